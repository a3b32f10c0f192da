"""Manufactured solution for the Euler equations on the periodic unit square (test
infrastructure): a smooth subsonic field w_ex, its source s = div f_c(w_ex) (the steady
residual of Eq. hdg_ls2-hdg_ls3 vanishes for w_ex when the source term -(phi, s) is added),
and L2 projections onto the pinned element and edge bases, evaluated with the oracle's
quadrature and basis routines."""
from __future__ import annotations

import math

import numpy as np

import oracle as O

GAMMA = 1.4
TWO_PI = 2.0 * math.pi


def primitive(x, y):
    """rho, u, v, p of the manufactured field (periodic, Mach about 0.6, works for complex x, y)."""
    rho = 1.0 + 0.15 * np.sin(TWO_PI * (x + y))
    u = 0.5 + 0.1 * np.sin(TWO_PI * x) * np.cos(TWO_PI * y)
    v = 0.3 + 0.1 * np.cos(TWO_PI * x) * np.sin(TWO_PI * y)
    p = 1.0 / GAMMA + 0.05 * np.cos(TWO_PI * (x - y))
    return rho, u, v, p


def conserved(x, y):
    rho, u, v, p = primitive(x, y)
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)], -1)


def flux(w):
    """Euler flux f_x, f_y of conserved states w[..., 4] (Sec. 2.1)."""
    rho, mu, mv, E = w[..., 0], w[..., 1], w[..., 2], w[..., 3]
    u, v = mu / rho, mv / rho
    p = (GAMMA - 1.0) * (E - 0.5 * rho * (u * u + v * v))
    fx = np.stack([mu, mu * u + p, mu * v, (E + p) * u], -1)
    fy = np.stack([mv, mv * u, mv * v + p, (E + p) * v], -1)
    return fx, fy


def source(x, y):
    """s = d f_x(w_ex)/dx + d f_y(w_ex)/dy by complex step (exact to rounding)."""
    h = 1e-30
    fx, _ = flux(conserved(x + 1j * h, y + 0j))
    _, fy = flux(conserved(x + 0j, y + 1j * h))
    return (fx.imag + fy.imag) / h


def _elem_points(xy, xi, eta):
    x0 = xy[0]
    J = np.stack([xy[1] - x0, xy[2] - x0], 1)
    pts = x0 + np.stack([xi, eta], 1) @ J.T
    return pts, abs(np.linalg.det(J))


def project(m, fun, order=8):
    """Coefficients in U's layout (4 fields x n_p per element) of the L2 projection of fun(x, y)[.., 4]."""
    xi, eta, wq = O.tri_rule(order)
    out = np.zeros(m.u_len)
    for K in range(m.n_elem):
        p = int(m.elem_p[K]); nb = O.n_basis(p)
        phi, _, _ = O.dubiner(p, xi, eta)
        pts, _ = _elem_points(m.elem_xy[K].reshape(3, 2), xi, eta)
        f = fun(pts[:, 0], pts[:, 1])                       # [nq, 4]
        c = (phi * wq[:, None]).T @ f                       # [nb, 4]
        out[m.u_off[K]:m.u_off[K] + 4 * nb] = c.T.reshape(-1)
    return out


def project_traces(m, elem_vid, order=8):
    """Edge L2 projections of w_ex (orthonormal Legendre on [0, 1], s from the lower to the higher
    global vertex id)."""
    s, ws = O.edge_rule(order)
    L = np.zeros(m.lam_len)
    for e in range(m.n_face):
        K = int(m.face_el[e][0])
        xy = m.elem_xy[K].reshape(3, 2)
        vid = list(elem_vid[K])
        lo, hi = (vid.index(int(m.face_vid[e][0])), vid.index(int(m.face_vid[e][1])))
        pts = xy[lo][None, :] + s[:, None] * (xy[hi] - xy[lo])[None, :]
        w = conserved(pts[:, 0], pts[:, 1])
        nk = int(m.face_p[e]) + 1
        psi = O.legendre01(nk - 1, s)
        c = (psi * ws[:, None]).T @ w                      # [nk, 4]
        L[m.lam_off[e]:m.lam_off[e] + 4 * nk] = c.T.reshape(-1)
    return L


def l2_error(m, U, field=0, order=8):
    """|| w_h,field - w_ex,field ||_L2 over the mesh."""
    xi, eta, wq = O.tri_rule(order)
    err = 0.0
    for K in range(m.n_elem):
        p = int(m.elem_p[K]); nb = O.n_basis(p)
        phi, _, _ = O.dubiner(p, xi, eta)
        pts, det = _elem_points(m.elem_xy[K].reshape(3, 2), xi, eta)
        wh = phi @ U[m.u_off[K] + field * nb:m.u_off[K] + (field + 1) * nb]
        we = conserved(pts[:, 0], pts[:, 1])[:, field]
        err += det * float(wq @ (wh - we) ** 2)
    return math.sqrt(err)
