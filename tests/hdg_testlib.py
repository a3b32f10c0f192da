"""Shared helpers of the parity tests: build a seeded case, run the oracle and
the CUDA path on the same inputs, and compare them element by element."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1308_3995_gb300 import inputs as G


def oracle_params(wl, cfl=0.0):
    return O.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds, prandtl=wl.prandtl,
                    cfl=cfl)


def lib_params(wl, cfl=0.0, precision=0):
    from paper_1308_3995_gb300 import hdg
    return hdg.Params(model=wl.model, precision=precision, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds,
                      prandtl=wl.prandtl, cfl=cfl)


def rel_err(a, b, floor=1e-300):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / max(nb, floor))


def per_element_errors(m, Xg, Xo):
    """Relative error of each element's X (GPU column-major vs oracle row-major)."""
    errs = np.zeros(m.n_elem)
    for K in range(m.n_elem):
        n, nt = m.n(K), m.nt(K)
        xg = Xg[m.x_off[K]:m.x_off[K + 1]].reshape(nt + 1, n).T
        xo = Xo[m.x_off[K]:m.x_off[K + 1]].reshape(n, nt + 1)
        errs[K] = rel_err(xg, xo)
    return errs


def per_block_errors(m, Kg, Ko):
    errs = np.zeros(5 * m.n_face)
    for b in range(5 * m.n_face):
        s0, s1 = m.k_blkoff[b], m.k_blkoff[b + 1]
        errs[b] = rel_err(Kg[s0:s1], Ko[s0:s1])
    return errs


def per_face_errors(m, Eg, Eo):
    errs = np.zeros(m.n_face)
    for f in range(m.n_face):
        s0, s1 = m.lam_off[f], m.lam_off[f + 1]
        errs[f] = rel_err(Eg[s0:s1], Eo[s0:s1])
    return errs


def per_elem_vec_errors(m, a, b):
    errs = np.zeros(m.n_elem)
    for K in range(m.n_elem):
        s0, s1 = m.u_off[K], m.u_off[K + 1]
        errs[K] = rel_err(a[s0:s1], b[s0:s1])
    return errs
