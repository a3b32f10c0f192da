"""ctypes wrapper of the FP64 CPU oracle (``hdg_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product package never imports
it, and it never imports the product package.

Every function returns NumPy float64/int arrays.  The oracle follows the
paper's definitions (arXiv:1308.3995, Sec. 2 physics, Sec. 3.2 HDG weak form,
Sec. 3.3 pseudo time, Sec. 3.4 hybridization, Sec. 4 adjoint and adaptation);
see ``hdg_oracle.cpp``.  The block ILU(0) of the trace matrix (the paper's
incomplete-LU preconditioner, Sec. 3.4) is written here in NumPy, in the
textbook IKJ form.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hdg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_i32_p = ctypes.POINTER(ctypes.c_int32)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)


_LIBX = os.path.join(_HERE, "liboracle_ext.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain C++17, no FMA contraction): the binary64
    build, and the same source in long double (``-DORC_EXTENDED``)."""
    for lib_path, extra in ((_LIB, []), (_LIBX, ["-DORC_EXTENDED"])):
        if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
            tmp = lib_path + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-pthread", *extra, "-o", tmp, _SRC])
            os.replace(tmp, lib_path)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("reserved", ctypes.c_int32), ("gamma", ctypes.c_double),
                ("prandtl", ctypes.c_double), ("reynolds", ctypes.c_double), ("mach", ctypes.c_double),
                ("alpha", ctypes.c_double), ("cfl", ctypes.c_double), ("t_inf", ctypes.c_double),
                ("sc_eps0", ctypes.c_double), ("sc_beta", ctypes.c_double), ("aoa", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_gauss_jacobi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _c_double_p, _c_double_p]
        L.orc_tri_rule.argtypes = [ctypes.c_int, _c_double_p, _c_double_p, _c_double_p]
        L.orc_edge_rule.argtypes = [ctypes.c_int, _c_double_p, _c_double_p]
        L.orc_dubiner.argtypes = [ctypes.c_int, ctypes.c_int, _c_double_p, _c_double_p, _c_double_p,
                                  _c_double_p, _c_double_p]
        L.orc_legendre01.argtypes = [ctypes.c_int, ctypes.c_int, _c_double_p, _c_double_p]
        L.orc_euler_flux.argtypes = [_c_double_p, ctypes.c_double, _c_double_p]
        L.orc_mesh_set_source.argtypes = [ctypes.c_void_p, _c_double_p]
        L.orc_euler_flux.restype = None
        L.orc_ns_viscous_flux.argtypes = [_c_double_p, _c_double_p, ctypes.POINTER(OrcParams), _c_double_p]
        L.orc_ns_viscous_flux.restype = None
        L.orc_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, _c_double_p, _c_i32_p,
                                      ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int8),
                                      ctypes.POINTER(ctypes.c_void_p)]
        L.orc_mesh_destroy.argtypes = [ctypes.c_void_p]
        L.orc_mesh_destroy.restype = None
        L.orc_mesh_sizes.argtypes = [ctypes.c_void_p, _c_i64_p]
        L.orc_mesh_sizes.restype = None
        L.orc_mesh_arrays.argtypes = [ctypes.c_void_p] + [_c_i32_p] * 5 + [_c_i64_p] * 3 + [_c_i32_p, _c_i64_p]
        L.orc_mesh_arrays.restype = None
        P = ctypes.POINTER(OrcParams)
        L.orc_element_residual.argtypes = [ctypes.c_void_p, P, ctypes.c_int, _c_double_p, _c_double_p,
                                           _c_double_p, _c_double_p]
        L.orc_element_blocks.argtypes = [ctypes.c_void_p, P, ctypes.c_int, _c_double_p, _c_double_p] + \
            [_c_double_p] * 6
        L.orc_element_condense.argtypes = [ctypes.c_void_p, P, ctypes.c_int, _c_double_p, _c_double_p,
                                           _c_double_p, _c_double_p, _c_double_p]
        L.orc_condense.argtypes = [ctypes.c_void_p, P, _c_double_p, _c_double_p] + [_c_double_p] * 5 + \
            [_c_i32_p, ctypes.c_int, ctypes.c_int]
        L.orc_condense_mt.argtypes = [ctypes.c_void_p, P, _c_double_p, _c_double_p] + [_c_double_p] * 5 + \
            [_c_i32_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_recover.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p, _c_double_p]
        L.orc_global_residual.argtypes = [ctypes.c_void_p, P, _c_double_p, _c_double_p, _c_double_p]
        L.orc_monolithic.argtypes = [ctypes.c_void_p, P, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                     _c_double_p]
        L.orc_dense_solve.argtypes = [ctypes.c_int, _c_double_p, _c_double_p]
        L.orc_boundary_state.argtypes = [ctypes.c_int, _c_double_p, ctypes.c_double, ctypes.c_double, P,
                                         _c_double_p]
        L.orc_boundary_state.restype = None
        L.orc_cfl_law.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double]
        L.orc_cfl_law.restype = ctypes.c_double
        L.orc_smoothness.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_double_p]
        L.orc_smoothness.restype = ctypes.c_double
        L.orc_adapt_mark.argtypes = [ctypes.c_int, _c_double_p, _c_double_p, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int8)]
        L.orc_sc_epsilon.argtypes = [ctypes.c_void_p, P, ctypes.c_int, _c_double_p]
        L.orc_sc_epsilon.restype = ctypes.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_c_double_p)


def _i32(a):
    return a.ctypes.data_as(_c_i32_p)


def _i64(a):
    return a.ctypes.data_as(_c_i64_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------- tables
def gauss_jacobi(n: int, alpha: float, beta: float):
    x = np.zeros(n); w = np.zeros(n)
    assert lib().orc_gauss_jacobi(n, alpha, beta, _d(x), _d(w)) == 0
    return x, w


def tri_rule(p: int):
    m = (p + 2) ** 2
    xi, eta, w = np.zeros(m), np.zeros(m), np.zeros(m)
    assert lib().orc_tri_rule(p, _d(xi), _d(eta), _d(w)) == 0
    return xi, eta, w


def edge_rule(pe: int):
    s, w = np.zeros(pe + 2), np.zeros(pe + 2)
    assert lib().orc_edge_rule(pe, _d(s), _d(w)) == 0
    return s, w


def n_basis(p: int) -> int:
    return (p + 1) * (p + 2) // 2


def dubiner(p: int, xi, eta):
    xi, eta = _f64(xi), _f64(eta)
    m, nb = xi.size, n_basis(p)
    phi, dx, de = np.zeros((m, nb)), np.zeros((m, nb)), np.zeros((m, nb))
    assert lib().orc_dubiner(p, m, _d(xi), _d(eta), _d(phi), _d(dx), _d(de)) == 0
    return phi, dx, de


def legendre01(pe: int, s):
    s = _f64(s)
    psi = np.zeros((s.size, pe + 1))
    lib().orc_legendre01(pe, s.size, _d(s), _d(psi))
    return psi


# --------------------------------------------------------------------------- physics
def euler_flux(w, gamma=1.4):
    w = _f64(w); f = np.zeros((2, 4))
    lib().orc_euler_flux(_d(w), gamma, _d(f))
    return f


def ns_viscous_flux(w, q, params):
    w = _f64(w); q = _f64(q).reshape(2, 4); f = np.zeros((2, 4))
    P = params.c()
    lib().orc_ns_viscous_flux(_d(w), _d(q), ctypes.byref(P), _d(f))
    return f


@dataclass
class Params:
    """Flow / discretisation parameters (model 0 = Euler, 1 = NS mixed form)."""
    model: int = 0
    gamma: float = 1.4
    prandtl: float = 0.72
    reynolds: float = 5000.0
    mach: float = 0.5
    alpha: float = 1.5
    cfl: float = 0.0
    t_inf: float = 288.15
    sc_eps0: float = 0.0     # shock capturing off unless > 0 (paper's value: 0.2)
    sc_beta: float = 0.0
    aoa: float = 0.0         # free-stream angle of attack [degrees] (far-field state)

    def c(self) -> OrcParams:
        return OrcParams(self.model, 0, self.gamma, self.prandtl, self.reynolds, self.mach, self.alpha,
                         self.cfl, self.t_inf, self.sc_eps0, self.sc_beta, self.aoa)

    @property
    def nfield(self) -> int:
        return 12 if self.model == 1 else 4


def boundary_state(kind, w, n, params) -> np.ndarray:
    """Boundary state w_b(w) of Sec. 2.1/2.2: kind 1 slip wall, 2 far field (characteristic), 3 no-slip
    wall (rho, 0, 0, E); normal n."""
    wb = np.zeros(4)
    P = params.c()
    lib().orc_boundary_state(int(kind), _d(_f64(w)), float(n[0]), float(n[1]), ctypes.byref(P), _d(wb))
    return wb


def cfl_law(n, c0=1e6, c1=1e3, n0=4, cfl_prev=0.0, res_prev=1.0, res_cur=1.0) -> float:
    """CFL^n of Eq. (cfl) (Sec. 3.3)."""
    return float(lib().orc_cfl_law(int(n), float(c0), float(c1), int(n0), float(cfl_prev), float(res_prev),
                                   float(res_cur)))


def adapt_mark(eta2, sensor, theta=0.05, eps_s=1e-6):
    """Doerfler marking with the h/p choice (Sec. 4.3-4.4): codes 0 / 1 (p) / 2 (h), count marked."""
    eta2 = _f64(eta2); sensor = _f64(sensor)
    code = np.zeros(eta2.size, np.int8)
    nm = lib().orc_adapt_mark(int(eta2.size), _d(eta2), _d(sensor), float(theta), float(eps_s),
                              code.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)))
    return code, int(nm)


# --------------------------------------------------------------------------- mesh-level
class Mesh:
    """Oracle mesh: faces, sides and the documented layouts of U, Lambda, X, K."""

    def __init__(self, elem_xy, elem_vid, elem_p, nfield: int, elem_bc=None):
        xy = _f64(elem_xy).reshape(-1, 6)
        vid = np.ascontiguousarray(elem_vid, dtype=np.int32).reshape(-1, 3)
        p = np.ascontiguousarray(elem_p, dtype=np.int8).reshape(-1)
        self.n_elem = int(p.size)
        self.nfield = nfield
        bc = None if elem_bc is None else np.ascontiguousarray(elem_bc, dtype=np.int8).reshape(-1, 3)
        self.elem_bc = bc
        h = ctypes.c_void_p()
        st = lib().orc_mesh_create(self.n_elem, nfield, _d(xy), _i32(vid),
                                   p.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                   bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if bc is not None else None,
                                   ctypes.byref(h))
        if st != 0:
            raise ValueError(f"oracle rejected the mesh (status {st})")
        self._h = h
        sz = np.zeros(5, dtype=np.int64)
        lib().orc_mesh_sizes(h, _i64(sz))
        self.n_face, self.u_len, self.lam_len, self.x_len, self.k_len = (int(v) for v in sz)
        nf, ne = self.n_face, self.n_elem
        self.face_vid = np.zeros((nf, 2), np.int32)
        self.face_el = np.zeros((nf, 2), np.int32)
        self.face_lf = np.zeros((nf, 2), np.int32)
        self.face_p = np.zeros(nf, np.int32)
        self.elem_face = np.zeros((ne, 3), np.int32)
        self.u_off = np.zeros(ne + 1, np.int64)
        self.lam_off = np.zeros(nf + 1, np.int64)
        self.x_off = np.zeros(ne + 1, np.int64)
        self.k_col = np.zeros((nf, 5), np.int32)
        self.k_blkoff = np.zeros(5 * nf + 1, np.int64)
        lib().orc_mesh_arrays(h, _i32(self.face_vid), _i32(self.face_el), _i32(self.face_lf),
                              _i32(self.face_p), _i32(self.elem_face), _i64(self.u_off), _i64(self.lam_off),
                              _i64(self.x_off), _i32(self.k_col), _i64(self.k_blkoff))
        self.elem_p = p.astype(np.int32)
        self.elem_vid = vid
        self.elem_xy = xy

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_mesh_destroy(h)
            self._h = None

    # sizes of element K
    def n(self, K):
        return self.nfield * n_basis(int(self.elem_p[K]))

    def nt(self, K):
        return int(sum(4 * (self.face_p[e] + 1) for e in self.elem_face[K] if e >= 0))

    def element_residual(self, params, K, U, Lam):
        n, nt = self.n(K), self.nt(K)
        Nu, Nl = np.zeros(n), np.zeros(nt)
        P = params.c()
        lib().orc_element_residual(self._h, ctypes.byref(P), int(K), _d(_f64(U)), _d(_f64(Lam)), _d(Nu), _d(Nl))
        return Nu, Nl

    def smoothness(self, K, U):
        """Smoothness sensor S_K of Sec. 4.4."""
        return float(lib().orc_smoothness(self._h, int(K), _d(_f64(U))))

    def sc_epsilon(self, params, K, U):
        """Shock-capturing viscosity eps_K of element K (Sec. 3.2); 0 when off."""
        P = params.c()
        return float(lib().orc_sc_epsilon(self._h, ctypes.byref(P), int(K), _d(_f64(U))))

    def element_blocks(self, params, K, U, Lam):
        n, nt = self.n(K), self.nt(K)
        A, B, C, D = np.zeros((n, n)), np.zeros((n, nt)), np.zeros((nt, n)), np.zeros((nt, nt))
        F, H = np.zeros(n), np.zeros(nt)
        P = params.c()
        lib().orc_element_blocks(self._h, ctypes.byref(P), int(K), _d(_f64(U)), _d(_f64(Lam)),
                                 _d(A), _d(B), _d(C), _d(D), _d(F), _d(H))
        return A, B, C, D, F, H

    def element_condense(self, params, K, U, Lam):
        n, nt = self.n(K), self.nt(K)
        X, S, E = np.zeros((n, nt + 1)), np.zeros((nt, nt)), np.zeros(nt)
        P = params.c()
        st = lib().orc_element_condense(self._h, ctypes.byref(P), int(K), _d(_f64(U)), _d(_f64(Lam)),
                                        _d(X), _d(S), _d(E))
        return X, S, E, st

    def condense(self, params, U, Lam, k0=0, k1=0, threads=1):
        """Condensation and assembly of elements [k0, k1) (all if k1 <= k0); `threads` > 1 spreads the
        per-element work over host threads (bitwise the same outputs)."""
        X = np.zeros(self.x_len); Kv = np.zeros(self.k_len); E = np.zeros(self.lam_len)
        rU = np.zeros(self.u_len); rL = np.zeros(self.lam_len); st = np.zeros(self.n_elem, np.int32)
        P = params.c()
        lib().orc_condense_mt(self._h, ctypes.byref(P), _d(_f64(U)), _d(_f64(Lam)), _d(X), _d(Kv), _d(E), _d(rU),
                              _d(rL), _i32(st), int(k0), int(k1), int(threads))
        return dict(X=X, K=Kv, E=E, res_u=rU, res_lam=rL, status=st)

    def recover(self, X, dLam):
        dU = np.zeros(self.u_len)
        lib().orc_recover(self._h, _d(_f64(X)), _d(_f64(dLam)), _d(dU))
        return dU

    def global_residual(self, params, U, Lam):
        R = np.zeros(self.u_len + self.lam_len)
        P = params.c()
        lib().orc_global_residual(self._h, ctypes.byref(P), _d(_f64(U)), _d(_f64(Lam)), _d(R))
        return R[:self.u_len], R[self.u_len:]

    def monolithic(self, params, U, Lam, want_matrix=False):
        N = self.u_len + self.lam_len
        dU, dL = np.zeros(self.u_len), np.zeros(self.lam_len)
        J = np.zeros((N, N)) if want_matrix else None
        P = params.c()
        st = lib().orc_monolithic(self._h, ctypes.byref(P), _d(_f64(U)), _d(_f64(Lam)), _d(dU), _d(dL),
                                  _d(J) if want_matrix else None)
        if st != 0:
            raise RuntimeError(f"monolithic solve failed (status {st})")
        return (dU, dL, J) if want_matrix else (dU, dL)

    def global_jacobian(self, params, U, Lam):
        """Dense Jacobian of the global residual (plus pseudo-time mass if cfl > 0); the
        solve status is ignored, so a singular (pure-Newton periodic) matrix is returned too."""
        N = self.u_len + self.lam_len
        dU, dL, J = np.zeros(self.u_len), np.zeros(self.lam_len), np.zeros((N, N))
        P = params.c()
        st = lib().orc_monolithic(self._h, ctypes.byref(P), _d(_f64(U)), _d(_f64(Lam)), _d(dU), _d(dL), _d(J))
        if st == 2:
            raise ValueError("mesh too large for the dense Jacobian")
        return J

    def set_source(self, S=None):
        """Source s of Eq. (hdg_ls3) as the coefficients of its L2 projection in U's layout
        (w part); None: s = 0."""
        if S is None:
            lib().orc_mesh_set_source(self._h, None)
        else:
            self._src = _f64(S).copy()
            lib().orc_mesh_set_source(self._h, _d(self._src))

    def dense_K(self, Kv):
        """Expand the block-sparse trace matrix into a dense lam_len x lam_len array."""
        Kd = np.zeros((self.lam_len, self.lam_len))
        for f in range(self.n_face):
            nr = 4 * (self.face_p[f] + 1)
            for b in range(5):
                c = self.k_col[f, b]
                if c < 0:
                    continue      # unused slot next to a boundary face
                nc = 4 * (self.face_p[c] + 1)
                o = self.k_blkoff[5 * f + b]
                Kd[self.lam_off[f]:self.lam_off[f] + nr, self.lam_off[c]:self.lam_off[c] + nc] = \
                    Kv[o:o + nr * nc].reshape(nr, nc)
        return Kd


def dense_solve(A, b):
    A = _f64(A); x = _f64(b).copy()
    if lib().orc_dense_solve(A.shape[0], _d(A), _d(x)) != 0:
        raise RuntimeError("singular")
    return x


# ----------------------------------------------------------------------------- block ILU(0)
# The paper preconditions GMRES on the trace system with incomplete LU (Sec. 3.4, the
# paragraph after Eq. hybridsystem).  The oracle below is the textbook block ILU(0): the
# IKJ form of Gaussian elimination with blocks as entries, fill kept only where the block
# pattern of the matrix has a block (Saad, Iterative Methods for Sparse Linear Systems,
# 2nd ed., Sec. 10.3), in a caller-given elimination order of the block rows.
def trace_pattern(mesh) -> set:
    """Block pattern of the trace matrix: the pairs (face, face) that share an element."""
    P = set()
    for f in range(mesh.n_face):
        for b in range(5):
            c = int(mesh.k_col[f, b])
            if c >= 0:
                P.add((f, c))
    return P


def block_ilu0(A, offs, pattern, order):
    """Block ILU(0) of the dense block matrix ``A`` (block row/column b spans
    ``offs[b]:offs[b+1]``) eliminated in the block order ``order``.

    Returns ``(L, U, perm)``: with ``perm`` the scalar permutation that lists the
    blocks in ``order``, ``L`` (identity diagonal blocks, blocks only below) and
    ``U`` (blocks on and above the diagonal) factor ``A[perm][:, perm]``
    incompletely: (L U)_ij = A_ij on every block (i, j) of ``pattern``."""
    A = _f64(A)
    nb = len(offs) - 1
    pos = {b: i for i, b in enumerate(order)}
    size = [int(offs[b + 1] - offs[b]) for b in order]
    po = np.concatenate([[0], np.cumsum(size)]).astype(np.int64)
    perm = np.concatenate([np.arange(offs[b], offs[b + 1]) for b in order]).astype(np.int64)
    W = A[np.ix_(perm, perm)].copy()
    row = [[] for _ in range(nb)]              # pattern of each permuted block row
    for (i, j) in pattern:
        row[pos[i]].append(pos[j])
    rows = [set(r) for r in row]

    def B(i, j):
        return (slice(po[i], po[i + 1]), slice(po[j], po[j + 1]))

    for i in range(1, nb):
        for k in sorted(c for c in rows[i] if c < i):
            W[B(i, k)] = W[B(i, k)] @ np.linalg.inv(W[B(k, k)])
            for j in sorted(c for c in rows[i] if c > k):
                if j in rows[k]:
                    W[B(i, j)] -= W[B(i, k)] @ W[B(k, j)]
    L = np.eye(len(perm))
    U = np.zeros_like(W)
    for i in range(nb):
        for j in rows[i]:
            if j < i:
                L[B(i, j)] = W[B(i, j)]
            else:
                U[B(i, j)] = W[B(i, j)]
    return L, U, perm


def block_ilu0_apply(L, U, perm, r, transpose=False):
    """z = M^{-1} r (or M^{-T} r) for the preconditioner M = P^T L U P of ``block_ilu0``."""
    rp = _f64(r)[perm]
    if transpose:
        zp = np.linalg.solve(L.T, np.linalg.solve(U.T, rp))
    else:
        zp = np.linalg.solve(U, np.linalg.solve(L, rp))
    z = np.empty_like(zp)
    z[perm] = zp
    return z


# --------------------------------------------------------------------------- extended precision
_libx = None


def libx():
    """The oracle compiled in long double (80-bit extended on x86-64, binary128 on aarch64)."""
    global _libx
    if _libx is None:
        build()
        L = ctypes.CDLL(_LIBX)
        L.orc_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, _c_double_p, _c_i32_p,
                                      ctypes.POINTER(ctypes.c_int8), ctypes.POINTER(ctypes.c_int8),
                                      ctypes.POINTER(ctypes.c_void_p)]
        L.orc_mesh_destroy.argtypes = [ctypes.c_void_p]
        L.orc_mesh_destroy.restype = None
        P = ctypes.POINTER(OrcParams)
        L.orcx_element_condense.argtypes = [ctypes.c_void_p, P, ctypes.c_int] + [_c_double_p] * 7
        L.orcx_face_E.argtypes = [ctypes.c_void_p, P, ctypes.c_int, _c_double_p, _c_double_p, _c_double_p]
        L.orcx_mantissa_bits.argtypes = []
        _libx = L
    return _libx


def mantissa_bits_ext() -> int:
    return int(libx().orcx_mantissa_bits())


class ExtMesh:
    """The same mesh in the extended-precision build: the definition evaluated in long double
    (tables, geometry, residual, complex-step Jacobian, LU, Schur), inputs and results binary64.
    Sizes and layouts are those of ``Mesh`` on the same arrays."""

    def __init__(self, mesh: Mesh):
        self.m = mesh
        bc = mesh.elem_bc
        h = ctypes.c_void_p()
        st = libx().orc_mesh_create(mesh.n_elem, mesh.nfield, _d(mesh.elem_xy), _i32(mesh.elem_vid),
                                    np.ascontiguousarray(mesh.elem_p, dtype=np.int8).ctypes.data_as(
                                        ctypes.POINTER(ctypes.c_int8)),
                                    bc.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if bc is not None else None,
                                    ctypes.byref(h))
        if st != 0:
            raise ValueError(f"extended oracle rejected the mesh (status {st})")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _libx is not None:
            _libx.orc_mesh_destroy(h)
            self._h = None

    def element_condense(self, params, K, U, Lam, dLam):
        """X [n, nt+1] (row-major, X_F last), S [nt, nt], E_K [nt] and dU_K = X_F - X_B dLam_K [n]."""
        n, nt = self.m.n(K), self.m.nt(K)
        X, S, E, dU = np.zeros((n, nt + 1)), np.zeros((nt, nt)), np.zeros(nt), np.zeros(n)
        P = params.c()
        st = libx().orcx_element_condense(self._h, ctypes.byref(P), int(K), _d(_f64(U)), _d(_f64(Lam)),
                                          _d(_f64(dLam)), _d(X), _d(S), _d(E), _d(dU))
        return X, S, E, dU, st

    def face_E(self, params, f, U, Lam):
        """Assembled E of face f (both sides' contributions summed in long double)."""
        out = np.zeros(4 * (int(self.m.face_p[f]) + 1))
        P = params.c()
        st = libx().orcx_face_E(self._h, ctypes.byref(P), int(f), _d(_f64(U)), _d(_f64(Lam)), _d(out))
        if st != 0:
            raise ValueError(f"extended oracle: status {st} on face {f}")
        return out
