"""Shared helpers of the parity tests: build a seeded case, run the oracle and
the CUDA path on the same inputs, and compare them element by element."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1308_3995_gb300 import inputs as G


def oracle_params(wl, cfl=0.0, sc=0.0):
    return O.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds, prandtl=wl.prandtl,
                    cfl=cfl, sc_eps0=sc, aoa=wl.aoa)


def lib_params(wl, cfl=0.0, precision=0, sc=0.0):
    from paper_1308_3995_gb300 import hdg
    return hdg.Params(model=wl.model, precision=precision, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds,
                      prandtl=wl.prandtl, cfl=cfl, sc_eps0=sc, aoa=wl.aoa)


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


# ----------------------------------------------------------------------------- element-wise parity
def _blocks_split(om, K):
    sz = [4 * (int(om.face_p[e]) + 1) if e >= 0 else 0 for e in om.elem_face[K]]
    return np.concatenate([[0], np.cumsum(sz)]).astype(int)


def gather_trace(om, K, Lam):
    parts = [Lam[om.lam_off[e]:om.lam_off[e + 1]] for e in om.elem_face[K] if e >= 0]
    return np.concatenate(parts) if parts else np.zeros(0)


class ParityChecker:
    """Element-by-element comparison of the CUDA outputs with the oracle.

    Outputs with no cancellation (the local solves X_B and the trace blocks S)
    are compared by relative error per element / block.  Residual-type outputs
    (interior residual, trace residual, X_F, E, dU) are small differences of
    O(flux) terms for a near-converged state, so two FP64 evaluations in a
    different order differ by about u times the magnitude of those terms times
    cond(A); they are checked by backward error against the oracle's own
    element blocks, relative to the magnitude of the summed terms
    (|A||U| + |B||Lambda| for interior rows, |C||U| + |D||Lambda| for trace rows).
    Every returned number is an error already divided by its scale: the bar is
    ``err <= tol`` for all of them."""

    def __init__(self, om, P, U, Lam, dLam, g):
        self.om, self.P, self.U, self.Lam, self.dLam, self.g = om, P, U, Lam, dLam, g
        self.cache = {}

    def element(self, K):
        if K not in self.cache:
            om = self.om
            A, B, C, D, F, H = om.element_blocks(self.P, K, self.U, self.Lam)
            X, S, Ek, st = om.element_condense(self.P, K, self.U, self.Lam)
            UK = self.U[om.u_off[K]:om.u_off[K + 1]]
            LK = gather_trace(om, K, self.Lam)
            self.cache[K] = dict(A=A, B=B, C=C, D=D, F=F, H=H, X=X, S=S, Ek=Ek, st=st, UK=UK, LK=LK,
                                 su=np.abs(A) @ np.abs(UK) + np.abs(B) @ np.abs(LK),
                                 sl=np.abs(C) @ np.abs(UK) + np.abs(D) @ np.abs(LK))
        return self.cache[K]

    def gpu_X(self, K):
        om = self.om
        n, nt = om.n(K), om.nt(K)
        return self.g["X"][om.x_off[K]:om.x_off[K + 1]].reshape(nt + 1, n).T

    def check_element(self, K):
        om, e = self.om, self.element(K)
        nt = e["D"].shape[0]
        Xg = self.gpu_X(K)
        out = {}
        out["X_B"] = rel_err(Xg[:, :nt], e["X"][:, :nt])
        su = np.abs(e["su"]).max()
        out["X_F backward"] = np.abs(e["A"] @ Xg[:, nt] - e["F"]).max() / su
        ru = self.g["res_u"][om.u_off[K]:om.u_off[K + 1]]
        out["res_u"] = np.abs(ru - (-e["F"])).max() / su
        dl = gather_trace(om, K, self.dLam)
        du_ref = Xg[:, nt] - e["X"][:, :nt] @ dl
        du = self.g["dU"][om.u_off[K]:om.u_off[K + 1]]
        out["dU"] = np.abs(du - du_ref).max() / (np.abs(Xg[:, nt]) + np.abs(e["X"][:, :nt]) @ np.abs(dl)).max()
        off = _blocks_split(om, K)
        worst = 0.0
        for a in range(3):
            for b in range(3):
                if a == b:
                    continue
                ea, eb = om.elem_face[K][a], om.elem_face[K][b]
                if ea < 0 or eb < 0:   # boundary face: no trace block
                    continue
                slot = list(om.k_col[ea]).index(eb)
                o0, o1 = om.k_blkoff[5 * ea + slot], om.k_blkoff[5 * ea + slot + 1]
                worst = max(worst, rel_err(self.g["K"][o0:o1], e["S"][off[a]:off[a + 1], off[b]:off[b + 1]]))
        out["S off-diagonal"] = worst
        return out

    def check_face(self, f):
        om = self.om
        diag, e_ref, e_scale, r_ref, r_scale = 0.0, 0.0, 0.0, 0.0, 0.0
        for side in range(2):
            K = int(om.face_el[f, side])
            e = self.element(K)
            off = _blocks_split(om, K)
            a = list(om.elem_face[K]).index(f)
            rows = slice(off[a], off[a + 1])
            nt = e["D"].shape[0]
            Xg = self.gpu_X(K)
            diag = diag + e["S"][rows, rows]
            e_ref = e_ref + (e["H"] - e["C"] @ Xg[:, nt])[rows]
            e_scale = e_scale + (np.abs(e["H"]) + np.abs(e["C"]) @ np.abs(Xg[:, nt]) + e["sl"])[rows]
            r_ref = r_ref + (-e["H"])[rows]
            r_scale = r_scale + e["sl"][rows]
        slot = list(om.k_col[f]).index(f)
        o0, o1 = om.k_blkoff[5 * f + slot], om.k_blkoff[5 * f + slot + 1]
        l0, l1 = om.lam_off[f], om.lam_off[f + 1]
        return {"S diagonal (two sides)": rel_err(self.g["K"][o0:o1], diag),
                "E": np.abs(self.g["E"][l0:l1] - e_ref).max() / np.abs(e_scale).max(),
                "res_lam": np.abs(self.g["res_lam"][l0:l1] - r_ref).max() / np.abs(r_scale).max()}

    def run(self, elems, faces):
        worst = {}
        for K in elems:
            assert self.element(K)["st"] == 0
            for k, v in self.check_element(int(K)).items():
                worst[k] = max(worst.get(k, 0.0), v)
        for f in faces:
            for k, v in self.check_face(int(f)).items():
                worst[k] = max(worst.get(k, 0.0), v)
        return worst
