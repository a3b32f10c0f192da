"""The FP64 bar on residual-type outputs, settled against an extended-precision
evaluation of the same definition.

E = H - C X_F, X_F = A^{-1} F and the reconstruction dU are differences of
O(flux) terms (the Newton iterate's residual is about 1e-3 of the terms it
sums), so every binary64 evaluation of them carries a rounding error of about
u * sum|terms| * cond(A_K).  Here the oracle compiled in long double (binary128
on aarch64) gives the reference; the GPU's binary64 results and the binary64
oracle are both measured against it on sampled elements and faces of the
full-size workloads (16,384-triangle Euler p = 3 and the 65,536-triangle
Navier-Stokes degree mix).  The GPU must be within 1e-12 of the reference over
the sample, and per element / face no further from it than the binary64 oracle
is, within a factor that allows for a different summation order."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import lib_params, oracle_params
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _gpu_step(wl, precision):
    from paper_1308_3995_gb300 import hdg
    c = G.make_case(wl)
    ctx = hdg.Context(0)
    mesh = hdg.Mesh(ctx, c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
    U, Lam, dLam = G.case_state(c, mesh.face_vid, mesh.face_p)
    sysm = hdg.System(ctx, mesh, lib_params(wl, precision=precision))
    dev = torch.device("cuda:0")
    Ut, Lt, dLt = (torch.from_numpy(a).to(dev) for a in (U, Lam, dLam))
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    sysm.condense(Ut, Lt)
    sysm.recover(dLt, dUt)
    torch.cuda.synchronize()
    v = {k: t.cpu().numpy() for k, t in sysm.views().items()}
    v["dU"] = dUt.cpu().numpy()
    return c, U, Lam, dLam, v


@pytest.mark.parametrize("name,precision,bar", [("euler_p3_16k", 0, 1e-12), ("ns_mixp_65k", 0, 1e-12),
                                                ("euler_p3_16k", 1, 1e-10), ("ns_mixp_65k", 1, 1e-10)])
def test_residual_type_outputs_against_extended_precision(name, precision, bar):
    wl = G.WORKLOADS[name]
    c, U, Lam, dLam, v = _gpu_step(wl, precision)
    m = O.Mesh(c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
    mx = O.ExtMesh(m)
    P = oracle_params(wl)
    rng = np.random.default_rng(5)
    elems = sorted(rng.choice(m.n_elem, 8, replace=False).tolist())
    faces = sorted(rng.choice(m.n_face, 8, replace=False).tolist())
    # binary64 oracle on the sampled elements and on both sides of the sampled faces
    need = sorted(set(elems) | {int(k) for f in faces for k in m.face_el[f]})
    o64 = {K: m.element_condense(P, K, U, Lam) for K in need}
    rows = {"X_B": [], "X_F": [], "dU": [], "E": []}
    for K in elems:
        X, S, E, dUx, st = mx.element_condense(P, K, U, Lam, dLam)
        assert st == 0
        n, nt = m.n(K), m.nt(K)
        Xg = v["X"][m.x_off[K]:m.x_off[K + 1]].reshape(nt + 1, n).T     # column-major on the GPU
        Xo = o64[K][0]
        dl = np.concatenate([dLam[m.lam_off[e]:m.lam_off[e + 1]] for e in m.elem_face[K] if e >= 0])
        dUo = Xo[:, nt] - Xo[:, :nt] @ dl
        dUg = v["dU"][m.u_off[K]:m.u_off[K + 1]]
        rows["X_B"].append((Xg[:, :nt], Xo[:, :nt], X[:, :nt]))
        rows["X_F"].append((Xg[:, nt], Xo[:, nt], X[:, nt]))
        rows["dU"].append((dUg, dUo, dUx))
    for f in faces:
        Ex = mx.face_E(P, f, U, Lam)
        Eo = np.zeros_like(Ex)
        for K in m.face_el[f]:
            nt, roff = m.nt(K), 0
            for e in m.elem_face[K]:
                if e < 0:
                    continue
                ln = 4 * (int(m.face_p[e]) + 1)
                if e == f:
                    Eo += o64[int(K)][2][roff:roff + ln]
                roff += ln
        rows["E"].append((v["E"][m.lam_off[f]:m.lam_off[f + 1]], Eo, Ex))
    report = {}
    for key, items in rows.items():
        g_err = [_rel(g, x) for g, o, x in items]
        o_err = [_rel(o, x) for g, o, x in items]
        glob = _rel(np.concatenate([np.ravel(g) for g, o, x in items]),
                    np.concatenate([np.ravel(x) for g, o, x in items]))
        report[key] = (max(g_err), max(o_err), glob)
        assert glob <= bar, f"{name} {key}: GPU {glob:.2e} from the extended reference over the sample"
        if precision == 0:
            for ge, oe in zip(g_err, o_err):
                assert ge <= max(bar, 4.0 * oe), f"{name} {key}: GPU {ge:.2e}, binary64 oracle {oe:.2e}"
    print(f"\n{name} {'fp64' if precision == 0 else 'float2'} vs long double ({O.mantissa_bits_ext()}-bit "
          f"significand): " + "; ".join(f"{k} GPU max {a:.2e} / oracle max {b:.2e} / GPU over sample {c:.2e}"
                                         for k, (a, b, c) in report.items()))
