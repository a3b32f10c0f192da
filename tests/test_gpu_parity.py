"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by
element, on the same seeded inputs.  Bar: 1e-12 relative per element / block
(FP64 path); layouts, bucket ids and integer data bit-exact."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import (lib_params, oracle_params, per_block_errors, per_elem_vec_errors, per_element_errors,
                         per_face_errors, rel_err)
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_3995_gb300 import hdg
    return hdg.Context(0)


def build_case(wl):
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    U, Lam, dLam = G.case_state(case, om.face_vid, om.face_p)
    return case, om, U, Lam, dLam


def run_gpu(ctx, case, wl, U, Lam, dLam, cfl=0.0, repeat=1):
    from paper_1308_3995_gb300 import hdg
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    sysm = hdg.System(ctx, mesh, lib_params(wl, cfl))
    dev = torch.device("cuda:0")
    Ut = torch.from_numpy(U).to(dev)
    Lt = torch.from_numpy(Lam).to(dev)
    dLt = torch.from_numpy(dLam).to(dev)
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    outs = []
    for _ in range(repeat):
        sysm.condense(Ut, Lt)
        sysm.recover(dLt, dUt)
        torch.cuda.synchronize()
        v = sysm.views()
        o = {k: t.cpu().numpy().copy() for k, t in v.items()}
        o["dU"] = dUt.cpu().numpy().copy()
        outs.append(o)
    return mesh, sysm, outs


def assert_layout_equal(mesh, om):
    for name in ("face_vid", "face_el", "face_p", "elem_face", "u_off", "lam_off", "x_off", "k_col", "k_blkoff"):
        a, b = getattr(mesh, name), getattr(om, name)
        assert np.array_equal(np.asarray(a).ravel(), np.asarray(b).ravel()), name


def full_parity(ctx, wl, cfl=0.0):
    case, om, U, Lam, dLam = build_case(wl)
    mesh, sysm, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam, cfl)
    assert_layout_equal(mesh, om)
    r = om.condense(oracle_params(wl, cfl), U, Lam)
    dUo = om.recover(r["X"], dLam)
    assert np.all(g["status"] == 0) and np.all(r["status"] == 0)
    errs = {
        "X": per_element_errors(om, g["X"], r["X"]).max(),
        "K": per_block_errors(om, g["K"], r["K"]).max(),
        "E": per_face_errors(om, g["E"], r["E"]).max(),
        "res_lam": per_face_errors(om, g["res_lam"], r["res_lam"]).max(),
        "res_u": per_elem_vec_errors(om, g["res_u"], r["res_u"]).max(),
        "dU": per_elem_vec_errors(om, g["dU"], dUo).max(),
    }
    print(wl.name, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < TOL, (k, v)
    return errs


def test_config1_euler_p1_256(ctx):
    """256 triangles, Euler p = 1, Mach 0.5 + density bump: every output element by element."""
    full_parity(ctx, G.WORKLOADS["euler_p1_256"])


@pytest.mark.parametrize("p", [2, 3, 4])
def test_euler_uniform_p_jittered(ctx, p):
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 6, 8, p=p)
    full_parity(ctx, wl)


def test_euler_mixed_p_ragged(ctx):
    """Degrees 1..4 mixed (p_e = max), odd grid so buckets have ragged sizes."""
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 7, 5, model=0)
    full_parity(ctx, wl)


def test_euler_pseudo_time(ctx):
    """Finite CFL adds the local-time-step mass (Sec. 3.3) to the W block."""
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 5, 6, p=3)
    full_parity(ctx, wl, cfl=10.0)


def test_euler_supersonic_shock_band(ctx):
    wl = G.small_variant(G.WORKLOADS["euler_p3_262k_shock"], 8, 12)
    full_parity(ctx, wl)


def test_free_stream_residual_vanishes(ctx):
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 6, 5, model=0)
    case, om, U, Lam, dLam = build_case(wl)
    winf = case.fld.w_inf
    U[:] = 0.0
    Lam[:] = 0.0
    for K in range(om.n_elem):
        nb = O.n_basis(int(om.elem_p[K]))
        U[om.u_off[K] + np.arange(4) * nb] = winf / np.sqrt(2.0)
    for e in range(om.n_face):
        nk = om.face_p[e] + 1
        Lam[om.lam_off[e] + np.arange(4) * nk] = winf
    _, _, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam)
    scale = np.abs(O.euler_flux(winf)).max()
    assert np.abs(g["res_u"]).max() < 1e-13 * scale
    assert np.abs(g["res_lam"]).max() < 1e-13 * scale


def test_repeatable_bitwise(ctx):
    """Two-sided sums in fixed order: repeated condensation is bitwise identical."""
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 9, 7, model=0)
    case, om, U, Lam, dLam = build_case(wl)
    _, _, outs = run_gpu(ctx, case, wl, U, Lam, dLam, repeat=3)
    for o in outs[1:]:
        for k in ("X", "K", "E", "res_u", "res_lam", "dU"):
            assert np.array_equal(o[k], outs[0][k]), k


def test_full_size_config2_sampled(ctx):
    """16,384-element Euler p = 3 workload in the benchmark's launch configuration:
    sampled elements and faces against the oracle computed one element at a time."""
    wl = G.WORKLOADS["euler_p3_16k"]
    case, om, U, Lam, dLam = build_case(wl)
    mesh, sysm, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam)
    assert_layout_equal(mesh, om)
    assert np.all(g["status"] == 0)
    P = oracle_params(wl)
    rng = np.random.default_rng(5)
    faces = rng.choice(om.n_face, 12, replace=False)
    elems = sorted(set(int(k) for f in faces for k in om.face_el[f]) | set(int(k) for k in rng.choice(om.n_elem, 8)))
    loc = {}
    for K in elems:
        X, S, Ek, st = om.element_condense(P, K, U, Lam)
        assert st == 0
        loc[K] = (X, S, Ek)
        n, nt = om.n(K), om.nt(K)
        xg = g["X"][om.x_off[K]:om.x_off[K + 1]].reshape(nt + 1, n).T
        assert rel_err(xg, X) < TOL
        # reconstruction from the oracle's own local solve
        dl = np.concatenate([dLam[om.lam_off[e]:om.lam_off[e + 1]] for e in om.elem_face[K]])
        du = X[:, nt] - X[:, :nt] @ dl
        assert rel_err(g["dU"][om.u_off[K]:om.u_off[K + 1]], du) < TOL
        # off-diagonal blocks come from this element alone
        sz = [4 * (om.face_p[e] + 1) for e in om.elem_face[K]]
        off = np.concatenate([[0], np.cumsum(sz)])
        for a in range(3):
            for b in range(3):
                if a == b:
                    continue
                ea, eb = om.elem_face[K][a], om.elem_face[K][b]
                slot = list(om.k_col[ea]).index(eb)
                o0, o1 = om.k_blkoff[5 * ea + slot], om.k_blkoff[5 * ea + slot + 1]
                assert rel_err(g["K"][o0:o1], S[off[a]:off[a + 1], off[b]:off[b + 1]]) < TOL
    for f in faces:
        diag = 0.0
        e_sum = 0.0
        for side in range(2):
            K = int(om.face_el[f, side])
            X, S, Ek = loc[K]
            sz = [4 * (om.face_p[e] + 1) for e in om.elem_face[K]]
            off = np.concatenate([[0], np.cumsum(sz)])
            a = list(om.elem_face[K]).index(f)
            diag = diag + S[off[a]:off[a + 1], off[a]:off[a + 1]]
            e_sum = e_sum + Ek[off[a]:off[a + 1]]
        slot = list(om.k_col[f]).index(f)
        o0, o1 = om.k_blkoff[5 * f + slot], om.k_blkoff[5 * f + slot + 1]
        assert rel_err(g["K"][o0:o1], diag) < TOL
        assert rel_err(g["E"][om.lam_off[f]:om.lam_off[f + 1]], e_sum) < TOL


def test_step_host_matches_device_path(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 6, 6)
    case, om, U, Lam, dLam = build_case(wl)
    _, _, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    sysm = hdg.System(ctx, mesh, lib_params(wl))
    Uh = torch.from_numpy(U).pin_memory()
    Lh = torch.from_numpy(Lam).pin_memory()
    dLh = torch.from_numpy(dLam).pin_memory()
    dUh = torch.empty(mesh.u_len, dtype=torch.float64).pin_memory()
    sysm.step_host(Uh, Lh, dLh, dUh)
    assert np.array_equal(dUh.numpy(), g["dU"])
    assert sysm.launches >= 2


def test_bad_mesh_rejected(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p1_256"], 4, 4)
    case = G.make_case(wl)
    xy = case.mesh.elem_xy.copy()
    xy[3] = xy[3][::-1]  # clockwise element
    with pytest.raises(hdg.HdgError) as ei:
        hdg.Mesh(ctx, xy, case.mesh.elem_vid, case.elem_p, 4)
    assert ei.value.status == hdg.HDG_EINVAL
    with pytest.raises(hdg.HdgError):
        hdg.Mesh(ctx, case.mesh.elem_xy[:-1], case.mesh.elem_vid[:-1], case.elem_p[:-1], 4)  # open mesh
    p = case.elem_p.copy(); p[0] = 7
    with pytest.raises(hdg.HdgError):
        hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, p, 4)
