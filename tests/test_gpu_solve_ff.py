"""The GPU trace solve with its products, preconditioner sweeps and Gram-Schmidt
in double-word arithmetic on the binary32 pipe (hdg_solver_set_arithmetic(S, 1)),
against the dense solve of the oracle's own K, E (Eq. hybridsystem), for K and
for K^T (the lane-ordered matrix copies are built per transpose flag), and the
true residual of the full-size system; the iteration count matches the binary64
solver's."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import lib_params, oracle_params, rel_err
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_3995_gb300 import hdg
    return hdg.Context(0)


def _setup(ctx, wl, cfl):
    from paper_1308_3995_gb300 import hdg
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, _ = G.case_state(case, om.face_vid, om.face_p)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl, cfl))
    dev = torch.device("cuda:0")
    sysm.condense(torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev))
    return om, U, Lam, mesh, sysm


@pytest.mark.parametrize("precond", [0, 1, 2, 3])
@pytest.mark.parametrize("name,nx,ny,kw", [("euler_p3_16k", 5, 6, {}), ("ns_mixp_65k", 4, 5, {}),
                                           ("euler_box_8k", 6, 6, {})])
def test_float_float_solve_matches_dense_oracle_solve(ctx, name, nx, ny, kw, precond):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    r = om.condense(oracle_params(wl, 10.0), U, Lam)
    ref = O.dense_solve(om.dense_K(r["K"]), r["E"])
    its = {}
    for arith in (0, 1):
        solver = hdg.Solver(sysm, restart=30, precond=precond)
        solver.set_arithmetic(arith)
        x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
        it, rel = solver.solve(x, rtol=1e-12, max_iter=2000)
        err = rel_err(x.cpu().numpy(), ref)
        its[arith] = it
        print(wl.name, precond, "arith", arith, "iterations", it, f"rel {rel:.1e} err {err:.1e}")
        assert rel <= 1e-12 and err < 1e-10
        solver.close()
    assert abs(its[1] - its[0]) <= 2


@pytest.mark.parametrize("precond", [0, 2])
def test_float_float_solve_full_size_true_residual(ctx, precond):
    from paper_1308_3995_gb300 import hdg
    wl = G.WORKLOADS["euler_p3_16k"]
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    solver = hdg.Solver(sysm, restart=30, precond=precond)
    solver.set_arithmetic(1)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    it, rel = solver.solve(x, rtol=1e-12, max_iter=800)
    y = torch.empty_like(x)
    solver.matvec(x, y)          # binary64 product
    torch.cuda.synchronize()
    E = sysm.views()["E"].cpu().numpy()
    true_rel = np.linalg.norm(E - y.cpu().numpy()) / np.linalg.norm(E)
    print("float-float GMRES", precond, "iterations", it, f"preconditioned {rel:.1e} true {true_rel:.1e}")
    assert rel <= 1e-12 and true_rel < 1e-10


def test_arithmetic_is_validated(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p1_256"], 4, 4)
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    solver = hdg.Solver(sysm)
    with pytest.raises(hdg.HdgError) as ei:
        solver.set_arithmetic(2)
    assert ei.value.status == hdg.HDG_EINVAL


@pytest.mark.parametrize("precond", [0, 1, 2, 3])
@pytest.mark.parametrize("name,nx,ny,kw", [("ns_mixp_65k", 4, 5, {}), ("euler_p3_16k", 4, 4, {"p": 4}),
                                           ("ns_mixp_65k", 5, 4, {"model": 0})])
def test_float_float_transposed_solve_matches_dense_oracle(ctx, name, nx, ny, kw, precond):
    """K^T x = r with mixed face sizes (every pair of lane orders), after a solve with K on the same
    solver (the copies are rebuilt for the transpose), against the oracle's dense K^T."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    r = om.condense(oracle_params(wl, 10.0), U, Lam)
    Kd = om.dense_K(r["K"])
    rhs = np.random.default_rng(5).standard_normal(mesh.lam_len)
    solver = hdg.Solver(sysm, restart=30, precond=precond)
    solver.set_arithmetic(1)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    it, rel = solver.solve(x, rtol=1e-12, max_iter=2000)
    assert rel <= 1e-12 and rel_err(x.cpu().numpy(), O.dense_solve(Kd, r["E"])) < 1e-10
    x.zero_()
    it, rel = solver.solve(x, rtol=1e-12, max_iter=2000, rhs=torch.from_numpy(rhs).to("cuda:0"), transpose=True)
    err = rel_err(x.cpu().numpy(), np.linalg.solve(Kd.T, rhs))
    print(wl.name, precond, "transposed, iterations", it, f"rel {rel:.1e} err {err:.1e}")
    assert rel <= 1e-12 and err < 1e-10
    solver.close()


def test_float_float_needs_setup_before_binary64_apply(ctx):
    """After a double-word solve with block Jacobi only the binary32 pivot inverses are current:
    the binary64 preconditioner apply asks for a setup, and gives M^{-1} r after one."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 4, 4)
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    solver = hdg.Solver(sysm, restart=30, precond=0)
    solver.set_arithmetic(1)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    solver.solve(x, rtol=1e-10, max_iter=500)
    rv = torch.from_numpy(np.random.default_rng(2).standard_normal(mesh.lam_len)).to("cuda:0")
    z = torch.empty_like(rv)
    with pytest.raises(hdg.HdgError) as ei:
        solver.precond_apply(rv, z)
    assert ei.value.status == hdg.HDG_EINVAL
    solver.setup()
    solver.precond_apply(rv, z)
    torch.cuda.synchronize()
    # z_e = K_ee^{-1} r_e with the oracle's diagonal blocks
    Kd = om.dense_K(om.condense(oracle_params(wl, 10.0), U, Lam)["K"])
    rn, ref, lo = rv.cpu().numpy(), np.empty(mesh.lam_len), 0
    for pe in mesh.face_p:
        m = 4 * (int(pe) + 1)
        ref[lo:lo + m] = np.linalg.solve(Kd[lo:lo + m, lo:lo + m], rn[lo:lo + m])
        lo += m
    assert rel_err(z.cpu().numpy(), ref) < 1e-12
    solver.close()


def test_float_float_refused_in_a_callers_workspace(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p1_256"], 4, 4)
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    nb = hdg.Solver.workspace_bytes(mesh, 30, 0)
    ws = torch.empty(nb // 8 + 64, dtype=torch.float64, device="cuda:0")
    solver = hdg.Solver(sysm, restart=30, precond=0, workspace=(ws.data_ptr(), ws.numel() * 8))
    with pytest.raises(hdg.HdgError) as ei:
        solver.set_arithmetic(1)
    assert ei.value.status == hdg.HDG_ENOMEM
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    it, rel = solver.solve(x, rtol=1e-10, max_iter=500)        # still binary64 and working
    assert rel <= 1e-10
    solver.close()


@pytest.mark.parametrize("precond", [0, 2, 3])
def test_float_float_solver_planned_in_a_callers_workspace(ctx, precond):
    """hdg_solver_create_ws_arith(..., arith 1, ...): the double-word copies planned into the caller's
    workspace (a larger plan than binary64's), the solver starts in float-float arithmetic and matches
    the dense oracle solve, twice in a row."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 4, 5)
    om, U, Lam, mesh, sysm = _setup(ctx, wl, 10.0)
    r = om.condense(oracle_params(wl, 10.0), U, Lam)
    ref = O.dense_solve(om.dense_K(r["K"]), r["E"])
    n0 = hdg.Solver.workspace_bytes(mesh, 30, precond, 0)
    n1 = hdg.Solver.workspace_bytes(mesh, 30, precond, 1)
    assert n1 > n0
    ws = torch.empty(n1 // 8 + 64, dtype=torch.float64, device="cuda:0")
    solver = hdg.Solver(sysm, restart=30, precond=precond, workspace=(ws.data_ptr(), n1), arith=1)
    solver.set_arithmetic(1)                    # already planned: no allocation, no error
    for _ in range(2):
        x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
        it, rel = solver.solve(x, rtol=1e-12, max_iter=2000)
        assert rel <= 1e-12 and rel_err(x.cpu().numpy(), ref) < 1e-10
    solver.close()
    with pytest.raises(hdg.HdgError) as ei:      # a binary64-sized workspace is too short for arith 1
        hdg.Solver(sysm, restart=30, precond=precond, workspace=(ws.data_ptr(), n0), arith=1)
    assert ei.value.status == hdg.HDG_EINVAL
