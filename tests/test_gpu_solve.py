"""GPU trace solve (Sec. 3.4, Eq. hybridsystem: K dLambda = E) and the pseudo-transient
Newton update (Sec. 3.3) against the FP64 oracle: the dense solve of the oracle's own K and E,
and the oracle's monolithic Newton steps on tiny meshes."""
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


def setup(ctx, wl, cfl, precision=0):
    from paper_1308_3995_gb300 import hdg
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, dLam = G.case_state(case, om.face_vid, om.face_p)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl, cfl, precision))
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    return case, om, U, Lam, mesh, sysm, Ut, Lt


PRECOND_NAMES = ["block Jacobi", "block SGS", "block ILU(0)", "block ILU(0) binary32"]


@pytest.mark.parametrize("precond", [0, 1, 2, 3])
@pytest.mark.parametrize("name,nx,ny,kw", [("euler_p3_16k", 5, 6, {}), ("ns_mixp_65k", 4, 5, {}),
                                           ("ns_mixp_65k", 5, 5, {"model": 0})])
def test_trace_solve_matches_dense_oracle_solve(ctx, name, nx, ny, kw, precond):
    """GMRES + block Jacobi on the GPU's K, E against the dense LU solve of the oracle's K, E."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    cfl = 10.0
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, cfl)
    sysm.condense(Ut, Lt)
    solver = hdg.Solver(sysm, restart=30, precond=precond)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    it, rel = solver.solve(x, rtol=1e-13, max_iter=400)
    r = om.condense(oracle_params(wl, cfl), U, Lam)
    ref = O.dense_solve(om.dense_K(r["K"]), r["E"])
    err = rel_err(x.cpu().numpy(), ref)
    print(wl.name, PRECOND_NAMES[precond], "iterations", it, "rel. residual", f"{rel:.1e}",
          "error vs dense oracle", f"{err:.1e}")
    assert rel <= 1e-13 and err < 1e-10
    # the matrix-vector product against the dense oracle matrix
    v = torch.from_numpy(np.random.default_rng(3).standard_normal(mesh.lam_len)).to("cuda:0")
    y = torch.empty_like(v)
    solver.matvec(v, y)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), om.dense_K(r["K"]) @ v.cpu().numpy()) < 1e-13
    solver.close(); sysm.close(); mesh.close()


@pytest.mark.parametrize("precond", [0, 2, 3])
def test_trace_solve_full_size_true_residual(ctx, precond):
    """16,384-element p = 3 workload at CFL 10: the true residual ||E - K dLambda|| (matrix-vector
    product checked row by row against the host copy of K) is small after the solve."""
    from paper_1308_3995_gb300 import hdg
    wl = G.WORKLOADS["euler_p3_16k"]
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, 10.0)
    sysm.condense(Ut, Lt)
    solver = hdg.Solver(sysm, restart=30, precond=precond)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    it, rel = solver.solve(x, rtol=1e-12, max_iter=600)
    y = torch.empty_like(x)
    solver.matvec(x, y)
    torch.cuda.synchronize()
    v = sysm.views()
    E = v["E"].cpu().numpy()
    Kh = v["K"].cpu().numpy()
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    rng = np.random.default_rng(5)
    for e in rng.choice(mesh.n_face, 40, replace=False):   # rows of face e, from the host copy
        m = 4 * (mesh.face_p[e] + 1)
        acc = np.zeros(m)
        for b in range(5):
            c = mesh.k_col.reshape(-1)[5 * e + b]
            mb = 4 * (mesh.face_p[c] + 1)
            blk = Kh[mesh.k_blkoff[5 * e + b]:mesh.k_blkoff[5 * e + b + 1]].reshape(m, mb)
            acc += blk @ xh[mesh.lam_off[c]:mesh.lam_off[c] + mb]
        assert rel_err(yh[mesh.lam_off[e]:mesh.lam_off[e] + m], acc) < 1e-13
    true_rel = np.linalg.norm(E - yh) / np.linalg.norm(E)
    print(PRECOND_NAMES[precond], "iterations", it, "preconditioned", f"{rel:.1e}", "true", f"{true_rel:.1e}")
    assert rel <= 1e-12 and true_rel < 1e-10
    solver.close(); sysm.close(); mesh.close()


@pytest.mark.parametrize("name,nx,ny,kw", [("euler_p1_256", 3, 3, {"jitter": 0.2}),
                                           ("ns_mixp_65k", 3, 3, {"p": 2, "probs": None})])
def test_newton_steps_match_oracle_monolithic(ctx, name, nx, ny, kw):
    """Three pseudo-transient Newton steps with the CFL law (Eq. cfl, c0 = 10, n0 = 2): condense,
    GPU trace solve, reconstruct, update -- against the oracle's monolithic Newton steps (the
    Jacobian of the global residual by complex step, dense solve), state and residual norm."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, 1.0)
    if om.u_len + om.lam_len > 4000:
        pytest.skip("too large for the dense monolithic solve")
    solver = hdg.Solver(sysm, restart=40)
    dL = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    dU = torch.zeros(mesh.u_len, dtype=torch.float64, device="cuda:0")
    Uo, Lo = U.copy(), Lam.copy()
    cfl_g = cfl_o = 0.0
    rg_prev = ro_prev = None
    for n in range(1, 4):
        # oracle: residual norm of the current state, CFL law, monolithic step
        Ru, Rl = om.global_residual(oracle_params(wl), Uo, Lo)
        ro = float(np.sqrt((Ru ** 2).sum() + (Rl ** 2).sum()))
        cfl_o = O.cfl_law(n, c0=10.0, c1=1.0, n0=2, cfl_prev=cfl_o, res_prev=ro_prev or ro, res_cur=ro)
        dUo, dLo = om.monolithic(oracle_params(wl, cfl_o), Uo, Lo)
        Uo, Lo, ro_prev = Uo + dUo, Lo + dLo, ro
        # GPU: condense at this step's CFL (its residual is that of the current state)
        sysm.condense(Ut, Lt)                  # residual only; the CFL is applied below
        rg = sysm.residual_norm()
        cfl_g = hdg.cfl_law(n, c0=10.0, c1=1.0, n0=2, cfl_prev=cfl_g, res_prev=rg_prev or rg, res_cur=rg)
        sysm.set_cfl(cfl_g)
        sysm.condense(Ut, Lt)
        dL.zero_()
        solver.solve(dL, rtol=1e-14, max_iter=1000)
        sysm.recover(dL, dU)
        sysm.newton_update(Ut, Lt, dU, dL)
        torch.cuda.synchronize()
        rg_prev = rg
        print(n, f"cfl {cfl_g:.4g}", f"res {rg:.3e} / {ro:.3e}")
        assert abs(rg - ro) < 1e-10 * ro and abs(cfl_g - cfl_o) < 1e-9 * cfl_o
        assert rel_err(Ut.cpu().numpy(), Uo) < 1e-10 and rel_err(Lt.cpu().numpy(), Lo) < 1e-10
    solver.close(); sysm.close(); mesh.close()


def test_trace_solve_reports_timeout_and_singular_blocks(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 4, 4)
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, 10.0)
    sysm.condense(Ut, Lt)
    solver = hdg.Solver(sysm, restart=10)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hdg.HdgError) as ei:
        solver.solve(x, rtol=1e-15, max_iter=2)
    assert ei.value.status == hdg.HDG_ETIMEOUT
    it, rel = solver.solve(x.zero_(), rtol=1e-15, max_iter=2, check=False)
    assert it == 2 and rel > 1e-15
    sysm.views()["K"].zero_()                              # every diagonal block singular
    with pytest.raises(hdg.HdgError) as ei:
        solver.solve(x.zero_(), rtol=1e-10, max_iter=10)
    assert ei.value.status == hdg.HDG_ESINGULAR
    solver.close(); sysm.close(); mesh.close()


@pytest.mark.parametrize("name,nx,ny,kw,precision", [("euler_p1_256", 3, 3, {"jitter": 0.2}, 0),
                                                     ("euler_p3_16k", 3, 3, {}, 0),
                                                     ("ns_mixp_65k", 3, 4, {"model": 0}, 0),
                                                     ("euler_p3_16k", 3, 3, {}, 1),
                                                     ("ns_mixp_65k", 3, 3, {}, 0),
                                                     ("ns_mixp_65k", 3, 3, {}, 1),
                                                     ("ns_wall_channel_8k", 3, 3, {}, 0),
                                                     ("ns_mixp_65k", 3, 3, {"p": 4, "probs": None}, 0)])
@pytest.mark.parametrize("precond", [0, 1, 2, 3])
def test_hybridized_adjoint_matches_transposed_monolithic_solve(ctx, name, nx, ny, kw, precision, precond):
    """Sec. 4.2: the adjoint of the Newton matrix (pseudo-time mass included, CFL 10) with right-hand
    side [F~; 0]: GPU adjoint local solves, E~ = -X_B^T F~, GMRES on K^T, reconstruction -- against
    the dense solve of the transposed monolithic Jacobian of the oracle (complex step).  Navier-Stokes
    (periodic and between no-slip walls): F~ on all of [Q; W], through the transposed in-element q
    elimination."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    cfl = 10.0
    case, om, U, Lam, mesh, primal, Ut, Lt = setup(ctx, wl, cfl, precision)
    adj = hdg.System(ctx, mesh, lib_params(wl, cfl, precision))
    Ft = np.random.default_rng(11).standard_normal(mesh.u_len)       # stands in for J'(U)
    Ftt = torch.from_numpy(Ft).to("cuda:0")
    primal.condense(Ut, Lt)
    adj.adjoint_condense(primal, Ut, Lt, Ftt)
    solver = hdg.Solver(primal, restart=40, precond=precond)
    lt = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    ut = torch.zeros(mesh.u_len, dtype=torch.float64, device="cuda:0")
    it, rel = solver.solve(lt, rtol=1e-14, max_iter=1000, rhs=adj.views()["E"], transpose=True)
    adj.recover(lt, ut)
    torch.cuda.synchronize()
    _, _, J = om.monolithic(oracle_params(wl, cfl), U, Lam, want_matrix=True)
    z = np.linalg.solve(J.T, np.concatenate([Ft, np.zeros(om.lam_len)]))
    eu, el = rel_err(ut.cpu().numpy(), z[:om.u_len]), rel_err(lt.cpu().numpy(), z[om.u_len:])
    print(wl.name, ["fp64", "float2"][precision], "iterations", it, f"adjoint U~ {eu:.1e} Lambda~ {el:.1e}")
    tol = [1e-10, 1e-9][precision]
    assert eu < tol and el < tol
    # the transposed product against the oracle's dense K^T
    r = om.condense(oracle_params(wl, cfl), U, Lam)
    v = torch.from_numpy(np.random.default_rng(4).standard_normal(mesh.lam_len)).to("cuda:0")
    y = torch.empty_like(v)
    solver.matvec(v, y, transpose=True)
    torch.cuda.synchronize()
    assert rel_err(y.cpu().numpy(), om.dense_K(r["K"]).T @ v.cpu().numpy()) < [1e-13, 1e-11][precision]
    solver.close(); adj.close(); primal.close(); mesh.close()


def test_adjoint_rejects_mismatched_systems(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 3, 3)
    case, om, U, Lam, mesh, primal, Ut, Lt = setup(ctx, wl, 10.0)
    other = hdg.System(ctx, mesh, lib_params(wl, 5.0))
    Ft = torch.zeros(mesh.u_len, dtype=torch.float64, device="cuda:0")
    with pytest.raises(hdg.HdgError) as ei:
        other.adjoint_condense(primal, Ut, Lt, Ft)
    assert ei.value.status == hdg.HDG_EINVAL
    other.close(); primal.close(); mesh.close()


@pytest.mark.parametrize("name,nx,ny,kw,cfl", [("euler_p3_16k", 5, 6, {}, 10.0),
                                               ("ns_mixp_65k", 4, 5, {}, 10.0),
                                               ("ns_mixp_65k", 5, 4, {"model": 0}, 0.0),
                                               ("euler_channel_8k", 5, 4, {"p": 2}, 10.0),
                                               ("euler_box_8k", 4, 4, {"p": 3}, 0.0)])
def test_block_ilu0_preconditioner_matches_oracle(ctx, name, nx, ny, kw, cfl):
    """z = M^{-1} r and M^{-T} r of the GPU block ILU(0) against the oracle's textbook block
    ILU(0) of the same K, eliminated in the GPU's color sequence (any order within a color gives
    the same factors); the coloring leaves no two faces of one element in one color."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, cfl)
    sysm.condense(Ut, Lt)
    solver = hdg.Solver(sysm, restart=10, precond=2)
    solver.setup()
    solver32 = hdg.Solver(sysm, restart=10, precond=3)
    solver32.setup()
    color, nc = solver.colors()
    P = O.trace_pattern(om)
    assert nc <= 8 and all(color[i] != color[j] for (i, j) in P if i != j)
    Kd = om.dense_K(sysm.views()["K"].cpu().numpy())
    offs = np.asarray(om.lam_off[:om.n_face + 1], dtype=np.int64)
    order = np.argsort(color.astype(np.int64) * om.n_face + np.arange(om.n_face), kind="stable")
    L, Uf, perm = O.block_ilu0(Kd, offs, P, order)
    rng = np.random.default_rng(7)
    for transpose in (False, True):
        r = rng.standard_normal(mesh.lam_len)
        z = torch.empty(mesh.lam_len, dtype=torch.float64, device="cuda:0")
        solver.precond_apply(torch.from_numpy(r).to("cuda:0"), z, transpose=transpose)
        torch.cuda.synchronize()
        ref = O.block_ilu0_apply(L, Uf, perm, r, transpose=transpose)
        err = np.abs(z.cpu().numpy() - ref).max() / np.abs(ref).max()
        # binary32 factors: the same incomplete factorization to binary32 rounding
        solver32.precond_apply(torch.from_numpy(r).to("cuda:0"), z, transpose=transpose)
        torch.cuda.synchronize()
        err32 = np.abs(z.cpu().numpy() - ref).max() / np.abs(ref).max()
        print(wl.name, "colors", nc, "transpose" if transpose else "", f"{err:.1e}", f"binary32 factors {err32:.1e}")
        assert err < 1e-11 and err32 < 1e-4
    solver32.close(); solver.close(); sysm.close(); mesh.close()


def test_solver_api_rejects_bad_use(ctx):
    """Host-side checks of the solver calls: a workspace smaller than planned or misaligned, a
    switch to an ILU(0) kind the workspace was not planned for, an unknown kind, applying the
    preconditioner before it is set up; a zero right-hand side returns zero at once."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 3, 4)
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, 10.0)
    sysm.condense(Ut, Lt)
    need = hdg.Solver.workspace_bytes(mesh, 20, 0)
    assert hdg.Solver.workspace_bytes(mesh, 20, 2) > need and hdg.Solver.workspace_bytes(mesh, 20, 3) > need
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda:0")
    with pytest.raises(hdg.HdgError) as ei:
        hdg.Solver(sysm, 20, 0, workspace=(buf.data_ptr(), need - 256))
    assert ei.value.status == hdg.HDG_EINVAL
    with pytest.raises(hdg.HdgError) as ei:
        hdg.Solver(sysm, 20, 0, workspace=(buf.data_ptr() + 8, need))
    assert ei.value.status == hdg.HDG_EINVAL
    s = hdg.Solver(sysm, 20, 0, workspace=(buf.data_ptr(), need))
    with pytest.raises(hdg.HdgError) as ei:
        s.set_preconditioner(2)                     # not planned in the caller's workspace
    assert ei.value.status == hdg.HDG_ENOMEM
    with pytest.raises(hdg.HdgError) as ei:
        s.set_preconditioner(4)
    assert ei.value.status == hdg.HDG_EINVAL
    r = torch.randn(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    z = torch.empty_like(r)
    with pytest.raises(hdg.HdgError) as ei:
        s.precond_apply(r, z)                       # no setup yet
    assert ei.value.status == hdg.HDG_EINVAL
    s.setup()
    s.precond_apply(r, z)
    x = torch.ones(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    it, rel = s.solve(x, rtol=1e-10, rhs=torch.zeros_like(r))
    torch.cuda.synchronize()
    assert it == 0 and float(x.abs().max()) == 0.0
    s.close(); sysm.close(); mesh.close()


def test_source_and_cfl_are_frozen_by_a_captured_graph(ctx):
    """A captured step holds the system's parameters: changing the CFL or the source afterwards is
    refused (HDG_EINVAL) instead of silently not taking effect."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 3, 4)
    case, om, U, Lam, mesh, sysm, Ut, Lt = setup(ctx, wl, 10.0)
    dLt = torch.zeros(mesh.lam_len, dtype=torch.float64, device="cuda:0")
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device="cuda:0")
    sysm.graph_create(Ut, Lt, dLt, dUt)
    with pytest.raises(hdg.HdgError) as ei:
        sysm.set_cfl(5.0)
    assert ei.value.status == hdg.HDG_EINVAL
    with pytest.raises(hdg.HdgError) as ei:
        sysm.set_source(torch.zeros(mesh.u_len, dtype=torch.float64, device="cuda:0"))
    assert ei.value.status == hdg.HDG_EINVAL
    sysm.close(); mesh.close()
