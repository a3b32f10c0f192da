"""Bounded domains (Sec. 2.1, 3.2): slip-wall and characteristic far-field boundary operators in the
element kernel, boundary faces without trace unknowns, and a steady Newton solve on the GPU --
against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import ParityChecker, lib_params, oracle_params, rel_err
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL, TOL_MIXED = 1e-12, 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_3995_gb300 import hdg
    return hdg.Context(0)


def _setup(ctx, wl, cfl=0.0, precision=0, sc=0.0):
    from paper_1308_3995_gb300 import hdg
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, dLam = G.case_state(case, om.face_vid, om.face_p)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl, cfl, precision, sc))
    return case, om, U, Lam, dLam, mesh, sysm


def _run(sysm, mesh, U, Lam, dLam):
    dev = torch.device("cuda:0")
    Ut, Lt, dLt = (torch.from_numpy(a).to(dev) for a in (U, Lam, dLam))
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    sysm.condense(Ut, Lt)
    sysm.recover(dLt, dUt)
    torch.cuda.synchronize()
    g = {k: t.cpu().numpy().copy() for k, t in sysm.views().items()}
    g["dU"] = dUt.cpu().numpy()
    return g


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p,cfl,sc", [(1, 0.0, 0.0), (2, 0.0, 0.0), (3, 10.0, 0.0), (4, 0.0, 0.0),
                                      (None, 0.0, 0.0), (3, 0.0, 0.2)])
def test_channel_parity(ctx, precision, p, cfl, sc):
    """Every element and face of a channel mesh (slip wall below, far field above), element by element."""
    kw = {"p": p} if p else {"p": None, "probs": (0.4, 0.3, 0.2, 0.1)}
    wl = G.small_variant(G.WORKLOADS["euler_channel_8k"], 6, 5, **kw)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, cfl, precision, sc)
    for name in ("face_vid", "face_el", "face_p", "elem_face", "u_off", "lam_off", "x_off", "k_col", "k_blkoff"):
        assert np.array_equal(np.asarray(getattr(mesh, name)).ravel(), np.asarray(getattr(om, name)).ravel()), name
    assert (np.asarray(mesh.k_col) < 0).any()
    g = _run(sysm, mesh, U, Lam, dLam)
    assert np.all(g["status"] == 0)
    chk = ParityChecker(om, oracle_params(wl, cfl, sc), U, Lam, dLam, g)
    errs = chk.run(range(om.n_elem), range(om.n_face))
    print(wl.name, p, cfl, sc, ["fp64", "float2"][precision], {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < [TOL, TOL_MIXED][precision], (k, v)
    sysm.close(); mesh.close()


def test_channel_free_stream_residual_vanishes(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_channel_8k"], 8, 6, p=3)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl)
    winf = G.conserved(*G.free_stream(wl.mach, 0.0))
    U = np.zeros(mesh.u_len); L = np.zeros(mesh.lam_len)
    nb = 10
    for f in range(4):
        U.reshape(-1, 4 * nb)[:, f * nb] = winf[f] / np.sqrt(2)
        L.reshape(-1, 16)[:, f * 4] = winf[f]
    g = _run(sysm, mesh, U, L, np.zeros(mesh.lam_len))
    assert np.abs(g["res_u"]).max() < 1e-14 and np.abs(g["res_lam"]).max() < 1e-14
    sysm.close(); mesh.close()


def test_channel_newton_steps_match_oracle_monolithic(ctx):
    """Three Newton steps (CFL law, c0 = 10, n0 = 2) on a small channel: GPU condense + GMRES trace
    solve + reconstruction + update against the oracle's monolithic Newton steps."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_channel_8k"], 4, 4, p=2)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, 1.0)
    assert om.u_len + om.lam_len <= 4000
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    solver = hdg.Solver(sysm, restart=40)
    dL = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    dU = torch.zeros(mesh.u_len, dtype=torch.float64, device=dev)
    Uo, Lo = U.copy(), Lam.copy()
    cfl_g = cfl_o = 0.0
    rg_prev = ro_prev = None
    for n in range(1, 4):
        Ru, Rl = om.global_residual(oracle_params(wl), Uo, Lo)
        ro = float(np.sqrt((Ru ** 2).sum() + (Rl ** 2).sum()))
        cfl_o = O.cfl_law(n, c0=10.0, c1=1.0, n0=2, cfl_prev=cfl_o, res_prev=ro_prev or ro, res_cur=ro)
        dUo, dLo = om.monolithic(oracle_params(wl, cfl_o), Uo, Lo)
        Uo, Lo, ro_prev = Uo + dUo, Lo + dLo, ro
        sysm.condense(Ut, Lt)
        rg = sysm.residual_norm()
        cfl_g = hdg.cfl_law(n, c0=10.0, c1=1.0, n0=2, cfl_prev=cfl_g, res_prev=rg_prev or rg, res_cur=rg)
        sysm.set_cfl(cfl_g)
        sysm.condense(Ut, Lt)
        dL.zero_()
        solver.solve(dL, rtol=1e-14, max_iter=2000)
        sysm.recover(dL, dU)
        sysm.newton_update(Ut, Lt, dU, dL)
        torch.cuda.synchronize()
        rg_prev = rg
        print(n, f"cfl {cfl_g:.4g}", f"res {rg:.3e} / {ro:.3e}")
        assert abs(rg - ro) < 1e-10 * ro
        assert rel_err(Ut.cpu().numpy(), Uo) < 1e-10 and rel_err(Lt.cpu().numpy(), Lo) < 1e-10
    solver.close(); sysm.close(); mesh.close()


@pytest.mark.parametrize("c0,c1,n0,precond", [(1e6, 1e3, 4, 0), (10.0, 10.0, 3, 0)])
def test_box_steady_solve_converges(ctx, c0, c1, n0, precond):
    """A steady Newton solve on the GPU: 8,192-element box with far field on all sides (Euler p = 2,
    Mach 0.5 at 10 degrees, density bump): pseudo time with the CFL law of Eq. (cfl) (the paper's
    c0 = 1e6, c1 = 1e3, n0 = 4, and a gentler ramp), GMRES to 1e-11 each step, until the residual has
    dropped by 1e-10; the converged state is the free stream."""
    from paper_1308_3995_gb300 import hdg
    wl = G.WORKLOADS["euler_box_8k"]
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, 1.0)
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    solver = hdg.Solver(sysm, restart=50, precond=precond)
    dL = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    dU = torch.zeros(mesh.u_len, dtype=torch.float64, device=dev)
    cfl, r_prev, r0 = 0.0, None, None
    hist, its = [], []
    for n in range(1, 40):
        sysm.condense(Ut, Lt)
        r = sysm.residual_norm()
        r0 = r0 or r
        hist.append(r)
        if r < 1e-10 * r0:
            break
        cfl = hdg.cfl_law(n, c0=c0, c1=c1, n0=n0, cfl_prev=cfl, res_prev=r_prev or r, res_cur=r)
        sysm.set_cfl(cfl)
        sysm.condense(Ut, Lt)
        dL.zero_()
        it, _ = solver.solve(dL, rtol=1e-11, max_iter=5000)
        its.append(it)
        sysm.recover(dL, dU)
        sysm.newton_update(Ut, Lt, dU, dL)
        r_prev = r
    print("residual history", " ".join(f"{h:.2e}" for h in hist), "GMRES iterations", its)
    assert hist[-1] < 1e-10 * hist[0]
    winf = G.conserved(*G.free_stream(wl.mach, wl.aoa))
    Uh = Ut.cpu().numpy().reshape(-1, 4, 6)
    assert np.abs(Uh[:, :, 0] * np.sqrt(2) - winf).max() < 1e-8 and np.abs(Uh[:, :, 1:]).max() < 1e-8
    solver.close(); sysm.close(); mesh.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_box_parity(ctx, precision):
    wl = G.small_variant(G.WORKLOADS["euler_box_8k"], 6, 5, p=3)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, 0.0, precision)
    g = _run(sysm, mesh, U, Lam, dLam)
    chk = ParityChecker(om, oracle_params(wl), U, Lam, dLam, g)
    errs = chk.run(range(om.n_elem), range(om.n_face))
    print(wl.name, ["fp64", "float2"][precision], {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < [TOL, TOL_MIXED][precision], (k, v)
    sysm.close(); mesh.close()


def test_channel_adjoint_matches_transposed_monolithic(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_channel_8k"], 4, 3, p=2)
    cfl = 10.0
    case, om, U, Lam, dLam, mesh, primal = _setup(ctx, wl, cfl)
    adj = hdg.System(ctx, mesh, lib_params(wl, cfl))
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    Ft = np.random.default_rng(12).standard_normal(mesh.u_len)
    primal.condense(Ut, Lt)
    adj.adjoint_condense(primal, Ut, Lt, torch.from_numpy(Ft).to(dev))
    solver = hdg.Solver(primal, restart=40)
    lt = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    ut = torch.zeros(mesh.u_len, dtype=torch.float64, device=dev)
    solver.solve(lt, rtol=1e-14, max_iter=2000, rhs=adj.views()["E"], transpose=True)
    adj.recover(lt, ut)
    torch.cuda.synchronize()
    _, _, J = om.monolithic(oracle_params(wl, cfl), U, Lam, want_matrix=True)
    z = np.linalg.solve(J.T, np.concatenate([Ft, np.zeros(om.lam_len)]))
    assert rel_err(ut.cpu().numpy(), z[:om.u_len]) < 1e-10 and rel_err(lt.cpu().numpy(), z[om.u_len:]) < 1e-10
    solver.close(); adj.close(); primal.close(); mesh.close()


def test_boundary_kinds_checked_against_the_model(ctx):
    """Navier-Stokes meshes take no-slip walls and far field, not the slip wall (HDG_ENOTSUP: the
    channel's bottom); the no-slip wall is not an Euler boundary (HDG_EINVAL)."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_channel_8k"], 4, 3, model=1)
    case = G.make_case(wl)
    with pytest.raises(hdg.HdgError) as ei:
        hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    assert ei.value.status == hdg.HDG_ENOTSUP
    wl = G.small_variant(G.WORKLOADS["ns_wall_channel_8k"], 4, 3, model=0, p=2, probs=None)
    case = G.make_case(wl)
    with pytest.raises(hdg.HdgError) as ei:
        hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    assert ei.value.status == hdg.HDG_EINVAL


# ----------------------------------------------------------------------------- Navier-Stokes walls
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("p,cfl,sc", [(1, 0.0, 0.0), (2, 10.0, 0.0), (3, 0.0, 0.0), (4, 0.0, 0.0),
                                      (None, 0.0, 0.0), (None, 10.0, 0.0), (2, 0.0, 0.2)])
def test_ns_wall_channel_parity(ctx, precision, p, cfl, sc):
    """Navier-Stokes between no-slip adiabatic walls (Sec. 2.2, 3.2), every element and face against
    the oracle: wall flux, its Jacobian in the rho and E columns, the wall term of the gradient
    equations inside the in-element q elimination."""
    kw = {"p": p, "probs": None} if p else {}
    wl = G.small_variant(G.WORKLOADS["ns_wall_channel_8k"], 5, 4, **kw)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, cfl, precision, sc)
    for name in ("face_vid", "face_el", "face_p", "elem_face", "u_off", "lam_off", "x_off", "k_col", "k_blkoff"):
        assert np.array_equal(np.asarray(getattr(mesh, name)).ravel(), np.asarray(getattr(om, name)).ravel()), name
    g = _run(sysm, mesh, U, Lam, dLam)
    assert np.all(g["status"] == 0)
    chk = ParityChecker(om, oracle_params(wl, cfl, sc), U, Lam, dLam, g)
    errs = chk.run(range(om.n_elem), range(om.n_face))
    print(wl.name, p, cfl, sc, ["fp64", "float2"][precision], {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < [TOL, TOL_MIXED][precision], (k, v)
    sysm.close(); mesh.close()


def test_ns_wall_channel_rest_state_residual_vanishes(ctx):
    """Fluid at rest between no-slip adiabatic walls: every residual row is zero on the GPU too."""
    wl = G.small_variant(G.WORKLOADS["ns_wall_channel_8k"], 8, 6, p=3, probs=None)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl)
    w0 = G.conserved(1.2, 0.0, 0.0, 0.9 * 0.4)
    nb = 10
    U = np.zeros(mesh.u_len); L = np.zeros(mesh.lam_len)
    for f in range(4):
        U.reshape(-1, 12 * nb)[:, 8 * nb + f * nb] = w0[f] / np.sqrt(2)
        L.reshape(-1, 16)[:, f * 4] = w0[f]
    g = _run(sysm, mesh, U, L, dLam)
    assert np.abs(g["res_u"]).max() < 1e-13 and np.abs(g["res_lam"]).max() < 1e-13
    sysm.close(); mesh.close()


def test_ns_wall_channel_newton_step_matches_oracle_monolithic(ctx):
    """One pseudo-transient Newton step (CFL 10) with walls: GPU condensation, GMRES + block ILU(0)
    trace solve, reconstruction -- against the oracle's monolithic step (complex-step Jacobian of the
    global residual, dense solve)."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["ns_wall_channel_8k"], 3, 3)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, 10.0)
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    sysm.condense(Ut, Lt)
    solver = hdg.Solver(sysm, restart=40, precond=2)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    it, rel = solver.solve(x, rtol=1e-13, max_iter=2000)
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    sysm.recover(x, dUt)
    torch.cuda.synchronize()
    dU, dL = om.monolithic(oracle_params(wl, 10.0), U, Lam)
    eU, eL = rel_err(dUt.cpu().numpy(), dU), rel_err(x.cpu().numpy(), dL)
    print(wl.name, "iterations", it, f"dU {eU:.1e} dLambda {eL:.1e}")
    assert eU < 1e-9 and eL < 1e-9
    solver.close(); sysm.close(); mesh.close()


# ----------------------------------------------------------------------------- Navier-Stokes far field
def _ns_far(kind, nx, ny, **kw):
    """The Navier-Stokes box (far field on all four sides, corner elements with two far-field faces)
    or the boundary layer (no-slip wall below, far field above; flow at 10 degrees so that the far
    field's normal velocity stays clear of the characteristic switch at v_n = 0)."""
    if kind == "box":
        return G.small_variant(G.WORKLOADS["ns_box_8k"], nx, ny, **kw)
    return G.small_variant(G.WORKLOADS["ns_wall_channel_8k"], nx, ny, domain="wall_far_channel", aoa=10.0, **kw)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind,p,cfl,sc", [("box", 1, 0.0, 0.0), ("box", 2, 10.0, 0.0), ("box", 3, 0.0, 0.0),
                                           ("box", 4, 0.0, 0.0), ("box", None, 10.0, 0.0), ("box", 2, 0.0, 0.2),
                                           ("layer", 2, 0.0, 0.0), ("layer", None, 10.0, 0.0)])
def test_ns_far_field_parity(ctx, precision, kind, p, cfl, sc):
    """Navier-Stokes characteristic far field (Sec. 2.1, 3.2), every element and face against the
    oracle: the far-field flux with the viscous flux at the far-field state, its Jacobian in all four
    columns, and the gradient equations' far-field term that couples the fields inside the in-element
    q elimination (A', C', X_q)."""
    kw = {"p": p, "probs": None} if p else {"p": None, "probs": (0.4, 0.3, 0.2, 0.1)}
    wl = _ns_far(kind, 5, 4, **kw)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, cfl, precision, sc)
    assert (case.mesh.elem_bc == 2).any()
    g = _run(sysm, mesh, U, Lam, dLam)
    assert np.all(g["status"] == 0)
    chk = ParityChecker(om, oracle_params(wl, cfl, sc), U, Lam, dLam, g)
    errs = chk.run(range(om.n_elem), range(om.n_face))
    print(wl.name, p, cfl, sc, ["fp64", "float2"][precision], {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < [TOL, TOL_MIXED][precision], (k, v)
    sysm.close(); mesh.close()


def test_ns_far_field_free_stream_residual_vanishes(ctx):
    """The uniform free stream with zero gradient is a steady state of the far-field box on the GPU."""
    wl = _ns_far("box", 6, 5, p=3)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl)
    w0 = G.conserved(*G.free_stream(wl.mach, wl.aoa))
    nb = 10
    U = np.zeros(mesh.u_len); L = np.zeros(mesh.lam_len)
    for f in range(4):
        U.reshape(-1, 12 * nb)[:, 8 * nb + f * nb] = w0[f] / np.sqrt(2)
        L.reshape(-1, 16)[:, f * 4] = w0[f]
    g = _run(sysm, mesh, U, L, dLam)
    assert np.abs(g["res_u"]).max() < 1e-13 and np.abs(g["res_lam"]).max() < 1e-13
    sysm.close(); mesh.close()


@pytest.mark.parametrize("kind", ["box", "layer"])
def test_ns_far_field_newton_step_matches_oracle_monolithic(ctx, kind):
    """One pseudo-transient Newton step (CFL 10) with far-field faces: GPU condensation, GMRES + block
    ILU(0) trace solve, reconstruction -- against the oracle's monolithic step."""
    from paper_1308_3995_gb300 import hdg
    wl = _ns_far(kind, 3, 3)
    case, om, U, Lam, dLam, mesh, sysm = _setup(ctx, wl, 10.0)
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    sysm.condense(Ut, Lt)
    solver = hdg.Solver(sysm, restart=40, precond=2)
    x = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    it, rel = solver.solve(x, rtol=1e-13, max_iter=2000)
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    sysm.recover(x, dUt)
    torch.cuda.synchronize()
    dU, dL = om.monolithic(oracle_params(wl, 10.0), U, Lam)
    eU, eL = rel_err(dUt.cpu().numpy(), dU), rel_err(x.cpu().numpy(), dL)
    print(wl.name, "iterations", it, f"dU {eU:.1e} dLambda {eL:.1e}")
    assert eU < 1e-9 and eL < 1e-9
    solver.close(); sysm.close(); mesh.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ns_far_field_adjoint_matches_transposed_monolithic(ctx, precision):
    """The hybridized adjoint (Sec. 4.2) with far-field faces: the transposed q elimination with the
    field-coupling far-field term, K^T solve and reconstruction, against the dense solve of the
    transposed monolithic Jacobian of the oracle."""
    from paper_1308_3995_gb300 import hdg
    wl = _ns_far("box", 3, 3, p=2)
    cfl = 10.0
    case, om, U, Lam, dLam, mesh, primal = _setup(ctx, wl, cfl, precision)
    adj = hdg.System(ctx, mesh, lib_params(wl, cfl, precision))
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    Ft = np.random.default_rng(13).standard_normal(mesh.u_len)
    primal.condense(Ut, Lt)
    adj.adjoint_condense(primal, Ut, Lt, torch.from_numpy(Ft).to(dev))
    solver = hdg.Solver(primal, restart=40, precond=2)
    lt = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    ut = torch.zeros(mesh.u_len, dtype=torch.float64, device=dev)
    solver.solve(lt, rtol=1e-14, max_iter=2000, rhs=adj.views()["E"], transpose=True)
    adj.recover(lt, ut)
    torch.cuda.synchronize()
    _, _, J = om.monolithic(oracle_params(wl, cfl), U, Lam, want_matrix=True)
    z = np.linalg.solve(J.T, np.concatenate([Ft, np.zeros(om.lam_len)]))
    eu, el = rel_err(ut.cpu().numpy(), z[:om.u_len]), rel_err(lt.cpu().numpy(), z[om.u_len:])
    print(wl.name, ["fp64", "float2"][precision], f"adjoint U~ {eu:.1e} Lambda~ {el:.1e}")
    tol = [1e-10, 1e-9][precision]
    assert eu < tol and el < tol
    solver.close(); adj.close(); primal.close(); mesh.close()
