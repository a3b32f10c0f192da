"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by
element, on the same seeded inputs.  Bar (FP64 path): 1e-12, as relative error
per element / block for the local solves X_B and the trace blocks, and as
backward error relative to the magnitude of the summed terms for the
residual-type outputs (see hdg_testlib.ParityChecker); layouts bit-exact."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import ParityChecker, lib_params, oracle_params, rel_err
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
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, dLam = G.case_state(case, om.face_vid, om.face_p)
    return case, om, U, Lam, dLam


def run_gpu(ctx, case, wl, U, Lam, dLam, cfl=0.0, repeat=1, precision=0, sc=0.0):
    from paper_1308_3995_gb300 import hdg
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl, cfl, precision, sc))
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


def full_parity(ctx, wl, cfl=0.0, precision=0, tol=TOL, sc=0.0):
    """Every element and every face of a small case, element by element."""
    case, om, U, Lam, dLam = build_case(wl)
    mesh, sysm, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam, cfl, precision=precision, sc=sc)
    assert_layout_equal(mesh, om)
    assert np.all(g["status"] == 0)
    chk = ParityChecker(om, oracle_params(wl, cfl, sc), U, Lam, dLam, g)
    errs = chk.run(range(om.n_elem), range(om.n_face))
    # plain normwise relative errors over the mesh, for the record
    r = om.condense(oracle_params(wl, cfl, sc), U, Lam)
    info = {"normwise E": rel_err(g["E"], r["E"]), "normwise dU": rel_err(g["dU"], om.recover(r["X"], dLam))}
    print(wl.name, ["fp64", "float2"][precision], {k: f"{v:.1e}" for k, v in {**errs, **info}.items()})
    for k, v in errs.items():
        assert v < tol, (k, v)
    return errs


# float-float path (binary32 pairs on the FP32 pipe): bar 1e-10 (mixed-precision tolerance)
TOL_MIXED = 1e-10


@pytest.mark.parametrize("name,nx,ny,kw", [
    ("euler_p1_256", 8, 16, {}),
    ("euler_p3_16k", 6, 8, {}),
    ("euler_p3_16k", 5, 6, {"p": 4}),
    ("ns_mixp_65k", 7, 5, {"model": 0}),
    ("euler_p3_262k_shock", 8, 12, {}),
])
def test_float2_parity(ctx, name, nx, ny, kw):
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    errs = full_parity(ctx, wl, precision=1, tol=TOL_MIXED)
    # float-float carries ~48 bits: it lands far inside the mixed bar
    assert max(errs.values()) < 1e-11


def test_float2_pseudo_time(ctx):
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 5, 6, p=3)
    full_parity(ctx, wl, cfl=10.0, precision=1, tol=TOL_MIXED)


def test_float2_full_size_config2_sampled(ctx):
    wl = G.WORKLOADS["euler_p3_16k"]
    case, om, U, Lam, dLam = build_case(wl)
    mesh, sysm, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam, precision=1)
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(6)
    faces = rng.choice(om.n_face, 16, replace=False)
    elems = sorted(set(int(k) for f in faces for k in om.face_el[f]) | set(int(k) for k in rng.choice(om.n_elem, 16)))
    errs = ParityChecker(om, oracle_params(wl), U, Lam, dLam, g).run(elems, faces)
    print(wl.name, "float2", {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < TOL_MIXED, (k, v)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_ns_uniform_p(ctx, p, precision):
    """Navier-Stokes mixed form (12 fields), Re 5000, Pr 0.72: q eliminated in-element."""
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 4, 3, p=p, probs=None)
    full_parity(ctx, wl, precision=precision, tol=[TOL, TOL_MIXED][precision])


@pytest.mark.parametrize("precision", [0, 1])
def test_ns_mixed_p(ctx, precision):
    """Config-3 degree mix (40/30/20/10 %, p_e = max) on a small jittered mesh."""
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 5, 4)
    full_parity(ctx, wl, precision=precision, tol=[TOL, TOL_MIXED][precision])


def test_ns_pseudo_time(ctx):
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 4, 3, p=2, probs=None)
    full_parity(ctx, wl, cfl=10.0)


def _sampled(ctx, wl, precision, n_faces, n_elems, seed, tol, sc=0.0):
    case, om, U, Lam, dLam = build_case(wl)
    mesh, sysm, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam, precision=precision, sc=sc)
    assert_layout_equal(mesh, om)
    assert np.all(g["status"] == 0)
    rng = np.random.default_rng(seed)
    faces = rng.choice(om.n_face, n_faces, replace=False)
    elems = sorted(set(int(k) for f in faces for k in om.face_el[f]) |
                   set(int(k) for k in rng.choice(om.n_elem, n_elems)))
    chk = ParityChecker(om, oracle_params(wl, 0.0, sc), U, Lam, dLam, g)
    errs = chk.run(elems, faces)
    # error per field of the stored local solves (rows grouped by field)
    nf = case.nfield
    per_field = np.zeros(nf)
    for K in elems:
        e = chk.element(K)
        nt = e["D"].shape[0]
        Xg = chk.gpu_X(K)
        nb = Xg.shape[0] // nf
        for f in range(nf):
            rows = slice(f * nb, (f + 1) * nb)
            per_field[f] = max(per_field[f], rel_err(Xg[rows, :nt], e["X"][rows, :nt]))
    print(wl.name, ["fp64", "float2"][precision], {k: f"{v:.1e}" for k, v in errs.items()},
          "X_B per field", " ".join(f"{v:.1e}" for v in per_field))
    for k, v in errs.items():
        assert v < tol, (k, v)
    assert per_field.max() < tol


@pytest.mark.parametrize("precision", [0, 1])
def test_config3_ns_mixp_full_size_sampled(ctx, precision):
    """65,536-triangle Navier-Stokes workload with the 40/30/20/10 % degree mix."""
    _sampled(ctx, G.WORKLOADS["ns_mixp_65k"], precision, 8, 8, 7, [TOL, TOL_MIXED][precision])


@pytest.mark.parametrize("precision", [0, 1])
def test_ns_mixed_trace_size_launch_groups(ctx, precision):
    """A degree bucket whose trace sizes differ (a face takes the larger degree
    of its two sides) is launched in groups of trace sizes with equal resident
    CTAs per SM, each sized by its largest trace: on the Navier-Stokes degree
    mix (1,024 triangles) the p = 1 bucket, trace sizes 24 .. 60, splits.  One
    element of every (degree, trace size) class and every face of those
    elements checked against the oracle."""
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 16, 32)
    case, om, U, Lam, dLam = build_case(wl)
    mesh, sysm, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam, precision=precision)
    assert_layout_equal(mesh, om)
    assert np.all(g["status"] == 0)
    n_buckets = len(set(int(p) for p in case.elem_p))
    # condensation launches (at least one bucket in two groups) + one reconstruction per bucket
    assert sysm.launches > 2 * n_buckets
    nt = np.zeros(om.n_elem, np.int64)
    for K in range(om.n_elem):
        for f in om.elem_face[K]:
            if f >= 0:
                nt[K] += 4 * (int(om.face_p[f]) + 1)
    first = {}
    for K in range(om.n_elem):
        first.setdefault((int(case.elem_p[K]), int(nt[K])), K)
    classes_p1 = sorted(t for (p, t) in first if p == 1)
    assert classes_p1[0] <= 44 and classes_p1[-1] >= 48  # both sides of the p = 1 occupancy step
    elems = sorted(first.values())
    faces = sorted(set(int(f) for K in elems for f in om.elem_face[K] if f >= 0))
    chk = ParityChecker(om, oracle_params(wl, 0.0, 0.0), U, Lam, dLam, g)
    errs = chk.run(elems, faces)
    tol = [TOL, TOL_MIXED][precision]
    for k, v in errs.items():
        assert v < tol, (k, v)


@pytest.mark.parametrize("precision", [1, 0])
def test_config4_shock_full_size_sampled(ctx, precision):
    """262,144-triangle Euler p = 3 workload, Mach 1.5 with an oblique shock band:
    the float-float path against the FP64 oracle, error per field."""
    _sampled(ctx, G.WORKLOADS["euler_p3_262k_shock"], precision, 12, 12, 8, [TOL, TOL_MIXED][precision])


# shock capturing (Sec. 3.2): eps_0 = 0.2, beta = 0 (the paper's values), eps_K frozen in the Jacobian
SC_EPS0 = 0.2


@pytest.mark.parametrize("precision", [0, 1])
def test_config4_shock_capturing_full_size_sampled(ctx, precision):
    """The 262,144-triangle Mach 1.5 shock-band workload with shock capturing on."""
    _sampled(ctx, G.WORKLOADS["euler_p3_262k_shock"], precision, 8, 8, 9, [TOL, TOL_MIXED][precision], sc=SC_EPS0)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,nx,ny,kw", [
    ("euler_p3_262k_shock", 8, 12, {}),                   # Euler p = 3, shock band
    ("euler_p3_262k_shock", 6, 7, {"p": 4}),               # Euler p = 4
    ("ns_mixp_65k", 5, 6, {"model": 0}),                   # Euler, ragged p mix
    ("ns_mixp_65k", 4, 5, {}),                             # Navier-Stokes, p mix (q in place of grad w)
    ("ns_mixp_65k", 3, 4, {"p": 4}),                       # Navier-Stokes p = 4
])
def test_shock_capturing_parity(ctx, precision, name, nx, ny, kw):
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    full_parity(ctx, wl, precision=precision, tol=[TOL, TOL_MIXED][precision], sc=SC_EPS0)
    # the term is not negligible here: switching it off moves the local solves far beyond the bar
    case, om, U, Lam, dLam = build_case(wl)
    x_on, *_ = om.element_condense(oracle_params(wl, 0.0, SC_EPS0), 0, U, Lam)
    x_off, *_ = om.element_condense(oracle_params(wl), 0, U, Lam)
    assert rel_err(x_on, x_off) > 1e-6


def test_shock_capturing_with_pseudo_time(ctx):
    wl = G.small_variant(G.WORKLOADS["euler_p3_262k_shock"], 5, 6)
    full_parity(ctx, wl, cfl=10.0, sc=SC_EPS0)


def test_nonfinite_state_flags_its_element_only(ctx):
    """Failure detection: a non-finite coefficient in one element's state sets that
    element's status to 2 (non-finite) and leaves every other element at 0."""
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 6, 6)
    case, om, U, Lam, dLam = build_case(wl)
    K = 17
    U[om.u_off[K] + 3] = np.nan
    for precision in (0, 1):
        _, _, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam, precision=precision)
        bad = np.nonzero(g["status"])[0]
        assert list(bad) == [K] and g["status"][K] == 2


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
    rng = np.random.default_rng(5)
    faces = rng.choice(om.n_face, 16, replace=False)
    elems = sorted(set(int(k) for f in faces for k in om.face_el[f]) | set(int(k) for k in rng.choice(om.n_elem, 16)))
    errs = ParityChecker(om, oracle_params(wl), U, Lam, dLam, g).run(elems, faces)
    print(wl.name, {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < TOL, (k, v)


def test_step_host_matches_device_path(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 6, 6)
    case, om, U, Lam, dLam = build_case(wl)
    _, _, (g,) = run_gpu(ctx, case, wl, U, Lam, dLam)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
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


@pytest.mark.parametrize("name,kw", [("ns_mixp_65k", {"model": 0}), ("ns_mixp_65k", {}), ("euler_p3_16k", {})])
def test_graph_replay_and_concurrent_buckets_match_plain_path(ctx, name, kw):
    """The captured step (degree buckets on their own streams, joined) replays to the
    same bits as the plain enqueue, and keeps doing so on repeated replays."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], 7, 6, **kw)
    case, om, U, Lam, dLam = build_case(wl)
    _, _, (ref,) = run_gpu(ctx, case, wl, U, Lam, dLam)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl))
    dev = torch.device("cuda:0")
    Ut, Lt, dLt = (torch.from_numpy(a).to(dev) for a in (U, Lam, dLam))
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    sysm.graph_create(Ut, Lt, dLt, dUt)
    for _ in range(3):
        dUt.fill_(float("nan"))
        sysm.graph_launch()
        torch.cuda.synchronize()
        v = sysm.views()
        assert np.array_equal(v["K"].cpu().numpy(), ref["K"])
        assert np.array_equal(v["E"].cpu().numpy(), ref["E"])
        assert np.array_equal(v["X"].cpu().numpy(), ref["X"])
        assert np.array_equal(dUt.cpu().numpy(), ref["dU"])


@pytest.mark.parametrize("name,kw", [("ns_mixp_65k", {}), ("ns_mixp_65k", {"model": 0}), ("euler_p3_16k", {})])
@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_launch_shapes_keep_results_bitwise(ctx, name, kw, precision):
    """The autotuner only changes the grid of each degree bucket's launch; every output stays bitwise
    the same, and the chosen shapes are in range."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], 12, 14, **kw)
    case, om, U, Lam, dLam = build_case(wl)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl, 0.0, precision))
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    sysm.condense(Ut, Lt)
    torch.cuda.synchronize()
    before = {k: t.cpu().numpy().copy() for k, t in sysm.views().items()}
    shapes = sysm.autotune(Ut, Lt)
    assert set(shapes) == set(int(p) for p in np.unique(case.elem_p))
    assert all(0 <= v <= 32 for v in shapes.values())
    for _ in range(2):
        sysm.condense(Ut, Lt)
        torch.cuda.synchronize()
        after = {k: t.cpu().numpy() for k, t in sysm.views().items()}
        for k in before:
            assert np.array_equal(before[k], after[k]), k
    print(wl.name, ["fp64", "float2"][precision], "shapes", shapes)
    sysm.close()
    mesh.close()


def test_bucket_times_of_a_mixed_degree_launch(ctx):
    """Per-degree device times of a condensation whose degree buckets run concurrently: one positive
    time per present degree, none for a single-degree mesh."""
    from paper_1308_3995_gb300 import hdg
    dev = torch.device("cuda:0")
    for name, kw, want in (("ns_mixp_65k", {}, None), ("euler_p3_16k", {}, set())):
        wl = G.small_variant(G.WORKLOADS[name], 12, 14, **kw)
        case, om, U, Lam, dLam = build_case(wl)
        mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
        sysm = hdg.System(ctx, mesh, lib_params(wl, 0.0, 0))
        sysm.condense(torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev))
        t = sysm.bucket_times()
        present = set(int(p) for p in np.unique(case.elem_p))
        expect = present if want is None else want
        assert set(t) == expect and all(v > 0.0 for v in t.values()), (name, t)
        print(name, t)
        sysm.close()
        mesh.close()


def test_degenerate_stabilisation_is_refused(ctx):
    """alpha = 0 (no pseudo time) makes every local block singular -- the constant mode's rows of
    A_K vanish, pinned on the oracle -- so the library refuses it at system creation (HDG_EINVAL)
    instead of returning a field of zero-pivot statuses; a small positive alpha is accepted."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 4, 5)
    case, om, U, Lam, dLam = build_case(wl)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    prm = lib_params(wl, 0.0, 0)
    prm.alpha = 0.0
    with pytest.raises(hdg.HdgError) as ei:
        hdg.System(ctx, mesh, prm)
    assert ei.value.status == hdg.HDG_EINVAL
    prm.alpha = 1e-3
    sysm = hdg.System(ctx, mesh, prm)
    sysm.close(); mesh.close()
