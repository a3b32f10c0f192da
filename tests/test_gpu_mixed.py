"""Tensor-core local solves with iterative refinement (precisions HDG_MIXED_TF32
and HDG_MIXED_BF16, the mixed-precision local solves of Sec. 3.4): residual and
Jacobian assembled in binary64, LU and solves in binary32 with mma.sync
tensor-core updates, X refined against binary64 residuals.  Parity with the
FP64 oracle element by element at the mixed-precision bar 1e-10 after
refinement (the same checker as the FP64 path); an element that cannot meet
refine_tol within refine_max corrections is flagged (status 3)."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import ParityChecker, oracle_params
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-10


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_3995_gb300 import hdg
    return hdg.Context(0)


def _run(ctx, wl, precision, refine_max, refine_tol=1e-13, cfl=0.0):
    from paper_1308_3995_gb300 import hdg
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, dLam = G.case_state(case, om.face_vid, om.face_p)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    prm = hdg.Params(model=wl.model, precision=precision, mach=wl.mach, alpha=wl.alpha, cfl=cfl, aoa=wl.aoa,
                     refine_max=refine_max, refine_tol=refine_tol)
    sysm = hdg.System(ctx, mesh, prm)
    dev = torch.device("cuda:0")
    Ut, Lt, dLt = (torch.from_numpy(a).to(dev) for a in (U, Lam, dLam))
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    sysm.condense(Ut, Lt)
    sysm.recover(dLt, dUt)
    torch.cuda.synchronize()
    g = {k: t.cpu().numpy().copy() for k, t in sysm.views().items()}
    g["dU"] = dUt.cpu().numpy()
    return om, U, Lam, dLam, g


CASES = [("euler_p1_256", 8, 16, {}), ("euler_p3_16k", 6, 8, {}), ("euler_p3_16k", 5, 6, {"p": 4}),
         ("ns_mixp_65k", 7, 5, {"model": 0}), ("euler_channel_8k", 6, 6, {}), ("euler_p3_262k_shock", 8, 8, {})]


@pytest.mark.parametrize("precision,refine_max", [(2, 4), (3, 24)])
@pytest.mark.parametrize("name,nx,ny,kw", CASES)
def test_refined_tensor_core_solves_match_oracle(ctx, precision, refine_max, name, nx, ny, kw):
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    om, U, Lam, dLam, g = _run(ctx, wl, precision, refine_max)
    assert np.all(g["status"] == 0), "every element converged"
    chk = ParityChecker(om, oracle_params(wl), U, Lam, dLam, g)
    errs = chk.run(range(om.n_elem), range(om.n_face))
    print(wl.name, ["", "", "tf32x3", "bf16"][precision], {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < TOL_MIXED, (k, v)


def test_refinement_with_pseudo_time(ctx):
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 5, 6)
    om, U, Lam, dLam, g = _run(ctx, wl, 2, 4, cfl=10.0)
    assert np.all(g["status"] == 0)
    errs = ParityChecker(om, oracle_params(wl, 10.0), U, Lam, dLam, g).run(range(om.n_elem), range(om.n_face))
    assert max(errs.values()) < TOL_MIXED, errs


def test_unconverged_refinement_is_flagged(ctx):
    """BF16 updates with a single correction cannot reach 1e-13: every element reports status 3
    (refinement not converged) while its X is still the (finite) last iterate."""
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 4, 4)
    om, U, Lam, dLam, g = _run(ctx, wl, 3, 1)
    assert np.all(g["status"] == 3)
    assert np.all(np.isfinite(g["X"]))
    # no refinement at all (refine_max = 0) is a plain binary32 tensor-core solve: no flag, 1e-3-ish accuracy
    om, U, Lam, dLam, g = _run(ctx, wl, 2, 0)
    assert np.all(g["status"] == 0)
    errs = ParityChecker(om, oracle_params(wl), U, Lam, dLam, g).run(range(om.n_elem), [])
    print(f"\nunrefined tensor-core solve (TF32x3 updates): X_B {errs['X_B']:.1e}")
    assert 1e-12 < errs["X_B"] < 1e-4


def test_mixed_precision_is_refused_where_not_built(ctx):
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 4, 4)
    case = G.make_case(wl)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    with pytest.raises(hdg.HdgError) as ei:
        hdg.System(ctx, mesh, hdg.Params(model=1, precision=hdg.HDG_MIXED_TF32, mach=0.5, alpha=1.5))
    assert ei.value.status == hdg.HDG_ENOTSUP
