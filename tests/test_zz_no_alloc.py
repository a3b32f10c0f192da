"""hdg_condense_noalloc: the allocation-free condensation entry point, for
callers that cannot allocate device memory when they call (latency-bound
serving loops, hosts whose device memory belongs to another allocator).

It must give the same outputs as hdg_condense on the same inputs, on two calls
in a row (the second call runs on the work array the first one left behind),
and reject meshes whose work space exceeds its fixed 64 MiB array.  This file is
collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _rel(a, b):
    a = a.double().cpu().numpy(); b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _compare_two_calls(wl):
    from paper_1308_3995_gb300 import hdg
    case = G.make_case(wl)
    ctx = hdg.Context(0)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, _ = G.case_state(case, mesh.face_vid, mesh.face_p)
    prm = hdg.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha)
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    # reference: the allocating entry point
    sysm = hdg.System(ctx, mesh, prm)
    sysm.condense(Ut, Lt)
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in sysm.views().items()}
    f64 = dict(dtype=torch.float64, device=dev)
    out = {"X": torch.empty(mesh.x_len, **f64), "K": torch.empty(mesh.k_len, **f64),
           "E": torch.empty(mesh.lam_len, **f64), "res_u": torch.empty(mesh.u_len, **f64),
           "res_lam": torch.empty(mesh.lam_len, **f64),
           "status": torch.empty(mesh.n_elem, dtype=torch.int32, device=dev)}
    for call in range(2):
        for k, t in out.items():  # poison the outputs so a skipped write would show
            t.fill_(-7 if k == "status" else float("nan"))
        hdg.hdg_condense_noalloc(mesh, prm, Ut, Lt, out["X"], out["K"], out["E"], out["res_u"], out["res_lam"],
                                 out["status"])
        torch.cuda.synchronize()
        assert torch.equal(out["status"], ref["status"]), f"call {call}: status differs"
        for k in ("X", "K", "E", "res_u", "res_lam"):
            assert not torch.isnan(out[k]).any(), f"call {call}: {k} not fully written"
            err = _rel(out[k], ref[k])
            assert err <= TOL, f"call {call}: {k} differs from hdg_condense by {err:.2e}"


def test_noalloc_matches_condense_mixed_degrees():
    _compare_two_calls(G.small_variant(G.WORKLOADS["ns_mixp_65k"], 9, 7, model=0))


def test_noalloc_matches_condense_full_size():
    """The 16,384-element Euler p = 3 workload fits the fixed work array."""
    _compare_two_calls(G.WORKLOADS["euler_p3_16k"])


def test_noalloc_rejects_oversize_mesh():
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_16k"], 96, 128, p=4)  # 36,864 faces at p_e = 4: ~130 MB
    case = G.make_case(wl)
    ctx = hdg.Context(0)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    prm = hdg.Params(model=0, mach=wl.mach, alpha=wl.alpha)
    dev = torch.device("cuda:0")
    one = torch.zeros(1, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(hdg.HdgError) as ei:
        hdg.hdg_condense_noalloc(mesh, prm, one, one, one, one, one, one, one, st)
    assert ei.value.status == hdg.HDG_EINVAL
    assert "64 MiB" in str(ei.value)
