"""hdg_condense_noalloc: the allocation-free condensation entry point, for
callers that cannot allocate device memory when they call (latency-bound
serving loops, hosts whose device memory belongs to another allocator).

It must give the same outputs as hdg_condense on the same inputs, on two calls
in a row (the second call runs on the work array the first one left behind),
across calls on meshes of different sizes and degrees (the array keeps the
previous mesh's layout), on a bounded mesh (far-field and slip-wall faces,
unused K slots), and reject meshes whose work space exceeds its fixed 64 MiB array.  This file is
collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

from hdg_testlib import lib_params
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _rel(a, b):
    a = a.double().cpu().numpy(); b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class _Case:
    """A mesh, its inputs on cuda:0 and the outputs of the allocating entry point."""

    def __init__(self, ctx, wl):
        from paper_1308_3995_gb300 import hdg
        case = G.make_case(wl)
        self.mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield,
                             case.mesh.elem_bc)
        U, Lam, _ = G.case_state(case, self.mesh.face_vid, self.mesh.face_p)
        self.prm = lib_params(wl)
        dev = torch.device("cuda:0")
        self.U, self.Lam = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
        sysm = hdg.System(ctx, self.mesh, self.prm)
        sysm.condense(self.U, self.Lam)
        torch.cuda.synchronize()
        self.ref = {k: v.clone() for k, v in sysm.views().items()}
        m = self.mesh
        f64 = dict(dtype=torch.float64, device=dev)
        self.out = {"X": torch.empty(m.x_len, **f64), "K": torch.empty(m.k_len, **f64),
                    "E": torch.empty(m.lam_len, **f64), "res_u": torch.empty(m.u_len, **f64),
                    "res_lam": torch.empty(m.lam_len, **f64),
                    "status": torch.empty(m.n_elem, dtype=torch.int32, device=dev)}

    def call_and_check(self, label):
        from paper_1308_3995_gb300 import hdg
        out = self.out
        for k, t in out.items():  # poison the outputs so a skipped write would show
            t.fill_(-7 if k == "status" else float("nan"))
        hdg.hdg_condense_noalloc(self.mesh, self.prm, self.U, self.Lam, out["X"], out["K"], out["E"],
                                 out["res_u"], out["res_lam"], out["status"])
        torch.cuda.synchronize()
        assert torch.equal(out["status"], self.ref["status"]), f"{label}: status differs"
        for k in ("X", "K", "E", "res_u", "res_lam"):
            assert not torch.isnan(out[k]).any(), f"{label}: {k} not fully written"
            err = _rel(out[k], self.ref[k])
            assert err <= TOL, f"{label}: {k} differs from hdg_condense by {err:.2e}"


def _two_calls(wl):
    from paper_1308_3995_gb300 import hdg
    c = _Case(hdg.Context(0), wl)
    for call in range(2):
        c.call_and_check(f"call {call}")


def test_noalloc_matches_condense_mixed_degrees():
    _two_calls(G.small_variant(G.WORKLOADS["ns_mixp_65k"], 9, 7, model=0))


def test_noalloc_matches_condense_full_size():
    """The 16,384-element Euler p = 3 workload fits the fixed work array."""
    _two_calls(G.WORKLOADS["euler_p3_16k"])


@pytest.mark.parametrize("name", ["euler_channel_8k", "euler_box_8k"])
def test_noalloc_matches_condense_bounded_mesh(name):
    """Slip wall and far field (channel), far field on all sides (box): boundary faces carry no trace
    unknowns, the far-field state enters the element kernel, K rows next to the boundary have empty slots."""
    _two_calls(G.small_variant(G.WORKLOADS[name], 12, 10))


def test_noalloc_large_then_small_then_large():
    """The array keeps the last call's contents, laid out for the last mesh: a call on a smaller mesh
    with other degrees, and a call on the first mesh after it, must each still match hdg_condense."""
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    a = _Case(ctx, G.WORKLOADS["euler_p3_16k"])
    b = _Case(ctx, G.small_variant(G.WORKLOADS["ns_mixp_65k"], 11, 9, model=0))
    a.call_and_check("mesh A, first")
    b.call_and_check("mesh B (smaller, mixed degrees)")
    a.call_and_check("mesh A, again")


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
