"""Batched condensation across systems (hdg_batch_*): the elements of several
requests -- different meshes, degree maps, Mach numbers, bounded and periodic
domains, Euler and Navier-Stokes -- condensed with one launch per (model,
degree) group.  Every system's outputs must be those of condensing it alone
with hdg_condense / hdg_recover (the same kernel source compiled for the work
list: equal up to the compiler's contraction of multiply-adds, within the FP64
bar 1e-12 relative; statuses identical), for plain launches, autotuned shapes
and graph replays; repeated batched steps are bitwise identical."""
import numpy as np
import pytest

from hdg_testlib import lib_params
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _workloads():
    return [
        G.small_variant(G.WORKLOADS["ns_mixp_65k"], 9, 7, model=0, mach=0.7),        # Euler, p mix
        G.small_variant(G.WORKLOADS["euler_p3_16k"], 10, 12),                        # Euler p = 3
        G.small_variant(G.WORKLOADS["euler_channel_8k"], 8, 8),                      # slip wall + far field
        G.small_variant(G.WORKLOADS["ns_mixp_65k"], 6, 8),                           # NS, p mix
        G.small_variant(G.WORKLOADS["ns_wall_channel_8k"], 6, 6),                    # NS between walls
        G.small_variant(G.WORKLOADS["euler_p3_262k_shock"], 8, 8, p=4, mach=1.9),    # Euler p = 4, shock band
    ]


class _Req:
    def __init__(self, ctx, wl, precision):
        from paper_1308_3995_gb300 import hdg
        c = G.make_case(wl)
        self.mesh = hdg.Mesh(ctx, c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
        self.U, self.Lam, self.dLam = G.case_state(c, self.mesh.face_vid, self.mesh.face_p)
        self.prm = lib_params(wl, precision=precision, cfl=5.0 if wl.model == 0 else 0.0)
        self.alone = hdg.System(ctx, self.mesh, self.prm)
        self.batched = hdg.System(ctx, self.mesh, self.prm)
        Ut, Lt, dLt = (torch.from_numpy(a).to(DEV) for a in (self.U, self.Lam, self.dLam))
        dU = torch.empty(self.mesh.u_len, dtype=torch.float64, device=DEV)
        self.alone.condense(Ut, Lt)
        self.alone.recover(dLt, dU)
        torch.cuda.synchronize()
        self.ref = {k: v.clone() for k, v in self.alone.views().items()}
        self.ref["dU"] = dU
        io = self.batched.io_views()
        io["U"].copy_(Ut)
        io["Lam"].copy_(Lt)
        io["dLam"].copy_(dLt)

    def poison(self):
        for k, t in self.batched.views().items():
            t.fill_(-7 if k == "status" else float("nan"))
        self.batched.io_views()["dU"].fill_(float("nan"))

    def outputs(self):
        got = {k: v.clone() for k, v in self.batched.views().items()}
        got["dU"] = self.batched.io_views()["dU"].clone()
        return got

    def check(self, label, tol=1e-12):
        got = self.outputs()
        worst = 0.0
        for k, ref in self.ref.items():
            if k == "status":
                assert torch.equal(got[k], ref), f"{label}: element status differs"
                continue
            assert not torch.isnan(got[k]).any(), f"{label}: {k} not fully written"
            err = float((got[k] - ref).norm() / ref.norm().clamp_min(1e-300))
            worst = max(worst, err)
            assert err <= tol, f"{label}: {k} differs from the system condensed alone by {err:.2e}"
        return got, worst


def _reqs(precision):
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    return ctx, [_Req(ctx, wl, precision) for wl in _workloads()]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_alone(precision):
    from paper_1308_3995_gb300 import hdg
    ctx, reqs = _reqs(precision)
    b = hdg.Batch(ctx, [r.batched for r in reqs])
    groups = b.groups()
    assert {(m, p) for m, p, _ in groups} == {(0, 1), (0, 2), (0, 3), (0, 4), (1, 1), (1, 2), (1, 3), (1, 4)}
    assert sum(n for _, _, n in groups) == sum(r.mesh.n_elem for r in reqs)
    first, worst = {}, 0.0
    for rep in range(2):
        for r in reqs:
            r.poison()
        b.condense()
        b.recover()
        torch.cuda.synchronize()
        # one condensation and one reconstruction launch per run of trace sizes, at least one per group
        assert b.launches >= 2 * len(groups)
        for i, r in enumerate(reqs):
            got, w = r.check(f"precision {precision}, call {rep}, system {i}")
            worst = max(worst, w)
            if rep == 0:
                first[i] = got
            else:                                   # a repeated batched step is bitwise the same
                for k in got:
                    assert torch.equal(got[k], first[i][k]), f"system {i}: {k} not reproducible"
    print(f"\nbatched vs alone, precision {precision}: max relative difference {worst:.2e}")


def test_batch_autotune_and_graph_replay_match_alone():
    from paper_1308_3995_gb300 import hdg
    ctx, reqs = _reqs(0)
    b = hdg.Batch(ctx, [r.batched for r in reqs])
    shapes = b.autotune()
    assert set(shapes) == {(m, p) for m, p, _ in b.groups()}
    host = [[torch.from_numpy(a).pin_memory() for a in (r.U, r.Lam, r.dLam)] for r in reqs]
    dUh = [torch.empty(r.mesh.u_len, dtype=torch.float64).pin_memory() for r in reqs]
    b.graph_create([h[0] for h in host], [h[1] for h in host], [h[2] for h in host], dUh)
    for rep in range(2):
        for r in reqs:
            r.poison()
        for d in dUh:
            d.fill_(float("nan"))
        b.graph_launch()
        torch.cuda.synchronize()
        for i, r in enumerate(reqs):
            got, _ = r.check(f"graph replay {rep}, system {i}")
            assert torch.equal(dUh[i], got["dU"].cpu()), f"graph replay {rep}: host dU of system {i}"


def test_batch_step_host_async_matches_alone():
    from paper_1308_3995_gb300 import hdg
    ctx, reqs = _reqs(1)
    b = hdg.Batch(ctx, [r.batched for r in reqs])
    host = [[torch.from_numpy(a).pin_memory() for a in (r.U, r.Lam, r.dLam)] for r in reqs]
    dUh = [torch.full((r.mesh.u_len,), float("nan"), dtype=torch.float64).pin_memory() for r in reqs]
    for r in reqs:
        r.poison()
    b.step_host_async([h[0] for h in host], [h[1] for h in host], [h[2] for h in host], dUh)
    torch.cuda.synchronize()
    for i, r in enumerate(reqs):
        got, _ = r.check(f"step_host_async, system {i}")
        assert torch.equal(dUh[i], got["dU"].cpu())


def test_batch_rejects_mixed_precision_and_duplicates():
    """Systems of different precisions, a system given twice, and the tensor-core refinement precisions
    (built for single-system condensation only) are refused."""
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    wl = G.small_variant(G.WORKLOADS["euler_p1_256"], 4, 4)
    c = G.make_case(wl)
    mesh = hdg.Mesh(ctx, c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield)
    a = hdg.System(ctx, mesh, lib_params(wl, precision=0))
    f = hdg.System(ctx, mesh, lib_params(wl, precision=1))
    for systems in ([a, f], [a, a]):
        with pytest.raises(hdg.HdgError) as ei:
            hdg.Batch(ctx, systems)
        assert ei.value.status == hdg.HDG_EINVAL
    t = hdg.System(ctx, mesh, lib_params(wl, precision=hdg.HDG_MIXED_TF32))
    with pytest.raises(hdg.HdgError) as ei:
        hdg.Batch(ctx, [t])
    assert ei.value.status == hdg.HDG_ENOTSUP
