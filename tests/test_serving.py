"""Continuous-batching request loop: host-side logic on CPU, and on the GPU the
property that each request's result is the same alone and in the mix."""
import math

import numpy as np
import pytest

from paper_1308_3995_gb300 import serving as SV


# ----------------------------------------------------------------------------- CPU
def test_arena_first_fit_alignment_and_coalescing():
    a = SV.Arena(10_000)
    o1 = a.alloc(100)
    o2 = a.alloc(1000)
    o3 = a.alloc(300)
    assert (o1, o2) == (0, 256) and o3 == 256 + 1024
    assert all(o % 256 == 0 for o in (o1, o2, o3))
    assert a.alloc(10_000) is None
    a.free(o2)
    assert a.alloc(1024) == 256               # reuses the hole
    a.free(256)
    a.free(o1)
    a.free(o3)
    assert a.free_list == [(0, 10_000)] and a.bytes_used == 0


def test_arena_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(0)
    a = SV.Arena(1 << 20)
    live = {}
    for _ in range(2000):
        if live and rng.uniform() < 0.45:
            off = list(live)[int(rng.integers(len(live)))]
            a.free(off)
            live.pop(off)
        else:
            n = int(rng.integers(1, 50_000))
            off = a.alloc(n)
            if off is not None:
                live[off] = SV.Arena._round(n)
        spans = sorted(live.items())
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2
        assert sum(live.values()) + sum(s for _, s in a.free_list) == a.capacity


def test_request_mix_and_poisson_schedule():
    wls = SV.request_workloads(400, seed=3, min_elems=1000, max_elems=64000)
    n = np.array([2 * w.nx * w.ny for w in wls])
    assert n.min() >= 900 and n.max() <= 70000
    # log-uniform sizes: the median sits near the geometric mean of the bounds
    assert 5000 < np.median(n) < 12000
    models = np.array([w.model for w in wls])
    assert 0.4 < models.mean() < 0.6
    assert all((w.field == "shock") == (w.mach > 1.1) for w in wls)
    assert SV.request_workloads(5, seed=3)[2].seed == SV.request_workloads(5, seed=3)[2].seed
    t = SV.poisson_arrivals(20000, rate_per_s=50.0, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 50.0) < 0.02 / 50.0 * 10


def test_report_percentiles():
    r = SV.Report("x", 100, 1000, 2.0, [i / 1000 for i in range(1, 101)])
    assert r.pct(50) == 0.050 and r.pct(99) == 0.099 and r.pct(100) == 0.100
    assert math.isclose(r.throughput, 500.0)


# ----------------------------------------------------------------------------- GPU
def _small_stream(n, seed):
    wls = SV.request_workloads(n, seed=seed, min_elems=600, max_elems=4000)
    return [SV.Request(i, float(t), w) for i, (w, t) in enumerate(zip(wls, SV.poisson_arrivals(n, 200.0, seed)))]


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    reqs = SV.prepare(ctx, _small_stream(8, seed=11))
    mixed = SV.Server(ctx, arena_bytes=2 << 30, slots=4, precision=hdg.HDG_FLOAT2, keep_outputs=True)
    rep = mixed.run(reqs, "mixed")
    assert rep.n == 8 and len(rep.latencies_s) == 8 and rep.makespan_s > 0
    in_mix = {r.rid: r.dU.copy() for r in reqs}
    alone = SV.Server(ctx, arena_bytes=2 << 30, slots=1, precision=hdg.HDG_FLOAT2, keep_outputs=True)
    for r in reqs:
        r.arrival_s = 0.0
        alone.run([r], "alone")
        # same kernels, own buffers: bitwise the same result alone and in the mix
        assert np.array_equal(r.dU, in_mix[r.rid]), r.rid
    # and the plain binary64 path agrees with the float-float one at the mixed-precision bar
    plain = SV.Server(ctx, arena_bytes=2 << 30, slots=1, precision=hdg.HDG_FP64, keep_outputs=True)
    for r in reqs:
        plain.run([r], "plain")
        err = np.linalg.norm(r.dU - in_mix[r.rid]) / np.linalg.norm(r.dU)
        assert err < 1e-10, (r.rid, err)
    # the served float-float steps against the oracle's condensation and reconstruction
    _check_against_oracle(sorted(reqs, key=lambda q: q.n_elem)[:2], in_mix, 1e-10)


def _check_against_oracle(reqs, results, bar):
    import oracle as O
    from hdg_testlib import oracle_params
    for r in reqs:
        c = r.case
        om = O.Mesh(c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
        res = om.condense(oracle_params(r.wl), r.U.numpy(), r.Lam.numpy())
        dU = om.recover(res["X"], r.dLam.numpy())
        err = np.linalg.norm(results[r.rid] - dU) / np.linalg.norm(dU)
        assert err < bar, (r.rid, err)


@pytest.mark.gpu
def test_batched_launches_give_each_result_as_alone():
    """Requests admitted together are condensed by one launch per (model, degree) group; each
    result is the one the request gets alone (own launches, one slot) within 1e-12, and matches
    the oracle at the mixed-precision bar."""
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    reqs = SV.prepare(ctx, _small_stream(10, seed=13))
    batched = SV.Server(ctx, arena_bytes=2 << 30, slots=8, precision=hdg.HDG_FLOAT2, keep_outputs=True,
                        batched=True, max_inflight=2)
    rep = batched.run(reqs, "batched")
    assert rep.n == 10 and batched.arena.bytes_used == 0
    in_batch = {r.rid: r.dU.copy() for r in reqs}
    alone = SV.Server(ctx, arena_bytes=2 << 30, slots=1, precision=hdg.HDG_FLOAT2, keep_outputs=True)
    for r in reqs:
        r.arrival_s = 0.0
        alone.run([r], "alone")
        err = np.linalg.norm(r.dU - in_batch[r.rid]) / np.linalg.norm(r.dU)
        assert err <= 1e-12, (r.rid, err)
    _check_against_oracle(sorted(reqs, key=lambda q: q.n_elem)[:2], in_batch, 1e-10)


@pytest.mark.gpu
def test_admission_waits_for_arena_room_and_rejects_oversize():
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    reqs = SV.prepare(ctx, _small_stream(5, seed=12))
    for r in reqs:
        r.arrival_s = 0.0
    # an arena that holds about one request at a time still serves them all, one by one
    sizes = []
    for r in reqs:
        m = hdg.Mesh(ctx, r.case.mesh.elem_xy, r.case.mesh.elem_vid, r.case.elem_p, r.case.nfield)
        sizes.append(m.workspace_bytes(hdg.Params(model=r.wl.model)))
        m.close()
    tight = SV.Server(ctx, arena_bytes=int(max(sizes) * 1.2), slots=4, precision=hdg.HDG_FLOAT2, keep_outputs=True)
    rep = tight.run(reqs, "tight")
    assert rep.n == 5 and all(r.dU is not None and np.all(np.isfinite(r.dU)) for r in reqs)
    assert tight.arena.bytes_used == 0
    tiny = SV.Server(ctx, arena_bytes=int(min(sizes) // 2), slots=2, precision=hdg.HDG_FLOAT2)
    with pytest.raises(hdg.HdgError) as ei:
        tiny.run(reqs[:1], "tiny")
    assert ei.value.status == hdg.HDG_ENOMEM


@pytest.mark.gpu
def test_solve_mode_requests_match_the_oracle_newton_step():
    """Requests as whole Newton steps (float-float condensation at CFL 10, GPU trace solve with block
    ILU(0) in double-word arithmetic, here to a relative residual of 1e-12, reconstruction): each
    result is bitwise the same alone and in the mix, and the smallest ones agree with the oracle's
    dense solve of its own K, E and its reconstruction within the mixed-precision bar 1e-10."""
    import oracle as O
    from hdg_testlib import oracle_params
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    wls = SV.request_workloads(6, seed=21, min_elems=60, max_elems=400)
    reqs = SV.prepare(ctx, [SV.Request(i, 0.002 * i, w) for i, w in enumerate(wls)])
    mixed = SV.Server(ctx, arena_bytes=2 << 30, slots=3, precision=hdg.HDG_FLOAT2, keep_outputs=True, solve=True,
                      rtol=1e-12)
    rep = mixed.run(reqs, "mixed-solve")
    assert rep.n == 6 and len(rep.gmres_iterations) == 6 and min(rep.gmres_iterations) > 0
    assert mixed.arena.bytes_used == 0
    in_mix = {r.rid: (r.dU.copy(), r.dLam_host.numpy().copy()) for r in reqs}
    alone = SV.Server(ctx, arena_bytes=2 << 30, slots=1, precision=hdg.HDG_FLOAT2, keep_outputs=True, solve=True,
                      rtol=1e-12)
    for r in reqs:
        r.arrival_s = 0.0
        alone.run([r], "alone")
        assert np.array_equal(r.dU, in_mix[r.rid][0]) and np.array_equal(r.dLam_host.numpy(), in_mix[r.rid][1])
    for r in sorted(reqs, key=lambda q: q.n_elem)[:2]:
        c = r.case
        om = O.Mesh(c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
        res = om.condense(oracle_params(r.wl, cfl=10.0), r.U.numpy(), r.Lam.numpy())
        dL = O.dense_solve(om.dense_K(res["K"]), res["E"])
        dU = om.recover(res["X"], dL)
        eL = np.linalg.norm(in_mix[r.rid][1] - dL) / np.linalg.norm(dL)
        eU = np.linalg.norm(in_mix[r.rid][0] - dU) / np.linalg.norm(dU)
        print(r.wl.name, r.n_elem, "elements, iterations", r.iters, f"dLambda {eL:.1e} dU {eU:.1e}")
        assert eL < 1e-10 and eU < 1e-10
