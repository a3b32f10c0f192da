"""Continuous-batching request loop for steady-flow Newton steps.

Requests (each a mesh, a degree map, a flow model, a state and a trace update)
arrive on a Poisson schedule.  The server admits them in arrival order while a
stream slot is free and its device arena can hold the request's footprint
(``hdg_sys_workspace_bytes``: the local solves X, the trace system K and E,
residuals and staging); an admitted request's whole step -- host->device
copies, condensation, reconstruction, device->host copy of dU -- is enqueued
on its own stream with ``hdg_step_host_async``, so requests that arrive while
others are on the GPU overlap with them.  A completion is observed through a
CUDA event; the request then releases its slot and its arena range at once.
Systems and solvers are carved from one arena tensor allocated at start-up;
while requests are in flight the only device allocations are the small mesh
plans made at admission (``hdg_mesh_create``: topology, offsets, degree
buckets), and nothing is freed until the run ends, so no call made here
synchronises the device.

With ``solve=True`` a request is a whole pseudo-transient Newton step of
Sec. 3.3 instead: condensation at a finite CFL, the GPU trace solve of
K dLambda = E to a relative residual of 1e-10 (GMRES, block ILU(0) by
default), reconstruction, and dU, dLambda copied back
(``hdg_solve_step_host``).  The trace solve reads its residual estimate back every few GMRES
iterations, so the call blocks its host thread: each stream slot then has
a worker thread that runs its requests' steps (the library releases the
interpreter lock during the call); the system and the solver both live in
the request's arena range.

With ``batched=True`` (step mode) admitted requests are not launched one by
one: the requests admitted since the last launch form one batch
(``hdg_batch_create_in``, its work list carved from the arena and uploaded on
the batch's stream) whose condensation is one kernel launch per (model,
degree) group over all of their elements, followed by one reconstruction
launch per group (``hdg_batch_step_host_async``, with every request's copies
on the same stream).  Up to ``max_inflight`` batches run at once, each on its
own stream; a batch completes all of its requests together.

The plain baseline is the same loop with one slot and binary64 arithmetic
(requests served one at a time, in arrival order; its trace solves in binary64
too, ``solver_arith=0``).

Latency is measured on the host clock from a request's arrival time to the
moment its completion event is observed; throughput is elements / makespan.
"""
from __future__ import annotations

import bisect
import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hdg
from . import inputs as G


# ----------------------------------------------------------------------------- arena
class Arena:
    """First-fit allocator of 256-byte-aligned ranges in [0, capacity)."""

    ALIGN = 256

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free_list = [(0, self.capacity)]      # sorted (offset, size)
        self.used = {}                             # offset -> size

    @classmethod
    def _round(cls, n: int) -> int:
        return (int(n) + cls.ALIGN - 1) // cls.ALIGN * cls.ALIGN

    def alloc(self, nbytes: int):
        n = self._round(max(1, nbytes))
        for i, (off, size) in enumerate(self.free_list):
            if size >= n:
                if size == n:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + n, size - n)
                self.used[off] = n
                return off
        return None

    def free(self, off: int):
        n = self.used.pop(off)
        i = bisect.bisect_left(self.free_list, (off, 0))
        self.free_list.insert(i, (off, n))
        # coalesce with neighbours
        merged = []
        for o, s in self.free_list:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self.free_list = merged

    @property
    def bytes_used(self) -> int:
        return sum(self.used.values())


# ----------------------------------------------------------------------------- requests
@dataclass
class Request:
    rid: int
    arrival_s: float
    wl: G.Workload
    n_elem: int = 0
    # host data (built before the run; pinned torch tensors when prepared)
    case: object = None
    U: object = None
    Lam: object = None
    dLam: object = None
    face_vid: object = None
    face_p: object = None
    # results
    dU: object = None
    dU_host: object = None
    dLam_host: object = None   # trace update computed by the solve (solve mode)
    iters: int = 0             # GMRES iterations of the solve (solve mode)
    mesh: object = None
    admitted_s: float = math.nan
    done_s: float = math.nan


def request_workloads(n: int, seed: int, min_elems: int = 1000, max_elems: int = 64000) -> list:
    """Seeded request mix: sizes log-uniform in [min_elems, max_elems]
    (nx = round(sqrt(N/4)), ny = 2 nx), Euler or Navier-Stokes 50/50, a uniform
    degree p ~ U{1..4} or the 40/30/20/10 % mix (50/50), Mach ~ U(0.3, 2.0)
    with an oblique normal-shock band above Mach 1.1, Fourier modes below."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = math.exp(rng.uniform(math.log(min_elems), math.log(max_elems)))
        nx = max(3, int(round(math.sqrt(N / 4.0))))
        model = int(rng.integers(2))
        if rng.uniform() < 0.5:
            p, probs = int(rng.integers(1, 5)), None
        else:
            p, probs = None, (0.4, 0.3, 0.2, 0.1)
        mach = float(rng.uniform(0.3, 2.0))
        fld = "shock" if mach > 1.1 else "fourier"
        out.append(G.Workload(f"req{i}", nx, 2 * nx, 0.2, model, p, probs, fld, mach, 0.0,
                              seed=int(rng.integers(1 << 30)), extra={"kvec": (1, 0)}))
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def prepare(ctx: hdg.Context, reqs: list, pin: bool = True):
    """Build each request's host inputs (mesh, degrees, state, trace update) and
    its pinned result buffer; the face list comes from the library's mesh plan."""
    import torch
    for r in reqs:
        case = G.make_case(r.wl)
        m = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
        U, Lam, dLam = G.case_state(case, m.face_vid, m.face_p)
        r.case, r.face_vid, r.face_p = case, m.face_vid.copy(), m.face_p.copy()
        r.n_elem = case.mesh.n_elem
        m.close()
        t = (torch.from_numpy(U), torch.from_numpy(Lam), torch.from_numpy(dLam), torch.empty(U.size, dtype=torch.float64),
             torch.empty(Lam.size, dtype=torch.float64))
        if pin:
            t = tuple(x.pin_memory() for x in t)
        r.U, r.Lam, r.dLam, r.dU_host, r.dLam_host = t
    return reqs


# ----------------------------------------------------------------------------- server
@dataclass
class Report:
    mode: str
    n: int
    elements: int
    makespan_s: float
    latencies_s: list = field(default_factory=list)
    gmres_iterations: list = field(default_factory=list)

    @property
    def throughput(self) -> float:
        return self.elements / self.makespan_s

    def pct(self, q: float) -> float:
        lat = sorted(self.latencies_s)
        if not lat:
            return math.nan
        k = min(len(lat) - 1, max(0, int(math.ceil(q / 100.0 * len(lat))) - 1))
        return lat[k]

    def as_dict(self) -> dict:
        d = {"mode": self.mode, "requests": self.n, "elements": self.elements,
             "makespan_s": self.makespan_s, "elements_per_s": self.throughput,
             "p50_ms": 1e3 * self.pct(50), "p99_ms": 1e3 * self.pct(99),
             "mean_ms": 1e3 * float(np.mean(self.latencies_s)) if self.latencies_s else math.nan}
        if self.gmres_iterations:
            d["gmres_iterations_median"] = float(np.median(self.gmres_iterations))
            d["gmres_iterations_max"] = int(max(self.gmres_iterations))
        return d


class Server:
    BATCH_REGION = 1 << 16   # device bytes of one batch's work list (about 400 B per request)

    def __init__(self, ctx: hdg.Context, arena_bytes: int, slots: int, precision: int, keep_outputs: bool = False,
                 solve: bool = False, precond: int = 2, rtol: float = 1e-10, cfl: float = 10.0,
                 restart: int = 30, max_iter: int = 5000, batched: bool = False, max_inflight: int = 2,
                 batch_max_elems: int = 0, solver_arith: int | None = None):
        import torch
        if batched and solve:
            raise ValueError("batched launches serve step requests (solve=False)")
        self.batched, self.max_inflight = bool(batched), int(max_inflight)
        self.batch_max_elems = int(batch_max_elems)   # 0: a batch takes every admitted request
        # GMRES arithmetic of solve requests (hdg_solver_set_arithmetic): float-float (about twice as fast
        # per iteration, same converged solution) unless asked; its double-word copies are planned into
        # the request's arena region
        self.solver_arith = 1 if solver_arith is None else int(solver_arith)
        self.ctx, self.slots, self.precision, self.keep = ctx, int(slots), int(precision), keep_outputs
        self.solve, self.precond, self.rtol, self.cfl = bool(solve), int(precond), float(rtol), float(cfl)
        self.restart, self.max_iter = int(restart), int(max_iter)
        self.dev = torch.device(f"cuda:{ctx.device}")
        self.buf = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.dev)
        self.arena = Arena(int(arena_bytes))
        self.streams = [torch.cuda.Stream(device=self.dev)
                        for _ in range(self.max_inflight if self.batched else self.slots)]

    def _params(self, wl):
        return hdg.Params(model=wl.model, precision=self.precision, mach=wl.mach, alpha=wl.alpha,
                          reynolds=wl.reynolds, prandtl=wl.prandtl, cfl=self.cfl if self.solve else 0.0)

    def _worker(self, slot: int, jobs: "queue.Queue", done: "queue.Queue", t0_box: list):
        """Runs the Newton steps of the requests given to one stream slot (solve mode)."""
        import torch
        torch.cuda.set_device(self.dev)
        st = self.streams[slot]
        while True:
            job = jobs.get()
            if job is None:
                return
            r, off, n_sys, n_sol, prm = job
            try:
                base = self.buf.data_ptr() + off
                sysm = hdg.System(self.ctx, r.mesh, prm, workspace=(base, n_sys))
                sol = hdg.Solver(sysm, self.restart, self.precond, workspace=(base + n_sys, n_sol),
                                 arith=self.solver_arith)
                r.iters, _ = sol.step_host(r.U, r.Lam, r.dU_host, r.dLam_host, self.rtol, self.max_iter, st)
                r.done_s = time.perf_counter() - t0_box[0]
                if self.keep:
                    r.dU = r.dU_host.numpy().copy()
                sol.close()          # arena-backed: frees no device memory
                sysm.close()
                done.put((r, slot, off, None))
            except Exception as exc:  # noqa: BLE001 - handed to the main loop
                done.put((r, slot, off, exc))

    def run(self, reqs: list, mode: str = "") -> Report:
        import torch
        order = sorted(reqs, key=lambda r: r.arrival_s)
        free_slots = list(range(self.slots))
        waiting, active, meshes = [], [], []
        pending, inflight = [], []          # batched mode: admitted, not launched / launched batches
        # batched mode: one arena region per stream for the work list of the batch launched on it
        bregions = [self.arena.alloc(self.BATCH_REGION) for _ in range(self.max_inflight)] if self.batched else []
        nxt = 0
        done_q, workers, jobs = queue.Queue(), [], []
        t0_box = [0.0]
        if self.solve:
            for k in range(self.slots):
                jobs.append(queue.Queue())
                th = threading.Thread(target=self._worker, args=(k, jobs[k], done_q, t0_box), daemon=True)
                th.start()
                workers.append(th)
        n_active = 0
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        t0_box[0] = t0
        try:
            while nxt < len(order) or waiting or n_active:
                now = time.perf_counter() - t0
                while nxt < len(order) and order[nxt].arrival_s <= now:
                    waiting.append(order[nxt])
                    nxt += 1
                # admit in arrival order while a slot and arena room are available; the head
                # request's mesh is planned once and kept until it is admitted
                while waiting and free_slots:
                    r = waiting[0]
                    wl = r.wl
                    if r.mesh is None:
                        r.mesh = hdg.Mesh(self.ctx, r.case.mesh.elem_xy, r.case.mesh.elem_vid, r.case.elem_p,
                                          r.case.nfield)
                        meshes.append(r.mesh)
                    mesh = r.mesh
                    prm = self._params(wl)
                    n_sys = Arena._round(mesh.workspace_bytes(prm))
                    n_sol = hdg.Solver.workspace_bytes(mesh, self.restart, self.precond, self.solver_arith) if self.solve else 0
                    need = n_sys + n_sol
                    if need > self.arena.capacity:
                        raise hdg.HdgError(hdg.HDG_ENOMEM, f"request {r.rid} needs {need} bytes, arena holds "
                                                           f"{self.arena.capacity}")
                    off = self.arena.alloc(need)
                    if off is None:
                        break
                    waiting.pop(0)
                    slot = free_slots.pop(0)
                    r.admitted_s = time.perf_counter() - t0
                    n_active += 1
                    if self.solve:
                        jobs[slot].put((r, off, n_sys, n_sol, prm))
                        continue
                    if self.batched:
                        sysm = hdg.System(self.ctx, mesh, prm, workspace=(self.buf.data_ptr() + off, n_sys))
                        pending.append((r, slot, off, sysm))
                        continue
                    sysm = hdg.System(self.ctx, mesh, prm, workspace=(self.buf.data_ptr() + off, n_sys))
                    dU = r.dU_host
                    st = self.streams[slot]
                    sysm.step_host_async(r.U, r.Lam, r.dLam, dU, st)
                    ev = torch.cuda.Event()
                    ev.record(st)
                    active.append((r, slot, off, sysm, dU, ev))
                # batched mode: the requests admitted since the last launch go out as one batch
                if self.batched and pending and len(inflight) < self.max_inflight:
                    take, tot = 0, 0                 # in admission order, up to batch_max_elems elements
                    while take < len(pending) and (take == 0 or not self.batch_max_elems or
                                                   tot + pending[take][0].n_elem <= self.batch_max_elems):
                        tot += pending[take][0].n_elem
                        take += 1
                    batch_items, pending = pending[:take], pending[take:]
                    systems = [it[3] for it in batch_items]
                    nb = hdg.Batch.workspace_bytes(systems)
                    if nb > self.BATCH_REGION:
                        raise hdg.HdgError(hdg.HDG_ENOMEM, f"batch work list of {nb} bytes > {self.BATCH_REGION}")
                    k = next(i for i in range(self.max_inflight) if i not in [b[4] for b in inflight])
                    boff = bregions[k]
                    if True:
                        st = self.streams[k]
                        bt = hdg.Batch(self.ctx, systems, workspace=(self.buf.data_ptr() + boff, nb),
                                       stream=st.cuda_stream)
                        reqs_b = [it[0] for it in batch_items]
                        bt.step_host_async([q.U for q in reqs_b], [q.Lam for q in reqs_b], [q.dLam for q in reqs_b],
                                           [q.dU_host for q in reqs_b], st)
                        ev = torch.cuda.Event()
                        ev.record(st)
                        inflight.append((bt, batch_items, ev, boff, k))
                # completions
                if self.batched:
                    still = []
                    for item in inflight:
                        bt, members, ev, boff, k = item
                        if not ev.query():
                            still.append(item)
                            continue
                        tdone = time.perf_counter() - t0
                        bt.close()                         # frees no device memory (arena-backed work list)
                        for r, slot, off, sysm in members:
                            r.done_s = tdone
                            if self.keep:
                                r.dU = r.dU_host.numpy().copy()
                            sysm.close()
                            self.arena.free(off)
                            free_slots.append(slot)
                            n_active -= 1
                    inflight = still
                elif self.solve:
                    while True:
                        try:
                            r, slot, off, exc = done_q.get_nowait()
                        except queue.Empty:
                            break
                        if exc is not None:
                            raise exc
                        self.arena.free(off)
                        free_slots.append(slot)
                        n_active -= 1
                else:
                    still = []
                    for item in active:
                        r, slot, off, sysm, dU, ev = item
                        if ev.query():
                            r.done_s = time.perf_counter() - t0
                            if self.keep:
                                r.dU = dU.numpy().copy()
                            sysm.close()                 # frees nothing on the device (arena-backed)
                            self.arena.free(off)
                            free_slots.append(slot)
                            n_active -= 1
                        else:
                            still.append(item)
                    active = still
                if not n_active and not waiting and nxt < len(order):
                    wait = order[nxt].arrival_s - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                elif n_active:
                    time.sleep(2e-5)
        finally:
            for q in jobs:
                q.put(None)
            for th in workers:
                th.join(timeout=60)
        for off in bregions:
            self.arena.free(off)
        makespan = max(r.done_s for r in order) - min(r.arrival_s for r in order)
        torch.cuda.synchronize(self.dev)
        for m in meshes:
            m.close()
        for r in order:
            r.mesh = None
        rep = Report(mode, len(order), sum(r.n_elem for r in order), makespan,
                     [r.done_s - r.arrival_s for r in order],
                     [r.iters for r in order] if self.solve else [])
        return rep
