"""Benchmark of one HDG Newton step's element work on GB300.

A step is one pass of the whole hot path over the workload: residual and
Jacobian by quadrature, LU of every local block, local solves X, Schur
complement and condensed right-hand side, assembly of the block-sparse trace
system, and reconstruction dU = X_F - X_B dLambda (dLambda a seeded stand-in
for the global trace solve).  Default workload: 2D Euler HDG, p = 3,
16,384 jittered periodic triangles, Mach 0.8, FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  ``value``: condensed elements per second over
all ranks, device-timed with CUDA events on the launching stream, L2 flushed
between timed steps.  ``e2e``: the same metric through hdg_step_host with
pinned host buffers (copies included).  ``--impl reference`` times the CPU
FP64 oracle on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "condensed elements/sec per p; p50/p99 solve latency vs plain FP64 at 1e-10 rel"
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 FP64 rate (recipe table); see the design doc
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def dense_condensation_flops(n: int, nt: int) -> float:
    """Algorithmic FP64 flops of one element's dense condensation:
    LU 2/3 n^3, local solves 2 n^2 (nt+1), Schur 2 nt^2 n, condensed RHS 2 nt n."""
    return 2.0 / 3.0 * n ** 3 + 2.0 * n * n * (nt + 1) + 2.0 * nt * nt * n + 2.0 * nt * n


def algorithmic_bytes(n: int, nt: int) -> float:
    """FP64 HBM bytes of one element: inputs (n + nt + 6) + S (nt^2) + E (nt) + X (n (nt+1))."""
    return 8.0 * ((n + nt + 6) + nt * nt + nt + n * (nt + 1))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(wl, n_elem, extra):
    cfg = {"workload": f"{wl.name}: 2D {'Euler' if wl.model == 0 else 'Navier-Stokes mixed-form'} HDG, "
                       f"{'p=' + str(wl.p) if wl.p else 'p in 1..4 mixed'}, {n_elem} jittered periodic triangles "
                       f"({wl.nx}x{wl.ny} cells), Mach {wl.mach}",
           "elements": n_elem, "model": "euler" if wl.model == 0 else "ns_mixed", "p": wl.p,
           "l2": "flushed (256 MB write) between timed steps", "parallelism": "replicas"}
    cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------- CPU oracle timing
def time_oracle_sample(wl, target_s: float = 12.0, max_elems: int | None = None):
    """Time the oracle (as it stands) on a bounded contiguous sample of the workload."""
    import numpy as np

    import oracle as O
    from paper_1308_3995_gb300 import inputs as G
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    U, Lam, dLam = G.case_state(case, om.face_vid, om.face_p)
    P = O.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds, prandtl=wl.prandtl)
    # calibrate on 32 elements, then size the sample to about target_s seconds
    t0 = time.perf_counter()
    om.condense(P, U, Lam, 0, 32)
    per = (time.perf_counter() - t0) / 32
    n = max(32, min(om.n_elem, int(target_s / max(per, 1e-6))))
    if max_elems:
        n = min(n, max_elems)
    return om, P, U, Lam, dLam, n


def run_reference(args, wl, rank):
    if rank != 0:
        return 0
    import oracle as O  # noqa: F401
    om, P, U, Lam, dLam, n = time_oracle_sample(wl, target_s=max(1.0, 120.0 / max(1, args.steps + args.warmup)))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        om.condense(P, U, Lam, 0, n)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = n * len(times) / tot
    sample = f"elements 0..{n - 1} of {om.n_elem} per step (condensation + assembly), single thread"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "elements/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded periodic jittered mesh, Newton iterate)",
            "config": workload_config(wl, om.n_elem, {"sample_elements": n}),
            "cpu_baseline": {"value": val, "unit": "elements/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args, wl, ws, rank, local):
    import numpy as np
    import torch

    from paper_1308_3995_gb300 import hdg
    from paper_1308_3995_gb300 import inputs as G

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    case = G.make_case(wl)
    ctx = hdg.Context(local)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield)
    U, Lam, dLam = G.case_state(case, mesh.face_vid, mesh.face_p)
    prm = hdg.Params(model=wl.model, precision=args.precision, mach=wl.mach, alpha=wl.alpha,
                     reynolds=wl.reynolds, prandtl=wl.prandtl)
    sysm = hdg.System(ctx, mesh, prm)
    Ut, Lt, dLt = (torch.from_numpy(a).to(dev) for a in (U, Lam, dLam))
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        sysm.condense(Ut, Lt, stream)
        sysm.recover(dLt, dUt, stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    launches_per_step = sysm.launches
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(1.0)
        ev[i][0].record(stream)
        sysm.condense(Ut, Lt, stream)
        ev[i][1].record(stream)
        sysm.recover(dLt, dUt, stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    cond_ms = [e[0].elapsed_time(e[1]) for e in ev]
    rec_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    n_elem = mesh.n_elem
    value = ws * n_elem * args.steps / (total_ms * 1e-3)
    status_bad = int((sysm.views()["status"] != 0).sum())

    # end to end through the C ABI with pinned host buffers (copies in the timed region)
    Uh, Lh, dLh = (torch.from_numpy(a).pin_memory() for a in (U, Lam, dLam))
    dUh = torch.empty(mesh.u_len, dtype=torch.float64).pin_memory()
    for _ in range(2):
        sysm.step_host(Uh, Lh, dLh, dUh, stream)
    e2e_s = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sysm.step_host(Uh, Lh, dLh, dUh, stream)
        e2e_s.append(time.perf_counter() - t0)
    e2e_val = ws * n_elem / statistics.mean(e2e_s)
    h2d = 8 * (mesh.u_len + 2 * mesh.lam_len)
    d2h = 8 * mesh.u_len

    # roofline of the dominant kernel (condensation): algorithmic FP64 flops per launch / duration
    from collections import Counter
    nts = Counter()
    for K in range(n_elem):
        nts[(int(mesh.elem_p[K]), int(sum(4 * (mesh.face_p[e] + 1) for e in mesh.elem_face[K])))] += 1
    flops = sum(c * dense_condensation_flops(case.nfield * (p + 1) * (p + 2) // 2, nt) for (p, nt), c in nts.items())
    abytes = sum(c * algorithmic_bytes(case.nfield * (p + 1) * (p + 2) // 2, nt) for (p, nt), c in nts.items())
    cond_s = statistics.mean(cond_ms) * 1e-3
    achieved = flops / cond_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
            "kernel": "k_condense_euler_f64 (FP64 pipe)",
            "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": abytes,
            "launch_ms": 1e3 * cond_s, "achieved_hbm_gbs": abytes / cond_s / 1e9,
            "peak_note": "nominal FP64 1.25 TFLOP/s (recipe); no measured FP64 peak file"}
    lat = sorted(step_ms)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]
    extra = {"precision": "fp64" if args.precision == 0 else "mixed", "p50_step_ms": p50, "p99_step_ms": p99,
             "condense_ms": statistics.mean(cond_ms), "recover_ms": statistics.mean(rec_ms),
             "elem_status_nonzero": status_bad}
    line = {"metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded periodic jittered mesh, Newton iterate)",
            "config": workload_config(wl, n_elem, extra),
            "e2e": {"value": e2e_val, "unit": "elements/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps, "roofline": roof, "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        om, P, U2, L2, _, n = time_oracle_sample(wl, target_s=12.0)
        t0 = time.perf_counter()
        om.condense(P, U2, L2, 0, n)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
                                "sample": f"elements 0..{n - 1} of {om.n_elem} (condensation + assembly), "
                                          f"single thread, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="euler_p3_16k")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", default=None, help="override the grid, e.g. 48x96 (profiling runs)")
    args = ap.parse_args(argv)
    from paper_1308_3995_gb300 import inputs as G
    wl = G.WORKLOADS[args.workload]
    if args.cells:
        nx, ny = (int(v) for v in args.cells.lower().split("x"))
        wl = G.small_variant(wl, nx, ny)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, wl, rank)
    return run_ours(args, wl, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
