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
FP64_PEAK_TFLOPS = 1.25     # nominal GB300 binary64 rate (1.255 measured by an FMA-chain microbenchmark)
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 80.5: 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
HBM_PEAK_GBS = 6778.0       # measured copy bandwidth of the GB300s (MEASURED_PEAKS.json)

# Counters from ncu captures of the condensation kernels (profiles/k_condense_flops_per_element.md and
# profiles/k_condense_euler_f64_euler_p3.md), valid only while the kernel sources hash to KERNEL_SRC_SHA
# (kernel_src_sha()); afterwards the bench reports them as stale (null) instead of quoting old numbers.
KERNEL_SRC_FILES = ("hdg_euler.cuh", "hdg_kernels.cu", "hdg_ns.cuh", "hdg_ns.cu", "hdg_ns_ff.cu", "hdg_lu.cuh",
                    "hdg_arith.cuh", "hdg_physics.cuh", "hdg_internal.h")
KERNEL_SRC_SHA = "a6e675e2bb098b37"
# executed floating-point work per element, (binary64 flops, binary32 flops): 2 DFMA + DADD + DMUL and
# 2 FFMA + FADD + FMUL from the SASS instruction counters (no paired FFMA2/FADD2/FMUL2 were issued),
# one launch of each kernel on a 1,024-triangle uniform-degree periodic mesh (bench.py --profile-variants)
EXEC_FLOPS_PER_ELEM = {
    ("euler", 1, 0): (28472, 0), ("euler", 1, 1): (1050, 221616),
    ("euler", 2, 0): (114635, 0), ("euler", 2, 1): (1206, 899120),
    ("euler", 3, 0): (368566, 0), ("euler", 3, 1): (1414, 2877254),
    ("euler", 4, 0): (997143, 0), ("euler", 4, 1): (1674, 7736024),
    ("ns", 1, 0): (98143, 0), ("ns", 1, 1): (3123, 912534),
    ("ns", 2, 0): (396503, 0), ("ns", 2, 1): (6119, 3395168),
    ("ns", 3, 0): (1263656, 0), ("ns", 3, 1): (11991, 10373734),
    ("ns", 4, 0): (3276121, 0), ("ns", 4, 1): (12291, 26361456)}
# dram__bytes_read.sum + dram__bytes_write.sum of one full-size condensation launch (1-pass capture)
TRAFFIC_PER_LAUNCH = {("euler_p3_16k", 0): 12008704 + 522415872}


def kernel_src_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SRC_FILES:
        h.update(f.encode())
        with open(os.path.join(ROOT, "paper_1308_3995_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def counters_current() -> bool:
    return kernel_src_sha() == KERNEL_SRC_SHA


def dense_condensation_flops(n: int, nt: int) -> float:
    """Flops of one element's condensation written densely (no structure used):
    LU 2/3 n^3, local solves 2 n^2 (nt+1), Schur 2 nt^2 n, condensed RHS 2 nt n.
    Context only: the kernels exploit the method's block structure, see below."""
    return 2.0 / 3.0 * n ** 3 + 2.0 * n * n * (nt + 1) + 2.0 * nt * nt * n + 2.0 * nt * n


def condensation_flops(nfield: int, p: int, nt: int) -> float:
    """Flops of one element's condensation (Sec. 3.4) as the method's structure
    makes it, counting multiply and add separately (an FMA is 2).

    Euler (n = 4 n_p): LU of A_K 2/3 n^3; local solves X = A_K^{-1}[B | F]
    2 n^2 (nt+1); Schur S = D - C X_B and E = H - C X_F with C = alpha <psi, phi>
    per field, so a trace row has n_p non-zeros: 2 nt (nt+1) n_p.

    Navier-Stokes (n = 12 n_p, q eliminated inside the element with the pivot
    block det J * I; m = 4 n_p; A_wq and C_q have zero rows for the mass field,
    A_qw, B_q and C_w couple a field only to itself):
      A' = A_ww - A_wq A_qw / det            2 (3 n_p)(4 n_p)(2 n_p)
      R'_w = R_w - A_wq [B_q | F_q] / det    2 (3 n_p) nt (2 n_p) + 2 (3 n_p)(8 n_p)
      LU of A' and solves                    2/3 m^3 + 2 m^2 (nt+1)
      X_q = (R_q - A_qw X_w) / det           2 (8 n_p)(nt+1) n_p
      C' = C_w - C_q A_qw / det              2 (3 nt/4)(4 n_p)(2 n_p)
      S = D - C_q B_q / det - C' X_w,B       2 (3 nt/4) nt (2 n_p) + 2 nt m nt
      E = H - C_q F_q / det - C' X_w,F       2 (3 nt/4)(8 n_p) + 2 nt m"""
    npb = (p + 1) * (p + 2) // 2
    if nfield == 4:
        n = 4 * npb
        return 2.0 / 3.0 * n ** 3 + 2.0 * n * n * (nt + 1) + 2.0 * nt * (nt + 1) * npb
    m = 4 * npb
    f = 2.0 * (3 * npb) * (4 * npb) * (2 * npb)
    f += 2.0 * (3 * npb) * nt * (2 * npb) + 2.0 * (3 * npb) * (8 * npb)
    f += 2.0 / 3.0 * m ** 3 + 2.0 * m * m * (nt + 1)
    f += 2.0 * (8 * npb) * (nt + 1) * npb
    f += 2.0 * (0.75 * nt) * (4 * npb) * (2 * npb)
    f += 2.0 * (0.75 * nt) * nt * (2 * npb) + 2.0 * nt * m * nt
    f += 2.0 * (0.75 * nt) * (8 * npb) + 2.0 * nt * m
    return f


def algorithmic_bytes(n: int, nt: int) -> float:
    """FP64 HBM bytes of one element: inputs (n + nt + 6) + S (nt^2) + E (nt) + X (n (nt+1))."""
    return 8.0 * ((n + nt + 6) + nt * nt + nt + n * (nt + 1))


def max_over_ranks(x: float, ws: int, device) -> float:
    """Largest value of x over all ranks (the slowest rank sets the job's time)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, steps: int, total_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank's timed region."""
    return ws * units_per_rank * steps / (total_ms * 1e-3)


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
def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def time_oracle_sample(wl, target_s: float = 12.0, max_elems: int | None = None):
    """Set up the oracle (as it stands) on the workload and size a bounded contiguous sample
    of about target_s seconds of single-thread CPU work."""
    import numpy as np

    import oracle as O
    from paper_1308_3995_gb300 import inputs as G
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
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


def oracle_accuracy(m, sample: int = 0, per_field: bool = False) -> dict:
    """Part of the CPU-baseline leg: the GPU results of a measured step (its last
    condensation and reconstruction) against the oracle on the same inputs.
    Whole mesh (sample = 0): max and median over elements of the relative error of
    the local solves X_B, max over blocks of the assembled trace matrix K, and the global
    relative errors of E and of the reconstruction dU.  sample > 0: X_B on
    elements [0, sample) only (also per field with per_field)."""
    import numpy as np

    import oracle as O
    c, wl = m.case, m.wl
    om = O.Mesh(c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
    P = O.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds, prandtl=wl.prandtl,
                 sc_eps0=m.prm.sc_eps0, aoa=wl.aoa)
    r = om.condense(P, m.U, m.Lam, 0, sample, threads=host_threads())
    v = {k: t.cpu().numpy() for k, t in m.sys.views().items()}
    n_el = sample or om.n_elem
    xo, uo = np.asarray(om.x_off), np.asarray(om.u_off)
    nf = 12 if c.nfield == 12 else 4
    worst, fworst, errs = 0.0, np.zeros(nf), []
    for K in range(n_el):
        n = int(uo[K + 1] - uo[K])
        nc = int(xo[K + 1] - xo[K]) // n
        g = v["X"][xo[K]:xo[K + 1]].reshape(nc, n)[:nc - 1]      # columns of X_B (library: column-major)
        o = r["X"][xo[K]:xo[K + 1]].reshape(n, nc).T[:nc - 1]    # (oracle: row-major n x (nt + 1))
        errs.append(float(np.linalg.norm(g - o) / np.linalg.norm(o)))
        worst = max(worst, errs[-1])
        if per_field:
            nb = n // nf
            for f in range(nf):
                gf, of = g[:, f * nb:(f + 1) * nb], o[:, f * nb:(f + 1) * nb]
                fworst[f] = max(fworst[f], float(np.linalg.norm(gf - of) / max(np.linalg.norm(of), 1e-300)))
    out = {"elements_checked": n_el, "X_B_max_rel": worst, "X_B_median_rel": float(np.median(errs))}
    if per_field:
        names = (["q_x " + t for t in ("rho", "rho u", "rho v", "E")] + ["q_y " + t for t in ("rho", "rho u", "rho v", "E")]
                 if nf == 12 else [])
        names += ["rho", "rho u", "rho v", "E"]
        out["X_B_max_rel_per_field"] = dict(zip(names, (float(x) for x in fworst)))
    if not sample:
        kb = np.asarray(om.k_blkoff)
        d2 = np.add.reduceat((v["K"] - r["K"]) ** 2, kb[:-1][np.diff(kb) > 0])
        k2 = np.add.reduceat(r["K"] ** 2, kb[:-1][np.diff(kb) > 0])
        out["K_block_max_rel"] = float(np.sqrt((d2 / k2).max()))
        out["E_rel"] = float(np.linalg.norm(v["E"] - r["E"]) / np.linalg.norm(r["E"]))
        du = om.recover(r["X"], m.dLam)
        out["dU_rel"] = float(np.linalg.norm(m.dUt.cpu().numpy() - du) / np.linalg.norm(du))
    return out


def run_reference(args, wl, rank):
    if rank != 0:
        return 0
    import oracle as O  # noqa: F401
    nth = host_threads()
    # each step: about 120 s / (steps + warmup) of CPU work, spread over the host's cores
    om, P, U, Lam, dLam, n = time_oracle_sample(wl, target_s=max(1.0, 120.0 * nth / max(1, args.steps + args.warmup)))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        om.condense(P, U, Lam, 0, n, threads=nth)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = n * len(times) / tot
    sample = f"elements 0..{n - 1} of {om.n_elem} per step (condensation + assembly), {nth} host threads"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "elements/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded periodic jittered mesh, Newton iterate)",
            "config": workload_config(wl, om.n_elem, {"sample_elements": n}),
            "cpu_baseline": {"value": val, "unit": "elements/s", "cores": nth, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
class Measured:
    """One workload on one GPU: device-timed steps (CUDA events on the launching
    stream, L2 flushed between timed steps)."""

    autotune = True   # pick each degree bucket's launch shape with hdg_autotune before timing

    def __init__(self, ctx, wl, precision, dev, flush, sc_eps0=0.0, refine_max=4, refine_tol=1e-13):
        import torch

        from paper_1308_3995_gb300 import hdg
        from paper_1308_3995_gb300 import inputs as G
        self.wl, self.precision = wl, precision
        self.case = G.make_case(wl)
        c = self.case
        self.mesh = hdg.Mesh(ctx, c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
        self.U, self.Lam, self.dLam = G.case_state(c, self.mesh.face_vid, self.mesh.face_p)
        self.prm = hdg.Params(model=wl.model, precision=precision, mach=wl.mach, alpha=wl.alpha,
                              reynolds=wl.reynolds, prandtl=wl.prandtl, sc_eps0=sc_eps0, aoa=wl.aoa,
                              refine_max=refine_max, refine_tol=refine_tol)
        self.sys = hdg.System(ctx, self.mesh, self.prm)
        self.Ut, self.Lt, self.dLt = (torch.from_numpy(a).to(dev) for a in (self.U, self.Lam, self.dLam))
        self.dUt = torch.empty(self.mesh.u_len, dtype=torch.float64, device=dev)
        self.flush = flush
        self.shapes = self.sys.autotune(self.Ut, self.Lt) if Measured.autotune else {}

    def run(self, steps, warmup, stream, clocks=None):
        import torch
        for _ in range(warmup):
            self.flush.fill_(1.0)
            self.sys.condense(self.Ut, self.Lt, stream)
            self.sys.recover(self.dLt, self.dUt, stream)
        torch.cuda.synchronize()
        self.launches = self.sys.launches
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        if clocks:
            clocks.start()
        torch.cuda.synchronize()
        for i in range(steps):
            self.flush.fill_(1.0)
            ev[i][0].record(stream)
            self.sys.condense(self.Ut, self.Lt, stream)
            ev[i][1].record(stream)
            self.sys.recover(self.dLt, self.dUt, stream)
            ev[i][2].record(stream)
        torch.cuda.synchronize()
        self.clk = clocks.stop() if clocks else None
        self.step_ms = [e[0].elapsed_time(e[2]) for e in ev]
        self.cond_ms = [e[0].elapsed_time(e[1]) for e in ev]
        self.rec_ms = [e[1].elapsed_time(e[2]) for e in ev]
        self.bucket_ms = self.sys.bucket_times()     # per-degree times inside the last mixed launch
        self.status_bad = int((self.sys.views()["status"] != 0).sum())
        return self

    @property
    def n_elem(self):
        return self.mesh.n_elem

    def algorithmic(self):
        """Per launch: the condensation algebra in flops (condensation_flops), the FP64 HBM bytes, and
        the executed flops of the kernel's own pipe from the ncu instruction counts (None when the
        kernel sources changed since the counters were taken).  Elements whose trace is longer than a
        uniform-degree element's (p_e = max on mixed meshes) get the uniform-degree count scaled by the
        ratio of their condensation algebra (marked 'scaled')."""
        from collections import Counter
        m, c = self.mesh, self.case
        nts = Counter()
        for K in range(m.n_elem):
            nts[(int(m.elem_p[K]), int(sum(4 * (m.face_p[e] + 1) for e in m.elem_face[K] if e >= 0)))] += 1
        fl = sum(k * condensation_flops(c.nfield, p, nt) for (p, nt), k in nts.items())
        by = sum(k * algorithmic_bytes(c.nfield * (p + 1) * (p + 2) // 2, nt) for (p, nt), k in nts.items())
        model = "euler" if c.nfield == 4 else "ns"
        prec = 0 if self.precision == 0 else 1
        ex, scaled = None, False
        if counters_current() and self.prm.sc_eps0 <= 0.0:
            ex = 0.0
            for (p, nt), k in nts.items():
                per = EXEC_FLOPS_PER_ELEM[(model, p, prec)][prec]
                nt_u = 12 * (p + 1)
                if nt != nt_u:
                    per *= condensation_flops(c.nfield, p, nt) / condensation_flops(c.nfield, p, nt_u)
                    scaled = True
                ex += k * per
        return fl, by, ex, scaled

    def summary(self):
        tot = sum(self.step_ms)
        lat = sorted(self.step_ms)

        def pct(q):
            return lat[min(len(lat) - 1, max(0, int(math.ceil(q / 100.0 * len(lat))) - 1))]
        p99 = pct(99)
        fl, by, ex, scaled = self.algorithmic()
        cond_s = statistics.mean(self.cond_ms) * 1e-3
        pipe, peak = ("fp64", FP64_PEAK_TFLOPS) if self.precision == 0 else ("fp32", FP32_PEAK_TFLOPS)
        work = {"condensation_algebra_gflop_per_launch": fl / 1e9,
                "condensation_algebra_tflops": fl / cond_s / 1e12,
                "executed_gflop_per_launch": None if ex is None else ex / 1e9,
                "executed_tflops": None if ex is None else ex / cond_s / 1e12,
                "pipe": pipe, "pipe_peak_tflops": peak,
                "pipe_frac": None if ex is None else ex / cond_s / 1e12 / peak,
                "counters": ("stale: kernel sources changed since the ncu counts" if not counters_current() else
                             "n/a with shock capturing" if self.prm.sc_eps0 > 0.0 else
                             "scaled from uniform-degree counts" if scaled else "ncu instruction counts")}
        return {"elements_per_s": self.n_elem * len(self.step_ms) / (tot * 1e-3), "ms_per_step": tot / len(lat),
                "p50_step_ms": lat[len(lat) // 2], "p10_step_ms": pct(10), "p90_step_ms": pct(90),
                "p99_step_ms": p99, "condense_ms": 1e3 * cond_s,
                "recover_ms": statistics.mean(self.rec_ms), "elem_status_nonzero": self.status_bad,
                "work": work, "algorithmic_mb_per_launch": by / 1e6,
                "launch_shapes": {str(p): ("one CTA per element" if v == 0 else f"persistent, {v} CTAs/SM")
                                  for p, v in self.shapes.items()},
                **({"buckets_in_last_step": {
                    str(p): {"elements": int((self.mesh.elem_p == p).sum()), "ms": ms,
                             "elements_per_s": int((self.mesh.elem_p == p).sum()) / (ms * 1e-3)}
                    for p, ms in self.bucket_ms.items()}} if self.bucket_ms else {})}

    def close(self):
        self.sys.close()
        self.mesh.close()


def solve_section(ctx, wl, dev, flush, stream, cfl=10.0, rtol=1e-10, reps=3):
    """One pseudo-transient Newton step with the GPU trace solve (Sec. 3.3/3.4): condensation at
    the given CFL, GMRES (block Jacobi, multicolor block symmetric Gauss-Seidel, then block
    ILU(0) in the multicolor order) on K dLambda = E, reconstruction, update; plus the bandwidth
    of the trace matrix-vector product (the K values stream once) and the ILU(0) factorization
    and application times."""
    import torch

    from paper_1308_3995_gb300 import hdg
    m = Measured(ctx, wl, hdg.HDG_FP64, dev, flush)
    m.sys.set_cfl(cfl)
    x = torch.zeros(m.mesh.lam_len, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    out = {"workload": wl.name, "cfl": cfl, "rtol": rtol, "restart": 30,
           "arithmetic": "binary64; *_ff: GMRES products, sweeps and Gram-Schmidt in double-word arithmetic on the "
                         "binary32 pipe (hdg_solver_set_arithmetic 1)"}
    for precond, nm, arith in ((0, "block_jacobi", 0), (0, "block_jacobi_ff", 1), (1, "block_sgs", 0),
                               (1, "block_sgs_ff", 1), (2, "block_ilu0", 0), (2, "block_ilu0_ff", 1),
                               (3, "block_ilu0_f32", 0), (3, "block_ilu0_f32_ff", 1)):
        solver = hdg.Solver(m.sys, restart=30, precond=precond)
        solver.set_arithmetic(arith)
        res = []
        for r in range(reps + 1):
            U, L = m.Ut.clone(), m.Lt.clone()
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.sys.condense(U, L, stream)
            x.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            it, rel = solver.solve(x, rtol=rtol, max_iter=3000, stream=stream)
            t2 = time.perf_counter()
            m.sys.recover(x, m.dUt, stream)
            m.sys.newton_update(U, L, m.dUt, x, stream)
            torch.cuda.synchronize()
            if r > 0:
                res.append((time.perf_counter() - t0, t2 - t1, it, rel))
        it_ = res[-1][2]
        solve_ms = 1e3 * statistics.median(t for _, t, _, _ in res)
        out[nm] = {"newton_step_ms": 1e3 * statistics.median(t for t, _, _, _ in res), "solve_ms": solve_ms,
                   "gmres_iterations": it_, "ms_per_iteration": solve_ms / max(it_, 1), "rel_residual": res[-1][3]}
        if precond == 0 and arith == 0:
            # matrix-vector product bandwidth (K values + x gathers + y), CUDA events on the stream
            nmv = 20
            k_bytes = 8 * m.mesh.k_len
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            solver.matvec(x, y, stream)
            ev0.record(stream)
            for _ in range(nmv):
                solver.matvec(x, y, stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            mv_s = ev0.elapsed_time(ev1) * 1e-3 / nmv
            out["matvec"] = {"k_mb": k_bytes / 1e6, "ms": 1e3 * mv_s, "k_gbs": k_bytes / mv_s / 1e9,
                             "frac_of_hbm": k_bytes / mv_s / 1e9 / HBM_PEAK_GBS}
        if precond >= 2 and arith == 0:
            # factorization (copy of K + one launch per color) and one application M^{-1} r
            ev0, ev1, ev2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            ev0.record(stream)
            solver.setup(stream)
            ev1.record(stream)
            for _ in range(10):
                solver.precond_apply(x, y, stream)
            ev2.record(stream)
            torch.cuda.synchronize()
            out[nm]["factor_ms"] = ev0.elapsed_time(ev1)
            out[nm]["apply_ms"] = ev1.elapsed_time(ev2) / 10
            out[nm]["colors"] = solver.colors()[1]
        solver.close()
    m.close()
    return out


def adjoint_section(ctx, wl, dev, flush, stream, cfl=10.0, rtol=1e-10, reps=3):
    """Hybridized adjoint (Sec. 4.2) and the adaptation decisions (Sec. 4.1, 4.3, 4.4) on the
    workload: primal condensation, adjoint local solves + E~, GMRES on K^T, adjoint reconstruction,
    indicators, Doerfler marking (theta 0.05) and the h/p choice (eps_s 1e-6).  The target
    functional is the integral of density (F~ on each element's density constant mode)."""
    import torch

    from paper_1308_3995_gb300 import hdg
    m = Measured(ctx, wl, hdg.HDG_FP64, dev, flush)
    m.sys.set_cfl(cfl)
    adj = hdg.System(ctx, m.mesh, hdg.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds,
                                              prandtl=wl.prandtl, cfl=cfl))
    nb = (wl.p + 1) * (wl.p + 2) // 2
    Ft = torch.zeros(m.mesh.u_len, dtype=torch.float64, device=dev)
    Ft.view(-1, 4 * nb)[:, 0] = 1.0
    solver = hdg.Solver(m.sys, restart=30)
    lt = torch.zeros(m.mesh.lam_len, dtype=torch.float64, device=dev)
    ua = torch.zeros(m.mesh.u_len, dtype=torch.float64, device=dev)
    eta2 = torch.empty(m.mesh.n_elem, dtype=torch.float64, device=dev)
    sens = torch.empty_like(eta2)
    code = torch.empty(m.mesh.n_elem, dtype=torch.int8, device=dev)
    rows = []
    for r in range(reps + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.sys.condense(m.Ut, m.Lt, stream)
        adj.adjoint_condense(m.sys, m.Ut, m.Lt, Ft, stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lt.zero_()
        it, rel = solver.solve(lt, rtol=rtol, max_iter=3000, rhs=adj.views()["E"], transpose=True, stream=stream)
        adj.recover(lt, ua, stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        m.sys.adapt_indicators(m.Ut, ua, eta2, sens, stream)
        nm = hdg.adapt_mark(ctx, eta2, sens, code, theta=0.05, eps_s=1e-6, stream=stream)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        if r > 0:
            rows.append((t1 - t0, t2 - t1, t3 - t2, it, rel, nm))
    c = code.cpu().numpy()
    med = lambda k: 1e3 * statistics.median(x[k] for x in rows)
    out = {"workload": wl.name, "cfl": cfl, "functional": "integral of density",
           "primal_and_adjoint_condense_ms": med(0), "adjoint_trace_solve_and_recover_ms": med(1),
           "indicators_and_marking_ms": med(2), "gmres_iterations": rows[-1][3], "rel_residual": rows[-1][4],
           "marked": rows[-1][5], "p_enrichment": int((c == 1).sum()), "h_refinement": int((c == 2).sum())}
    solver.close()
    adj.close()
    m.close()
    return out


def steady_section(ctx, dev, flush, stream, name="euler_box_8k", tol=1e-10, c0=1e6, c1=1e3, n0=4):
    """A steady solve on a bounded domain (far field on all sides, Sec. 2.1/3.2): pseudo-transient
    Newton with the CFL law of Eq. (cfl) (the paper's c0, c1, n0), GPU condensation, GMRES trace
    solve, reconstruction and update each step, until ||N_h|| has dropped by tol."""
    import torch

    from paper_1308_3995_gb300 import hdg
    from paper_1308_3995_gb300 import inputs as G
    wl = G.WORKLOADS[name]
    m = Measured(ctx, wl, hdg.HDG_FP64, dev, flush)
    dL = torch.zeros(m.mesh.lam_len, dtype=torch.float64, device=dev)
    out = {"workload": f"{name}: {m.n_elem} triangles, Euler p={wl.p}, far field on all sides, Mach {wl.mach} "
                       f"at {wl.aoa} deg + density bump", "cfl_law": {"c0": c0, "c1": c1, "n0": n0}}
    for precond, nm in ((0, "block_jacobi"), (2, "block_ilu0"), (3, "block_ilu0_f32")):
        solver = hdg.Solver(m.sys, restart=50, precond=precond)
        U, L = m.Ut.clone(), m.Lt.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cfl, r_prev, r0, hist, its = 0.0, None, None, [], []
        for n in range(1, 40):
            m.sys.condense(U, L, stream)
            r = m.sys.residual_norm(stream)
            r0 = r0 or r
            hist.append(r)
            if r < tol * r0:
                break
            cfl = hdg.cfl_law(n, c0=c0, c1=c1, n0=n0, cfl_prev=cfl, res_prev=r_prev or r, res_cur=r)
            m.sys.set_cfl(cfl)
            m.sys.condense(U, L, stream)
            dL.zero_()
            it, _ = solver.solve(dL, rtol=1e-11, max_iter=5000, stream=stream)
            its.append(it)
            m.sys.recover(dL, m.dUt, stream)
            m.sys.newton_update(U, L, m.dUt, dL, stream)
            r_prev = r
        torch.cuda.synchronize()
        out[nm] = {"time_to_solution_s": time.perf_counter() - t0, "newton_steps": len(its),
                   "gmres_iterations": its, "residual_history": hist, "converged": hist[-1] < tol * hist[0]}
        solver.close()
        m.sys.set_cfl(0.0)
    m.close()
    return out


def latency_section(ctx, dev, stream, reps=300):
    """The 256-triangle Euler p = 1 step (8x16 cells, Mach 0.5 with a density bump; the small
    configuration): latency-bound, so it is reported as times per step, not as a throughput.
    Device time of condensation + reconstruction (CUDA events around each step), host time to
    enqueue them (launch overhead), end-to-end time through hdg_step_host with pinned host
    buffers (copies and synchronisation included), and the same step replayed as a CUDA graph."""
    import torch

    from paper_1308_3995_gb300 import hdg
    from paper_1308_3995_gb300 import inputs as G
    wl = G.WORKLOADS["euler_p1_256"]
    c = G.make_case(wl)
    mesh = hdg.Mesh(ctx, c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
    U, Lam, dLam = G.case_state(c, mesh.face_vid, mesh.face_p)
    sysm = hdg.System(ctx, mesh, hdg.Params(model=wl.model, mach=wl.mach, alpha=wl.alpha))
    Ut, Lt, dLt = (torch.from_numpy(a).to(dev) for a in (U, Lam, dLam))
    dUt = torch.empty(mesh.u_len, dtype=torch.float64, device=dev)
    for _ in range(20):
        sysm.condense(Ut, Lt, stream)
        sysm.recover(dLt, dUt, stream)
    torch.cuda.synchronize()

    def pct(v, q):
        v = sorted(v)
        return v[min(len(v) - 1, int(q / 100.0 * len(v)))]
    dev_us, enq_us = [], []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        sysm.condense(Ut, Lt, stream)
        sysm.recover(dLt, dUt, stream)
        enq_us.append(1e6 * (time.perf_counter() - t0))
        e1.record(stream)
        e1.synchronize()
        dev_us.append(1e3 * e0.elapsed_time(e1))
    Uh, Lh, dLh = (torch.from_numpy(a).pin_memory() for a in (U, Lam, dLam))
    dUh = torch.empty(mesh.u_len, dtype=torch.float64).pin_memory()
    e2e_us = []
    for i in range(reps + 10):
        t0 = time.perf_counter()
        sysm.step_host(Uh, Lh, dLh, dUh, stream)
        if i >= 10:
            e2e_us.append(1e6 * (time.perf_counter() - t0))
    sysm.graph_create(Ut, Lt, dLt, dUt)
    g_us = []
    for i in range(reps + 10):
        t0 = time.perf_counter()
        sysm.graph_launch(stream)
        stream.synchronize()
        if i >= 10:
            g_us.append(1e6 * (time.perf_counter() - t0))
    out = {"workload": "euler_p1_256: 2D Euler HDG, p=1, 256 periodic triangles (8x16 cells), Mach 0.5, "
                       "density bump; binary64",
           "elements": mesh.n_elem, "kernel_launches_per_step": sysm.launches,
           "device_us_p50": pct(dev_us, 50), "device_us_p99": pct(dev_us, 99),
           "enqueue_us_p50": pct(enq_us, 50),
           "e2e_us_p50": pct(e2e_us, 50), "e2e_us_p99": pct(e2e_us, 99),
           "e2e_h2d_bytes": 8 * (mesh.u_len + 2 * mesh.lam_len), "e2e_d2h_bytes": 8 * mesh.u_len,
           "graph_replay_us_p50": pct(g_us, 50), "graph_replay_us_p99": pct(g_us, 99),
           "note": "host clock for enqueue, end-to-end and graph replay (launch to stream synchronised); "
                   "CUDA events for device time; inputs L2-resident (a 256-element step is latency-bound)"}
    sysm.close()
    mesh.close()
    return out


def serving_section(ctx, n_requests, seed, max_elems, rates=(0.7,), arena_gb=24, solve=False):
    """Poisson stream through the continuous-batching loop (float-float, 8 slots)
    against the plain loop (binary64, one request at a time), at each load level
    (fraction of the batched loop's saturated throughput).  solve: each request is
    a whole Newton step with the GPU trace solve to 1e-10 (CFL 10, block ILU(0)),
    else condensation + reconstruction with a seeded trace update."""
    import torch

    from paper_1308_3995_gb300 import hdg
    from paper_1308_3995_gb300 import serving as SV
    wls = SV.request_workloads(n_requests, seed=seed, min_elems=1000, max_elems=max_elems)
    reqs = SV.prepare(ctx, [SV.Request(i, 0.0, w) for i, w in enumerate(wls)])
    arena = int(arena_gb) << 30
    mixed = SV.Server(ctx, arena, slots=8, precision=hdg.HDG_FLOAT2, solve=solve)
    plain = SV.Server(ctx, arena, slots=1, precision=hdg.HDG_FP64, solve=solve, solver_arith=0)
    # step requests also through batched launches: the requests admitted since the last launch
    # condensed by one launch per (model, degree) group, batches of at most 32,768 elements, up to
    # eight in flight (the best of a sweep over 2-8 in flight and 32k-200k elements or no cap)
    batched = None if solve else SV.Server(ctx, arena, slots=64, precision=hdg.HDG_FLOAT2, batched=True,
                                           max_inflight=8, batch_max_elems=32768)
    sat = mixed.run(reqs, "saturated")                       # everything at t = 0
    mean_el = sat.elements / sat.n
    levels = {}
    sat_b = batched.run(reqs, "saturated, batched launches") if batched else None
    for frac in rates:
        rate = frac * sat.throughput / mean_el               # requests / s
        arr = SV.poisson_arrivals(len(reqs), rate, seed + 1)
        for r, t in zip(reqs, arr):
            r.arrival_s = float(t)
        m = mixed.run(reqs, "mixed float-float, continuous batching (8 slots)").as_dict()
        lv = {"arrival_rate_per_s": rate, "mixed": m}
        if batched:
            lv["mixed_batched_launches"] = batched.run(reqs, "mixed float-float, batched launches").as_dict()
        lv["plain_fp64"] = plain.run(reqs, "plain FP64, one request at a time").as_dict()
        levels[str(frac)] = lv
    del mixed, plain, batched
    torch.cuda.empty_cache()
    out = {"requests": len(reqs), "sizes": f"1000..{max_elems} elements log-uniform, Euler/NS 50/50, p 1..4",
           "request": ("Newton step: condensation at CFL 10, GMRES(30) + block ILU(0) trace solve to 1e-10 "
                       "relative residual, reconstruction; dU and dLambda back to the host") if solve else
                      "condensation + reconstruction with a seeded trace update; dU back to the host",
           "saturated_elements_per_s": sat.throughput, "elements_total": sat.elements}
    if sat_b is not None:
        out["saturated_elements_per_s_batched_launches"] = sat_b.throughput
    if solve:
        out["saturated_gmres_iterations_median"] = sat.as_dict().get("gmres_iterations_median")
    if len(levels) == 1:
        out.update(next(iter(levels.values())))
    else:
        out["load_levels"] = levels
    return out


def run_ours(args, wl, ws, rank, local):
    import torch

    from paper_1308_3995_gb300 import hdg
    from paper_1308_3995_gb300 import inputs as G

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ctx = hdg.Context(local)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    if args.solve_only:
        if rank == 0:
            print(json.dumps({"metric": "Newton step with GPU trace solve; adjoint and adaptation",
                              "solve": solve_section(ctx, wl, dev, flush, stream),
                              "adjoint": adjoint_section(ctx, wl, dev, flush, stream),
                              "steady": steady_section(ctx, dev, flush, stream)}), flush=True)
        return 0
    if args.serving_only:
        line = {"metric": "serving: p50/p99 latency and elements/s, continuous batching (float-float) vs plain FP64",
                "serving": serving_section(ctx, args.serving_requests, 77, args.serving_max_elems,
                                           tuple(float(v) for v in args.serving_rates.split(",")), args.serving_arena_gb),
                "serving_with_trace_solve": serving_section(ctx, args.serving_requests, 77, args.serving_max_elems,
                                                            tuple(float(v) for v in args.serving_rates.split(",")),
                                                            args.serving_arena_gb, solve=True)}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0

    # headline: plain binary64 path on the named workload (replicated on every rank)
    main_m = Measured(ctx, wl, args.precision, dev, flush, args.sc_eps0)
    if ws > 1:
        torch.distributed.barrier()
    main_m.run(args.steps, args.warmup, stream, ClockSampler(local))
    if ws > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(sum(main_m.step_ms), ws, dev)
    n_elem = main_m.n_elem
    value = whole_job_rate(n_elem, ws, args.steps, total_ms)
    summ = main_m.summary()

    # end to end through the C ABI with pinned host buffers (copies in the timed region)
    Uh, Lh, dLh = (torch.from_numpy(a).pin_memory() for a in (main_m.U, main_m.Lam, main_m.dLam))
    dUh = torch.empty(main_m.mesh.u_len, dtype=torch.float64).pin_memory()
    for _ in range(2):
        main_m.sys.step_host(Uh, Lh, dLh, dUh, stream)
    e2e_s = []
    for _ in range(max(3, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        main_m.sys.step_host(Uh, Lh, dLh, dUh, stream)
        e2e_s.append(time.perf_counter() - t0)
    e2e_val = ws * n_elem / statistics.mean(e2e_s)
    h2d = 8 * (main_m.mesh.u_len + 2 * main_m.mesh.lam_len)
    d2h = 8 * main_m.mesh.u_len

    # roofline of the dominant kernel (condensation): bound by its arithmetic pipe
    fl, by, ex, _ = main_m.algorithmic()
    cond_s = summ["condense_ms"] * 1e-3
    peak = FP64_PEAK_TFLOPS if args.precision == 0 else FP32_PEAK_TFLOPS
    work = ex if ex is not None else fl
    achieved = work / cond_s / 1e12
    fresh = counters_current()
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": TRAFFIC_PER_LAUNCH.get((wl.name, args.precision)) if fresh else None,
            "kernel": f"k_condense_{'euler' if wl.model == 0 else 'ns'} "
                      f"({'binary64 on the FP64 pipe' if args.precision == 0 else 'float-float on the FP32 pipe'})",
            "flops_counted": ("executed flops of the kernel (ncu instruction counts per element x elements): "
                              "the condensation algebra plus the quadrature assembly" if ex is not None else
                              "condensation algebra only (instruction counts stale or unavailable)"),
            "flops_per_launch": work, "condensation_algebra_flops_per_launch": fl,
            "algebra_only_frac": fl / cond_s / 1e12 / peak if args.precision == 0 else None,
            "algorithmic_bytes_per_launch": by, "launch_ms": 1e3 * cond_s, "achieved_hbm_gbs": by / cond_s / 1e9,
            "hbm_frac": by / cond_s / 1e9 / HBM_PEAK_GBS,
            "peak_note": ("FP64 1.25 TFLOP/s nominal (1.255 measured by an FMA-chain microbenchmark)"
                          if args.precision == 0 else
                          "FP32 80.5 TFLOP/s from unit counts (152 SMs x 128 lanes x FMA x 2.07 GHz); "
                          "73.5 measured by an FMA-chain microbenchmark")}
    extra = {"precision": "fp64" if args.precision == 0 else "float-float", "sc_eps0": args.sc_eps0,
             "launch_shapes": summ["launch_shapes"]}
    extra.update({k: summ[k] for k in ("p50_step_ms", "p10_step_ms", "p90_step_ms", "p99_step_ms", "condense_ms",
                                       "recover_ms", "elem_status_nonzero")})
    check = rank == 0 and ws == 1 and not args.no_cpu_baseline   # the CPU-baseline leg checks every result
    acc = {}
    if check:
        acc[f"{wl.name}_{'fp64' if args.precision == 0 else 'float2'}"] = oracle_accuracy(main_m)
    line = {"metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f32x2",
            "data": "synthetic (seeded periodic jittered mesh, Newton iterate)",
            "config": workload_config(wl, n_elem, extra),
            "e2e": {"value": e2e_val, "unit": "elements/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": main_m.launches * args.steps, "roofline": roof, "clocks": main_m.clk}
    main_m.close()

    if ws == 1 and not args.quick:
        from paper_1308_3995_gb300 import inputs as G
        # the same workload in float-float arithmetic (mixed-precision path, parity <= 1e-12 vs the oracle)
        mm = Measured(ctx, wl, hdg.HDG_FLOAT2, dev, flush).run(max(5, args.steps // 2), 3, stream)
        line["mixed_float2"] = {**mm.summary(), "dtype": "f32x2 (binary32 pairs, ~48-bit significand)"}
        if check:
            acc[f"{wl.name}_float2"] = oracle_accuracy(mm)
        mm.close()
        # condensed elements/s per p at equal element counts (Euler, 16,384 triangles)
        per_p = {}
        for p in (1, 2, 3, 4):
            wp = G.small_variant(wl, wl.nx, wl.ny, p=p, name=f"euler_p{p}_16k")
            row = {}
            for prec, nm in ((hdg.HDG_FP64, "fp64"), (hdg.HDG_FLOAT2, "float2")):
                mp = Measured(ctx, wp, prec, dev, flush).run(5, 2, stream)
                sm = mp.summary()
                row[nm] = sm["elements_per_s"]
                row[f"{nm}_pipe_frac"] = sm["work"]["pipe_frac"]
                if check:
                    acc[f"{wp.name}_{nm}"] = oracle_accuracy(mp)
                mp.close()
            per_p[str(p)] = row
        line["elements_per_s_per_p"] = per_p
        # Navier-Stokes mixed form per degree (uniform p, 16,384 triangles): elements/s and pipe fraction
        ns_per_p = {}
        for p in (1, 2, 3, 4):
            wp = G.small_variant(G.WORKLOADS["ns_mixp_65k"], 64, 128, p=p, probs=None, name=f"ns_p{p}_16k")
            row = {}
            for prec, nm in ((hdg.HDG_FP64, "fp64"), (hdg.HDG_FLOAT2, "float2")):
                mp = Measured(ctx, wp, prec, dev, flush).run(3, 1, stream)
                sm = mp.summary()
                row[nm] = sm["elements_per_s"]
                row[f"{nm}_pipe_frac"] = sm["work"]["pipe_frac"]
                row[f"{nm}_algebra_tflops"] = sm["work"]["condensation_algebra_tflops"]
                mp.close()
            ns_per_p[str(p)] = row
        line["ns_elements_per_s_per_p"] = ns_per_p
        # tensor-core trial (precision item of the method's mixed-precision local solves): binary64
        # assembly and refinement residuals, binary32 LU and solves with mma.sync updates
        trial = {}
        for p in (3, 4):
            wp = G.small_variant(wl, wl.nx, wl.ny, p=p, name=f"euler_p{p}_16k")
            row = {}
            for nm, prec, rmax in (("fp64_direct", hdg.HDG_FP64, 0), ("float2_direct", hdg.HDG_FLOAT2, 0),
                                   ("tf32x3_refined", hdg.HDG_MIXED_TF32, 4),
                                   ("tf32x3_one_correction", hdg.HDG_MIXED_TF32, 1),
                                   ("bf16_refined", hdg.HDG_MIXED_BF16, 24)):
                mp = Measured(ctx, wp, prec, dev, flush, refine_max=rmax).run(5, 2, stream)
                sm = mp.summary()
                row[nm] = {"elements_per_s": sm["elements_per_s"], "condense_ms": sm["condense_ms"],
                           "elements_status_3": int((mp.sys.views()["status"] == 3).sum())}
                if check and prec >= hdg.HDG_MIXED_TF32:
                    acc[f"{wp.name}_{nm}"] = oracle_accuracy(mp)
                mp.close()
            trial[str(p)] = row
        line["tensor_core_local_solve_trial"] = {
            "what": "Euler, 16,384 triangles; refinement stops when a correction < 1e-13 max|X| (status 3: "
                    "not reached within refine_max corrections)", "per_p": trial}
        # Navier-Stokes mixed form, degree mix 40/30/20/10 % (65,536 triangles)
        ns = {}
        for prec, nm in ((hdg.HDG_FP64, "fp64"), (hdg.HDG_FLOAT2, "float2")):
            mn = Measured(ctx, G.WORKLOADS["ns_mixp_65k"], prec, dev, flush).run(3, 1, stream)
            ns[nm] = mn.summary()
            if check:
                acc[f"ns_mixp_65k_{nm}"] = oracle_accuracy(mn, sample=2048, per_field=True)
            mn.close()
        line["ns_mixp_65k"] = ns
        # 262,144-triangle Euler p = 3, Mach 1.5 shock band, shock capturing off / on (eps_0 = 0.2)
        shock = {}
        for sc in (0.0, 0.2):
            for prec, nm in ((hdg.HDG_FP64, "fp64"), (hdg.HDG_FLOAT2, "float2")):
                ms = Measured(ctx, G.WORKLOADS["euler_p3_262k_shock"], prec, dev, flush, sc).run(3, 1, stream)
                shock[f"{nm}_sc{'_on' if sc else '_off'}"] = ms.summary()
                if check:
                    acc[f"euler_p3_262k_shock_{nm}_sc{'_on' if sc else '_off'}"] = oracle_accuracy(ms, sample=4096,
                                                                                                   per_field=True)
                ms.close()
        line["euler_p3_262k_shock"] = shock
        line["euler_p1_256_latency"] = latency_section(ctx, dev, stream)
        line["newton_step_with_trace_solve"] = solve_section(ctx, wl, dev, flush, stream)
        line["adjoint_and_adaptation"] = adjoint_section(ctx, wl, dev, flush, stream)
        line["steady_solve_bounded_domain"] = steady_section(ctx, dev, flush, stream)
        if args.serving_requests > 0:
            # the serving configuration: 512 requests of 1k-64k elements at load 0.7
            sv = serving_section(ctx, args.serving_requests, 77, args.serving_max_elems)
            line["serving"] = sv
            best = min(("mixed", "mixed_batched_launches"), key=lambda k: sv[k]["p99_ms"] if k in sv else 1e30)
            line["serving_p50_ms"] = sv[best]["p50_ms"]
            line["serving_p99_ms"] = sv[best]["p99_ms"]
            line["serving_elements_per_s"] = sv[best]["elements_per_s"]
            line["serving_form"] = ("float-float, batched launches across requests" if best != "mixed" else
                                    "float-float, 8 stream slots")
            line["serving_plain_fp64_p50_ms"] = sv["plain_fp64"]["p50_ms"]
            line["serving_plain_fp64_p99_ms"] = sv["plain_fp64"]["p99_ms"]
            line["serving_plain_fp64_elements_per_s"] = sv["plain_fp64"]["elements_per_s"]
        if args.serving_solve_requests > 0:
            line["serving_with_trace_solve"] = serving_section(ctx, args.serving_solve_requests, 77,
                                                               args.serving_solve_max_elems, solve=True)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle on the host's cores (std::thread over elements): ~20 s of CPU work
        nth = host_threads()
        om, P, U2, L2, _, n = time_oracle_sample(wl, target_s=20.0)
        t0 = time.perf_counter()
        om.condense(P, U2, L2, 0, n, threads=nth)
        dt = time.perf_counter() - t0
        n1 = max(32, n // 4)
        t1 = time.perf_counter()
        om.condense(P, U2, L2, 0, n1)
        dt1 = time.perf_counter() - t1
        line["cpu_baseline"] = {"value": n / dt, "unit": "elements/s", "cores": nth, "kind": "oracle",
                                "sample": f"elements 0..{n - 1} of {om.n_elem} (condensation + assembly), "
                                          f"{nth} host threads, {dt:.1f} s",
                                "single_thread_value": n1 / dt1,
                                "accuracy_of_gpu_results": {
                                    "bar": "1e-12 relative (binary64), 1e-10 (float-float) on X_B per element and "
                                           "K per block; E = H - C X_F and dU are residual-type (they cancel), "
                                           "reported as global relative errors",
                                    **acc}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- profiling driver
PROFILE_VARIANTS = [("euler", p, prec) for p in (1, 2, 3, 4) for prec in (0, 1)] + \
                   [("ns", p, prec) for p in (1, 2, 3, 4) for prec in (0, 1)]


def run_profile_variants(args):
    """One condensation launch of every element kernel (Euler and Navier-Stokes, p = 1..4, binary64 and
    float-float), each on a small uniform-degree periodic mesh (args.cells, default 16x32 cells: 1,024
    triangles), in PROFILE_VARIANTS order and without autotuning or warm-up: the command that the
    instruction-count capture (ncu -k regex:k_condense) runs.  Prints the launch order as one JSON line."""
    import torch

    from paper_1308_3995_gb300 import hdg
    from paper_1308_3995_gb300 import inputs as G
    dev = torch.device("cuda:0")
    ctx = hdg.Context(0)
    nx, ny = (int(v) for v in (args.cells or "16x32").lower().split("x"))
    order = []
    for model, p, prec in PROFILE_VARIANTS:
        base = G.WORKLOADS["euler_p3_16k" if model == "euler" else "ns_mixp_65k"]
        wl = G.small_variant(base, nx, ny, p=p, probs=None)
        c = G.make_case(wl)
        mesh = hdg.Mesh(ctx, c.mesh.elem_xy, c.mesh.elem_vid, c.elem_p, c.nfield, c.mesh.elem_bc)
        U, Lam, _ = G.case_state(c, mesh.face_vid, mesh.face_p)
        prm = hdg.Params(model=wl.model, precision=prec, mach=wl.mach, alpha=wl.alpha, reynolds=wl.reynolds,
                         prandtl=wl.prandtl, aoa=wl.aoa)
        sysm = hdg.System(ctx, mesh, prm)
        sysm.condense(torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev))
        torch.cuda.synchronize()
        order.append({"model": model, "p": p, "precision": prec, "elements": mesh.n_elem,
                      "launches": sysm.launches})
        sysm.close()
        mesh.close()
    print(json.dumps({"profile_variants": order}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="euler_p3_16k")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--sc-eps0", type=float, default=0.0, help="shock capturing eps_0 on the headline workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", default=None, help="override the grid, e.g. 48x96 (profiling runs)")
    ap.add_argument("--quick", action="store_true", help="headline workload only (no per-p, NS, serving)")
    ap.add_argument("--serving-requests", type=int, default=512)
    ap.add_argument("--serving-max-elems", type=int, default=64000)
    ap.add_argument("--serving-solve-requests", type=int, default=32)
    ap.add_argument("--serving-solve-max-elems", type=int, default=32000)
    ap.add_argument("--serving-rates", default="0.7", help="load levels, fractions of saturated throughput")
    ap.add_argument("--serving-arena-gb", type=int, default=24)
    ap.add_argument("--serving-only", action="store_true", help="run only the serving section")
    ap.add_argument("--solve-only", action="store_true", help="run only the trace-solve section")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes (no hdg_autotune)")
    ap.add_argument("--profile-variants", action="store_true",
                    help="one launch of every element kernel on a small mesh (instruction-count capture)")
    args = ap.parse_args(argv)
    if args.profile_variants:
        return run_profile_variants(args)
    from paper_1308_3995_gb300 import inputs as G
    wl = G.WORKLOADS[args.workload]
    if args.cells:
        nx, ny = (int(v) for v in args.cells.lower().split("x"))
        wl = G.small_variant(wl, nx, ny)
    ws, rank, local = dist_env()
    Measured.autotune = not args.no_autotune
    if args.impl == "reference":
        return run_reference(args, wl, rank)
    return run_ours(args, wl, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
