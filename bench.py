"""Benchmark: GaBP edge-updates/s on the random sparse symmetric workload (n = 2^20).

One step = one complete solve of A x = b to relative residual 1e-10 through the
C ABI: FP32 joint rounds (precision and mean messages together until the
precisions are stationary), frozen coefficients, FP32 mean rounds and FP64
iterative refinement (the precision state is recomputed every step, nothing is
cached between steps).  value = directed edges x rounds of all steps / device
time.  The plain FP64 GaBP solve of the same system is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its
own right-hand side on its own GPU (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N_NODES = 1 << 20
PICKS = 8
DIAG = 1.1
SEED = 2
TOL = 1e-10
METRIC = "GaBP edge-updates/s (solve to relative residual 1e-10, FP32 messages + FP64 refinement)"
WORKLOAD = (f"random sparse symmetric diagonally dominant A, n=2^20, {PICKS} uniform picks per row symmetrised, "
            f"values U(-1,1), diagonal {DIAG} x row abs-sum, b ~ N(0,1)")


def kernel_source_sha(source, kernel):
    """sha256 of a kernel's own definition (from its template / __global__ line to
    the closing brace in column 0) plus the shared device helpers (devutil.cuh):
    a committed ncu summary stays valid while neither changes."""
    import hashlib

    import re

    lines = open(os.path.join(ROOT, source)).read().split("\n")
    pat = re.compile(r"__global__.*\b" + re.escape(kernel) + r"\s*\(")
    start = next(i for i, l in enumerate(lines) if pat.search(l))
    if start > 0 and lines[start - 1].startswith("template"):
        start -= 1
    end = next(i for i in range(start + 1, len(lines)) if lines[i] == "}")
    body = "\n".join(lines[start:end + 1])
    helpers = open(os.path.join(ROOT, "paper_0811_2518_gb300", "csrc", "devutil.cuh")).read()
    return hashlib.sha256((body + "\n" + helpers).encode()).hexdigest()


def _profiled_traffic(summary, source, kernel, scale_to=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current source of the kernel (the summary records kernel_source_sha)."""
    ps, src = os.path.join(ROOT, "profiles", summary), os.path.join(ROOT, source)
    if not (os.path.exists(ps) and os.path.exists(src)):
        return None
    try:
        sha = kernel_source_sha(source, kernel)
    except StopIteration:
        return None
    vals = {}
    for line in open(ps):
        if ":" in line:
            k, v = line.split(":", 1)
            v = v.strip().split()
            if v:
                vals[k.strip(" -*`")] = v[0].strip("`")
    if vals.get("kernel_source_sha256") != sha:
        return None
    try:
        traffic = float(vals["dram_bytes_per_launch"])
        if scale_to is not None:  # captured on a smaller case: scale by the units processed
            traffic *= scale_to / float(vals["algorithmic_bytes_captured"])
        return traffic
    except (KeyError, ValueError):
        return None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (every 100 ms, one streaming process) of SM clock and throttle
    reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._proc = None
        self._th = None
        self._t_begin = 0.0

    def start(self):
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return

        def run():
            for line in self._proc.stdout:
                v = [x.strip() for x in line.split(",")]
                if len(v) >= 7:
                    self.samples.append((time.perf_counter(), v))

        self._th = threading.Thread(target=run, daemon=True)
        self._th.start()
        t0 = time.perf_counter()
        while not self.samples and time.perf_counter() - t0 < 2.0:  # the sampler is running
            time.sleep(0.01)
        self._t_begin = time.perf_counter()

    def stop(self):
        t_end = time.perf_counter()
        time.sleep(0.15)  # the sample that covers the end of the region
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._th:
            self._th.join(timeout=5)
        window = [v for t, v in self.samples if self._t_begin <= t <= t_end + 0.1]
        if not window and self.samples:  # region shorter than the sampling period: the nearest sample
            window = [min(self.samples, key=lambda tv: abs(tv[0] - t_end))[1]]
        self.samples = window
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in self.samples for j in range(4) if s[3 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def oracle_rounds_sample(m, b, rounds=3):
    """The oracle (Algorithm 2, plain C) on `rounds` rounds of matrix m, input checks outside the timed
    rounds: edge-updates/s on all host cores (OpenMP build) and on one core (one round)."""
    import oracle

    oracle.gabp_broadcast(m, b, max_iter=0, tol=0.0)
    par = oracle.host_threads()
    edges = int(m.rowptr[-1]) - m.n  # off-diagonal entries = directed edges
    out = {"rounds": rounds, "edges": edges}
    if par:
        _, dt = oracle.broadcast_timed(m, b, rounds, threads=True)
        out.update({"all_cores": edges * rounds / dt, "cores": par})
    _, dt1 = oracle.broadcast_timed(m, b, 1, threads=False)
    out["one_core"] = edges / dt1
    return out


def oracle_threads():
    """Threads of the all-cores oracle build (None when gcc had no OpenMP)."""
    import oracle

    return oracle.host_threads()


def host_cpu():
    """CPU model and core count of the host the oracle runs on."""
    import platform

    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                model = (model + " / " if model else "") + line.split(":", 1)[1].strip()
    except Exception:
        pass
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def cpu_baseline_sample(m, b, rounds=5, what="the full n=2^20 matrix", single_rounds=2):
    """The FP64 oracle (Algorithm 2, plain C) on a bounded sample: `rounds` synchronous rounds over
    the matrix `m` on all host cores (the OpenMP build of the same file), and `single_rounds` on one
    core; the input checks run once before, outside the timed rounds."""
    import oracle

    oracle.gabp_broadcast(m, b, max_iter=0, tol=0.0)  # input checks (and the build)
    threads = oracle.host_threads()
    out = {"unit": "edge-updates/s", "kind": "oracle", "host": host_cpu()}
    _, dt1 = oracle.broadcast_timed(m, b, single_rounds, threads=False)
    single = {"value": m.num_edges * single_rounds / dt1, "cores": 1,
              "sample": f"{single_rounds} rounds over {what} ({m.num_edges} directed edges), {dt1:.1f} s"}
    if threads:
        _, dt = oracle.broadcast_timed(m, b, rounds, threads=True)
        out.update({"value": m.num_edges * rounds / dt, "cores": threads,
                    "sample": f"{rounds} rounds of the FP64 broadcast oracle over {what} ({m.num_edges} directed "
                              f"edges) on {threads} threads, input checks outside the timed rounds, {dt:.1f} s",
                    "single_core": single})
    else:
        out.update(single)
        out["sample"] = "one core (no OpenMP build): " + single["sample"]
    return out


REFERENCE_BUDGET_S = 150.0  # the whole --impl reference run (warm-up + timed steps)


def run_reference(args, rank, world):
    """The oracle as the reference arm: every step is one synchronous round of the FP64 oracle
    (Algorithm 2, plain C, the OpenMP build on all host cores) over a sample of the benchmark
    workload -- the full n = 2^20 matrix when (warmup + steps) such rounds fit the time budget, else
    a smaller matrix of the same family (same picks, values and diagonal rule, n a power of two)
    sized so that the whole run does.  The input checks run once, outside the steps."""
    if rank != 0:
        return 0
    import oracle

    t_all = time.perf_counter()
    m = synth.random_sym(N_NODES, PICKS, DIAG, SEED)
    b = synth.rhs(m.n, SEED)
    total = args.warmup + args.steps
    oracle.gabp_broadcast(m, b, max_iter=0, tol=0.0)  # input checks once (and the build)
    threads = oracle.host_threads()
    par = threads is not None
    _, t_round = oracle.broadcast_timed(m, b, 1, threads=par)  # the first warm-up step, also the size probe
    n_s, what = m.n, "the full n=2^20 matrix"
    if total * t_round > REFERENCE_BUDGET_S:
        while n_s > (1 << 14) and total * t_round * n_s / m.n > REFERENCE_BUDGET_S:
            n_s //= 2
        m = synth.random_sym(n_s, PICKS, DIAG, SEED)
        b = synth.rhs(m.n, SEED)
        oracle.gabp_broadcast(m, b, max_iter=0, tol=0.0)
        what = f"random_sym(n={n_s}) of the same family"
    vals = []
    for st in range(1, total):
        _, dt = oracle.broadcast_timed(m, b, 1, threads=par)
        if st >= args.warmup:
            vals.append(m.num_edges / dt)
    if not vals:  # steps = 0 or only the probe ran
        vals = [m.num_edges / t_round]
    v = float(np.mean(vals))
    ms = m.num_edges / v * 1e3
    cores = threads if par else 1
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "edge-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N_NODES, "sample_n": m.n, "sample_edges": m.num_edges,
                       "sample_per_step": f"1 oracle round over {what}"},
            "cpu_baseline": {"value": v, "unit": "edge-updates/s", "cores": cores, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"1 round of the FP64 broadcast oracle per step over {what} on {cores} "
                                       f"thread(s), input checks once before the steps"},
            "e2e": {"value": v, "unit": "edge-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=0,
                    help="sub-warp width of the R = 1 kernels (0 = the library's autotuner)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch every kernel on its own instead of replaying captured CUDA graphs (for "
                         "per-kernel profilers; results are the same)")
    ap.add_argument("--unroll", type=int, default=0,
                    help="with --lanes: slots per lane of the FP32 round kernels (0 = the library default)")
    ap.add_argument("--batched-grid", type=int, default=128,
                    help="edge length m of the m^3 grid of the batched leg (128 = the 64-RHS workload)")
    ap.add_argument("--multi-mode", type=int, default=0,
                    help="independent-systems kernel: 0 autotune, 1 grid-persistent, 2 teams, 3 grid-persistent "
                         "on the sliced layout")
    ap.add_argument("--multi-systems", type=int, default=512,
                    help="number of random geometric graphs of the independent-systems leg (512 = the workload)")
    ap.add_argument("--dense-n", type=int, default=8192,
                    help="points of the dense kernel-regression leg (n x n dense matrix)")
    ap.add_argument("--legs", default="fp32,fp64,e2e,oracle,edge,c1,lsq,dense,batched,multi,grad,fix",
                    help="comma list of timed legs (fp32 is the headline; the others add keys)")
    args = ap.parse_args()
    gkw = {"graphs": 0} if args.no_graphs else {}  # solver options of every handle below

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import paper_0811_2518_gb300 as gb
    from paper_0811_2518_gb300.replicas import Replicas

    reps = Replicas()  # one replica per GPU (weak scaling); the group only times and counts

    def barrier():
        reps.barrier()
        torch.cuda.synchronize()

    m = synth.random_sym(N_NODES, PICKS, DIAG, SEED)
    b = synth.rhs(m.n, SEED + rank)
    E = m.num_edges
    dev = torch.device("cuda", local)
    b_dev = torch.from_numpy(b).to(dev)
    x_dev = torch.empty_like(b_dev)

    s32 = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, reuse_precisions=0, profile=1, lanes=args.lanes, **gkw,
                             unroll=args.unroll if args.lanes else 0)
    s64 = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP64, profile=1, lanes=args.lanes, **gkw)

    def step(s):
        _, st, it, rel = s.solve(b_dev, tol=TOL, max_iter=2000, x=x_dev)
        if st != gb.GABP_OK:
            raise RuntimeError(f"solve status {st} relres {rel}")
        return s.stats()["rounds"], rel

    # ---- FP32 + refinement (headline): the library's default path -- the whole refinement loop
    # as one CUDA graph with device-side decisions, no per-phase timers -- over `steps` solves
    sd = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, reuse_precisions=0, lanes=args.lanes, **gkw,
                            unroll=args.unroll if args.lanes else 0)
    for _ in range(args.warmup):
        step(sd)
    sd.profile(reset=True)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record()
    rounds = 0
    rel = None
    for _ in range(args.steps):
        r, rel = step(sd)
        rounds += r
    ev1.record()
    barrier()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = float(clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0)  # the timed region's SM clock
    x_fp32 = x_dev.cpu().numpy()  # the headline's answer, compared with the oracle below
    ms_local = ev0.elapsed_time(ev1)
    launches_timed = sd.profile(reset=True)["launches"]
    sd.close()
    # the same solves once more through the host-driven loop with CUDA-event timers per phase
    # (round counts, phase times and the dominant kernel's live launch time for the roofline)
    for _ in range(args.warmup):
        step(s32)
    s32.profile(reset=True)
    for _ in range(args.steps):
        step(s32)
    prof = s32.profile(reset=True)
    # whole job: every rank's edge-updates over the slowest rank's time
    ms_total = reps.max(ms_local, device=dev)
    value = reps.job_rate(E * rounds, ms_local / 1e3, device=dev)
    ms_step = ms_total / args.steps

    # roofline of the dominant kernel (largest phase time in the timed region)
    peak, peak_kind = _peaks()
    ph = max(("mean32", "prec32"), key=lambda k: prof["ms"][k])
    n = m.n
    # algorithmic bytes per launch (what the method itself must move per round, node arrays taken as
    # L2-resident): FP32 mean round at one right-hand side 16 B per directed edge (coefficient 4, sender
    # index 4, h read 4, h write 4) + 8 B per node; FP32 full round (precision and mean messages, the
    # "prec32" phase of a solve with joint rounds) 24 B per edge (A 4, sender 4, (P, h) read 8, (P, h)
    # write 8) + 12 B per node.  The implementation's own bytes (recompute form: both coefficients,
    # previous-round chains, node rings) are reported beside them.
    bytes_launch = (16 * E + 8 * n) if ph == "mean32" else (24 * E + 12 * n)
    impl_bytes = (20 * E + 24 * n) if ph == "mean32" else (28 * E + 36 * n)
    dur_ms = prof["ms"][ph] / max(prof["rounds"][ph], 1)
    achieved = bytes_launch / (dur_ms / 1e3) / 1e9
    kname = "k32_mean" if ph == "mean32" else "k32_joint"
    _ts = s32.tuned()
    tuned = {"k32_mean": _ts["mean32"], "k32_joint": _ts["prec32"]}  # (lanes per row, slots per lane)
    if args.lanes:  # pinned: the library's mapping of (lanes, unroll)
        _L = min(args.lanes, 16)
        tuned = {k: (_L, args.unroll or (1 if _L >= 16 else 4)) for k in tuned}

    legs = set(args.legs.split(","))

    # the random-gather ceiling the mean round meets on this graph: one 4-byte load per slot from a
    # random row of an n-float array (torch's index_select over the round's own sender indices),
    # timed like the round (CUDA events, L2-resident source, E indices streamed)
    gather = None
    if "fp32" in legs:
        src = torch.randn(n, device=dev, dtype=torch.float32)
        idx = torch.from_numpy(m.col[m.col != np.repeat(np.arange(n), np.diff(m.rowptr))].astype(np.int64)).to(dev)
        out = torch.empty(idx.numel(), device=dev, dtype=torch.float32)
        for _ in range(3):
            torch.index_select(src, 0, idx, out=out)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(20):
            torch.index_select(src, 0, idx, out=out)
        g1.record()
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / 20
        gather = {"what": "index_select of the E sender indices of the benchmark graph from an n-float array "
                          "(4-byte random gathers, 8-byte indices streamed): the gather part of a mean round alone",
                  "ms": gms, "gathers_per_s": idx.numel() / (gms / 1e3),
                  "mean_round_ms": dur_ms if ph == "mean32" else None,
                  "mean_round_vs_gather_only": (dur_ms / gms) if ph == "mean32" else None}
        del src, idx, out

    ms64, r64, k64, p64, x_fp64, ms64fz = None, 0, 1, {"ms": {"fp64": 0.0}}, None, None
    # ---- plain FP64 GaBP on the same system (time to 1e-10)
    for _ in range(max(1, args.warmup) if "fp64" in legs else 0):
        step(s64)
    if "fp64" in legs:
        s64.profile(reset=True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        k64 = max(1, min(args.steps, 5))
        for _ in range(k64):
            rr, _ = step(s64)
            r64 += rr
        e1.record()
        barrier()
        ms64 = e0.elapsed_time(e1) / k64
        p64 = s64.profile(reset=True)
        x_fp64 = x_dev.cpu().numpy()
        # the same with the precision freeze (options.freeze_precisions): on this graph the
        # precisions settle about when the means do, so few rounds run frozen
        sfz = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP64, freeze_precisions=1, **gkw)
        for _ in range(max(1, args.warmup)):
            step(sfz)
        barrier()
        e0.record()
        rfz = 0
        for _ in range(k64):
            rr, relfz = step(sfz)
            rfz += rr
        e1.record()
        barrier()
        fz = sfz.stats()
        ms64fz = {"ms_per_solve": e0.elapsed_time(e1) / k64, "rounds": rfz / k64, "relres": relfz,
                  "freeze_round": fz["freeze_round"], "verifications": fz["freeze_checks"],
                  "max_abs_diff_vs_fp64_plain": float(np.max(np.abs(x_dev.cpu().numpy() - x_fp64)))}
        sfz.close()

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    # (default options: the refinement loop runs as one CUDA graph, no per-phase timing events)
    e2e_rounds, e2e_s = 0, None
    if "e2e" in legs:
        se = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP32_REFINE, reuse_precisions=0, lanes=args.lanes, **gkw,
                                unroll=args.unroll if args.lanes else 0)
        bh = torch.from_numpy(b).pin_memory().numpy()
        xh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        for _ in range(max(1, args.warmup)):
            se.solve_host(bh, xh, tol=TOL, max_iter=2000)
        barrier()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            st, it, rr = se.solve_host(bh, xh, tol=TOL, max_iter=2000)
            if st != gb.GABP_OK:
                raise RuntimeError(f"e2e solve status {st}")
            e2e_rounds += se.stats()["rounds"]
        barrier()
        e2e_s = time.perf_counter() - t1
        se.close()

    # ---- batched: 128^3 heterogeneous diffusion grid, 64 right-hand sides in one launch sequence,
    # serial schedule (red-black on this grid) and, for comparison, the parallel schedule
    batched = None
    if "batched" in legs:
        try:
            s32.close()
            s64.close()
            mg = synth.grid3d(args.batched_grid, 1.05, 3)
            Rb = 64
            Bb = torch.from_numpy(synth.rhs_batch(mg.n, Rb, 3 + rank)).to(dev)
            Eg, ng = mg.num_edges, mg.n
            res = {}
            for sched in (1, 0):
                sb = gb.Solver.from_csr(mg, profile=1, reuse_precisions=0, schedule=sched, **gkw)
                Xb, stb, itb, relb = sb.solve_batched(Bb, tol=TOL)
                sb.profile(reset=True)
                barrier()
                eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                eb0.record()
                Xb, stb, itb, relb = sb.solve_batched(Bb, tol=TOL, X=Xb)
                eb1.record()
                barrier()
                res[sched] = (eb0.elapsed_time(eb1), sb.profile(reset=True), sb.stats(), stb, itb, float(np.max(relb)),
                              sb.serial_colours()[1] if sched else 1)
                sb.close()
            # plain FP64 GaBP on one right-hand side of the same grid (time to 1e-10), both schedules: the
            # batched solve is compared with 64 x that
            fp64_one = {}
            for sched in (0, 1, 2, 3):  # 2, 3: the parallel and serial schedules with the precision freeze
                s1 = gb.Solver.from_csr(mg, precision=gb.GABP_PREC_FP64, schedule=int(sched in (1, 3)),
                                        freeze_precisions=int(sched >= 2), **gkw)
                b1 = Bb[0].contiguous()
                x1, st1, it1, rel1 = s1.solve(b1, tol=TOL, max_iter=5000)
                barrier()
                e10, e11 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e10.record()
                x1, st1, it1, rel1 = s1.solve(b1, tol=TOL, max_iter=5000, x=x1)
                e11.record()
                barrier()
                fp64_one[("parallel", "serial", "parallel_frozen_precisions", "serial_frozen_precisions")[sched]] = {
                    "ms_one_rhs": e10.elapsed_time(e11), "rounds": int(it1), "status": int(st1), "relres": rel1,
                    "ms_x64": 64 * e10.elapsed_time(e11), "freeze_round": s1.stats()["freeze_round"]}
                s1.close()
                del x1
            cpu_b = None
            if not args.no_cpu_baseline and rank == 0:
                cpu_b = oracle_rounds_sample(mg, synth.rhs_batch(mg.n, 1, 3)[0])
            msb, pb, stats_b, stb, itb, maxrel, ncol = res[1]
            mean_ms = pb["ms"]["mean32"] / max(pb["rounds"]["mean32"], 1)  # one sweep (all colour passes)
            # per sweep: every slot once (R messages read + written, coefficient pair, sender) and every row once
            # (R firing aggregates read + written, R right-hand sides, segment bounds / colour / row pointer)
            bytes_b = Eg * (8 * Rb + 12) + ng * (12 * Rb + 20)
            # the method's own bytes per sweep: per edge R mean messages read and written (8 R) and the frozen
            # coefficient with the reverse index (8), per node the R aggregates (8 R)
            alg_b = Eg * (8 * Rb + 8) + 8 * Rb * ng
            # DRAM bytes from a capture of the 64^3 case (a few GB on the device; the 128^3 x 64 workload is
            # too large to capture under ncu), scaled to this sweep by the implementation's bytes
            traffic_b = _profiled_traffic("kbs_pass_grid3d_64_64rhs.md", "paper_0811_2518_gb300/csrc/batched.cu",
                                          "kbs_pass", scale_to=bytes_b)
            traffic_note_b = ("DRAM bytes per sweep, scaled from one captured pass of the 64^3 case (the two "
                              "red-black passes move equal bytes) by the implementation's bytes")
            batched = {"workload": f"{args.batched_grid}^3 7-point grid, face coefficients LogNormal(0,1), diagonal 1.05 x "
                                   "row abs-sum, 64 right-hand sides N(0,1)", "n": ng, "edges": Eg, "rhs": Rb,
                       "schedule": f"serial (one message store, {ncol} colours: red-black on this grid)",
                       "status": stb, "ms_per_solve": msb, "inner_sweeps": itb, "refine_steps": stats_b["refine_steps"],
                       "max_relres": maxrel, "rhs_edge_updates_per_s": stats_b["edge_updates"] / (msb / 1e3),
                       "ms_per_rhs": msb / Rb,
                       "parallel_schedule": {"ms_per_solve": res[0][0], "inner_rounds": res[0][4],
                                             "max_relres": res[0][5]},
                       "fp64_plain_one_rhs": fp64_one, "cpu_oracle_one_rhs": cpu_b,
                       "batched_vs_64_fp64": {k: v["ms_x64"] / msb for k, v in fp64_one.items()},
                       "roofline": {"bound": "hbm", "kernel": "kbs_pass (one sweep = all colour passes)",
                                    "achieved": alg_b / (mean_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                                    "frac": alg_b / (mean_ms / 1e3) / 1e9 / peak,
                                    "algorithmic_bytes_per_sweep": alg_b,
                                    "algorithmic_bytes_rule": "E (8 R + 8) + 8 R n per sweep, R = 64",
                                    "traffic": traffic_b,
                                    "traffic_over_algorithmic": None if traffic_b is None else traffic_b / alg_b,
                                    "traffic_note": traffic_note_b,
                                    "impl_bytes_per_sweep": bytes_b,
                                    "impl_frac": bytes_b / (mean_ms / 1e3) / 1e9 / peak, "sweep_ms": mean_ms}}
        except Exception as exc:  # one GPU: keep the headline line, record the failed leg
            if world > 1:
                raise
            batched = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- 512 independent random-geometric-graph systems in one persistent launch
    multi = None
    if "multi" in legs:
        try:
            mats = synth.rgg_batch(args.multi_systems, 1024, 65536, 2.0, 4)
            bigm = synth.block_diag(mats)
            offm = bigm.meta["offsets"]
            bm = torch.from_numpy(synth.rhs(bigm.n, 4 + rank)).to(dev)
            sm = gb.Solver.from_csr(bigm, multi_mode=args.multi_mode, **gkw)
            xm, stm, stsm, itsm, relm = sm.solve_systems(bm, offm, tol=TOL)  # first call autotunes the split
            sm.profile(reset=True)
            reps_m = 5  # timed batches (each one launch); the median is reported
            times_m = []
            for _ in range(reps_m):
                barrier()
                em0, em1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                em0.record()
                xm, stm, stsm, itsm, relm = sm.solve_systems(bm, offm, tol=TOL, x=xm)
                em1.record()
                barrier()
                times_m.append(em0.elapsed_time(em1))
            msm = float(np.median(times_m))
            pm = sm.profile(reset=True)
            stm_ = sm.stats()
            tuned_m = sm.tuned()
            # plain FP64 GaBP on every system by itself (a handle per system, created before the timing):
            # the sum of the 512 solve times, each to its own 1e-10
            hs = [gb.Solver.from_csr(ms_, precision=gb.GABP_PREC_FP64, **gkw) for ms_ in mats]
            bms = [bm[int(offm[i]):int(offm[i + 1])].contiguous() for i in range(len(mats))]
            xms = [torch.empty_like(v) for v in bms]
            for h_, bv, xv in zip(hs, bms, xms):
                h_.solve(bv, tol=TOL, max_iter=20000, x=xv)
            barrier()
            ep0, ep1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ep0.record()
            rounds_p = 0
            for h_, bv, xv in zip(hs, bms, xms):
                _, stp, itp, _ = h_.solve(bv, tol=TOL, max_iter=20000, x=xv)
                rounds_p += int(itp)
            ep1.record()
            barrier()
            ms_per_sys = ep0.elapsed_time(ep1)
            for h_ in hs:
                h_.close()
            del hs, bms, xms
            multi = {"workload": f"{args.multi_systems} random geometric graphs, sizes ~ n^-2 on [1024, 65536], "
                                 "radius for degree 6, "
                                 "weights -U(0.5,1), diagonal 1.1 x row abs-sum, one b ~ N(0,1) each",
                     "systems": len(mats), "n_total": bigm.n, "edges_total": bigm.num_edges, "status": int(stm),
                     "ms_per_batch": msm, "ms_per_batch_all": times_m, "kernel_ms": pm["ms"]["multi"] / reps_m,
                     "kernel": "grid-persistent" if (args.multi_mode in (1, 3) or tuned_m["multi_mode"] == 1) else "teams",
                     "grid_shape": {"lanes_per_row": tuned_m["multi_grid"][0], "slots_per_lane": tuned_m["multi_grid"][1],
                                    "sliced_layout": tuned_m["multi_grid_sliced"]},
                     "edge_updates": stm_["edge_updates"],
                     "edge_updates_per_s": stm_["edge_updates"] / (msm / 1e3),
                     "rounds_per_system": {"min": int(itsm.min()), "median": int(np.median(itsm)), "max": int(itsm.max())},
                     "max_relres": float(relm.max()), "launches_per_batch": 1,
                     "fp64_plain_per_system": {"ms_all_systems": ms_per_sys, "rounds_total": rounds_p,
                                               "how": "one FP64 handle per system, solved one after another"},
                     "batch_vs_fp64_per_system": ms_per_sys / msm,
                     "cpu_oracle": (oracle_rounds_sample(bigm, synth.rhs(bigm.n, 4))
                                    if not args.no_cpu_baseline and rank == 0 else None)}
            sm.close()
        except Exception as exc:  # one GPU: keep the headline line, record the failed leg
            if world > 1:
                raise
            multi = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- differentiable solve: n = 2^22, degree ~6, forward + hand-written backward
    grad = None
    if "grad" in legs:
        try:
            from paper_0811_2518_gb300 import autograd as ga

            mc = synth.random_sym(1 << 22, 3, 1.2, 5)
            rp_t = torch.from_numpy(mc.rowptr).to(dev)
            cl_t = torch.from_numpy(mc.col).to(dev)
            xs_t = torch.from_numpy(synth.rhs(mc.n, 105)).to(dev)
            b_c = synth.rhs(mc.n, 5 + rank)

            vals0 = torch.from_numpy(mc.val).to(dev)
            b0 = torch.from_numpy(b_c).to(dev)

            def fwd_bwd(solver=None):
                vals = vals0.detach().clone().requires_grad_(True)
                bt = b0.detach().clone().requires_grad_(True)
                xg = ga.gabp_solve_autograd(rp_t, cl_t, vals, bt, tol=TOL, solver=solver)
                loss = 0.5 * torch.sum((xg - xs_t) ** 2)
                loss.backward()
                return vals.grad, bt.grad

            def timed(f, reps=3):
                f()
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    f()
                e1.record()
                barrier()
                return e0.elapsed_time(e1) / reps

            ms_fresh = timed(fwd_bwd)
            shared = gb.Solver(mc.n, rp_t, cl_t, vals0, precision=gb.GABP_PREC_FP32_REFINE, **gkw)
            ms_shared = timed(lambda: fwd_bwd(shared))
            shared.close()
            grad = {"workload": "random sparse symmetric A, n=2^22, 3 picks per row (degree ~6), U(-1,1), diagonal "
                                "1.2 x row abs-sum; loss 0.5||x - x*||^2; FP32 messages + FP64 refinement",
                    "n": mc.n, "edges": mc.num_edges, "ms_forward_backward": ms_fresh,
                    "includes": "handle creation (validation, reverse index), forward solve (precision state "
                                "recomputed), adjoint solve on the same precision state, dL/dA and dL/db; inputs "
                                "already on the device",
                    "ms_forward_backward_shared_solver": ms_shared,
                    "cpu_oracle": (oracle_rounds_sample(mc, b_c) if not args.no_cpu_baseline and rank == 0
                                   else None),
                    "shared_solver": "one handle for the pattern, new values set each step (gabp_set_values) "
                                     "instead of a new handle"}
        except Exception as exc:  # one GPU: keep the headline line, record the failed leg
            if world > 1:
                raise
            grad = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- convergence fix on a non-walk-summable SPD matrix (n = 4096, diagonal 0.9 x row abs-sum):
    # the double loop (FP32 inner GaBP solves on A + Gamma) and the single loop (one FP64 round per step)
    fix = None
    if "fix" in legs:
        try:
            mf = synth.random_sym(4096, 3, 0.9, 5)
            bf = torch.from_numpy(synth.rhs(mf.n, 5)).to(dev)
            fix = {"workload": "random sparse symmetric A, n=4096, 3 picks per row, diagonal 0.9 x row abs-sum "
                               "(SPD, rho(|R|) = 1/0.9 > 1), uniform loading Gamma = 0.25 diag(A), to 1e-10"}
            for name, kw in (("double_loop", {}), ("single_loop", {"fix_single_loop": 1, "fix_step": 0.5})):
                sf = gb.Solver.from_csr(mf, gamma_mode=1, gamma=0.25, max_refine=2000, **kw, **gkw)
                sf.solve(bf, tol=TOL, max_iter=200000)
                barrier()
                ef0, ef1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ef0.record()
                xf, stf, itf, relf = sf.solve(bf, tol=TOL, max_iter=200000)
                ef1.record()
                barrier()
                fix[name] = {"ms": ef0.elapsed_time(ef1), "status": int(stf), "gabp_rounds": int(itf),
                             "outer_steps": sf.stats()["refine_steps"] if not kw else int(itf), "relres": relf}
                sf.close()
        except Exception as exc:  # one GPU: keep the headline line, record the failed leg
            if world > 1:
                raise
            fix = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- the oracle's FP64 solution of the benchmark system (all host cores, to 1e-13): the error of
    # every result of this system against it
    errors = None
    if "oracle" in legs and rank == 0 and world == 1:
        import oracle

        ro, dto = oracle.broadcast_timed(m, b, 200, threads=oracle.host_threads() is not None, tol=1e-13)
        xo = ro["x"]

        def err(x):
            return None if x is None else {"max_abs_over_max": float(np.max(np.abs(x - xo)) / np.max(np.abs(xo))),
                                           "rel_2norm": float(np.linalg.norm(x - xo) / np.linalg.norm(xo))}

        errors = {"oracle": {"rounds": ro["iters"], "relres": ro["relres"], "status": ro["status"], "s": dto},
                  "fp32_refine": err(x_fp32), "fp64_node": err(x_fp64)}

    # ---- the same system with the edge-centric FP64 variant (GABP_VARIANT_EDGE)
    edge = None
    if "edge" in legs:
        try:
            s64e = gb.Solver.from_csr(m, precision=gb.GABP_PREC_FP64, variant=gb.GABP_VARIANT_EDGE, profile=1,
                                      lanes=args.lanes, **gkw)
            step(s64e)
            barrier()
            ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ke, re_ = max(1, min(args.steps, 3)), 0
            ee0.record()
            for _ in range(ke):
                rr, rel_e = step(s64e)
                re_ += rr
            ee1.record()
            barrier()
            mse = ee0.elapsed_time(ee1) / ke
            edge = {"ms_per_solve": mse, "rounds": re_ / ke, "edge_updates_per_s": E * (re_ / ke) / (mse / 1e3),
                    "relres": rel_e}
            if errors is not None:
                edge["error_vs_oracle"] = err(x_dev.cpu().numpy())
            s64e.close()
        except Exception as exc:
            if world > 1:
                raise
            edge = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- the 32 x 32 grid (n = 1024), plain FP64 GaBP to 1e-12: parallel and serial schedules, and
    # Steffensen's iterations on the serial schedule; errors against the oracle's FP64 solution
    c1 = None
    if "c1" in legs:
        try:
            import oracle

            g1 = synth.grid2d(32, -1.0, 4.5)
            b1 = synth.rhs(g1.n, 1)
            ref1 = oracle.gabp_broadcast(g1, b1, max_iter=2000, tol=1e-12)
            bt1 = torch.from_numpy(b1).to(dev)
            c1 = {"workload": "32x32 5-point grid, off-diagonal -1, diagonal 4.5, b ~ N(0,1), to 1e-12",
                  "oracle_rounds": ref1["iters"]}
            if not args.no_cpu_baseline and rank == 0:  # the oracle's own time to 1e-12 (checks excluded)
                _, t1c = oracle.broadcast_timed(g1, b1, 2000, threads=False, tol=1e-12)
                c1["oracle_ms_one_core"] = t1c * 1e3
                if oracle.host_threads():
                    _, tac = oracle.broadcast_timed(g1, b1, 2000, threads=True, tol=1e-12)
                    c1["oracle_ms_all_cores"] = tac * 1e3
            for name, kw in (("parallel", {}), ("parallel_frozen_precisions", {"freeze_precisions": 1}),
                             ("serial", {"schedule": 1}),
                             ("serial_steffensen", {"schedule": 1, "accel": 2}),
                             ("parallel_steffensen", {"accel": 2})):
                sc = gb.Solver.from_csr(g1, precision=gb.GABP_PREC_FP64, **kw, **gkw)
                xc, stc, itc, relc = sc.solve(bt1, tol=1e-12, max_iter=2000)
                times = []
                for _ in range(20):
                    ec0, ec1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ec0.record()
                    xc, stc, itc, relc = sc.solve(bt1, tol=1e-12, max_iter=2000, x=xc)
                    ec1.record()
                    torch.cuda.synchronize()
                    times.append(ec0.elapsed_time(ec1))
                xn = xc.cpu().numpy()
                c1[name] = {"ms_per_solve": float(np.median(times)), "status": int(stc), "rounds": int(itc),
                            "relres": relc,
                            "error_vs_oracle": float(np.max(np.abs(xn - ref1["x"])) / np.max(np.abs(ref1["x"])))}
                sc.close()
        except Exception as exc:
            if world > 1:
                raise
            c1 = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- dense kernel-regression system: Gaussian kernel on n points in [0, 1]^3 (sigma 0.1), main
    # diagonal weighted to 1.1 x the row sum; FP32 + refinement and plain FP64 to 1e-10
    dense = None
    if "dense" in legs:
        try:
            nd = args.dense_n
            Ad = synth.rbf_kernel_system(nd, 3, 0.1, 1.1, 9)
            bdn = synth.rhs(nd, 9)
            Adt = torch.from_numpy(Ad).to(dev)
            bdt = torch.from_numpy(bdn).to(dev)
            dense = {"workload": f"dense {nd} x {nd} kernel matrix: Gaussian kernel (sigma 0.1) on {nd} points uniform "
                                 "in [0,1]^3, main diagonal 1.1 x the row sum; b ~ N(0,1); to 1e-10",
                     "n": nd}
            for name, prec in (("fp32_refine", gb.GABP_PREC_FP32_REFINE), ("fp64", gb.GABP_PREC_FP64)):
                sdn = gb.Solver.from_dense(Adt, precision=prec, reuse_precisions=0, **gkw)
                Edn = sdn.nnz - nd
                xd_, std_, itd_, reld_ = sdn.solve(bdt, tol=TOL, max_iter=2000)
                times = []
                for _ in range(3):
                    ed0, ed1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ed0.record()
                    xd_, std_, itd_, reld_ = sdn.solve(bdt, tol=TOL, max_iter=2000, x=xd_)
                    ed1.record()
                    torch.cuda.synchronize()
                    times.append(ed0.elapsed_time(ed1))
                rounds_d = sdn.stats()["rounds"]
                msd = float(np.median(times))
                xh = xd_.cpu().numpy()
                entry = {"ms_per_solve": msd, "status": int(std_), "rounds": int(rounds_d), "relres": reld_,
                         "host_relres": float(np.linalg.norm(bdn - Ad @ xh) / np.linalg.norm(bdn)),
                         "edge_updates_per_s": Edn * rounds_d / (msd / 1e3), "edges": Edn}
                if prec == gb.GABP_PREC_FP32_REFINE:  # the mean round's live time from a profiled run
                    sdn.set_options(profile=1, device_loop=0)
                    sdn.solve(bdt, tol=TOL, max_iter=2000, x=xd_)
                    sdn.profile(reset=True)
                    sdn.solve(bdt, tol=TOL, max_iter=2000, x=xd_)
                    pd = sdn.profile(reset=True)
                    mean_ms = pd["ms"]["mean32"] / max(pd["rounds"]["mean32"], 1)
                    alg = 16 * Edn + 8 * nd
                    entry["roofline"] = {"bound": "hbm", "kernel": "k32_mean", "launch_ms": mean_ms,
                                         "algorithmic_bytes_per_launch": alg,
                                         "algorithmic_bytes_rule": "16 B per directed edge + 8 B per node",
                                         "achieved": alg / (mean_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                                         "frac": alg / (mean_ms / 1e3) / 1e9 / peak,
                                         # a complete pattern's mean round reads no column indices
                                         "impl_frac": (16 * Edn + 24 * nd) / (mean_ms / 1e3) / 1e9 / peak}
                    x32 = xh
                else:
                    entry["max_abs_diff_fp32_refine_vs_fp64"] = float(np.max(np.abs(xh - x32)))
                dense[name] = entry
                sdn.close()
            if not args.no_cpu_baseline and rank == 0:  # the oracle scans rows: a 1024-point instance
                As = synth.rbf_kernel_system(1024, 3, 0.1, 1.1, 9)
                dense["cpu_oracle_n1024"] = oracle_rounds_sample(synth.from_dense(As), synth.rhs(1024, 9), rounds=2)
            del Adt, Ad
        except Exception as exc:
            if world > 1:
                raise
            dense = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- regularised least squares through the augmented symmetric system: J 2^20 x 2^19, 8 entries
    # per row N(0,1)/sqrt(8), gamma = 1, y ~ N(0,1), to 1e-10 (FP32 + refinement and plain FP64)
    lsq = None
    if "lsq" in legs:
        try:
            from scipy.sparse import csr_matrix

            J = synth.random_rect(1 << 20, 1 << 19, 8, 21)
            yl = synth.rhs(J.m, 22 + rank)
            S = csr_matrix((J.val, J.col, J.rowptr), shape=(J.m, J.k))
            jty = S.T @ yl
            yt = torch.from_numpy(yl).to(dev)
            Ea = 2 * J.nnz
            lsq = {"workload": "J 2^20 x 2^19 sparse, 8 entries per row N(0,1)/sqrt(8), gamma = 1, y ~ N(0,1): "
                               "x = (J^T J + gamma I)^{-1} J^T y via [[I, J^T], [J, -gamma I]] (n = 1572864, "
                               f"{Ea} directed edges), to relative residual 1e-10", "edges": Ea}
            for name, prec in (("fp32_refine", gb.GABP_PREC_FP32_REFINE), ("fp64", gb.GABP_PREC_FP64)):
                sl = gb.LSQSolver.from_rect(J, 1.0, precision=prec, reuse_precisions=0, **gkw)
                xl, _, stl, itl, rell = sl.solve_lsq(yt, tol=TOL, max_iter=5000)
                barrier()
                el0, el1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                kl, rounds_l = 3, 0
                el0.record()
                for _ in range(kl):
                    xl, _, stl, itl, rell = sl.solve_lsq(yt, tol=TOL, max_iter=5000)
                    rounds_l += sl.stats()["rounds"]
                el1.record()
                barrier()
                msl = el0.elapsed_time(el1) / kl
                xn = xl.cpu().numpy()
                lsq[name] = {"ms_per_solve": msl, "status": int(stl), "rounds": rounds_l / kl, "relres": rell,
                             "edge_updates_per_s": Ea * (rounds_l / kl) / (msl / 1e3),
                             "normal_equation_residual": float(np.linalg.norm(S.T @ (yl - S @ xn) - xn) /
                                                               np.linalg.norm(jty))}
                sl.close()
            if not args.no_cpu_baseline and rank == 0:
                import oracle

                lsq["cpu_oracle"] = oracle_rounds_sample(oracle.lsq_augmented(J, 1.0),
                                                         np.concatenate([np.zeros(J.k), yl]))
            del S, J
        except Exception as exc:
            if world > 1:
                raise
            lsq = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(m, b, rounds=5)

    traffic_main = _profiled_traffic(f"{kname}_random_sym_n1048576.md", "paper_0811_2518_gb300/csrc/solve32.cu",
                                     kname)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "edge-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "edges": E, "nnz": m.nnz, "rhs": 1, "tol": TOL,
                       "precision": "FP32 messages, FP64 residual and update",
                       "rounds_per_step": rounds / args.steps, "final_relres": rel,
                       "l2": "inputs larger than L2: 268 MB of edge state read and written per round",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "path": "default options: the refinement loop as one CUDA graph with device-side "
                               "decisions; phases_ms_per_step and the roofline's launch time come from a "
                               "second run of the same solves with per-phase CUDA-event timers"},
            "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic_main,
                         "algorithmic_bytes_per_launch": bytes_launch,
                         "algorithmic_bytes_rule": ("16 B per directed edge + 8 B per node (FP32 mean round, one "
                                                    "right-hand side)" if ph == "mean32" else
                                                    "24 B per directed edge + 12 B per node (FP32 full round)"),
                         "impl_bytes_per_launch": impl_bytes, "impl_frac": impl_bytes / (dur_ms / 1e3) / 1e9 / peak,
                         "traffic_over_algorithmic": None if traffic_main is None else traffic_main / bytes_launch,
                         "launch_ms": dur_ms,
                         "shape": {"lanes_per_row": tuned[kname][0], "slots_per_lane": tuned[kname][1]},
                         "random_gather_reference": gather},
            "phases_ms_per_step": {k: v / args.steps for k, v in prof["ms"].items()},
            "rounds_per_step_by_phase": {k: v / args.steps for k, v in prof["rounds"].items()},
            "gpu_launches": launches_timed,
            "time_to_1e-10_ms": {"fp32_refine": ms_step, "fp64_plain": ms64,
                                 "fp64_frozen_precisions": None if ms64fz is None else ms64fz["ms_per_solve"]},
            "fp64_frozen_precisions": ms64fz,
            "fp64_plain": None if ms64 is None else {
                "ms_per_solve": ms64, "rounds": r64 / k64, "edge_updates_per_s": E * (r64 / k64) / (ms64 / 1e3),
                "phase_ms": p64["ms"]["fp64"] / k64,
                "roofline": {"bound": "fp64 alu", "kernel": "k64_node",
                             # FP64 instructions of a round, counted by ncu's per-opcode counters: per message
                             # 4 DADD + 4 DFMA + 3 DMUL, per row 3 + 5 + 1; GB300 retires 2 FP64 operations per
                             # SM and clock (1.25 TFLOP/s FMA at 2.07 GHz on 152 SMs)
                             "fp64_ops_per_round": 11 * E + 9 * n,
                             "fp64_peak_ops_per_s": 2.0 * n_sms * clk_mhz * 1e6,
                             "alu_frac": (11 * E + 9 * n) / (p64["ms"]["fp64"] / max(p64["rounds"]["fp64"], 1) / 1e3)
                                         / (2.0 * n_sms * clk_mhz * 1e6),
                             "algorithmic_bytes_per_round": 48 * E + 24 * n,
                             "algorithmic_bytes_rule": "48 B per directed edge (A 8, sender 4, reverse index 4, "
                                                       "reverse message 16, new message 16) + 24 B per node",
                             "round_ms": p64["ms"]["fp64"] / max(p64["rounds"]["fp64"], 1),
                             "hbm_frac": (48 * E + 24 * n) / (p64["ms"]["fp64"] / max(p64["rounds"]["fp64"], 1)
                                                             / 1e3) / 1e9 / peak}},
            "fp64_edge_variant": edge,
            "errors_vs_oracle": errors,
            "grid32_fp64": c1,
            "lsq_rect_1048576x524288": lsq,
            f"dense_rbf_n{args.dense_n}": dense,
            "e2e": None if e2e_s is None else {
                "value": E * e2e_rounds / e2e_s, "unit": "edge-updates/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n, "ms_per_step": e2e_s / args.steps * 1e3},
            "clocks": clk,
            "wall_timed_s": wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if batched is not None:
            line["batched_grid3d_64rhs"] = batched
        if multi is not None:
            line[f"multi_rgg_{args.multi_systems}"] = multi
        if grad is not None:
            line["autograd_n4194304"] = grad
        if fix is not None:
            line["convergence_fix_n4096"] = fix
        print(json.dumps(line), flush=True)
    s32.close()
    s64.close()
    reps.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
