"""Benchmark: ANOVA fast-summation matvec throughput (Gpts/s) on the
precision form (N = 1e6, d = 28, nine windows: 3 x 3-D at n = 32, 4 x 2-D and
2 x 1-D at n = 64, m = 6, sigma = 2), plus KRR solves/s, p50/p99 step latency
and, as a secondary key, the same figures on the mid workload (N = 1e5, three
3-D windows) where the plain FP64 solve is timed beside the mixed one.

A step is one full ANOVA matvec K alpha (all windows: spread, FFT, multiply,
inverse FFT, gather, weighted window sum) in FP32 through the C ABI, inputs
resident in HBM.  L2 is flushed before every step (256 MB write outside the
per-step events).  With --gpus N (torchrun) every rank runs an independent
replica (the path has no exchange step); value = points of all ranks / max
time over ranks.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method used for parity) on the same workload on the host cores, rank 0 only:
every step is the oracle's fast summation of a bounded slice of the
workload's points.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ANOVA fastsum matvec Gpts/s & KRR solves/s at rel err 1e-5; p50/p99 latency"
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.md")
CSRC = os.path.join(ROOT, "paper_2111_10140_gb300", "csrc")


def fp32_peak_tflops():
    return 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def tf32_peak_tflops():
    pk, _ = measured_peaks()
    return float(pk["bf16_tflops"]) * (1.1 / 2.25)


def source_sha(files):
    """sha256 (first 16 hex digits) of the concatenated sources a kernel is built from."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch(kernel, workload, path=None):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu summary, or None when there is none or when the kernel's
    sources have changed since the counters were taken.  Rows of the table in
    profiles/dram_traffic.md: | kernel | workload | bytes per launch | sources | sha |"""
    try:
        with open(path or TRAFFIC_FILE) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    for ln in lines:
        cells = [c.strip().strip("`") for c in ln.strip().strip("|").split("|")]
        if len(cells) < 5 or cells[0] != kernel or cells[1] != workload:
            continue
        try:
            nbytes = int(cells[2].replace(",", ""))
            files = [x.strip() for x in cells[3].split("+")]
            if source_sha(files) != cells[4]:
                return None
        except (ValueError, OSError):
            return None
        return nbytes
    return None


def max_over_ranks(ms, ws, device=None):
    """The largest per-rank time (all_reduce MAX over the process group); ms itself at ws == 1."""
    if ws == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gpts(n_per_rank, ws, steps, total_ms):
    """Whole-job throughput of ws replicas, each processing n_per_rank points per step."""
    return ws * n_per_rank * steps / (total_ms * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(w):
    """The `config` object of both arms: the workload by its sizes (no plan choices)."""
    dims = [len(x) for x in w.windows]
    desc = "+".join(f"{dims.count(k)}x{k}D" for k in (3, 2, 1) if dims.count(k))
    return {"workload": w.name, "N": w.N, "d": w.d, "windows": desc,
            "n": sorted(set(w.n), reverse=True), "m": w.m, "sigma": w.sigma, "eps_B": w.epsB, "ell": w.ell,
            "lambda": w.lam, "tol": w.tol}


def run_reference(args):
    """Time the FP64 CPU oracle's fast summation: every step is the oracle's
    fast summation of a slice of `--ref-sample` consecutive points of the
    benchmark workload (slices rotate through the N points)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2111_10140_gb300 import workloads as W
    oracle.build()
    w = W.precision_form()
    ns = min(args.ref_sample, w.N)
    cores = len(os.sched_getaffinity(0))
    times = []
    for it in range(args.warmup + args.steps):
        lo = (it * ns) % (w.N - ns + 1)
        Xs, alpha = w.X[lo:lo + ns], w.alpha[lo:lo + ns]
        t0 = time.perf_counter()
        oracle.fastsum(None, Xs, w.windows, w.eta, w.ell, w.n, w.m, alpha, sigma=w.sigma, epsB=w.epsB, p=w.p)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    value = ns / t / 1e9
    sample = (f"each step: the oracle's FP64 fast summation (OpenMP) of {ns} consecutive points of the "
              f"{w.N}-point workload (slices rotate), same windows, n, m, sigma, eps_B")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": "Gpts/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(ns, what="fastsum", data=None, workload=None):
    """One timed oracle run on a bounded sample: the fast summation of the
    first ns points of `workload` (default the precision form; about 10-30 s
    of CPU work), or with what="features" the window construction (z-score
    fit on all rows of `data` = (X, labels), MIS on the first ns rows)."""
    import oracle
    from paper_2111_10140_gb300 import workloads as W
    if what == "features":
        from oracle import features as F
        X, labels = data
        t0 = time.perf_counter()
        F.zscore_fit(X)
        t_fit = time.perf_counter() - t0
        t0 = time.perf_counter()
        F.mis(X[:ns], labels[:ns], int(labels.max()) + 1)
        t_mis = time.perf_counter() - t0
        return {"zscore_fit_s": t_fit, "mis_s": t_mis, "mis_rows": ns, "cores": 1, "kind": "oracle",
                "sample": f"numpy z-score fit on {X.shape[0]} x {X.shape[1]}; Python-loop MIS on the first {ns} rows"}
    oracle.build()
    w = workload if workload is not None else W.precision_form()
    ns = min(ns, w.N)
    t0 = time.perf_counter()
    oracle.fastsum(None, w.X[:ns], w.windows, w.eta, w.ell, w.n, w.m, w.alpha[:ns], sigma=w.sigma,
                   epsB=w.epsB, p=w.p)
    t = time.perf_counter() - t0
    return {"value": ns / t / 1e9, "unit": "Gpts/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"one oracle fast summation (FP64, OpenMP) of the first {ns} of the {w.N} points of "
                      f"{w.name}, same windows/n/m/sigma/eps_B; {t:.2f} s"}


STAGES = ["spread", "fft", "gather", "window_sum", "spread_3d_kernel", "gather_3d_kernel"]


def time_matvec(B, plan, alpha, out, flush, steps, warmup, stream, lead_in_s=0.0):
    """Per-step CUDA-event times of anova_matvec with an L2 flush before every step."""
    import torch
    for _ in range(warmup):
        flush.fill_(1.0)
        B.anova_matvec(plan, alpha, out)
    torch.cuda.synchronize()
    # keep the GPU busy before the timed region so that the 200 ms clock samples straddle it
    t_end = time.perf_counter() + lead_in_s
    while time.perf_counter() < t_end:
        for _ in range(20):
            B.anova_matvec(plan, alpha, out)
        torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        B.anova_matvec(plan, alpha, out)
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def stage_profile(B, plan, alpha, out, flush, steps):
    """Milliseconds and launches per stage over `steps` profiled matvecs (library events)."""
    import torch
    B.anova_set_profiling(plan, True)
    B.anova_stage_times(plan)   # reset
    for i in range(steps):
        flush.fill_(float(i))
        B.anova_matvec(plan, alpha, out)
    torch.cuda.synchronize()
    ms, la = B.anova_stage_times(plan)
    B.anova_set_profiling(plan, False)
    return dict(zip(STAGES, ms)), dict(zip(STAGES, la))


def dominant_roofline(B, plan, w, stage_ms, stage_la, steps):
    """Roofline of the slower of the 3-D spread and 3-D gather kernels (one launch
    each per matvec, covering every 3-D window), timed live by library events on
    the launch stream.  Algorithmic work: one FP32 multiply-add (2 flop) per tap
    (2m+1)^3, node and 3-D window."""
    P3 = sum(1 for x in w.windows if len(x) == 3)
    l3 = next(l for l, x in enumerate(w.windows) if len(x) == 3)
    R = B.anova_plan_window_bins(plan, l3)["region"]
    names = B.anova_dense3_kernels(plan)
    key = "spread_3d_kernel" if stage_ms["spread_3d_kernel"] >= stage_ms["gather_3d_kernel"] else "gather_3d_kernel"
    kernel = (names["spread"] if key == "spread_3d_kernel" else names["gather"]).replace("<R>", f"<{R}>")
    launches = max(1, stage_la[key])
    per_launch_ms = stage_ms[key] / launches
    units = w.N * P3 * steps / launches                      # node-windows per launch
    taps = (2 * w.m + 1) ** 3
    flops = 2.0 * taps * units
    achieved = flops / (per_launch_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    tc_flops = 3.0 * flops                                    # three tensor-core products per FP32 multiply-add
    f16 = "tch" in kernel                                     # FP16-split form: against the FP16 (= bf16) peak
    tc_peak = float(measured_peaks()[0]["bf16_tflops"]) if f16 else tf32_peak_tflops()
    _, src = measured_peaks()
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic_per_launch(kernel, w.name),
            "units_per_launch": units, "flop_per_unit": 2 * taps,
            "peak_source": f"derived FP32 FMA peak ({FP32_PEAK_NOTE}); algorithmic FP32 multiply-adds "
                           f"(executed on tcgen05 / mma.sync tensor cores as 3xTF32)",
            "tensor_view": {"achieved": tc_flops / (per_launch_ms * 1e-3) / 1e12, "peak": tc_peak,
                            "frac": tc_flops / (per_launch_ms * 1e-3) / 1e12 / tc_peak,
                            "what": "the FP32-accurate contraction as 3 " + ("FP16" if f16 else "TF32") +
                                    " products per multiply-add, unpadded",
                            "peak_source": f"{src} bf16 burst (MEASURED_PEAKS.json)" +
                                           ("" if f16 else " x nominal tf32/bf16 ratio 1.1/2.25")},
            "per_launch_ms": per_launch_ms,
            "stage_ms_per_step": {k: v / steps for k, v in stage_ms.items()}}


_DIRECT = {}


def accuracy_vs_direct(B, torch, np, X, w, out, rows_n, seed, dev):
    """Relative 2-norm error of the FP32 product against the FP64 direct sum on sampled rows
    (the direct sums are computed once per workload, rows and seed)."""
    rows = torch.from_numpy(np.sort(np.random.default_rng(seed).choice(w.N, rows_n, replace=False))).to(dev)
    key = (w.name, rows_n, seed)
    if key not in _DIRECT:
        dref = torch.empty(rows_n, dtype=torch.float64, device=dev)
        B.anova_direct_matvec(X[rows].contiguous(), X, w.windows, w.ell, torch.from_numpy(w.alpha).to(dev), dref,
                              dtype=B.FP64)
        _DIRECT[key] = dref
    dref = _DIRECT[key]
    torch.cuda.synchronize()
    err = (torch.linalg.norm(out.double()[rows] - dref) / torch.linalg.norm(dref)).item()
    return {"rel_err_vs_direct": err, "sample_rows": rows_n, "direct": "anova_direct_matvec FP64",
            "target": 1e-5, "meets_target": bool(err <= 1e-5)}


def krr_solve(B, torch, plan, w, dev, maxit, what):
    y = torch.from_numpy(w.y).to(dev)
    sol = torch.zeros_like(y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, its, rel = B.krr_cg_solve(plan, w.lam, y, sol, w.tol, maxit)
    t = time.perf_counter() - t0
    return {"solves_per_s": 1.0 / t, "seconds": t, "iterations": int(its[0]), "relres": float(rel[0]),
            "status": int(st), "converged": bool(st == B.OK and rel[0] <= w.tol), "precision": what,
            "tol": w.tol, "lambda": w.lam}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    from paper_2111_10140_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:   # one builder; the other ranks load its library after the barrier
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()

    # the CPU baseline runs before any kernel work (rank 0, N = 1 only)
    cpu = cpu_baseline(args.cpu_sample) if (rank == 0 and ws == 1 and not args.skip_cpu) else None

    w = W.precision_form(N=args.points, seed=2 + rank)
    N = w.N
    X = torch.from_numpy(w.X).to(dev)
    # bin sides per window dimension from the library's autotuner (outside any timed region)
    if args.bin_side:
        sides = [int(v) for v in args.bin_side.split(",")]
    elif not args.no_autotune:
        sides, _ = B.anova_autotune_bins(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                         precision=B.FP32, reps=5)
    else:
        sides = [0, 0, 0]
    torch.cuda.synchronize()
    t_plan = time.perf_counter()
    plan = B.anova_fastsum_plan_bins(X, w.windows, w.ell, sides, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                     precision=B.MIXED)
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t_plan) * 1e3
    # kernel forms (3-D spread, 3-D gather, 1-D / 2-D schedule): given, or from the library's tuner
    # when the bin sides are tuned too
    if args.forms:
        f = [int(v) for v in args.forms.split(",")]
        B.anova_plan_set_kernels(plan, B.SPREAD3_FORMS[f[0]], B.GATHER3_FORMS[f[1]], f[2])
        kernels, kernels_how = B.anova_plan_get_kernels(plan), "given"
    elif not args.bin_side and not args.no_autotune:
        try:
            kernels, _ = B.anova_autotune_kernels(plan, reps=5)
            kernels_how = "autotuned"
        except B.AnovaError as e:   # the plan keeps its forms; the headline still runs
            kernels, kernels_how = B.anova_plan_get_kernels(plan), f"default (tuner failed: {e})"
    else:
        kernels, kernels_how = B.anova_plan_get_kernels(plan), "default"
    alpha = torch.from_numpy(w.alpha).to(dev).float()
    out = torch.empty_like(alpha)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.__enter__()
    step_ms = time_matvec(B, plan, alpha, out, flush, args.steps, args.warmup, stream, lead_in_s=0.6)
    if ws > 1:
        dist.barrier()
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    ms_per_step = total_ms / args.steps
    value = aggregate_gpts(N, ws, args.steps, total_ms)

    # stage breakdown and the dominant kernel from a second, profiled pass (events between the stages)
    stage_ms, stage_la = stage_profile(B, plan, alpha, out, flush, args.steps)
    launches = int(sum(stage_la[k] for k in STAGES[:4]))
    roofline = dominant_roofline(B, plan, w, stage_ms, stage_la, args.steps)

    B.anova_matvec(plan, alpha, out)
    accuracy = accuracy_vs_direct(B, torch, np, X, w, out, args.check_rows, 7, dev)

    # the same product with the 3-D spread and gather on FP32 FMA kernels (no tensor cores), for comparison
    fsteps = max(5, args.steps // 2)
    B.anova_plan_set_tensor_cores(plan, False)
    fma_ms = time_matvec(B, plan, alpha, out, flush, fsteps, args.warmup, stream)
    fma_stage, _ = stage_profile(B, plan, alpha, out, flush, fsteps)
    fma_names = B.anova_dense3_kernels(plan)
    B.anova_matvec(plan, alpha, out)
    fma_acc = accuracy_vs_direct(B, torch, np, X, w, out, args.check_rows, 7, dev)
    B.anova_plan_set_kernels(plan, kernels["spread3"], kernels["gather3"], kernels["schedule"])
    no_tensor = {"ms_per_matvec": statistics.median(fma_ms), "gpts": N / statistics.median(fma_ms) / 1e6,
                 "spread_3d_kernel_ms": fma_stage["spread_3d_kernel"] / fsteps,
                 "gather_3d_kernel_ms": fma_stage["gather_3d_kernel"] / fsteps,
                 "kernels": fma_names, "rel_err_vs_direct": fma_acc["rel_err_vs_direct"],
                 "what": "3-D spread and gather on FP32 FMA kernels (anova_plan_set_tensor_cores off), same plan"}

    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    a_host = torch.from_numpy(w.alpha.astype(np.float32)).pin_memory()
    o_host = torch.empty(N, dtype=torch.float32).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        s_ev, e_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_ev.record(stream)
        alpha.copy_(a_host, non_blocking=True)
        B.anova_matvec(plan, alpha, out)
        o_host.copy_(out, non_blocking=True)
        e_ev.record(stream)
        e_ev.synchronize()
        if i >= args.warmup:
            e2e_ms.append(s_ev.elapsed_time(e_ev))
    e2e_value = aggregate_gpts(N, ws, args.steps, max_over_ranks(sum(e2e_ms), ws, dev))

    # KRR solves/s (mixed precision: FP32 inner CG, FP64 refinement) to the workload's tolerance
    krr = None if args.skip_krr else krr_solve(B, torch, plan, w, dev, 20000,
                                               "mixed (FP32 inner CG, FP64 refinement)")
    if krr is not None and not args.skip_fp64:
        # the FP64 product the refinement's residuals use (same plan, FP64 coefficients)
        a64 = torch.from_numpy(w.alpha).to(dev)
        o64 = torch.empty_like(a64)
        B.anova_matvec(plan, a64, o64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            B.anova_matvec(plan, a64, o64)
        e1.record(stream)
        e1.synchronize()
        krr["fp64_matvec_ms"] = e0.elapsed_time(e1) / 3
        krr["fp32_matvec_ms"] = ms_per_step
        del a64, o64
    clk.__exit__(None, None, None)
    plan.close()
    del X

    # secondary key: the mid workload, where the plain FP64 solve is timed beside the mixed one
    mid = None
    if not args.skip_mid:
        wm = W.plain_mid(seed=1 + rank)
        Xm = torch.from_numpy(wm.X).to(dev)
        sm, _ = B.anova_autotune_bins(Xm, wm.windows, wm.ell, n=wm.n, m=wm.m, sigma=wm.sigma, eps_B=wm.epsB,
                                      p=wm.p, precision=B.FP32, reps=5)
        pm = B.anova_fastsum_plan_bins(Xm, wm.windows, wm.ell, sm, n=wm.n, m=wm.m, sigma=wm.sigma, eps_B=wm.epsB,
                                       p=wm.p, precision=B.MIXED)
        try:
            mkern, _ = B.anova_autotune_kernels(pm, reps=5)
        except B.AnovaError as e:
            mkern = dict(B.anova_plan_get_kernels(pm), tuner_failed=str(e))
        am = torch.from_numpy(wm.alpha).to(dev).float()
        om = torch.empty_like(am)
        mid_ms = time_matvec(B, pm, am, om, flush, args.steps, args.warmup, stream)
        mst, mla = stage_profile(B, pm, am, om, flush, args.steps)
        mroof = dominant_roofline(B, pm, wm, mst, mla, args.steps)
        B.anova_matvec(pm, am, om)
        macc = accuracy_vs_direct(B, torch, np, Xm, wm, om, 2048, 7, dev)
        mkrr = None if args.skip_krr else krr_solve(B, torch, pm, wm, dev, 5000,
                                                    "mixed (FP32 inner CG, FP64 refinement)")
        pm.close()
        mkrr64 = None
        if not args.skip_krr and not args.skip_fp64:
            p64 = B.anova_fastsum_plan(Xm, wm.windows, wm.ell, n=wm.n, m=wm.m, sigma=wm.sigma, eps_B=wm.epsB,
                                       p=wm.p, precision=B.FP64)
            mkrr64 = krr_solve(B, torch, p64, wm, dev, 5000, "plain FP64 CG on the FP64 operator")
            a64 = torch.from_numpy(wm.alpha).to(dev)
            o64 = torch.empty_like(a64)
            B.anova_matvec(p64, a64, o64)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                B.anova_matvec(p64, a64, o64)
            e1.record(stream)
            e1.synchronize()
            mkrr64["fp64_matvec_ms"] = e0.elapsed_time(e1) / 5
            p64.close()
        mid = {"config": workload_config(wm), "bin_side_1d_2d_3d": sm, "kernels": mkern,
               "value": wm.N * len(mid_ms) / (sum(mid_ms) * 1e-3) / 1e9, "unit": "Gpts/s",
               "ms_per_step": sum(mid_ms) / len(mid_ms), "roofline": mroof, "accuracy": macc,
               "krr": mkrr, "krr_plain_fp64": mkrr64}
        del Xm

    # the other forms of the path on reduced configurations (rank 0 of a one-GPU run; outside the clocks window)
    forms = None
    if rank == 0 and ws == 1 and not args.skip_forms:
        del flush
        torch.cuda.empty_cache()
        forms = other_forms(args)

    q = sorted(step_ms)
    lat = {"p50": q[len(q) // 2], "p99": q[min(len(q) - 1, int(0.99 * len(q)))], "unit": "ms"}
    if rank == 0:
        cfg = workload_config(w)
        cfg.update({"precision": "fp32 operator (spread, FFT, gather); FP64 CG scalars and refinement",
                    "l2": "flushed before every step (256 MB write outside the step events)",
                    "parallelism": f"replicas x{ws}"})
        line = {"metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg,
                "plan": {"bin_side_1d_2d_3d": sides,
                         "bin_sides": "given" if args.bin_side else ("autotuned" if not args.no_autotune else "rule"),
                         "create_ms": plan_ms,
                         "kernels": kernels, "kernels_chosen": kernels_how,
                         "create_note": "anova_fastsum_plan_bins (frames, binning, D_k, FP32 weight tables, "
                                        "FP64 data), wall clock, outside the timed steps"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "Gpts/s", "h2d_bytes_per_step": 4 * N,
                        "d2h_bytes_per_step": 4 * N},
                "gpu_launches": launches, "latency_ms": lat, "accuracy": accuracy, "no_tensor_cores": no_tensor,
                "krr": krr,
                "plain_mid": mid,
                "forms": forms,
                "clocks": dict(clk.summary(), window="0.6 s busy lead-in, timed steps, profiled steps, e2e steps "
                                                     "and the KRR solve of the headline workload")}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def other_forms(args):
    """Window construction, serving and batching in the default run (the modes
    --features, --serve and --batch on their own print the same records):
    serving on its full configuration, window construction with fewer timed
    calls, batching on a configuration small enough for a few seconds.  Each
    entry is that mode's record plus `reduced`, which names what differs from
    the mode's full configuration (None: nothing)."""
    import copy
    out = {}

    def run(key, fn, a, reduced):
        # a failing form is reported in its entry; the headline line is printed regardless
        try:
            out[key] = dict(fn(a), reduced=reduced)
        except Exception as e:
            out[key] = {"error": f"{type(e).__name__}: {e}", "reduced": reduced}

    a = copy.copy(args)
    a.steps, a.warmup, a.features_cpu_rows = 10, 3, 2000
    run("window_construction", features_result, a, "10 timed calls each; CPU oracle on 2000 rows")
    run("serving", serve_result, copy.copy(args), None)
    a = copy.copy(args)
    a.batch_problems, a.batch_rhs, a.batch_sample, a.batch_lambda_min = 16, 4, 2, 1e-3
    run("batching", batch_result, a, "16 problems x 4 right-hand sides, lambda >= 1e-3, "
                                     "2 problems timed one at a time (full: 64 x 16, 1e-4, 8)")
    return out


def run_crossover(args):
    """Direct O(N^2 P) GPU sum vs the fast summation on the mid workload's shape."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    from paper_2111_10140_gb300 import workloads as W
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    for N in [1000, 3000, 10_000, 30_000, 100_000, 300_000, 1_000_000]:
        w = W.plain_mid(N=N)
        X = torch.from_numpy(w.X).to(dev)
        a64 = torch.from_numpy(w.alpha).to(dev)
        plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                    precision=B.FP32)
        a32, o32 = a64.float(), torch.empty(N, dtype=torch.float32, device=dev)
        od = torch.empty(N, dtype=torch.float64, device=dev)

        def timeit(fn, reps):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1) / reps

        t_fast = timeit(lambda: B.anova_matvec(plan, a32, o32), 20)
        reps = 3 if N <= 300_000 else 1
        t_dir = timeit(lambda: B.anova_direct_matvec(X, X, w.windows, w.ell, a64, od, dtype=B.FP32), reps)
        err = (torch.linalg.norm(o32.double() - od) / torch.linalg.norm(od)).item()
        print(json.dumps({"crossover": True, "N": N, "fast_ms": t_fast, "direct_fp32_ms": t_dir,
                          "speedup": t_dir / t_fast, "rel_diff": err}), flush=True)
        plan.close()


def run_serve(args):
    print(json.dumps(serve_result(args)), flush=True)


def serve_result(args):
    """Serving form: a Poisson stream of requests (mean `--serve-rate` per s),
    70 % predictions of M test points (log-uniform in [1e2, 1e5]) against a
    resident model (N log-uniform in [1e4, 1e6]) and 30 % fits of new problems
    (N log-uniform in [1e3, 1e6]), d 9..28, 3..9 windows, served by the
    library's request server under a 150 GB budget (FP32 bulk, FP64
    refinement to residual 1e-6).  Fits whose expected queue wait exceeds
    `--serve-fit-wait-ms` are refused at submission (counted).  Fitted stream
    models are released as soon as their fit is done.  Prints one line with
    latency percentiles per kind (fits also per half of the run) and the
    served throughput."""
    import threading
    import time

    import numpy as np
    import torch

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    from paper_2111_10140_gb300 import workloads as W
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    logu = lambda lo, hi: int(round(10 ** rng.uniform(np.log10(lo), np.log10(hi))))

    def to_dev(w):
        return (torch.from_numpy(w.X).to(dev), torch.from_numpy(w.y).to(dev))

    # resident models (fitted before the stream starts) with held-out test rows
    res_N = [logu(1e4, 1e6) for _ in range(args.serve_models)]
    res = [W.serving_problem(N, seed=1000 + k, M_test=100_000) for k, N in enumerate(res_N)]
    res_dev = [to_dev(w) + (torch.from_numpy(w.meta["Z"]).to(dev),) for w in res]
    fit_pool = [W.serving_problem(logu(1e3, 1e6), seed=2000 + k) for k in range(args.serve_fit_pool)]
    fit_dev = [to_dev(w) for w in fit_pool]
    torch.cuda.synchronize()
    sv = B.Server(n_workers=args.serve_workers, hbm_budget_bytes=150 << 30)
    stop = threading.Event()
    # the server's workers and the releaser stop on every exit path
    try:
        t0 = time.perf_counter()
        models = [sv.submit_fit(X, w.windows, w.ell, y, w.lam, n=w.n, m=w.m, eps_B=w.epsB, tol=w.tol)
                  for w, (X, y, _) in zip(res, res_dev)]
        init = [sv.wait(t) for t in models]
        t_init = time.perf_counter() - t0
        # fits whose expected queue wait exceeds the bound are refused at submission
        # (the rate estimate comes from the resident models' fits above)
        sv.set_fit_wait_bound(args.serve_fit_wait_ms)
        refused = 0
        # the stream
        n_req = int(args.serve_rate * args.serve_seconds)
        arrivals = np.cumsum(rng.exponential(1.0 / args.serve_rate, size=n_req))
        kinds = rng.uniform(size=n_req) < 1.0 - args.serve_fit_share
        fit_tickets, pred = [], []
        done_fits = []

        def releaser():
            k = 0
            while True:
                while k >= len(fit_tickets):
                    if stop.is_set() and k >= len(fit_tickets):
                        return
                    time.sleep(0.002)
                r = sv.wait(fit_tickets[k][0])
                done_fits.append((fit_tickets[k][1], r))
                if r["status"] in (B.OK, B.ENOCONV):
                    sv.release(fit_tickets[k][0])
                k += 1

        th = threading.Thread(target=releaser, daemon=True)
        th.start()
        outs = []
        rows = 0
        t0 = time.perf_counter()
        for i in range(n_req):
            now = time.perf_counter() - t0
            if arrivals[i] > now:
                time.sleep(arrivals[i] - now)
            if kinds[i]:
                k = int(rng.integers(len(res)))
                M = logu(1e2, 1e5)
                Zt = res_dev[k][2]
                off = int(rng.integers(0, Zt.shape[0] - M + 1))
                o = torch.empty(M, dtype=torch.float64, device=dev)
                outs.append(o)
                pred.append((sv.submit_predict(models[k], Zt[off:off + M], o), M))
                rows += M
            else:
                k = int(rng.integers(len(fit_pool)))
                w, (X, y) = fit_pool[k], fit_dev[k]
                try:
                    fit_tickets.append((sv.submit_fit(X, w.windows, w.ell, y, w.lam, n=w.n, m=w.m, eps_B=w.epsB,
                                                      tol=w.tol), w.N))
                except B.AnovaError as e:
                    if e.status != B.EBUSY:
                        raise
                    refused += 1
        t_sub = time.perf_counter() - t0
        plat = np.array([sv.wait(t)["latency_ms"] for t, _ in pred])
        stop.set()
        th.join()
        t_all = time.perf_counter() - t0
        flat = np.array([r["latency_ms"] for _, r in done_fits])
        half = len(flat) // 2
        fitted = sum(N for N, r in done_fits)
        bad = sum(r["status"] not in (B.OK, B.ENOCONV) for _, r in done_fits)
        pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
        return {
            "serve": True,
            "workload": "Poisson stream of predictions (M log-uniform 1e2..1e5) on resident models and "
                        "fits (N log-uniform 1e3..1e6; share fit_share); d 9..28, 3..9 windows of 1-3 features",
            "offered_rate_rps": args.serve_rate, "seconds_offered": args.serve_seconds, "workers": args.serve_workers,
            "resident_models_N": res_N, "initial_fits_s": round(t_init, 3),
            "initial_fit_iters": [r["iterations"] for r in init],
            "requests": n_req, "predicts": len(pred), "fits": len(done_fits), "failed_fits": int(bad),
            "fit_share": args.serve_fit_share,
            "predict_p50_ms": pct(plat, 50), "predict_p99_ms": pct(plat, 99),
            "predict_p50_ms_first_half": pct(plat[:len(plat) // 2], 50),
            "predict_p50_ms_second_half": pct(plat[len(plat) // 2:], 50),
            "fit_p50_ms": pct(flat, 50), "fit_p99_ms": pct(flat, 99),
            "fit_wait_bound_ms": args.serve_fit_wait_ms, "fits_refused": refused,
            "fit_p50_ms_first_half": pct(flat[:half], 50), "fit_p50_ms_second_half": pct(flat[half:], 50),
            "submit_s": round(t_sub, 3), "drain_s": round(t_all, 3),
            "achieved_rps": n_req / t_all, "predicted_rows_per_s": rows / t_all, "fitted_points_per_s": fitted / t_all,
        }
    finally:
        stop.set()
        sv.close()


def run_batch(args):
    print(json.dumps(batch_result(args)), flush=True)


def batch_result(args):
    """Batching form: 64 problems (N log-uniform in [2^10, 2^17], d 6..15, own
    windows of 1-3 features, ell in [0.05, 0.5], lambda in [1e-4, 1e-1]) with
    16 right-hand sides each.  Timed: (a) krr_batch_cg_solve (FP32 operator,
    FP64 CG vectors, graph replay) to a recursive residual of tol; (b)
    krr_batch_cg_solve_refined to an FP64 residual of tol; against the same
    systems one at a time through krr_cg_solve: FP32 plans for (a), and the
    plain FP64 path (FP64 plans) for (b), the single-system times taken on one
    right-hand side of the first `--batch-sample` problems and scaled to all
    systems by their share of the batch's node-window work."""
    import time

    import numpy as np
    import torch

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    from paper_2111_10140_gb300 import workloads as W
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    probs = W.batch_form(args.batch_problems, seed=3, nrhs=args.batch_rhs,
                         lam_range=(args.batch_lambda_min, 1e-1))
    t0 = time.perf_counter()
    Xs = [torch.from_numpy(w.X).to(dev) for w in probs]
    plans = [B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=B.MIXED)
             for X, w in zip(Xs, probs)]
    batch = B.Batch(plans, args.batch_rhs)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    y = torch.empty(batch.size, dtype=torch.float64, device=dev)
    for p, w in enumerate(probs):
        batch.block(y, p).copy_(torch.from_numpy(w.meta["Y"]))
    alpha = torch.empty_like(y)
    lams = [w.lam for w in probs]
    tol, maxit = args.batch_tol, args.batch_maxit

    def timed(fn):
        # one run: it includes the graph captures (a few per solve, milliseconds)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    (st32, its32, rr32), t32 = timed(lambda: batch.cg_solve(lams, y, alpha, tol, maxit))
    (st64, its64, rr64), t64 = timed(lambda: batch.cg_solve(lams, y, alpha, tol, maxit, refined=True))
    ns = len(probs) * args.batch_rhs
    # systems the refined solve leaves above tol, each with an upper bound on its
    # condition number: kappa(K + lambda I) <= (lambda_max(K) + lambda) / lambda,
    # lambda_max(K) by 30 power iterations of the problem's FP64 operator
    exceptions, lmax = [], {}
    for p, r in zip(*np.nonzero(rr64 > tol)):
        p, r = int(p), int(r)
        if p not in lmax:
            v = torch.from_numpy(np.random.default_rng(9).standard_normal(probs[p].N)).to(dev)
            kv = torch.empty_like(v)
            est = 0.0
            for _ in range(30):
                v /= torch.linalg.norm(v)
                B.anova_matvec(plans[p], v, kv)
                est = float(torch.linalg.norm(kv))
                v, kv = kv, v
            lmax[p] = est
        w = probs[p]
        exceptions.append({"problem": p, "rhs": r, "N": w.N, "windows": [len(x) for x in w.windows],
                           "ell": round(w.ell, 4), "lambda": w.lam, "relres_fp64": float(rr64[p, r]),
                           "iters": int(its64[p, r]), "kappa_upper": (lmax[p] + w.lam) / w.lam})
    work = np.array([w.N * len(w.windows) for w in probs], dtype=float)
    K = min(args.batch_sample, len(probs))
    share = work[:K].sum() / work.sum()
    single = {}
    for name, prec in (("fp32", B.FP32), ("fp64", B.FP64)):
        tt, it_s, rel_s = 0.0, [], []
        for p in range(K):
            w = probs[p]
            pl = B.anova_fastsum_plan(Xs[p], w.windows, w.ell, n=w.n, m=w.m, eps_B=w.epsB, precision=prec)
            y1 = torch.from_numpy(w.meta["Y"][0]).to(dev)
            a1 = torch.zeros_like(y1)
            B.krr_cg_solve(pl, w.lam, y1, a1, tol, maxit)    # warm
            torch.cuda.synchronize()
            s0 = time.perf_counter()
            _, it1, r1 = B.krr_cg_solve(pl, w.lam, y1, a1, tol, maxit)
            torch.cuda.synchronize()
            tt += time.perf_counter() - s0
            it_s.append(int(it1[0]))
            rel_s.append(float(r1[0]))
            pl.close()
        single[name] = {"sample_s": round(tt, 4), "est_all_systems_s": round(tt * args.batch_rhs / share, 3),
                        "iters": it_s, "relres_max": max(rel_s),
                        "converged": int(sum(r <= (10 if name == "fp32" else 1) * tol for r in rel_s))}
    res = {
        "batch": True,
        "workload": f"{len(probs)} problems, N log-uniform 2^10..2^17 (total {sum(w.N for w in probs)}), "
                    f"{args.batch_rhs} right-hand sides each, d 6..15, 1-5 windows of 1-3 features, "
                    f"lambda log-uniform {args.batch_lambda_min:g}..1e-1",
        "systems": ns, "tol": tol, "setup_s": round(t_setup, 3),
        "fp32_operator": {"status": int(st32), "solve_s": round(t32, 4), "systems_per_s": ns / t32,
                          "converged_fp32_residual": int((rr32 <= 10 * tol).sum()),
                          "iters_median": float(np.median(its32)), "iters_max": int(its32.max()),
                          "relres_fp32_median": float(np.median(rr32)), "relres_fp32_max": float(rr32.max()),
                          "speedup_vs_single_fp32": single["fp32"]["est_all_systems_s"] / t32},
        "fp64_refined": {"status": int(st64), "solve_s": round(t64, 4), "systems_per_s": ns / t64,
                         "iters_median": float(np.median(its64)), "relres_fp64_max": float(rr64.max()),
                         "converged": int((rr64 <= tol).sum()),
                         "speedup_vs_single_fp64": single["fp64"]["est_all_systems_s"] / t64,
                         # both at an FP64 residual <= tol: systems brought to tol per second
                         "converged_per_s": float((rr64 <= tol).sum()) / t64,
                         "single_fp64_converged_per_s": single["fp64"]["converged"] / single["fp64"]["sample_s"],
                         "exceptions": exceptions},
        "single_sample_problems": K, "single_sample_work_share": round(float(share), 4),
        "single": single,
    }
    batch.close()
    for pl in plans:
        pl.close()
    return res


def run_precision(args):
    """Precision form (N = 1e6, d = 28, nine windows of 1-3 features): FP32 and
    FP64 products, the mixed-precision KRR solve to 1e-8 against the FP64
    operator, and the FP32 product's error against the FP64 direct sum on a
    10 000-row subsample."""
    import time

    import numpy as np
    import torch

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    from paper_2111_10140_gb300 import workloads as W
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    w = W.precision_form()
    X = torch.from_numpy(w.X).to(dev)
    sides, _ = B.anova_autotune_bins(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                     precision=B.FP32, reps=10)
    plan = B.anova_fastsum_plan_bins(X, w.windows, w.ell, sides, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                     precision=B.MIXED)
    a64 = torch.from_numpy(w.alpha).to(dev)
    a32 = a64.float()
    o64, o32 = torch.empty_like(a64), torch.empty_like(a32)

    def timeit(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    t32 = timeit(lambda: B.anova_matvec(plan, a32, o32), 20)
    t64 = timeit(lambda: B.anova_matvec(plan, a64, o64), 3)
    B.anova_set_profiling(plan, True)
    B.anova_matvec(plan, a32, o32)
    torch.cuda.synchronize()
    stages = B.anova_stage_times(plan)[0]
    B.anova_set_profiling(plan, False)
    rows = torch.from_numpy(np.sort(np.random.default_rng(3).choice(w.N, 10_000, replace=False))).to(dev)
    dref = torch.empty(rows.numel(), dtype=torch.float64, device=dev)
    B.anova_direct_matvec(X[rows].contiguous(), X, w.windows, w.ell, a64, dref)
    B.anova_matvec(plan, a32, o32)
    B.anova_matvec(plan, a64, o64)
    torch.cuda.synchronize()
    err32 = (torch.linalg.norm(o32.double()[rows] - dref) / torch.linalg.norm(dref)).item()
    err64 = (torch.linalg.norm(o64[rows] - dref) / torch.linalg.norm(dref)).item()
    y = torch.from_numpy(w.y).to(dev)
    alpha = torch.zeros_like(y)
    torch.cuda.synchronize()
    s0 = time.perf_counter()
    st, its, rr = B.krr_cg_solve(plan, w.lam, y, alpha, w.tol, 20000)
    torch.cuda.synchronize()
    t_krr = time.perf_counter() - s0
    print(json.dumps({
        "precision_form": True, "workload": w.name, "N": w.N, "windows": [len(x) for x in w.windows],
        "bin_side_1d_2d_3d": sides, "fp32_matvec_ms": t32, "fp64_matvec_ms": t64,
        "fp32_stage_ms": dict(zip(["spread", "fft", "gather", "window_sum"], [round(x, 4) for x in stages])),
        "rel_err_vs_direct_10k": {"fp32": err32, "fp64": err64},
        "krr_mixed": {"status": int(st), "seconds": round(t_krr, 3), "iterations": int(its[0]),
                      "relres_fp64": float(rr[0]), "tol": w.tol, "lambda": w.lam}}), flush=True)
    plan.close()


def run_features(args):
    print(json.dumps(features_result(args)), flush=True)


def features_result(args):
    """Window construction on the GPU at the precision form's shape (N rows,
    d = 28, six Student-t columns, columns on their own scales, two classes):
    z-score fit, z-score apply (in place) and the MIS scores, each call timed
    with CUDA events after an L2 flush; the kernels are HBM-bound, so the
    figure is algorithmic bytes (one read of X, plus one write for apply, plus
    the labels for MIS) / time against the measured copy bandwidth."""
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    N, d = args.features_n, 28
    rng = np.random.default_rng(2)
    Xh = rng.standard_normal((N, d))
    for c in (0, 4, 8, 10, 13, 17):
        Xh[:, c] = rng.standard_t(3.0, N)
    Xh = Xh * rng.uniform(0.5, 3.0, d) + rng.uniform(-2.0, 2.0, d)
    lab = ((Xh[:, 0] + 0.5 * Xh[:, 3] - Xh[:, 7]) > 0).astype(np.int32)
    cpu = None if args.skip_cpu else cpu_baseline(args.features_cpu_rows, "features", (Xh, lab))
    X = torch.from_numpy(Xh).to(dev)
    labels = torch.from_numpy(lab).to(dev)
    Xw = torch.empty_like(X)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    mean, sd = B.anova_zscore_fit(X)

    def timed(fn, before=None):
        ts = []
        for i in range(args.warmup + args.steps):
            if before is not None:
                before()
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    t_fit = timed(lambda: B.anova_zscore_fit(X))
    t_apply = timed(lambda: B.anova_zscore_apply(Xw, mean, sd), before=lambda: Xw.copy_(X))
    scores = []
    t_mis = timed(lambda: scores.append(B.anova_mis(X, labels, 2)))
    windows = B.anova_windows_from_mis(scores[-1], 0.0)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm, src = float(json.load(f)["hbm_gbs"]), "measured copy (MEASURED_PEAKS.json)"
    except Exception:
        hbm, src = 6800.0, "fallback figure"
    xb = N * d * 8

    def row(ms, nbytes):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"ms": ms, "algorithmic_bytes": nbytes, "GB/s": gbs, "frac_of_hbm": gbs / hbm}

    return {"features": True, "N": N, "d": d, "hbm_peak_gbs": hbm, "peak_source": src,
            "zscore_fit": row(t_fit, xb), "zscore_apply": row(t_apply, 2 * xb),
            "mis": dict(row(t_mis, xb + 4 * N), note="synchronous call: includes the host's score formation"),
            "top_windows": windows[:3], "cpu_baseline": cpu, "steps": args.steps, "warmup": args.warmup,
            "l2": "flushed before every call (256 MB write outside the events)"}


def run_autotune(args):
    """Bin sides chosen by anova_autotune_bins for the mid workload and the
    precision form, against the default rule."""
    import torch

    import __graft_entry__
    from paper_2111_10140_gb300 import binding as B
    from paper_2111_10140_gb300 import workloads as W
    __graft_entry__.build()
    for w in (W.plain_mid(), W.precision_form()):
        X = torch.from_numpy(w.X).cuda()
        sides, ms = B.anova_autotune_bins(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                          precision=B.FP32, reps=20)
        d_sides, d_ms = None, None
        plan = B.anova_fastsum_plan(X, w.windows, w.ell, n=w.n, m=w.m, sigma=w.sigma, eps_B=w.epsB, p=w.p,
                                    precision=B.FP32)
        d_sides = sorted({(len(win), B.anova_plan_window_bins(plan, l)["bin_side"]) for l, win in enumerate(w.windows)})
        plan.close()
        print(json.dumps({"autotune": True, "workload": w.name, "chosen_bin_side_1d_2d_3d": sides,
                          "ms_per_fp32_matvec": ms, "default_rule_sides": d_sides}), flush=True)
        del X
        torch.cuda.empty_cache()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=100_000)
    ap.add_argument("--ref-sample", type=int, default=40_000)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-krr", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--check-rows", type=int, default=10_000)
    ap.add_argument("--skip-mid", action="store_true", help="no secondary mid-workload figures")
    ap.add_argument("--skip-forms", action="store_true",
                    help="no reduced window-construction, serving and batching runs after the headline")
    ap.add_argument("--points", type=int, default=1_000_000,
                    help="points of the headline workload (1e6 = the precision form; smaller only for profiler "
                         "captures of the same kernels)")
    ap.add_argument("--no-autotune", action="store_true", help="bin sides from the default rule")
    ap.add_argument("--bin-side", default="", help="bin sides for 1-D,2-D,3-D windows (e.g. 0,0,4), no autotuning")
    ap.add_argument("--forms", default="",
                    help="kernel forms 'spread3,gather3,schedule' as anova_autotune_kernels codes (e.g. 3,3,2), "
                         "no kernel tuning")
    ap.add_argument("--crossover", action="store_true",
                    help="direct vs fast matvec time over N (the paper's Fig. 1 on synthetic data); prints one line per N")
    ap.add_argument("--serve", action="store_true",
                    help="Poisson stream of prediction (and fit) requests through the request server")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-models", type=int, default=4)
    ap.add_argument("--serve-fit-pool", type=int, default=6)
    ap.add_argument("--serve-fit-share", type=float, default=0.3, help="share of the requests that are fits")
    ap.add_argument("--serve-fit-wait-ms", type=float, default=5000.0,
                    help="refuse fits whose expected queue wait exceeds this (0: admit every fit)")
    ap.add_argument("--precision-form", action="store_true",
                    help="precision form (N = 1e6, nine windows): products, mixed KRR to 1e-8, error vs direct")
    ap.add_argument("--autotune", action="store_true", help="bin sides chosen by the autotuner (mid, precision form)")
    ap.add_argument("--batch", action="store_true",
                    help="batching form: many problems x right-hand sides in one batched CG")
    ap.add_argument("--batch-problems", type=int, default=64)
    ap.add_argument("--batch-rhs", type=int, default=16)
    ap.add_argument("--batch-tol", type=float, default=1e-6)
    ap.add_argument("--batch-maxit", type=int, default=3000)
    ap.add_argument("--batch-sample", type=int, default=8)
    ap.add_argument("--batch-lambda-min", type=float, default=1e-4)
    ap.add_argument("--features", action="store_true",
                    help="window construction (z-score fit / apply, MIS) at the precision form's shape")
    ap.add_argument("--features-n", type=int, default=1_000_000)
    ap.add_argument("--features-cpu-rows", type=int, default=20_000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.crossover:
        run_crossover(args)
    elif args.serve:
        run_serve(args)
    elif args.batch:
        run_batch(args)
    elif args.autotune:
        run_autotune(args)
    elif args.precision_form:
        run_precision(args)
    elif args.features:
        run_features(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
