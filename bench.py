#!/usr/bin/env python
"""Benchmark of the FGFRFT online hot path on GB300.

Workload (the image-graph batch): 32x32 4-connected grid graph (N = 1024),
Laplacian GFT F, truncation L = 32, 64 transform orders uniform in [-2, 2], each
applied to 256 smooth Gaussian-random-field signals (length scale 4 px) plus
N(0, 0.1^2) noise -- 16384 signals per step, synthetic and seeded.

One step = the whole online path for that batch through the C ABI
(fgfrft_apply on 16384 columns in 64 runs of equal order): per-order
coefficients, one fused pass over the stored powers that assembles all 64
operators (split-fp16), the signal split, and one tcgen05 GEMM over the 64
groups.  The signals are real, so they are passed as real float32 arrays
(FGFRFT_REAL_SIGNALS; real float32 outputs too when every Q is real); the same
step on complex64 buffers is reported beside it.  The offline precompute (FP64
powers and projector) is not timed (the paper times only the online phase).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the same workload (a bounded sample of orders per step) instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "order-updates/s, signals/s, p99 latency vs plain FGFRFT on GB300 @ rel err≤1e-5"
UNIT = "order-updates/s"
WORKLOAD = "image-graph batch: 32x32 grid graph N=1024, L=32, 64 orders x 256 GRF signals"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="image-graph",
                    choices=["image-graph", "point-cloud", "precision", "serving", "stacked"],
                    help="image-graph is the headline line; the others report the remaining configs")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--serving-scale", default="full", choices=["full", "small"])
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[0.3, 0.6, 0.9, 1.2, 2.0, 4.0],
                    help="arrival rates as fractions of the measured sequential capacity")
    ap.add_argument("--no-target", action="store_true",
                    help="skip the N=4096, L=64 leg (single-order assembly, stacked GEMM) of the default run")
    ap.add_argument("--no-serving", action="store_true", help="skip the small serving sweep of the default run")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def reduce_max(x: float, device="cuda") -> float:
    """Maximum of x over all ranks (x itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_max_s: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / t_max_s


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper part of the clock distribution is the loaded region
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_traffic(kernel: str, workload_key: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(path))[f"{kernel}@{workload_key}"]
    except Exception:
        return None
    src = os.path.join(ROOT, "paper_2602_20870_gb300", "csrc", rec["source"])
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except Exception:
        return None
    return rec["bytes_per_launch"] if sha == rec.get("source_sha256_16") else None


def workload():
    from paper_2602_20870_gb300 import workloads as W
    return W.image_graph()


# ----------------------------------------------------------------------------- CPU oracle
class OracleOnline:
    """The FP64 oracle's online step (Algorithm 1 with stored powers, then Q X per order)
    on the host cores.  Offline work (spectral projector, powers) is done once here and
    excluded from the timings, as in the paper's timings."""

    def __init__(self, wl):
        from oracle import fgfrft_oracle as O
        self.O = O
        self.wl = wl
        self.sp = O.spectral(wl.F)
        self.P = O.projector(wl.F, self.sp)
        self.M = O.powers(wl.F, wl.L, self.P)

    def run(self, seconds: float, max_orders: int | None = None, start: int = 0, Y_gpu=None):
        wl, O = self.wl, self.O
        orders = wl.meta["orders"]
        per = wl.meta["per_order"]
        done, t0 = 0, time.perf_counter()
        errs = []
        for g in range(start, start + len(orders)):
            g %= len(orders)
            if max_orders is not None and done >= max_orders:
                break
            Xg = wl.X[g * per:(g + 1) * per].T
            Q = O.fgfrft_power(wl.F, float(orders[g]), wl.L, self.P, self.M)
            Yg = Q @ Xg
            done += 1
            if Y_gpu is not None and len(errs) < 4:
                errs.append((np.linalg.norm(Y_gpu[g * per:(g + 1) * per] - Yg.T), np.linalg.norm(Yg)))
            if time.perf_counter() - t0 > seconds:
                break
        el = time.perf_counter() - t0
        err = None
        if errs:
            err = math.sqrt(sum(e * e for e, _ in errs)) / math.sqrt(sum(n * n for _, n in errs))
        return done, el, err


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    wl = workload()
    per = wl.meta["per_order"]
    n_orders = len(wl.meta["orders"])
    # each step: a bounded sample of 2 orders (x 256 signals) of the workload
    sample = 2
    ora = OracleOnline(wl)
    for k in range(args.warmup):
        ora.run(1e9, max_orders=sample, start=sample * k)
    times, step_s = [], []
    for k in range(args.steps):
        done, el, _ = ora.run(1e9, max_orders=sample, start=sample * (k + args.warmup))
        times.append(el / done)
        step_s.append(el)
    per_order = statistics.mean(times)
    value = 1.0 / per_order
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # a step of this arm is the bounded sample (2 orders x 256 signals): its measured time
        "ms_per_step": statistics.mean(step_s) * 1e3,
        "ms_per_full_batch_extrapolated": per_order * n_orders * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 1024, "L": 32, "orders": n_orders, "signals_per_order": per,
                   "sample_per_step": f"{sample} orders x {per} signals"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{sample} orders x {per} signals per step, FP64 numpy/scipy"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2602_20870_gb300 import build as BUILD
    BUILD.build()
    from paper_2602_20870_gb300 import fgfrft as FG

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    wl = workload()
    N, L = wl.N, wl.L
    n_orders = len(wl.meta["orders"])
    B = wl.B
    plan = FG.Plan(wl.F, L)  # offline (untimed): FP64 powers and projector on this GPU
    alpha = np.ascontiguousarray(wl.alpha)
    X = torch.as_tensor(wl.X, dtype=torch.complex64).cuda()
    Y = torch.empty_like(X)
    stream = torch.cuda.current_stream()
    # The signals are real (GRF fields): they are kept as real float32 and the library's
    # real-signal interface reads them (and writes real outputs when Q is real).  The same
    # step on complex64 buffers is timed below for comparison.
    real_x = not bool(np.any(wl.X.imag))
    real_q = plan.real and plan.r_neg1 == 0  # every assembled Q_g is real
    real_out = real_x and real_q
    if real_x:
        Xr = torch.as_tensor(wl.X.real, dtype=torch.float32).cuda()
        Yr = torch.empty(Xr.shape, dtype=torch.float32 if real_out else torch.complex64, device=Xr.device)

    def step(path="auto", complex_io=False):
        if real_x and not complex_io and path != "plain":
            plan.apply(alpha, Xr, L, path=path, out=Yr, real_io=True, real_output=real_out)
        else:
            plan.apply(alpha, X, L, path=path, out=Y)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K device-resident steps through the public call as a user runs them
    # (one CUDA event between steps, for the per-step latencies), then the same K steps with
    # the library's per-kernel CUDA events, which give the per-kernel durations of the
    # rooflines; those events add small gaps between launches, so that pass is reported beside
    # the value, not as it
    clocks = ClockSampler(local)
    clocks.start()
    # the sampler's first readings come while the GPU keeps running untimed steps (an idle
    # GPU would lower its clocks and slow the first timed step)
    t_busy, n_busy = time.perf_counter() + 0.3, 0
    while time.perf_counter() < t_busy:
        step()
        n_busy += 1
        if n_busy % 32 == 0:  # the host does not run far ahead of the device
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    FG.timing_reset()  # the launch counters count with or without the per-kernel events
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = sum(v[0] for v in FG.timing_read().values())
    per_step = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_max = reduce_max(ev[0].elapsed_time(ev[-1]))
    ms_step = t_max / args.steps
    value = whole_job_rate(n_orders * args.steps, ws, t_max / 1e3)
    # the instrumented pass: every launch of the step between two CUDA events on its stream
    FG.timing_reset()
    FG.timing_enable(True)
    e0k, e1k = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0k.record(stream)
    for _ in range(args.steps):
        step()
    e1k.record(stream)
    torch.cuda.synchronize()
    barrier()
    FG.timing_enable(False)
    kt = FG.timing_read()
    clk = clocks.stop()
    total_ms = e0k.elapsed_time(e1k)
    ms_step_ev = reduce_max(total_ms) / args.steps
    # the same step on complex64 device buffers
    for _ in range(3):
        step(complex_io=True)
    torch.cuda.synchronize()
    e0c, e1c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0c.record(stream)
    for _ in range(args.steps):
        step(complex_io=True)
    e1c.record(stream)
    torch.cuda.synchronize()
    ms_step_c = reduce_max(e0c.elapsed_time(e1c)) / args.steps
    if real_x:
        Y.copy_(Yr)  # the result checked against the oracle: the real-signal step's output

    # ---- dominant kernel and its roofline (live CUDA events around each launch)
    peaks, peak_src = measured_peaks()
    rooflines = {}
    if kt["tc_gemm"][1]:
        avg_ms = kt["tc_gemm"][2] / kt["tc_gemm"][1]
        # Q_g X_g over the groups: flops per (i, j, k) = 8 complex x complex, 4 real x complex,
        # 2 real x real
        flops = (2.0 if real_q and real_x else 4.0 if (real_q or real_x) else 8.0) * N * N * B
        # bytes: split Q planes read + split X planes read + Y written (real float32 outputs
        # when both are real)
        byts = ((4.0 if real_q else 8.0) * n_orders * N * N + (4.0 if real_x else 8.0) * B * N +
                (4.0 if real_out else 8.0) * B * N)
        tpeak = peaks.get("bf16_tflops_sustained", 1700.0)  # fp16 dense tensor rate = bf16
        hpeak = peaks.get("hbm_gbs", 6800.0)
        tflops = flops / (avg_ms * 1e-3) / 1e12
        gbs = byts / (avg_ms * 1e-3) / 1e9
        # the roof that bounds it: the executed tensor work (3 split products) per byte against
        # the ridge point of the two peaks
        hbm_bound = 3 * flops / byts < tpeak * 1e12 / (hpeak * 1e9)
        rooflines["tc_gemm"] = {
            "bound": "hbm" if hbm_bound else "tensor", "kernel": "tc_gemm_kernel",
            "achieved": gbs if hbm_bound else tflops, "peak": hpeak if hbm_bound else tpeak,
            "unit": "GB/s" if hbm_bound else "TFLOP/s",
            "frac": gbs / hpeak if hbm_bound else tflops / tpeak,
            "real_operators": real_q, "real_signals": real_x,
            "peak_source": f"{peak_src} hbm_gbs" if hbm_bound else
                           f"{peak_src} bf16_tflops_sustained (fp16 dense rate equals bf16)",
            "algorithmic_per_launch": byts if hbm_bound else flops,
            "algorithmic_flops_per_launch": flops, "executed_tensor_flops_per_launch": 3 * flops,
            "bytes_per_launch": byts, "avg_launch_ms": avg_ms,
            "tflops": tflops, "tensor_frac": tflops / tpeak, "hbm_gbs": gbs, "hbm_frac": gbs / hpeak}
    if kt["assemble_multi"][1]:
        avg_ms = kt["assemble_multi"][2] / kt["assemble_multi"][1]
        # stack read once + operators written.  The pair stack (real F without a -1 eigenvalue)
        # holds 2 L_max real split values (4 bytes) per entry pair of the block-upper region,
        # N (N + 128) / 2 rows; the full entry-major copy 2L + 2 blocks per entry (8 bytes, 4 for
        # real F)
        if plan.pair:
            stack_b = 4.0 * 2 * plan.L_max * N * (N + 128) / 2
        else:
            stack_b = (4.0 if plan.real else 8.0) * (2 * L + 2) * N * N
        byts = stack_b + (4.0 if real_q else 8.0) * n_orders * N * N
        peak = peaks.get("hbm_gbs", 6800.0)
        achieved = byts / (avg_ms * 1e-3) / 1e9
        # the signal split runs beside it on an auxiliary stream, inside the same interval:
        # signals read (4 or 8 bytes per entry) + split planes written (2 or 4 fp16 planes)
        split_b = (4.0 if real_x else 8.0) * B * N + (4.0 if real_x else 8.0) * B * plan.N
        rooflines["assemble_multi"] = {
            "bound": "hbm", "kernel": "tc_gemm_kernel (fused multi-order assembly)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs",
            "algorithmic_per_launch": byts, "avg_launch_ms": avg_ms,
            "pair_stack": bool(plan.pair),
            "window_with_signal_split": {
                "bytes": byts + split_b, "gbs": (byts + split_b) / (avg_ms * 1e-3) / 1e9,
                "frac": (byts + split_b) / (avg_ms * 1e-3) / 1e9 / peak,
                "note": "the split's traffic moves inside the assembly's interval on an auxiliary stream"}}
    dom = max(rooflines, key=lambda k: kt[k][2])
    roof = dict(rooflines[dom])
    for r in rooflines.values():
        r["traffic"] = kernel_traffic(r["kernel"], "image-graph")
    roof["traffic"] = rooflines[dom]["traffic"]
    kernels = {k: {"launches": v[0], "ms_total": v[2], "share": v[2] / max(total_ms, 1e-9)} for k, v in kt.items()
               if v[0]}

    # ---- plain per-order FP32 path (the comparison path), same workload
    k_plain = max(3, args.steps // 4)
    for _ in range(2):
        step("plain")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    FG.timing_reset()
    FG.timing_enable(True)
    e0.record(stream)
    for _ in range(k_plain):
        step("plain")
    e1.record(stream)
    torch.cuda.synchronize()
    FG.timing_enable(False)
    kt_plain = FG.timing_read()
    plain_ms = e0.elapsed_time(e1) / k_plain
    # single-order assembly (K1) inside the plain path: the paper's online update
    n1, t1, ms1 = kt_plain["assemble_single"]
    # 2L+1 powers + P read (8 bytes per entry, 4 for real F from the real split planes), Q written
    k1_bytes = (4.0 if plan.real else 8.0) * (2 * L + 2) * N * N + 8.0 * N * N
    k1_gbs = k1_bytes / (ms1 / max(t1, 1) * 1e-3) / 1e9 if t1 else None

    # ---- end to end through the public API from pinned host buffers: every step copies its
    # signals to the device and its result back; FG.Pipeline overlaps the copies of one
    # step with the transform of the next (three streams, double-buffered device tensors)
    Xh = torch.as_tensor(wl.X, dtype=torch.complex64).pin_memory()
    Yh = torch.empty(Xh.shape, dtype=Xh.dtype).pin_memory()
    pipe = FG.Pipeline(plan, tuple(Xh.shape), L)
    for _ in range(3):
        pipe.submit(alpha, Xh, Yh)
    pipe.wait()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pipe.submit(alpha, Xh, Yh)
    pipe.wait()
    e2e_s = reduce_max(time.perf_counter() - t0)
    e2e_value = whole_job_rate(n_orders * args.steps, ws, e2e_s)
    # the same, one synchronous call per step (no overlap between steps)
    k_serial = max(3, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(k_serial):
        plan.apply(alpha, Xh, L, out=Yh)
        torch.cuda.synchronize()
    e2e_serial = n_orders * k_serial / (time.perf_counter() - t0)
    nbytes = X.numel() * 8
    e2e_complex = {"value": e2e_value, "serial_value": e2e_serial, "h2d_bytes_per_step": nbytes,
                   "d2h_bytes_per_step": nbytes}
    # the signals are real: the same calls with real float32 host buffers (and real outputs
    # when Q is real), half the bytes over the host link
    e2e_mode = "pipelined (copies of step k+1 / k-1 overlap the transform of step k), complex64 host buffers"
    if real_x:
        Xrh = torch.as_tensor(wl.X.real, dtype=torch.float32).pin_memory()
        Yrh = torch.empty(Xrh.shape, dtype=torch.float32 if real_out else torch.complex64).pin_memory()
        pipe_r = FG.Pipeline(plan, tuple(Xrh.shape), L, real_io=True, real_output=real_out)
        for _ in range(3):
            pipe_r.submit(alpha, Xrh, Yrh)
        pipe_r.wait()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pipe_r.submit(alpha, Xrh, Yrh)
        pipe_r.wait()
        e2e_s = reduce_max(time.perf_counter() - t0)
        e2e_value = whole_job_rate(n_orders * args.steps, ws, e2e_s)
        t0 = time.perf_counter()
        for _ in range(k_serial):
            plan.apply(alpha, Xrh, L, out=Yrh, real_io=True, real_output=real_out)
            torch.cuda.synchronize()
        e2e_serial = n_orders * k_serial / (time.perf_counter() - t0)
        nbytes_in = Xrh.numel() * 4
        nbytes_out = Yrh.numel() * Yrh.element_size()
        e2e_mode = ("pipelined (copies of step k+1 / k-1 overlap the transform of step k), real float32 host "
                    "signals" + (" and outputs (Q is real)" if real_out else ", complex64 outputs"))
    else:
        nbytes_in = nbytes_out = nbytes

    # ---- the same step captured once into a CUDA graph and replayed: the call's host work and
    # the gaps between its launches leave the loop (the orders and host tables are part of the
    # captured call, re-uploaded by every replay)
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        e0g, e1g = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0g.record(stream)
        for _ in range(args.steps):
            g.replay()
        e1g.record(stream)
        torch.cuda.synchronize()
        ms_g = reduce_max(e0g.elapsed_time(e1g)) / args.steps
        graph_replay = {"ms_per_step": ms_g, "value": whole_job_rate(n_orders * args.steps, ws, ms_g * args.steps / 1e3)}
    except Exception as exc:  # reported, not fatal: the eager numbers above stand
        graph_replay = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("fp16 hi/lo split operands x3 products on tcgen05 tensor cores, f32 accumulate (fused "
                  "multi-order assembly and grouped apply); FP64 offline"), "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "L": L, "orders": n_orders, "signals_per_order": B // n_orders,
                   "path": "assembled (fused multi-order assembly + tcgen05 grouped GEMM)",
                   "signals": ("real float32 signals and outputs (FGFRFT_REAL_SIGNALS / _REAL_OUTPUT)"
                               if real_out else "real float32 signals" if real_x else "complex64 signals"),
                   "l2": "inputs larger than L2 (pair stack 151 MB + assembled split operators 268 MB + "
                         "signals 67 MB in, 67 MB out per step)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "signals_per_s": whole_job_rate(B * args.steps, ws, t_max / 1e3),
        "ms_per_step_with_kernel_events": ms_step_ev,
        "complex64_buffers": {"ms_per_step": ms_step_c, "value": n_orders / (ms_step_c / 1e3) * ws},
        "graph_replay": graph_replay,
        "latency_ms": {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99))},
        "plain_fp32": {"ms_per_step": plain_ms, "order_updates_per_s": n_orders / (plain_ms / 1e3),
                       "io": "complex64 device buffers",
                       # the like-for-like pairing: both paths on complex64 buffers
                       "speedup_vs_plain": plain_ms / ms_step_c,
                       "speedup_vs_plain_pairing": "optimized step on complex64 buffers vs plain path on "
                                                   "complex64 buffers",
                       "speedup_headline_real_io_vs_plain": plain_ms / ms_step,
                       "assemble_single": {"launches": n1, "avg_us": 1e3 * ms1 / max(t1, 1),
                                           "bytes_per_launch": k1_bytes, "achieved_gbs": k1_gbs,
                                           "frac_of_hbm": (k1_gbs / peaks.get("hbm_gbs", 6800.0)) if k1_gbs else None},
                       "simt_gemm_ms_per_step": kt_plain["simt_gemm"][2] / k_plain},
        "roofline": roof,
        "roofline_kernels": rooflines,
        "kernels": kernels,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes_in, "d2h_bytes_per_step": nbytes_out,
                "mode": e2e_mode, "serial_value": e2e_serial, "complex64_buffers": e2e_complex},
        "gpu_launches": launches,
        "clocks": clk,
    }

    if rank == 0 and not args.no_cpu_baseline:
        Yc = Y.cpu().numpy().astype(np.complex128)
        done, el, err = OracleOnline(wl).run(args.cpu_seconds, Y_gpu=Yc)
        line["cpu_baseline"] = {"value": done / el, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"{done} of {n_orders} orders x {B // n_orders} signals, FP64 "
                                          f"numpy (Algorithm 1 with stored powers, then Q X); offline excluded",
                                "rel_err_gpu_vs_fp64": err}
        line["rel_err_vs_fp64"] = err
    # ---- the other legs of the default run (one GPU only: a scaling run times the headline)
    if ws == 1:
        del plan
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        if not args.no_target:
            line["target_n4096_l64"] = leg_target(args, local)
        if not args.no_serving:
            line["serving_small"] = leg_serving(args, local, scale="small", requests=2000, rates=[0.6, 2.0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- default-run legs
def _events_ms(fn, steps, warmup):
    """Device time per call of fn on the current stream (CUDA events), after warmup calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _kernel_ms(FG, cls, fn, steps, warmup):
    """(mean CUDA-event time per launch of kernel class cls, launches) while fn runs steps times."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    FG.timing_reset()
    FG.timing_enable(True)
    for _ in range(steps):
        fn()
    torch.cuda.synchronize()
    FG.timing_enable(False)
    n, t, ms = FG.timing_read()[cls]
    return ms / max(t, 1), n


def _oracle_projector_for(F):
    """FP64 P for the oracle comparisons: real eigenvalues certify r_-1 = 0 cheaply (P = 0)."""
    import scipy.linalg
    from oracle import fgfrft_oracle as O
    lam = scipy.linalg.eigvals(F.real if not np.any(F.imag) else F)
    if np.min(np.abs(lam + 1.0)) > 1e-6:
        return np.zeros(F.shape, dtype=np.complex128)
    return O.projector(F)


def leg_target(args, gpu_index):
    """The target configuration, N = 4096 (4096-point RGG), L = 64, 1024 complex signals:
    single-order assembly from the half stack (K1h) and from the full real split stack (K1r)
    against the HBM roof; the stacked split GEMM with per-column orders against the tensor
    roof; the assembled (one shared order) and plain FP32 paths; each with its error against
    the FP64 oracle on sampled columns.  Offline precompute outside the timed regions."""
    import torch
    from paper_2602_20870_gb300 import fgfrft as FG
    from paper_2602_20870_gb300 import workloads as W
    wl = W.precision()
    N, L, B = wl.N, wl.L, wl.B
    peaks, src = measured_peaks()
    hpeak = peaks.get("hbm_gbs", 6800.0)
    tpeak = peaks.get("bf16_tflops_sustained", 1700.0)
    out = {"workload": wl.name, "orders": "per column U[-2, 2] (stacked); 0.37 shared (assembled, plain)"}
    t0 = time.perf_counter()
    half = FG.Plan(wl.F, L, storage=FG.STORE_HALF | FG.STORE_SPLIT_F16)
    out["offline_precompute_s_half_plus_split"] = time.perf_counter() - t0
    X = torch.as_tensor(wl.X, dtype=torch.complex64).cuda()
    clk = ClockSampler(gpu_index)
    clk.start()
    time.sleep(0.3)
    # K1h: one order from the half stack (L + 2 blocks read as pairs of transposed tiles)
    ms, n = _kernel_ms(FG, "assemble_single", lambda: half.assemble([0.37], L), 10, 3)
    byts = (4.0 if half.real else 8.0) * (L + 1 + (1 if half.r_neg1 > 0 else 0)) * N * N + 8.0 * N * N
    out["assemble_single_half"] = {
        "kernel": "assemble_half_kernel", "bound": "hbm", "avg_launch_ms": ms, "launches": n,
        "order_updates_per_s": 1e3 / ms, "algorithmic_bytes_per_launch": byts,
        "achieved_gbs": byts / (ms * 1e-3) / 1e9, "peak_gbs": hpeak,
        "frac_of_hbm": byts / (ms * 1e-3) / 1e9 / hpeak, "peak_source": f"{src} hbm_gbs"}
    # per-column orders on the stacked split GEMM (all 130 stored blocks as K-major operands)
    ms_st = _events_ms(lambda: half.apply(wl.alpha, X, L, path="stacked"), 4, 1)
    kst, nst = _kernel_ms(FG, "tc_gemm", lambda: half.apply(wl.alpha, X, L, path="stacked"), 3, 0)
    fl = (4.0 if half.real else 8.0) * (2 * L + 2) * N * N * B  # algorithmic (real F: real x complex)
    out["stacked_per_column"] = {
        "kernel": "tc_gemm_kernel<128> (stacked)", "bound": "tensor", "ms_per_call": ms_st,
        "signals_per_s": B / (ms_st * 1e-3), "gemm_avg_launch_ms": kst,
        "algorithmic_flops": fl, "algorithmic_tflops": fl / (kst * 1e-3) / 1e12,
        "executed_tensor_tflops": 3 * fl / (kst * 1e-3) / 1e12,
        "tensor_frac_executed": 3 * fl / (kst * 1e-3) / 1e12 / tpeak,
        "tensor_frac_algorithmic": fl / (kst * 1e-3) / 1e12 / tpeak,
        "peak_tflops": tpeak, "peak_source": f"{src} bf16_tflops_sustained (fp16 dense rate equals bf16)"}
    Ys = half.apply(wl.alpha, X, L, path="stacked").cpu().numpy()
    shared = np.full(B, 0.37)
    ms_as = _events_ms(lambda: half.apply(shared, X, L, path="assembled"), 4, 1)
    Ya = half.apply(shared, X, L, path="assembled").cpu().numpy()
    ms_pl = _events_ms(lambda: half.apply(shared, X, L, path="plain"), 3, 1)
    Yp = half.apply(shared, X, L, path="plain").cpu().numpy()
    out["assembled_shared"] = {"ms_per_call": ms_as, "signals_per_s": B / (ms_as * 1e-3)}
    out["plain_fp32_shared"] = {"ms_per_call": ms_pl, "signals_per_s": B / (ms_pl * 1e-3)}
    out["clocks_half_and_gemm"] = clk.stop()
    del half
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # K1r: one order from the full stack's two real split planes (2L + 2 blocks)
    t0 = time.perf_counter()
    split = FG.Plan(wl.F, L, storage=FG.STORE_SPLIT_F16)
    out["offline_precompute_s_split"] = time.perf_counter() - t0
    clk = ClockSampler(gpu_index)
    clk.start()
    time.sleep(0.3)
    ms, n = _kernel_ms(FG, "assemble_single", lambda: split.assemble([0.37], L), 10, 3)
    byts = (4.0 if split.real else 8.0) * (2 * L + 2) * N * N + 8.0 * N * N
    out["assemble_single_full"] = {
        "kernel": "assemble_single_real_kernel" if split.real else "assemble_single_kernel", "bound": "hbm",
        "avg_launch_ms": ms, "launches": n, "order_updates_per_s": 1e3 / ms, "algorithmic_bytes_per_launch": byts,
        "achieved_gbs": byts / (ms * 1e-3) / 1e9, "peak_gbs": hpeak,
        "frac_of_hbm": byts / (ms * 1e-3) / 1e9 / hpeak, "peak_source": f"{src} hbm_gbs"}
    out["clocks_full"] = clk.stop()
    del split
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if not args.no_cpu_baseline:
        from oracle import fgfrft_oracle as O
        t0 = time.perf_counter()
        P = _oracle_projector_for(wl.F)
        cols = np.arange(0, B, 128)
        ref_s = O.apply_power(wl.F, wl.alpha[cols], L, wl.X[cols].T, P).T
        ref_1 = O.apply_power(wl.F, 0.37, L, wl.X[cols].T, P).T
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        out["rel_err_vs_fp64"] = {"stacked_split (bar 5e-5)": rel(Ys[cols], ref_s),
                                  "assembled_split (bar 5e-5)": rel(Ya[cols], ref_1),
                                  "plain_fp32 (bar 1e-5)": rel(Yp[cols], ref_1),
                                  "sample": f"{len(cols)} of {B} columns, FP64 oracle (signal recursion)",
                                  "oracle_s": time.perf_counter() - t0}
    return out


def leg_serving(args, gpu_index, scale="small", requests=2000, rates=(0.6, 2.0)):
    """Continuous batching against the plain one-request-at-a-time FP32 path (a short sweep)."""
    import torch
    from paper_2602_20870_gb300 import fgfrft as FG
    from paper_2602_20870_gb300 import serving as S
    from paper_2602_20870_gb300 import workloads as W
    sizes = [256, 512, 1024, 1024, 2048, 2048, 4096, 4096] if scale == "full" else \
        [64, 128, 256, 256, 512, 512, 1024, 1024]
    L_max = 64 if scale == "full" else 32
    Ls = (16, 32, 64) if L_max == 64 else (8, 16, 32)
    t0 = time.perf_counter()
    plans = [FG.Plan(W.rgg_gft(n, 500 + i), L_max, storage=FG.STORE_C64 | FG.STORE_SPLIT_F16)
             for i, n in enumerate(sizes)]
    offline_s = time.perf_counter() - t0
    resident = sum(p.plan_bytes for p in plans)
    budget = 150 * 2 ** 30
    sample = W.serving_requests(sizes, 200, rate_per_s=1e9, seed=55, Ls=Ls, lazy=True)
    S.sequential(plans, sample[:20], time_scale=0.0)
    t0 = time.perf_counter()
    S.sequential(plans, sample, time_scale=0.0)
    capacity = len(sample) / (time.perf_counter() - t0)
    sweep = []
    for frac in rates:
        reqs = W.serving_requests(sizes, requests, rate_per_s=frac * capacity, seed=5, Ls=Ls, lazy=True)
        srv = S.Server(plans, budget - resident, max_cols=512, max_inflight_per_graph=2)
        clk = ClockSampler(gpu_index)
        clk.start()
        t0 = time.perf_counter()
        res = S.replay(srv, reqs, timeout_s=3600)
        torch.cuda.synchronize()
        span = time.perf_counter() - t0
        clocks_b = clk.stop()
        clk = ClockSampler(gpu_index)
        clk.start()
        seq = S.sequential(plans, reqs)
        clocks_s = clk.stop()
        seq_span = max(r.done for r in seq)
        sweep.append({"rate_frac_of_capacity": frac, "rate_per_s": frac * capacity,
                      "batched": {**S.latency_stats(res), "throughput_rps": len(reqs) / span,
                                  "launches": srv.launches, "max_reserved_gb": srv.max_reserved / 2 ** 30,
                                  "clocks": clocks_b},
                      "sequential_plain": {**S.latency_stats(seq), "throughput_rps": len(reqs) / seq_span,
                                           "clocks": clocks_s}})
    del plans
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"scale": scale, "graphs": sizes, "L_max": L_max, "requests_per_point": requests,
            "sequential_capacity_rps": capacity, "resident_plan_gb": resident / 2 ** 30,
            "offline_precompute_s": offline_s, "sweep": sweep}


# ----------------------------------------------------------------------------- other configs
def _device_time(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_point_cloud(args):
    """Differentiation config: Y and dY/dalpha in one pass, then the adjoint and the
    alpha-gradient (a full forward + backward of the transform), 384 columns."""
    import torch
    from paper_2602_20870_gb300 import build as BUILD
    BUILD.build()
    from paper_2602_20870_gb300 import fgfrft as FG
    from paper_2602_20870_gb300 import workloads as W
    wl = W.point_cloud()
    N, L, B = wl.N, wl.L, wl.B
    plan = FG.Plan(wl.F, L)
    X = torch.as_tensor(wl.X, dtype=torch.complex64).cuda()
    G = torch.as_tensor(W.complex_normal(wl.X.shape, np.random.default_rng(3)), dtype=torch.complex64).cuda()
    out = {}
    clk = ClockSampler(0)
    clk.start()
    time.sleep(0.3)
    for path in ("stacked", "stacked_fp32"):
        def step():
            Y, D = plan.forward_dual(wl.alpha, X, L, path=path)
            plan.backward(wl.alpha, G, D, L, path=path)
        ms = _device_time(step, args.steps, args.warmup)
        # algorithmic flops: the block products A_b X (shared by Y and the dual, whose
        # coefficients are applied to the same products) and A_b G of the adjoint; a real
        # factor halves a complex multiply-add (8 -> 4 -> 2 flops)
        def per_mac(sig_real):
            return 8.0 / (2 if plan.real else 1) / (2 if sig_real else 1)
        x_real = bool(np.all(np.imag(wl.X) == 0))
        flops = (per_mac(x_real) + per_mac(False)) * (2 * L + 2) * N * N * B
        out[path] = {"ms_per_step": ms, "signals_per_s": B / (ms / 1e3), "algorithmic_tflops": flops / ms / 1e9}
    line = {"metric": "signals/s (forward + dY/dalpha + adjoint + alpha-gradient)", "workload": wl.name,
            "value": out["stacked"]["signals_per_s"], "unit": "signals/s", "paths": out, "clocks": clk.stop()}
    if not args.no_cpu_baseline:
        from oracle import fgfrft_oracle as O
        cols = np.arange(0, B, 47)
        Y, D = plan.forward_dual(wl.alpha, X, L, path="stacked")
        sp = O.spectral(wl.F)
        P = O.projector(wl.F, sp)
        t0 = time.perf_counter()
        Yr = O.apply_power(wl.F, wl.alpha[cols], L, wl.X[cols].T, P).T
        Dr = O.dalpha_apply(wl.F, wl.alpha[cols], L, wl.X[cols].T, P).T
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(cols) / el, "unit": "signals/s (forward + dual)", "cores": cpu_cores(),
                                "kind": "oracle", "sample": f"{len(cols)} columns",
                                "rel_err_Y": _rel(Y.cpu().numpy()[cols], Yr),
                                "rel_err_D": _rel(D.cpu().numpy()[cols], Dr)}
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args):
    """Precision config (N = 4096, L = 64, 1024 columns): the default run's target leg alone."""
    from paper_2602_20870_gb300 import build as BUILD
    BUILD.build()
    out = leg_target(args, 0)
    line = {"metric": "signals/s and order-updates/s", "unit": "signals/s",
            "value": out["stacked_per_column"]["signals_per_s"], **out}
    print(json.dumps(line), flush=True)
    return 0


def run_stacked(args):
    """The stacked split GEMM with per-column orders on a small case (image-graph graph,
    N = 1024, L = 32, 512 complex signals with orders U[-2, 2], split storage only, about
    0.6 GB on the device): Y[:, j] = sum over the 66 stored blocks of c_b(alpha_j) A_b X[:, j]
    as one tcgen05 GEMM (Def. 2), with its tensor-roofline fraction and error against FP64."""
    import torch
    from paper_2602_20870_gb300 import build as BUILD
    BUILD.build()
    from paper_2602_20870_gb300 import fgfrft as FG
    from paper_2602_20870_gb300 import workloads as W
    wl = W.image_graph()
    N, L, B = wl.N, wl.L, 512
    rng = np.random.default_rng(12)
    X = W.complex_normal((B, N), rng)
    alpha = rng.uniform(-2.0, 2.0, size=B)
    plan = FG.Plan(wl.F, L, storage=FG.STORE_SPLIT_F16)
    Xd = torch.as_tensor(X, dtype=torch.complex64).cuda()
    peaks, src = measured_peaks()
    tpeak = peaks.get("bf16_tflops_sustained", 1700.0)
    clk = ClockSampler(0)
    clk.start()
    time.sleep(0.3)
    ms = _device_time(lambda: plan.apply(alpha, Xd, L, path="stacked"), args.steps, args.warmup)
    kms, n = _kernel_ms(FG, "tc_gemm", lambda: plan.apply(alpha, Xd, L, path="stacked"), args.steps, 1)
    clocks = clk.stop()
    fl = (4.0 if plan.real else 8.0) * (2 * L + 2) * N * N * B
    line = {"metric": "signals/s (stacked split GEMM, per-column orders)", "workload":
            f"image-graph graph N={N}, L={L}, {B} complex signals, per-column orders", "unit": "signals/s",
            "value": B / (ms * 1e-3), "ms_per_call": ms, "gemm_avg_launch_ms": kms, "launches": n,
            "roofline": {"bound": "tensor", "kernel": "tc_gemm_kernel<128> (stacked)",
                         "achieved": fl / (kms * 1e-3) / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                         "frac": fl / (kms * 1e-3) / 1e12 / tpeak, "algorithmic_flops": fl,
                         "executed_tensor_frac": 3 * fl / (kms * 1e-3) / 1e12 / tpeak,
                         "peak_source": f"{src} bf16_tflops_sustained (fp16 dense rate equals bf16)",
                         "traffic": kernel_traffic("tc_gemm_kernel<128> (stacked)", "stacked")},
            "clocks": clocks}
    if not args.no_cpu_baseline:
        from oracle import fgfrft_oracle as O
        cols = np.arange(0, B, 64)
        Y = plan.apply(alpha, Xd, L, path="stacked").cpu().numpy()
        P = _oracle_projector_for(wl.F)
        ref = O.apply_power(wl.F, alpha[cols], L, X[cols].T, P).T
        line["rel_err_vs_fp64 (bar 5e-5)"] = _rel(Y[cols], ref)
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Serving config: Poisson arrivals over 8 resident graphs, continuous batching against
    the plain one-request-at-a-time FP32 path, at the given fractions of the sequential
    capacity (clocks recorded during each timed run)."""
    from paper_2602_20870_gb300 import build as BUILD
    BUILD.build()
    out = leg_serving(args, 0, scale=args.serving_scale, requests=args.serving_requests, rates=args.serving_rates)
    line = {"metric": "serving p50/p99 latency and throughput vs plain sequential FP32", "unit": "requests/s",
            "value": out["sweep"][-1]["batched"]["throughput_rps"], **out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "point-cloud":
        return run_point_cloud(args)
    if args.workload == "precision":
        return run_precision(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "stacked":
        return run_stacked(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
