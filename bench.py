#!/usr/bin/env python
"""Throughput benchmark of the Gauss-polynomial bilateral filter on GB300.

Workload (default): one 4096 x 4096 FP32 image (16.8 Mpx; 512 rectangles +
noise std 15, seeded), sigma_s = 10, sigma_r = 20, order N = 20 (K = 22
channels), Deriche recursive Gaussian.  A step is one full forward pass
(stats -> row pass -> column pass + combine) over the image, through the
library's C ABI.  Metric: Mpixel/s (higher is better).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank filters its own image (independent problems, weak
scaling, no collective on the data path); value = all ranks' pixels / max
rank time.  --impl reference times the FP64 CPU oracle (Algorithm 1) on the
host cores instead (rank 0 only).
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

EXTRA_WORKLOADS = {
    # batched: 64 images, sides U{256..2048}, 3 planes each, per-image sigma_s in [1, 16], sigma_r in [10, 60]
    "gpf-batched-64img-3ch-N20-iir": "uneven-batch",
    # differentiation: 16 x 512^2, sigma_s 5, sigma_r 25, N 20, forward + hand-written backward
    "gpf-16x512x512-ss5-sr25-N20-fwdbwd": "batch512-fwdbwd",
    # runtime against sigma_s with the recursive filter: 1024^2, sigma_s in {2, 5, 10, 20}, sigma_r 30, N 20
    "gpf-1024x1024-sr30-N20-iir-sigma-sweep": "rects-ramp1024-sweep",
    # joint (cross) filter: data = the 4096^2 image, guide = a second seeded 4096^2 image, K = 42 channels
    "gpf-joint-4096x4096-ss10-sr20-N20-iir": "joint",
}

WORKLOADS = {
    # name: (H, W, sigma_s, sigma_r, order, spatial, generator)
    "gpf-4096x4096-ss10-sr20-N20-iir": (4096, 4096, 10.0, 20.0, 20, "iir", "rects4096"),
    "gpf-256x256-ss3-sr30-N20-fir": (256, 256, 3.0, 30.0, 20, "fir", "rects256"),
    "gpf-2048x2048-ss10-sr20-N20-iir": (2048, 2048, 10.0, 20.0, 20, "iir", "rects4096-crop"),
    "gpf-1024x1024-ss2-sr30-N20-fir": (1024, 1024, 2.0, 30.0, 20, "fir", "rects-ramp1024"),
    # box variant of S: 3 passes of a flat kernel matched to sigma_s = 3 (r = 3), fused kernel
    "gpf-1024x1024-ss3-sr30-N20-box3": (1024, 1024, 3.0, 30.0, 20, "box", "rects-ramp1024"),
}
DEFAULT = "gpf-4096x4096-ss10-sr20-N20-iir"
FALLBACK_HBM_GBS = 6800.0


def make_input(gen, H, W, rank):
    import synthetic
    if gen == "rects4096":
        if rank == 0:
            return synthetic.rects4096_image()
        return synthetic.make_image(H, W, 512, 15.0, 0.0, synthetic.seed_for(3, rank))
    if gen == "rects4096-crop":
        return synthetic.make_image(H, W, 128, 15.0, 0.0, synthetic.seed_for(3, 100 + rank))
    if gen == "rects-ramp1024":
        if rank == 0:
            return synthetic.rects_ramp1024_image()
        return synthetic.make_image(H, W, 64, 10.0, 60.0, synthetic.seed_for(2, rank))
    if gen == "rects256":
        if rank == 0:
            return synthetic.rects256_image()
        return synthetic.make_image(H, W, 16, 10.0, 0.0, synthetic.seed_for(1, rank))
    raise ValueError(gen)


def reduce_max(value: float, dist, device) -> float:
    """Max of `value` over the ranks: the slowest rank's time is the job's time."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(px_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job Mpixel/s: every rank filters its own image each step (weak scaling)."""
    return px_per_rank * world * steps / (total_ms / 1e3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.path = tempfile.mktemp(prefix="bench_clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        self.interval = interval_ms
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu=timestamp,{self.FIELDS}",
                                          "--format=csv,noheader,nounits", f"-lms", str(self.interval)],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[5:10]))
            except (ValueError, IndexError):
                continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.05 <= r[0] <= self.t1 + 0.05]
        window = "timed"
        if not inside:
            inside = rows
            window = "process (timed region shorter than the sampling interval)"
        reasons = set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in inside:
            for n, v in zip(names[1:], r[3][1:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("bf_gp_device.cuh", "bf_gp.cu"):
        h.update(open(os.path.join(ROOT, "paper_1505_00077_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_launch"])


def cpu_baseline(img, ss, sr, N, spatial, budget_s=20.0):
    """The FP64 oracle (as it stands) on the host cores: full image, repeated
    until ~budget_s of CPU work has been done (at least once)."""
    import numpy as np

    import oracle
    oracle.build()
    f = img.astype(np.float64)
    runs, t_total = 0, 0.0
    while True:
        t = time.perf_counter()
        oracle.gp_bf(f, ss, sr, N, spatial)
        t_total += time.perf_counter() - t
        runs += 1
        if t_total >= budget_s or runs >= 5 or t_total / runs * (runs + 1) > 2 * budget_s:
            break
    px = f.size * runs
    return {"value": px / t_total / 1e6, "unit": "Mpixel/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{runs} run(s) of the FP64 Algorithm-1 oracle on the full {f.shape[0]}x{f.shape[1]} image "
                      f"({spatial}, sigma_s={ss}, sigma_r={sr}, N={N}), {t_total:.1f} s"}


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    H, W, ss, sr, N, spatial, gen = WORKLOADS[args.workload]
    oracle.build()
    img = make_input(gen, H, W, 0).astype(np.float64)
    # bounded sample per step: a band of rows (its own image) sized so that
    # warmup + steps take about args.ref_budget seconds
    band = min(H, 128)
    t = time.perf_counter()
    oracle.gp_bf(img[:band], ss, sr, N, spatial)
    rate = band * W / max(1e-6, time.perf_counter() - t)  # px/s
    per_step = args.ref_budget / max(1, args.steps + args.warmup)
    rows = int(max(8, min(H, per_step * rate / W)))
    sample = img[:rows]
    for _ in range(args.warmup):
        oracle.gp_bf(sample, ss, sr, N, spatial)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.gp_bf(sample, ss, sr, N, spatial)
    dt = time.perf_counter() - t
    value = rows * W * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": "Mpixel/s", "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "H": H, "W": W, "sigma_s": ss, "sigma_r": sr, "order": N,
                       "spatial": spatial, "sample_rows": rows},
            "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"first {rows} rows ({rows}x{W}) of the workload image per step"},
            "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(EXTRA_WORKLOADS), default=DEFAULT)
    ap.add_argument("--engine", choices=["auto", "tensor", "cuda-core", "tcgen05"], default="auto",
                    help="recursive filter engine: auto (tensor-core rows, CUDA-core columns), tensor, cuda-core")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--ref-budget", type=float, default=90.0, help="seconds of oracle work for --impl reference")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    rank, world, local = dist_env()
    if args.impl == "reference":
        if args.workload in EXTRA_WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm covers the single-image workloads"}))
            return 0
        return run_reference(args, rank, world)
    if args.workload in EXTRA_WORKLOADS:
        return run_extra(args, rank, world, local)

    import numpy as np
    import torch

    import paper_1505_00077_gb300 as bf

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    H, W, ss, sr, N, spatial, gen = WORKLOADS[args.workload]
    bf.build()
    img = make_input(gen, H, W, rank)
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    opts = bf.make_opts(N, spatial, engine={"auto": 0, "cuda-core": 1, "tensor": 2, "tcgen05": 3}[args.engine])
    tune = spatial in ("fir", "iir") and args.engine == "auto"
    ws_bytes = bf.bf_gp_workspace_size(1, H, W, ss, opts)
    if tune:  # room for every candidate the autotuner times (the two-pass FIR form is the largest)
        ws_bytes = max([ws_bytes] + [bf.bf_gp_workspace_size(1, H, W, ss, bf.make_opts(N, spatial, engine=e,
                                                                                       fir_two_pass=spatial == "fir"))
                                     for e in range(4)])
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    K = N + 2
    tuned = None
    if tune:
        # recursive filter: engine and row-pass CTA size; window sum: fused tile height or the two-pass
        # form; from the autotuner, before the measured region
        opts, _ = bf.bf_gp_autotune(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, opts, ws.data_ptr(), ws_bytes,
                                    sp, reps=20)
        tuned = {"engine": int(opts.engine), "fir_two_pass": int(opts.fir_two_pass), "fir_tile": int(opts.fir_tile),
                 "row_threads": int(opts.row_threads), "how": "bf_gp_autotune (20 timed runs per candidate)"}

    fused = spatial == "box" or (spatial == "fir" and not opts.fir_two_pass)
    working_set = (12 * H * W) if fused else (ws_bytes + 8 * H * W)
    small = working_set < 2 * 129e6
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda") if small else None

    def step():
        # one forward pass through the public entry point: stats, then rows + columns
        # (recursive filter or two-pass FIR) or the fused FIR tile kernel
        bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, opts, ws.data_ptr(), ws_bytes, sp)

    for _ in range(args.warmup):
        step()
    status = bf.bf_gp_get_device_status(ws.data_ptr(), sp)
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    sampler.mark("t0")
    if small:
        # working set below the 129 MB L2: each step is timed alone, with the L2
        # flushed (a 512 MB buffer overwritten) between steps, outside the events
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            pairs[i][0].record(stream)
            step()
            pairs[i][1].record(stream)
        barrier()
        sampler.mark("t1")
        clocks = sampler.stop()
        total_ms = sum(a.elapsed_time(b) for a, b in pairs)
    else:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            step()
        t_end.record(stream)
        barrier()
        sampler.mark("t1")
        clocks = sampler.stop()
        total_ms = t_start.elapsed_time(t_end)

    # per-kernel times (CUDA events on the launching stream), after the timed region
    n_ph = max(1, min(args.steps, 50))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(n_ph)]
    for i in range(n_ph):
        e = evs[i]
        e[0].record(stream)
        bf.bf_gp_phase_stats(x.data_ptr(), 1, H, W, W, ss, sr, opts, ws.data_ptr(), ws_bytes, sp)
        e[1].record(stream)
        if fused:
            step()
            e[2].record(stream)
        else:
            bf.bf_gp_phase_rows(x.data_ptr(), 1, H, W, W, ss, sr, opts, ws.data_ptr(), ws_bytes, sp)
            e[2].record(stream)
            bf.bf_gp_phase_cols(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, opts, ws.data_ptr(), ws_bytes, sp)
        e[3].record(stream)
    torch.cuda.synchronize()
    stats_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / n_ph
    rows_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / n_ph
    cols_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / n_ph
    if fused:  # e[1] -> e[2] is a whole forward (stats + fused kernel)
        fused_ms = max(rows_ms - stats_ms, 1e-6)
        rows_ms = cols_ms = 0.0
    total_ms = reduce_max(total_ms, dist, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_throughput(H * W, world, args.steps, total_ms)

    # end to end through the public host entry point (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        need = bf.bf_gp_host_workspace_size(1, H, W, ss, opts)
        ws_h = torch.empty(need, dtype=torch.uint8, device="cuda")
        fh = torch.from_numpy(img).pin_memory()
        yh = torch.empty_like(fh).pin_memory()
        for _ in range(2):
            bf.bf_gp_forward_host(fh.data_ptr(), yh.data_ptr(), 1, H, W, ss, sr, opts, ws_h.data_ptr(), need, sp)
        barrier()
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            bf.bf_gp_forward_host(fh.data_ptr(), yh.data_ptr(), 1, H, W, ss, sr, opts, ws_h.data_ptr(), need, sp)
        barrier()
        dt = time.perf_counter() - t
        dt = reduce_max(dt, dist, "cuda")
        e2e = {"value": job_throughput(H * W, world, args.e2e_steps, dt * 1e3), "unit": "Mpixel/s",
               "h2d_bytes_per_step": 4 * H * W, "d2h_bytes_per_step": 4 * H * W,
               "how": "bf_gp_forward_host, wall clock: the statistics pass reads the pinned host f and stores the "
                      "device copy, forward, the last pass stores y straight into mapped pinned host memory"}
        # the host path must agree with the device path bit for bit
        step()
        torch.cuda.synchronize()
        if not torch.equal(yh, y.cpu()):
            print("warning: host entry point result differs from the device path", file=sys.stderr)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    bytes_rows = (4 + 4 * K) * H * W       # read f, write K row-filtered planes
    bytes_cols = (4 * K + 8) * H * W       # read K planes + f, write y
    # the kernels of the engine that ran: 0 row_tc + col_iir, 1 row_iir + col_iir, 2 row_tc + col_tc,
    # 3 row_iir + col_tc5
    rk = ("row_tc" if opts.engine in (0, 2) else "row_iir") if spatial == "iir" else "row_fir"
    ck = ("col_iir", "col_iir", "col_tc", "col_tc5")[opts.engine] if spatial == "iir" else "col_fir"
    if fused:
        # FP32 FMA per pixel of the separable filter (row + column, 2w + 1 taps each) and the combine,
        # against the FP32 FMA rate of the SMs (152 SMs x 128 lanes x the measured maximum SM clock)
        w_half = int(math.ceil(3 * ss - 1e-12))  # W = ceil(3 sigma_s), the default window
        # window sum: 2 w + 1 multiply-adds per sample and direction; box variant (3 passes): two
        # running-sum additions per pass and direction
        fma_px = K * ((4 * 3 if spatial == "box" else 2 * (2 * w_half + 1)) + 3)
        alu_peak = 152 * 128 * float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]) * 1e6 \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 152 * 128 * 2.07e9
        achieved = fma_px * H * W / (fused_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": "fir_fused", "achieved": achieved, "peak": alu_peak / 1e12,
                    "unit": "T FMA/s", "frac": achieved / (alu_peak / 1e12),
                    "peak_kind": "derived (152 SMs x 128 FP32 lanes x sm_max_mhz of MEASURED_PEAKS.json)",
                    "algorithmic_fma_per_launch": fma_px * H * W, "kernel_ms": fused_ms,
                    "traffic": committed_traffic("fir_fused", args.workload)}
    else:
        dominant = (rk, rows_ms, bytes_rows) if rows_ms >= cols_ms else (ck, cols_ms, bytes_cols)
        achieved = dominant[2] / (dominant[1] / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": dominant[0], "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_kind": f"{peak_kind} (hbm_gbs)",
                    "algorithmic_bytes_per_launch": dominant[2], "kernel_ms": dominant[1],
                    "traffic": committed_traffic(dominant[0], args.workload)}
    line = {
        "metric": "Mpixel/s", "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "H": H, "W": W, "planes_per_gpu": 1, "sigma_s": ss, "sigma_r": sr,
                   "order": N, "channels": K, "spatial": spatial, "engine": args.engine, "tuned": tuned,
                   "parallelism": f"replicas x{world}",
                   "l2": (f"working set {working_set / 1e6:.1f} MB < 2 x 129 MB L2: each step timed alone, "
                          "L2 flushed (512 MB written) between steps" if small else
                          f"working set {working_set / 1e9:.2f} GB per step > 129 MB L2 (no flush needed)")},
        "phases_ms": ({"stats": stats_ms, "fir_fused": fused_ms} if fused else
                      {"stats": stats_ms, "rows": rows_ms, "cols": cols_ms}),
        "roofline": roofline,
        "gpu_launches": (3 if fused else 4) * args.steps,
        "device_status": status,
    }
    step_bytes = (12 if fused else 8 * K + 16) * H * W
    line["step_roofline"] = {"bound": "hbm", "algorithmic_bytes_per_step": step_bytes,
                             "frac": step_bytes / (ms_per_step / 1e3) / 1e9 / peak}
    if clocks is not None:
        line["clocks"] = clocks
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(img, ss, sr, N, spatial)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _clock_wrap(local, fn):
    sampler = ClockSampler(local)
    sampler.start()
    sampler.mark("t0")
    out = fn()
    sampler.mark("t1")
    return out, sampler.stop()


def run_extra(args, rank, world, local):
    """Batched (uneven batch), forward + backward (16 x 512^2), sigma_s-sweep (1024^2) and joint-filter
    workloads, one GPU."""
    import numpy as np
    import torch

    import paper_1505_00077_gb300 as bf
    import synthetic

    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    bf.build()
    peak, peak_kind = measured_peaks()
    kind = EXTRA_WORKLOADS[args.workload]
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def timed(fn, steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    if kind == "joint":
        H = W = 4096
        fd = torch.from_numpy(synthetic.rects4096_image()).cuda()
        gd = torch.from_numpy(synthetic.make_image(H, W, 512, 15.0, 0.0, synthetic.seed_for(3, 900))).cuda()
        y = torch.empty_like(fd)
        opts = bf.make_opts(20, "iir")
        need = bf.bf_gp_joint_workspace_size(1, H, W, 10.0, opts)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        K = 42

        def fwd():
            bf.bf_gp_forward_joint(fd.data_ptr(), gd.data_ptr(), y.data_ptr(), 1, H, W, W, 10.0, 20.0, opts,
                                   ws.data_ptr(), need, sp)
        for _ in range(args.warmup):
            fwd()
        steps = max(1, args.steps)
        ms, clocks = _clock_wrap(local, lambda: timed(fwd, steps))
        bytes_step = (8 * K + 20) * H * W  # stats (guide), rows read guide + data and write K planes, columns
        line = {"metric": "Mpixel/s", "value": H * W / (ms / 1e3) / 1e6, "unit": "Mpixel/s", "n_gpus": 1,
                "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "H": H, "W": W, "sigma_s": 10.0, "sigma_r": 20.0, "order": 20,
                           "channels": K, "spatial": "iir", "how": "bf_gp_forward_joint, CUDA-core passes"},
                "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": bytes_step,
                                  "achieved": bytes_step / (ms / 1e3) / 1e9, "peak": peak,
                                  "frac": bytes_step / (ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind},
                "gpu_launches": 4 * steps,
                "device_status": bf.bf_gp_get_device_status(ws.data_ptr(), sp)}
        if clocks:
            line["clocks"] = clocks
        print(json.dumps(line), flush=True)
        return 0

    if kind == "rects-ramp1024-sweep":
        img = synthetic.rects_ramp1024_image()
        x = torch.from_numpy(img).cuda()
        y = torch.empty_like(x)
        H, W = x.shape
        opts = bf.make_opts(20, "iir")
        per = {}
        steps = max(1, args.steps)
        clocks = None
        for ss in (2.0, 5.0, 10.0, 20.0):
            need = bf.bf_gp_workspace_size(1, H, W, ss, opts)
            ws = torch.empty(need, dtype=torch.uint8, device="cuda")

            def fwd():
                bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, 30.0, opts, ws.data_ptr(), need, sp)
            for _ in range(args.warmup):
                fwd()
            if ss == 10.0:
                ms, clocks = _clock_wrap(local, lambda: timed(fwd, steps))
            else:
                ms = timed(fwd, steps)
            per[f"{ss:g}"] = ms
        mean_ms = sum(per.values()) / len(per)
        line = {"metric": "Mpixel/s", "value": H * W / (mean_ms / 1e3) / 1e6, "unit": "Mpixel/s", "n_gpus": 1,
                "steps": steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "H": H, "W": W, "sigma_s": list(per), "sigma_r": 30.0,
                           "order": 20, "spatial": "iir", "how": "bf_gp_forward per sigma_s, mean time"},
                "ms_per_sigma_s": per, "max_over_min": max(per.values()) / min(per.values()),
                "gpu_launches": 4 * steps * len(per)}
        if clocks:
            line["clocks"] = clocks
        print(json.dumps(line), flush=True)
        return 0

    if kind == "uneven-batch":
        specs = synthetic.uneven_batch_specs()
        planes = []
        K = 22
        for spec in specs:
            img = synthetic.uneven_batch_image(spec)
            for c in range(3):
                x = torch.from_numpy(np.ascontiguousarray(img[c])).cuda()
                planes.append((x, torch.empty_like(x), spec[3], spec[4], 20))
        px = sum(x.numel() for x, *_ in planes)
        # each plane runs with the engine the autotuner measures fastest for its shape (timed before the
        # measured region; shape classes repeat, so most planes reuse a stored choice)
        bfilt = bf.BatchedFilter(planes, autotune=True)
        engines = bfilt.engines
        for _ in range(args.warmup):
            bfilt.run()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bfilt.run()
        steps = max(1, min(args.steps, 50))
        for _ in range(2):
            g.replay()
        ms, clocks = _clock_wrap(local, lambda: timed(g.replay, steps))
        status = bfilt.status()
        # the same batch as one persistent launch (engine 0 for every plane), captured and replayed
        gp = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gp):
            bfilt.run_persistent()
        for _ in range(2):
            gp.replay()
        ms_pers = timed(gp.replay, max(1, min(args.steps, 20)))
        status_pers = bfilt.status()
        # plain form: the single-image path plane by plane (same kernels, 4 launches per plane)
        popts = [bf.make_opts(o, "iir", engine=e) for (x, y, ss, sr, o), e in zip(planes, engines)]
        maxws = max(bf.bf_gp_workspace_size(1, p[0].shape[0], p[0].shape[1], p[2], po) for p, po in zip(planes, popts))
        ws = torch.empty(maxws, dtype=torch.uint8, device="cuda")

        def plain():
            for (x, y, ss, sr, o), po in zip(planes, popts):
                bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, x.shape[0], x.shape[1], x.shape[1], ss, sr,
                                 po, ws.data_ptr(), maxws, sp)
        plain()
        ms_plain = timed(plain, max(1, min(args.steps, 5)))
        bytes_step = (8 * K + 16) * px
        line = {"metric": "Mpixel/s", "value": px / (ms / 1e3) / 1e6, "unit": "Mpixel/s", "n_gpus": 1,
                "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "planes": len(planes), "pixels": px, "order": 20,
                           "spatial": "iir", "how": "CUDA graph of bf_gp_batched (every plane's forward on 8 streams forked from and joined into the capturing stream, then a status gather), replayed",
                           "engines": {str(e): engines.count(e) for e in sorted(set(engines))},
                           "engine_choice": "bf_gp_batched_plan_tune (per plane, before the timed region)"},
                "plain_loop": {"value": px / (ms_plain / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": ms_plain,
                               "how": "bf_gp_forward plane by plane, same kernels and engines, no graph"},
                "persistent": {"value": px / (ms_pers / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": ms_pers,
                               "device_status": status_pers,
                               "how": "CUDA graph of bf_gp_batched_persistent: one launch of resident 4-CTA clusters "
                                      "taking statistics, row and column items from a counter (engine 0 kernels' "
                                      "arithmetic for every plane), replayed"},
                "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": bytes_step,
                                  "achieved": bytes_step / (ms / 1e3) / 1e9, "peak": peak,
                                  "frac": bytes_step / (ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind},
                "gpu_launches": (4 * len(planes) + 1) * steps,
                "device_status": status}
        if clocks:
            line["clocks"] = clocks
        print(json.dumps(line), flush=True)
        return 0

    # forward + backward on a 16 x 512^2 batch (planes in one call)
    xb = synthetic.batch512(16)[:, 0]
    B, H, W = xb.shape
    K = 22
    x = torch.from_numpy(np.ascontiguousarray(xb)).cuda()
    gy = torch.from_numpy(np.random.default_rng(5).normal(size=xb.shape).astype(np.float32)).cuda()
    opts = bf.make_opts(20, "iir")
    need = bf.bf_gp_workspace_size(B, H, W, 5.0, opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    saved = torch.empty((B, 4, H, W), dtype=torch.float32, device="cuda")
    gx = torch.empty_like(x)
    gsr = torch.empty(B, dtype=torch.float32, device="cuda")

    def fwd():
        bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), B, H, W, W, 5.0, 25.0, opts, ws.data_ptr(), need, sp)

    def fwdbwd():
        bf.bf_gp_forward_train(x.data_ptr(), y.data_ptr(), saved.data_ptr(), B, H, W, W, 5.0, 25.0, opts,
                               ws.data_ptr(), need, sp)
        bf.bf_gp_backward(x.data_ptr(), gy.data_ptr(), saved.data_ptr(), gx.data_ptr(), gsr.data_ptr(), B, H, W, W,
                          5.0, 25.0, opts, ws.data_ptr(), need, sp)

    def plain_fwd():  # the single-image form: one call per image
        for i in range(B):
            bf.bf_gp_forward(x[i].data_ptr(), y[i].data_ptr(), 1, H, W, W, 5.0, 25.0, opts, ws.data_ptr(), need, sp)

    for _ in range(args.warmup):
        fwdbwd()
        fwd()
        plain_fwd()
    steps = max(1, args.steps)
    ms, clocks = _clock_wrap(local, lambda: timed(fwdbwd, steps))
    ms_fwd = timed(fwd, steps)
    ms_plain = timed(plain_fwd, steps)
    px = B * H * W
    # algorithmic bytes per pixel: the forward that saves its sums, 8K + 16 plus 16 (P~, Q~ and the two
    # derivative sums written); the backward, 8K + 56: statistics 4, the adjoint row pass reads f, dL/dy and
    # two saved sums (16) and writes K planes, the adjoint column pass reads the K planes, f, dL/dy and the
    # four saved sums (24) and writes dL/dh (4), the finish reads and writes the gradient (8)
    bytes_step = ((8 * K + 32) + (8 * K + 56)) * px
    line = {"metric": "Mpixel/s", "value": px / (ms / 1e3) / 1e6, "unit": "Mpixel/s", "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "batch": B, "H": H, "W": W, "sigma_s": 5.0, "sigma_r": 25.0,
                       "order": 20, "spatial": "iir", "step": "bf_gp_forward_train + bf_gp_backward"},
            "fwd_only": {"value": px / (ms_fwd / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": ms_fwd},
            "plain_single_image_fwd": {"value": px / (ms_plain / 1e3) / 1e6, "unit": "Mpixel/s",
                                       "ms_per_step": ms_plain},
            "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": bytes_step,
                              "achieved": bytes_step / (ms / 1e3) / 1e9, "peak": peak,
                              "frac": bytes_step / (ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind},
            "gpu_launches": 8 * steps}
    if clocks:
        line["clocks"] = clocks
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
