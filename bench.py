#!/usr/bin/env python
"""Benchmark of the butterfly-filtering hot path on GB300.

Workload (one step): the GW-like pair -- two 64 s series at 4096 Hz
(262,144 samples each) of coloured Gaussian noise with a common power-law
chirp -- plus their two time-randomised controls, searched against a bank of
65,536 ascending power-law templates of 4096 samples (1 s).  A step runs every
stage of the path: template synthesis, the two controls, series preparation
(split rows, FP64 prefix norms), the batched split-BF16 tensor-core correlation
of all four series in one launch, the fused epilogue (max/argmax, sigma,
tails), finalize (histogram of maxima, time-frequency map painting) and the
skew-normal fits of the maxima and the two-detector coincidence pseudo-spectra
of data and controls -- all through the C ABI.

metric: lag-correlations per second (one normalised length-M inner product of
one template at one lag), whole job.  Printed as one JSON line by rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this project
has) on a bounded sample of the same workload.  Under torchrun every rank runs
an independent replica (the search of one batch is not sharded across GPUs).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "correlations/s on 1 GB300, split-BF16 vs FP32 at |err|<=2e-5; serve p50/p99 ms"
UNIT = "correlations/s"

# DRAM traffic of the tensor-core correlation kernel measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, one launch of the
# --kernel-case capture), per 128-template tile: every CTA works on the same
# template tile at once, so each template block is read from DRAM once and the
# traffic grows with the number of template tiles, not with the lag tiles.
# Keyed by (hash of the kernel source the counters were taken on, lags per
# tile); a changed kernel reports null until it is captured again.
TRAFFIC_BYTES_PER_TEMPLATE_TILE = {
    ("d4820c4a9ba61a1a", 256): (272.17e6 + 0.68e6) / 128,   # the 16 s x 16,384-template capture
}


def kernel_source_hash() -> str:
    """Hash of the tensor-core kernel's code (// comments and blank lines
    stripped), so that the DRAM traffic captured for it is reported only while
    the code is the one captured."""
    with open(os.path.join(ROOT, "paper_1802_01685_gb300", "csrc", "corr_tc.cu")) as f:
        lines = [l.split("//", 1)[0].rstrip() for l in f]
    code = "\n".join(l for l in lines if l.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


# ------------------------------------------------------------------ helpers

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"bf16_burst": d["bf16_tflops"], "bf16_sustained": d["bf16_tflops_sustained"],
                "hbm": d["hbm_gbs"], "source": "measured"}
    return {"bf16_burst": 1900.0, "bf16_sustained": 1700.0, "hbm": 6800.0, "source": "fallback"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_dist(world: int, backend: str, device=None):
    """Barrier and max-over-ranks for N independent replicas (each rank runs
    the whole workload on its own GPU; nothing is exchanged but timings)."""
    import torch
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        if device is not None:
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    return barrier, max_over_ranks


def whole_job_value(units_per_step: float, steps: int, world: int, max_elapsed_ms: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_step * steps / (max_elapsed_ms / 1e3)


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local):
    import torch

    import __graft_entry__
    from paper_1802_01685_gb300 import bf, synth

    __graft_entry__.build()
    torch.cuda.set_device(local)
    barrier, max_over_ranks = make_dist(world, "nccl", torch.device("cuda", local))

    w = synth.gw_pair()
    fs, M = w["fs"], w["M"]
    seeds = w["control_seeds"]
    cfg = bf.bf_config_default()
    cfg.device = local
    ctx = bf.bf_init(cfg)
    xs_host = [torch.from_numpy(x).pin_memory() for x in w["series"]]
    xs = [x.cuda() for x in xs_host]
    ctrl = [torch.empty_like(x) for x in xs]
    N = xs[0].numel()
    K = synth.grid_size(w["grid"])
    L = N - M + 1
    corr_per_step = 4 * L * K
    opts = bf.make_opts(precision="split_bf16", want_map=True, want_hist=True)
    kernel_ms = []
    stage_ms = {}
    shapes = set()
    fits = {}
    coincidences = {}

    def step(record=False):
        t0 = time.perf_counter()
        bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16)
        t1 = time.perf_counter()
        for x, c, sd in zip(xs, ctrl, seeds):
            bf.bf_control_randomize(ctx, x, sd, c)
        t2 = time.perf_counter()
        res = bf.bf_correlate(ctx, bank, xs + ctrl, fs, opts)
        # skew-normal fits of the maxima: data (series 0, 1) vs controls (2, 3)
        fit = [bf.bf_result_fit_max(res, s) for s in range(4)]
        # two-detector pseudo-spectra: data pair (0, 1) and control pair (2, 3)
        coinc = [bf.bf_result_coincidence(res, a, b, 50.0, 0) for a, b in ((0, 1), (2, 3))]
        t3 = time.perf_counter()
        info = bf.bf_result_info_get(res)
        if record:
            fits.update({name: {k: round(fit[i][k], 6) for k in ("xi", "omega", "alpha")}
                         for i, name in enumerate(("data_0", "data_1", "control_0", "control_1"))})
            coincidences.update({name: {k: int(v.sum()) for k, v in c.items()}
                                 for name, c in zip(("data", "control"), coinc)})
            kernel_ms.append(info.kernel_ms)
            shapes.add(info.tile_lags)
            for k, v in (("bank_synthesis", t1 - t0), ("controls", t2 - t1), ("correlate", t3 - t2)):
                stage_ms.setdefault(k, []).append(1e3 * v)
        bf.bf_result_destroy(res)
        bf.bf_bank_destroy(bank)
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = bf.bf_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        info = step(record=True)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = bf.bf_kernel_launches() - launches0
    barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1))
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_value(corr_per_step, args.steps, world, elapsed_ms)

    # roofline of the dominant kernel (the split-BF16 tcgen05 correlation), on
    # the method's work: 2M flops per lag-correlation (one length-M inner
    # product).  The split issues three BF16 MMAs per operand pair, 6M tensor
    # flops per lag-correlation, reported beside it.
    peaks = measured_peaks()
    k_ms = float(np.mean(kernel_ms))
    useful_flops = 2 * M * corr_per_step
    issued_flops = 3 * useful_flops
    achieved = useful_flops / (k_ms / 1e3) / 1e12
    issued = issued_flops / (k_ms / 1e3) / 1e12
    th = kernel_source_hash()
    lt = sorted(shapes)[0] if len(shapes) == 1 else None
    traffic = None
    if (th, lt) in TRAFFIC_BYTES_PER_TEMPLATE_TILE:
        traffic = round(TRAFFIC_BYTES_PER_TEMPLATE_TILE[(th, lt)] * (K // 128))
    roofline = {"bound": "tensor", "achieved": round(achieved, 1),
                "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
                "frac": round(achieved / peaks["bf16_sustained"], 4), "traffic": traffic,
                "kernel": f"k_corr_tc<3,{lt}> (split-BF16, {lt} lags per tile, K in 2048-sample chunks)",
                "kernel_ms": round(k_ms, 2),
                "peak_source": f"{peaks['source']} bf16_tflops_sustained (the kernel runs ~0.8 s "
                               "inside a step)",
                "algorithmic_flops_per_launch": useful_flops,
                "work": "2M flops per lag-correlation, M = 4096; one launch = 4 series x 258049 "
                        "lags x 65536 templates",
                "issued_tflops": round(issued, 1),
                "issued_frac": round(issued / peaks["bf16_sustained"], 4),
                "issued_note": "split-BF16 issues three BF16 MMAs per operand pair (6M tensor "
                               "flops per lag-correlation); issued_frac is the tensor pipe's "
                               "load against the cuBLAS-measured rate"}
    # measured FP32 / FP64 FMA rates, the peaks of the ALU-bound paths
    alu = probe_alu(bf)

    # end to end through the public API with pinned host buffers
    e2e = run_e2e(args, ctx, bf, torch, w, xs_host, opts, corr_per_step)

    # plain FP32 SIMT path on the same workload (one step)
    fp32 = None
    if not args.no_fp32:
        fp32 = run_fp32(ctx, bf, torch, w, xs, ctrl, corr_per_step, alu)

    # the paper's FFT route on the same step
    fft = None
    if not args.no_fft:
        fft = run_fft(ctx, bf, w, xs, ctrl, corr_per_step, alu)

    # the split-FP16 tensor-core route on the same step
    f16 = None
    if not args.no_fp16:
        f16 = run_split_fp16(ctx, bf, w, xs, ctrl, corr_per_step)

    # oracle on a bounded sample, and accuracy of the timed path on that sample
    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu:
        cpu, accuracy = run_cpu_sample(ctx, bf, w, xs_host, args.cpu_templates)

    serve = None
    if rank == 0 and not args.no_serve:
        serve = run_serve(ctx, bf, synth, args)

    bf.bf_destroy(ctx)
    if serve is not None and not args.no_config5:
        serve["config5"] = run_config5(bf, synth)
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (split hi/lo operands, f32 accumulate)",
        "metric_unit_note": "one correlation = one template at one lag (a length-M normalised "
                            "inner product); the FP32 path and serving p50/p99 are in fp32_path "
                            "and serve",
        "data": "synthetic (seeded numpy PCG64; coloured Gaussian noise + power-law chirp)",
        "config": {"workload": "gw_pair: 2 x 262144 samples at 4096 Hz + 2 time-randomised "
                               "controls, 65536 power-law templates x 4096 samples",
                   "series": 4, "samples_per_series": N, "templates": K, "template_len": M,
                   "lags_per_series": L, "correlations_per_step": corr_per_step,
                   "precision": "split_bf16", "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (split bank 1.07 GB re-synthesised every step)",
                   "stages_in_step": ["bank_synthesis", "controls", "series_prep",
                                      "correlation+epilogue", "finalize+hist+map",
                                      "skew-normal fit of maxima",
                                      "coincidence pseudo-spectra (delta f 50 Hz)"]},
        "stage_ms": {k: round(float(np.mean(v)), 2) for k, v in stage_ms.items()},
        "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "alu_peaks": alu, "e2e": e2e,
        "fp32_path": fp32, "fft_path": fft, "split_fp16_path": f16, "accuracy_vs_oracle": accuracy, "cpu_baseline": cpu, "serve": serve,
        "maxima_fit": fits,
        "coincidence_counts": coincidences,
        "paper_unit": {
            "unit": "template-segment correlations/s: one template against one 16 s segment of "
                    "2^16 samples at all lags, i.e. 2^16 lag-correlations",
            "value": round(value / 65536.0),
            "e2e": round(e2e["value"] / 65536.0) if e2e else None,
            "fft_path": round(fft["value"] / 65536.0) if fft else None,
            "paper": "over one million per second on 12 AMD Fiji GPUs (FFT route, OpenCL): "
                     "context, another machine"},
    }


def run_e2e(args, ctx, bf, torch, w, xs_host, opts, corr_per_step):
    """The step end to end through the public API: inputs from pinned host
    memory, results back into pinned host memory. A step's results are copied
    on a second stream, into one of two sets of host buffers, while the next
    step's correlation runs (after its controls, whose device-to-host copies
    would otherwise queue behind them): maxima, argmaxes, sigmas and
    histograms by bf_result_copy_to_host_async, and each map's painted cells
    by bf_result_copy_map_cells_async (the map itself, cell by cell). The
    result and its bank are destroyed once the copies are done. The last
    step's copies run and end inside the timed region."""
    fs = w["fs"]
    seeds = w["control_seeds"]
    N = xs_host[0].numel()
    ctrl_host = [torch.empty_like(x).pin_memory() for x in xs_host]
    copy_stream = torch.cuda.Stream()
    res_host = None                     # two sets of pinned host buffers, allocated once
    done = []                           # (result, bank) not yet copied
    inflight = []                       # (result, bank, buffer set) whose copies are enqueued
    n_copied = 0
    d2h = [0]
    cells_max = [0]
    CELL_CAP = 1 << 20                  # painted cells per map that fit the buffers

    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()

    def enqueue_copies():
        nonlocal res_host, n_copied
        for res, bank in done:
            if res_host is None:
                K = bf.bf_result_info_get(res).n_templates
                nbins = bf.bf_result_info_get(res).hist_bins
                res_host = [[{"max": pinned((K,), torch.float32), "argmax": pinned((K,), torch.int32),
                              "sigma": pinned((K,), torch.float32),
                              "hist": pinned((nbins,), torch.int32).view(np.uint32),
                              "cell": pinned((CELL_CAP,), torch.int32).view(np.uint32),
                              "value": pinned((CELL_CAP,), torch.float32),
                              "count": pinned((1,), torch.int32).view(np.uint32)}
                             for s in range(4)] for _ in range(2)]
            d2h[0] = 0
            hs = res_host[n_copied % 2]
            for s in range(4):
                r = bf.bf_result_copy_to_host_async(res, s, hs[s], copy_stream.cuda_stream, want_hist=True)
                d2h[0] += sum(a.nbytes for a in r.values() if a is not None)
                bf.bf_result_copy_map_cells_async(res, s, hs[s]["cell"], hs[s]["value"], hs[s]["count"],
                                                  copy_stream.cuda_stream)
            n_copied += 1
            inflight.append((res, bank, hs))
        done.clear()

    def retire():
        copy_stream.synchronize()
        for res, bank, hs in inflight:
            for s in range(4):
                n = int(hs[s]["count"][0])
                if n > CELL_CAP:
                    raise RuntimeError(f"{n} painted cells: more than the {CELL_CAP} the buffers hold")
                cells_max[0] = max(cells_max[0], n)
                d2h[0] += 4 + 8 * n             # the count, then (cell, value) per painted cell
            bf.bf_result_destroy(res)
            bf.bf_bank_destroy(bank)
        inflight.clear()

    phases = {}

    def step(record=False):
        t = [time.perf_counter()]
        bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16)
        t.append(time.perf_counter())
        for x, c, sd in zip(xs_host, ctrl_host, seeds):
            bf.bf_control_randomize(ctx, x, sd, c)
        t.append(time.perf_counter())
        enqueue_copies()                                # the previous step's results
        res = bf.bf_correlate(ctx, bank, xs_host + ctrl_host, fs, opts)
        t.append(time.perf_counter())
        retire()
        t.append(time.perf_counter())
        done.append((res, bank))
        if record:
            for name, a, b in (("bank_synthesis", 0, 1), ("controls", 1, 2), ("correlate", 2, 3),
                               ("wait_for_previous_copies", 3, 4)):
                phases.setdefault(name, []).append(1e3 * (t[b] - t[a]))

    def flush():
        enqueue_copies()
        retire()

    step()
    flush()
    n = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(n):
        step(record=True)
    t_last = time.perf_counter()
    flush()
    last_ms = 1e3 * (time.perf_counter() - t_last)
    ev1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / n
    h2d = 2 * N * 4 + 4 * N * 4                     # control inputs + the four searched series
    out = {"value": corr_per_step / (ms / 1e3), "unit": UNIT, "ms_per_step": round(ms, 2),
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h[0] + 2 * N * 4,
           "steps": n, "inputs": "pinned host float32; each step's results copied on a second stream "
                                 "into pinned host buffers (two sets, allocated once) while the next "
                                 "step correlates: maxima, argmaxes, sigmas and histograms by "
                                 "bf_result_copy_to_host_async, each map's painted cells by "
                                 "bf_result_copy_map_cells_async (written by the kernels into mapped "
                                 "pinned memory); the last step's copies run and end inside the "
                                 "timed region",
           "map_cells_max": cells_max[0],
           "phase_ms": {k: round(float(np.mean(v)), 2) for k, v in phases.items()},
           "last_step_copies_ms": round(last_ms, 2),
           "clocks": clocks}
    return out


def probe_alu(bf) -> dict:
    """FP32 and FP64 FMA rates measured on this device (bf_probe_alu_peaks)."""
    import torch
    f32, f64 = bf.bf_probe_alu_peaks(torch.cuda.current_device())
    return {"fp32_tflops": round(f32, 2), "fp64_tflops": round(f64, 3),
            "how": "independent FMA chains filling every SM, best of three ~40 ms launches, "
                   "CUDA events; two flops per FMA"}


def run_fp32(ctx, bf, torch, w, xs, ctrl, corr_per_step, alu):
    fs = w["fs"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_FP32)
    warm = bf.make_opts(precision="fp32", bank_end=1024, want_map=True)
    bf.bf_result_destroy(bf.bf_correlate(ctx, bank, xs + ctrl, fs, warm))
    opts = bf.make_opts(precision="fp32", want_map=True, want_hist=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = bf.bf_correlate(ctx, bank, xs + ctrl, fs, opts)
    wall = time.perf_counter() - t0
    info = bf.bf_result_info_get(res)
    bf.bf_result_destroy(res)
    bf.bf_bank_destroy(bank)
    tflops = 2 * w["M"] * corr_per_step / (info.kernel_ms / 1e3) / 1e12
    return {"value": corr_per_step / wall, "unit": UNIT, "ms_per_step": round(1e3 * wall, 1),
            "kernel_ms": round(info.kernel_ms, 1),
            "kernel_tflops": round(tflops, 1),
            "roofline": {"bound": "alu", "achieved": round(tflops, 1), "peak": alu["fp32_tflops"],
                         "unit": "TFLOP/s", "frac": round(tflops / alu["fp32_tflops"], 4),
                         "peak_source": "measured FP32 FMA rate (alu_peaks)",
                         "work": "2M flops per lag-correlation, one FMA per sample pair"},
            "note": "bank synthesis excluded; same series, bank and outputs, FP32 SIMT kernel"}


def run_split_fp16(ctx, bf, w, xs, ctrl, corr_per_step, steps=3):
    """The same step on the split-FP16 tensor-core route: bank synthesised in
    the FP16 layout, series scaled by a power of two on the device, three
    FP16 MMAs per operand pair, histogram and map."""
    fs, M = w["fs"], w["M"]
    opts = bf.make_opts(precision="split_fp16", want_map=True, want_hist=True)

    def step():
        t0 = time.perf_counter()
        bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_FP16)
        res = bf.bf_correlate(ctx, bank, xs + ctrl, fs, opts)
        wall = time.perf_counter() - t0
        info = bf.bf_result_info_get(res)
        bf.bf_result_destroy(res)
        bf.bf_bank_destroy(bank)
        return wall, info.kernel_ms, info.tile_lags

    step()
    walls, kms, lts = zip(*[step() for _ in range(steps)])
    wall, k_ms = float(np.mean(walls)), float(np.mean(kms))
    return {"value": corr_per_step / wall, "unit": UNIT, "ms_per_step": round(1e3 * wall, 1),
            "kernel_ms": round(k_ms, 1), "tile_lags": sorted(set(lts)),
            "issued_tflops": round(3 * 2 * M * corr_per_step / (k_ms / 1e3) / 1e12, 1),
            "note": "bank synthesis included (FP16 hi/lo of 2^8 h); three FP16 MMAs per "
                    "operand pair into FP32, like split-BF16"}


def run_fft(ctx, bf, w, xs, ctrl, corr_per_step, alu, steps=3):
    """The same step through the FFT route (the paper's own route): bank from
    the chirp parameters, template spectra, segment spectra and the fused
    inverse-FFT correlation, with histogram and map."""
    fs, M = w["fs"], w["M"]
    opts = bf.make_opts(precision="fft_fp32", want_map=True, want_hist=True)

    def step():
        t0 = time.perf_counter()
        bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_GENERATED)
        res = bf.bf_correlate(ctx, bank, xs + ctrl, fs, opts)
        wall = time.perf_counter() - t0
        info = bf.bf_result_info_get(res)
        bf.bf_result_destroy(res)
        bf.bf_bank_destroy(bank)
        return wall, info.kernel_ms

    step()
    sampler = ClockSampler(torch_device_index())
    sampler.start()
    walls, kms = zip(*[step() for _ in range(steps)])
    clocks = sampler.stop()
    wall, k_ms = float(np.mean(walls)), float(np.mean(kms))
    N = 8192                      # complex points per transform
    V = 2 * N - M + 1             # lags per transform: one template, 16384-sample segments
    K = synth_grid_size(w)
    n_transforms = K * sum(-(-(x.numel() - M + 1) // V) for x in xs + ctrl)
    fft_flops = n_transforms * 5 * N * np.log2(N)
    return {"value": corr_per_step / wall, "unit": UNIT, "ms_per_step": round(1e3 * wall, 1),
            "kernel_ms": round(k_ms, 1),
            "kernel_value": corr_per_step / (k_ms / 1e3),
            "transforms": int(n_transforms),
            "fft_tflops_nominal": round(fft_flops / (k_ms / 1e3) / 1e12, 1),
            "roofline": {"bound": "alu", "achieved": round(fft_flops / (k_ms / 1e3) / 1e12, 1),
                         "peak": alu["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": round(fft_flops / (k_ms / 1e3) / 1e12 / alu["fp32_tflops"], 4),
                         "peak_source": "measured FP32 FMA rate (alu_peaks)",
                         "work": "5 N log2 N nominal flops per N-point complex transform",
                         "note": "on-chip bound: the profile puts shared-memory wavefronts and "
                                 "issue at about half their peaks each; no DRAM bound"},
            "roofline_smem": smem_roofline(n_transforms, k_ms, clocks),
            "clocks": clocks,
            "note": "FP32 complex FFTs of 8192 points carrying real segments of 16384 samples "
                    "(even/odd packing), overlap-save with 16385 - M lags per segment, one "
                    "template per transform; ms_per_step includes the template spectra "
                    "(computed from the chirp parameters every step); kernel_ms is the segment "
                    "spectra plus the correlation kernel; fft_tflops_nominal counts 5 N log2 N "
                    "per N-point complex transform"}


# shared-memory wavefronts per 8192-point transform of the real-route
# correlation kernel (ncu l1tex__data_pipe_lsu_wavefronts_mem_shared.sum over
# the transforms of the 16 s x 16,384-template case): the passes' loads and
# stores, twiddles, the mirror exchange, the staged segment spectrum and the
# final stage's loads
FFT_SMEM_WAVEFRONTS = 4170


def torch_device_index() -> int:
    import torch
    return torch.cuda.current_device()


def smem_roofline(n_transforms, k_ms, clocks):
    """The FFT route's shared-memory roofline: wavefronts per second over the
    SMs' peak of one wavefront per SM per cycle at the sampled SM clock."""
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clocks.get("sm_mhz") or None
    achieved = n_transforms * FFT_SMEM_WAVEFRONTS / (k_ms / 1e3)
    peak = n_sm * mhz * 1e6 if mhz else None
    return {"bound": "shared-memory wavefronts", "achieved": round(achieved / 1e9, 1),
            "peak": round(peak / 1e9, 1) if peak else None, "unit": "G wavefronts/s",
            "frac": round(achieved / peak, 4) if peak else None,
            "per_transform": FFT_SMEM_WAVEFRONTS,
            "note": "wavefronts per transform from ncu on the 16 s x 16,384-template case; peak = "
                    "one wavefront per SM per cycle at the median SM clock sampled during the "
                    "FFT steps; the kernel time includes the template and segment spectra"}


def synth_grid_size(w):
    from paper_1802_01685_gb300 import synth
    return synth.grid_size(w["grid"])


def run_cpu_sample(ctx, bf, w, xs_host, n_templates):
    import oracle
    fs, M = w["fs"], w["M"]
    g = w["grid"]
    p = oracle.grid(g["tracks"], g["senses"], g["durations"], g["f_min"], g["f_max"], g["I"], g["J"])
    K = len(p["track"])
    idx = np.linspace(0, K - 1, n_templates).astype(np.int64)
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}
    x = xs_host[0].numpy()
    t0 = time.perf_counter()
    ref = oracle.search(x, fs, sub, M)
    dt = time.perf_counter() - t0
    L = len(x) - M + 1
    cpu = {"value": n_templates * L / dt, "unit": UNIT, "cores": oracle.num_threads(),
           "kind": "oracle", "seconds": round(dt, 2),
           "sample": f"{n_templates} templates spread over the 65536-template bank x all "
                     f"{L} lags of series 0 (FP64 direct correlation, OpenMP over templates)"}
    # accuracy of the timed GPU path on the same sample
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16 | bf.BF_BANK_SPLIT_FP16)
    acc = {}
    for prec in ("split_bf16", "bf16", "fft_fp32", "split_fp16"):
        res = bf.bf_correlate(ctx, bank, [xs_host[0]], fs, bf.make_opts(precision=prec))
        got = bf.bf_result_copy_to_host(res, 0)
        bf.bf_result_destroy(res)
        err = np.abs(got["max"][idx].astype(np.float64) - ref["max"])
        acc[prec] = {"max_abs_err_of_max_rho": float(err.max()),
                     "argmax_equal": int((got["argmax"][idx] == ref["argmax"]).sum()),
                     "templates": int(n_templates)}
    bf.bf_bank_destroy(bank)
    return cpu, acc


def run_serve(ctx, bf, synth, args, precision="split_bf16", baseline=True):
    """Finite seeded stream of mixed requests (lengths 4-64 s, 2048/4096 Hz,
    Gaussian or Poisson-count, bank slices of 2^12..2^16 templates) arriving
    as a Poisson process; continuous batching; p50/p99 from submission.  The
    statistics are the context's, so each precision runs in a context of its
    own."""
    reqs = synth.serving_stream(seed=8, n_requests=args.serve_requests, rate_hz=args.serve_rate,
                                t_min=4.0, t_max=64.0, k_min_log2=12, k_max_log2=16)
    banks = {}
    for fs in (2048.0, 4096.0):
        spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0],
                               20.0, min(1000.0, fs / 2 - 24), 128, 128)
        banks[fs] = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_SPLIT_BF16)
    series = [synth.request_series(r) for r in reqs]
    t0 = time.perf_counter()
    tickets = []
    corr = 0.0
    for r, x in zip(reqs, series):
        while time.perf_counter() - t0 < r["arrival_s"]:
            time.sleep(0.0005)
        opts = bf.make_opts(precision=precision, bank_end=r["n_templates"])
        tickets.append(bf.bf_serve_submit(ctx, banks[r["fs"]], x, r["fs"], opts))
        corr += (len(x) - int(r["fs"]) + 1) * r["n_templates"]
    for t in tickets:
        st, res = bf.bf_serve_poll(ctx, t, -1)
        if res:
            bf.bf_result_destroy(res)
    wall = time.perf_counter() - t0
    s = bf.bf_serve_stats_get(ctx)
    for b in banks.values():
        bf.bf_bank_destroy(b)
    out = {"requests": len(reqs), "rate_hz": args.serve_rate, "p50_ms": round(s.p50_ms, 2),
           "p99_ms": round(s.p99_ms, 2), "sustained_correlations_per_s": corr / wall,
           "busy_correlations_per_s": s.correlations_per_s, "launches": int(s.launches),
           "precision": precision,
           "stream": "seeded Poisson arrivals; 4-64 s series; 2048/4096 Hz; 2^12-2^16 templates"}
    if baseline and not args.no_fp32:
        out["fp32_one_at_a_time"] = run_serve_fp32_baseline(ctx, bf, synth, reqs, series)
    if baseline and not args.no_fft:
        # the same stream through the FFT route, in a fresh context
        ctx2 = bf.bf_init()
        try:
            f = run_serve(ctx2, bf, synth, args, precision="fft_fp32", baseline=False)
        finally:
            bf.bf_destroy(ctx2)
        out["fft_route"] = {k: f[k] for k in ("p50_ms", "p99_ms", "sustained_correlations_per_s",
                                               "busy_correlations_per_s", "launches")}
    return out


def run_serve_fp32_baseline(ctx, bf, synth, reqs, series):
    """The same stream, replayed in real time through the plain FP32 path one
    request at a time (each waits for the previous one); latency from arrival."""
    banks = {}
    for fs in (2048.0, 4096.0):
        spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0],
                               20.0, min(1000.0, fs / 2 - 24), 128, 128)
        banks[fs] = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, bf.BF_BANK_FP32)
    lat, corr = [], 0.0
    t0 = time.perf_counter()
    for r, x in zip(reqs, series):
        while time.perf_counter() - t0 < r["arrival_s"]:
            time.sleep(0.0005)
        res = bf.bf_correlate(ctx, banks[r["fs"]], [x], r["fs"],
                              bf.make_opts(precision="fp32", bank_end=r["n_templates"]))
        bf.bf_result_copy_to_host(res, 0)
        bf.bf_result_destroy(res)
        lat.append(1e3 * (time.perf_counter() - t0 - r["arrival_s"]))
        corr += (len(x) - int(r["fs"]) + 1) * r["n_templates"]
    wall = time.perf_counter() - t0
    for b in banks.values():
        bf.bf_bank_destroy(b)
    lat = np.sort(np.array(lat))
    pct = lambda q: float(lat[min(len(lat) - 1, int(np.ceil(q * len(lat))) - 1)])
    return {"p50_ms": round(pct(0.5), 2), "p99_ms": round(pct(0.99), 2),
            "sustained_correlations_per_s": corr / wall}


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank, world, local):
    """The FP64 CPU oracle timed as it stands on the host cores, each step a
    bounded sample of the same workload: the four series (two data, two
    controls) against a fixed slice of the bank."""
    if rank != 0:
        return None
    import oracle
    from paper_1802_01685_gb300 import synth
    oracle.build()
    w = synth.gw_pair()
    fs, M = w["fs"], w["M"]
    g = w["grid"]
    p = oracle.grid(g["tracks"], g["senses"], g["durations"], g["f_min"], g["f_max"], g["I"], g["J"])
    K = len(p["track"])
    idx = np.linspace(0, K - 1, args.ref_templates).astype(np.int64)
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}
    series = list(w["series"]) + [oracle.permute(x, sd) for x, sd in zip(w["series"], w["control_seeds"])]
    L = len(series[0]) - M + 1

    def step():
        for x in series:
            oracle.search(x, fs, sub, M)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    corr = 4 * L * args.ref_templates
    v = corr / dt
    sample = (f"{args.ref_templates} of 65536 templates x 4 series x {L} lags per step "
              f"(FP64 direct correlation)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded numpy PCG64)",
            "config": {"workload": "gw_pair (bounded sample)", "templates_per_step": args.ref_templates},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_kernel_case(tile_lags: int, precision: str = "split_bf16"):
    """Moderate case of the correlation kernels for profiler captures: one
    16 s series at 4096 Hz against 16,384 power-law templates (split bank
    268 MB, template spectra 537 MB, both larger than L2); two launches of
    the given tile shape (no autotuner launches) or of the FFT route, each
    printed with its CUDA-event time."""
    from paper_1802_01685_gb300 import bf, synth
    import __graft_entry__
    __graft_entry__.build()
    w = synth.gw_pair(n=65536, I=128, J=128)
    ctx = bf.bf_init()
    storage = bf.BF_BANK_SPLIT_FP16 if precision == "split_fp16" else bf.BF_BANK_SPLIT_BF16
    bank = bf.bf_bank_create_grid(ctx, w["grid"], w["fs"], 1.0, storage)
    for _ in range(2):
        res = bf.bf_correlate(ctx, bank, [w["series"][0]], w["fs"],
                              bf.make_opts(precision=precision, tile_lags=tile_lags))
        info = bf.bf_result_info_get(res)
        print(json.dumps({"kernel_case": "gw_pair 16 s x 16384 templates", "precision": precision,
                          "kernel_ms": info.kernel_ms,
                          "tile_lags": info.tile_lags, "correlations": info.correlations}), flush=True)
        bf.bf_result_destroy(res)
    bf.bf_bank_destroy(bank)
    bf.bf_destroy(ctx)


def run_fft_step(steps: int, warmup: int):
    """The GW-pair step on the FFT route alone, for launch lists: the two
    series and their time-reversed copies (standing in for the controls,
    same lengths) against the 65,536-template bank made from its parameters
    (template spectra synthesised chunk by chunk), warm-up steps first; prints
    each timed step's wall and CUDA-event kernel times."""
    import torch
    from paper_1802_01685_gb300 import bf, synth
    import __graft_entry__
    __graft_entry__.build()
    w = synth.gw_pair()
    fs = w["fs"]
    ctx = bf.bf_init()
    xs = [torch.from_numpy(x).cuda() for x in w["series"]]
    xs = xs + [x.flip(0).contiguous() for x in xs]
    opts = bf.make_opts(precision="fft_fp32", want_map=True, want_hist=True)
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_GENERATED)
        res = bf.bf_correlate(ctx, bank, xs, fs, opts)
        wall = time.perf_counter() - t0
        info = bf.bf_result_info_get(res)
        if i >= warmup:
            print(json.dumps({"fft_step": i - warmup, "wall_ms": round(1e3 * wall, 2),
                              "kernel_ms": round(info.kernel_ms, 2)}), flush=True)
        bf.bf_result_destroy(res)
        bf.bf_bank_destroy(bank)
    bf.bf_destroy(ctx)


def run_workload_plan(ctx, bf, w, idx, ref):
    """The GRB batch as a plan: the 42-series search captured once as a CUDA
    graph (autotuned tile shape, one persistent correlation launch) and
    replayed on the same series; times the capture and two replays."""
    fs, xs = w["fs"], w["series"]
    bank = bf.bf_bank_create_grid(ctx, w["grid"], fs, 1.0, bf.BF_BANK_SPLIT_BF16)
    t0 = time.perf_counter()
    plan = bf.bf_plan_create(ctx, bank, [len(x) for x in xs], fs, bf.make_opts(precision="split_bf16"))
    t1 = time.perf_counter()
    runs = []
    try:
        for _ in range(2):
            ta = time.perf_counter()
            res = bf.bf_plan_run(plan, xs)
            info = bf.bf_result_info_get(res)
            runs.append(time.perf_counter() - ta)
        got = bf.bf_result_copy_to_host(res, 0)
    finally:
        bf.bf_plan_destroy(plan)
        bf.bf_bank_destroy(bank)
    return {"precision": "split_bf16", "capture_s": round(t1 - t0, 3),
            "replay_s": [round(r, 3) for r in runs], "tile_lags": int(info.tile_lags),
            "correlations_per_s": info.correlations / min(runs),
            "oracle_check": {"templates": len(idx), "series": 0,
                             "max_abs_err_of_max_rho": float(np.abs(got["max"][idx] - ref["max"]).max()),
                             "argmax_equal": int((got["argmax"][idx] == ref["argmax"]).sum())}}


def serve_stream(ctx, bf, banks, reqs, series, precision, time_scale=1.0):
    """Replays a request stream in real time (arrivals stretched by
    time_scale) through the serving loop; returns the loop's statistics and
    the wall time."""
    t0 = time.perf_counter()
    tickets = []
    for r, x in zip(reqs, series):
        while time.perf_counter() - t0 < r["arrival_s"] * time_scale:
            time.sleep(0.0005)
        opts = bf.make_opts(precision=precision, bank_end=r["n_templates"])
        tickets.append(bf.bf_serve_submit(ctx, banks[r["fs"]], x, r["fs"], opts))
    for t in tickets:
        st, res = bf.bf_serve_poll(ctx, t, -1)
        if res:
            bf.bf_result_destroy(res)
    return bf.bf_serve_stats_get(ctx), time.perf_counter() - t0


def run_config5(bf, synth, n_sustained=100):
    """The serving workload at its stated size: 200 requests arriving as a
    Poisson process at 50 per second, series of 4-256 s at 2048 or 4096 Hz,
    bank slices of 2^12..2^20 templates, an HBM budget of 150 GB.  That
    offered load is far above one GPU's capacity, so the first n_sustained
    requests are also replayed with the arrivals stretched to 70 % of the
    capacity measured in the offered run.  Split-BF16 (stored banks) with the
    shortest-first policy; the FFT route (generated banks: the stored spectra
    of two 2^20-template banks would not fit the budget) with both policies
    offered, shortest-first replayed.  Each run in a fresh context."""
    reqs = synth.serving_stream(seed=8, n_requests=200, rate_hz=50.0, t_min=4.0, t_max=256.0,
                                k_min_log2=12, k_max_log2=20)
    series = [synth.request_series(r) for r in reqs]

    def work(rs, xs):
        return float(sum((len(x) - int(r["fs"]) + 1) * r["n_templates"] for r, x in zip(rs, xs)))

    corr = work(reqs, series)
    out = {"workload": "serving: 200 requests, Poisson arrivals at 50/s, 4-256 s at 2048/4096 Hz, "
                       "2^12..2^20 templates, HBM budget 150 GB",
           "requests": len(reqs), "rate_hz": 50.0, "correlations": corr,
           "sustainable_requests": n_sustained}
    policies = {"shortest": bf.BF_SERVE_SHORTEST, "fair": bf.BF_SERVE_FAIR}
    runs = [("split_bf16", bf.BF_BANK_SPLIT_BF16, "shortest", "offered"),
            ("split_bf16", bf.BF_BANK_SPLIT_BF16, "shortest", "sustainable"),
            ("fft_fp32", bf.BF_BANK_GENERATED, "shortest", "offered"),
            ("fft_fp32", bf.BF_BANK_GENERATED, "fair", "offered"),
            ("fft_fp32", bf.BF_BANK_GENERATED, "shortest", "sustainable")]
    for precision, storage, policy, label in runs:
        res = out.setdefault(precision, {"banks": "stored split-BF16" if storage != bf.BF_BANK_GENERATED
                                         else "generated (spectra made per iteration per request)"})
        rs, xs = (reqs, series) if label == "offered" else (reqs[:n_sustained], series[:n_sustained])
        c = work(rs, xs)
        scale = 1.0
        if label == "sustainable":
            # arrivals stretched so the offered rate is ~70 % of the capacity just measured
            cap = res[f"offered_{policy}"]["busy_correlations_per_s"]
            scale = max(1.0, c / (0.7 * cap) / max(rs[-1]["arrival_s"], 1e-9))
        cfg = bf.bf_config_default()
        cfg.hbm_budget = 150 << 30
        cfg.serve_policy = policies[policy]
        ctx = bf.bf_init(cfg)
        try:
            banks = {}
            for fs in (2048.0, 4096.0):
                spec = synth.grid_spec([synth.LINEAR, synth.POWERLAW], [synth.ASC, synth.DESC], [1.0],
                                       20.0, min(1000.0, fs / 2 - 24), 512, 512)
                banks[fs] = bf.bf_bank_create_grid(ctx, spec, fs, 1.0, storage)
                # untimed: the autotuner's choice, the twiddle tables
                warm = np.zeros(int(2 * fs), np.float32)
                bf.bf_result_destroy(bf.bf_correlate(ctx, banks[fs], [warm], fs,
                                                     bf.make_opts(precision=precision, bank_end=4096)))
            st, wall = serve_stream(ctx, bf, banks, rs, xs, precision, scale)
            res[f"{label}_{policy}"] = {
                "rate_hz": round(50.0 / scale, 3), "requests": len(rs), "p50_ms": round(st.p50_ms, 1),
                "p99_ms": round(st.p99_ms, 1), "wall_s": round(wall, 1),
                "sustained_correlations_per_s": c / wall,
                "busy_correlations_per_s": st.correlations_per_s,
                "completed": int(st.completed), "rejected": int(st.rejected)}
            for b in banks.values():
                bf.bf_bank_destroy(b)
        finally:
            bf.bf_destroy(ctx)
    return out


def run_serving_workload():
    import __graft_entry__
    from paper_1802_01685_gb300 import bf, synth
    __graft_entry__.build()
    print(json.dumps(run_config5(bf, synth)), flush=True)


def k_block_fraction(p, fs, M):
    """Fraction of the 64-sample K blocks the tensor-core kernel runs: a
    128-template tile skips the blocks outside the union of its templates'
    supports (centred sweeps of round(D fs) samples; a descending support is
    the mirror of the ascending one)."""
    MD = np.floor(p["D"] * fs + 0.5).astype(np.int64)
    a0 = (M - MD) // 2
    a1 = a0 + MD
    lo = np.where(p["sense"] == 0, a0, np.where(p["sense"] == 1, M - a1, np.minimum(a0, M - a1)))
    hi = np.where(p["sense"] == 0, a1, np.where(p["sense"] == 1, M - a0, np.maximum(a1, M - a0)))
    K = len(MD)
    pad = -K % 128
    lo = np.concatenate([lo, np.full(pad, M)]).reshape(-1, 128).min(axis=1)
    hi = np.concatenate([hi, np.zeros(pad, np.int64)]).reshape(-1, 128).max(axis=1)
    blocks = -(-hi // 64) - lo // 64
    return float(blocks.sum() / (len(blocks) * -(-M // 64)))


def run_workload(name: str, n_check: int):
    """One timed search of a paper-sized workload other than the GW pair, with
    a sampled oracle check: 'grb_batch' (42 Poisson light curves of 20-200 s
    at 2000 Hz, 1,048,576 linear templates, one batched launch, mean
    spectrum) or 'full_bank' (32 s at 2048 Hz, 8,640,000 templates over both
    tracks, both senses and nine sweep times, stored and generated banks,
    histogram and map).  Each also runs through the FFT route: the GRB bank
    keeps its spectra (made in the untimed warm-up call), the full bank makes
    them chunk by chunk inside the timed call."""
    import oracle
    import __graft_entry__
    from paper_1802_01685_gb300 import bf, synth
    __graft_entry__.build()
    w = synth.grb_batch() if name == "grb_batch" else synth.full_bank()
    fs, M, xs = w["fs"], w["M"], w["series"]
    ctx = bf.bf_init()
    modes = [("stored", bf.BF_BANK_SPLIT_BF16, "split_bf16")]
    if name == "full_bank":
        modes.append(("generated", bf.BF_BANK_GENERATED, "split_bf16"))
        modes.append(("fft_generated", bf.BF_BANK_GENERATED, "fft_fp32"))
    else:
        modes.append(("fft_stored", bf.BF_BANK_SPLIT_BF16, "fft_fp32"))
    g = w["grid"]
    p = oracle.grid(g["tracks"], g["senses"], g["durations"], g["f_min"], g["f_max"], g["I"], g["J"])
    K = len(p["track"])
    idx = np.linspace(0, K - 1, n_check).astype(np.int64)
    sub = {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}
    out = {"workload": name, "series": len(xs), "samples": int(sum(len(x) for x in xs)),
           "templates": K, "template_len": M}
    ref = oracle.search(xs[0], fs, sub, M)
    if name == "grb_batch":
        out["plan"] = run_workload_plan(ctx, bf, w, idx, ref)
    for mode, storage, prec in modes:
        t0 = time.perf_counter()
        bank = bf.bf_bank_create_grid(ctx, g, fs, 1.0, storage)
        t1 = time.perf_counter()
        opts = bf.make_opts(precision=prec, want_map=(name == "full_bank"))
        warm = bf.make_opts(precision=prec, bank_end=4096)
        bf.bf_result_destroy(bf.bf_correlate(ctx, bank, xs, fs, warm))
        t2 = time.perf_counter()
        res = bf.bf_correlate(ctx, bank, xs, fs, opts)
        t3 = time.perf_counter()
        info = bf.bf_result_info_get(res)
        got = bf.bf_result_copy_to_host(res, 0)
        mean = bf.bf_result_copy_mean_max(res)
        bf.bf_result_destroy(res)
        bf.bf_bank_destroy(bank)
        out[mode] = {"precision": prec, "bank_create_s": round(t1 - t0, 3),
                     "warmup_s": round(t2 - t1, 3), "search_s": round(t3 - t2, 3),
                     "kernel_ms": round(info.kernel_ms, 1), "correlations": info.correlations,
                     "correlations_per_s": info.correlations / (t3 - t2),
                     "tails": int(info.n_candidates),
                     "oracle_check": {"templates": n_check, "series": 0,
                                      "max_abs_err_of_max_rho": float(np.abs(got["max"][idx] - ref["max"]).max()),
                                      "argmax_equal": int((got["argmax"][idx] == ref["argmax"]).sum()),
                                      "mean_of_maxima_finite": bool(np.all(np.isfinite(mean)))}}
        if prec != "fft_fp32":
            frac = k_block_fraction(p, fs, M)
            out[mode]["k_blocks_run"] = round(frac, 4)
            out[mode]["issued_tflops"] = round(3 * 2 * 64 * -(-M // 64) * frac * info.correlations
                                               / (info.kernel_ms / 1e3) / 1e12, 1)
    bf.bf_destroy(ctx)
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["gw_pair", "grb_batch", "full_bank", "serving"], default="gw_pair",
                    help="gw_pair is the benchmark line; the others print one measurement each")
    ap.add_argument("--check-templates", type=int, default=16)
    ap.add_argument("--kernel-case", action="store_true",
                    help="run only the moderate profiling case of the tensor-core kernel")
    ap.add_argument("--tile-lags", type=int, default=256,
                    help="tile shape of --kernel-case (256, the split routes' shape)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-fft", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--fft", action="store_true", help="--kernel-case: the FFT route")
    ap.add_argument("--fp16", action="store_true", help="--kernel-case: the split-FP16 route")
    ap.add_argument("--fft-step", action="store_true",
                    help="run only the GW-pair step on the FFT route (--steps timed after --warmup)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-config5", action="store_true",
                    help="skip the stated serving stream (200 requests at 50/s, about 10 minutes)")
    ap.add_argument("--cpu-templates", type=int, default=384)
    ap.add_argument("--ref-templates", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-rate", type=float, default=8.0)
    args = ap.parse_args()
    if args.kernel_case:
        run_kernel_case(args.tile_lags, "fft_fp32" if args.fft else
                        ("split_fp16" if args.fp16 else "split_bf16"))
        return
    if args.fft_step:
        run_fft_step(args.steps, args.warmup)
        return
    if args.workload == "serving":
        run_serving_workload()
        return
    if args.workload != "gw_pair":
        run_workload(args.workload, args.check_templates)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = dist_env()
    out = run_reference(args, rank, world, local) if args.impl == "reference" else \
        run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
