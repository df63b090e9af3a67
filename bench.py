#!/usr/bin/env python3
"""Benchmark: VEGAS events/s on one GB300 (LO Drell-Yan, 4 dims, 100 bins,
10 iterations x 1e6 calls, FP32 integrand with FP64/exact accumulation).

A step is one stage of that workload, one vegas_iterate call: 10 VEGAS
iterations, each every step of the hot path (Philox uniforms, grid map,
phase space and matrix element, the combination of all events and the grid
refinement; Section 2.1) over 1e6 events.  Steps are timed with CUDA events
on the library's launching stream (torch's current stream), the L2 cache is
flushed between steps, and the whole timed region is bracketed by a barrier
and a device synchronisation.  The same measurement with one iteration per
step is reported beside it (single_iteration).  See ``--help`` for the options;
``--impl reference`` times the CPU oracle instead (the reference arm).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NCALL = 1_000_000
ITMX = 10  # iterations per step: the workload's 10 x 1e6 calls
NDIM, NBINS = 4, 100
METRIC = "VEGAS events/s (LO Drell-Yan, d=4, 100 bins, 10 iterations x 1e6 calls)"
WORKLOAD = "drell_yan_lo_14tev_d4_n100_10x1e6calls"
UNIT = "events/s"
L2_FLUSH_BYTES = 256 << 20
# FP32 floating-point operations per event of the FP32 fills, counted from the
# source (gv_integrands.cuh, gv_fill.cuh): an fma counts 2, an add, multiply,
# division, square root or transcendental call (exp, log, sincos counted as
# 2) counts 1; integer work (Philox, bins, exact sums) is not counted.
#   Drell-Yan, d=4: grid map 4 x (fma + fma) = 16, integrand 83 arithmetic
#     operations + 8 transcendental calls + 3 divisions: 110.
#   3-jet, d=5: grid map 20; the cut test 4; an event inside the cuts adds
#     the momenta, the Euler rotation (18 + 45), the invariants and |M|^2:
#     144 in all, 24 for a cut event.  The cuts keep (1 - 3 y_cut)^2 / 2 =
#     0.4705 of the unit square, so 0.4705 x 144 + 0.5295 x 24 = 80.5.
#   NLO-shaped, d=13: Drell-Yan 110 + 9 more axes of grid map (36) and of
#     exp(beta cos 2 pi x)/I0 (8 each: 72) + 1 = 219.
#   Drell-Yan adjoint: forward 110 + reverse sweep 72 + 5 channel weights = 187.
FLOPS_PER_EVENT_FP32 = 16 + 83 + 8 + 3
FLOPS_EE3J_FP32 = 0.4705 * 144 + 0.5295 * 24
FLOPS_DYNLO_FP32 = 110 + 36 + 72 + 1
FLOPS_ADJOINT_FP32 = 110 + 72 + 5
# FP64 operations per event of the plain FP64 Drell-Yan fill (the same
# convention, with the table-driven exp (21 operations) and log (25), the
# library square root (15) and divisions (15 each) counted by their FP64
# operations): 83 + 3 x 21 + 25 + 15 + 3 x 15 + grid map 4 x 5 = 251.
FP64_OPS_PER_EVENT_DY = 83 + 3 * 21 + 25 + 15 + 3 * 15 + 4 * 5
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
# Per events-per-thread shape of the FP32 Drell-Yan fill (1e6 calls, 977
# tiles), from one-kernel ncu captures (profiles/fill_drell_yan_fp32_ept*_1e6.md):
# the DRAM bytes (read + write) of one launch, and its warp instructions
# (smsp__inst_executed.sum).  The fill is issue-bound, so its instruction rate
# against one warp instruction per cycle per SM sub-partition (4 per SM) is its
# binding roofline.  Valid while the fill's sources are the ones captured
# (their SHA-256 below) and only for the shape the timed run used; otherwise
# both are reported as unknown (null).
FILL_CAPTURES = {4: {"traffic_bytes": 83_456, "warp_instructions": 21_418_973},
                 8: {"traffic_bytes": 121_600, "warp_instructions": 19_412_189}}
SMSP_PER_SM = 4
FILL_SOURCES = ("gv_fill.cuh", "gv_fill_inst.cuh", "gv_fill_dy_f32.cu", "gv_integrands.cuh",
                "gv_common.cuh")
FILL_SOURCES_SHA256 = "b6e6780f442ab04756baca4c51db64638d12551e4734af9a48e958c1e9bed140"
# HBM copy bandwidth measured by the driver on the GB300s (used when
# MEASURED_PEAKS.json is absent: the profiling recipe's fallback)
HBM_FALLBACK_GBS = 6800.0


def _fill_sources_captured():
    import hashlib

    h = hashlib.sha256()
    try:
        for f in FILL_SOURCES:
            with open(os.path.join(ROOT, "paper_1503_06182_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return False
    return h.hexdigest() == FILL_SOURCES_SHA256


def _fill_capture(ept, key):
    """A captured figure of the fill at this events-per-thread shape (None if
    the sources changed since the capture or the shape was not captured)."""
    if not _fill_sources_captured():
        return None
    return FILL_CAPTURES.get(ept, {}).get(key)


def _fill_issue(fill_avg_ms, sm_mhz, ept):
    """The fill's warp-instruction issue rate against its peak (None if the
    sources changed since the capture, or the timed shape was not captured)."""
    wi = _fill_capture(ept, "warp_instructions")
    if wi is None or not fill_avg_ms:
        return None
    achieved = wi / (fill_avg_ms * 1e-3) / 1e12
    peak = SM_COUNT * SMSP_PER_SM * sm_mhz * 1e6 / 1e12
    return {"unit": "T warp instructions/s", "warp_instructions_per_launch": wi,
            "events_per_thread": ept,
            "instructions_per_event": wi * 32 / NCALL, "achieved": achieved,
            "peak": peak, "frac": achieved / peak,
            "peak_source": "derived: 152 SMs x 4 sub-partitions x 1 warp instruction per cycle "
                           "at the median SM clock of the timed region"}


def _fp32_peak_derived_tflops():
    """Dense FP32 peak from unit counts and the maximum SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def _hbm_peak():
    """(GB/s, source) of the HBM copy peak."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


def measure_peaks(v, ms=60.0):
    """The arithmetic pipes' rates on this GPU now (vegas_pipe_peak probes):
    FFMA and DFMA in TFLOP/s, IMAD and MUFU (ex2) in T ops/s."""
    return {"ffma_tflops": v.vegas_pipe_peak(v.VEGAS_PIPE_FFMA, ms) / 1e12,
            "dfma_tflops": v.vegas_pipe_peak(v.VEGAS_PIPE_DFMA, ms) / 1e12,
            "imad_tops": v.vegas_pipe_peak(v.VEGAS_PIPE_IMAD, ms) / 1e12,
            "mufu_ex2_tops": v.vegas_pipe_peak(v.VEGAS_PIPE_MUFU, ms) / 1e12,
            "how": "vegas_pipe_peak: 8 independent chains per thread, 8 x 256-thread CTAs "
                   "per SM, about 60 ms each, CUDA events, this run's clock"}


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the whole job is as slow as its
    slowest replica); the value itself on a single process."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 50):
        self.index, self.period = index, period_ms
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.period)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        return self

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0: float, t1: float):
        sel = [r for t, r in self.rows if t0 <= t <= t1] or [r for _, r in self.rows[-3:]]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        sm = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in sel for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(sel)}


# ---------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    from paper_1503_06182_gb300 import vegas as v
    from paper_1503_06182_gb300.workloads import DY, DY_PARAMS, SEED

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    seed = SEED + rank  # replicas draw independent events
    K, W = args.steps, args.warmup

    def make(precision):
        g = v.Vegas(NDIM, NBINS, seed, precision=precision)
        v.vegas_set_stream(g.h, stream.cuda_stream)
        if args.ept:
            g.set(v.VEGAS_OPT_EPT, args.ept)
        return g

    def timed_steps(g, nsteps, itmx=ITMX, flush_between=True):
        """Device time (ms) of each of nsteps stages of itmx iterations, L2
        flushed in between."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(nsteps)]
        with torch.cuda.stream(stream):
            for a, b in evs:
                if flush_between:
                    flush.fill_(1)
                a.record(stream)
                g.launch(NCALL, itmx, DY, DY_PARAMS)
                b.record(stream)
        stream.synchronize()
        res = g.fetch(itmx)
        return [a.elapsed_time(b) for a, b in evs], res

    sampler = ClockSampler(torch.cuda.current_device()).start() if rank == 0 else None
    g32 = make("fp32")
    # warm-up (also autotunes events per thread and captures the graphs)
    for _ in range(W):
        g32.iterate(NCALL, ITMX, DY, DY_PARAMS)
        g32.iterate(NCALL, 1, DY, DY_PARAMS)
    barrier()
    t_wall0 = time.time()
    step_ms, _ = timed_steps(g32, K)
    barrier()
    t_wall1 = time.time()
    tot_ms = max_over_ranks(sum(step_ms), dev)
    value = world * K * ITMX * NCALL / (tot_ms * 1e-3)

    # end to end through the blocking C ABI: host params in, host results out
    e2e_ms = []
    p = np.asarray(DY_PARAMS, dtype=np.float64)
    for _ in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        g32.iterate(NCALL, ITMX, DY, p)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_tot = max_over_ranks(sum(e2e_ms), dev)
    e2e_value = world * K * ITMX * NCALL / (e2e_tot * 1e-3)
    # the same with one iteration per step (each iteration a stage of its own)
    one_ms, _ = timed_steps(g32, K, itmx=1)
    one_tot = max_over_ranks(sum(one_ms), dev)
    t_wall2 = time.time()

    # roofline of the dominant kernel (fill): library-side CUDA events on the
    # same stream around every fill launch
    v.vegas_set_option(g32.h, v.VEGAS_OPT_TIMING, 1)
    kernels = (v.VEGAS_KERNEL_FILL, v.VEGAS_KERNEL_REDUCE)  # the refinement is in the reduce
    for kid in kernels:
        v.vegas_kernel_time(g32.h, kid, reset=True)
    for _ in range(max(K // ITMX, 5)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        g32.iterate(NCALL, ITMX, DY, DY_PARAMS)
    kavg = []
    for kid in kernels:
        ms, n = v.vegas_kernel_time(g32.h, kid)
        kavg.append(ms / max(n, 1))
    v.vegas_set_option(g32.h, v.VEGAS_OPT_TIMING, 0)
    fill_avg = kavg[0]
    achieved = FLOPS_PER_EVENT_FP32 * NCALL / (fill_avg * 1e-3) / 1e12
    peaks = measure_peaks(v)
    peak = peaks["ffma_tflops"]
    hbm, hbm_src = _hbm_peak()
    # the reduce (one launch per iteration): algorithmic bytes = the tile
    # partials and tile scales read, the FP64 sums written, the refined grid
    # pack (edges, widths, Jacobian factors in FP64 and FP32) rewritten
    n_tiles = (NCALL + 1023) // 1024
    nacc = 2 + NDIM * NBINS
    grid_pack = 8 * (3 * NDIM * NBINS + NDIM) + 4 * (4 * NDIM * NBINS + NDIM)
    red_bytes = n_tiles * nacc * 16 + n_tiles * 4 + nacc * 8 + grid_pack
    red_gbs = red_bytes / (kavg[1] * 1e-3) / 1e9

    # plain FP64 path and equal-error comparison: one 10-iteration stage of each
    # form from the same grid and seed (the same events)
    g64 = make("fp64")
    for _ in range(max(2, W // 2)):
        g64.iterate(NCALL, ITMX, DY, DY_PARAMS)
    k64 = max(3, min(K, 10))
    ms64, _ = timed_steps(g64, k64)
    value64 = world * ITMX * NCALL / (sum(ms64) / k64 * 1e-3)
    v.vegas_set_option(g64.h, v.VEGAS_OPT_TIMING, 1)
    v.vegas_kernel_time(g64.h, v.VEGAS_KERNEL_FILL, reset=True)
    g64.iterate(NCALL, ITMX, DY, DY_PARAMS)
    ms, n = v.vegas_kernel_time(g64.h, v.VEGAS_KERNEL_FILL)
    v.vegas_set_option(g64.h, v.VEGAS_OPT_TIMING, 0)
    fill64 = ms / max(n, 1)
    ach64 = FP64_OPS_PER_EVENT_DY * NCALL / (fill64 * 1e-3) / 1e12
    sig = {}
    for prec in ("fp32", "fp64"):
        g = v.Vegas(NDIM, NBINS, 4321, precision=prec)
        try:
            g.iterate(NCALL // 10, 5, DY, DY_PARAMS)  # warm-up stage (paper: 4 x 1,000)
            I, e, c, _, _ = g.iterate(NCALL, 10, DY, DY_PARAMS)
            sig[prec] = (I, e, c)
        finally:
            g.close()
    t32 = tot_ms / world / K
    t64 = sum(ms64) / k64
    eff_ratio = (1.0 / (sig["fp32"][1] ** 2 * t32)) / (1.0 / (sig["fp64"][1] ** 2 * t64))
    ept = v.vegas_get_ept(g32.h)
    g32.close()
    g64.close()
    form_rates = {} if args.no_forms else forms(v, stream, seed, peaks)

    clocks = sampler.summary(t_wall0 - 0.1, t_wall2 + 0.1) if sampler else None
    if sampler:
        sampler.stop()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    cpu = cpu_baseline(args) if (world == 1 and not args.no_cpu_baseline) else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": tot_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "integrand": "drell_yan",
                   "ndim": NDIM, "nbins": NBINS, "ncall_per_iteration": NCALL,
                   "itmx_per_step": ITMX,
                   "step": "one vegas_iterate stage of 10 iterations x 1e6 calls",
                   "precision": "fp32 integrand; Jacobian as fp32 mantissas times integer "
                                "exponents; exact integer sums rounded once to fp64",
                   "seed": 1234, "events_per_thread": ept,
                   "l2": "flushed between steps (256 MiB device write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        # per step: the 10 parameters in; the state (44 B) and 10 iteration
        # records (160 B) written by the device into mapped host memory
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 128,
                "d2h_bytes_per_step": 44 + 16 * ITMX},
        "gpu_launches": 2 * ITMX * K,
        "single_iteration": {"value": world * K * NCALL / (one_tot * 1e-3), "unit": UNIT,
                             "ms_per_iteration": one_tot / K,
                             "note": "one iteration per step (a stage of its own), L2 flushed"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": _fill_capture(ept, "traffic_bytes"),
                     "kernel": "gv_fill_kernel<drell_yan, float>",
                     "kernel_avg_ms": fill_avg, "reduce_refine_avg_ms": kavg[1],
                     "peak_source": "measured in this run: FFMA probe (vegas_pipe_peak)",
                     "peak_derived": _fp32_peak_derived_tflops(),
                     "frac_of_derived": achieved / _fp32_peak_derived_tflops(),
                     "flops_per_event": FLOPS_PER_EVENT_FP32,
                     "issue": _fill_issue(fill_avg, (clocks or {}).get("sm_mhz") or SM_MAX_MHZ,
                                          ept),
                     "reduce": {"kernel": "gv_reduce_slots_kernel (sums, refinement, record)",
                                "bound": "latency", "algorithmic_bytes": red_bytes,
                                "achieved_gbs": red_gbs, "peak_gbs": hbm,
                                "peak_source": hbm_src, "frac": red_gbs / hbm}},
        "peaks_measured": peaks,
        "fp64_path": {"value": value64, "unit": UNIT,
                      "roofline": {"bound": "fp64", "kernel": "gv_fill_kernel<drell_yan, double>",
                                   "kernel_avg_ms": fill64, "fp64_ops_per_event":
                                       FP64_OPS_PER_EVENT_DY, "achieved": ach64,
                                   "peak": peaks["dfma_tflops"], "unit": "TFLOP/s",
                                   "frac": ach64 / peaks["dfma_tflops"],
                                   "peak_source": "measured in this run: DFMA probe"}},
        "forms": form_rates,
        "equal_error": {"sigma_fp32": sig["fp32"][1], "sigma_fp64": sig["fp64"][1],
                        "integral_fp32": sig["fp32"][0], "integral_fp64": sig["fp64"][0],
                        "efficiency_ratio_fp32_over_fp64": eff_ratio},
        "clocks": clocks,
    }
    if cpu:
        out["cpu_baseline"] = cpu
        if not args.no_forms:
            out["cpu_baselines"] = cpu_baselines()
    print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def forms(v, stream, seed, peaks, only=None):
    """The other workloads, each a warm-up stage then one timed stage on the
    bench stream (device time between CUDA events; L2 not flushed inside a
    stage, as in a real run): 3-jet 10 x 1e7 FP32; Drell-Yan adjoint 10 x 1e8
    FP32 on a frozen grid; 64 batched integrations x 10 iterations (one graph);
    the plain FP64 Gauss case 5 x 1e5; the NLO-shaped 13-axis case 10 x 1e6
    FP32; Drell-Yan 10 x 1e6 FP32 filling a 60-bin m_ll histogram; Drell-Yan
    10 x 1e6 FP32 with VEGAS+ stratification, with its integration efficiency
    1/(sigma^2 t) against plain VEGAS on the same workload (each arm's time the
    median of five stages timed like the headline's).  Each FP32 form
    also reports its fill kernel's FP32 roofline fraction (a separate stage
    with per-kernel timing) and its difference from the FP64 form on the same
    events (the FP64 path matches the oracle to 1e-12)."""
    import numpy as np
    import torch

    from paper_1503_06182_gb300.workloads import (DY, DY_PARAMS, DYNLO, DYNLO_PARAMS, EE3J,
                                                  EE3J_PARAMS, GAUSS, GAUSS_PARAMS, batch_spec)

    ffma = peaks["ffma_tflops"]

    def want(name):
        return only is None or name in only

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            out = fn()
            b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b), out

    def fill_ms(g, fn):
        """Average fill-kernel time of one more stage, with per-kernel events."""
        v.vegas_set_option(g.h, v.VEGAS_OPT_TIMING, 1)
        v.vegas_kernel_time(g.h, v.VEGAS_KERNEL_FILL, reset=True)
        fn()
        ms, n = v.vegas_kernel_time(g.h, v.VEGAS_KERNEL_FILL)
        v.vegas_set_option(g.h, v.VEGAS_OPT_TIMING, 0)
        return ms / max(n, 1)

    def vs64(I, e, I64, e64, ms=None, ms64=None, events=None):
        r = {"integral_fp64": I64, "error_fp64": e64,
             "rel_diff_integral": abs(I - I64) / abs(I64),
             "diff_in_sigma": abs(I - I64) / e64 if e64 > 0 else None,
             "rel_diff_error": abs(e - e64) / e64 if e64 > 0 else None}
        if ms and ms64 and events:
            # events/s of the FP64 form, and the integration efficiency
            # 1/(sigma^2 t) of the FP32 form over the FP64 form's
            r["value_fp64"] = events / (ms64 * 1e-3)
            r["efficiency_ratio_fp32_over_fp64"] = (e64 ** 2 * ms64) / (e ** 2 * ms) if e > 0 else None
        return r

    res = {}
    for name, (iid, params, d, n, ncall, itmx, prec, hist, flops) in {
            "ee3j_d5_n100_10x1e7_fp32": (EE3J, EE3J_PARAMS, 5, 100, 10_000_000, 10, "fp32", None,
                                         FLOPS_EE3J_FP32),
            "gauss_d4_n50_5x1e5_fp64": (GAUSS, GAUSS_PARAMS, 4, 50, 100_000, 5, "fp64", None,
                                        None),
            "dy_nlo_shaped_d13_n50_10x1e6_fp32": (DYNLO, DYNLO_PARAMS, 13, 50, 1_000_000, 10,
                                                  "fp32", None, FLOPS_DYNLO_FP32),
            "dy_mll_hist60_d4_n100_10x1e6_fp32": (DY, DY_PARAMS, 4, 100, 1_000_000, 10, "fp32",
                                                  (60, 60.0, 120.0), FLOPS_PER_EVENT_FP32)}.items():
        if not want(name):
            continue
        out = {}
        edges = None
        for p in ((prec, "fp64") if prec == "fp32" else (prec,)):
            g = v.Vegas(d, n, seed, precision=p)
            v.vegas_set_stream(g.h, stream.cuda_stream)
            if hist:
                g.hist_set(*hist)
            try:
                g.iterate(ncall, itmx, iid, params)  # warm-up stage (adapts, tunes, captures)
                if edges is None:
                    edges = g.grid
                else:  # the FP64 form from the FP32 form's grid: the same events follow
                    g.grid = edges
                st = g.state()
                ms, (I, e, c, _, _) = timed(lambda: g.iterate(ncall, itmx, iid, params))
                hv = g.hist()[0] if hist else None
                fm = None
                if p == prec and flops:
                    g.restore(st)
                    fm = fill_ms(g, lambda: g.iterate(ncall, itmx, iid, params))
            finally:
                g.close()
            out[p] = (ms, I, e, c, fm, hv)
        ms, I, e, c, fm, hv = out[prec]
        r = {"value": ncall * itmx / (ms * 1e-3), "unit": UNIT, "integral": I, "error": e,
             "chi2_dof": c}
        if fm:
            ach = flops * ncall / (fm * 1e-3) / 1e12
            r["fill_roofline"] = {"fill_avg_ms": fm, "flops_per_event": flops,
                                  "achieved_tflops": ach, "frac_of_measured_ffma": ach / ffma}
        if "fp64" in out and prec == "fp32":
            r["fp32_vs_fp64"] = vs64(I, e, out["fp64"][1], out["fp64"][2], ms, out["fp64"][0],
                                     ncall * itmx)
            if hist:
                h32, h64 = hv, out["fp64"][5]
                nz = h64 != 0
                r["fp32_vs_fp64"]["hist_max_rel_diff_bin"] = float(
                    np.max(np.abs(h32[nz] - h64[nz]) / np.abs(h64[nz])))
        res[name] = r
    if want("dy_vegasplus_d4_n100_10x1e6_fp32"):
        # VEGAS+ against plain VEGAS: the same workload, events/s and efficiency
        # Each arm: a warm-up stage (grid and allocation adapt), then five
        # stages timed like the headline's (device events around the stage's
        # launch, L2 flushed before it): the time is their median, the result
        # the first one's.
        plus = {}
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=stream.device)
        for strat, prec in ((0, "fp32"), (1, "fp32"), (1, "fp64")):
            g = v.Vegas(NDIM, NBINS, seed, precision=prec)
            v.vegas_set_stream(g.h, stream.cuda_stream)
            g.set(v.VEGAS_OPT_STRAT, strat)
            try:
                g.iterate(NCALL, 10, DY, DY_PARAMS)
                ts, first = [], None
                for _ in range(5):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        flush.fill_(1)
                        a.record(stream)
                        g.launch(NCALL, 10, DY, DY_PARAMS)
                        b.record(stream)
                    out = g.fetch(10)
                    ts.append(a.elapsed_time(b))
                    first = first or out
                ms = float(np.median(ts))
                I, e, c = first[0], first[1], first[2]
            finally:
                g.close()
            plus[(strat, prec)] = (ms, I, e, c)
        ms, I, e, c = plus[(1, "fp32")]
        p0 = plus[(0, "fp32")]
        res["dy_vegasplus_d4_n100_10x1e6_fp32"] = {
            "value": NCALL * 10 / (ms * 1e-3), "unit": UNIT, "integral": I, "error": e, "chi2_dof": c,
            "events_note": "target 1e6 calls per iteration; VEGAS+ runs up to 1e6 + 2 nh",
            "error_plain_vegas": p0[2], "ms_plain_vegas": p0[0],
            "efficiency_ratio_over_plain": (p0[2] ** 2 * p0[0]) / (e ** 2 * ms),
            "fp32_vs_fp64": vs64(I, e, plus[(1, "fp64")][1], plus[(1, "fp64")][2], ms,
                                 plus[(1, "fp64")][0], NCALL * 10)}
    if want("dy_adjoint_d4_n100_10x1e8_fp32"):
        # gradient: frozen grid adapted by a forward warm-up, then the adjoint stage
        adj = {}
        edges = None
        for prec in ("fp32", "fp64"):
            g = v.Vegas(NDIM, NBINS, seed, precision=prec)
            v.vegas_set_stream(g.h, stream.cuda_stream)
            try:
                g.iterate(NCALL, 5, DY, DY_PARAMS)
                if edges is None:
                    edges = g.grid
                else:  # the FP64 gradient on the FP32 form's frozen grid: the same events
                    g.grid = edges
                g.set(v.VEGAS_OPT_ADAPT, 0)
                st = g.state()
                # warm-up stage of the timed size: events per thread are tuned per size
                g.adjoint(100_000_000, 10, DY_PARAMS)
                g.restore(st)
                ms, (grad, gerr, I, e, _) = timed(lambda: g.adjoint(100_000_000, 10, DY_PARAMS))
                fm = None
                if prec == "fp32":
                    g.restore(st)
                    fm = fill_ms(g, lambda: g.adjoint(100_000_000, 10, DY_PARAMS))
            finally:
                g.close()
            adj[prec] = (ms, np.asarray(grad), np.asarray(gerr), I, e, fm)
        ms, grad, gerr, I, e, fm = adj["fp32"]
        g64, ge64 = adj["fp64"][1], adj["fp64"][2]
        ach = FLOPS_ADJOINT_FP32 * 1e8 / (fm * 1e-3) / 1e12
        res["dy_adjoint_d4_n100_10x1e8_fp32"] = {
            "value": 1e9 / (ms * 1e-3), "unit": UNIT, "grad": list(grad), "grad_err": list(gerr),
            "fill_roofline": {"fill_avg_ms": fm, "flops_per_event": FLOPS_ADJOINT_FP32,
                              "achieved_tflops": ach, "frac_of_measured_ffma": ach / ffma},
            "fp32_vs_fp64": {"grad_fp64": list(g64), "value_fp64": 1e9 / (adj["fp64"][0] * 1e-3),
                             "max_diff_over_abs_plus_sigma":
                             float(np.max(np.abs(grad - g64) / (np.abs(g64) + ge64))),
                             "integral_rel_diff": abs(I - adj["fp64"][3]) / abs(adj["fp64"][3])}}
    if want("batch64_10it_fp32"):
        # batched: 64 integrations of uneven dimension, calls and integrand
        spec = batch_spec(64, seed)
        members = [(m.ndim, m.ncall, m.integrand, m.params) for m in spec]
        bat = {}
        for prec in ("fp32", "fp64"):
            B = v.VegasBatch(members, NBINS, seed, precision=prec)
            v.vegas_batch_set_stream(B.h, stream.cuda_stream)
            try:
                B.iterate(1)  # tunes events per thread
                B.iterate(10)  # captures the 10-iteration graph
                ms, out = timed(lambda: B.iterate(10))
            finally:
                B.close()
            bat[prec] = (ms, out)
        tot = sum(m.ncall for m in spec) * 10
        (ms, o32), o64 = bat["fp32"], bat["fp64"][1]
        # events-weighted FP32 flops of the members' integrands (the Gaussian:
        # grid map 4 d + d (sub, fma) + exp and scale 3)
        fl = {GAUSS: lambda d: 4 * d + 3 * d + 3, DY: lambda d: FLOPS_PER_EVENT_FP32 + 4 * (d - 4),
              EE3J: lambda d: FLOPS_EE3J_FP32 + 4 * (d - 5)}
        flops_b = sum(fl[m.integrand](m.ndim) * m.ncall for m in spec) / sum(m.ncall for m in spec)
        ach = flops_b * tot / (ms * 1e-3) / 1e12
        res["batch64_10it_fp32"] = {
            "value": tot / (ms * 1e-3), "unit": UNIT, "events_per_iteration": tot // 10,
            "stage_roofline": {"flops_per_event": flops_b, "achieved_tflops": ach,
                               "frac_of_measured_ffma": ach / ffma,
                               "note": "whole stage (fills, reduce, refinement) over the FFMA peak"},
            "fp32_vs_fp64": {"value_fp64": tot / (bat["fp64"][0] * 1e-3),
                             "max_rel_diff_integral": float(np.max(np.abs(o32[0] - o64[0]) /
                                                                    np.abs(o64[0]))),
                             "max_diff_in_sigma": float(np.max(np.abs(o32[0] - o64[0]) / o64[1]))}}
    if want("paper_shaped"):
        res["paper_shaped"] = paper_shaped(v, stream, seed, timed)
    return res


def run_only(names):
    """Only the named forms (for a profiler's launch list of one workload)."""
    import torch

    from paper_1503_06182_gb300 import vegas as v
    from paper_1503_06182_gb300.workloads import SEED

    stream = torch.cuda.Stream()
    peaks = {"ffma_tflops": v.vegas_pipe_peak(v.VEGAS_PIPE_FFMA, 20.0) / 1e12}
    print(json.dumps({"forms": forms(v, stream, SEED, peaks, only=set(names))}))


def paper_shaped(v, stream, seed, timed):
    """The paper's run shape (Section 3.2): a warm-up stage of 4 x 1,000 and a
    production stage of 10 x 10,000 events, here on the 10- and 13-axis
    Gaussian (the process of the paper is not available).  Latency-bound on
    a GPU: reported, not targeted."""
    from paper_1503_06182_gb300.workloads import GAUSS, GAUSS_PARAMS

    out = {}
    for d in (10, 13):
        for prec in ("fp64", "fp32"):
            g = v.Vegas(d, 50, seed, precision=prec)
            v.vegas_set_stream(g.h, stream.cuda_stream)
            try:
                g.iterate(1000, 4, GAUSS, GAUSS_PARAMS)  # tunes and captures
                g.iterate(10_000, 10, GAUSS, GAUSS_PARAMS)
                ms_w, _ = timed(lambda: g.iterate(1000, 4, GAUSS, GAUSS_PARAMS))
                ms_p, (I, e, c, _, _) = timed(lambda: g.iterate(10_000, 10, GAUSS, GAUSS_PARAMS))
            finally:
                g.close()
            out[f"gauss_d{d}_n50_4x1e3+10x1e4_{prec}"] = {
                "ms_warmup": ms_w, "ms_production": ms_p,
                "events_per_s": 104_000 / ((ms_w + ms_p) * 1e-3), "integral": I, "error": e}
    return out


# ---------------------------------------------------------------------------- CPU oracle
def _oracle_rate(seconds_target: float):
    """The oracle as it stands on this host's cores on a bounded sample of
    the same workload (whole 1e6-event iterations of the same config)."""
    import oracle
    from paper_1503_06182_gb300.workloads import DY, DY_PARAMS, SEED

    oracle.build()
    # calibrate with one iteration, then run a bounded number of iterations
    t0 = time.perf_counter()
    r = oracle.iterate(NDIM, NBINS, SEED, NCALL, 1, DY, DY_PARAMS)
    t1 = time.perf_counter() - t0
    n_it = max(1, min(200, int(seconds_target / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.iterate(NDIM, NBINS, SEED, NCALL, n_it, DY, DY_PARAMS, edges=r.edges,
                   iteration=r.iteration)
    dt = time.perf_counter() - t0
    return n_it * NCALL / dt, n_it, dt, oracle.get_threads()


def cpu_baseline(args):
    rate, n_it, dt, cores = _oracle_rate(args.cpu_seconds)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_it} iterations x 1e6 events of the same workload (FP64), {dt:.1f} s"}


def cpu_baselines():
    """The oracle (FP64, OpenMP over this host's cores) on every configuration,
    each on a bounded sample of its workload; events/s is the sample's rate.
    Also the per-core rate of the Gaussian configuration (one thread) and the
    paper-shaped runs.  A few seconds of CPU work in all."""
    import oracle
    from paper_1503_06182_gb300.workloads import (DY, DY_PARAMS, EE3J, EE3J_PARAMS, GAUSS,
                                                  GAUSS_PARAMS, SEED, batch_spec)

    oracle.build()
    cores = oracle.get_threads()
    out = {}

    def rate(name, events, fn, sample, reps=1, **extra):
        dt = float("inf")
        for _ in range(reps):  # the fastest of reps runs (short samples)
            t0 = time.perf_counter()
            fn()
            dt = min(dt, time.perf_counter() - t0)
        if reps > 1:
            sample += f" (fastest of {reps})"
        out[name] = {"value": events / dt, "unit": UNIT, "cores": extra.pop("cores", cores),
                     "kind": "oracle", "sample": f"{sample}, {dt:.3f} s", **extra}

    rate("gauss_d4_n50_5x1e5", 5 * 100_000,
         lambda: oracle.iterate(4, 50, SEED, 100_000, 5, GAUSS, GAUSS_PARAMS),
         "the whole 5 x 1e5 stage", reps=5)
    oracle.set_threads(1)
    try:
        rate("gauss_d4_n50_1e5_one_core", 100_000,
             lambda: oracle.iterate(4, 50, SEED, 100_000, 1, GAUSS, GAUSS_PARAMS),
             "one 1e5-event iteration on one thread", reps=5, cores=1)
    finally:
        oracle.set_threads(cores)
    r = oracle.iterate(5, 100, SEED, 1_000_000, 1, EE3J, EE3J_PARAMS)
    rate("ee3j_d5_n100_10x1e7", 10_000_000,
         lambda: oracle.iterate(5, 100, SEED, 10_000_000, 1, EE3J, EE3J_PARAMS, edges=r.edges,
                                iteration=1), "one 1e7-event iteration of the 10 x 1e7 stage")
    r = oracle.iterate(NDIM, NBINS, SEED, 1_000_000, 3, DY, DY_PARAMS)
    rate("dy_adjoint_d4_n100_10x1e8", 10_000_000,
         lambda: oracle.adjoint(NDIM, NBINS, SEED, 10_000_000, 1, DY_PARAMS, edges=r.edges,
                                iteration=3),
         "one 1e7-event gradient iteration; the workload is 10 x 1e8, so its rate is this "
         "sample's scaled linearly", scaled=True)
    spec = batch_spec(64, SEED)
    rate("batch64_1iteration", sum(m.ncall for m in spec),
         lambda: [oracle.iterate(m.ndim, NBINS, SEED, m.ncall, 1, m.integrand, m.params,
                                 batch=m.index) for m in spec],
         "one iteration of each of the 64 integrations, one after the other")
    for d in (10, 13):
        rate(f"gauss_d{d}_n50_4x1e3+10x1e4", 104_000,
             lambda: oracle.iterate(d, 50, SEED, 10_000, 10, GAUSS, GAUSS_PARAMS,
                                    edges=oracle.iterate(d, 50, SEED, 1000, 4, GAUSS,
                                                         GAUSS_PARAMS).edges, iteration=4),
             "the paper's run shape: 4 x 1,000 warm-up + 10 x 10,000 production events", reps=5)
    return out


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, same config and metric;
    each step one whole 1e6-event iteration."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1503_06182_gb300.workloads import DY, DY_PARAMS, SEED

    oracle.build()
    r = oracle.iterate(NDIM, NBINS, SEED, NCALL, max(1, args.warmup), DY, DY_PARAMS)
    edges, it = r.edges, r.iteration
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.iterate(NDIM, NBINS, SEED, NCALL, 1, DY, DY_PARAMS, edges=edges, iteration=it)
        times.append(time.perf_counter() - t0)
        edges, it = r.edges, r.iteration
    tot = sum(times)
    value = args.steps * NCALL / tot
    cores = oracle.get_threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "integrand": "drell_yan",
                   "ndim": NDIM, "nbins": NBINS, "ncall_per_iteration": NCALL,
                   "itmx_per_step": 1,
                   "step": "a bounded sample of the stage: one whole 1e6-event iteration",
                   "precision": "fp64 oracle (C + OpenMP), compensated sums"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} whole 1e6-event iterations"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def oracle_scaling(threads=None, runs=5, warmup=(4, 10_000), production=(10, 100_000), ndim=NDIM,
                   nbins=NBINS):
    """The paper's thread-scaling table (Section 3.2, Tables 1-8) for the
    oracle on this host's cores: a two-stage run (warm-up stage discarded,
    then the production stage, as in the paper's 4 x 1,000 + 10 x 10,000
    events, here scaled up since this integrand is far cheaper than MCFM's),
    timed `runs` times per thread count: min / avg / max, acceleration
    T_1 / T_n and efficiency acceleration / n.  Also checks the paper's
    invariant: the same result for every thread count."""
    import oracle
    from paper_1503_06182_gb300.workloads import DY, DY_PARAMS, SEED

    oracle.build()
    maxt = oracle.get_threads()
    if threads is None:
        threads = sorted({1, 2, 4, 8, maxt} | ({16} if maxt >= 16 else set()))
        threads = [t for t in threads if t <= maxt]
    rows, ref = [], None
    for t in threads:
        oracle.set_threads(t)
        times = []
        for _ in range(runs):
            t0 = time.perf_counter()
            w = oracle.iterate(ndim, nbins, SEED, warmup[1], warmup[0], DY, DY_PARAMS)
            r = oracle.iterate(ndim, nbins, SEED, production[1], production[0], DY, DY_PARAMS,
                               edges=w.edges, iteration=w.iteration)
            times.append(time.perf_counter() - t0)
        res = (r.integral, r.error)
        if ref is None:
            ref = res
        rows.append({"threads": t, "min_s": min(times), "avg_s": sum(times) / len(times),
                     "max_s": max(times), "integral": r.integral, "error": r.error,
                     "identical_to_1_thread": res == ref})
    oracle.set_threads(maxt)
    t1 = rows[0]["avg_s"]
    for row in rows:
        row["acceleration"] = t1 / row["avg_s"]
        row["efficiency"] = row["acceleration"] / row["threads"]
    return {"workload": f"drell_yan d={ndim} N={nbins}: {warmup[0]} x {warmup[1]} warm-up + "
                        f"{production[0]} x {production[1]} production, FP64 oracle",
            "runs": runs, "rows": rows}


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gvegas", "reference"], default="gvegas")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="CPU work of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ept", type=int, default=0, choices=(0, 1, 2, 4, 8),
                    help="events per thread of the fill kernel (0: autotuned)")
    ap.add_argument("--only", default=None,
                    help="comma-separated names of forms to run alone (profiling); prints "
                         "their results instead of the benchmark line")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the extra workloads reported under 'forms'")
    ap.add_argument("--oracle-scaling", action="store_true",
                    help="print the oracle's thread-scaling table (CPU only) and exit")
    args = ap.parse_args()
    if args.only:
        run_only(args.only.split(","))
        return
    if args.oracle_scaling:
        print(json.dumps({"oracle_scaling": oracle_scaling()}))
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
