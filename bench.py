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
# FP32 floating-point operations per event of the FP32 Drell-Yan fill, counted
# from the source: grid map 4 x (fma + fma) = 16; integrand 83 arithmetic
# operations (fma counted as 2) + 8 transcendental calls (3 exp, 4 log, 1 sqrt)
# counted as 1 each + 3 divisions counted as 1 each.
FLOPS_PER_EVENT_FP32 = 16 + 83 + 8 + 3
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes (read + write) of one fill launch of this workload, from the ncu
# capture summarised in profiles/fill_drell_yan_fp32_ept4_1e6.md, valid while
# the fill's sources are the ones captured (their SHA-256 below); otherwise the
# traffic is reported as unknown (null).
FILL_TRAFFIC_BYTES = 80_384
FILL_SOURCES = ("gv_fill.cuh", "gv_fill_inst.cuh", "gv_fill_dy_f32.cu", "gv_integrands.cuh",
                "gv_common.cuh")
FILL_SOURCES_SHA256 = "d2aaa5757c0a219f965c90d1e96b5eb96b1d1b014057b79110c2cda22077ca3c"


def _fill_traffic():
    import hashlib

    h = hashlib.sha256()
    try:
        for f in FILL_SOURCES:
            with open(os.path.join(ROOT, "paper_1503_06182_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return FILL_TRAFFIC_BYTES if h.hexdigest() == FILL_SOURCES_SHA256 else None


def _fp32_peak_tflops():
    """Dense FP32 peak from unit counts and the maximum SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


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
    peak = _fp32_peak_tflops()

    # plain FP64 path and equal-error comparison: one 10-iteration stage of each
    # form from the same grid and seed (the same events)
    g64 = make("fp64")
    for _ in range(max(2, W // 2)):
        g64.iterate(NCALL, ITMX, DY, DY_PARAMS)
    k64 = max(3, min(K, 10))
    ms64, _ = timed_steps(g64, k64)
    value64 = world * ITMX * NCALL / (sum(ms64) / k64 * 1e-3)
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
    form_rates = {} if args.no_forms else forms(v, stream, seed)

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
                   "precision": "fp32 integrand, fp64 Jacobian, exact integer sums",
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
                     "frac": achieved / peak, "traffic": _fill_traffic(),
                     "kernel": "gv_fill_kernel<drell_yan, float>",
                     "kernel_avg_ms": fill_avg, "reduce_refine_avg_ms": kavg[1],
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                     "flops_per_event": FLOPS_PER_EVENT_FP32},
        "fp64_path": {"value": value64, "unit": UNIT},
        "forms": form_rates,
        "equal_error": {"sigma_fp32": sig["fp32"][1], "sigma_fp64": sig["fp64"][1],
                        "integral_fp32": sig["fp32"][0], "integral_fp64": sig["fp64"][0],
                        "efficiency_ratio_fp32_over_fp64": eff_ratio},
        "clocks": clocks,
    }
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def forms(v, stream, seed):
    """The other workloads, each a warm-up stage then one timed stage on the
    bench stream (device time between CUDA events; L2 not flushed inside a
    stage, as in a real run): 3-jet 10 x 1e7 FP32; Drell-Yan adjoint 10 x 1e8
    FP32 on a frozen grid; 64 batched integrations x 10 iterations (one graph);
    the plain FP64 Gauss case 5 x 1e5; the NLO-shaped 13-axis case 10 x 1e6
    FP32; Drell-Yan 10 x 1e6 FP32 filling a 60-bin m_ll histogram; Drell-Yan
    10 x 1e6 FP32 with VEGAS+ stratification, with its integration efficiency
    1/(sigma^2 t) against plain VEGAS on the same workload."""
    import torch

    from paper_1503_06182_gb300.workloads import (DY, DY_PARAMS, DYNLO, DYNLO_PARAMS, EE3J,
                                                  EE3J_PARAMS, GAUSS, GAUSS_PARAMS, batch_spec)

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            out = fn()
            b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b), out

    res = {}
    for name, (iid, params, d, n, ncall, itmx, prec, hist) in {
            "ee3j_d5_n100_10x1e7_fp32": (EE3J, EE3J_PARAMS, 5, 100, 10_000_000, 10, "fp32", None),
            "gauss_d4_n50_5x1e5_fp64": (GAUSS, GAUSS_PARAMS, 4, 50, 100_000, 5, "fp64", None),
            "dy_nlo_shaped_d13_n50_10x1e6_fp32": (DYNLO, DYNLO_PARAMS, 13, 50, 1_000_000, 10,
                                                  "fp32", None),
            "dy_mll_hist60_d4_n100_10x1e6_fp32": (DY, DY_PARAMS, 4, 100, 1_000_000, 10, "fp32",
                                                  (60, 60.0, 120.0))}.items():
        g = v.Vegas(d, n, seed, precision=prec)
        v.vegas_set_stream(g.h, stream.cuda_stream)
        if hist:
            g.hist_set(*hist)
        try:
            g.iterate(ncall, itmx, iid, params)  # warm-up stage (adapts, tunes, captures)
            ms, (I, e, c, _, _) = timed(lambda: g.iterate(ncall, itmx, iid, params))
        finally:
            g.close()
        res[name] = {"value": ncall * itmx / (ms * 1e-3), "unit": UNIT, "integral": I,
                     "error": e, "chi2_dof": c}
    # VEGAS+ against plain VEGAS: the same workload, events/s and efficiency
    plus = {}
    for strat in (0, 1):
        g = v.Vegas(NDIM, NBINS, seed, precision="fp32")
        v.vegas_set_stream(g.h, stream.cuda_stream)
        g.set(v.VEGAS_OPT_STRAT, strat)
        try:
            g.iterate(NCALL, 10, DY, DY_PARAMS)  # warm-up stage: grid and allocation adapt
            ms, (I, e, c, _, _) = timed(lambda: g.iterate(NCALL, 10, DY, DY_PARAMS))
        finally:
            g.close()
        plus[strat] = (ms, I, e, c)
    ms, I, e, c = plus[1]
    res["dy_vegasplus_d4_n100_10x1e6_fp32"] = {
        "value": NCALL * 10 / (ms * 1e-3), "unit": UNIT, "integral": I, "error": e, "chi2_dof": c,
        "events_note": "target 1e6 calls per iteration; VEGAS+ runs up to 1e6 + 2 nh",
        "error_plain_vegas": plus[0][2], "ms_plain_vegas": plus[0][0],
        "efficiency_ratio_over_plain": (plus[0][2] ** 2 * plus[0][0]) / (e ** 2 * ms)}
    # gradient: frozen grid adapted by a forward warm-up, then the adjoint stage
    g = v.Vegas(NDIM, NBINS, seed, precision="fp32")
    v.vegas_set_stream(g.h, stream.cuda_stream)
    try:
        g.iterate(NCALL, 5, DY, DY_PARAMS)
        g.set(v.VEGAS_OPT_ADAPT, 0)
        # warm-up stage of the timed size: events per thread are tuned per size
        g.adjoint(100_000_000, 10, DY_PARAMS)
        ms, (grad, gerr, _, _, _) = timed(lambda: g.adjoint(100_000_000, 10, DY_PARAMS))
    finally:
        g.close()
    res["dy_adjoint_d4_n100_10x1e8_fp32"] = {"value": 1e9 / (ms * 1e-3), "unit": UNIT,
                                              "grad": list(grad), "grad_err": list(gerr)}
    # batched: 64 integrations of uneven dimension, calls and integrand
    spec = batch_spec(64, seed)
    members = [(m.ndim, m.ncall, m.integrand, m.params) for m in spec]
    B = v.VegasBatch(members, NBINS, seed, precision="fp32")
    v.vegas_batch_set_stream(B.h, stream.cuda_stream)
    try:
        B.iterate(1)  # tunes events per thread
        B.iterate(10)  # captures the 10-iteration graph
        ms, _ = timed(lambda: B.iterate(10))
    finally:
        B.close()
    tot = sum(m.ncall for m in spec) * 10
    res["batch64_10it_fp32"] = {"value": tot / (ms * 1e-3), "unit": UNIT,
                                "events_per_iteration": tot // 10}
    return res


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
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the extra workloads reported under 'forms'")
    ap.add_argument("--oracle-scaling", action="store_true",
                    help="print the oracle's thread-scaling table (CPU only) and exit")
    args = ap.parse_args()
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
