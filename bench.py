#!/usr/bin/env python3
"""Benchmark: FGGC reconstruction on one GB300 (and N independent GPUs).

Headline workload (default, --config 4): the 3-D WKB problem with eps = 1/64,
the 2^24 largest-amplitude packets of a 32^3 (q) x 16^3 (p) mesh, V = |x|^2/2,
propagated to t = 0.5 (RK4, dt = 1e-4, once, outside the timed region), output
256^3 points on [-pi, pi)^3, FP32 bulk arithmetic with FP64 phase reduction,
complex64 output, Q4P2 neighbours.

One step = one fgr_reconstruct_fggc call (A3-A5) on the device-resident
packets; value = packets / mean step time (CUDA events on the launching
stream; L2 flushed by a 512 MiB write between steps, outside the events).
Beside it: the direct sum (A2) of the same packets, the FGGC/direct speed-up
where their relative L2 difference is <= 1e-5, the end-to-end rate through
the C ABI with pinned host buffers, and the roofline of the step's dominant
kernel.  Extras: the 1-D pipeline with its RK4 step (workload 2), the 2-D
reconstruction (workload 3), batched requests, the serving workload and the
oracle on the host cores.

--impl reference runs the FP64 CPU oracle (the only reference this method has)
on a bounded packet sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "packets reconstructed/s, FGGC vs direct sum at rel L2<=1e-5; serving p50/p99 ms"
WORKLOADS = {
    1: "wkb-1d eps=1/64 grid=1024 M=4096 (64q x 64p) V=1-cos(x) t=0.5 fp64 Q4P2",
    2: "wkb-1d eps=1/1024 grid=32768 M=262144 (512q x 512p) V=1-cos(x) t=1.0 rk4 dt=1e-4 fp32/complex64 Q4P2",
    3: "wkb-2d eps=1/256 grid=1024^2 M=4194304 (64^2q x 32^2p) V=cos(x1)+cos(x2)+2 t=0.5 fp32/complex64 Q4P2",
    4: "wkb-3d eps=1/64 grid=256^3 M=16777216 (top 2^24 by |a| of 32^3q x 16^3p) V=|x|^2/2 t=0.5 "
       "fp32/complex64 Q4P2",
}
# FP64 FMA rate of this GB300 measured by a DFMA probe (2 FMA per clock per SM,
# 152 SMs at 2.07 GHz; nominal 1.26 TFLOP/s)
FP64_PEAK_TFLOPS = 1.19
# FP32 FMA rate measured by an FFMA probe on this GB300 (nominal 152 x 128 x 2
# x 2.07e9 = 80.5 TFLOP/s)
FP32_PEAK_TFLOPS = 74.6
# float2 reductions per second in L2 measured on this GB300 by a probe of
# reductions to random addresses of a 64 MiB buffer (one 8-byte reduction per
# lane, no two lanes of a warp on one 32-byte sector); 32 consecutive ones per
# warp reach 855e9 per second
L2_RED_PEAK_GPS = 222.8
L2_RED_COALESCED_GPS = 855.1
# TF32 tensor rate: the measured bf16 GEMM rate (MEASURED_PEAKS.json, burst)
# times the nominal TF32/bf16 ratio 1.1/2.25; a tcgen05.mma rate probe on this
# GB300 (M 128, K 8, operands in shared memory) measured 4093 FLOP per clock
# per SM at N >= 128 and 2725 at N = 64 (the direct sum's shape)
BF16_MEASURED_TFLOPS = 1933.7
TF32_PEAK_TFLOPS = BF16_MEASURED_TFLOPS * 1.1 / 2.25


def _rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:  # noqa: BLE001
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 5 + i and s[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of x over the ranks of the default process group (x itself for
    one rank).  Only timings cross ranks; every rank reconstructs its own batch."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rk4_nsteps(t: float, dt: float) -> int:
    """Step count rule of fgr_propagate (include/fgr.h)."""
    r = t / dt
    n = round(r)
    return int(n) if abs(r - n) <= 1e-9 * max(n, 1.0) else int(math.ceil(r))


# DRAM bytes (read + written) of one launch of the binned scatter kernel on the
# 3-D workload (d, packets), from the ncu launch list of the headline command
# (mean of 4 launches); to be retaken whenever the kernel changes.
SCATTER_TRAFFIC_BYTES = {(3, 16777216): 4148112512}
# Algorithmic FP64 work of one RK4 packet-step per dimension: 4 stages of
# about 40 FLOPs each.
RK4_ALG_FLOPS_PER_PACKET_STEP = 160
# FP64 FLOPs the RK4 kernel executes per packet-step (FMA = 2), counted by ncu
# on GB300 (DFMA x 2 + DMUL + DADD of rk4_kernel), 1-D cosine potential:
# 69.83 DFMA + 35.18 DMUL + 14.02 DADD (262144 packets, 100 steps).
RK4_EXEC_FLOPS_PER_PACKET_STEP = {(1, "cossum"): 188.86}
# DRAM bytes of one RK4 launch on the 1-D workload (ncu, same capture): the
# packet arrays are read once; the written state stays in L2 at kernel end.
RK4_TRAFFIC_BYTES = {(1, "cossum", 262144): 10530816}


def run_ours(args):
    """The headline: FGGC reconstruction of the 3-D workload (2^24 propagated
    packets onto 256^3 points, FP32/complex64, Q4P2).  One step = one
    fgr_reconstruct_fggc call on device-resident packets (its node-box zeroing,
    binning, coefficient scatter and grid passes); the packets are propagated
    once before the timed region.  The direct sum of the same packets, the
    FGGC/direct speed-up at equal accuracy, the end-to-end rate through the C
    ABI with pinned host buffers and the roofline of the step's dominant
    kernel are reported beside it."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads import config_workload

    rank, local, world = _rank_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w = config_workload(args.config)
    d, eps, grid = w["d"], w["eps"], w["grid"]
    pk = w["packets"]
    M = int(pk["s"].size)
    prec = fgr.FGR_FP32 if w["precision"] == "fp32" else fgr.FGR_FP64
    ctx = fgr.Context(d, grid, eps, fgr.make_options(precision=prec))
    pot = fgr.make_potential(**w["potential"])
    shape = tuple(grid["n"][:d])
    cdt = torch.complex64 if prec == fgr.FGR_FP32 else torch.complex128
    stream = torch.cuda.current_stream(dev)

    # packets at t = 0, propagated once (A1; outside the timed region)
    arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device=dev) for k in "qpsa"]
    packets = fgr.make_packets(*arrs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fgr.fgr_propagate(ctx.handle, packets, pot, w["t"], w["dt"], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    propagate_ms = e0.elapsed_time(e1)

    u_f = torch.zeros(shape, dtype=cdt, device=dev)
    u_d = torch.zeros(shape, dtype=cdt, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
    torch.cuda.synchronize()
    # the library's per-stage CUDA events (recorded on this stream) give the
    # dominant kernel's own duration in every timed step (level 1: events only;
    # the grid passes' term count takes an extra kernel per pass and is taken
    # once after the timed steps)
    fgr.fgr_set_timing(ctx.handle, 1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage = {"prep_ms": [], "bin_ms": [], "scatter_ms": [], "grid_ms": [], "pass_ms": [], "pass_terms": []}
    launches = 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()                      # L2 flushed between steps, outside the events
            evs[i][0].record(stream)
            fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
            evs[i][1].record(stream)
            st = fgr.fgr_get_stats(ctx.handle)
            stage["prep_ms"].append(st.prep_ms)
            stage["bin_ms"].append(st.coeff_ms)
            stage["scatter_ms"].append(st.scatter_ms)
            stage["grid_ms"].append(st.grid_ms)
            stage["pass_ms"].append(st.pass_ms)
            launches += int(st.launches)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    fgr.fgr_set_timing(ctx.handle, 2)
    fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
    stage["pass_terms"].append(fgr.fgr_get_stats(ctx.handle).pass_terms)
    fgr.fgr_set_timing(ctx.handle, False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    nodes = int(fgr.fgr_get_stats(ctx.handle).nodes)

    # the direct sum of the same packets (A2) and the other FGGC variants
    recon = reconstruct_runs(fgr, ctx, packets, u_d, grid, d, eps, prec, flush, stream, None, runs=20,
                             direct_runs=args.direct_runs)
    ud, uf = u_d.cpu().numpy(), u_f.cpu().numpy()
    rel = float(np.linalg.norm(uf - ud) / max(np.linalg.norm(ud), 1e-300))
    droof = None
    if d >= 2 and prec == fgr.FGR_FP32:
        droof = direct_roofline(window_pairs(arrs[0].cpu().numpy(), grid, eps), recon["direct"]["median_ms"])

    # end to end through the C ABI: packets in pinned host memory, u back to
    # pinned host memory, both copies inside the timed region
    host = [torch.empty(x.shape, dtype=x.dtype, pin_memory=True) for x in arrs]
    for h, x in zip(host, arrs):
        h.copy_(x)
    hpk = fgr.make_packets(*[h.numpy() for h in host])
    hu = torch.empty(shape, dtype=cdt, pin_memory=True)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fgr.fgr_reconstruct_fggc(ctx.handle, hpk, hu.numpy())   # H2D of the packets, D2H of u
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_rel = float(np.linalg.norm(hu.numpy() - uf) / max(np.linalg.norm(uf), 1e-300))
    h2d = sum(h.numel() * h.element_size() for h in host)
    d2h = hu.numel() * hu.element_size()
    del host, hu

    def agg(xs):
        return max_over_ranks(statistics.mean(xs), world)

    ms_step = agg(step_ms)
    ms_e2e = agg(e2e_ms)
    kern = {k: statistics.mean(v) for k, v in stage.items()}
    roof = reconstruction_roofline(d, M, nodes, kern, ms_step)
    total_packets = M * world
    out = None
    if rank == 0:
        direct = recon["direct"]
        out = {
            "metric": METRIC,
            "value": total_packets / (ms_step * 1e-3),
            "unit": "packets/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32/complex64 reconstruction (f64 phase reduction); f64 trajectories (untimed)",
            "data": "synthetic (seeded analytic WKB data, cut-off FFT initial decomposition)",
            "config": {"workload": WORKLOADS[args.config], "packets_per_gpu": M, "grid": list(shape),
                       "eps": eps, "strategy": "Q4P2 cq=1/2 cp=pi/8",
                       "step": "fgr_reconstruct_fggc of the propagated packets (A3-A5), device-resident",
                       "l2": "flushed (512 MiB write) between timed steps, outside the events",
                       "parallelism": "replicas"},
            "headline": {
                "fggc_packets_per_s": total_packets / (ms_step * 1e-3),
                "fggc_ms_mean": ms_step, "fggc_ms_median": statistics.median(step_ms),
                "fggc_ms_min": min(step_ms), "fggc_ms_max": max(step_ms),
                "direct_packets_per_s": direct["packets_per_s"], "direct_ms_median": direct["median_ms"],
                "direct_runs": direct["runs"], "direct_path": direct.get("path", "CUDA cores"),
                "direct_roofline": droof,
                "speedup_fggc_over_direct": (direct["median_ms"] / statistics.median(step_ms)
                                             if rel <= 1e-5 else "not at equal accuracy"),
                "rel_l2_fggc_vs_direct": rel,
                "propagate_ms_untimed": propagate_ms,
                "fggc_stage_ms_mean": kern, "nodes": nodes,
            },
            "stages": {"reconstruct_runs": recon},
            "roofline": roof,
            "e2e": {"value": total_packets / (ms_e2e * 1e-3), "unit": "packets/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "call": "fgr_reconstruct_fggc with pinned host packets and a pinned host output",
                    "rel_l2_vs_device_call": e2e_rel},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
    ctx.close()
    del arrs, packets, u_f, u_d
    torch.cuda.empty_cache()
    if rank == 0:
        if args.extra:
            out["workloads"] = {}
            for cfg in [int(x) for x in args.extra.split(",") if x]:
                if cfg == 2:
                    out["workloads"]["config2_pipeline"] = pipeline_bench(2, args, flush)
                else:
                    out["workloads"]["config%d" % cfg] = reconstruct_bench(cfg, args, flush)
        if args.fft:
            out["fft_grid_stage"] = fft_grid_bench(args, flush)
        if args.batch:
            out["batched_direct"] = batch_bench(args, flush)
        if args.serving:
            out["serving"] = serving_bench(args, local)
        if args.cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, args)
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def reconstruction_roofline(d, M, nodes, kern, ms_step):
    """Roofline block of the FGGC step's dominant kernel, from the library's
    per-stage CUDA events of the timed steps (kern: mean per stage).

    Scatter (K3+K4): unit = one contribution A e^{iS/eps} c_k of a packet to a
    node (eq. 2.25), an 8-byte reduction in L2 as the method states it, M 8^d
    per launch (Q4P2), against the best rate at which this GB300's L2 absorbs
    8-byte reductions (a warp on 32 consecutive cells, probed); the binned 3-D
    kernel sums a cell's contributions in registers first, so it issues fewer
    reductions than contributions.  Grid passes (K5): unit = one node-point
    term W[a, b] g(x_m - a dq) (a real x complex multiply-add, 4 FLOPs), counted
    on the device per launch (occupied b-range x window points over every
    (row, a) line), against the measured FP32 FMA rate."""
    contrib = M * 8 ** d
    scatter_ms, pass_ms = kern["scatter_ms"], kern["pass_ms"]
    if scatter_ms >= pass_ms:
        out = {"kernel": "coefficient + scatter (K3+K4: binned_scatter_kernel in 3-D)", "bound": "l2",
               "achieved": contrib / (scatter_ms * 1e-3) / 1e9, "peak": L2_RED_COALESCED_GPS,
               "unit": "G contributions/s", "traffic": SCATTER_TRAFFIC_BYTES.get((d, M)),
               "launch_ms": scatter_ms, "units_per_launch": contrib,
               "unit_def": "one contribution of a packet to a node (eq. 2.25): an 8-byte L2 reduction as the "
                           "method states it; M 8^d per launch",
               "peak_source": "float2 reductions by warps on 32 consecutive cells of a 64 MiB buffer, probe on "
                              "this GB300 (scattered ones: 222.8e9/s)"}
    else:
        terms = kern["pass_terms"]
        out = {"kernel": "grid_pass_kernel (K5, all passes)", "bound": "alu",
               "achieved": 4.0 * terms / (pass_ms * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
               "unit": "TFLOP/s", "traffic": None, "launch_ms": pass_ms,
               "units_per_launch": terms,
               "unit_def": "one node-point term W[a,b] g(x_m - a dq): a real x complex multiply-add (4 FLOPs); "
                           "per pass the occupied b-range x window points of every (row, a) line",
               "peak_source": "FFMA probe on this GB300 (74.6 TFLOP/s; nominal 80.5 at 2.07 GHz)"}
    out["frac"] = out["achieved"] / out["peak"]
    out["share_of_step"] = out["launch_ms"] / ms_step
    out["stage_ms"] = {"scatter": scatter_ms, "passes": pass_ms}
    return out


def window_pairs(q, grid, eps, R=6.0):
    """Packet-point pairs inside the box windows (the rule of the direct sum:
    m_lo = ceil((Q - R sqrt(eps) - lo) / h), m_hi = floor((Q + R sqrt(eps) - lo) / h),
    clipped to the grid), summed over the packets."""
    import numpy as np
    d = int(grid["d"])
    rs = R * np.sqrt(eps)
    prod = np.ones(q.shape[1], dtype=np.float64)
    for l in range(d):
        n, lo = int(grid["n"][l]), float(grid["lo"][l])
        h = (float(grid["hi"][l]) - lo) / n
        mlo = np.maximum(np.ceil((q[l] - rs - lo) / h), 0)
        mhi = np.minimum(np.floor((q[l] + rs - lo) / h), n - 1)
        prod *= np.maximum(mhi - mlo + 1, 0)
    return float(prod.sum())


def direct_roofline(pairs, direct_ms):
    """Roofline block of the direct sum (FP32, d >= 2: tcgen05 kernel).  Unit:
    a packet-point pair inside the windows, one complex multiply-add (8 real
    FLOPs) run on the tensor pipe as three TF32 products (hi x hi, hi x lo,
    lo x hi): 24 TF32 FLOPs per pair, against the TF32 tensor rate."""
    ach = 24.0 * pairs / (direct_ms * 1e-3) / 1e12
    return {"kernel": "direct_tc_kernel (K2 on tcgen05, 3 x TF32)", "bound": "tensor", "achieved": ach,
            "peak": TF32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / TF32_PEAK_TFLOPS,
            "units_per_launch": pairs, "pairs_per_s": pairs / (direct_ms * 1e-3), "launch_ms": direct_ms,
            "unit_def": "packet-point pair inside the windows = one complex multiply-add, 24 TF32 FLOPs as "
                        "three TF32 products",
            "peak_source": "measured bf16 GEMM rate x nominal TF32/bf16 ratio 1.1/2.25 (of measured)"}


def pipeline_bench(cfg: int, args, flush):
    """The 1-D workload as a whole pipeline: copy the t = 0 packets into the
    working buffers, fgr_propagate (A1, 10^4 RK4 steps), fgr_reconstruct_fggc
    (A3-A5) and fgr_reconstruct_direct (A2) of the same batch; CUDA events
    between the calls give the stage times; the roofline of the RK4 launch."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads import config_workload

    w = config_workload(cfg)
    d, eps, grid = w["d"], w["eps"], w["grid"]
    pk = w["packets"]
    M = int(pk["s"].size)
    prec = fgr.FGR_FP32 if w["precision"] == "fp32" else fgr.FGR_FP64
    ctx = fgr.Context(d, grid, eps, fgr.make_options(precision=prec))
    pot = fgr.make_potential(**w["potential"])
    t_final, dt = w["t"], w["dt"]
    shape = tuple(grid["n"][:d])
    cdt = torch.complex64 if prec == fgr.FGR_FP32 else torch.complex128
    init = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
    work = [x.clone() for x in init]
    packets = fgr.make_packets(*work)
    u_f = torch.zeros(shape, dtype=cdt, device="cuda")
    u_d = torch.zeros(shape, dtype=cdt, device="cuda")
    stream = torch.cuda.current_stream()

    def step(ev=None):
        for wbuf, ibuf in zip(work, init):
            wbuf.copy_(ibuf)
        if ev:
            ev[0].record(stream)
        fgr.fgr_propagate(ctx.handle, packets, pot, t_final, dt, stream)
        if ev:
            ev[1].record(stream)
        fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
        if ev:
            ev[2].record(stream)
        fgr.fgr_reconstruct_direct(ctx.handle, packets, u_d, stream)
        if ev:
            ev[3].record(stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    fgr.fgr_autotune(ctx.handle, packets, u_d, 3, stream)
    tuning = fgr.fgr_get_tuning(ctx.handle)
    nsteps = 5
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(nsteps)]
    for i in range(nsteps):
        flush.zero_()
        step(evs[i])
    torch.cuda.synchronize()
    prop_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    fggc_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    direct_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    step_ms = statistics.mean(e[0].elapsed_time(e[3]) for e in evs)
    ud, uf = u_d.cpu().numpy(), u_f.cpu().numpy()
    rel = float(np.linalg.norm(uf - ud) / max(np.linalg.norm(ud), 1e-300))
    droof = None
    if d >= 2 and prec == fgr.FGR_FP32:
        droof = direct_roofline(window_pairs(arrs[0].cpu().numpy(), grid, eps), recon["direct"]["median_ms"])
    recon = reconstruct_runs(fgr, ctx, packets, u_d, grid, d, eps, prec, flush, stream, ud, runs=20)
    decomp = decompose_runs(fgr, ctx, w, init, pot, stream, flush, runs=20)
    fgr.fgr_set_timing(ctx.handle, True)
    fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
    st = fgr.fgr_get_stats(ctx.handle)
    fggc_stages = {"prep_ms": st.prep_ms, "bin_ms": st.coeff_ms, "coeff_scatter_ms": st.scatter_ms,
                   "grid_ms": st.grid_ms, "nodes": int(st.nodes)}
    fgr.fgr_set_timing(ctx.handle, False)
    kind = w["potential"]["kind"]
    steps_rk4 = rk4_nsteps(t_final, dt)
    # algorithmic FP64 work of one packet-step (4 stages, about 40 d FLOPs
    # each) against the measured DFMA rate; the FLOPs the kernel executes
    # (counted by ncu) are kept beside it
    alg = RK4_ALG_FLOPS_PER_PACKET_STEP * d * M * steps_rk4
    exe = RK4_EXEC_FLOPS_PER_PACKET_STEP.get((d, kind))
    ctx.close()
    return {
        "workload": WORKLOADS[cfg], "packets": M,
        "step": "propagate (A1) + fggc reconstruct (A3-A5) + direct sum (A2), same batch, 5 steps",
        "step_ms": step_ms, "packets_per_s": M / (step_ms * 1e-3),
        "propagate_ms": prop_ms, "fggc_ms": fggc_ms, "direct_ms": direct_ms,
        "fggc_packets_per_s": M / (fggc_ms * 1e-3), "direct_packets_per_s": M / (direct_ms * 1e-3),
        "rel_l2_fggc_vs_direct": rel,
        "reconstruct_20_runs": recon, "decompose_20_runs": decomp, "fggc_stage_split": fggc_stages,
        "autotuned": {"direct_ctas_per_sm": tuning[0], "grid_pass_ctas_per_sm": tuning[1],
                      "grid_pass_tile": tuning[2]},
        "rk4_roofline": {"kernel": "rk4_kernel (fgr_propagate)", "bound": "alu",
                         "achieved": alg / (prop_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": alg / (prop_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "flops_per_launch": alg,
                         "flops_counted": "algorithmic: 4 stages x 40 d FP64 FLOPs per packet-step",
                         "peak_source": "DFMA probe on this GB300 (2 FP64 FMA per clock per SM at 2.07 GHz)",
                         "executed_flops_per_packet_step": exe,
                         "traffic": RK4_TRAFFIC_BYTES.get((d, kind, M))},
    }


def reconstruct_runs(fgr, ctx, packets, u_ref, grid, d, eps, prec, flush, stream, ud, runs=20, direct_runs=None):
    """Median/min/max ms of `runs` reconstructions per method (`direct_runs`
    for the direct sum, whose 3-D runs take seconds); FGGC with the Q4P2 and
    Q2P2 neighbour sets and Q4P2 through a plan, relative L2 difference from
    the direct sum.  The direct sum is left in u_ref; with ud None its result
    becomes the reference."""
    import numpy as np
    import torch

    q2 = fgr.Context(d, grid, eps, fgr.make_options(precision=prec, nq=2, np_=2))
    out = {}
    methods = [("direct", fgr.fgr_reconstruct_direct, ctx), ("fggc_q4p2", fgr.fgr_reconstruct_fggc, ctx),
               ("fggc_q2p2", fgr.fgr_reconstruct_fggc, q2)]
    fma = None
    if d >= 2 and prec == fgr.FGR_FP32:
        # the direct sum on the CUDA cores (FGR_FLAG_DIRECT_FMA) beside the default tensor-core path
        fma = fgr.Context(d, grid, eps, fgr.make_options(precision=prec, flags=fgr.FGR_FLAG_DIRECT_FMA))
        methods.insert(1, ("direct_cuda_cores", fgr.fgr_reconstruct_direct, fma))
    for name, fn, c in methods:
        u = u_ref if name == "direct" else torch.zeros_like(u_ref)
        nrun = direct_runs if (name.startswith("direct") and direct_runs) else runs
        t0 = time.perf_counter()
        fn(c.handle, packets, u, stream)
        torch.cuda.synchronize()
        for _ in range(2 if time.perf_counter() - t0 < 0.5 else 0):
            fn(c.handle, packets, u, stream)
        ms = []
        for _ in range(nrun):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(c.handle, packets, u, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        got = u.cpu().numpy()
        if name == "direct" and ud is None:
            ud = got
        rel = float(np.linalg.norm(got - ud) / max(np.linalg.norm(ud), 1e-300))
        med = statistics.median(ms)
        out[name] = {"runs": nrun, "median_ms": med, "min_ms": min(ms), "max_ms": max(ms),
                     "packets_per_s": int(packets.m) / (med * 1e-3), "rel_l2_vs_direct": rel}
        if name != "direct":
            del u
    u = torch.zeros_like(u_ref)
    q2.close()
    if fma is not None:
        fma.close()
        out["direct"]["path"] = "tensor cores (tcgen05.mma, 3 x TF32)"
        out["direct"]["speedup_vs_cuda_cores"] = out["direct_cuda_cores"]["median_ms"] / out["direct"]["median_ms"]
    # FGGC Q4P2 through a plan: the node box fixed once for this packet set,
    # so a call waits for nothing on the host (the unplanned call reads the
    # box bounds back every time)
    plan = fgr.fgr_fggc_plan_create(ctx.handle, packets, 2, stream)
    try:
        for _ in range(3):
            fgr.fgr_reconstruct_fggc_planned(ctx.handle, plan, packets, u, stream)
        ms = []
        for _ in range(runs):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fgr.fgr_reconstruct_fggc_planned(ctx.handle, plan, packets, u, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        got = u.cpu().numpy()
        med = statistics.median(ms)
        out["fggc_q4p2_planned"] = {
            "median_ms": med, "min_ms": min(ms), "max_ms": max(ms), "packets_per_s": int(packets.m) / (med * 1e-3),
            "rel_l2_vs_direct": float(np.linalg.norm(got - ud) / max(np.linalg.norm(ud), 1e-300)),
            "overflow": fgr.fgr_fggc_plan_overflow(plan)}
    finally:
        fgr.fgr_fggc_plan_destroy(plan)
    for k in ("fggc_q4p2", "fggc_q2p2", "fggc_q4p2_planned"):
        ok = out[k]["rel_l2_vs_direct"] <= 1e-5
        out[k]["speedup_vs_direct_at_equal_accuracy"] = (
            out["direct"]["median_ms"] / out[k]["median_ms"] if ok else "not at equal accuracy")
    return out


def decompose_runs(fgr, ctx, w, init, pot, stream, flush, runs=20, multistep=True, moved=None):
    """Median/min/max ms of `runs` initial decompositions (eq. 2.8) of the
    workload's u0 onto its t = 0 packet positions, and of one multi-step FGGC
    step (Algorithm 3: decompose, apply the learned flow, FGGC) whose flow is
    those positions propagated over the workload's time from unit amplitude.
    For d >= 2 also the tensor-product decomposition of the same mesh
    (fgr_decompose_tensor) and, given the propagated packets `moved`, one
    multi-step FGGC step over the tensor mesh whose learned amplitude factors
    are A(t) / A(0) of the workload (eq. 2.6 is linear in A)."""
    import math
    import numpy as np
    import torch
    from workloads.wkb import _FAMILIES

    d, eps, grid = w["d"], w["eps"], w["grid"]
    m = int(init[2].numel())
    axes = [np.linspace(grid["lo"][l], grid["hi"][l], grid["n"][l], endpoint=False) for l in range(d)]
    x = np.stack(np.meshgrid(*axes, indexing="ij"))
    cdt = torch.complex64 if w["precision"] == "fp32" else torch.complex128
    u0 = torch.tensor(_FAMILIES[w["family"]].u0(x, eps), dtype=cdt, device=init[0].device)
    q, p = init[0].clone(), init[1].clone()
    s, a = torch.empty_like(init[2]), torch.empty_like(init[3])
    mesh = fgr.make_packets(q, p, s, a)

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        n = runs if time.perf_counter() - t0 < 1.0 else 3
        for _ in range(2):
            fn()
        ms = []
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        return {"runs": n, "median_ms": med, "min_ms": min(ms), "max_ms": max(ms), "packets_per_s": m / (med * 1e-3)}

    out = {"decompose": timed(lambda: fgr.fgr_decompose(ctx.handle, u0, mesh, stream))}
    # window points per packet: (2 R sqrt(eps) / h + 1)^d with the context's R
    R = 6.0 if w["precision"] == "fp32" else 8.0
    pts = math.prod(2 * R * math.sqrt(eps) / ((grid["hi"][l] - grid["lo"][l]) / grid["n"][l]) + 1
                    for l in range(d))
    out["decompose"]["window_points_per_packet"] = pts
    out["decompose"]["gpoints_per_s"] = m * pts / (out["decompose"]["median_ms"] * 1e-3) / 1e9
    if d >= 2:
        from workloads import workload_axes
        axes_np, sel_np = workload_axes(w)
        dev = init[0].device
        axes = fgr.make_axes([(torch.tensor(q, device=dev), torch.tensor(p, device=dev)) for q, p in axes_np])
        sel = torch.tensor(sel_np, device=dev)
        at = torch.empty((2, m), dtype=torch.float64, device=dev)
        out["decompose_tensor"] = timed(lambda: fgr.fgr_decompose_tensor(ctx.handle, axes, u0, m, sel, at, stream))
        ap, aq = torch.complex(a[0], a[1]), torch.complex(at[0], at[1])
        out["decompose_tensor"]["rel_l2_vs_per_packet_kernel"] = float(torch.linalg.norm(aq - ap) /
                                                                       torch.linalg.norm(ap))
        out["decompose_tensor"]["speedup_vs_per_packet_kernel"] = (out["decompose"]["median_ms"] /
                                                                   out["decompose_tensor"]["median_ms"])
        out["decompose_tensor"]["mesh"] = "%d-dim tensor product of %d-entry axes, %d packets selected" % (
            d, axes_np[0][0].size, m)
        if moved is not None:
            a0 = torch.complex(init[3][0], init[3][1])
            at_ = torch.complex(moved[3][0], moved[3][1])
            fac = torch.where(a0 != 0, at_ / torch.where(a0 != 0, a0, torch.ones_like(a0)), torch.zeros_like(a0))
            flow = fgr.make_packets(moved[0], moved[1], moved[2], torch.stack([fac.real, fac.imag]).contiguous())
            u1 = torch.empty_like(u0)
            out["multistep_tensor_1_step"] = timed(
                lambda: fgr.fgr_fggc_multistep_tensor(ctx.handle, axes, sel, flow, u0, u1, 1, stream))
            out["multistep_tensor_1_step"]["note"] = ("tensor decomposition + learned factors + FGGC; "
                                                      "factors A(t)/A(0) of the workload's propagation, untimed")
    if multistep:
        fq, fp = init[0].clone(), init[1].clone()
        fs = torch.zeros_like(init[2])
        fa = torch.zeros_like(init[3])
        fa[0] = 1.0
        flow = fgr.make_packets(fq, fp, fs, fa)
        fgr.fgr_propagate(ctx.handle, flow, pot, w["t"], w["dt"], stream)
        u1 = torch.empty_like(u0)
        out["multistep_1_step"] = timed(lambda: fgr.fgr_fggc_multistep(ctx.handle, mesh, flow, u0, u1, 1, stream))
        out["multistep_1_step"]["note"] = "decompose + flow amplitudes + FGGC; RK4 of the flow learned once, untimed"
    return out


def reconstruct_bench(cfg: int, args, flush):
    """FGGC and direct reconstruction of another workload (propagated once on
    the GPU, not timed), L2 flushed between timed runs."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads import config_workload
    w = config_workload(cfg)
    d, eps, grid = w["d"], w["eps"], w["grid"]
    M = int(w["packets"]["s"].size)
    prec = fgr.FGR_FP32 if w["precision"] == "fp32" else fgr.FGR_FP64
    cdt = torch.complex64 if prec == fgr.FGR_FP32 else torch.complex128
    ctx = fgr.Context(d, grid, eps, fgr.make_options(precision=prec))
    arrs = [torch.tensor(np.ascontiguousarray(w["packets"][k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
    pk = fgr.make_packets(*arrs)
    init = [x.clone() for x in arrs]
    t0 = time.perf_counter()
    fgr.fgr_propagate(ctx.handle, pk, fgr.make_potential(**w["potential"]), w["t"], w["dt"])
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    shape = tuple(grid["n"][:d])
    uf = torch.zeros(shape, dtype=cdt, device="cuda")
    ud = torch.zeros(shape, dtype=cdt, device="cuda")
    stream = torch.cuda.current_stream()
    fgr.fgr_autotune(ctx.handle, pk, ud, 3, stream)
    res, spread = {}, {}
    q2 = fgr.Context(d, grid, eps, fgr.make_options(precision=prec, nq=2, np_=2))
    fma = fgr.Context(d, grid, eps, fgr.make_options(precision=prec, flags=fgr.FGR_FLAG_DIRECT_FMA))
    uq2 = torch.zeros(shape, dtype=cdt, device="cuda")
    ufma = torch.zeros(shape, dtype=cdt, device="cuda")
    for name, fn, c, u in (("direct", fgr.fgr_reconstruct_direct, ctx, ud),
                           ("direct_cuda_cores", fgr.fgr_reconstruct_direct, fma, ufma),
                           ("fggc", fgr.fgr_reconstruct_fggc, ctx, uf),
                           ("fggc_q2p2", fgr.fgr_reconstruct_fggc, q2, uq2)):
        t0 = time.perf_counter()
        fn(c.handle, pk, u, stream)
        torch.cuda.synchronize()
        # 20 timed runs, fewer where one run takes seconds (the 3-D direct sum)
        runs = 20 if time.perf_counter() - t0 < 1.0 else 3
        ms = []
        for _ in range(runs):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(c.handle, pk, u, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = statistics.median(ms)
        spread[name] = {"runs": runs, "median_ms": res[name], "min_ms": min(ms), "max_ms": max(ms)}
    q2.close()
    fma.close()
    a, b, c2 = uf.cpu().numpy(), ud.cpu().numpy(), uq2.cpu().numpy()
    rel = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    rel_fma = float(np.linalg.norm(ufma.cpu().numpy() - b) / max(np.linalg.norm(b), 1e-300))
    del ufma
    rel_q2 = float(np.linalg.norm(c2 - b) / max(np.linalg.norm(b), 1e-300))
    fgr.fgr_set_timing(ctx.handle, True)
    fgr.fgr_reconstruct_fggc(ctx.handle, pk, uf, stream)
    st = fgr.fgr_get_stats(ctx.handle)
    tuned = list(fgr.fgr_get_tuning(ctx.handle))
    decomp = decompose_runs(fgr, ctx, w, init, None, stream, flush, multistep=False, moved=arrs)
    del init
    ctx.close()
    return {"workload": w["name"], "packets": M, "propagate_s_untimed": t_prop,
            "fggc_ms": res["fggc"], "direct_ms": res["direct"],
            "fggc_packets_per_s": M / (res["fggc"] * 1e-3), "direct_packets_per_s": M / (res["direct"] * 1e-3),
            "fggc_over_direct": res["direct"] / res["fggc"], "rel_l2_fggc_vs_direct": rel,
            "direct_path": "tensor cores (tcgen05.mma, 3 x TF32)",
            "direct_cuda_cores_ms": res["direct_cuda_cores"], "rel_l2_direct_cuda_cores_vs_direct": rel_fma,
            "direct_roofline": direct_roofline(window_pairs(arrs[0].cpu().numpy(), grid, eps), res["direct"]),
            "runs": spread, "fggc_q2p2_ms": res["fggc_q2p2"], "rel_l2_fggc_q2p2_vs_direct": rel_q2,
            "fggc_q2p2_over_direct": (res["direct"] / res["fggc_q2p2"] if rel_q2 <= 1e-5
                                      else "not at equal accuracy (rel L2 > 1e-5)"),
            "fggc_nodes": int(st.nodes), "autotuned_ctas_per_sm_and_tile": tuned,
            "decompose": decomp,
            "fggc_stage_split_ms": {"bounds_alloc": st.prep_ms, "coeff_scatter": st.scatter_ms, "grid": st.grid_ms}}


def fft_grid_bench(args, flush):
    """FGGC with the DFT grid stage (FGR_FLAG_FFT_GRID) beside the direct grid
    stage on the commensurate meshes of Examples 4 and 5 (Sec. 4.4: h = eps,
    N = 16 / sqrt(eps) = 1024 and 128): the fixed mesh of each example with
    the amplitudes of u0 (fgr_decompose_tensor), propagated under V2 over
    T / 32 (one restart interval of the 32-step split; untimed), FP32, Q2P2;
    median of 20 reconstructions each, L2 flushed before every run."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads.examples import EXAMPLES, example_axis, example_grid, example_u0

    stream = torch.cuda.current_stream()
    out = {}
    for ex in (4, 5):
        e = EXAMPLES[ex]
        d, eps = e["d"], e["eps"]
        grid = example_grid(ex)
        q, p = example_axis(ex)
        aq, ap = torch.tensor(q, device="cuda"), torch.tensor(p, device="cuda")
        L = q.size
        idx = torch.arange(L ** d, device="cuda")
        Q = torch.stack([aq[(idx // (L ** (d - 1 - l))) % L] for l in range(d)]).contiguous()
        P = torch.stack([ap[(idx // (L ** (d - 1 - l))) % L] for l in range(d)]).contiguous()
        del idx
        m = Q.shape[1]
        S = torch.zeros(m, dtype=torch.float64, device="cuda")
        A = torch.zeros((2, m), dtype=torch.float64, device="cuda")
        u0 = torch.tensor(example_u0(ex), dtype=torch.complex64, device="cuda")
        opts = {name: fgr.make_options(precision=fgr.FGR_FP32, nq=2, np_=2, flags=fl)
                for name, fl in (("direct_stage", 0), ("dft_stage", fgr.FGR_FLAG_FFT_GRID))}
        res = {"packets": m, "grid": grid["n"], "eps": eps, "N_dft": int(round(16 / math.sqrt(eps)))}
        outs = {}
        with fgr.Context(d, grid, eps, opts["direct_stage"]) as c0:
            fgr.fgr_decompose_tensor(c0.handle, fgr.make_axes([(aq, ap)] * d), u0, m, None, A, stream)
            pk = fgr.make_packets(Q, P, S, A)
            fgr.fgr_propagate(c0.handle, pk, fgr.make_potential(**e["potentials"]["V2"]), e["T"] / 32, e["dt"],
                              stream)
        for name, o in opts.items():
            with fgr.Context(d, grid, eps, o) as c:
                u = torch.zeros(tuple(grid["n"]), dtype=torch.complex64, device="cuda")
                for _ in range(3):
                    fgr.fgr_reconstruct_fggc(c.handle, pk, u, stream)
                ms = []
                for _ in range(20):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    fgr.fgr_reconstruct_fggc(c.handle, pk, u, stream)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                fgr.fgr_set_timing(c.handle, True)
                fgr.fgr_reconstruct_fggc(c.handle, pk, u, stream)
                st = fgr.fgr_get_stats(c.handle)
                fgr.fgr_set_timing(c.handle, False)
                outs[name] = u.cpu().numpy()
                res[name] = {"median_ms": statistics.median(ms), "min_ms": min(ms), "max_ms": max(ms),
                             "packets_per_s": m / (statistics.median(ms) * 1e-3), "grid_stage_ms": st.grid_ms,
                             "pass_kernels_ms": st.pass_ms}
        a, b = outs["dft_stage"], outs["direct_stage"]
        res["rel_l2_dft_vs_direct_stage"] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        res["grid_stage_speedup"] = res["direct_stage"]["grid_stage_ms"] / res["dft_stage"]["grid_stage_ms"]
        out["example%d" % ex] = res
        del Q, P, S, A, pk, u0
        torch.cuda.empty_cache()
    return out


def batch_bench(args, flush):
    """Many small reconstructions: direct sums as one fgr_reconstruct_direct call
    each on one stream, against one fgr_reconstruct_direct_batch call, eager and
    replayed from a CUDA graph; FGGC as one fgr_reconstruct_fggc call each,
    as planned calls (fgr_reconstruct_fggc_planned) and as one
    fgr_reconstruct_fggc_batch call, eager and replayed from CUDA graphs.  64 1-D requests, grids 1024..8192 points, 2k..16k
    uniformly placed packets, eps in [1/1024, 1/256], FP32; L2 flushed before
    each timed run."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads import random_packets, mesh_for

    rng = np.random.default_rng(11)
    opt = fgr.make_options(precision=fgr.FGR_FP32)
    ctxs, pks, outs, keep = [], [], [], []
    packets = 0
    for r in range(64):
        n = int(2 ** rng.integers(10, 14))
        eps = float(2.0 ** -rng.uniform(8, 10))
        m = int(np.exp(rng.uniform(np.log(2048), np.log(16384))))
        pk = random_packets(100 + r, 1, m, q_range=(-3.2, 3.2), p_range=(-4, 4), s_range=(-1, 1),
                            mesh=mesh_for(1, eps))
        arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
        grid = dict(d=1, n=[n], lo=[-np.pi], hi=[np.pi])
        ctxs.append(fgr.Context(1, grid, eps, opt))
        pks.append(fgr.make_packets(*arrs))
        outs.append(torch.zeros(n, dtype=torch.complex64, device="cuda"))
        keep.append(arrs)
        packets += m
    s = torch.cuda.Stream()
    torch.cuda.synchronize()

    def single():
        for c, p, u in zip(ctxs, pks, outs):
            fgr.fgr_reconstruct_direct(c.handle, p, u, s)

    def batched():
        fgr.fgr_reconstruct_direct_batch(ctxs, pks, outs, s)

    ref = None
    for fn in (single, batched):  # warm-up; results must agree
        fn()
        torch.cuda.synchronize()
        cur = [u.clone() for u in outs]
        if ref is None:
            ref = cur
    worst = max(float(torch.linalg.norm(a - b) / max(float(torch.linalg.norm(b)), 1e-30))
                for a, b in zip(cur, ref))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        batched()
        g.capture_end()
    torch.cuda.synchronize()

    def timed(fn):
        ms = []
        for _ in range(max(3, args.steps)):
            with torch.cuda.stream(s):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    with torch.cuda.stream(s):
        t_single = timed(single)
        t_batch = timed(batched)
        t_graph = timed(g.replay)

    # the same requests by FGGC: one fgr_reconstruct_fggc each (each waits for
    # its node bounds) against planned calls, eager and replayed from a graph
    plans = [fgr.fgr_fggc_plan_create(c.handle, p, 2) for c, p in zip(ctxs, pks)]

    def fggc_single():
        for c, p, u in zip(ctxs, pks, outs):
            fgr.fgr_reconstruct_fggc(c.handle, p, u, s)

    def fggc_planned():
        for c, pl, p, u in zip(ctxs, plans, pks, outs):
            fgr.fgr_reconstruct_fggc_planned(c.handle, pl, p, u, s)

    fggc_single()
    torch.cuda.synchronize()
    ref_f = [u.clone() for u in outs]
    fggc_planned()
    torch.cuda.synchronize()
    worst_f = max(float(torch.linalg.norm(a - b) / max(float(torch.linalg.norm(b)), 1e-30))
                  for a, b in zip(outs, ref_f))
    gf = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gf.capture_begin()
        fggc_planned()
        gf.capture_end()
    torch.cuda.synchronize()

    def fggc_batched():
        fgr.fgr_reconstruct_fggc_batch(ctxs, plans, pks, outs, s)

    fggc_batched()
    torch.cuda.synchronize()
    worst_b = max(float(torch.linalg.norm(a - b) / max(float(torch.linalg.norm(b)), 1e-30))
                  for a, b in zip(outs, ref_f))
    gb = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        gb.capture_begin()
        fggc_batched()
        gb.capture_end()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        tf_single = timed(fggc_single)
        tf_planned = timed(fggc_planned)
        tf_graph = timed(gf.replay)
        tf_batch = timed(fggc_batched)
        tf_batch_graph = timed(gb.replay)
    for pl in plans:
        fgr.fgr_fggc_plan_destroy(pl)
    for c in ctxs:
        c.close()
    return {"requests": len(outs), "packets": packets, "single_calls_ms": t_single, "batch_ms": t_batch,
            "graph_replay_ms": t_graph, "requests_per_s_graph": len(outs) / (t_graph * 1e-3),
            "speedup_batch_vs_single": t_single / t_batch, "speedup_graph_vs_single": t_single / t_graph,
            "max_rel_l2_batch_vs_single": worst,
            "fggc_single_calls_ms": tf_single, "fggc_planned_ms": tf_planned,
            "fggc_planned_graph_replay_ms": tf_graph, "fggc_batch_ms": tf_batch,
            "fggc_batch_graph_replay_ms": tf_batch_graph,
            "fggc_requests_per_s_batch_graph": len(outs) / (tf_batch_graph * 1e-3),
            "max_rel_l2_fggc_planned_vs_single": worst_f, "max_rel_l2_fggc_batch_vs_single": worst_b,
            "mix": "64 x 1-D, grids 1024..8192, 2k..16k packets, eps 1/1024..1/256, fp32"}


def serving_bench(args, device_index: int):
    """Continuous-batching server under a Poisson stream (the serving workload):
    a pool of packet sets with d in {1, 2}, eps log-uniform in [1/1024, 1/64],
    M = 2^L with L uniform in [12, log2(max packets)] (WKB data on a q x p mesh),
    propagated once to t = 0.5 on the GPU and kept resident; each request picks
    a set, a grid (1-D: 1024..32768 points, 2-D: 256^2..1024^2, powers of two)
    and a method (direct / FGGC) uniformly; FP32.  Capacity = the saturated
    request rate (a burst submitted at once); Poisson streams of 2000 requests
    at 0.5x, 0.8x and 1.0x capacity; p50/p99 of submit-to-done latency and
    packets/s per level."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads import wkb_packets, WKB_TANH

    rng = np.random.default_rng(0)
    srv = fgr.fgr_server_create(150 << 30, args.serve_inflight)
    sets = []
    pot1 = fgr.make_potential("cossum", c0=1.0, amp=-1.0, k=1.0)
    pot2 = fgr.make_potential("cossum", c0=2.0, amp=1.0, k=1.0)
    lmax = int(round(math.log2(args.serve_max_packets)))
    t_setup = time.perf_counter()
    for i in range(args.serve_sets):
        d = 1 + (i % 2)
        eps = float(2.0 ** -rng.uniform(6, 10))
        L = int(rng.integers(12, lmax + 1))
        half = L // d                       # log2 of nq * np per dimension
        nq, np_ = 2 ** ((half + 1) // 2), 2 ** (half // 2)
        pk = wkb_packets(d, eps, nq, np_, WKB_TANH)
        arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda") for k in "qpsa"]
        grid0 = dict(d=d, n=[16] * d, lo=[-3.0] * d, hi=[3.0] * d)
        with fgr.Context(d, grid0, eps) as c:
            fgr.fgr_propagate(c.handle, fgr.make_packets(*arrs), pot1 if d == 1 else pot2, 0.5, 1e-4)
        torch.cuda.synchronize()
        sid = fgr.fgr_register_packets(srv, d, fgr.make_packets(*arrs))
        sets.append((sid, d, eps, int(pk["s"].size)))
        del arrs
    t_setup = time.perf_counter() - t_setup
    opt = fgr.make_options(precision=fgr.FGR_FP32)

    def draw():
        sid, d, eps, m = sets[rng.integers(len(sets))]
        if d == 1:
            n = [int(2 ** rng.integers(10, 16))]
        else:
            n = [int(2 ** rng.integers(8, 11))] * 2
        grid = dict(d=d, n=n, lo=[-np.pi] * d, hi=[np.pi] * d)
        return sid, d, eps, m, grid, int(rng.integers(0, 2))

    # isolated service times
    iso = []
    for _ in range(args.serve_probe):
        sid, d, eps, m, grid, method = draw()
        u = torch.zeros(tuple(grid["n"]), dtype=torch.complex64, device="cuda")
        t = fgr.fgr_submit(srv, fgr.make_request(method, grid, eps, opt, sid, u))
        r = fgr.fgr_poll(srv, t, -1)
        iso.append(r.t_done_ms - r.t_start_ms)
    # capacity = the saturated rate: a burst submitted at once keeps every
    # slot busy (the load levels below are fractions of it)
    burst = [draw() for _ in range(4 * args.serve_probe)]
    bouts = [torch.zeros(tuple(g["n"]), dtype=torch.complex64, device="cuda") for (_, _, _, _, g, _) in burst]
    tb0 = time.perf_counter()
    bt = [fgr.fgr_submit(srv, fgr.make_request(mth, g, e, opt, sid, u))
          for (sid, d, e, m, g, mth), u in zip(burst, bouts)]
    for t in bt:
        fgr.fgr_poll(srv, t, -1)
    burst_rate = len(burst) / (time.perf_counter() - tb0)
    capacity = burst_rate
    del bouts
    # the longest single requests of the mix, alone: every set with either
    # method on its dimension's finest grid (best of 2 runs each; the first run
    # of an FGGC request also builds the plan the server caches)
    alone = []
    for sid, d, eps, m in sets:
        n = [32768] if d == 1 else [1024, 1024]
        grid = dict(d=d, n=n, lo=[-np.pi] * d, hi=[np.pi] * d)
        u = torch.zeros(tuple(n), dtype=torch.complex64, device="cuda")
        for method in (0, 1):
            times = []
            for _ in range(2):
                r = fgr.fgr_poll(srv, fgr.fgr_submit(srv, fgr.make_request(method, grid, eps, opt, sid, u)), -1)
                times.append(r.t_done_ms - r.t_start_ms)
            alone.append({"method": ("direct", "fggc")[method], "d": d, "packets": m, "eps": eps, "grid": n,
                          "service_ms": min(times), "first_ms": times[0]})
        del u
    alone.sort(key=lambda x: -x["service_ms"])
    levels = {}
    for frac in (0.5, 0.8, 1.0):
        lam = frac * capacity
        reqs = [draw() for _ in range(args.serve_requests)]
        outs = [torch.zeros(tuple(g["n"]), dtype=torch.complex64, device="cuda") for (_, _, _, _, g, _) in reqs]
        gaps = rng.exponential(1.0 / lam, size=len(reqs))
        tickets = []
        t0 = time.perf_counter()
        due = t0
        for (sid, d, eps, m, grid, method), u, gap in zip(reqs, outs, gaps):
            due += gap
            while time.perf_counter() < due:
                time.sleep(max(0.0, min(0.001, due - time.perf_counter())))
            tickets.append(fgr.fgr_submit(srv, fgr.make_request(method, grid, eps, opt, sid, u)))
        res = [fgr.fgr_poll(srv, t, -1) for t in tickets]
        t1 = time.perf_counter()
        lat = np.array([r.t_done_ms - r.t_submit_ms for r in res])
        wait = np.array([r.t_start_ms - r.t_submit_ms for r in res])
        svc = np.array([r.t_done_ms - r.t_start_ms for r in res])
        tail = lat >= np.percentile(lat, 99)
        by_method = {}
        for mth_, name in ((0, "direct"), (1, "fggc")):
            sel = np.array([q[5] == mth_ for q in reqs])
            if sel.any():
                by_method[name] = {"p50_ms": float(np.percentile(lat[sel], 50)),
                                   "p99_ms": float(np.percentile(lat[sel], 99))}
        kinds = {}
        for (sid_, d_, e_, m_, g_, mth_), t_ in zip(reqs, tail):
            if t_:
                key = "%s %d-D" % (("direct", "fggc")[mth_], d_)
                kinds[key] = kinds.get(key, 0) + 1
        ok = all(r.status == 0 for r in res)
        packets = sum(q[3] for q in reqs)
        levels["%.1fx" % frac] = {"lambda_req_per_s": lam, "p50_ms": float(np.percentile(lat, 50)),
                                  "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                                  "by_method": by_method,
                                  "tail_1pct": {"wait_ms_median": float(np.median(wait[tail])),
                                                "service_ms_median": float(np.median(svc[tail])),
                                                "kinds": kinds},
                                  "packets_per_s": packets / (t1 - t0),
                                  "requests": len(reqs), "all_ok": ok}
        del outs
    fgr.fgr_server_destroy(srv)
    ms = [m for (_, _, _, m) in sets]
    return {"sets": len(sets), "packets_min": min(ms), "packets_max": max(ms), "setup_s_untimed": t_setup,
            "inflight": args.serve_inflight, "max_batch": 16, "isolated_service_ms_mean": float(np.mean(iso)),
            "isolated_service_ms_p50": float(np.percentile(iso, 50)),
            "capacity_req_per_s": capacity, "capacity_def": "saturated rate of a burst of %d requests" % len(burst),
            "isolated_capacity_req_per_s": 1e3 / float(np.mean(iso)),
            "largest_requests_alone": alone[:4], "largest_request_ms": alone[0]["service_ms"],
            "levels": levels,
            "mix": "d in {1,2}; grids 1-D 1024..32768, 2-D 256^2..1024^2; direct/fggc 50/50; fp32"}


def _oracle_job(job):
    """One oracle reconstruction of a packet chunk on the full grid (runs in a
    spawned worker process); returns (seconds, squared norm of the field)."""
    import numpy as np

    from oracle import fga, fggc, lsa
    kind, pk, grid, eps, dq, dp, R = job
    t0 = time.perf_counter()
    if kind == "fggc":
        u = fggc.reconstruct(pk, grid, eps, dq, dp, lsa.Strategy(nq=4, np_=2), R=R)
    else:
        u = fga.direct_sum(pk, grid, eps, dq, dp, R=R)
    return time.perf_counter() - t0, float(np.vdot(u, u).real)


def _oracle_sample(w, count: int, seed: int = 0):
    """`count` packets of the workload (uniform sample without replacement,
    seeded), propagated to the workload's t by the oracle's RK4."""
    import numpy as np

    from oracle import trajectories
    pk = w["packets"]
    M = pk["s"].size
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(M, size=min(count, M), replace=False))
    sub = {k: np.ascontiguousarray(pk[k][..., idx]) for k in ("q", "p", "s", "a")}
    t0 = time.perf_counter()
    prop = trajectories.propagate(sub, w["potential"], w["t"], w["dt"])
    return prop, idx, time.perf_counter() - t0


def _chunks(pk: dict, n: int):
    """The packet set split into n consecutive chunks (FGGC and the direct sum
    are linear in the packets, so the chunks' fields add up to the whole)."""
    import numpy as np
    m = pk["s"].size
    cuts = np.linspace(0, m, n + 1).astype(int)
    return [{k: np.ascontiguousarray(pk[k][..., a:b]) for k in ("q", "p", "s", "a")}
            for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def oracle_pool(workers: int):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def cpu_baseline(w, args, pool=None):
    """The FP64 oracle, as it stands, on bounded packet samples of the
    workload on the host cores: FGGC (Algorithm 2: aggregation onto the nodes,
    eq. 2.25, then eq. 2.24 node by node) and the direct sum (eq. 2.10) of
    propagated packets on the full output grid, single-threaded and spread
    over all cores (one spawned process per core, each reconstructing its own
    chunk of the sample; their partial fields are not summed)."""
    R = 6 if w["precision"] == "fp32" else 8
    mesh = w["mesh"]
    cores = os.cpu_count() or 1
    own_pool = pool is None
    if own_pool:
        pool = oracle_pool(cores)
    try:
        res = {}
        for kind, n1, nall in (("fggc", args.cpu_fggc_single, args.cpu_fggc_all),
                               ("direct", args.cpu_direct_single, args.cpu_direct_all)):
            sub, _, _ = _oracle_sample(w, max(n1, nall), seed=0)
            one = _chunks(sub, max(1, sub["s"].size // max(n1, 1)))[0]
            t_single, _ = _oracle_job((kind, one, w["grid"], w["eps"], mesh.dq, mesh.dp, R))
            jobs = [(kind, c, w["grid"], w["eps"], mesh.dq, mesh.dp, R) for c in _chunks(sub, cores)]
            t0 = time.perf_counter()
            list(pool.imap_unordered(_oracle_job, jobs))
            t_all = time.perf_counter() - t0
            res[kind] = {"single_thread_packets_per_s": one["s"].size / t_single,
                         "single_thread_sample": int(one["s"].size), "single_thread_s": t_single,
                         "all_core_packets_per_s": sub["s"].size / t_all, "all_core_sample": int(sub["s"].size),
                         "all_core_s": t_all}
    finally:
        if own_pool:
            pool.close()
            pool.join()
    f = res["fggc"]
    return {"value": f["all_core_packets_per_s"], "unit": "packets/s", "cores": cores, "kind": "oracle",
            "sample": "FGGC of %d propagated packets (uniform sample, seed 0) on the full %s grid over %d processes "
                      "(%.1f s); single-threaded %d packets in %.1f s = %.3g packets/s; direct sum %.3g packets/s "
                      "on %d cores, %.3g on one" % (
                          f["all_core_sample"], "x".join(str(n) for n in w["grid"]["n"][:w["d"]]), cores,
                          f["all_core_s"], f["single_thread_sample"], f["single_thread_s"],
                          f["single_thread_packets_per_s"], res["direct"]["all_core_packets_per_s"], cores,
                          res["direct"]["single_thread_packets_per_s"]),
            "fggc": res["fggc"], "direct": res["direct"]}


def run_reference(args):
    """The oracle's FGGC reconstruction of the headline workload on the host
    cores: each step reconstructs a fresh packet sample (one chunk per core,
    spawned processes) on the full grid; value = sampled packets / step time."""
    rank, _, world = _rank_env()
    if rank != 0:
        return None
    from workloads import config_workload
    w = config_workload(args.config)
    R = 6 if w["precision"] == "fp32" else 8
    mesh = w["mesh"]
    cores = os.cpu_count() or 1
    per_step = max(cores, args.ref_sample)
    sub, _, t_prop = _oracle_sample(w, per_step * (args.warmup + args.steps), seed=1)
    pool = oracle_pool(cores)
    times = []
    try:
        allc = _chunks(sub, args.warmup + args.steps)
        for i, step_pk in enumerate(allc):
            jobs = [("fggc", c, w["grid"], w["eps"], mesh.dq, mesh.dp, R) for c in _chunks(step_pk, cores)]
            t0 = time.perf_counter()
            list(pool.imap_unordered(_oracle_job, jobs))
            if i >= args.warmup:
                times.append((time.perf_counter() - t0, step_pk["s"].size))
    finally:
        pool.close()
        pool.join()
    tot_s = sum(t for t, _ in times)
    tot_p = sum(n for _, n in times)
    value = tot_p / tot_s
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "packets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config], "packets_per_step": tot_p // len(times),
                       "step": "oracle FGGC reconstruction (Algorithm 2) of a packet sample on the full grid"},
            "cpu_baseline": {"value": value, "unit": "packets/s", "cores": cores, "kind": "oracle",
                             "sample": "%d propagated packets per step (uniform sample, seed 1; oracle RK4 %.1f s, "
                                       "untimed), one chunk per process on %d processes, full grid"
                                       % (tot_p // len(times), t_prop, cores)},
            "e2e": {"value": value, "unit": "packets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """One short pass of every kernel on the benchmark workload, for ncu:
    propagate to t = 0.01 (100 RK4 steps), then one FGGC and one direct
    reconstruction of the propagated packets, one batched direct sum of
    eight copies of that request and one initial decomposition of the
    reconstructed wave onto the propagated positions (3-D workloads: FGGC, and
    the direct sum with at most 2^21 packets kept); for d >= 2 one
    tensor-product decomposition of that wave onto the t = 0 mesh."""
    import numpy as np
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads import config_workload
    w = config_workload(args.config)
    d, eps, grid = w["d"], w["eps"], w["grid"]
    prec = fgr.FGR_FP32 if w["precision"] == "fp32" else fgr.FGR_FP64
    pk = w["packets"]
    pick = None
    if args.profile_packets and args.profile_packets < pk["s"].size:
        # the largest amplitudes, in their original order (a smaller case of the same shape)
        amp = np.hypot(pk["a"][0], pk["a"][1])
        pick = np.sort(np.argsort(-amp, kind="stable")[:args.profile_packets])
        pk = {k: np.ascontiguousarray(pk[k][..., pick]) for k in "qpsa"}
    with fgr.Context(d, grid, eps, fgr.make_options(precision=prec)) as ctx:
        arrs = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda")
                for k in "qpsa"]
        pk = fgr.make_packets(*arrs)
        fgr.fgr_propagate(ctx.handle, pk, fgr.make_potential(**w["potential"]), 0.01, w["dt"])
        cdt = torch.complex64 if prec == fgr.FGR_FP32 else torch.complex128
        u = torch.zeros(tuple(grid["n"][:d]), dtype=cdt, device="cuda")
        fgr.fgr_reconstruct_fggc(ctx.handle, pk, u)
        if d < 3 or (pick is not None and pick.size <= 1 << 21):
            # the full 3-D direct sum takes about a second: only on a reduced case
            fgr.fgr_reconstruct_direct(ctx.handle, pk, u)
        if d < 3:
            outs = [torch.zeros_like(u) for _ in range(8)]
            fgr.fgr_reconstruct_direct_batch([ctx] * 8, [pk] * 8, outs)
            fgr.fgr_decompose(ctx.handle, u, pk)
        if d >= 2:  # the same mesh as a tensor product, decomposed by contractions
            from workloads import workload_axes
            axes_np, sel_np = workload_axes(w)
            if pick is not None:
                sel_np = sel_np[pick]
            axes = fgr.make_axes([(torch.tensor(q, device="cuda"), torch.tensor(p, device="cuda"))
                                  for q, p in axes_np])
            sel = torch.tensor(np.ascontiguousarray(sel_np), device="cuda")
            at = torch.empty((2, sel.numel()), dtype=torch.float64, device="cuda")
            fgr.fgr_decompose_tensor(ctx.handle, axes, u, sel.numel(), sel, at)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": "config %d" % args.config, "ok": True}))


def multistep_study(args):
    """Runtimes of single-step FGA and multi-step FGGC (Algorithm 3, Q2P2) on
    Examples 4 and 5 of Sec. 4.4 for the T_evo x T_multi splits of Tables 19
    and 22: per split the learning of the flow (RK4 of the fixed mesh over
    T / T_multi from unit amplitude) and the T_multi steps (decomposition by
    tensor-product contractions, learned amplitude factors, FGGC), timed with
    CUDA events (the second of two runs, or the first where it takes over a
    second); FGA = decomposition, RK4 over T and the direct sum.  The errors of the same runs against the exact harmonic
    solution are checked by tests/test_gpu_examples.py."""
    import torch

    import paper_2504_21785_gb300 as fgr
    from workloads.examples import EXAMPLES, SPLITS, example_axis, example_grid, example_u0

    prec = fgr.FGR_FP32 if args.study_precision == "fp32" else fgr.FGR_FP64
    cdt = torch.complex64 if prec == fgr.FGR_FP32 else torch.complex128
    stream = torch.cuda.current_stream()
    out = {"study": "multistep (Sec. 4.4, Tables 19 and 22)", "precision": args.study_precision, "cases": []}

    def timed(fn):
        # the first run is timed too; runs under a second are timed again
        # (warm memory pool) and the second time is reported
        ms = 0.0
        for rep in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if ms > 1000.0:
                break
        return ms

    for ex in (4, 5):
        e = EXAMPLES[ex]
        d, eps = e["d"], e["eps"]
        grid = example_grid(ex)
        u0 = torch.tensor(example_u0(ex), dtype=cdt, device="cuda")
        q, p = example_axis(ex)
        aq, ap = torch.tensor(q, device="cuda"), torch.tensor(p, device="cuda")
        L = q.size
        idx = torch.arange(L ** d, device="cuda")
        Q = torch.stack([aq[(idx // (L ** (d - 1 - l))) % L] for l in range(d)]).contiguous()
        P = torch.stack([ap[(idx // (L ** (d - 1 - l))) % L] for l in range(d)]).contiguous()
        m = Q.shape[1]
        axes = fgr.make_axes([(aq, ap)] * d)
        with fgr.Context(d, grid, eps, fgr.make_options(precision=prec, nq=2, np_=2)) as ctx:
            for vname, pot in e["potentials"].items():
                potv = fgr.make_potential(**pot)
                case = {"example": ex, "potential": vname, "d": d, "eps": eps, "T": e["T"], "packets": m,
                        "grid": grid["n"], "splits": {}}
                # single-step FGA
                s = torch.zeros(m, dtype=torch.float64, device="cuda")
                a = torch.zeros((2, m), dtype=torch.float64, device="cuda")
                Qw, Pw = Q.clone(), P.clone()
                pk = fgr.make_packets(Qw, Pw, s, a)
                u = torch.zeros_like(u0)

                def fga():
                    Qw.copy_(Q)
                    Pw.copy_(P)
                    fgr.fgr_decompose_tensor(ctx.handle, axes, u0, m, None, a, stream)
                    s.zero_()
                    fgr.fgr_propagate(ctx.handle, pk, potv, e["T"], e["dt"], stream)
                    fgr.fgr_reconstruct_direct(ctx.handle, pk, u, stream)
                case["fga_ms"] = timed(fga)
                for M in SPLITS:
                    fs = torch.zeros(m, dtype=torch.float64, device="cuda")
                    fa = torch.zeros((2, m), dtype=torch.float64, device="cuda")
                    Fq, Fp = Q.clone(), P.clone()
                    flow = fgr.make_packets(Fq, Fp, fs, fa)

                    def learn():
                        Fq.copy_(Q)
                        Fp.copy_(P)
                        fs.zero_()
                        fa.zero_()
                        fa[0] = 1.0
                        fgr.fgr_propagate(ctx.handle, flow, potv, e["T"] / M, e["dt"], stream)
                    learn_ms = timed(learn)
                    steps_ms = timed(lambda: fgr.fgr_fggc_multistep_tensor(ctx.handle, axes, None, flow, u0, u, M,
                                                                            stream))
                    case["splits"]["%dx%d" % (round(e["T"] / e["dt"]) // M, M)] = {
                        "learn_ms": learn_ms, "steps_ms": steps_ms, "total_ms": learn_ms + steps_ms,
                        "per_step_ms": steps_ms / M}
                    del flow, Fq, Fp, fs, fa
                out["cases"].append(case)
        del Q, P, idx
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--direct-runs", type=int, default=5,
                    help="timed runs of the direct sum beside the headline (each takes seconds in 3-D)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-fggc-single", type=int, default=2, help="oracle FGGC packets, one process")
    ap.add_argument("--cpu-fggc-all", type=int, default=0, help="oracle FGGC packets over all cores (0: 2 per core)")
    ap.add_argument("--cpu-direct-single", type=int, default=32)
    ap.add_argument("--cpu-direct-all", type=int, default=0, help="0: 32 per core")
    ap.add_argument("--ref-sample", type=int, default=0, help="oracle packets per reference step (0: one per core)")
    ap.add_argument("--extra", default="2,3", help="other workloads: 2 = 1-D pipeline with RK4, 3 = 2-D ('' for none)")
    ap.add_argument("--no-serving", dest="serving", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-fft", dest="fft", action="store_false",
                    help="skip the DFT grid stage on the meshes of Examples 4-5")
    ap.add_argument("--serve-sets", type=int, default=32)
    ap.add_argument("--serve-max-packets", type=int, default=1 << 22)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-probe", type=int, default=40)
    ap.add_argument("--serve-inflight", type=int, default=4)
    ap.add_argument("--profile-packets", type=int, default=0,
                    help="with --profile: keep only this many largest-amplitude packets")
    ap.add_argument("--profile", action="store_true",
                    help="run every kernel once on a short case (for ncu) and exit")
    ap.add_argument("--study", choices=["multistep", "serving"], default=None,
                    help="print the runtimes of the multi-step examples of Sec. 4.4, or the serving "
                         "workload's numbers alone, and exit")
    ap.add_argument("--study-precision", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args()
    cores = os.cpu_count() or 1
    args.cpu_fggc_all = args.cpu_fggc_all or 2 * cores
    args.cpu_direct_all = args.cpu_direct_all or 32 * cores
    if args.profile:
        run_profile_case(args)
        return
    if args.study == "multistep":
        print(json.dumps(multistep_study(args)))
        return
    if args.study == "serving":
        print(json.dumps(serving_bench(args, 0)))
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
