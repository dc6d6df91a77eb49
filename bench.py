#!/usr/bin/env python3
"""Benchmark: FGGC reconstruction on one GB300 (and N independent GPUs).

Workload (default): the 1-D WKB problem with eps = 1/1024, 512 (q) x 512 (p) =
262144 packets, V = 1 - cos x, t = 1.0 (RK4, dt = 1e-4), output 32768 points on
[-pi, pi), FP32 bulk arithmetic with FP64 phase reduction, complex64 output.

One step = Algorithm 2 on one batch: copy the t = 0 packets into the working
buffers, fgr_propagate to t (A1), fgr_reconstruct_fggc (A3-A5).  value =
packets / step time.  In the same run the direct sum (A2) reconstructs the same
propagated batch; its packets/s and the FGGC-vs-direct relative L2 are reported
beside it.  L2 is flushed (a 512 MiB write) between timed steps; only the steps
are inside the CUDA events.

--impl reference runs the FP64 CPU oracle (the only reference this method has)
on a bounded sample of the same workload.
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
WORKLOAD = "wkb-1d eps=1/1024 grid=32768 M=262144 (512q x 512p) V=1-cos(x) t=1.0 rk4 dt=1e-4 fp32/complex64 Q4P2"
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (no measured FP64 peak on file)


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


# FP64 FLOPs the RK4 kernel executes per packet-step (FMA = 2), counted by ncu
# on GB300 (DFMA x 2 + DMUL + DADD of rk4_kernel), 1-D cosine potential:
# 69.83 DFMA + 35.18 DMUL + 14.02 DADD (262144 packets, 100 steps).
RK4_FP64_FLOPS_PER_PACKET_STEP = {(1, "cossum"): 188.86}
# DRAM bytes of one RK4 launch on the bench workload (ncu, same capture): the
# packet arrays are read once; the written state stays in L2 at kernel end.
RK4_TRAFFIC_BYTES = {(1, "cossum", 262144): 10530816}


def run_ours(args):
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
    t_final, dt = w["t"], w["dt"]
    shape = tuple(grid["n"][:d])
    cdt = torch.complex64 if prec == fgr.FGR_FP32 else torch.complex128

    init = [torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device=dev) for k in "qpsa"]
    work = [x.clone() for x in init]
    packets = fgr.make_packets(*work)
    u_f = torch.zeros(shape, dtype=cdt, device=dev)
    u_d = torch.zeros(shape, dtype=cdt, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    launches = {"n": 0}

    def stats_launches():
        launches["n"] += int(fgr.fgr_get_stats(ctx.handle).launches)

    def step(ev=None):
        for wbuf, ibuf in zip(work, init):
            wbuf.copy_(ibuf)
        if ev:
            ev[0].record(stream)
        fgr.fgr_propagate(ctx.handle, packets, pot, t_final, dt, stream)
        stats_launches()
        if ev:
            ev[1].record(stream)
        fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
        stats_launches()
        if ev:
            ev[2].record(stream)
        fgr.fgr_reconstruct_direct(ctx.handle, packets, u_d, stream)
        stats_launches()
        if ev:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # launch shapes picked by the library's autotuner on the propagated batch
    fgr.fgr_autotune(ctx.handle, packets, u_d, 3, stream)
    tuning = fgr.fgr_get_tuning(ctx.handle)
    launches["n"] = 0
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            step(evs[i])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    prop_ms = [e[0].elapsed_time(e[1]) for e in evs]
    fggc_ms = [e[1].elapsed_time(e[2]) for e in evs]
    direct_ms = [e[2].elapsed_time(e[3]) for e in evs]
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    gpu_launches = launches["n"]
    ud, uf = u_d.cpu().numpy(), u_f.cpu().numpy()
    rel = float(np.linalg.norm(uf - ud) / max(np.linalg.norm(ud), 1e-300))

    # reconstruction alone on the propagated batch: median, min and max of 20
    # runs each (L2 flushed before every run), FGGC with Q4P2 and Q2P2
    recon = reconstruct_runs(fgr, ctx, packets, u_d, grid, d, eps, prec, flush, stream, ud, runs=20)
    # initial decomposition of u0 onto the t = 0 packet positions, and one step
    # of multi-step FGGC with the flow learned from them (outside the timed region)
    decomp = decompose_runs(fgr, ctx, w, init, pot, stream, flush, runs=20)

    # stage split of FGGC (context timing on; outside the timed region)
    fgr.fgr_set_timing(ctx.handle, True)
    fgr.fgr_reconstruct_fggc(ctx.handle, packets, u_f, stream)
    st = fgr.fgr_get_stats(ctx.handle)
    fggc_stages = {"bounds_alloc_ms": st.prep_ms, "coeff_scatter_ms": st.scatter_ms, "grid_ms": st.grid_ms,
                   "nodes": int(st.nodes)}
    fgr.fgr_reconstruct_direct(ctx.handle, packets, u_d, stream)
    st = fgr.fgr_get_stats(ctx.handle)
    direct_stages = {"bin_ms": st.prep_ms, "sum_ms": st.direct_ms}
    fgr.fgr_set_timing(ctx.handle, False)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    host = {k: np.ascontiguousarray(pk[k]) for k in "qpsa"}
    hwork = {k: np.empty_like(v) for k, v in host.items()}
    hu = np.zeros(shape, dtype=np.complex64 if prec == fgr.FGR_FP32 else np.complex128)
    hu_d = np.zeros_like(hu)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        for k in "qpsa":
            hwork[k][...] = host[k]
        hp = fgr.make_packets(hwork["q"], hwork["p"], hwork["s"], hwork["a"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fgr.fgr_propagate(ctx.handle, hp, pot, t_final, dt)       # H2D, RK4, D2H of the packets
        fgr.fgr_reconstruct_fggc(ctx.handle, hp, hu)               # H2D of the packets, D2H of u
        fgr.fgr_reconstruct_direct(ctx.handle, hp, hu_d)           # H2D of the packets, D2H of u
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    pbytes = sum(v.nbytes for v in host.values())
    h2d = 3 * pbytes
    d2h = pbytes + hu.nbytes + hu_d.nbytes

    def agg(xs):
        return max_over_ranks(statistics.mean(xs), world)

    ms_step = agg(step_ms)
    ms_prop = agg(prop_ms)
    ms_fggc = agg(fggc_ms)
    ms_direct = agg(direct_ms)
    ms_e2e = agg(e2e_ms)
    total_packets = M * world
    kind = w["potential"]["kind"]
    fpps = RK4_FP64_FLOPS_PER_PACKET_STEP.get((d, kind))
    flops = fpps * M * rk4_nsteps(t_final, dt) if fpps else None
    achieved_tflops = flops / (ms_prop * 1e-3) / 1e12 if flops else None
    out = None
    if rank == 0:
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
            "dtype": "f64 trajectories + f32/complex64 reconstruction",
            "data": "synthetic (seeded analytic WKB data, cut-off FFT initial decomposition)",
            "config": {"workload": WORKLOAD, "packets_per_gpu": M, "grid": list(shape), "eps": eps,
                       "t": t_final, "dt": dt, "strategy": "Q4P2 cq=1/2 cp=pi/8",
                       "step": "propagate (A1) + fggc reconstruct (A3-A5) + direct sum (A2), same batch",
                       "l2": "flushed (512 MiB write) between timed steps", "parallelism": "replicas",
                       "autotuned": {"direct_ctas_per_sm": tuning[0], "grid_pass_ctas_per_sm": tuning[1],
                                     "grid_pass_tile": tuning[2]}},
            "stages": {
                "propagate_ms": ms_prop,
                "fggc_reconstruct_ms": ms_fggc,
                "direct_reconstruct_ms": ms_direct,
                "fggc_reconstruct_packets_per_s": total_packets / (ms_fggc * 1e-3),
                "direct_reconstruct_packets_per_s": total_packets / (ms_direct * 1e-3),
                "fggc_over_direct_reconstruct": ms_direct / ms_fggc,
                "fggc_over_direct_pipeline": (ms_prop + ms_direct) / (ms_prop + ms_fggc),
                "rel_l2_fggc_vs_direct": rel,
                "reconstruct_20_runs": recon,
                "decompose_20_runs": decomp,
                "fggc_stage_split": fggc_stages,
                "direct_stage_split": direct_stages,
            },
            "roofline": {"kernel": "rk4_kernel (fgr_propagate)", "bound": "alu",
                         "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved_tflops / FP64_PEAK_TFLOPS if achieved_tflops else None,
                         "traffic": RK4_TRAFFIC_BYTES.get((d, kind, M)),
                         "peak_source": "nominal FP64 rate of the profiling recipe (MEASURED_PEAKS.json has no "
                                        "FP64 figure; a pure-DFMA probe measured 1.19 TFLOP/s)",
                         "flops_per_launch": flops,
                         "flops_counted": "FP64 FLOPs executed per packet-step (ncu: 2 DFMA + DMUL + DADD)"},
            "e2e": {"value": total_packets / (ms_e2e * 1e-3), "unit": "packets/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
        }
        if args.extra:
            out["workloads"] = {}
            for cfg in [int(x) for x in args.extra.split(",") if x]:
                out["workloads"]["config%d" % cfg] = reconstruct_bench(cfg, args, flush)
        if args.batch:
            out["batched_direct"] = batch_bench(args, flush)
        if args.serving:
            out["serving"] = serving_bench(args, local)
        if args.cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_sample)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def reconstruct_runs(fgr, ctx, packets, u_ref, grid, d, eps, prec, flush, stream, ud, runs=20):
    """Median/min/max ms of `runs` reconstructions per method; FGGC with the
    Q4P2 and Q2P2 neighbour sets and Q4P2 through a plan, relative L2
    difference from the direct sum."""
    import numpy as np
    import torch

    q2 = fgr.Context(d, grid, eps, fgr.make_options(precision=prec, nq=2, np_=2))
    u = torch.zeros_like(u_ref)
    out = {}
    for name, fn, c in (("direct", fgr.fgr_reconstruct_direct, ctx), ("fggc_q4p2", fgr.fgr_reconstruct_fggc, ctx),
                        ("fggc_q2p2", fgr.fgr_reconstruct_fggc, q2)):
        for _ in range(3):
            fn(c.handle, packets, u, stream)
        ms = []
        for _ in range(runs):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(c.handle, packets, u, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        got = u.cpu().numpy()
        rel = float(np.linalg.norm(got - ud) / max(np.linalg.norm(ud), 1e-300))
        med = statistics.median(ms)
        out[name] = {"median_ms": med, "min_ms": min(ms), "max_ms": max(ms),
                     "packets_per_s": int(packets.m) / (med * 1e-3), "rel_l2_vs_direct": rel}
    q2.close()
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
    uq2 = torch.zeros(shape, dtype=cdt, device="cuda")
    for name, fn, c, u in (("direct", fgr.fgr_reconstruct_direct, ctx, ud),
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
    a, b, c2 = uf.cpu().numpy(), ud.cpu().numpy(), uq2.cpu().numpy()
    rel = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
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
            "runs": spread, "fggc_q2p2_ms": res["fggc_q2p2"], "rel_l2_fggc_q2p2_vs_direct": rel_q2,
            "fggc_q2p2_over_direct": (res["direct"] / res["fggc_q2p2"] if rel_q2 <= 1e-5
                                      else "not at equal accuracy (rel L2 > 1e-5)"),
            "fggc_nodes": int(st.nodes), "autotuned_ctas_per_sm_and_tile": tuned,
            "decompose": decomp,
            "fggc_stage_split_ms": {"bounds_alloc": st.prep_ms, "coeff_scatter": st.scatter_ms, "grid": st.grid_ms}}


def batch_bench(args, flush):
    """Many small reconstructions: direct sums as one fgr_reconstruct_direct call
    each on one stream, against one fgr_reconstruct_direct_batch call, eager and
    replayed from a CUDA graph; FGGC as one fgr_reconstruct_fggc call each
    against planned calls (fgr_reconstruct_fggc_planned), eager and replayed
    from a CUDA graph.  64 1-D requests, grids 1024..8192 points, 2k..16k
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
    with torch.cuda.stream(s):
        tf_single = timed(fggc_single)
        tf_planned = timed(fggc_planned)
        tf_graph = timed(gf.replay)
    for pl in plans:
        fgr.fgr_fggc_plan_destroy(pl)
    for c in ctxs:
        c.close()
    return {"requests": len(outs), "packets": packets, "single_calls_ms": t_single, "batch_ms": t_batch,
            "graph_replay_ms": t_graph, "requests_per_s_graph": len(outs) / (t_graph * 1e-3),
            "speedup_batch_vs_single": t_single / t_batch, "speedup_graph_vs_single": t_single / t_graph,
            "max_rel_l2_batch_vs_single": worst,
            "fggc_single_calls_ms": tf_single, "fggc_planned_ms": tf_planned, "fggc_graph_replay_ms": tf_graph,
            "fggc_requests_per_s_graph": len(outs) / (tf_graph * 1e-3),
            "max_rel_l2_fggc_planned_vs_single": worst_f,
            "mix": "64 x 1-D, grids 1024..8192, 2k..16k packets, eps 1/1024..1/256, fp32"}


def serving_bench(args, device_index: int):
    """Continuous-batching server under a Poisson stream (the serving workload):
    a pool of packet sets with d in {1, 2}, eps log-uniform in [1/1024, 1/64],
    M = 2^L with L uniform in [12, log2(max packets)] (WKB data on a q x p mesh),
    propagated once to t = 0.5 on the GPU and kept resident; each request picks
    a set, a grid (1-D: 1024..32768 points, 2-D: 256^2..1024^2, powers of two)
    and a method (direct / FGGC) uniformly; FP32.  Capacity = 1 / mean isolated
    service time; p50/p99 of submit-to-done latency and packets/s at 0.5x, 0.8x
    and 1.0x capacity."""
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
    capacity = 1e3 / float(np.mean(iso))
    # saturated throughput: a burst submitted at once, all slots busy
    burst = [draw() for _ in range(args.serve_probe)]
    bouts = [torch.zeros(tuple(g["n"]), dtype=torch.complex64, device="cuda") for (_, _, _, _, g, _) in burst]
    tb0 = time.perf_counter()
    bt = [fgr.fgr_submit(srv, fgr.make_request(mth, g, e, opt, sid, u))
          for (sid, d, e, m, g, mth), u in zip(burst, bouts)]
    for t in bt:
        fgr.fgr_poll(srv, t, -1)
    burst_rate = len(burst) / (time.perf_counter() - tb0)
    del bouts
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
        ok = all(r.status == 0 for r in res)
        packets = sum(q[3] for q in reqs)
        levels["%.1fx" % frac] = {"lambda_req_per_s": lam, "p50_ms": float(np.percentile(lat, 50)),
                                  "p99_ms": float(np.percentile(lat, 99)), "packets_per_s": packets / (t1 - t0),
                                  "requests": len(reqs), "all_ok": ok}
        del outs
    fgr.fgr_server_destroy(srv)
    ms = [m for (_, _, _, m) in sets]
    return {"sets": len(sets), "packets_min": min(ms), "packets_max": max(ms), "setup_s_untimed": t_setup,
            "inflight": args.serve_inflight, "max_batch": 16, "isolated_service_ms_mean": float(np.mean(iso)),
            "isolated_service_ms_p50": float(np.percentile(iso, 50)),
            "capacity_req_per_s": capacity, "burst_req_per_s": burst_rate, "levels": levels,
            "mix": "d in {1,2}; grids 1-D 1024..32768, 2-D 256^2..1024^2; direct/fggc 50/50; fp32"}


def cpu_baseline(w, sample: int):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    `sample` packets propagated (C RK4, OpenMP) and reconstructed by the
    oracle's FGGC and by its direct sum on the full output grid."""
    import numpy as np

    from oracle import fga, fggc, lsa, trajectories
    pk = w["packets"]
    M = pk["s"].size
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(M, size=min(sample, M), replace=False))
    sub = {k: np.ascontiguousarray(pk[k][..., idx]) for k in ("q", "p", "s", "a")}
    mesh = w["mesh"]
    t0 = time.perf_counter()
    prop = trajectories.propagate(sub, w["potential"], w["t"], w["dt"])
    t1 = time.perf_counter()
    R = 6 if w["precision"] == "fp32" else 8
    fggc.reconstruct(prop, w["grid"], w["eps"], mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2), R=R)
    t2 = time.perf_counter()
    fga.direct_sum(prop, w["grid"], w["eps"], mesh.dq, mesh.dp, R=R)
    t3 = time.perf_counter()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": idx.size / (t3 - t0), "unit": "packets/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d packets (uniform sample, seed 0): propagate %.2f s (C RK4, OpenMP %d threads) "
                      "+ FGGC reconstruct %.2f s + direct sum %.2f s (numpy, 1 thread) on the full grid"
                      % (idx.size, M, t1 - t0, cores, t2 - t1, t3 - t2)}


def run_reference(args):
    rank, _, world = _rank_env()
    if rank != 0:
        return None
    from workloads import config_workload
    w = config_workload(args.config)
    times, vals = [], []
    last = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(w, args.ref_sample)
        if i >= args.warmup:
            vals.append(cb["value"])
            last = cb
    value = statistics.mean(vals)
    ms = args.ref_sample / value * 1e3
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "packets/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "packets_per_step": args.ref_sample,
                       "step": "propagate + fggc reconstruct + direct sum of a packet sample (oracle)"},
            "cpu_baseline": {"value": value, "unit": "packets/s", "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": value, "unit": "packets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """One short pass of every kernel on the benchmark workload, for ncu:
    propagate to t = 0.01 (100 RK4 steps), then one FGGC and one direct
    reconstruction of the propagated packets, one batched direct sum of
    eight copies of that request and one initial decomposition of the
    reconstructed wave onto the propagated positions (FGGC only for 3-D
    workloads); for d >= 2 one tensor-product decomposition of that wave onto
    the t = 0 mesh."""
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
        if d < 3:  # the 3-D direct sum takes seconds: FGGC only there
            fgr.fgr_reconstruct_direct(ctx.handle, pk, u)
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
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-sample", type=int, default=2048)
    ap.add_argument("--ref-sample", type=int, default=512)
    ap.add_argument("--extra", default="3", help="other workloads to reconstruct, e.g. 3,4 ('' for none)")
    ap.add_argument("--no-serving", dest="serving", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--serve-sets", type=int, default=32)
    ap.add_argument("--serve-max-packets", type=int, default=1 << 22)
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-probe", type=int, default=40)
    ap.add_argument("--serve-inflight", type=int, default=4)
    ap.add_argument("--profile-packets", type=int, default=0,
                    help="with --profile: keep only this many largest-amplitude packets")
    ap.add_argument("--profile", action="store_true",
                    help="run every kernel once on a short case (for ncu) and exit")
    ap.add_argument("--study", choices=["multistep"], default=None,
                    help="print the runtimes of the multi-step examples of Sec. 4.4 and exit")
    ap.add_argument("--study-precision", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args()
    if args.profile:
        run_profile_case(args)
        return
    if args.study == "multistep":
        print(json.dumps(multistep_study(args)))
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
