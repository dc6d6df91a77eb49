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


def rk4_nsteps(t: float, dt: float) -> int:
    """Step count rule of fgr_propagate (include/fgr.h)."""
    r = t / dt
    n = round(r)
    return int(n) if abs(r - n) <= 1e-9 * max(n, 1.0) else int(math.ceil(r))


def rk4_flops_per_packet_step(d: int) -> int:
    """Algorithmic FP64 operations of one RK4 step of eq. 2.3-2.7 for a separable
    cosine potential, per packet (sin and cos counted as one operation each,
    a division as one): 4 right-hand sides of (per dimension 2 trig + 27
    arithmetic, plus 9 for S and A) and 4 state updates of 2 ops per variable."""
    nvar = 6 * d + 3
    rhs = d * (2 + 27) + 9
    return 4 * rhs + 4 * 2 * nvar + 2 * nvar


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

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches["n"] = 0
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
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
    step_ms = [a + b for a, b in zip(prop_ms, fggc_ms)]
    gpu_launches = launches["n"]

    # direct sum on the same propagated batch (A2), same stream, L2 flushed between runs
    dev_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for _ in range(max(1, args.warmup)):
        fgr.fgr_reconstruct_direct(ctx.handle, packets, u_d, stream)
    for i in range(args.steps):
        flush.zero_()
        dev_ev[i][0].record(stream)
        fgr.fgr_reconstruct_direct(ctx.handle, packets, u_d, stream)
        dev_ev[i][1].record(stream)
    torch.cuda.synchronize()
    direct_ms = [e[0].elapsed_time(e[1]) for e in dev_ev]
    ud, uf = u_d.cpu().numpy(), u_f.cpu().numpy()
    rel = float(np.linalg.norm(uf - ud) / max(np.linalg.norm(ud), 1e-300))

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
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        for k in "qpsa":
            hwork[k][...] = host[k]
        hp = fgr.make_packets(hwork["q"], hwork["p"], hwork["s"], hwork["a"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fgr.fgr_propagate(ctx.handle, hp, pot, t_final, dt)       # H2D, RK4, D2H of the packets
        fgr.fgr_reconstruct_fggc(ctx.handle, hp, hu)               # H2D of the packets, D2H of u
        t1 = time.perf_counter()
        if i >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
    pbytes = sum(v.nbytes for v in host.values())
    h2d = 2 * pbytes
    d2h = pbytes + hu.nbytes

    def agg(xs):
        t = torch.tensor([statistics.mean(xs)], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    ms_step = agg(step_ms)
    ms_prop = agg(prop_ms)
    ms_fggc = agg(fggc_ms)
    ms_direct = agg(direct_ms)
    ms_e2e = agg(e2e_ms)
    total_packets = M * world
    flops = rk4_flops_per_packet_step(d) * M * rk4_nsteps(t_final, dt)
    achieved_tflops = flops / (ms_prop * 1e-3) / 1e12
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
                       "step": "propagate (A1) + fggc reconstruct (A3-A5)",
                       "l2": "flushed (512 MiB write) between timed steps", "parallelism": "replicas"},
            "stages": {
                "propagate_ms": ms_prop,
                "fggc_reconstruct_ms": ms_fggc,
                "direct_reconstruct_ms": ms_direct,
                "fggc_reconstruct_packets_per_s": total_packets / (ms_fggc * 1e-3),
                "direct_reconstruct_packets_per_s": total_packets / (ms_direct * 1e-3),
                "fggc_over_direct_reconstruct": ms_direct / ms_fggc,
                "fggc_over_direct_pipeline": (ms_prop + ms_direct) / (ms_prop + ms_fggc),
                "rel_l2_fggc_vs_direct": rel,
                "fggc_stage_split": fggc_stages,
                "direct_stage_split": direct_stages,
            },
            "roofline": {"kernel": "rk4_kernel<1> (fgr_propagate)", "bound": "alu",
                         "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved_tflops / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "nominal FP64 rate of the profiling recipe (not in MEASURED_PEAKS.json)",
                         "flops_per_launch": flops},
            "e2e": {"value": total_packets / (ms_e2e * 1e-3), "unit": "packets/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches,
            "clocks": clk.summary(),
        }
        if args.cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(w, args.cpu_sample)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def cpu_baseline(w, sample: int):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    `sample` packets propagated (C RK4, OpenMP) and reconstructed by the
    oracle's FGGC on the full output grid."""
    import numpy as np

    from oracle import fggc, lsa, trajectories
    pk = w["packets"]
    M = pk["s"].size
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(M, size=min(sample, M), replace=False))
    sub = {k: np.ascontiguousarray(pk[k][..., idx]) for k in ("q", "p", "s", "a")}
    mesh = w["mesh"]
    t0 = time.perf_counter()
    prop = trajectories.propagate(sub, w["potential"], w["t"], w["dt"])
    t1 = time.perf_counter()
    fggc.reconstruct(prop, w["grid"], w["eps"], mesh.dq, mesh.dp, lsa.Strategy(nq=4, np_=2),
                     R=6 if w["precision"] == "fp32" else 8)
    t2 = time.perf_counter()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": idx.size / (t2 - t0), "unit": "packets/s", "cores": cores, "kind": "oracle",
            "sample": "%d of %d packets (uniform sample, seed 0): propagate %.2f s (C RK4, OpenMP %d threads) "
                      "+ FGGC reconstruct %.2f s (numpy, 1 thread) on the full grid"
                      % (idx.size, M, t1 - t0, cores, t2 - t1)}


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
                       "step": "propagate + fggc reconstruct of a packet sample (oracle)"},
            "cpu_baseline": {"value": value, "unit": "packets/s", "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": value, "unit": "packets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


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
    args = ap.parse_args()
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
