"""GPU-side helpers for the parity tests: run the library through its C ABI on
numpy inputs (device copies made with torch) and return numpy results."""

from __future__ import annotations

import numpy as np

import paper_2504_21785_gb300 as fgr


def _torch():
    import torch
    return torch


def to_device(pk: dict):
    torch = _torch()
    return tuple(torch.tensor(np.ascontiguousarray(pk[k]), dtype=torch.float64, device="cuda")
                 for k in ("q", "p", "s", "a"))


def options(precision="fp64", nq=4, np_=2, window_r=0.0, cq=0.5, cp=np.pi / 8, flags=0):
    prec = fgr.FGR_FP64 if precision == "fp64" else fgr.FGR_FP32
    return fgr.make_options(precision=prec, nq=nq, np_=np_, window_r=window_r, cq=cq, cp=cp, flags=flags)


def reconstruct(method: str, pk: dict, grid: dict, eps: float, opt, on_device=True, ctx=None):
    """Runs fgr_reconstruct_{direct,fggc}; returns u as a numpy complex array."""
    torch = _torch()
    shape = tuple(int(n) for n in grid["n"][: grid["d"]])
    dtype = torch.complex128 if opt.precision == fgr.FGR_FP64 else torch.complex64
    own = ctx is None
    if own:
        ctx = fgr.Context(grid["d"], grid, eps, opt)
    try:
        fn = fgr.fgr_reconstruct_fggc if method == "fggc" else fgr.fgr_reconstruct_direct
        if on_device:
            arrs = to_device(pk)
            u = torch.zeros(shape, dtype=dtype, device="cuda")
            fn(ctx.handle, fgr.make_packets(*arrs), u)
            torch.cuda.synchronize()
            return u.cpu().numpy()
        host = [np.ascontiguousarray(pk[k], dtype=np.float64) for k in ("q", "p", "s", "a")]
        u = np.zeros(shape, dtype=np.complex128 if dtype == torch.complex128 else np.complex64)
        fn(ctx.handle, fgr.make_packets(*host), u)
        return u
    finally:
        if own:
            ctx.close()


def propagate(pk: dict, d: int, potential: dict, t: float, dt: float, on_device=True):
    torch = _torch()
    grid = dict(d=d, n=[8] * d, lo=[-1.0] * d, hi=[1.0] * d)
    with fgr.Context(d, grid, 1.0) as ctx:
        pot = fgr.make_potential(**potential)
        if on_device:
            arrs = to_device(pk)
            fgr.fgr_propagate(ctx.handle, fgr.make_packets(*arrs), pot, t, dt)
            torch.cuda.synchronize()
            return {k: v.cpu().numpy() for k, v in zip(("q", "p", "s", "a"), arrs)}
        host = {k: np.array(pk[k], dtype=np.float64, order="C", copy=True) for k in ("q", "p", "s", "a")}
        fgr.fgr_propagate(ctx.handle, fgr.make_packets(host["q"], host["p"], host["s"], host["a"]),
                          pot, t, dt)
        return host


def rel_l2(x, ref) -> float:
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(np.asarray(x) - ref) / (den if den > 0 else 1.0))
