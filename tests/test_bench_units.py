"""The unit counts behind bench.py's direct-sum roofline: window_pairs (the
packet-point pairs inside the box windows, eq. 2.10) equals the oracle's
window rule summed over the packets, and brute-force enumeration of the grid
points within R sqrt(eps) of each centre on a small grid (CPU only)."""

import math

import numpy as np

import bench
from oracle import fga
from workloads import random_packets


def _grid(d, n):
    return dict(d=d, n=list(n), lo=[-math.pi] * d, hi=[math.pi] * d)


def test_window_pairs_equals_the_oracle_windows():
    eps = 1 / 256
    for d, n in ((1, (3001,)), (2, (70, 101)), (3, (20, 17, 23))):
        pk = random_packets(7 + d, d, 500, q_range=(-3.6, 3.6))   # windows leave the grid at both ends
        grid = _grid(d, n)
        want = np.ones(500)
        for l in range(d):
            lo, hi = fga.window_bounds(pk["q"][l], grid, l, eps, 6.0)
            want *= np.maximum(hi - lo + 1, 0)
        assert bench.window_pairs(pk["q"], grid, eps) == float(want.sum())


def test_window_pairs_by_enumeration():
    eps = 1 / 64
    grid = _grid(2, (40, 33))
    pk = random_packets(12, 2, 60, q_range=(-3.4, 3.4))
    rs = 6.0 * math.sqrt(eps)
    total = 0
    for j in range(60):
        cnt = 1
        for l in range(2):
            n = grid["n"][l]
            h = 2 * math.pi / n
            x = -math.pi + h * np.arange(n)
            cnt *= int(np.sum(np.abs(x - pk["q"][l, j]) <= rs))
        total += cnt
    assert bench.window_pairs(pk["q"], grid, eps) == total


def test_direct_roofline_fields():
    r = bench.direct_roofline(1e12, 10.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["achieved"], 24 * 1e12 / 0.01 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / bench.TF32_PEAK_TFLOPS)
    assert math.isclose(bench.TF32_PEAK_TFLOPS, bench.BF16_MEASURED_TFLOPS * 1.1 / 2.25)
