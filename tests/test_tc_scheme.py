"""The arithmetic scheme of the tensor-core direct sum, checked on the CPU in
numpy: (1) the complex product U = F_row F_last^T of eq. 2.10's per-dimension
factors equals the real product of the operand layout the kernel writes
(A[row][2r + c] = (Re, Im) F_row; B[j] = (Re, -Im) F_last and
B[N + j] = (Im, Re) F_last), read back as Re in columns j and Im in N + j;
(2) splitting each factor into hi = x truncated to TF32 and lo = x - hi (read
by the tensor core as lo truncated to TF32) and summing hi*hi + hi*lo + lo*hi
reproduces each product to better than 3 x 2^-20 of |a| |b| (the three dropped
terms, lo*lo and the two truncations of lo, are each below 2^-20)."""

import numpy as np


def _tf32_trunc(x):
    """x (float32) with the 13 low mantissa bits cleared."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32)


def test_complex_product_as_real_operands():
    rng = np.random.default_rng(0)
    rows, n, rec = 128, 64, 16
    f_row = rng.normal(size=(rec, rows)) + 1j * rng.normal(size=(rec, rows))
    f_last = rng.normal(size=(rec, n)) + 1j * rng.normal(size=(rec, n))
    A = np.zeros((rows, 2 * rec))
    B = np.zeros((2 * n, 2 * rec))
    A[:, 0::2], A[:, 1::2] = f_row.real.T, f_row.imag.T
    B[:n, 0::2], B[:n, 1::2] = f_last.real.T, -f_last.imag.T
    B[n:, 0::2], B[n:, 1::2] = f_last.imag.T, f_last.real.T
    D = A @ B.T
    U = f_row.T @ f_last          # sum over records of the outer products
    assert np.allclose(D[:, :n] + 1j * D[:, n:], U, rtol=1e-12, atol=1e-12)


def test_three_tf32_products_reach_fp32_accuracy():
    rng = np.random.default_rng(1)
    # factors over the range the kernel meets: Gaussian tails times amplitudes
    a = (rng.normal(size=200000) * np.exp(rng.uniform(-30, 5, 200000))).astype(np.float32)
    b = (rng.normal(size=200000) * np.exp(rng.uniform(-30, 5, 200000))).astype(np.float32)
    ah, bh = _tf32_trunc(a), _tf32_trunc(b)
    al, bl = (a - ah).astype(np.float32), (b - bh).astype(np.float32)   # exact in FP32
    al_t, bl_t = _tf32_trunc(al), _tf32_trunc(bl)                          # what the tensor core reads
    # each product of two TF32 values is exact in FP64
    approx = (ah.astype(np.float64) * bh + ah.astype(np.float64) * bl_t + al_t.astype(np.float64) * bh)
    exact = a.astype(np.float64) * b.astype(np.float64)
    rel = np.abs(approx - exact) / (np.abs(a.astype(np.float64)) * np.abs(b.astype(np.float64)))
    assert rel.max() < 3 * 2.0 ** -20
    assert np.median(rel) < 2.0 ** -21
    # a single TF32 product is not enough for FP32 results
    one = ah.astype(np.float64) * bh
    assert (np.abs(one - exact) / np.abs(exact)).max() > 2.0 ** -12
