"""WKB initial data, phase-space meshes and packet sets (inputs only).

Conventions shared by every consumer of these inputs:

* Uniform output grid per dimension: x_m = lo + m*(hi-lo)/n, m in [0, n).
* Mesh strategy (eq. 3.5): dq = cq*sqrt(eps), dp = cp*sqrt(eps); the paper's
  recommended mesh (Remark after Table 4) is cq = 1/2, cp = pi/8.
* q-nodes per dimension: q_a = (a - Nq/2)*dq, a in [0, Nq).
* p-nodes per q (Remark 1: the p-mesh sits around grad S0(q)):
  p_b = (round(dS0(q)/dp) + b - Np/2)*dp, b in [0, Np).
* Packet linear index: (a_1..a_d, b_1..b_d) in row-major order.
* Packet arrays (structure of arrays, float64):
  q[d][M], p[d][M], s[M], a[2][M] (real plane, imaginary plane).

The initial amplitudes are A(0,q,p) = 2^{d/2} u0hat(q,p) (eq. 2.6) with
u0hat from eq. 2.8, evaluated by the cut-off FFT of Remark 1: for each q the
y-integral is a trapezoid sum over one period of the p-lattice phase, which is
a length-L DFT.  The WKB data used here are separable, u0(x) = prod_l u0_l(x_l),
so u0hat and A factor per dimension as well.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Mesh:
    """Phase-space mesh of eq. 3.5 for one value of eps."""

    d: int
    eps: float
    cq: float = 0.5
    cp: float = math.pi / 8

    @property
    def sigma(self) -> float:
        return math.sqrt(self.eps)

    @property
    def dq(self) -> float:
        return self.cq * math.sqrt(self.eps)

    @property
    def dp(self) -> float:
        return self.cp * math.sqrt(self.eps)


def mesh_for(d: int, eps: float, cq: float = 0.5, cp: float = math.pi / 8) -> Mesh:
    return Mesh(d=d, eps=eps, cq=cq, cp=cp)


# --------------------------------------------------------------------------
# WKB data u0 = sqrt(n0) exp(i S0 / eps) (eq. 1.2), separable per dimension.
# Each family gives, per dimension l, sqrt(n0)_l(y), S0_l(y) and dS0_l(y).
# --------------------------------------------------------------------------

class _Family:
    name = "base"

    def sqrt_n0(self, l: int, y):
        raise NotImplementedError

    def s0(self, l: int, y):
        raise NotImplementedError

    def ds0(self, l: int, y):
        raise NotImplementedError

    def u0(self, x, eps):
        """u0 on points x with shape (d, ...); product of the per-dim factors."""
        x = np.asarray(x, dtype=np.float64)
        out = np.ones(x.shape[1:], dtype=np.complex128)
        for l in range(x.shape[0]):
            out = out * self.sqrt_n0(l, x[l]) * np.exp(1j * self.s0(l, x[l]) / eps)
        return out


class _Tanh(_Family):
    """n0 = exp(-25|x|^2), S0 = -log(2 cosh(5 x_1))/5 (the 1-D and 2-D workloads)."""

    name = "tanh"

    def sqrt_n0(self, l, y):
        return np.exp(-12.5 * np.asarray(y) ** 2)

    def s0(self, l, y):
        y = np.asarray(y, dtype=np.float64)
        if l != 0:
            return np.zeros_like(y)
        # log(2 cosh z) = |z| + log1p(exp(-2|z|)), stable for large |z|
        z = 5.0 * y
        return -(np.abs(z) + np.log1p(np.exp(-2.0 * np.abs(z)))) / 5.0

    def ds0(self, l, y):
        y = np.asarray(y, dtype=np.float64)
        if l != 0:
            return np.zeros_like(y)
        return -np.tanh(5.0 * y)


class _Linear(_Family):
    """n0 = exp(-25|x|^2), S0 = x_1 + ... + x_d (the 3-D harmonic workload)."""

    name = "linear"

    def sqrt_n0(self, l, y):
        return np.exp(-12.5 * np.asarray(y) ** 2)

    def s0(self, l, y):
        return np.asarray(y, dtype=np.float64).copy()

    def ds0(self, l, y):
        return np.ones_like(np.asarray(y, dtype=np.float64))


WKB_TANH = _Tanh()
WKB_LINEAR = _Linear()


def _next_pow2(n: int) -> int:
    return 1 << max(0, int(n - 1).bit_length())


def _amplitude_table_1d(fam: _Family, l: int, mesh: Mesh, nq: int, np_: int):
    """Per-dimension factor sqrt(2) * u0hat_l(q_a, p_{a,b}) on the (a, b) mesh.

    Returns (q[nq], p[nq, np_], amp[nq, np_]) with amp complex128.
    """
    eps, dq, dp = mesh.eps, mesh.dq, mesh.dp
    a = np.arange(nq)
    q = (a - nq // 2) * dq
    centre = np.rint(fam.ds0(l, q) / dp).astype(np.int64)
    beta = centre[:, None] + (np.arange(np_)[None, :] - np_ // 2)  # p lattice index
    p = beta * dp
    # Cut-off FFT (Remark 1): with h = 2*pi*eps/(dp*L) the kernel
    # exp(-i beta dp (y-q)/eps) at y = q + k h is exp(-2 pi i beta k / L).
    L = _next_pow2(max(4 * np_, 256))
    h = 2.0 * math.pi * eps / (dp * L)
    k = np.arange(-L // 2, L // 2)
    y = q[:, None] + k[None, :] * h
    f = (fam.sqrt_n0(l, y) * np.exp(1j * fam.s0(l, y) / eps)
         * np.exp(-((k * h) ** 2) / (2.0 * eps))[None, :])
    x = np.zeros((nq, L), dtype=np.complex128)
    x[:, np.mod(k, L)] = f
    spec = np.fft.fft(x, axis=1) * h
    u0hat = np.take_along_axis(spec, np.mod(beta, L), axis=1)
    return q, p, math.sqrt(2.0) * u0hat


def wkb_packets(d: int, eps: float, nq: int, np_: int, family: _Family = WKB_TANH,
                cq: float = 0.5, cp: float = math.pi / 8):
    """All packets of the (nq per dim) x (np_ per dim) phase-space mesh at t = 0.

    Returns a dict with q (d,M), p (d,M), s (M,), a (2,M) float64 arrays, and the
    mesh.  M = nq^d * np_^d; the packet index is (a_1..a_d, b_1..b_d) row-major.
    """
    mesh = Mesh(d=d, eps=eps, cq=cq, cp=cp)
    tabs = [_amplitude_table_1d(family, l, mesh, nq, np_) for l in range(d)]
    # index grids in (a_1..a_d, b_1..b_d) order
    shape = (nq,) * d + (np_,) * d
    idx = np.indices(shape, sparse=True)
    qs, ps = [], []
    amp = np.ones(shape, dtype=np.complex128)
    for l in range(d):
        ql, pl, al = tabs[l]
        ia, ib = idx[l], idx[d + l]
        qs.append(np.broadcast_to(ql[ia], shape))
        ps.append(np.broadcast_to(pl[ia, ib], shape))
        amp = amp * al[ia, ib]
    M = int(np.prod(shape))
    q = np.stack([x.reshape(M) for x in qs]).astype(np.float64)
    p = np.stack([x.reshape(M) for x in ps]).astype(np.float64)
    a = amp.reshape(M)
    return {
        "q": np.ascontiguousarray(q),
        "p": np.ascontiguousarray(p),
        "s": np.zeros(M, dtype=np.float64),
        "a": np.ascontiguousarray(np.stack([a.real, a.imag])),
        "mesh": mesh,
    }


def mesh_axes(d: int, eps: float, nq: int, np_: int, family: _Family = WKB_TANH,
              cq: float = 0.5, cp: float = math.pi / 8):
    """The mesh of wkb_packets as a tensor product of per-dimension lists.

    Returns (axes, sel): axes[l] = (q, p), nq * np_ pairs ordered (a, b)
    row-major; sel[j] = the row-major tensor-product index of wkb_packets'
    packet j, so packet j sits at (axes[l][0][i_l], axes[l][1][i_l]).
    """
    mesh = Mesh(d=d, eps=eps, cq=cq, cp=cp)
    axes = []
    for l in range(d):
        a = np.arange(nq)
        q = (a - nq // 2) * mesh.dq
        centre = np.rint(family.ds0(l, q) / mesh.dp).astype(np.int64)
        beta = centre[:, None] + (np.arange(np_)[None, :] - np_ // 2)
        axes.append((np.ascontiguousarray(np.repeat(q, np_)), np.ascontiguousarray((beta * mesh.dp).reshape(-1))))
    idx = np.indices((nq,) * d + (np_,) * d).reshape(2 * d, -1)
    L = nq * np_
    sel = np.zeros(idx.shape[1], dtype=np.int64)
    for l in range(d):
        sel = sel * L + idx[l] * np_ + idx[d + l]
    return axes, sel


def workload_axes(w: dict):
    """(axes, sel) of a config_workload's t = 0 packets (kept ones only where
    the workload keeps the largest amplitudes)."""
    axes, sel = mesh_axes(w["d"], w["eps"], w["nq"], w["np_"], _FAMILIES[w["family"]])
    keep = w["packets"].get("kept_index")
    if keep is not None:
        sel = sel[keep]
    return axes, np.ascontiguousarray(sel)


def select_top(packets: dict, pref: float, threshold: float, cap: int) -> dict:
    """Keep packets with pref*|A| > threshold; if more than `cap` remain keep the
    `cap` largest, ties broken towards the lower packet index."""
    a = packets["a"]
    mag = pref * np.hypot(a[0], a[1])
    keep = np.nonzero(mag > threshold)[0]
    if keep.size > cap:
        m = mag[keep]
        kth = np.partition(m, keep.size - cap)[keep.size - cap]  # cap-th largest
        above = keep[m > kth]
        ties = keep[m == kth][: cap - above.size]
        keep = np.sort(np.concatenate([above, ties]))
    out = dict(packets)
    out["q"] = np.ascontiguousarray(packets["q"][:, keep])
    out["p"] = np.ascontiguousarray(packets["p"][:, keep])
    out["s"] = np.ascontiguousarray(packets["s"][keep])
    out["a"] = np.ascontiguousarray(packets["a"][:, keep])
    out["kept_index"] = keep
    return out


# --------------------------------------------------------------------------
# The five workloads (uniform grids on [-pi, pi)^d).
# --------------------------------------------------------------------------

CONFIGS = {
    1: dict(name="d1_eps1/64_n1024_M4096_fp64", d=1, eps=1 / 64, n=1024, nq=64, np_=64,
            family="tanh", potential=dict(kind="cossum", c0=1.0, amp=-1.0, k=1.0),
            t=0.5, dt=1e-4, precision="fp64"),
    2: dict(name="d1_eps1/1024_n32768_M262144_fp32", d=1, eps=1 / 1024, n=32768, nq=512, np_=512,
            family="tanh", potential=dict(kind="cossum", c0=1.0, amp=-1.0, k=1.0),
            t=1.0, dt=1e-4, precision="fp32"),
    3: dict(name="d2_eps1/256_n1024^2_M4194304_fp32", d=2, eps=1 / 256, n=1024, nq=64, np_=32,
            family="tanh", potential=dict(kind="cossum", c0=2.0, amp=1.0, k=1.0),
            t=0.5, dt=1e-4, precision="fp32"),
    4: dict(name="d3_eps1/64_n256^3_M16777216_fp32", d=3, eps=1 / 64, n=256, nq=32, np_=16,
            family="linear", potential=dict(kind="harmonic", omega=1.0),
            t=0.5, dt=1e-4, precision="fp32", threshold=1e-8, cap=1 << 24),
}

_FAMILIES = {"tanh": WKB_TANH, "linear": WKB_LINEAR}


def config_workload(cfg: int, **override) -> dict:
    """Packets (t = 0), grid and run parameters of one workload."""
    c = dict(CONFIGS[cfg])
    c.update(override)
    d = c["d"]
    pk = wkb_packets(d, c["eps"], c["nq"], c["np_"], _FAMILIES[c["family"]])
    mesh = pk["mesh"]
    if "threshold" in c:
        pref = (mesh.dq * mesh.dp) ** d / (2 * math.pi * c["eps"]) ** (1.5 * d)
        pk = select_top(pk, pref, c["threshold"], c["cap"])
    c["packets"] = pk
    c["mesh"] = mesh
    c["grid"] = dict(d=d, n=[c["n"]] * d, lo=[-math.pi] * d, hi=[math.pi] * d)
    return c


# --------------------------------------------------------------------------
# Seeded random packet sets for unit tests and edge cases.
# --------------------------------------------------------------------------

def random_packets(seed: int, d: int, m: int, q_range=(-1.0, 1.0), p_range=(-1.0, 1.0),
                   s_range=(-1.0, 1.0), mesh: Mesh | None = None, on_node_fraction=0.0):
    """m packets with uniform Q, P, S and complex-normal A.

    With a mesh and on_node_fraction > 0, that fraction of the packets is moved
    exactly onto mesh nodes (Q = a*dq, P = b*dp as float64 products).
    """
    rng = np.random.default_rng(seed)
    q = rng.uniform(q_range[0], q_range[1], size=(d, m))
    p = rng.uniform(p_range[0], p_range[1], size=(d, m))
    s = rng.uniform(s_range[0], s_range[1], size=m)
    a = rng.standard_normal((2, m))
    if mesh is not None and on_node_fraction > 0 and m > 0:
        k = max(1, int(on_node_fraction * m))
        sel = rng.choice(m, size=k, replace=False)
        q[:, sel] = np.floor(q[:, sel] / mesh.dq) * mesh.dq
        p[:, sel] = np.floor(p[:, sel] / mesh.dp) * mesh.dp
    return {"q": np.ascontiguousarray(q), "p": np.ascontiguousarray(p),
            "s": s, "a": np.ascontiguousarray(a), "mesh": mesh}
