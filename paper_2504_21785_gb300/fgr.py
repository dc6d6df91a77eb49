"""ctypes binding of libfgr (include/fgr.h): argument marshalling only.

Every function keeps its C name.  Arrays may be numpy arrays (host) or torch
tensors (host or CUDA); their data pointers are passed straight to the library,
which does all of the computation.  Nothing here falls back to a CPU path: if
libfgr.so is missing or cannot be loaded, every call raises.
"""

from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfgr.so")

FGR_OK, FGR_E_INVALID, FGR_E_NOMEM, FGR_E_CUDA, FGR_E_NOT_READY = 0, 1, 2, 3, 4
FGR_E_TIMEOUT, FGR_E_CAPACITY, FGR_E_CANCELLED, FGR_E_INTERNAL = 5, 6, 7, 8
FGR_FP64, FGR_FP32 = 0, 1
FGR_V_FREE, FGR_V_COSSUM, FGR_V_HARMONIC = 0, 1, 2
STATUS_NAMES = {0: "FGR_OK", 1: "FGR_E_INVALID", 2: "FGR_E_NOMEM", 3: "FGR_E_CUDA",
                4: "FGR_E_NOT_READY", 5: "FGR_E_TIMEOUT", 6: "FGR_E_CAPACITY",
                7: "FGR_E_CANCELLED", 8: "FGR_E_INTERNAL"}


class FgrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class fgr_grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class fgr_options(ctypes.Structure):
    _fields_ = [("cq", ctypes.c_double), ("cp", ctypes.c_double), ("nq", ctypes.c_int32),
                ("np", ctypes.c_int32), ("window_r", ctypes.c_double), ("rcond", ctypes.c_double),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32)]


class fgr_packets(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("q", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("s", ctypes.c_void_p), ("a", ctypes.c_void_p), ("on_device", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


FGR_MAX_DIM = 3


class fgr_axis(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("q", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class fgr_potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("c0", ctypes.c_double),
                ("amp", ctypes.c_double), ("k", ctypes.c_double), ("omega", ctypes.c_double)]


class fgr_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n1", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("eps", ctypes.c_double), ("dq", ctypes.c_double),
                ("dp", ctypes.c_double), ("pref", ctypes.c_double), ("window_r", ctypes.c_double),
                ("eigenvalues", ctypes.c_double * 16)]


class fgr_stats(ctypes.Structure):
    _fields_ = [("prep_ms", ctypes.c_double), ("coeff_ms", ctypes.c_double),
                ("scatter_ms", ctypes.c_double), ("grid_ms", ctypes.c_double),
                ("direct_ms", ctypes.c_double), ("propagate_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("pairs", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("pass_ms", ctypes.c_double), ("pass_terms", ctypes.c_int64)]


class fgr_request(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("d", ctypes.c_int32), ("grid", fgr_grid),
                ("eps", ctypes.c_double), ("opt", fgr_options), ("set_id", ctypes.c_uint64),
                ("u_out", ctypes.c_void_p)]


class fgr_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


# Every exported symbol of include/fgr.h with (restype, argtypes).
P = ctypes.POINTER
vp = ctypes.c_void_p
SIGNATURES = {
    "fgr_default_options": (ctypes.c_int, [P(fgr_options)]),
    "fgr_create": (ctypes.c_int, [ctypes.c_int32, P(fgr_grid), ctypes.c_double, P(fgr_options), P(vp)]),
    "fgr_destroy": (None, [vp]),
    "fgr_last_error": (ctypes.c_char_p, []),
    "fgr_propagate": (ctypes.c_int, [vp, P(fgr_packets), P(fgr_potential), ctypes.c_double,
                                     ctypes.c_double, vp]),
    "fgr_decompose": (ctypes.c_int, [vp, vp, P(fgr_packets), vp]),
    "fgr_fggc_multistep": (ctypes.c_int, [vp, P(fgr_packets), P(fgr_packets), vp, vp, ctypes.c_int32, vp]),
    "fgr_decompose_tensor": (ctypes.c_int, [vp, P(fgr_axis), vp, ctypes.c_int64, vp, vp, vp]),
    "fgr_fggc_multistep_tensor": (ctypes.c_int, [vp, P(fgr_axis), vp, P(fgr_packets), vp, vp, ctypes.c_int32, vp]),
    "fgr_reconstruct_direct": (ctypes.c_int, [vp, P(fgr_packets), vp, vp]),
    "fgr_reconstruct_fggc": (ctypes.c_int, [vp, P(fgr_packets), vp, vp]),
    "fgr_reconstruct_fggc_noalloc": (ctypes.c_int, [vp, P(fgr_packets), vp, vp]),
    "fgr_reconstruct_direct_batch": (ctypes.c_int, [ctypes.c_int32, P(vp), P(P(fgr_packets)), P(vp), vp]),
    "fgr_fggc_plan_create": (ctypes.c_int, [vp, P(fgr_packets), ctypes.c_int32, P(vp), vp]),
    "fgr_reconstruct_fggc_planned": (ctypes.c_int, [vp, vp, P(fgr_packets), vp, vp]),
    "fgr_reconstruct_fggc_batch": (ctypes.c_int, [ctypes.c_int32, P(vp), P(vp), P(P(fgr_packets)), P(vp), vp]),
    "fgr_fggc_plan_overflow": (ctypes.c_int, [vp, P(ctypes.c_int32)]),
    "fgr_fggc_plan_info": (ctypes.c_int, [vp, P(ctypes.c_int64), P(ctypes.c_int32)]),
    "fgr_fggc_plan_destroy": (None, [vp]),
    "fgr_get_info": (ctypes.c_int, [vp, P(fgr_info)]),
    "fgr_autotune": (ctypes.c_int, [vp, P(fgr_packets), vp, ctypes.c_int32, vp]),
    "fgr_get_tuning": (ctypes.c_int, [vp, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]),
    "fgr_set_tuning": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "fgr_set_timing": (ctypes.c_int, [vp, ctypes.c_int32]),
    "fgr_get_stats": (ctypes.c_int, [vp, P(fgr_stats)]),
    "fgr_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int32, P(vp)]),
    "fgr_server_destroy": (None, [vp]),
    "fgr_server_set_max_batch": (ctypes.c_int, [vp, ctypes.c_int32]),
    "fgr_register_packets": (ctypes.c_int, [vp, ctypes.c_int32, P(fgr_packets), P(ctypes.c_uint64)]),
    "fgr_release_packets": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "fgr_submit": (ctypes.c_int, [vp, P(fgr_request), P(ctypes.c_uint64)]),
    "fgr_poll": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_int32, P(fgr_result)]),
    "fgr_cancel": (ctypes.c_int, [vp, ctypes.c_uint64]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libfgr.so (built in-tree by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libfgr.so is missing at %s: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def fgr_last_error() -> str:
    return (load().fgr_last_error() or b"").decode()


def _check(status):
    if status != FGR_OK:
        raise FgrError(status, fgr_last_error())
    return status


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------

def _ptr(x):
    """(address, on_device) of a contiguous numpy array or torch tensor."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):  # torch
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data, 0


def make_packets(q, p, s, a) -> fgr_packets:
    """fgr_packets view of q (d,M), p (d,M), s (M,), a (2,M) float64 arrays/tensors.

    The view holds references to the arrays, so they live as long as it does."""
    pq, dq = _ptr(q)
    pp, dp = _ptr(p)
    ps, ds = _ptr(s)
    pa, da = _ptr(a)
    if len({dq, dp, ds, da}) != 1:
        raise ValueError("packet arrays must all live on the host or all on the device")
    m = int(s.shape[0])
    view = fgr_packets(m, pq, pp, ps, pa, dq, 0)
    view._arrays = (q, p, s, a)
    return view


def make_axes(axes):
    """fgr_axis array from a list of (q, p) pairs of 1-D float64 arrays/tensors,
    one pair per dimension.  The array holds references to them."""
    arr = (fgr_axis * FGR_MAX_DIM)()
    keep = []
    for l, (q, p) in enumerate(axes):
        pq, dq = _ptr(q)
        pp, dp = _ptr(p)
        if dq != dp:
            raise ValueError("an axis's q and p must both live on the host or both on the device")
        arr[l] = fgr_axis(int(q.shape[0]), pq, pp, dq, 0)
        keep.append((q, p))
    arr._arrays = keep
    return arr


def make_grid(grid: dict) -> fgr_grid:
    g = fgr_grid()
    g.d = int(grid["d"])
    for l in range(g.d):
        g.n[l] = int(grid["n"][l])
        g.lo[l] = float(grid["lo"][l])
        g.hi[l] = float(grid["hi"][l])
    return g


def fgr_default_options() -> fgr_options:
    o = fgr_options()
    _check(load().fgr_default_options(ctypes.byref(o)))
    return o


FGR_FLAG_FFT_GRID = 1
FGR_FLAG_SNAP_CP = 2
FGR_FLAG_DIRECT_FMA = 4


def make_options(precision=FGR_FP64, cq=0.5, cp=math.pi / 8, nq=4, np_=2, window_r=0.0,
                 rcond=1e-14, flags=0) -> fgr_options:
    return fgr_options(cq, cp, nq, np_, window_r, rcond, precision, int(flags))


def make_potential(kind="free", c0=0.0, amp=0.0, k=1.0, omega=1.0) -> fgr_potential:
    kinds = {"free": FGR_V_FREE, "cossum": FGR_V_COSSUM, "harmonic": FGR_V_HARMONIC}
    return fgr_potential(kinds[kind] if isinstance(kind, str) else int(kind), 0, c0, amp, k, omega)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---------------------------------------------------------------------------
# the C entry points, one Python function each
# ---------------------------------------------------------------------------

def fgr_create(d: int, grid, eps: float, opt: fgr_options | None = None):
    g = grid if isinstance(grid, fgr_grid) else make_grid(grid)
    out = ctypes.c_void_p()
    _check(load().fgr_create(d, ctypes.byref(g), eps, ctypes.byref(opt) if opt else None,
                             ctypes.byref(out)))
    return out


def fgr_destroy(ctx):
    if ctx:
        load().fgr_destroy(ctx)


def fgr_propagate(ctx, packets: fgr_packets, potential: fgr_potential, t: float, dt: float,
                  stream=None):
    return _check(load().fgr_propagate(ctx, ctypes.byref(packets), ctypes.byref(potential), t, dt,
                                       _stream_handle(stream)))


def fgr_decompose(ctx, u_in, packets: fgr_packets, stream=None):
    """Writes the packets' amplitudes (a) and zero actions (s) from the wave u_in."""
    return _check(load().fgr_decompose(ctx, _ptr(u_in)[0], ctypes.byref(packets), _stream_handle(stream)))


def fgr_decompose_tensor(ctx, axes, u_in, m: int, sel, a_out, stream=None):
    """A(0) of the tensor-product mesh packets sel[j] (or all, in row-major order) into a_out (2, m)."""
    return _check(load().fgr_decompose_tensor(ctx, axes, _ptr(u_in)[0], int(m), _ptr(sel)[0], _ptr(a_out)[0],
                                              _stream_handle(stream)))


def fgr_fggc_multistep_tensor(ctx, axes, sel, flow: fgr_packets, u_in, u_out, steps: int, stream=None):
    """Multi-step FGGC with the mesh given as a tensor product (axes from make_axes)."""
    return _check(load().fgr_fggc_multistep_tensor(ctx, axes, _ptr(sel)[0], ctypes.byref(flow), _ptr(u_in)[0],
                                                   _ptr(u_out)[0], int(steps), _stream_handle(stream)))


def fgr_fggc_multistep(ctx, mesh: fgr_packets, flow: fgr_packets, u_in, u_out, steps: int, stream=None):
    """`steps` multi-step FGGC steps from u_in into u_out (mesh positions, learned flow)."""
    return _check(load().fgr_fggc_multistep(ctx, ctypes.byref(mesh), ctypes.byref(flow), _ptr(u_in)[0],
                                            _ptr(u_out)[0], int(steps), _stream_handle(stream)))


def fgr_reconstruct_direct(ctx, packets: fgr_packets, u_out, stream=None):
    return _check(load().fgr_reconstruct_direct(ctx, ctypes.byref(packets), _ptr(u_out)[0],
                                                _stream_handle(stream)))


def fgr_reconstruct_direct_batch(ctxs, packets, u_outs, stream=None):
    """One persistent direct-sum launch over len(ctxs) requests (<= 64)."""
    n = len(ctxs)
    if not (len(packets) == n == len(u_outs)):
        raise ValueError("ctxs, packets and u_outs must have the same length")
    c_ctx = (vp * n)(*[getattr(c, "handle", c) for c in ctxs])
    c_pk = (P(fgr_packets) * n)(*[ctypes.pointer(p) for p in packets])
    c_u = (vp * n)(*[_ptr(u)[0] for u in u_outs])
    return _check(load().fgr_reconstruct_direct_batch(n, c_ctx, c_pk, c_u, _stream_handle(stream)))


def fgr_fggc_plan_create(ctx, packets: fgr_packets, margin: int = 2, stream=None):
    """Plan handle (free with fgr_fggc_plan_destroy)."""
    out = vp()
    _check(load().fgr_fggc_plan_create(ctx, ctypes.byref(packets), int(margin), ctypes.byref(out),
                                       _stream_handle(stream)))
    return out.value


def fgr_reconstruct_fggc_planned(ctx, plan, packets: fgr_packets, u_out, stream=None):
    return _check(load().fgr_reconstruct_fggc_planned(ctx, plan, ctypes.byref(packets), _ptr(u_out)[0],
                                                      _stream_handle(stream)))


def fgr_reconstruct_fggc_batch(ctxs, plans, packets, u_outs, stream=None):
    """len(ctxs) (<= 64) planned FGGC reconstructions, one launch per stage
    for the requests of each dimension."""
    n = len(ctxs)
    if not (len(plans) == len(packets) == n == len(u_outs)):
        raise ValueError("ctxs, plans, packets and u_outs must have the same length")
    c_ctx = (vp * n)(*[getattr(c, "handle", c) for c in ctxs])
    c_pl = (vp * n)(*plans)
    c_pk = (P(fgr_packets) * n)(*[ctypes.pointer(p) for p in packets])
    c_u = (vp * n)(*[_ptr(u)[0] for u in u_outs])
    return _check(load().fgr_reconstruct_fggc_batch(n, c_ctx, c_pl, c_pk, c_u, _stream_handle(stream)))


def fgr_fggc_plan_overflow(plan) -> bool:
    v = ctypes.c_int32()
    _check(load().fgr_fggc_plan_overflow(plan, ctypes.byref(v)))
    return bool(v.value)


def fgr_fggc_plan_info(plan):
    """(node cells, empty)."""
    n, e = ctypes.c_int64(), ctypes.c_int32()
    _check(load().fgr_fggc_plan_info(plan, ctypes.byref(n), ctypes.byref(e)))
    return n.value, bool(e.value)


def fgr_fggc_plan_destroy(plan):
    if plan:
        load().fgr_fggc_plan_destroy(plan)


def fgr_reconstruct_fggc(ctx, packets: fgr_packets, u_out, stream=None):
    return _check(load().fgr_reconstruct_fggc(ctx, ctypes.byref(packets), _ptr(u_out)[0],
                                              _stream_handle(stream)))


def fgr_reconstruct_fggc_noalloc(ctx, packets: fgr_packets, u_out, stream=None):
    return _check(load().fgr_reconstruct_fggc_noalloc(ctx, ctypes.byref(packets), _ptr(u_out)[0],
                                                      _stream_handle(stream)))


def fgr_autotune(ctx, packets: fgr_packets, u_out, methods: int = 3, stream=None):
    return _check(load().fgr_autotune(ctx, ctypes.byref(packets), _ptr(u_out)[0], int(methods),
                                      _stream_handle(stream)))


def fgr_get_tuning(ctx):
    """(direct CTAs per SM, grid-pass CTAs per SM, grid-pass tile)."""
    a, b, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().fgr_get_tuning(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)))
    return a.value, b.value, t.value


def fgr_set_tuning(ctx, direct_ctas_per_sm: int, pass_ctas_per_sm: int, pass_tile: int = 0):
    return _check(load().fgr_set_tuning(ctx, int(direct_ctas_per_sm), int(pass_ctas_per_sm), int(pass_tile)))


def fgr_get_info(ctx) -> fgr_info:
    i = fgr_info()
    _check(load().fgr_get_info(ctx, ctypes.byref(i)))
    return i


def fgr_set_timing(ctx, enabled):
    """0/False off, 1/True per-stage events, 2 also the grid passes' terms."""
    return _check(load().fgr_set_timing(ctx, int(enabled)))


def fgr_get_stats(ctx) -> fgr_stats:
    s = fgr_stats()
    _check(load().fgr_get_stats(ctx, ctypes.byref(s)))
    return s


def fgr_server_create(hbm_budget_bytes: int, max_inflight: int):
    out = ctypes.c_void_p()
    _check(load().fgr_server_create(int(hbm_budget_bytes), int(max_inflight), ctypes.byref(out)))
    return out


def fgr_server_destroy(srv):
    if srv:
        load().fgr_server_destroy(srv)


def fgr_server_set_max_batch(srv, max_batch: int):
    return _check(load().fgr_server_set_max_batch(srv, int(max_batch)))


def fgr_register_packets(srv, d: int, packets: fgr_packets) -> int:
    sid = ctypes.c_uint64()
    _check(load().fgr_register_packets(srv, d, ctypes.byref(packets), ctypes.byref(sid)))
    return sid.value


def fgr_release_packets(srv, set_id: int):
    return _check(load().fgr_release_packets(srv, ctypes.c_uint64(set_id)))


def make_request(method: int, grid, eps: float, opt: fgr_options, set_id: int, u_out) -> fgr_request:
    g = grid if isinstance(grid, fgr_grid) else make_grid(grid)
    return fgr_request(int(method), g.d, g, float(eps), opt, int(set_id), _ptr(u_out)[0])


def fgr_submit(srv, req: fgr_request) -> int:
    t = ctypes.c_uint64()
    _check(load().fgr_submit(srv, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def fgr_poll(srv, ticket: int, timeout_ms: int = -1):
    """Returns an fgr_result once done, or None while the request still runs."""
    r = fgr_result()
    st = load().fgr_poll(srv, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r))
    if st == FGR_E_NOT_READY:
        return None
    _check(st)
    return r


def fgr_cancel(srv, ticket: int):
    return _check(load().fgr_cancel(srv, ctypes.c_uint64(ticket)))


class Context:
    """Owns one fgr_ctx (convenience around fgr_create / fgr_destroy)."""

    def __init__(self, d, grid, eps, opt: fgr_options | None = None):
        self.d = d
        self.grid = grid
        self.eps = eps
        self.handle = fgr_create(d, grid, eps, opt)

    def close(self):
        if getattr(self, "handle", None):
            fgr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self):
        return fgr_get_info(self.handle)
