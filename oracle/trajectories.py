"""Frozen Gaussian trajectories, eq. 2.3-2.7, by classical RK4 in FP64.

Test infrastructure only (see the package docstring).  The integrator itself is
plain C (c/rk4.c, OpenMP over packets), compiled on first use with gcc; this
module only marshals arrays.  ``build()`` compiles it ahead of time.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "rk4.c")
_LIB = os.path.join(_HERE, "c", "liboracle_rk4.so")
_lock = threading.Lock()
_lib = None

KINDS = {"free": 0, "cossum": 1, "harmonic": 2}


def build(force: bool = False) -> str:
    """Compile c/rk4.c into c/liboracle_rk4.so (gcc, -fopenmp, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_rk4.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_rk4.restype = ctypes.c_int
            lib.oracle_rk4_nsteps.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_rk4_nsteps.restype = ctypes.c_int64
            _lib = lib
    return _lib


def nsteps(t: float, dt: float) -> int:
    return int(_load().oracle_rk4_nsteps(t, dt))


def _ptr(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def propagate(packets: dict, potential: dict, t: float, dt: float = 1e-4,
              with_jacobian: bool = False):
    """Returns a new packet dict at time t (and the final Jacobians if asked).

    potential: {"kind": "free"|"cossum"|"harmonic", "c0", "amp", "k", "omega"}.
    Jacobians come back as an array (M, 4, d, d) holding F, G, H, K.
    """
    lib = _load()
    q = np.array(packets["q"], dtype=np.float64, order="C", copy=True)
    p = np.array(packets["p"], dtype=np.float64, order="C", copy=True)
    s = np.array(packets["s"], dtype=np.float64, order="C", copy=True)
    a = np.array(packets["a"], dtype=np.float64, order="C", copy=True)
    d, m = q.shape
    jac = np.zeros((m, 4, d, d)) if with_jacobian else None
    rc = lib.oracle_rk4(d, m, _ptr(q), _ptr(p), _ptr(s), _ptr(a),
                        KINDS[potential.get("kind", "free")], float(potential.get("c0", 0.0)),
                        float(potential.get("amp", 0.0)), float(potential.get("k", 1.0)),
                        float(potential.get("omega", 1.0)), float(t), float(dt),
                        _ptr(jac) if jac is not None else None)
    if rc != 0:
        raise ValueError("oracle_rk4 rejected its arguments")
    out = {"q": q, "p": p, "s": s, "a": a}
    if with_jacobian:
        return out, jac
    return out
