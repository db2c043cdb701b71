"""Build and load ``oracle/hier.c`` (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hier.c")
_LIB = os.path.join(_HERE, "_hier.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile hier.c with gcc (-ffp-contract=off keeps every sum unfused)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        I = ctypes.c_int
        L = ctypes.c_long
        D = ctypes.c_double
        P = ctypes.c_void_p
        _lib.oracle_fps.argtypes = [I, P, P, P, I, I, P, P]
        _lib.oracle_fps.restype = I
        _lib.oracle_fps_among.argtypes = [I, P, P, P, I, I, P, P, P]
        _lib.oracle_fps_among.restype = I
        _lib.oracle_balls.argtypes = [I, P, P, P, I, P, D, L, P, P, P]
        _lib.oracle_balls.restype = L
        _lib.oracle_nearest.argtypes = [I, P, P, P, I, P, P, P]
        _lib.oracle_nearest.restype = I
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fps(ptr, idx, w, start: int, count: int, candidates=None):
    """Farthest-point order of `count` vertices from `start`; with a boolean
    `candidates` mask only those vertices are chosen (distances still run over
    the whole graph)."""
    n = len(ptr) - 1
    order = np.empty(count, dtype=np.int32)
    field = np.empty(n, dtype=np.float64)
    if candidates is None:
        rc = lib().oracle_fps(n, _p(ptr), _p(idx), _p(w), int(start), int(count), _p(order), _p(field))
    else:
        cand = np.ascontiguousarray(candidates, dtype=np.uint8)
        if not cand[start] or count > int(cand.sum()):
            raise ValueError("start must be a candidate and count at most the number of candidates")
        rc = lib().oracle_fps_among(n, _p(ptr), _p(idx), _p(w), int(start), int(count), _p(cand),
                                    _p(order), _p(field))
    if rc != 0:
        raise MemoryError("oracle_fps failed")
    return order, field


def balls(ptr, idx, w, centres: np.ndarray, rho: float):
    n = len(ptr) - 1
    centres = np.ascontiguousarray(centres, dtype=np.int32)
    cap = max(1024, 16 * len(centres))
    while True:
        c = np.empty(cap, dtype=np.int32)
        v = np.empty(cap, dtype=np.int32)
        d = np.empty(cap, dtype=np.float64)
        cnt = lib().oracle_balls(n, _p(ptr), _p(idx), _p(w), len(centres), _p(centres),
                                 float(rho), cap, _p(c), _p(v), _p(d))
        if cnt >= 0:
            return c[:cnt], v[:cnt], d[:cnt]
        if cnt < -(1 << 61):
            raise MemoryError("oracle_balls failed")
        cap = -cnt


def nearest(ptr, idx, w, centres: np.ndarray):
    n = len(ptr) - 1
    centres = np.ascontiguousarray(centres, dtype=np.int32)
    label = np.empty(n, dtype=np.int32)
    dist = np.empty(n, dtype=np.float64)
    rc = lib().oracle_nearest(n, _p(ptr), _p(idx), _p(w), len(centres), _p(centres),
                              _p(label), _p(dist))
    if rc != 0:
        raise MemoryError("oracle_nearest failed")
    return label, dist
