"""ctypes front end of rgg.c (unstructured SpMV-style scatter forest)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import rng
from .forests import Forest

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgg.c")
_LIB = os.path.join(_HERE, "_build", "librgg.so")
_lock = threading.Lock()
_lib = None


class _Res(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int64), ("N", ctypes.c_int64), ("E", ctypes.c_int64),
                ("G", ctypes.c_int64), ("nleaves", ctypes.POINTER(ctypes.c_int64)),
                ("rrank", ctypes.POINTER(ctypes.c_int32)), ("rindex", ctypes.POINTER(ctypes.c_int64)),
                ("r", ctypes.c_double), ("ncell", ctypes.c_int64), ("deg_sample", ctypes.c_double)]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.rgg_generate.restype = ctypes.POINTER(_Res)
            lib.rgg_generate.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64]
            lib.rgg_free.argtypes = [ctypes.POINTER(_Res)]
            lib.rgg_free.restype = None
            _lib = lib
    return _lib


def cfg3_spmv(npoints: int = 1 << 24, levels: int = 8, degree: float = 14.0) -> Forest:
    """Random geometric graph of `npoints` points (expected degree `degree`) split into
    2^levels ranks by coordinate bisection; leaves = owned entries then ghost columns."""
    lib = _load()
    seed = rng.BASE_SEED + 3
    res = lib.rgg_generate(npoints, levels, degree, seed)
    if not res:
        raise ValueError("rgg_generate failed (npoints must be a multiple of 2^levels)")
    try:
        R = res.contents
        P, E = int(R.P), int(R.E)
        nleaves = np.ctypeslib.as_array(R.nleaves, shape=(P,)).copy()
        rr = np.ctypeslib.as_array(R.rrank, shape=(E,)).copy() if E else np.zeros(0, np.int32)
        ri = np.ctypeslib.as_array(R.rindex, shape=(E,)).copy() if E else np.zeros(0, np.int64)
        meta = {"npoints": npoints, "ranks": P, "ghosts": int(R.G), "radius": float(R.r),
                "ncell": int(R.ncell), "degree_sample": float(R.deg_sample)}
    finally:
        lib.rgg_free(res)
    off = np.concatenate([[0], np.cumsum(nleaves)])
    per = npoints // P
    return Forest(P, np.full(P, per), nleaves, [None] * P,
                  [rr[off[q]:off[q + 1]] for q in range(P)],
                  [ri[off[q]:off[q + 1]] for q in range(P)],
                  name=f"spmv{npoints}_{P}", meta=meta)
