"""Oracle for the star-forest operations: a plain single-threaded C reference (sf_oracle.c).

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
import this package.  The CUDA library and its Python binding never import, link or call it.

Functions take a forest object (anything with the attributes of sfgen.Forest) and numpy
arrays, and follow Sec. III.A-B: Bcast, Reduce and FetchAndOp over edges in canonical
order, with the blocked fold D of block K for floating point Reduce SUM (the paper leaves
that order open; the reading is stated in sf_oracle.c).

Parity status: every exported function (Bcast, Reduce, FetchAndOp, Gather, Scatter, the MAX
with location, the SUM reference) is pinned by tests/test_oracle_pins.py against the
worked example of Fig. 2, dense incidence-matrix products, library scatter routines,
closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsf_oracle.so")
_lock = threading.Lock()
_lib = None

DTYPE = {"int32": 0, "int64": 1, "fp32": 2, "fp64": 3, "bf16": 4}
NPTYPE = {"int32": np.int32, "int64": np.int64, "fp32": np.float32, "fp64": np.float64,
          "bf16": np.uint16}
OP = {"REPLACE": 0, "SUM": 1, "MIN": 2, "MAX": 3}

# Block of the deterministic fold D used for floating point Reduce SUM.
FOLD_BLOCK = 64

GCC_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


_PAR_SRC = os.path.join(_HERE, "sf_cpu_parallel.c")
_PAR_LIB = os.path.join(_HERE, "_build", "libsf_cpu_parallel.so")


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *GCC_FLAGS, "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    if src == _SRC:
        build_parallel(force)
    return out


def build_parallel(force: bool = False):
    """The multi-core CPU baseline of the benchmark (sf_cpu_parallel.c, OpenMP).  Returns its
    path, or None when the compiler has no OpenMP (the baseline is then reported missing)."""
    if not force and os.path.exists(_PAR_LIB) and os.path.getmtime(_PAR_LIB) >= os.path.getmtime(_PAR_SRC):
        return _PAR_LIB
    tmp = _PAR_LIB + f".{os.getpid()}.tmp"
    r = subprocess.run(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                        "-fno-fast-math", "-o", tmp, _PAR_SRC], capture_output=True)
    if r.returncode != 0:
        return None
    os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


class CpuParallel:
    """The benchmark step on all host cores (bench.py's multi-core CPU baseline; fp64, bs = 1):
    bcast_replace(root, leaf) and reduce_sum(leaf, root), in place.  Not the oracle."""

    def __init__(self, forest):
        path = build_parallel()
        if path is None:
            raise RuntimeError("no OpenMP compiler for the multi-core CPU baseline")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.cp_plan_create.argtypes = [ctypes.POINTER(_Forest)]
        lib.cp_plan_create.restype = vp
        lib.cp_plan_destroy.argtypes = [vp]
        lib.cp_bcast_replace_f64.argtypes = [vp, vp, vp]
        lib.cp_reduce_sum_f64.argtypes = [vp, vp, vp]
        lib.cp_threads.restype = ctypes.c_int
        self._lib = lib
        m = _Marshalled(forest)
        self._plan = lib.cp_plan_create(m.ref)
        self.threads = int(lib.cp_threads())

    def bcast_replace(self, root, leaf):
        assert root.dtype == np.float64 and leaf.dtype == np.float64 and leaf.flags.c_contiguous
        self._lib.cp_bcast_replace_f64(self._plan, _ptr(np.ascontiguousarray(root)), _ptr(leaf))

    def reduce_sum(self, leaf, root):
        assert root.dtype == np.float64 and leaf.dtype == np.float64 and root.flags.c_contiguous
        self._lib.cp_reduce_sum_f64(self._plan, _ptr(np.ascontiguousarray(leaf)), _ptr(root))

    def __del__(self):
        try:
            self._lib.cp_plan_destroy(self._plan)
        except Exception:
            pass


class _Forest(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32),
                ("nroots", ctypes.c_void_p), ("nleaves", ctypes.c_void_p),
                ("has_ilocal", ctypes.c_void_p), ("ilocal", ctypes.c_void_p),
                ("rrank", ctypes.c_void_p), ("rindex", ctypes.c_void_p)]


def _bind(lib):
    F = ctypes.POINTER(_Forest)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.oracle_layout.argtypes = [F, vp, vp]
    lib.oracle_layout.restype = i64
    lib.oracle_bcast.argtypes = [F, i32, i32, vp, vp, i32]
    lib.oracle_reduce.argtypes = [F, i32, i32, vp, vp, i32, i64]
    lib.oracle_fetch_and_op.argtypes = [F, i32, i32, vp, vp, vp, i32]
    lib.oracle_sum_reference.argtypes = [F, i32, i32, vp, vp, vp, vp]
    lib.oracle_reduce_maxloc.argtypes = [F, i32, i32, vp, vp, vp]
    lib.oracle_in_degree.argtypes = [F, vp]
    lib.oracle_gather.argtypes = [F, i32, i32, vp, vp, vp]
    lib.oracle_scatter.argtypes = [F, i32, i32, vp, vp]
    lib.oracle_f32_to_bf16.argtypes = [vp, vp, i64]
    lib.oracle_f32_to_bf16.restype = None
    return lib


def load(path: str | None = None):
    """The oracle library (built on first use).  A different `path` loads another build
    of the same source (used by the planted-mistake tests)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class _Marshalled:
    """Keeps the flattened forest arrays alive while C reads them."""

    def __init__(self, forest):
        self.has, self.il, self.rr, self.ri = forest.flat()
        self.nroots = np.ascontiguousarray(forest.nroots, np.int64)
        self.nleaves = np.ascontiguousarray(forest.nleaves, np.int64)
        self.s = _Forest(int(forest.nranks), self.nroots.ctypes.data, self.nleaves.ctypes.data,
                         self.has.ctypes.data, self.il.ctypes.data, self.rr.ctypes.data,
                         self.ri.ctypes.data)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data


def layout(forest, lib=None):
    """(rootoff[P+1], leafoff[P+1]) of the concatenated rank-major buffers."""
    lib = lib or load()
    m = _Marshalled(forest)
    ro = np.zeros(forest.nranks + 1, np.int64)
    lo = np.zeros(forest.nranks + 1, np.int64)
    lib.oracle_layout(m.ref, _ptr(ro), _ptr(lo))
    return ro, lo


def _check(dtype, bs, arr, units, name):
    if arr.dtype != NPTYPE[dtype] or arr.size != units * bs:
        raise ValueError(f"{name}: expected {units}x{bs} {dtype}, got {arr.dtype} size {arr.size}")


def bcast(forest, dtype: str, bs: int, rootdata, leafdata, op: str, lib=None):
    """Returns a new leaf array: leafdata after Bcast(op)."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    root = np.ascontiguousarray(rootdata)
    leaf = np.array(leafdata, copy=True, order="C")
    _check(dtype, bs, root, ro[-1], "rootdata")
    _check(dtype, bs, leaf, lo[-1], "leafdata")
    m = _Marshalled(forest)
    rc = lib.oracle_bcast(m.ref, DTYPE[dtype], bs, _ptr(root), _ptr(leaf), OP[op])
    assert rc == 0
    return leaf


def reduce(forest, dtype: str, bs: int, leafdata, rootdata, op: str, K: int = FOLD_BLOCK, lib=None):
    """Returns a new root array: rootdata after Reduce(op)."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    leaf = np.ascontiguousarray(leafdata)
    root = np.array(rootdata, copy=True, order="C")
    _check(dtype, bs, root, ro[-1], "rootdata")
    _check(dtype, bs, leaf, lo[-1], "leafdata")
    m = _Marshalled(forest)
    rc = lib.oracle_reduce(m.ref, DTYPE[dtype], bs, _ptr(leaf), _ptr(root), OP[op], K)
    assert rc == 0
    return root


def fetch_and_op(forest, dtype: str, bs: int, rootdata, leafdata, leafupdate, op: str, lib=None):
    """Returns (root after, leafupdate after) of FetchAndOp(op)."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    root = np.array(rootdata, copy=True, order="C")
    leaf = np.ascontiguousarray(leafdata)
    upd = np.array(leafupdate, copy=True, order="C")
    for a, n, nm in ((root, ro[-1], "rootdata"), (leaf, lo[-1], "leafdata"), (upd, lo[-1], "leafupdate")):
        _check(dtype, bs, a, n, nm)
    m = _Marshalled(forest)
    rc = lib.oracle_fetch_and_op(m.ref, DTYPE[dtype], bs, _ptr(root), _ptr(leaf), _ptr(upd), OP[op])
    assert rc == 0
    return root, upd


def sum_reference(forest, dtype: str, bs: int, leafdata, rootdata, lib=None):
    """(accurate r0 + sum, |r0| + sum|y|) per root element, in float64."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    leaf = np.ascontiguousarray(leafdata)
    root = np.ascontiguousarray(rootdata)
    _check(dtype, bs, root, ro[-1], "rootdata")
    _check(dtype, bs, leaf, lo[-1], "leafdata")
    s = np.zeros(ro[-1] * bs, np.float64)
    a = np.zeros(ro[-1] * bs, np.float64)
    m = _Marshalled(forest)
    rc = lib.oracle_sum_reference(m.ref, DTYPE[dtype], bs, _ptr(leaf), _ptr(root), _ptr(s), _ptr(a))
    assert rc == 0
    return s, a


def reduce_maxloc(forest, dtype: str, bs: int, leafdata, lib=None):
    """(max per root element or 0 if no leaves, first canonical edge reaching it or -1)."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    leaf = np.ascontiguousarray(leafdata)
    _check(dtype, bs, leaf, lo[-1], "leafdata")
    out = np.zeros(ro[-1] * bs, NPTYPE[dtype])
    arg = np.zeros(ro[-1] * bs, np.int64)
    m = _Marshalled(forest)
    rc = lib.oracle_reduce_maxloc(m.ref, DTYPE[dtype], bs, _ptr(leaf), _ptr(out), _ptr(arg))
    assert rc == 0
    return out, arg


def in_degree(forest, lib=None):
    lib = lib or load()
    ro, _ = layout(forest, lib)
    deg = np.zeros(ro[-1], np.int64)
    m = _Marshalled(forest)
    lib.oracle_in_degree(m.ref, _ptr(deg))
    return deg


def f32_to_bf16(x, lib=None):
    lib = lib or load()
    x = np.ascontiguousarray(x, np.float32)
    y = np.zeros(x.size, np.uint16)
    lib.oracle_f32_to_bf16(_ptr(x), _ptr(y), x.size)
    return y


def gather(forest, dtype: str, bs: int, leafdata, multirootdata, lib=None):
    """Returns a new multi-root array: multirootdata after Gather (one multi-root per edge;
    root u's k-th leaf in canonical order lands at (edges into roots below u) + k)."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    leaf = np.ascontiguousarray(leafdata)
    multi = np.array(multirootdata, copy=True, order="C")
    _check(dtype, bs, leaf, lo[-1], "leafdata")
    _check(dtype, bs, multi, forest.nedges, "multirootdata")
    m = _Marshalled(forest)
    n = ctypes.c_int64(-1)
    rc = lib.oracle_gather(m.ref, DTYPE[dtype], bs, _ptr(leaf), _ptr(multi), ctypes.addressof(n))
    assert rc == 0 and n.value == forest.nedges
    return multi


def scatter(forest, dtype: str, bs: int, multirootdata, leafdata, lib=None):
    """Returns a new leaf array: leafdata after Scatter (the reverse of gather; isolated
    leaves keep their values)."""
    lib = lib or load()
    ro, lo = layout(forest, lib)
    multi = np.ascontiguousarray(multirootdata)
    leaf = np.array(leafdata, copy=True, order="C")
    _check(dtype, bs, leaf, lo[-1], "leafdata")
    _check(dtype, bs, multi, forest.nedges, "multirootdata")
    m = _Marshalled(forest)
    rc = lib.oracle_scatter(m.ref, DTYPE[dtype], bs, _ptr(multi), _ptr(leaf))
    assert rc == 0
    return leaf
