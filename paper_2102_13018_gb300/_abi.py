"""ctypes declarations of the C ABI in include/sf.h (libsfgb.so, built in-tree)."""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsfgb.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "sf.h")

SF_INT32, SF_INT64, SF_FP32, SF_FP64, SF_BF16 = range(5)
SF_REPLACE, SF_SUM, SF_MIN, SF_MAX = range(4)
SF_MODE_AUTO, SF_MODE_ATOMIC, SF_MODE_DETERMINISTIC = range(3)
SF_PATH_AUTO, SF_PATH_FUSED, SF_PATH_THREE_PHASE, SF_PATH_ROOT_MAJOR = range(4)
SF_PLAN_AUTO, SF_PLAN_ROOT_MAJOR, SF_PLAN_DIAGONAL, SF_PLAN_DIAGONAL_STAGED = range(4)
SF_MEM_HOST, SF_MEM_DEVICE = 0, 1
SF_OP_BCAST, SF_OP_REDUCE, SF_OP_BARRIER = 0, 1, 2
SF_FOLD_BLOCK = 64
SF_NOALLOC_SCRATCH_BYTES = 16 << 20
SF_DEVSTAT_STAGE_TIMEOUT = 1
SF_DEVSTAT_TILE_REFUSED = 2
SF_MAX_UNIT_BYTES = 1 << 19

ERRORS = {0: "SF_SUCCESS", 1: "SF_ERR_ARG", 2: "SF_ERR_NULL", 3: "SF_ERR_RANGE", 4: "SF_ERR_DUP_LEAF",
          5: "SF_ERR_STATE", 6: "SF_ERR_NO_PENDING", 7: "SF_ERR_PENDING", 8: "SF_ERR_UNSUPPORTED",
          9: "SF_ERR_ALLOC", 10: "SF_ERR_CUDA", 11: "SF_ERR_ALIGN", 12: "SF_ERR_TOO_LARGE"}
CODES = {v: k for k, v in ERRORS.items()}


class SFError(RuntimeError):
    def __init__(self, code: int, where: str, lib=None):
        self.code = code
        self.name = ERRORS.get(code, str(code))
        msg = lib.sf_error_string(code).decode() if lib is not None else self.name
        super().__init__(f"{where}: {self.name} ({msg})")


class sf_node(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("index", ctypes.c_int64)]


class sf_unit(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("bs", ctypes.c_int32)]


class sf_batch_op(ctypes.Structure):
    _fields_ = [("sf", ctypes.c_void_p), ("kind", ctypes.c_int32), ("unit", sf_unit), ("op", ctypes.c_int32),
                ("src", ctypes.c_void_p), ("dst", ctypes.c_void_p)]


class sf_tuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("mode", ctypes.c_int32), ("vector_bytes", ctypes.c_int32),
                ("tile_edges", ctypes.c_int32), ("reduce_plan", ctypes.c_int32)]


class sf_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("nranks", "analyzed", "setup_done", "has_dup_roots")] + \
               [(n, ctypes.c_int64) for n in (
                   "nroots_total", "leaf_extent_total", "nedges", "max_in_degree", "connected_roots",
                   "multi_roots", "multi_edges", "segments", "self_edges", "runs", "runs_pattern", "runs_3d",
                   "edges_both_pattern", "edges_one_indexed", "edges_two_indexed", "rm_masked_runs",
                   "rm_masked_edges", "rm_pairs", "rm_chunks", "device_plan_bytes", "ts_tile_edges",
                   "rm_tile_edges", "rm_tile_blocks", "dg_chunks", "dg_roots", "dg_extra_leaves", "dg_list_roots",
                   "dg_rest_roots")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


def declared_functions(header: str = HEADER):
    """Names of the functions include/sf.h declares (for the export check)."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sf_[a-z0-9_]+)\s*\(", text)))


_lib = None


def load():
    """The library, loaded once.  Raises ImportError when it has not been built: the
    package has no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "python -c 'import __graft_entry__ as g; g.build()'")
    lib = ctypes.CDLL(LIB_PATH)
    P, vp, i32, i64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    H = P(vp)   # sf_t* / sf_t**
    lib.sf_create.argtypes = [i32, P(i64), P(i64), P(P(i64)), P(P(sf_node)), P(vp)]
    lib.sf_analyze.argtypes = [vp]
    lib.sf_setup.argtypes = [vp, vp]
    lib.sf_get_layout.argtypes = [vp, P(i64), P(i64)]
    lib.sf_get_info.argtypes = [vp, P(sf_info)]
    lib.sf_set_mode.argtypes = [vp, i32]
    lib.sf_set_path.argtypes = [vp, i32]
    lib.sf_set_reduce_plan.argtypes = [vp, i32]
    lib.sf_set_vector_bytes.argtypes = [vp, i32]
    lib.sf_set_tile_edges.argtypes = [vp, i32]
    lib.sf_get_tuning.argtypes = [vp, P(sf_tuning)]
    lib.sf_zero_leafless_roots.argtypes = [vp, sf_unit, vp, vp, vp]
    for name in ("sf_bcast_begin", "sf_bcast_end", "sf_reduce_begin", "sf_reduce_end", "sf_reduce_from_zero_begin",
                 "sf_reduce_from_zero_end"):
        getattr(lib, name).argtypes = [vp, sf_unit, vp, vp, i32, vp]
    for name in ("sf_fetch_and_op_begin", "sf_fetch_and_op_end"):
        getattr(lib, name).argtypes = [vp, sf_unit, vp, vp, vp, i32, vp]
    for name in ("sf_bcast_with_memtype_begin", "sf_bcast_with_memtype_end",
                 "sf_reduce_with_memtype_begin", "sf_reduce_with_memtype_end"):
        getattr(lib, name).argtypes = [vp, sf_unit, i32, vp, i32, vp, i32, vp]
    lib.sf_reduce_noalloc.argtypes = [vp, sf_unit, vp, vp, i32, vp]
    lib.sf_reduce_maxloc.argtypes = [vp, sf_unit, vp, vp, vp, vp]
    lib.sf_get_device_status.argtypes = [vp, vp, P(i32)]
    lib.sf_create_embedded_root_sf.argtypes = [vp, i64, P(i64), P(vp)]
    lib.sf_create_embedded_leaf_sf.argtypes = [vp, i64, P(i64), P(vp)]
    lib.sf_get_multi_sf.argtypes = [vp, vp, P(vp)]
    lib.sf_compose.argtypes = [vp, vp, P(vp)]
    lib.sf_compose_inverse.argtypes = [vp, vp, P(vp)]
    for name in ("sf_gather_begin", "sf_gather_end", "sf_scatter_begin", "sf_scatter_end"):
        getattr(lib, name).argtypes = [vp, sf_unit, vp, vp, vp]
    lib.sf_maxloc_scatter.argtypes = [vp, sf_unit, vp, vp, vp, vp]
    lib.sf_maxloc_grad.argtypes = [vp, sf_unit, vp, vp, vp, vp]
    lib.sf_batch_create.argtypes = [P(vp)]
    lib.sf_batch_run.argtypes = [vp, P(sf_batch_op), i32, i32, vp]
    lib.sf_batch_launches.argtypes = [vp, P(i32)]
    lib.sf_batch_destroy.argtypes = [vp]
    lib.sf_autotune.argtypes = [vp, sf_unit, i32, vp, vp, i32, i32, vp, P(i32)]
    lib.sf_destroy.argtypes = [vp]
    lib.sf_error_string.argtypes = [ctypes.c_int]
    lib.sf_error_string.restype = ctypes.c_char_p
    lib.sf_launch_count.argtypes = []
    lib.sf_launch_count.restype = i64
    for name in declared_functions():
        f = getattr(lib, name)
        if f.restype is ctypes.c_int and name not in ("sf_error_string",):
            f.restype = ctypes.c_int
    _lib = lib
    return lib


def check(rc: int, where: str):
    if rc != 0:
        raise SFError(rc, where, _lib)
