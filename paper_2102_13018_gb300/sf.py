"""StarForest: Python handle over the C ABI (argument marshalling only).

Every step of Bcast / Reduce / FetchAndOp runs in libsfgb's kernels; this module converts
arrays to pointers, infers the unit from a tensor's dtype and shape, and passes the current
torch CUDA stream.  PyTorch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import _abi
from ._abi import check, sf_info, sf_node, sf_tuning, sf_unit

OPS = {"REPLACE": _abi.SF_REPLACE, "SUM": _abi.SF_SUM, "MIN": _abi.SF_MIN, "MAX": _abi.SF_MAX}
MODES = {"auto": _abi.SF_MODE_AUTO, "atomic": _abi.SF_MODE_ATOMIC, "deterministic": _abi.SF_MODE_DETERMINISTIC}
PATHS = {"auto": _abi.SF_PATH_AUTO, "fused": _abi.SF_PATH_FUSED, "three_phase": _abi.SF_PATH_THREE_PHASE,
         "root_major": _abi.SF_PATH_ROOT_MAJOR}
PLANS = {"auto": _abi.SF_PLAN_AUTO, "root_major": _abi.SF_PLAN_ROOT_MAJOR, "diagonal": _abi.SF_PLAN_DIAGONAL,
         "diagonal_staged": _abi.SF_PLAN_DIAGONAL_STAGED}
DTYPE_NAMES = {"int32": _abi.SF_INT32, "int64": _abi.SF_INT64, "fp32": _abi.SF_FP32, "fp64": _abi.SF_FP64,
               "bf16": _abi.SF_BF16}


_TORCH_CODES = None
_CURRENT_STREAM = None


def _torch_dtype_code(t) -> int:
    global _TORCH_CODES
    if _TORCH_CODES is None:
        import torch
        _TORCH_CODES = {torch.int32: _abi.SF_INT32, torch.int64: _abi.SF_INT64, torch.float32: _abi.SF_FP32,
                        torch.float64: _abi.SF_FP64, torch.bfloat16: _abi.SF_BF16}
    code = _TORCH_CODES.get(t.dtype)
    if code is None:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return code


def _current_stream_handle() -> int:
    """The current torch CUDA stream's handle, or 0 (legacy default stream) without CUDA."""
    global _CURRENT_STREAM
    if _CURRENT_STREAM is None:
        try:
            import torch
            if torch.cuda.is_available():
                _CURRENT_STREAM = lambda: torch.cuda.current_stream().cuda_stream  # noqa: E731
            else:
                return 0
        except Exception:
            return 0
    return _CURRENT_STREAM()


def _numpy_dtype_code(a: np.ndarray, bf16: bool = False) -> int:
    if bf16:
        assert a.dtype == np.uint16
        return _abi.SF_BF16
    m = {np.dtype(np.int32): _abi.SF_INT32, np.dtype(np.int64): _abi.SF_INT64,
         np.dtype(np.float32): _abi.SF_FP32, np.dtype(np.float64): _abi.SF_FP64}
    return m[a.dtype]


class StarForest:
    """A star forest over `nranks` simulated ranks (Sec. III.A).

    nroots[p], nleaves[p]: sizes per rank; ilocal[p]: int array or None (contiguous leaves);
    iremote_rank[p], iremote_index[p]: root address of each leaf.
    """

    def __init__(self, nroots: Sequence[int], nleaves: Sequence[int], ilocal, iremote_rank, iremote_index):
        self._lib = _abi.load()
        P = len(nroots)
        self.nranks = P
        self._nroots = np.ascontiguousarray(nroots, dtype=np.int64)
        self._nleaves = np.ascontiguousarray(nleaves, dtype=np.int64)
        if len(self._nleaves) != P:
            raise ValueError("nroots and nleaves differ in length")
        i64p = ctypes.POINTER(ctypes.c_int64)
        nodep = ctypes.POINTER(sf_node)
        self._keep = []
        il_arr = (i64p * P)()
        ir_arr = (nodep * P)()
        node_dt = np.dtype([("rank", "<i4"), ("index", "<i8")], align=True)
        assert node_dt.itemsize == ctypes.sizeof(sf_node)
        for p in range(P):
            if ilocal is not None and ilocal[p] is not None:
                a = np.ascontiguousarray(ilocal[p], dtype=np.int64)
                self._keep.append(a)
                il_arr[p] = a.ctypes.data_as(i64p)
            n = int(self._nleaves[p])
            nodes = np.zeros(max(n, 1), dtype=node_dt)
            if n:
                nodes["rank"][:n] = np.asarray(iremote_rank[p], dtype=np.int32)[:n]
                nodes["index"][:n] = np.asarray(iremote_index[p], dtype=np.int64)[:n]
            self._keep.append(nodes)
            ir_arr[p] = ctypes.cast(nodes.ctypes.data, nodep)
        h = ctypes.c_void_p()
        check(self._lib.sf_create(P, self._nroots.ctypes.data_as(i64p), self._nleaves.ctypes.data_as(i64p),
                                  il_arr, ir_arr, ctypes.byref(h)), "sf_create")
        self._h = h
        self._keep = None   # sf_create copied everything
        ro = np.zeros(P + 1, np.int64)
        lo = np.zeros(P + 1, np.int64)
        check(self._lib.sf_get_layout(self._h, ro.ctypes.data_as(i64p), lo.ctypes.data_as(i64p)), "sf_get_layout")
        self.rootoff, self.leafoff = ro, lo
        self.nroots_total = int(ro[-1])
        self.leaf_extent = int(lo[-1])

    @classmethod
    def _wrap(cls, handle, owned: bool = True) -> "StarForest":
        """A StarForest around an existing handle (derived forests)."""
        self = cls.__new__(cls)
        self._lib = _abi.load()
        self._h = handle
        self._owned = owned
        inf = sf_info()
        check(self._lib.sf_get_info(self._h, ctypes.byref(inf)), "sf_get_info")
        P = inf.nranks
        self.nranks = P
        i64p = ctypes.POINTER(ctypes.c_int64)
        ro = np.zeros(P + 1, np.int64)
        lo = np.zeros(P + 1, np.int64)
        check(self._lib.sf_get_layout(self._h, ro.ctypes.data_as(i64p), lo.ctypes.data_as(i64p)), "sf_get_layout")
        self.rootoff, self.leafoff = ro, lo
        self.nroots_total = int(ro[-1])
        self.leaf_extent = int(lo[-1])
        return self

    @classmethod
    def from_forest(cls, f) -> "StarForest":
        """From any object with nroots, nleaves, ilocal, iremote_rank, iremote_index."""
        return cls(f.nroots, f.nleaves, f.ilocal, f.iremote_rank, f.iremote_index)

    # ---------------------------------------------------------------- lifecycle
    def analyze(self) -> "StarForest":
        check(self._lib.sf_analyze(self._h), "sf_analyze")
        return self

    def setup(self, stream=None) -> "StarForest":
        check(self._lib.sf_setup(self._h, self._stream(stream)), "sf_setup")
        return self

    def info(self) -> dict:
        inf = sf_info()
        check(self._lib.sf_get_info(self._h, ctypes.byref(inf)), "sf_get_info")
        return inf.as_dict()

    def set_mode(self, mode: str) -> "StarForest":
        check(self._lib.sf_set_mode(self._h, MODES[mode]), "sf_set_mode")
        return self

    def set_path(self, path: str) -> "StarForest":
        check(self._lib.sf_set_path(self._h, PATHS[path]), "sf_set_path")
        return self

    def set_reduce_plan(self, plan: str) -> "StarForest":
        """Plan of the deterministic Reduce: "auto", "root_major", "diagonal", "diagonal_staged"."""
        check(self._lib.sf_set_reduce_plan(self._h, PLANS[plan]), "sf_set_reduce_plan")
        return self

    def set_vector_bytes(self, nbytes: int) -> "StarForest":
        """Widest vector the kernels move per access (2, 4, 8, 16; 0 = 16)."""
        check(self._lib.sf_set_vector_bytes(self._h, int(nbytes)), "sf_set_vector_bytes")
        return self

    def set_tile_edges(self, edges: int) -> "StarForest":
        """Edges per CTA tile of the two-sided kernels (a power of two; 0 = the setup's)."""
        check(self._lib.sf_set_tile_edges(self._h, int(edges)), "sf_set_tile_edges")
        return self

    def tuning(self) -> dict:
        """The forest's current choices: Bcast path, Reduce mode and plan, vector bytes, tile edges."""
        t = sf_tuning()
        check(self._lib.sf_get_tuning(self._h, ctypes.byref(t)), "sf_get_tuning")
        paths = {v: n for n, v in PATHS.items()}
        modes = {v: n for n, v in MODES.items()}
        plans = {v: n for n, v in PLANS.items()}
        return {"path": paths[t.path], "mode": modes[t.mode], "vector_bytes": t.vector_bytes,
                "tile_edges": t.tile_edges, "reduce_plan": plans[t.reduce_plan]}

    def destroy(self):
        if getattr(self, "_h", None) and getattr(self, "_owned", True):
            check(self._lib.sf_destroy(self._h), "sf_destroy")
        self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) and getattr(self, "_owned", True):
                self._lib.sf_destroy(self._h)
        except Exception:
            pass

    # ---------------------------------------------------------------- derived forests
    def embedded_roots(self, selected) -> "StarForest":
        """Forest of the edges of the selected roots (global root units), same layout."""
        sel = np.ascontiguousarray(selected, dtype=np.int64)
        h = ctypes.c_void_p()
        check(self._lib.sf_create_embedded_root_sf(self._h, sel.size, sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                   ctypes.byref(h)), "sf_create_embedded_root_sf")
        return StarForest._wrap(h)

    def embedded_leaves(self, selected) -> "StarForest":
        """Forest of the edges of the selected leaves (global leaf units), same layout."""
        sel = np.ascontiguousarray(selected, dtype=np.int64)
        h = ctypes.c_void_p()
        check(self._lib.sf_create_embedded_leaf_sf(self._h, sel.size, sel.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                                   ctypes.byref(h)), "sf_create_embedded_leaf_sf")
        return StarForest._wrap(h)

    def compose(self, other: "StarForest") -> "StarForest":
        """AB: this forest's roots to other's leaves (this forest's leaves = other's roots)."""
        h = ctypes.c_void_p()
        check(self._lib.sf_compose(self._h, other._h, ctypes.byref(h)), "sf_compose")
        return StarForest._wrap(h)

    def compose_inverse(self, other: "StarForest") -> "StarForest":
        """AB: this forest's roots to other's roots through the shared leaves."""
        h = ctypes.c_void_p()
        check(self._lib.sf_compose_inverse(self._h, other._h, ctypes.byref(h)), "sf_compose_inverse")
        return StarForest._wrap(h)

    def multi_sf(self, stream=None) -> "StarForest":
        """The multi-forest (owned by this forest)."""
        h = ctypes.c_void_p()
        check(self._lib.sf_get_multi_sf(self._h, self._stream(stream), ctypes.byref(h)), "sf_get_multi_sf")
        return StarForest._wrap(h, owned=False)

    def gather(self, leafdata, multirootdata, bs=None, stream=None):
        m = self.multi_sf(stream)
        u = self._unit(multirootdata, m.nroots_total, bs)
        args = (self._h, u, self._ptr(leafdata), self._ptr(multirootdata), self._stream(stream))
        check(self._lib.sf_gather_begin(*args), "sf_gather_begin")
        check(self._lib.sf_gather_end(*args), "sf_gather_end")
        return multirootdata

    def scatter(self, multirootdata, leafdata, bs=None, stream=None):
        m = self.multi_sf(stream)
        u = self._unit(multirootdata, m.nroots_total, bs)
        args = (self._h, u, self._ptr(multirootdata), self._ptr(leafdata), self._stream(stream))
        check(self._lib.sf_scatter_begin(*args), "sf_scatter_begin")
        check(self._lib.sf_scatter_end(*args), "sf_scatter_end")
        return leafdata

    # ---------------------------------------------------------------- helpers
    @staticmethod
    def _stream(stream):
        if stream is None:
            return ctypes.c_void_p(_current_stream_handle())
        if isinstance(stream, int):
            return ctypes.c_void_p(stream)
        return ctypes.c_void_p(stream.cuda_stream)

    def _unit(self, t, units: int, bs: Optional[int]) -> sf_unit:
        code = _torch_dtype_code(t)
        if bs is None:
            if units == 0:
                bs = t.shape[-1] if t.dim() > 1 else 1
            else:
                if t.numel() % units:
                    raise ValueError(f"tensor of {t.numel()} elements is not {units} units")
                bs = t.numel() // units
        return sf_unit(code, int(bs))

    @staticmethod
    def _ptr(t):
        if t is None:
            return None
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(t.data_ptr())

    # ---------------------------------------------------------------- operations (device tensors)
    def bcast_begin(self, rootdata, leafdata, op: str = "REPLACE", bs: Optional[int] = None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_bcast_begin(self._h, u, self._ptr(rootdata), self._ptr(leafdata), OPS[op],
                                       self._stream(stream)), "sf_bcast_begin")

    def bcast_end(self, rootdata, leafdata, op: str = "REPLACE", bs: Optional[int] = None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_bcast_end(self._h, u, self._ptr(rootdata), self._ptr(leafdata), OPS[op],
                                     self._stream(stream)), "sf_bcast_end")

    def bcast(self, rootdata, leafdata, op: str = "REPLACE", bs: Optional[int] = None, stream=None):
        args = (self._h, self._unit(rootdata, self.nroots_total, bs), self._ptr(rootdata), self._ptr(leafdata),
                OPS[op], self._stream(stream))
        check(self._lib.sf_bcast_begin(*args), "sf_bcast_begin")
        check(self._lib.sf_bcast_end(*args), "sf_bcast_end")
        return leafdata

    def reduce_begin(self, leafdata, rootdata, op: str = "SUM", bs: Optional[int] = None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_reduce_begin(self._h, u, self._ptr(leafdata), self._ptr(rootdata), OPS[op],
                                        self._stream(stream)), "sf_reduce_begin")

    def reduce_end(self, leafdata, rootdata, op: str = "SUM", bs: Optional[int] = None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_reduce_end(self._h, u, self._ptr(leafdata), self._ptr(rootdata), OPS[op],
                                      self._stream(stream)), "sf_reduce_end")

    def reduce(self, leafdata, rootdata, op: str = "SUM", bs: Optional[int] = None, stream=None):
        args = (self._h, self._unit(rootdata, self.nroots_total, bs), self._ptr(leafdata), self._ptr(rootdata),
                OPS[op], self._stream(stream))
        check(self._lib.sf_reduce_begin(*args), "sf_reduce_begin")
        check(self._lib.sf_reduce_end(*args), "sf_reduce_end")
        return rootdata

    def reduce_from_zero(self, leafdata, rootdata, op: str = "SUM", bs: Optional[int] = None, stream=None):
        """rootdata = Reduce(op) of leafdata into roots that start at zero (every root written,
        roots without leaves get 0; the old rootdata is never read)."""
        args = (self._h, self._unit(rootdata, self.nroots_total, bs), self._ptr(leafdata), self._ptr(rootdata),
                OPS[op], self._stream(stream))
        check(self._lib.sf_reduce_from_zero_begin(*args), "sf_reduce_from_zero_begin")
        check(self._lib.sf_reduce_from_zero_end(*args), "sf_reduce_from_zero_end")
        return rootdata

    def zero_leafless_roots(self, rootdata, argleaf=None, bs: Optional[int] = None, stream=None):
        """Roots without leaves -> 0 (and their argleaf entries -> -1); other roots untouched."""
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_zero_leafless_roots(self._h, u, self._ptr(rootdata), self._ptr(argleaf),
                                               self._stream(stream)), "sf_zero_leafless_roots")
        return rootdata

    def all_leaves_connected(self) -> bool:
        """Whether every leaf unit of the layout has a root (a Bcast REPLACE then writes all)."""
        if getattr(self, "_all_connected", None) is None:
            self._all_connected = self.info()["nedges"] == self.leaf_extent
        return self._all_connected

    def fetch_and_op_begin(self, rootdata, leafdata, leafupdate, op: str = "SUM", bs=None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_fetch_and_op_begin(self._h, u, self._ptr(rootdata), self._ptr(leafdata),
                                              self._ptr(leafupdate), OPS[op], self._stream(stream)),
              "sf_fetch_and_op_begin")

    def fetch_and_op_end(self, rootdata, leafdata, leafupdate, op: str = "SUM", bs=None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_fetch_and_op_end(self._h, u, self._ptr(rootdata), self._ptr(leafdata),
                                            self._ptr(leafupdate), OPS[op], self._stream(stream)),
              "sf_fetch_and_op_end")

    def fetch_and_op(self, rootdata, leafdata, leafupdate, op: str = "SUM", bs=None, stream=None):
        self.fetch_and_op_begin(rootdata, leafdata, leafupdate, op, bs, stream)
        self.fetch_and_op_end(rootdata, leafdata, leafupdate, op, bs, stream)
        return leafupdate

    # ---------------------------------------------------------------- host-buffer variants
    def _mt(self, t):
        return _abi.SF_MEM_DEVICE if t.is_cuda else _abi.SF_MEM_HOST

    def bcast_memtype(self, rootdata, leafdata, op: str = "REPLACE", bs=None, stream=None):
        """Bcast where either buffer may be a CPU tensor (pinned for asynchronous copies)."""
        u = self._unit(rootdata, self.nroots_total, bs)
        args = (self._h, u, self._mt(rootdata), self._ptr(rootdata), self._mt(leafdata), self._ptr(leafdata),
                OPS[op], self._stream(stream))
        check(self._lib.sf_bcast_with_memtype_begin(*args), "sf_bcast_with_memtype_begin")
        check(self._lib.sf_bcast_with_memtype_end(*args), "sf_bcast_with_memtype_end")
        return leafdata

    def reduce_memtype(self, leafdata, rootdata, op: str = "SUM", bs=None, stream=None):
        u = self._unit(rootdata, self.nroots_total, bs)
        args = (self._h, u, self._mt(leafdata), self._ptr(leafdata), self._mt(rootdata), self._ptr(rootdata),
                OPS[op], self._stream(stream))
        check(self._lib.sf_reduce_with_memtype_begin(*args), "sf_reduce_with_memtype_begin")
        check(self._lib.sf_reduce_with_memtype_end(*args), "sf_reduce_with_memtype_end")
        return rootdata


    def device_status(self, stream=None) -> int:
        """Device status bits raised since the previous call (0: none), then cleared; syncs the stream."""
        st = ctypes.c_int32(0)
        check(self._lib.sf_get_device_status(self._h, self._stream(stream), ctypes.byref(st)), "sf_get_device_status")
        return int(st.value)

    def reduce_maxloc(self, leafdata, rootdata, argleaf, bs=None, stream=None):
        """rootdata = max over each root's leaves, argleaf = first leaf reaching it (int32)."""
        u = self._unit(rootdata, self.nroots_total, bs)
        check(self._lib.sf_reduce_maxloc(self._h, u, self._ptr(leafdata), self._ptr(rootdata), self._ptr(argleaf),
                                         self._stream(stream)), "sf_reduce_maxloc")
        return rootdata, argleaf

    def maxloc_scatter(self, argleaf, rootgrad, leafgrad, bs=None, stream=None):
        u = self._unit(rootgrad, self.nroots_total, bs)
        check(self._lib.sf_maxloc_scatter(self._h, u, self._ptr(argleaf), self._ptr(rootgrad), self._ptr(leafgrad),
                                          self._stream(stream)), "sf_maxloc_scatter")
        return leafgrad

    def maxloc_grad(self, argleaf, rootgrad, leafgrad, bs=None, stream=None):
        """Every connected leaf's gradient unit: rootgrad where argleaf names the leaf, else 0."""
        u = self._unit(rootgrad, self.nroots_total, bs)
        check(self._lib.sf_maxloc_grad(self._h, u, self._ptr(argleaf), self._ptr(rootgrad), self._ptr(leafgrad),
                                       self._stream(stream)), "sf_maxloc_grad")
        return leafgrad

    # ---------------------------------------------------------------- autotuner
    def autotune(self, kind: str, src, dst, op: str, bs=None, reps: int = 3, stream=None) -> str:
        """Time the Bcast variants (kind "bcast": path x vector width x tile size) or the Reduce
        variants (kind "reduce": mode x vector width, the plan of the deterministic mode, tile size
        for atomics) and keep the fastest; its path or mode becomes what "auto" means for this
        forest (tuning() has the rest, the tuned plan becomes what reduce plan "auto" means).
        src/dst are not modified."""
        root = src if kind == "bcast" else dst
        u = self._unit(root, self.nroots_total, bs)
        k = _abi.SF_OP_BCAST if kind == "bcast" else _abi.SF_OP_REDUCE
        c = ctypes.c_int32()
        check(self._lib.sf_autotune(self._h, u, k, self._ptr(src), self._ptr(dst), OPS[op], reps,
                                    self._stream(stream), ctypes.byref(c)), "sf_autotune")
        names = {v: n for n, v in (PATHS if kind == "bcast" else MODES).items()}
        return names[c.value]


class Batch:
    """Many forests' Bcast / Reduce operations in few launches (optionally one CUDA graph)."""

    def __init__(self):
        self._lib = _abi.load()
        h = ctypes.c_void_p()
        check(self._lib.sf_batch_create(ctypes.byref(h)), "sf_batch_create")
        self._h = h
        self._ops = None
        self._keep = None

    def set_ops(self, ops):
        """ops: list of ("bcast"|"reduce", StarForest, op, src, dst, bs) or "barrier"."""
        arr = (_abi.sf_batch_op * len(ops))()
        keep = []
        for i, o in enumerate(ops):
            if o == "barrier":
                arr[i].kind = _abi.SF_OP_BARRIER
                continue
            kind, sf, op, src, dst, bs = o
            root = src if kind == "bcast" else dst
            arr[i].sf = sf._h
            arr[i].kind = _abi.SF_OP_BCAST if kind == "bcast" else _abi.SF_OP_REDUCE
            arr[i].unit = sf._unit(root, sf.nroots_total, bs)
            arr[i].op = OPS[op]
            arr[i].src = src.data_ptr()
            arr[i].dst = dst.data_ptr()
            keep.append((sf, src, dst))
        self._ops, self._keep = arr, keep
        return self

    def run(self, use_graph: bool = False, stream=None):
        check(self._lib.sf_batch_run(self._h, self._ops, len(self._ops), int(use_graph),
                                     StarForest._stream(stream)), "sf_batch_run")

    def launches(self) -> int:
        n = ctypes.c_int32()
        check(self._lib.sf_batch_launches(self._h, ctypes.byref(n)), "sf_batch_launches")
        return n.value

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._lib.sf_batch_destroy(self._h)
        except Exception:
            pass


def launch_count() -> int:
    """Kernels libsfgb has launched in this process."""
    return int(_abi.load().sf_launch_count())
