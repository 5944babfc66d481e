"""Helpers for the GPU parity tests: numpy <-> torch CUDA tensors, oracle comparison."""
from __future__ import annotations

import numpy as np

import oracle
import sfgen

TOL = {"fp32": 1e-6, "fp64": 1e-13, "bf16": 1e-2}


def to_dev(a: np.ndarray, dtype: str):
    import torch
    if dtype == "bf16":
        return torch.from_numpy(a.view(np.int16).copy()).cuda().view(torch.bfloat16)
    return torch.from_numpy(a.copy()).cuda()


def to_host(t, dtype: str) -> np.ndarray:
    import torch
    if dtype == "bf16":
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def make_data(f, dtype: str, bs: int, seed: int, kind_root="signed", kind_leaf="signed"):
    ro, lo = oracle.layout(f)
    root = sfgen.data(dtype, int(ro[-1]) * bs, seed, 1, kind_root)
    leaf = sfgen.data(dtype, int(lo[-1]) * bs, seed, 2, kind_leaf)
    return root, leaf


def assert_bits_equal(got: np.ndarray, want: np.ndarray, what: str):
    if got.dtype.kind == "f":
        g, w = got.view(np.uint64 if got.itemsize == 8 else np.uint32), want.view(
            np.uint64 if want.itemsize == 8 else np.uint32)
    else:
        g, w = got, want
    bad = np.nonzero(g != w)[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} of {g.size} differ; first at {i}: got {got[i]!r} want {want[i]!r}")


def assert_atomic_sum_close(got, want, f, dtype, bs, leaf, root0, what):
    """|gpu - oracle| <= tol * deg * (|r0| + sum |y|) per root element."""
    deg = oracle.in_degree(f)
    _, absum = oracle.sum_reference(f, dtype, bs, leaf, root0)
    d = np.repeat(np.maximum(deg, 1), bs).astype(np.float64)
    g = got.astype(np.float64)
    w = want.astype(np.float64)
    err = np.abs(g - w)
    bound = TOL[dtype] * d * absum
    bad = np.nonzero(err > bound)[0]
    if bad.size:
        i = bad[0]
        raise AssertionError(f"{what}: {bad.size} outside bound; first at {i}: err {err[i]} bound {bound[i]}")
    return float(np.max(err / np.maximum(absum, 1e-300))) if err.size else 0.0


def signed_zero_forest(nroots=4000, seed=93):
    """Roots of in-degree 1..9 on three ranks, leaves in random rank order: the data below
    gives every root a mix of +0 and -0 leaves, so MIN/MAX ties are decided by canonical order."""
    deg = (np.arange(nroots) % 9) + 1
    owner = np.repeat(np.arange(nroots), deg)
    owner = owner[np.argsort(sfgen.rng.u64(seed, 1, owner.size), kind="stable")]
    per = -(-nroots // 3)
    cuts = np.linspace(0, owner.size, 4).astype(int)
    rr = [(owner[cuts[q]:cuts[q + 1]] // per).astype(np.int32) for q in range(3)]
    ri = [(owner[cuts[q]:cuts[q + 1]] % per).astype(np.int64) for q in range(3)]
    roots = np.array([min(per, nroots - p * per) for p in range(3)])
    return sfgen.Forest(3, roots, np.diff(cuts), [None] * 3, rr, ri, name="signed_zero")


def signed_zero_data(f, dtype, bs, seed):
    """Leaves +0 or -0 at random; roots -1, +0 or -0 (MAX) / +1, +0 or -0 (MIN)."""
    ro, lo = oracle.layout(f)
    npt = {"fp32": np.float32, "fp64": np.float64}[dtype]
    sgn = sfgen.rng.u64(seed, 1, int(lo[-1]) * bs) & np.uint64(1)
    leaf = np.where(sgn == 1, npt(-0.0), npt(0.0)).astype(npt)
    pick = sfgen.rng.u64(seed, 2, int(ro[-1]) * bs) % np.uint64(3)
    root = np.choose(pick.astype(np.int64), [npt(-1.0), npt(0.0), npt(-0.0)]).astype(npt)
    return root, leaf

