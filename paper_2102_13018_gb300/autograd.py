"""Differentiable star-forest operations (torch.autograd.Function), all computed by libsfgb.

Bcast with REPLACE is the linear map x -> P x (P the leaf-by-root incidence matrix, Sec. IV.A:
lvec = P x), so its adjoint is Reduce with SUM (y = P^T lvec), and vice versa.  Reduce MAX sends
each root's gradient to the first leaf, in canonical order, that reached the maximum.  Units
are rows of bs elements; fp32 and bf16 storage both accumulate in fp32 (bf16 Reduce SUM rounds
once per result).  Roots without leaves get 0 in the functional forms and no gradient.

Outputs are allocated uninitialised and written whole by the library: the Reduce runs from
zero (roots never read, roots without leaves zeroed by the library), and a Bcast output is
zero-filled only when some leaf of the layout has no root.
"""
from __future__ import annotations

import torch

from .sf import StarForest


def _units(t: torch.Tensor, n: int):
    if t.numel() % max(n, 1):
        raise ValueError(f"{t.numel()} elements are not {n} units")
    return t.numel() // max(n, 1)


def _leaf_out(sf: StarForest, bs: int, like: torch.Tensor) -> torch.Tensor:
    """The output of a Bcast REPLACE: uninitialised when every leaf has a root (all are written),
    else zeros (leaves without a root keep 0)."""
    make = torch.empty if sf.all_leaves_connected() else torch.zeros
    return make(sf.leaf_extent, bs, dtype=like.dtype, device=like.device)


class _Bcast(torch.autograd.Function):
    @staticmethod
    def forward(ctx, root, sf: StarForest):
        bs = _units(root, sf.nroots_total)
        root = root.contiguous()
        leaf = _leaf_out(sf, bs, root)
        sf.bcast(root, leaf, "REPLACE", bs=bs)
        ctx.sf, ctx.bs = sf, bs
        return leaf

    @staticmethod
    def backward(ctx, g):
        sf, bs = ctx.sf, ctx.bs
        groot = torch.empty(sf.nroots_total, bs, dtype=g.dtype, device=g.device)
        sf.reduce_from_zero(g.contiguous(), groot, "SUM", bs=bs)
        return groot, None


class _ReduceSum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, leaf, sf: StarForest):
        bs = _units(leaf, sf.leaf_extent)
        leaf = leaf.contiguous()
        root = torch.empty(sf.nroots_total, bs, dtype=leaf.dtype, device=leaf.device)
        sf.reduce_from_zero(leaf, root, "SUM", bs=bs)
        ctx.sf, ctx.bs = sf, bs
        return root

    @staticmethod
    def backward(ctx, g):
        sf, bs = ctx.sf, ctx.bs
        gleaf = _leaf_out(sf, bs, g)
        sf.bcast(g.contiguous(), gleaf, "REPLACE", bs=bs)
        return gleaf, None


class _ReduceMax(torch.autograd.Function):
    @staticmethod
    def forward(ctx, leaf, sf: StarForest):
        bs = _units(leaf, sf.leaf_extent)
        leaf = leaf.contiguous()
        root = torch.empty(sf.nroots_total, bs, dtype=leaf.dtype, device=leaf.device)
        arg = torch.empty((sf.nroots_total, bs), dtype=torch.int32, device=leaf.device)
        sf.zero_leafless_roots(root, arg, bs=bs)
        sf.reduce_maxloc(leaf, root, arg, bs=bs)
        ctx.sf, ctx.bs = sf, bs
        ctx.save_for_backward(arg)
        return root

    @staticmethod
    def backward(ctx, g):
        (arg,) = ctx.saved_tensors
        sf, bs = ctx.sf, ctx.bs
        # every connected leaf's unit is written (the selected elements of g, zeros elsewhere)
        gleaf = _leaf_out(sf, bs, g)
        sf.maxloc_grad(arg, g.contiguous(), gleaf, bs=bs)
        return gleaf, None


def bcast(sf: StarForest, root: torch.Tensor) -> torch.Tensor:
    """leaf = Bcast_REPLACE(root) into zeros; shape (leaf_extent, bs)."""
    return _Bcast.apply(root, sf)


def reduce(sf: StarForest, leaf: torch.Tensor, op: str = "SUM") -> torch.Tensor:
    """root = Reduce_op(leaf) into zeros (SUM) or the per-root maximum (MAX); (nroots, bs)."""
    if op == "SUM":
        return _ReduceSum.apply(leaf, sf)
    if op == "MAX":
        return _ReduceMax.apply(leaf, sf)
    raise ValueError("differentiable Reduce supports SUM and MAX")
