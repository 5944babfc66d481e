"""Pins for the oracle: what the paper and mathematics fix, checked without the oracle's
own code path (hand values from Fig. 2, dense incidence products, numpy scatter routines,
closed forms, invariants).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import sfgen
from tests import npref

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig2.json")))


def split(arr, off):
    return [arr[off[p]:off[p + 1]].tolist() for p in range(len(off) - 1)]


# ------------------------------------------------------------------ Fig. 2 worked example
def test_fig2_layout():
    ro, lo = oracle.layout(sfgen.fig2())
    assert ro.tolist() == GOLD["rootoff"]
    assert lo.tolist() == GOLD["leafoff"]


def test_fig2_in_degree_and_reduce_sum():
    f = sfgen.fig2()
    ro, lo = oracle.layout(f)
    deg = oracle.in_degree(f)
    assert split(deg, ro) == GOLD["in_degree"]
    root = oracle.reduce(f, "int32", 1, np.ones(lo[-1], np.int32), np.zeros(ro[-1], np.int32), "SUM")
    assert split(root, ro) == GOLD["in_degree"]
    rootf = oracle.reduce(f, "fp64", 1, np.ones(lo[-1]), np.zeros(ro[-1]), "SUM")
    assert split(rootf.astype(int), ro) == GOLD["in_degree"]


def test_fig2_bcast_replace():
    f = sfgen.fig2()
    ro, lo = oracle.layout(f)
    x = np.concatenate([100 * p + np.arange(f.nroots[p]) for p in range(3)]).astype(np.int64)
    leaf = oracle.bcast(f, "int64", 1, x, np.full(lo[-1], -1, np.int64), "REPLACE")
    assert split(leaf, lo) == GOLD["bcast_replace"]["leaves"]


def _fig2_leafvals(lo):
    return np.concatenate([10 * q + np.arange(lo[q + 1] - lo[q]) for q in range(3)])


def test_fig2_reduce_replace_last_edge_wins():
    f = sfgen.fig2()
    ro, lo = oracle.layout(f)
    y = _fig2_leafvals(lo).astype(np.int32)
    root = oracle.reduce(f, "int32", 1, y, np.full(ro[-1], -1, np.int32), "REPLACE")
    assert split(root, ro) == GOLD["reduce_replace"]["roots"]


def test_fig2_reduce_min():
    f = sfgen.fig2()
    ro, lo = oracle.layout(f)
    y = _fig2_leafvals(lo).astype(np.float64)
    root = oracle.reduce(f, "fp64", 1, y, np.full(ro[-1], 100.0), "MIN")
    assert split(root.astype(int), ro) == GOLD["reduce_min"]["roots"]


@pytest.mark.parametrize("dtype", ["int32", "int64", "fp64"])
def test_fig2_fetch_and_op_multisf(dtype):
    f = sfgen.fig2()
    ro, lo = oracle.layout(f)
    g = GOLD["fetch_and_op_sum"]
    npt = oracle.NPTYPE[dtype]
    r0 = np.concatenate([np.array(a) for a in g["root_init"]]).astype(npt)
    root, upd = oracle.fetch_and_op(f, dtype, 1, r0, np.ones(lo[-1], npt), np.full(lo[-1], -7, npt), "SUM")
    assert split(upd.astype(int), lo) == g["leafupdate"]
    assert split(root.astype(int), ro) == g["roots"]


# ------------------------------------------------------------------ dense incidence products
FORESTS = [sfgen.random_forest(s, P, 9, 12) for s, P in [(1, 1), (2, 3), (3, 5), (4, 4), (5, 7), (6, 2)]]


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("bs", [1, 3])
def test_bcast_is_incidence_product(f, bs):
    Pm, L, R = npref.incidence(f)
    nl, nr = Pm.shape
    x = sfgen.data("fp64", nr * bs, 11, 1).reshape(nr, bs)
    leaf0 = sfgen.data("fp64", nl * bs, 11, 2).reshape(nl, bs)
    connected = Pm.sum(axis=1) > 0
    got = oracle.bcast(f, "fp64", bs, x.ravel(), leaf0.ravel(), "REPLACE").reshape(nl, bs)
    want = np.where(connected[:, None], Pm @ x, leaf0)
    assert np.array_equal(got, want)
    got = oracle.bcast(f, "fp64", bs, x.ravel(), leaf0.ravel(), "SUM").reshape(nl, bs)
    want = leaf0 + Pm @ x       # one term per connected leaf: exact
    assert np.array_equal(got, want)


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("bs", [1, 2])
def test_reduce_sum_is_transpose_product_exact(f, bs):
    """Integer-valued doubles: every partial sum is exact, so any order equals P^T y."""
    Pm, L, R = npref.incidence(f)
    nl, nr = Pm.shape
    y = sfgen.data("int32", nl * bs, 12, 1).astype(np.float64).reshape(nl, bs)
    r0 = sfgen.data("int32", nr * bs, 12, 2).astype(np.float64).reshape(nr, bs)
    got = oracle.reduce(f, "fp64", bs, y.ravel(), r0.ravel(), "SUM").reshape(nr, bs)
    assert np.array_equal(got, r0 + Pm.T @ y)


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
def test_reduce_sum_fp_within_bound(f):
    """Random doubles: |oracle - exact| <= (deg+1) u sum|.| (any summation order)."""
    Pm, L, R = npref.incidence(f)
    nl, nr = Pm.shape
    y = sfgen.data("fp64", nl, 13, 1)
    r0 = sfgen.data("fp64", nr, 13, 2)
    got = oracle.reduce(f, "fp64", 1, y, r0, "SUM")
    deg = Pm.sum(axis=0)
    u = 2.0 ** -53
    for r in range(nr):
        terms = [r0[r]] + [y[l] for l in L[R == r]]
        exact = math.fsum(terms)
        assert abs(got[r] - exact) <= (deg[r] + 1) * u * sum(abs(t) for t in terms) + 1e-300


def test_adjoint_identity_exact():
    """<Bcast_REPLACE(x), y> = <x, Reduce_SUM(y)> over connected leaves (integers: exact)."""
    for f in FORESTS:
        Pm, L, R = npref.incidence(f)
        nl, nr = Pm.shape
        x = sfgen.data("int64", nr, 14, 1)
        y = sfgen.data("int64", nl, 14, 2)
        bx = oracle.bcast(f, "int64", 1, x, np.zeros(nl, np.int64), "REPLACE")
        ry = oracle.reduce(f, "int64", 1, y, np.zeros(nr, np.int64), "SUM")
        connected = Pm.sum(axis=1) > 0
        assert int((bx * y * connected).sum()) == int((x * ry).sum())


# ------------------------------------------------------------------ numpy scatter routines
@pytest.mark.parametrize("f", FORESTS + [sfgen.cfg1_plain_tiny()], ids=lambda f: f.name)
@pytest.mark.parametrize("dtype", ["int32", "int64", "fp32", "fp64"])
def test_reduce_min_max_sum_match_numpy_scatter(f, dtype):
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    npt = oracle.NPTYPE[dtype]
    kind = "wide" if dtype.startswith("int") else "signed"
    y = sfgen.data(dtype, lo[-1] * 2, 15, 1, kind).reshape(-1, 2)
    r0 = sfgen.data(dtype, ro[-1] * 2, 15, 2, kind).reshape(-1, 2)
    for op, ufunc in (("MIN", np.minimum), ("MAX", np.maximum)):
        want = r0.copy()
        ufunc.at(want, R, y[L])
        got = oracle.reduce(f, dtype, 2, y.ravel(), r0.ravel(), op).reshape(-1, 2)
        assert np.array_equal(got, want), op
    if dtype.startswith("int"):   # wraparound sum: numpy add.at wraps too
        want = r0.copy()
        with np.errstate(over="ignore"):
            np.add.at(want, R, y[L])
        got = oracle.reduce(f, dtype, 2, y.ravel(), r0.ravel(), "SUM").reshape(-1, 2)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["SUM", "MIN", "MAX"])
def test_bcast_ops_match_numpy_gather(f, op):
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    x = sfgen.data("int32", ro[-1], 16, 1, "wide")
    leaf0 = sfgen.data("int32", lo[-1], 16, 2, "wide")
    want = leaf0.copy()
    with np.errstate(over="ignore"):
        want[L] = {"SUM": np.add, "MIN": np.minimum, "MAX": np.maximum}[op](leaf0[L], x[R])
    assert np.array_equal(oracle.bcast(f, "int32", 1, x, leaf0, op), want)


def test_reduce_replace_last_edge_matches_numpy():
    for f in FORESTS:
        L, R = npref.edge_arrays(f)
        ro, lo = npref.offsets(f)
        y = sfgen.data("int64", lo[-1], 17, 1, "wide")
        r0 = sfgen.data("int64", ro[-1], 17, 2, "wide")
        last = np.full(ro[-1], -1, np.int64)
        np.maximum.at(last, R, np.arange(len(R)))      # last canonical edge of every root
        want = r0.copy()
        hit = last >= 0
        want[hit] = y[L[last[hit]]]
        assert np.array_equal(oracle.reduce(f, "int64", 1, y, r0, "REPLACE"), want)


def test_round_trip_one_to_one():
    """Ping-pong (Sec. VI.A): Reduce REPLACE after Bcast REPLACE restores the roots."""
    for f in [sfgen.one_to_one(s, P, n) for s, P, n in [(1, 1, 7), (2, 3, 50), (3, 8, 33)]] + [sfgen.pingpong(100)]:
        ro, lo = oracle.layout(f)
        x = sfgen.data("fp64", ro[-1] * 3, 18, 1)
        leaf = oracle.bcast(f, "fp64", 3, x, np.zeros(lo[-1] * 3), "REPLACE")
        back = oracle.reduce(f, "fp64", 3, leaf, np.zeros(ro[-1] * 3), "REPLACE")
        assert np.array_equal(back, x)


# ------------------------------------------------------------------ blocked fold D (hand values)
def star(n):
    """One root on rank 0, n leaves on rank 0 all pointing at it."""
    return sfgen.Forest(1, np.array([1]), np.array([n]), [None], [np.zeros(n, np.int32)],
                        [np.zeros(n, np.int64)], name=f"star{n}")


def test_fold_left_order_fp64():
    """Leaves (1, 1e16, -1e16): the left fold gives (1+1e16)-1e16 = 0 (1 is absorbed),
    any order that adds 1e16 and -1e16 first gives 1."""
    f = star(3)
    got = oracle.reduce(f, "fp64", 1, np.array([1.0, 1e16, -1e16]), np.array([0.0]), "SUM")
    assert got[0] == 0.0
    got = oracle.reduce(f, "fp64", 1, np.array([1e16, -1e16, 1.0]), np.array([0.0]), "SUM")
    assert got[0] == 1.0


def test_fold_root_added_last():
    """root + D(y), not ((root + y0) + y1): root 2^53, leaves 1, 1 -> D = 2 -> 2^53 + 2 exactly;
    adding the root first would absorb both ones (ties to even) and give 2^53."""
    f = star(2)
    got = oracle.reduce(f, "fp64", 1, np.array([1.0, 1.0]), np.array([2.0 ** 53]), "SUM")
    assert got[0] == 2.0 ** 53 + 2.0


def test_fold_blocks_of_64_fp32():
    """128 leaves: 2^24 then 127 ones (fp32).  Block 0 = fl(2^24 + 1 + ...) = 2^24 (each 1 is
    a tie rounded to even), block 1 = 64 exactly; D = 2^24 + 64.  A plain left fold would
    give 2^24, a block of 32 would give 2^24 + 96."""
    f = star(128)
    y = np.ones(128, np.float32)
    y[0] = 2.0 ** 24
    got = oracle.reduce(f, "fp32", 1, y, np.zeros(1, np.float32), "SUM")
    assert got[0] == np.float32(2.0 ** 24 + 64)


def test_fold_three_levels_fp32():
    """4097 leaves: 2^24 then 4096 ones.  Level 1: 65 blocks -> (2^24, 64 x 63, 1).  Level 2:
    65 > 64 so blocks again -> (2^24 + 4032, 1).  Level 3: 2^24 + 4033 is a tie between
    2^24 + 4032 (even significand) and 2^24 + 4034 -> 2^24 + 4032."""
    f = star(4097)
    y = np.ones(4097, np.float32)
    y[0] = 2.0 ** 24
    got = oracle.reduce(f, "fp32", 1, y, np.zeros(1, np.float32), "SUM")
    assert got[0] == np.float32(2.0 ** 24 + 4032)


def test_fold_bf16_accumulates_in_fp32_and_rounds_once():
    """bf16 leaves 1.0 x 300 into root 0: fp32 sum is 300 exactly; bf16(300) = 300 (needs 7
    significand bits: 300 = 0b100101100).  Rounding after every add would stall at 256."""
    f = star(300)
    one = np.array([0x3F80] * 300, np.uint16)
    got = oracle.reduce(f, "bf16", 1, one, np.zeros(1, np.uint16), "SUM")
    val = np.array([int(got[0]) << 16], np.uint32).view(np.float32)[0]
    assert val == 300.0


# ------------------------------------------------------------------ FetchAndOp invariants
@pytest.mark.parametrize("f", FORESTS + [sfgen.cfg1_plain_tiny()], ids=lambda f: f.name)
def test_fetch_and_op_multisf_invariant(f):
    """Roots at degree-prefix offsets, leaves 1 (Sec. III.B): each root's fetched values are
    exactly {o, ..., o+deg-1}, increasing in canonical order, and the root ends at o+deg."""
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    deg = np.bincount(R, minlength=ro[-1])
    off = np.concatenate([[0], np.cumsum(deg)[:-1]]).astype(np.int32)
    root, upd = oracle.fetch_and_op(f, "int32", 1, off, np.ones(lo[-1], np.int32),
                                    np.full(lo[-1], -1, np.int32), "SUM")
    assert np.array_equal(root, off + deg)
    order = np.argsort(R, kind="stable")          # edges grouped by root, canonical inside
    fetched = upd[L[order]]
    assert np.array_equal(fetched, np.arange(len(L)))


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
def test_fetch_and_op_prefix_sums_match_cumsum(f):
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = sfgen.data("int64", lo[-1], 19, 1, "wide")
    r0 = sfgen.data("int64", ro[-1], 19, 2, "wide")
    root, upd = oracle.fetch_and_op(f, "int64", 1, r0, y, np.zeros(lo[-1], np.int64), "SUM")
    want_root, want_upd = r0.copy(), np.zeros(lo[-1], np.int64)
    with np.errstate(over="ignore"):
        for r in np.unique(R):
            es = np.nonzero(R == r)[0]
            inc = np.cumsum(np.concatenate([[r0[r]], y[L[es]]]).astype(np.int64))
            want_upd[L[es]] = inc[:-1]
            want_root[r] = inc[-1]
    assert np.array_equal(root, want_root)
    assert np.array_equal(upd, want_upd)


def test_fetch_and_op_replace_is_a_chain_of_swaps():
    f = star(4)
    root, upd = oracle.fetch_and_op(f, "int32", 1, np.array([9], np.int32),
                                    np.array([1, 2, 3, 4], np.int32), np.zeros(4, np.int32), "REPLACE")
    assert root.tolist() == [4] and upd.tolist() == [9, 1, 2, 3]


def test_fetch_and_op_max_fetches_running_max():
    f = star(5)
    root, upd = oracle.fetch_and_op(f, "fp64", 1, np.array([0.5]), np.array([0.1, 0.9, 0.3, 1.5, -2.0]),
                                    np.zeros(5), "MAX")
    assert root.tolist() == [1.5] and upd.tolist() == [0.5, 0.5, 0.9, 0.9, 1.5]


# ------------------------------------------------------------------ helpers of the oracle
def test_bf16_rounding_matches_torch_cpu():
    torch = pytest.importorskip("torch")
    bits = sfgen.rng.u64(99, 1, 200000) >> np.uint64(32)
    x = bits.astype(np.uint32).view(np.float32)
    x = x[np.isfinite(x)]
    # ties and near-ties explicitly
    base = np.arange(0, 1 << 16, dtype=np.uint32) << np.uint32(16)
    extra = np.concatenate([base | 0x8000, base | 0x7FFF, base | 0x8001]).view(np.float32)
    x = np.concatenate([x, extra[np.isfinite(extra)]])
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = oracle.f32_to_bf16(x)
    assert np.array_equal(got, want)


def test_sum_reference_matches_fsum():
    f = sfgen.random_forest(21, 3, 6, 40)
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = sfgen.data("fp64", lo[-1], 20, 1) * 1e3
    r0 = sfgen.data("fp64", ro[-1], 20, 2)
    s, a = oracle.sum_reference(f, "fp64", 1, y, r0)
    for r in range(ro[-1]):
        terms = [r0[r]] + list(y[L[R == r]])
        ex = math.fsum(terms)
        assert abs(s[r] - ex) <= 4 * 2.0 ** -53 * abs(ex) + 1e-290
        assert a[r] == pytest.approx(sum(abs(t) for t in terms), rel=1e-12)


def test_maxloc_matches_lexsort():
    f = sfgen.random_forest(22, 4, 8, 30)
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = sfgen.data("int32", lo[-1], 21, 1)     # many ties (values < 1000, few edges)
    y[::3] = 5
    val, arg = oracle.reduce_maxloc(f, "int32", 1, y)
    e = np.arange(len(L))
    order = np.lexsort((e, -y[L].astype(np.int64), R))      # by root, value desc, edge asc
    first = np.ones(len(order), bool)
    first[1:] = R[order][1:] != R[order][:-1]
    want_val = np.zeros(ro[-1], np.int32)
    want_arg = np.full(ro[-1], -1, np.int64)
    want_val[R[order][first]] = y[L][order][first]
    want_arg[R[order][first]] = e[order][first]
    assert np.array_equal(val, want_val) and np.array_equal(arg, want_arg)


@pytest.mark.parametrize("dtype,bs", [("fp64", 3), ("bf16", 2), ("int64", 4)])
def test_maxloc_per_component_matches_lexsort(dtype, bs):
    """MAX with location element by element of multi-component units: per (root, component)
    the largest value and the first canonical edge holding it, from a numpy lexsort (bf16
    compared as the float32 values of its bit patterns).  Values on a coarse grid tie often."""
    f = sfgen.random_forest(23, 3, 10, 40)
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = sfgen.data(dtype, lo[-1] * bs, 24, 1)
    if dtype == "bf16":
        y = (y & np.uint16(0xFE00)) | np.uint16(0x3C00)   # few distinct values: ties
        key = (y.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    elif dtype == "fp64":
        y = np.round(y * 4) / 4
        key = y
    else:
        y = y % 7
        key = y.astype(np.float64)
    val, arg = oracle.reduce_maxloc(f, dtype, bs, y)
    e = np.arange(len(L))
    for c in range(bs):
        kc = key.reshape(-1, bs)[:, c]
        order = np.lexsort((e, -kc[L], R))      # by root, value descending, edge ascending
        first = np.ones(len(order), bool)
        first[1:] = R[order][1:] != R[order][:-1]
        want_arg = np.full(ro[-1], -1, np.int64)
        want_arg[R[order][first]] = e[order][first]
        got_arg = arg.reshape(-1, bs)[:, c]
        assert np.array_equal(got_arg, want_arg), f"component {c}"
        has = want_arg >= 0
        got_val = val.reshape(-1, bs)[:, c]
        assert np.array_equal(got_val[has], y.reshape(-1, bs)[L[want_arg[has]], c])
        assert not got_val[~has].any()


def test_empty_forest_and_isolated():
    f = sfgen.Forest(2, np.array([3, 0]), np.array([0, 0]), [None, None],
                     [np.zeros(0, np.int32)] * 2, [np.zeros(0, np.int64)] * 2)
    ro, lo = oracle.layout(f)
    assert ro.tolist() == [0, 3, 3] and lo.tolist() == [0, 0, 0]
    r = oracle.reduce(f, "fp64", 1, np.zeros(0), np.array([1.0, 2.0, 3.0]), "SUM")
    assert r.tolist() == [1.0, 2.0, 3.0]


# ------------------------------------------------------------------ the bf16 branch of the element op
def _f32_of_bf16(h):
    """float32 values of bf16 bit patterns (exact: a bf16 is the top half of a float32)."""
    return (np.asarray(h, np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def _bf16_full(n, seed, tag, scale=1.0):
    """n bf16 bit patterns with full 8-bit significands (so sums of two round), made by
    torch's own float32 -> bfloat16 conversion of uniform float32 values."""
    torch = pytest.importorskip("torch")
    x = sfgen.data("fp32", n, seed, tag) * np.float32(scale)
    return torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


def _torch_bf16(h):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(np.asarray(h, np.uint16).view(np.int16).copy()).view(torch.bfloat16)


def _bits(t):
    return t.view(pytest.importorskip("torch").int16).numpy().view(np.uint16)


@pytest.mark.parametrize("f", FORESTS + [sfgen.cfg1_plain_tiny()], ids=lambda f: f.name)
def test_bf16_reduce_min_max_match_numpy_scatter(f):
    """bf16 Reduce MIN/MAX = numpy minimum.at / maximum.at on the float32 values of the bit
    patterns (every bf16 is exactly a float32, and the result is one of the inputs)."""
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = _bf16_full(lo[-1] * 2, 23, 1).reshape(-1, 2)
    r0 = _bf16_full(ro[-1] * 2, 23, 2).reshape(-1, 2)
    for op, ufunc in (("MIN", np.minimum), ("MAX", np.maximum)):
        want = _f32_of_bf16(r0).copy()
        ufunc.at(want, R, _f32_of_bf16(y)[L])
        got = oracle.reduce(f, "bf16", 2, y.ravel(), r0.ravel(), op).reshape(-1, 2)
        assert np.array_equal(_f32_of_bf16(got), want), op


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["SUM", "MIN", "MAX"])
def test_bf16_bcast_ops_match_torch(f, op):
    """bf16 Bcast with an op: each leaf takes one root, combined and rounded by torch's own
    CPU bfloat16 arithmetic (SUM rounds the float32 sum to nearest even)."""
    torch = pytest.importorskip("torch")
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    x = _bf16_full(ro[-1] * 3, 24, 1, 4.0).reshape(-1, 3)
    leaf0 = _bf16_full(lo[-1] * 3, 24, 2, 4.0).reshape(-1, 3)
    lt, xt = _torch_bf16(leaf0), _torch_bf16(x)
    fn = {"SUM": torch.add, "MIN": torch.minimum, "MAX": torch.maximum}[op]
    want = lt.clone()
    idx_l, idx_r = torch.from_numpy(L), torch.from_numpy(R)
    want[idx_l] = fn(lt[idx_l], xt[idx_r])
    got = oracle.bcast(f, "bf16", 3, x.ravel(), leaf0.ravel(), op).reshape(-1, 3)
    assert np.array_equal(got, _bits(want))


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
def test_bf16_fetch_and_op_sum_rounds_every_op(f):
    """bf16 FetchAndOp SUM is a chain of bf16 additions, each rounded: replayed edge by edge
    in canonical order with torch CPU bfloat16 scalars."""
    torch = pytest.importorskip("torch")
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = _bf16_full(lo[-1], 25, 1)
    r0 = _bf16_full(ro[-1], 25, 2, 8.0)
    r = _torch_bf16(r0).clone()
    yt = _torch_bf16(y)
    upd = torch.zeros(lo[-1], dtype=torch.bfloat16)
    for e in range(len(L)):
        upd[L[e]] = r[R[e]]
        r[R[e]] = r[R[e]] + yt[L[e]]
    got_r, got_u = oracle.fetch_and_op(f, "bf16", 1, r0, y, np.zeros(lo[-1], np.uint16), "SUM")
    connected = np.zeros(lo[-1], bool)
    connected[L] = True
    assert np.array_equal(got_r, _bits(r))
    assert np.array_equal(got_u[connected], _bits(upd)[connected])


def test_bf16_rounding_per_op_differs_from_rounding_once():
    """Hand values.  bf16 has 8 significand bits, so 256 + 1 = 257 is a tie between 256 and
    258 and rounds to the even 256.  FetchAndOp SUM of leaves (1, 1) into root 256 rounds after
    each op: 256 -> 256 -> 256, fetching (256, 256).  Reduce SUM folds the leaves in float32
    first and rounds once: 256 + 2 = 258.  Bcast SUM of root 1 into leaf 256 gives 256, and
    1.0078125 + 2^-8 (a tie between 1.0078125 and 1.015625) gives the even 1.015625."""
    f = star(2)
    b256, b1, b258 = 0x4380, 0x3F80, 0x4381
    root, upd = oracle.fetch_and_op(f, "bf16", 1, np.array([b256], np.uint16), np.array([b1, b1], np.uint16),
                                    np.zeros(2, np.uint16), "SUM")
    assert root.tolist() == [b256] and upd.tolist() == [b256, b256]
    red = oracle.reduce(f, "bf16", 1, np.array([b1, b1], np.uint16), np.array([b256], np.uint16), "SUM")
    assert red.tolist() == [b258]
    one = sfgen.Forest(1, np.array([1]), np.array([1]), [None], [np.zeros(1, np.int32)], [np.zeros(1, np.int64)])
    assert oracle.bcast(one, "bf16", 1, np.array([b1], np.uint16), np.array([b256], np.uint16),
                        "SUM").tolist() == [b256]
    assert oracle.bcast(one, "bf16", 1, np.array([0x3B80], np.uint16), np.array([0x3F81], np.uint16),
                        "SUM").tolist() == [0x3F82]


def test_max_ties_keep_the_first_value_in_canonical_order():
    """MAX(a, b) = (a < b ? b : a) keeps the current value on a tie, so +0 and -0 (equal)
    resolve by order: the root keeps its own zero when a leaf brings the other one, and a root
    below zero takes the first zero in canonical order."""
    f = star(3)
    pz, nz = 0.0, -0.0
    got = oracle.reduce(f, "fp64", 1, np.array([nz, pz, nz]), np.array([-1.0]), "MAX")
    assert np.signbit(got[0])
    got = oracle.reduce(f, "fp64", 1, np.array([pz, nz, nz]), np.array([-1.0]), "MAX")
    assert got[0] == 0.0 and not np.signbit(got[0])
    got = oracle.reduce(f, "fp64", 1, np.array([pz, pz, pz]), np.array([nz]), "MAX")
    assert np.signbit(got[0])
    got = oracle.reduce(f, "fp32", 1, np.array([nz, pz, nz], np.float32), np.array([1.0], np.float32), "MIN")
    assert np.signbit(got[0])


def test_nan_leaf_never_wins_min_max():
    """The element op compares with < only, so a NaN leaf loses every MIN/MAX against a
    non-NaN root (NaN < x and x < NaN are both false).  NaN input is outside the library's
    contract for MIN/MAX; this pins what the oracle computes."""
    f = star(3)
    got = oracle.reduce(f, "fp64", 1, np.array([np.nan, 2.0, np.nan]), np.array([1.0]), "MAX")
    assert got[0] == 2.0
    got = oracle.reduce(f, "fp64", 1, np.array([np.nan, 0.5, np.nan]), np.array([1.0]), "MIN")
    assert got[0] == 0.5


# ------------------------------------------------------------------ Gather / Scatter (multi-forest)
def test_fig2_gather_and_scatter():
    f = sfgen.fig2()
    ro, lo = oracle.layout(f)
    g = GOLD["gather"]
    y = _fig2_leafvals(lo).astype(np.int32)
    multi = oracle.gather(f, "int32", 1, y, np.full(f.nedges, -9, np.int32))
    assert split(multi, g["multirootoff"]) == g["multiroots"]
    back = oracle.scatter(f, "int32", 1, 100 + np.arange(f.nedges, dtype=np.int32), np.full(lo[-1], -1, np.int32))
    assert split(back, lo) == GOLD["scatter"]["leaves"]


@pytest.mark.parametrize("f", FORESTS + [sfgen.cfg1_plain_tiny()], ids=lambda f: f.name)
def test_gather_is_a_stable_sort_by_root_and_scatter_inverts_it(f):
    """Gather lists the leaf units grouped by root, canonical order inside a root (a stable
    argsort of the root units); Scatter puts them back (isolated leaves untouched)."""
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    y = sfgen.data("fp64", lo[-1] * 2, 26, 1).reshape(-1, 2)
    order = np.argsort(R, kind="stable")
    multi = oracle.gather(f, "fp64", 2, y.ravel(), np.zeros(len(L) * 2)).reshape(-1, 2)
    assert np.array_equal(multi, y[L[order]])
    leaf0 = sfgen.data("fp64", lo[-1] * 2, 26, 2).reshape(-1, 2)
    back = oracle.scatter(f, "fp64", 2, multi.ravel(), leaf0.ravel()).reshape(-1, 2)
    want = leaf0.copy()
    want[L] = y[L]
    assert np.array_equal(back, want)


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
def test_gather_slots_are_the_fetch_and_op_multisf_offsets(f):
    """The paper's recipe (Sec. III.B): FetchAndOp SUM with roots at degree-prefix offsets and
    leaves of 1 fetches, for every leaf, its multi-root; Gather must put the leaf there."""
    L, R = npref.edge_arrays(f)
    ro, lo = npref.offsets(f)
    deg = np.bincount(R, minlength=ro[-1])
    off = np.concatenate([[0], np.cumsum(deg)[:-1]]).astype(np.int64)
    _, slot = oracle.fetch_and_op(f, "int64", 1, off, np.ones(lo[-1], np.int64), np.full(lo[-1], -1, np.int64), "SUM")
    y = sfgen.data("int64", lo[-1], 27, 1, "wide")
    multi = oracle.gather(f, "int64", 1, y, np.zeros(len(L), np.int64))
    assert np.array_equal(multi[slot[L]], y[L])
