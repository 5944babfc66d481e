"""The gather-then-fold kernels against the oracle, bit for bit (GB300): the deterministic
Reduce of multi-vector units (SUM/MIN/MAX with nv > 1 vectors per unit) and MAX with location
(values and leaf locations, ties resolved by canonical order).  Power-law and Zipf in-degrees,
a heavy star whose fold runs three levels, units up to the kernels' vector limits and past them
(the general kernels), vector widths 4/8/16 bytes, and the Reduce from zero."""
import numpy as np
import pytest

import oracle
import sfgen
from tests.gpu_util import assert_bits_equal, make_data, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import StarForest  # noqa: E402

FORESTS = [sfgen.cfg5_powerlaw(4096, 40000, 4), sfgen.zipf_forest(78, 2, 30000, 2000, 3),
           sfgen.owned_plus_ghosts(8, keep=0.7)]
_SF = {}


def sf_for(f):
    if f.name not in _SF:
        _SF[f.name] = StarForest.from_forest(f).setup().set_mode("deterministic")
    return _SF[f.name]


# (dtype, bs, vector bytes): 2 .. 512 vectors per unit, each vector width
UNITS = [("fp32", 64, 0), ("fp32", 64, 4), ("fp32", 64, 8), ("fp64", 5, 0), ("fp64", 3, 0), ("bf16", 64, 0),
         ("bf16", 24, 0), ("int32", 7, 0), ("int64", 3, 0), ("int64", 4, 16), ("fp32", 512, 4), ("fp32", 6, 8)]


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["SUM", "MIN", "MAX"])
@pytest.mark.parametrize("dtype,bs,vb", UNITS)
def test_flat_reduce_bit_exact(f, op, dtype, bs, vb):
    sf = sf_for(f).set_vector_bytes(vb)
    kind = "wide" if dtype.startswith("int") else "signed"
    root, leaf = make_data(f, dtype, bs, 1700, kind, kind)
    want = oracle.reduce(f, dtype, bs, leaf, root, op)
    l = to_dev(leaf, dtype)
    for call in range(2):   # the second call finds the arrival counters reset
        r = to_dev(root, dtype)
        sf.reduce(l, r, op, bs=bs)
        assert_bits_equal(to_host(r, dtype), want, f"flat {f.name} {op} {dtype}x{bs} vb{vb} call {call}")
    zeros = np.zeros_like(root)
    r = to_dev(np.full_like(root, 0x7F if dtype == "bf16" else 3), dtype)
    sf.reduce_from_zero(l, r, op, bs=bs)
    assert_bits_equal(to_host(r, dtype), oracle.reduce(f, dtype, bs, leaf, zeros, op),
                      f"flat from zero {f.name} {op} {dtype}x{bs} vb{vb}")
    assert_bits_equal(to_host(l, dtype), leaf, "leafdata must be untouched")
    sf.set_vector_bytes(0)
    assert sf.device_status() == 0


@pytest.mark.parametrize("dtype,bs,vb", [("fp32", 600, 4), ("fp64", 3000, 8)])
def test_units_past_the_flat_limits_keep_the_general_kernel(dtype, bs, vb):
    """600 vectors per unit (over 512), and 24 KB units (over one gather round)."""
    f = FORESTS[1]
    sf = sf_for(f).set_vector_bytes(vb)
    root, leaf = make_data(f, dtype, bs, 1701)
    for op in ("SUM", "MAX"):
        r = to_dev(root, dtype)
        sf.reduce(to_dev(leaf, dtype), r, op, bs=bs)
        assert_bits_equal(to_host(r, dtype), oracle.reduce(f, dtype, bs, leaf, root, op), f"{op} {dtype}x{bs}")
    sf.set_vector_bytes(0)
    assert sf.device_status() == 0


def test_heavy_star_multi_vector_three_fold_levels():
    """A star of 300,000 leaves (4688 blocks -> 74 -> 2 -> 1) with 8- and 64-element units."""
    n = 300000
    f = sfgen.Forest(1, np.array([3]), np.array([n]), [None], [np.zeros(n, np.int32)],
                     [(np.arange(n) % 7 == 0).astype(np.int64)], name="heavystar")
    sf = StarForest.from_forest(f).setup()
    for dtype, bs in (("fp32", 8), ("fp64", 2), ("bf16", 64)):
        root, leaf = make_data(f, dtype, bs, 1702)
        want = oracle.reduce(f, dtype, bs, leaf, root, "SUM")
        l = to_dev(leaf, dtype)
        for _ in range(2):
            r = to_dev(root, dtype)
            sf.reduce(l, r, "SUM", bs=bs)
            assert_bits_equal(to_host(r, dtype), want, f"heavy star {dtype}x{bs}")
    assert sf.device_status() == 0


def test_signed_zero_ties_multi_vector():
    """+0 / -0 leaves on shared roots: MIN/MAX keep the first of equal values in canonical order."""
    f = FORESTS[1]
    sf = sf_for(f)
    bs = 6
    ro, lo = oracle.layout(f)
    sgn = sfgen.rng.u64(1703, 1, int(lo[-1]) * bs) & np.uint64(1)
    leaf = np.where(sgn == 1, -0.0, 0.0)
    for op, low in (("MAX", -1.0), ("MIN", 1.0)):
        root = np.full(int(ro[-1]) * bs, low)
        r = to_dev(root, "fp64")
        sf.reduce(to_dev(leaf, "fp64"), r, op, bs=bs)
        assert_bits_equal(to_host(r, "fp64"), oracle.reduce(f, "fp64", bs, leaf, root, op), f"signed zeros {op}")


# MAX with location (the autograd MAX forward): gather-then-fold for units of 4/8/16-byte
# vectors, the general kernel otherwise; integer data in 0..999 makes ties on most roots, so the
# first maximum in canonical order decides the location
MAXLOC_UNITS = [("fp32", 64), ("bf16", 64), ("fp64", 2), ("int64", 3), ("bf16", 8), ("int32", 5), ("fp32", 1),
                ("bf16", 3)]


def _edge_leaves(f):
    ro, lo = oracle.layout(f)
    return np.concatenate([lo[q] + (np.arange(f.nleaves[q]) if f.ilocal[q] is None else np.asarray(f.ilocal[q]))
                           for q in range(f.nranks)]).astype(np.int64)


@pytest.mark.parametrize("f", FORESTS + [sfgen.zipf_forest(5, 3, 300000, 500, 4)], ids=lambda f: f.name)
@pytest.mark.parametrize("dtype,bs", MAXLOC_UNITS)
def test_maxloc_bit_exact(f, dtype, bs):
    sf = StarForest.from_forest(f).setup() if f.name.startswith("zipf3") else sf_for(f)
    _, leaf = make_data(f, dtype, bs, 1704)
    want_v, want_e = oracle.reduce_maxloc(f, dtype, bs, leaf)
    L = _edge_leaves(f)
    ro, lo = oracle.layout(f)
    root = to_dev(np.zeros(int(ro[-1]) * bs, oracle.NPTYPE[dtype]), dtype)
    arg = torch.full((int(ro[-1]) * bs,), -1, dtype=torch.int32, device="cuda")
    l = to_dev(leaf, dtype)
    for call in range(2):   # the second call finds the arrival counters reset
        sf.reduce_maxloc(l, root, arg, bs=bs)
        assert_bits_equal(to_host(root, dtype), want_v, f"maxloc value {f.name} {dtype}x{bs} call {call}")
        want_leaf = np.where(want_e >= 0, L[np.maximum(want_e, 0)], -1)
        got = arg.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want_leaf), f"maxloc location {f.name} {dtype}x{bs}: " \
            f"{int((got != want_leaf).sum())} differ"
    assert sf.device_status() == 0


def test_maxloc_heavy_star_three_fold_levels():
    n = 300000
    f = sfgen.Forest(1, np.array([3]), np.array([n]), [None], [np.zeros(n, np.int32)],
                     [(np.arange(n) % 7 == 0).astype(np.int64)], name="heavystar")
    sf = StarForest.from_forest(f).setup()
    L = _edge_leaves(f)
    for dtype, bs in (("fp32", 8), ("int32", 4), ("bf16", 16)):
        _, leaf = make_data(f, dtype, bs, 1705)
        want_v, want_e = oracle.reduce_maxloc(f, dtype, bs, leaf)
        root = to_dev(np.zeros(3 * bs, oracle.NPTYPE[dtype]), dtype)
        arg = torch.full((3 * bs,), -1, dtype=torch.int32, device="cuda")
        sf.reduce_maxloc(to_dev(leaf, dtype), root, arg, bs=bs)
        assert_bits_equal(to_host(root, dtype), want_v, f"heavy star maxloc {dtype}x{bs}")
        assert np.array_equal(arg.cpu().numpy().astype(np.int64), np.where(want_e >= 0, L[np.maximum(want_e, 0)], -1))
    assert sf.device_status() == 0


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("dtype,bs", [("fp32", 64), ("bf16", 64), ("fp64", 2), ("int32", 5), ("bf16", 3), ("fp32", 1)])
def test_maxloc_grad_writes_every_connected_leaf(f, dtype, bs):
    """The MAX backward: each connected leaf's unit becomes the root gradient where the oracle's
    location names that leaf and 0 elsewhere; leaves without a root keep what they held."""
    sf = sf_for(f)
    _, leaf = make_data(f, dtype, bs, 1706)
    _, want_e = oracle.reduce_maxloc(f, dtype, bs, leaf)
    L = _edge_leaves(f)
    argleaf = np.where(want_e >= 0, L[np.maximum(want_e, 0)], -1).astype(np.int32)
    ro, lo = oracle.layout(f)
    g = sfgen.data(dtype, int(ro[-1]) * bs, 1706, 3)
    held = sfgen.data(dtype, int(lo[-1]) * bs, 1706, 4)
    want = held.copy().reshape(-1, bs)
    want[L] = 0
    r, c = np.nonzero(argleaf.reshape(-1, bs) >= 0)
    want[argleaf.reshape(-1, bs)[r, c], c] = g.reshape(-1, bs)[r, c]
    out = to_dev(held, dtype)
    sf.maxloc_grad(torch.from_numpy(argleaf).cuda(), to_dev(g, dtype), out, bs=bs)
    assert_bits_equal(to_host(out, dtype), want.ravel(), f"maxloc grad {f.name} {dtype}x{bs}")
