"""The deterministic Reduce over diagonal chunks -- the root-streaming plan for forests whose
roots own a leaf at a fixed offset (the SpMV scatter of Sec. IV.A) -- and the root-major plan
of the roots it leaves out, against the oracle, bit for bit (GB300)."""
import numpy as np
import pytest

import oracle
import sfgen
from tests.gpu_util import assert_bits_equal, make_data, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import Batch, StarForest  # noqa: E402

FORESTS = [sfgen.owned_plus_ghosts(5), sfgen.owned_plus_ghosts(6, keep=0.6),
           sfgen.owned_plus_ghosts(7, nroots=(33, 4096, 1, 500), ghosts_per_rank=3000, heavy=1, shuffled_rank=3),
           sfgen.cfg3_spmv(1 << 15, 4)]
_SF = {}


PLANS = ["diagonal", "diagonal_staged"]


def sf_for(f, plan="diagonal"):
    if f.name not in _SF:
        sf = StarForest.from_forest(f).setup().set_mode("deterministic")
        assert sf.info()["dg_chunks"] > 0
        assert sf.tuning()["reduce_plan"] == "root_major"   # the default
        _SF[f.name] = sf
    return _SF[f.name].set_reduce_plan(plan)


# one vector per unit: bs = 1, or 16-byte units
UNITS = [("fp64", 1), ("fp32", 1), ("bf16", 1), ("int32", 1), ("int64", 1),
         ("fp64", 2), ("fp32", 4), ("bf16", 8), ("int32", 4), ("int64", 2)]


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["SUM", "MIN", "MAX"])
@pytest.mark.parametrize("dtype,bs", UNITS)
def test_diagonal_chunk_reduce_bit_exact(f, op, dtype, bs, plan):
    sf = sf_for(f, plan)
    assert sf.tuning()["reduce_plan"] == plan
    kind = "wide" if dtype.startswith("int") else "signed"
    root, leaf = make_data(f, dtype, bs, 1500, kind, kind)
    want = oracle.reduce(f, dtype, bs, leaf, root, op)
    l = to_dev(leaf, dtype)
    for call in range(2):
        r = to_dev(root, dtype)
        sf.reduce(l, r, op, bs=bs)
        assert_bits_equal(to_host(r, dtype), want, f"diag reduce {plan} {f.name} {op} {dtype}x{bs} call {call}")
    assert_bits_equal(to_host(l, dtype), leaf, "leafdata must be untouched")
    assert sf.device_status() == 0


@pytest.mark.parametrize("op", ["SUM", "MAX"])
def test_plans_agree_and_tuner_keeps_the_bits(op):
    """Every plan gives the same bits; the tuner may pick any of them and still does."""
    f = FORESTS[3]
    sf = sf_for(f, "auto")
    root, leaf = make_data(f, "fp64", 1, 1520, "signed", "signed")
    want = oracle.reduce(f, "fp64", 1, leaf, root, op)
    l = to_dev(leaf, "fp64")
    for plan in ["root_major"] + PLANS:
        r = to_dev(root, "fp64")
        sf.set_reduce_plan(plan).reduce(l, r, op)
        assert_bits_equal(to_host(r, "fp64"), want, f"plan {plan} {op}")
    sf.set_reduce_plan("auto")
    choice = sf.autotune("reduce", l, to_dev(root, "fp64"), op, reps=2)
    assert choice == "deterministic"
    assert sf.tuning()["reduce_plan"] in ["root_major"] + PLANS
    r = to_dev(root, "fp64")
    sf.reduce(l, r, op)
    assert_bits_equal(to_host(r, "fp64"), want, f"tuned plan {sf.tuning()['reduce_plan']} {op}")
    sf.set_reduce_plan("diagonal")


@pytest.mark.parametrize("dtype,bs", [("fp64", 3), ("bf16", 2), ("int32", 1)])
def test_other_units_and_replace_keep_the_root_major_plan(dtype, bs):
    """Units of several vectors, and REPLACE, run the root-major plan of every root."""
    f = FORESTS[0]
    sf = sf_for(f, "diagonal_staged")
    for op in ("REPLACE", "SUM", "MAX"):
        root, leaf = make_data(f, dtype, bs, 1501)
        r, l = to_dev(root, dtype), to_dev(leaf, dtype)
        sf.reduce(l, r, op, bs=bs)
        assert_bits_equal(to_host(r, dtype), oracle.reduce(f, dtype, bs, leaf, root, op), f"{op} {dtype}x{bs}")


@pytest.mark.parametrize("plan", PLANS)
def test_signed_zero_ties_on_diagonal_chunks(plan):
    """Two- and three-leaf roots of +0 / -0 leaves: the diagonal leaf keeps its canonical place."""
    f = FORESTS[0]
    sf = sf_for(f, plan)
    ro, lo = oracle.layout(f)
    sgn = sfgen.rng.u64(1502, 1, int(lo[-1])) & np.uint64(1)
    leaf = np.where(sgn == 1, -0.0, 0.0)
    pick = sfgen.rng.u64(1502, 2, int(ro[-1])) % np.uint64(3)
    for op, low in (("MAX", -1.0), ("MIN", 1.0)):
        root = np.choose(pick.astype(np.int64), [low, 0.0, -0.0])
        want = oracle.reduce(f, "fp64", 1, leaf, root, op)
        r = to_dev(root, "fp64")
        sf.reduce(to_dev(leaf, "fp64"), r, op)
        assert_bits_equal(to_host(r, "fp64"), want, f"signed zeros {op}")


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_of_diagonal_chunk_forests(use_graph):
    items = []
    for i, (f, (dtype, bs), op) in enumerate(zip(FORESTS, [("fp64", 1), ("fp32", 4), ("bf16", 1), ("int64", 1)],
                                                 ["SUM", "MAX", "SUM", "MIN"])):
        root, leaf = make_data(f, dtype, bs, 1510 + i)
        items.append((f, sf_for(f), dtype, bs, op, root, leaf, to_dev(root, dtype), to_dev(leaf, dtype)))
    b = Batch().set_ops([("reduce", sf, op, l, r, bs) for f, sf, dtype, bs, op, root, leaf, r, l in items])
    for run in range(2):
        for f, sf, dtype, bs, op, root, leaf, r, l in items:
            r.copy_(to_dev(root, dtype))
        b.run(use_graph=use_graph)
        torch.cuda.synchronize()
        for f, sf, dtype, bs, op, root, leaf, r, l in items:
            assert_bits_equal(to_host(r, dtype), oracle.reduce(f, dtype, bs, leaf, root, op),
                              f"batch {f.name} {op} {dtype}x{bs} run {run}")


def negative_offset_forest():
    """Rank 0 has roots but no leaves; rank 1 lists its owned leaves first (leaf i -> root (1, i)),
    so the diagonal leaf sits 5000 units below its root, then ghosts of rank 0's roots."""
    n0, n1, g = 5000, 7001, 3000
    ghost = sfgen.rng.randint(1600, 1, g, 0, n0)
    return sfgen.Forest(2, np.array([n0, n1]), np.array([0, n1 + g]), [None, None],
                        [np.zeros(0, np.int32), np.concatenate([np.ones(n1), np.zeros(g)]).astype(np.int32)],
                        [np.zeros(0, np.int64), np.concatenate([np.arange(n1), ghost]).astype(np.int64)],
                        name="negative_offset")


@pytest.mark.parametrize("plan", PLANS)
@pytest.mark.parametrize("dtype,bs", [("fp64", 1), ("fp32", 1), ("bf16", 1), ("fp64", 2), ("int64", 1)])
def test_negative_offset_and_unaligned_buffers(dtype, bs, plan):
    """A negative diagonal offset, and buffers that are not 16-byte aligned (one element into a
    larger allocation: the staged plan then reads with plain loads instead of bulk copies), give the
    oracle's bits; so does the Reduce from zero."""
    f = negative_offset_forest()
    sf = StarForest.from_forest(f).setup().set_mode("deterministic").set_reduce_plan(plan)
    info = sf.info()
    assert info["dg_chunks"] > 0 and info["dg_rest_roots"] > 0
    root, leaf = make_data(f, dtype, bs, 1601)
    for op in ("SUM", "MAX"):
        want = oracle.reduce(f, dtype, bs, leaf, root, op)
        for shift in (0, 1):
            rb = to_dev(np.concatenate([root[:1], root]), dtype)[1:] if shift else to_dev(root, dtype)
            lb = to_dev(np.concatenate([leaf[:1], leaf]), dtype)[1:] if shift else to_dev(leaf, dtype)
            sf.reduce(lb, rb, op, bs=bs)
            assert_bits_equal(to_host(rb, dtype), want, f"negative offset {op} {dtype}x{bs} shift {shift}")
        zeros = np.zeros_like(root)
        r = to_dev(np.full_like(root, 0xFF if dtype == "bf16" else 7), dtype)
        sf.reduce_from_zero(to_dev(leaf, dtype), r, op, bs=bs)
        assert_bits_equal(to_host(r, dtype), oracle.reduce(f, dtype, bs, leaf, zeros, op), f"from zero {op}")
    assert sf.device_status() == 0
