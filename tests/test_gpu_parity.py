"""CUDA path vs oracle, element by element, through the C ABI (GB300)."""
import numpy as np
import pytest

import oracle
import sfgen
from tests.gpu_util import (assert_atomic_sum_close, assert_bits_equal, make_data, signed_zero_data,
                            signed_zero_forest, to_dev, to_host)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import StarForest, SFError, launch_count  # noqa: E402


def small_forests():
    fs = [sfgen.fig2(), sfgen.cfg1_plain_tiny(), sfgen.cfg2_halo(64, 4), sfgen.cfg3_spmv(1 << 15, 4),
          sfgen.zipf_forest(77, 1, 20000, 3000, 4)]
    fs += [sfgen.random_forest(s, P, 300, 400) for s, P in [(41, 1), (42, 3), (43, 8)]]
    fs.append(sfgen.Forest(2, np.array([5, 0]), np.array([0, 0]), [None, None],
                           [np.zeros(0, np.int32)] * 2, [np.zeros(0, np.int64)] * 2, name="empty"))
    return fs


FORESTS = small_forests()
_SF = {}


def sf_for(f):
    if f.name not in _SF:
        _SF[f.name] = StarForest.from_forest(f).setup()
    return _SF[f.name]


DT = ["int32", "int64", "fp32", "fp64", "bf16"]


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("path", ["fused", "three_phase", "root_major"])
@pytest.mark.parametrize("op", ["REPLACE", "SUM", "MAX"])
@pytest.mark.parametrize("dtype,bs", [("fp64", 1), ("int32", 1), ("fp32", 3), ("bf16", 8), ("int64", 2),
                                      ("fp32", 2), ("bf16", 3)])
def test_bcast_bit_exact(f, path, op, dtype, bs):
    sf = sf_for(f).set_path(path)
    root, leaf = make_data(f, dtype, bs, 100)
    want = oracle.bcast(f, dtype, bs, root, leaf, op)
    r, l = to_dev(root, dtype), to_dev(leaf, dtype)
    sf.bcast(r, l, op, bs=bs)
    assert_bits_equal(to_host(l, dtype), want, f"bcast {f.name} {path} {op} {dtype}x{bs}")
    assert_bits_equal(to_host(r, dtype), root, "rootdata must be untouched")


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["REPLACE", "SUM", "MIN", "MAX"])
@pytest.mark.parametrize("dtype", DT)
def test_reduce_deterministic_bit_exact(f, op, dtype):
    sf = sf_for(f).set_mode("deterministic")
    # integers also over their full range, so SUM wraps around (two's complement)
    kinds = ("signed", "wide") if dtype.startswith("int") else ("signed",)
    for bs in (1, 5):
        for kind in kinds:
            root, leaf = make_data(f, dtype, bs, 200, kind, kind)
            want = oracle.reduce(f, dtype, bs, leaf, root, op)
            r, l = to_dev(root, dtype), to_dev(leaf, dtype)
            sf.reduce(l, r, op, bs=bs)
            assert_bits_equal(to_host(r, dtype), want, f"reduce det {f.name} {op} {dtype}x{bs} {kind}")
            assert_bits_equal(to_host(l, dtype), leaf, "leafdata must be untouched")
    assert sf.device_status() == 0


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["SUM", "MIN", "MAX"])
@pytest.mark.parametrize("dtype", ["int32", "int64", "fp32", "fp64"])
def test_reduce_atomic(f, op, dtype):
    bs = 2
    kind = "wide" if dtype.startswith("int") else "signed"   # integer SUM wraps around
    root, leaf = make_data(f, dtype, bs, 300, kind, kind)
    want = oracle.reduce(f, dtype, bs, leaf, root, op)
    r, l = to_dev(root, dtype), to_dev(leaf, dtype)
    sf = sf_for(f).set_mode("atomic")
    sf.reduce(l, r, op, bs=bs)
    got = to_host(r, dtype)
    sf.set_mode("deterministic")
    if op == "SUM" and dtype.startswith("fp"):
        assert_atomic_sum_close(got, want, f, dtype, bs, leaf, root, f"reduce atomic {f.name} {dtype}")
    else:
        assert_bits_equal(got, want, f"reduce atomic {f.name} {op} {dtype}")


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("op", ["SUM", "MAX", "REPLACE"])
@pytest.mark.parametrize("dtype,bs", [("int32", 1), ("fp64", 1), ("fp32", 4), ("int64", 3)])
def test_fetch_and_op_deterministic_bit_exact(f, op, dtype, bs):
    sf = sf_for(f).set_mode("deterministic")
    kind = "wide" if dtype.startswith("int") else "signed"   # integer SUM wraps around
    root, leaf = make_data(f, dtype, bs, 400, kind, kind)
    upd0 = sfgen.data(dtype, leaf.size, 400, 3)
    want_root, want_upd = oracle.fetch_and_op(f, dtype, bs, root, leaf, upd0, op)
    r, l, u = to_dev(root, dtype), to_dev(leaf, dtype), to_dev(upd0, dtype)
    sf.fetch_and_op(r, l, u, op, bs=bs)
    assert_bits_equal(to_host(r, dtype), want_root, f"fetch root {f.name} {op}")
    assert_bits_equal(to_host(u, dtype), want_upd, f"fetch leafupdate {f.name} {op}")


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("dtype", ["int32", "int64", "fp64"])
def test_fetch_and_op_atomic_multisf(f, dtype):
    """Atomic order is the hardware's: check the multi-SF invariant (Sec. III.B) and that the
    fetched values of each root are its running sums in some order of its leaves."""
    sf = sf_for(f).set_mode("atomic")
    ro, lo = oracle.layout(f)
    deg = oracle.in_degree(f)
    npt = oracle.NPTYPE[dtype]
    off = np.concatenate([[0], np.cumsum(deg)[:-1]]).astype(npt)
    ones = np.ones(lo[-1], npt)
    r, l, u = to_dev(off, dtype), to_dev(ones, dtype), to_dev(np.full(lo[-1], -1, npt), dtype)
    sf.fetch_and_op(r, l, u, "SUM", bs=1)
    sf.set_mode("deterministic")
    assert np.array_equal(to_host(r, dtype), off + deg)
    got_upd = to_host(u, dtype)
    from tests import npref
    L, R = npref.edge_arrays(f)
    for root in np.unique(R)[:2000]:
        fetched = np.sort(got_upd[L[R == root]])
        assert np.array_equal(fetched, off[root] + np.arange(deg[root])), root


def degree_ladder(nroots=3000, nranks=3, seed=91):
    """Root r has in-degree (r % 70) + 1: fold blocks of every length 1..64 plus two-block
    roots, starting at every offset of a 32-leaf warp step; leaves spread over the ranks in
    random order."""
    deg = (np.arange(nroots) % 70) + 1
    owner = np.repeat(np.arange(nroots), deg)
    perm = np.argsort(sfgen.rng.u64(seed, 1, owner.size), kind="stable")
    owner = owner[perm]
    per = -(-nroots // nranks)
    cuts = np.linspace(0, owner.size, nranks + 1).astype(int)
    rr = [(owner[cuts[q]:cuts[q + 1]] // per).astype(np.int32) for q in range(nranks)]
    ri = [(owner[cuts[q]:cuts[q + 1]] % per).astype(np.int64) for q in range(nranks)]
    roots = np.array([min(per, nroots - p * per) for p in range(nranks)])
    return sfgen.Forest(nranks, roots, np.diff(cuts), [None] * nranks, rr, ri, name="degree_ladder")


LADDER = degree_ladder()


@pytest.mark.parametrize("op", ["SUM", "MIN", "MAX"])
@pytest.mark.parametrize("dtype", DT)
def test_reduce_degree_ladder_bit_exact(op, dtype):
    sf = sf_for(LADDER).set_mode("deterministic")
    for bs in (1, 2):
        root, leaf = make_data(LADDER, dtype, bs, 260)
        r, l = to_dev(root, dtype), to_dev(leaf, dtype)
        for _ in range(2):          # the second call reuses reset arrival counters
            r.copy_(to_dev(root, dtype))
            sf.reduce(l, r, op, bs=bs)
            assert_bits_equal(to_host(r, dtype), oracle.reduce(LADDER, dtype, bs, leaf, root, op),
                              f"degree ladder {op} {dtype}x{bs}")
    assert sf.device_status() == 0


def test_reduce_heavy_root_recursive_fold():
    """A star of 300,000 leaves: 4688 blocks -> 74 -> 2 -> 1, three fold levels."""
    n = 300000
    f = sfgen.Forest(1, np.array([3]), np.array([n]), [None], [np.zeros(n, np.int32)],
                     [(np.arange(n) % 7 == 0).astype(np.int64)], name="heavystar")
    sf = StarForest.from_forest(f).setup()
    for dtype in ("fp32", "fp64", "bf16"):
        root, leaf = make_data(f, dtype, 1, 500)
        want = oracle.reduce(f, dtype, 1, leaf, root, "SUM")
        r, l = to_dev(root, dtype), to_dev(leaf, dtype)
        for _ in range(2):      # second call: the arrival counters must have been reset
            r.copy_(to_dev(root, dtype))
            sf.reduce(l, r, "SUM")
            assert_bits_equal(to_host(r, dtype), want, f"heavy star {dtype}")
    assert sf.device_status() == 0


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_memtype_host_buffers(dtype):
    f = sfgen.cfg1_plain_tiny()
    sf = sf_for(f)
    root, leaf = make_data(f, dtype, 1, 600)
    want_b = oracle.bcast(f, dtype, 1, root, leaf, "REPLACE")
    want_r = oracle.reduce(f, dtype, 1, leaf, root, "SUM")
    rh = torch.from_numpy(root.copy()).pin_memory()
    lh = torch.from_numpy(leaf.copy()).pin_memory()
    sf.bcast_memtype(rh, lh, "REPLACE")
    torch.cuda.synchronize()
    assert_bits_equal(lh.numpy(), want_b, "bcast host")
    lh2 = torch.from_numpy(leaf.copy()).pin_memory()
    rh2 = torch.from_numpy(root.copy()).pin_memory()
    sf.set_mode("deterministic")
    sf.reduce_memtype(lh2, rh2, "SUM")
    torch.cuda.synchronize()
    assert_bits_equal(rh2.numpy(), want_r, "reduce host")


def test_begin_end_protocol_errors():
    f = sfgen.cfg1_plain_tiny()
    sf = sf_for(f).set_path("three_phase")
    root, leaf = make_data(f, "fp64", 1, 700)
    r, l = to_dev(root, "fp64"), to_dev(leaf, "fp64")
    sf.bcast_begin(r, l, "REPLACE")
    with pytest.raises(SFError) as e:
        sf.bcast_begin(r, l, "REPLACE")
    assert e.value.name == "SF_ERR_PENDING"
    with pytest.raises(SFError) as e:
        sf.destroy()
    assert e.value.name == "SF_ERR_PENDING"
    # independent work between begin and end, then end completes the unpack
    x = torch.ones(1000, device="cuda") * 2
    sf.bcast_end(r, l, "REPLACE")
    assert_bits_equal(to_host(l, "fp64"), oracle.bcast(f, "fp64", 1, root, leaf, "REPLACE"), "three-phase end")
    with pytest.raises(SFError) as e:
        sf.bcast_end(r, l, "REPLACE")
    assert e.value.name == "SF_ERR_NO_PENDING"
    sf.set_path("fused")
    # two concurrent operations on one forest with different data (Sec. III.A)
    l2 = to_dev(leaf, "fp64")
    sf.bcast_begin(r, l, "REPLACE")
    sf.bcast_begin(r, l2, "REPLACE")
    sf.bcast_end(r, l2, "REPLACE")
    sf.bcast_end(r, l, "REPLACE")
    assert float(x.sum()) == 2000.0


def test_misaligned_pointer_rejected():
    f = sfgen.cfg1_plain_tiny()
    sf = sf_for(f)
    buf = torch.zeros(20000 * 8 + 1, dtype=torch.uint8, device="cuda")
    lib = sf._lib
    from paper_2102_13018_gb300 import _abi
    import ctypes
    u = _abi.sf_unit(_abi.SF_FP64, 1)
    p = ctypes.c_void_p(buf.data_ptr() + 1)
    assert lib.sf_bcast_begin(sf._h, u, p, p, 0, None) == _abi.CODES["SF_ERR_ALIGN"]


@pytest.mark.parametrize("dtype,bs", [("fp64", 1 << 16), ("bf16", 1 << 18)])
def test_largest_unit_matches_oracle(dtype, bs):
    """Units of exactly 512 KiB (the documented maximum): Bcast REPLACE and deterministic
    Reduce SUM over every vector of the unit."""
    f = sfgen.fig2()
    sf = sf_for(f).set_mode("deterministic")
    root, leaf = make_data(f, dtype, bs, 810)
    r, l = to_dev(root, dtype), to_dev(leaf, dtype)
    sf.bcast(r, l, "REPLACE", bs=bs)
    assert_bits_equal(to_host(l, dtype), oracle.bcast(f, dtype, bs, root, leaf, "REPLACE"), "bcast max unit")
    l2 = to_dev(leaf, dtype)
    sf.reduce(l2, r, "SUM", bs=bs)
    assert_bits_equal(to_host(r, dtype), oracle.reduce(f, dtype, bs, leaf, root, "SUM"), "reduce max unit")


def test_unit_above_the_limit_is_rejected():
    f = sfgen.fig2()
    sf = sf_for(f)
    bs = (1 << 16) + 1                      # fp64: 512 KiB + 8 bytes
    r = torch.zeros(9 * bs, dtype=torch.float64, device="cuda")
    l = torch.zeros(11 * bs, dtype=torch.float64, device="cuda")
    with pytest.raises(SFError) as e:
        sf.bcast(r, l, "REPLACE", bs=bs)
    assert e.value.name == "SF_ERR_ARG"


def test_launch_counter_advances():
    f = sfgen.fig2()
    sf = sf_for(f)
    root, leaf = make_data(f, "fp64", 1, 800)
    n0 = launch_count()
    sf.bcast(to_dev(root, "fp64"), to_dev(leaf, "fp64"))
    assert launch_count() > n0


@pytest.mark.parametrize("nbytes", [1 << 10, 1 << 16, 1 << 22])
def test_pingpong_round_trip_restores_roots(nbytes):
    """Sec. VI.A: Bcast REPLACE to rank 1, Reduce REPLACE back; the contiguous pattern on both
    sides means no index array is read."""
    n = nbytes // 8
    f = sfgen.pingpong(n)
    sf = StarForest.from_forest(f).setup()
    info = sf.info()
    assert info["edges_both_pattern"] == n
    x0 = torch.rand(n, dtype=torch.float64, device="cuda")
    x = x0.clone()
    lv = torch.zeros(n, dtype=torch.float64, device="cuda")
    for _ in range(3):
        sf.bcast(x, lv, "REPLACE")
        x.zero_()
        sf.reduce(lv, x, "REPLACE")
    assert torch.equal(x, x0)


SZ = signed_zero_forest()


@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
@pytest.mark.parametrize("op", ["MIN", "MAX"])
@pytest.mark.parametrize("bs", [1, 3])
def test_min_max_signed_zero_ties_bit_exact(dtype, op, bs):
    """Deterministic MIN/MAX must keep the first of equal values in canonical order, as the
    oracle does: +0 and -0 compare equal but differ in their bits."""
    sf = sf_for(SZ).set_mode("deterministic")
    root, leaf = signed_zero_data(SZ, dtype, bs, 94)
    if op == "MIN":
        root = np.where(root == -1.0, -root, root).astype(root.dtype)
    want = oracle.reduce(SZ, dtype, bs, leaf, root, op)
    assert np.signbit(want).any() and (~np.signbit(want)).any()
    r, l = to_dev(root, dtype), to_dev(leaf, dtype)
    sf.reduce(l, r, op, bs=bs)
    assert_bits_equal(to_host(r, dtype), want, f"signed zeros {op} {dtype}x{bs}")
    assert sf.device_status() == 0


def _small_ladder():
    f = degree_ladder(500, 2, 97)
    f.name = "degree_ladder_500"
    return f


FROM_ZERO_FORESTS = FORESTS + [sfgen.owned_plus_ghosts(5), _small_ladder()]


@pytest.mark.parametrize("f", FROM_ZERO_FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("mode", ["deterministic", "atomic"])
@pytest.mark.parametrize("op", ["REPLACE", "SUM", "MIN", "MAX"])
def test_reduce_from_zero_equals_reduce_into_zeros(f, mode, op):
    """sf_reduce_from_zero = a Reduce into roots that were all zero, without reading them:
    the root buffer starts as NaN garbage (all-ones bits for integers) here."""
    sf = sf_for(f).set_mode(mode)
    ro, lo = oracle.layout(f)
    for dtype, bs in (("fp64", 1), ("fp32", 4), ("bf16", 8), ("int32", 1), ("fp32", 64)):
        _, leaf = make_data(f, dtype, bs, 700)
        zeros = np.zeros(int(ro[-1]) * bs, oracle.NPTYPE[dtype])
        want = oracle.reduce(f, dtype, bs, leaf, zeros, op)
        garbage = np.full(int(ro[-1]) * bs, 0xFFFF if dtype == "bf16" else -1, oracle.NPTYPE[dtype])
        if dtype in ("fp32", "fp64"):
            garbage[:] = np.nan
        r = to_dev(garbage, dtype)
        sf.reduce_from_zero(to_dev(leaf, dtype), r, op, bs=bs)
        got = to_host(r, dtype)
        if mode == "atomic" and op == "SUM" and dtype in ("fp32", "fp64"):
            assert_atomic_sum_close(got, want, f, dtype, bs, leaf, zeros, f"from zero {f.name} {op}")
        else:
            assert_bits_equal(got, want, f"from zero {f.name} {mode} {op} {dtype}x{bs}")
    sf.set_mode("deterministic")
    assert sf.device_status() == 0


@pytest.mark.parametrize("f", [sfgen.random_forest(44, 4, 300, 200), sfgen.owned_plus_ghosts(6, keep=0.6)],
                         ids=lambda f: f.name)
def test_zero_leafless_roots(f):
    sf = sf_for(f)
    ro, _ = oracle.layout(f)
    deg = oracle.in_degree(f)
    bs = 3
    root = sfgen.data("fp32", int(ro[-1]) * bs, 710, 1)
    arg = np.arange(int(ro[-1]) * bs, dtype=np.int32)
    r, a = to_dev(root, "fp32"), torch.from_numpy(arg.copy()).cuda()
    sf.zero_leafless_roots(r, a, bs=bs)
    empty = np.repeat(deg == 0, bs)
    assert empty.any() and (~empty).any()
    assert_bits_equal(to_host(r, "fp32"), np.where(empty, np.float32(0), root), "leafless roots zeroed")
    assert np.array_equal(a.cpu().numpy(), np.where(empty, -1, arg))
