"""Parity at the full workload sizes, in the launch configurations bench.py times (GB300), every
element against the oracle:
  * the SpMV-style scatter: 2^24 roots of a random geometric graph in 256 ranks, fp64 and fp32,
    bs = 1 -- Bcast REPLACE (fused), Reduce SUM deterministic (bit-exact) and atomic (within the
    stated bound);
  * the 3-D halo: 256^3 grid in 4x4x4 ranks, 27-point ghosts, bs = 1 and 5;
  * the batch: 512 uneven forests, Bcast then Reduce each, replayed as one CUDA graph."""
import numpy as np
import pytest

import oracle
import sfgen
from tests.gpu_util import assert_atomic_sum_close, assert_bits_equal, make_data, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import Batch, StarForest  # noqa: E402


@pytest.fixture(scope="module")
def spmv():
    f = sfgen.cfg3_spmv(1 << 24, 8)
    return f, StarForest.from_forest(f).setup()


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_spmv_scatter_full_size(spmv, dtype):
    f, sf = spmv
    root, leaf = make_data(f, dtype, 1, 2400)
    x, lv = to_dev(root, dtype), to_dev(leaf, dtype)
    sf.set_path("fused").bcast(x, lv, "REPLACE")
    want_l = oracle.bcast(f, dtype, 1, root, leaf, "REPLACE")
    assert_bits_equal(to_host(lv, dtype), want_l, f"spmv bcast {dtype}")
    y = to_dev(root, dtype)
    sf.set_mode("deterministic").reduce(lv, y, "SUM")
    want = oracle.reduce(f, dtype, 1, want_l, root, "SUM")
    assert_bits_equal(to_host(y, dtype), want, f"spmv reduce deterministic {dtype}")
    assert sf.device_status() == 0
    y2 = to_dev(root, dtype)
    sf.set_mode("atomic").reduce(lv, y2, "SUM")
    assert_atomic_sum_close(to_host(y2, dtype), want, f, dtype, 1, want_l, root, f"spmv reduce atomic {dtype}")
    sf.set_mode("deterministic")


@pytest.fixture(scope="module")
def halo():
    f = sfgen.cfg2_halo()
    return f, StarForest.from_forest(f).setup()


@pytest.mark.parametrize("bs", [1, 5])
def test_halo_full_size(halo, bs):
    f, sf = halo
    root, leaf = make_data(f, "fp64", bs, 2500)
    x, lv = to_dev(root, "fp64"), to_dev(leaf, "fp64")
    sf.bcast(x, lv, "REPLACE", bs=bs)
    want_l = oracle.bcast(f, "fp64", bs, root, leaf, "REPLACE")
    assert_bits_equal(to_host(lv, "fp64"), want_l, f"halo ghost update bs={bs}")
    del lv
    lv = to_dev(leaf, "fp64")
    y = to_dev(root, "fp64")
    sf.set_mode("deterministic").reduce(lv, y, "SUM", bs=bs)
    want = oracle.reduce(f, "fp64", bs, leaf, root, "SUM")
    assert_bits_equal(to_host(y, "fp64"), want, f"halo ghost accumulate bs={bs}")
    assert sf.device_status() == 0
    y.copy_(x)
    sf.set_mode("atomic").reduce(lv, y, "SUM", bs=bs)
    assert_atomic_sum_close(to_host(y, "fp64"), want, f, "fp64", bs, leaf, root, f"halo atomic bs={bs}")
    sf.set_mode("deterministic")


def test_batched_512_forests_full_size():
    forests = sfgen.cfg4_batched(nforests=512)
    items = []
    for i, f in enumerate(forests):
        dt, bs, op = f.meta["dtype"], f.meta["bs"], f.meta["op"]
        sf = StarForest.from_forest(f).setup().set_mode("deterministic")
        root, leaf = make_data(f, dt, bs, 3000 + i)
        items.append(dict(f=f, sf=sf, dt=dt, bs=bs, op=op, root=root, leaf=leaf,
                          r=to_dev(root, dt), l=to_dev(leaf, dt), r2=to_dev(root, dt), l2=to_dev(leaf, dt)))
    ops = [("bcast", it["sf"], it["op"], it["r"], it["l"], it["bs"]) for it in items] + ["barrier"] + \
          [("reduce", it["sf"], it["op"], it["l2"], it["r2"], it["bs"]) for it in items]
    Batch().set_ops(ops).run(use_graph=True)
    torch.cuda.synchronize()
    for it in items:
        f, dt, bs, op = it["f"], it["dt"], it["bs"], it["op"]
        assert_bits_equal(to_host(it["l"], dt), oracle.bcast(f, dt, bs, it["root"], it["leaf"], op),
                          f"batch bcast {f.name} {op} {dt}x{bs}")
        assert_bits_equal(to_host(it["r2"], dt), oracle.reduce(f, dt, bs, it["leaf"], it["root"], op),
                          f"batch reduce {f.name} {op} {dt}x{bs}")
        assert it["sf"].device_status() == 0
