"""Batched execution and the autotuner vs the oracle and vs one call per forest (GB300)."""
import numpy as np
import pytest

import oracle
import sfgen
from tests.gpu_util import assert_atomic_sum_close, assert_bits_equal, make_data, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import Batch, SFError, StarForest, launch_count  # noqa: E402

FORESTS = sfgen.cfg4_batched(nforests=24, lo=1e2, hi=2e4)


def build(forests, modes=None):
    items = []
    for i, f in enumerate(forests):
        dt, bs, op = f.meta["dtype"], f.meta["bs"], f.meta["op"]
        sf = StarForest.from_forest(f).setup()
        if modes is not None:
            sf.set_mode(modes[i % len(modes)])
        else:
            sf.set_mode("deterministic")
        root, leaf = make_data(f, dt, bs, 1000 + i)
        items.append(dict(f=f, sf=sf, dt=dt, bs=bs, op=op, root=root, leaf=leaf))
    return items


def ops_for(items):
    bc = [("bcast", it["sf"], it["op"], it["r"], it["l"], it["bs"]) for it in items]
    rd = [("reduce", it["sf"], it["op"], it["l2"], it["r2"], it["bs"]) for it in items]
    return bc + ["barrier"] + rd


def fresh(items):
    for it in items:
        it["r"], it["l"] = to_dev(it["root"], it["dt"]), to_dev(it["leaf"], it["dt"])
        it["r2"], it["l2"] = to_dev(it["root"], it["dt"]), to_dev(it["leaf"], it["dt"])


def check(items, atomic=False):
    for it in items:
        f, dt, bs, op = it["f"], it["dt"], it["bs"], it["op"]
        want_l = oracle.bcast(f, dt, bs, it["root"], it["leaf"], op)
        assert_bits_equal(to_host(it["l"], dt), want_l, f"batch bcast {f.name} {op} {dt}x{bs}")
        want_r = oracle.reduce(f, dt, bs, it["leaf"], it["root"], op)
        got = to_host(it["r2"], dt)
        if atomic and op == "SUM" and dt.startswith("fp"):
            assert_atomic_sum_close(got, want_r, f, dt, bs, it["leaf"], it["root"], f"batch reduce {f.name}")
        else:
            assert_bits_equal(got, want_r, f"batch reduce {f.name} {op} {dt}x{bs}")


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(use_graph):
    items = build(FORESTS)
    fresh(items)
    b = Batch().set_ops(ops_for(items))
    n0 = launch_count()
    b.run(use_graph=use_graph)
    torch.cuda.synchronize()
    check(items)
    assert 0 < b.launches() < 2 * len(items)       # 2 operations per forest, grouped by variant
    assert launch_count() - n0 == b.launches()
    # a second run with the same list reuses the tables (and the graph): reset data first
    for it in items:
        it["r"].copy_(to_dev(it["root"], it["dt"]))
        it["l"].copy_(to_dev(it["leaf"], it["dt"]))
        it["r2"].copy_(to_dev(it["root"], it["dt"]))
        it["l2"].copy_(to_dev(it["leaf"], it["dt"]))
    b.run(use_graph=use_graph)
    torch.cuda.synchronize()
    check(items)


def test_batch_atomic_and_root_major_mix():
    items = build(FORESTS[:12], modes=["atomic", "deterministic"])
    for i, it in enumerate(items):
        it["sf"].set_path("root_major" if i % 3 == 0 else "fused")
    fresh(items)
    Batch().set_ops(ops_for(items)).run(use_graph=True)
    torch.cuda.synchronize()
    check(items, atomic=True)


def test_batch_equals_one_call_per_forest():
    items = build(FORESTS[:10])
    fresh(items)
    Batch().set_ops(ops_for(items)).run()
    torch.cuda.synchronize()
    for it in items:
        r, l = to_dev(it["root"], it["dt"]), to_dev(it["leaf"], it["dt"])
        it["sf"].bcast(r, l, it["op"], bs=it["bs"])
        l2 = to_dev(it["leaf"], it["dt"])
        it["sf"].reduce(l2, r, it["op"], bs=it["bs"])
        want_root = it["root"].copy()
        want = oracle.reduce(it["f"], it["dt"], it["bs"], it["leaf"], want_root, it["op"])
        assert_bits_equal(to_host(r, it["dt"]), want, "per-forest reduce")
        assert_bits_equal(to_host(it["r2"], it["dt"]), to_host(r, it["dt"]), "batch == per-forest")


def test_batch_errors():
    items = build(FORESTS[:2])
    fresh(items)
    it = items[0]
    b = Batch()
    b.set_ops([("reduce", it["sf"], it["op"], it["l2"], it["r2"], it["bs"])])
    b._ops[0].sf = None
    with pytest.raises(SFError) as e:
        b.run()
    assert e.value.name == "SF_ERR_NULL"


@pytest.mark.parametrize("kind", ["bcast", "reduce"])
def test_autotune_choice_is_valid_and_auto_stays_correct(kind):
    f = sfgen.cfg3_spmv(1 << 15, 4)
    sf = StarForest.from_forest(f).setup()
    root, leaf = make_data(f, "fp64", 1, 1100)
    r, l = to_dev(root, "fp64"), to_dev(leaf, "fp64")
    if kind == "bcast":
        choice = sf.autotune("bcast", r, l, "REPLACE")
        assert choice in ("fused", "root_major", "three_phase")
        assert_bits_equal(to_host(l, "fp64"), leaf, "autotune leaves dst untouched")
        sf.set_path("auto").bcast(r, l, "REPLACE")
        assert_bits_equal(to_host(l, "fp64"), oracle.bcast(f, "fp64", 1, root, leaf, "REPLACE"), "auto bcast")
    else:
        choice = sf.autotune("reduce", l, r, "SUM")
        assert choice in ("deterministic", "atomic")
        assert_bits_equal(to_host(r, "fp64"), root, "autotune leaves dst untouched")
        sf.set_mode("auto").reduce(l, r, "SUM")
        want = oracle.reduce(f, "fp64", 1, leaf, root, "SUM")
        assert_atomic_sum_close(to_host(r, "fp64"), want, f, "fp64", 1, leaf, root, "auto reduce")


def test_batch_rebuilds_after_a_forest_scratch_grows():
    """A batch keeps device tables that point at each forest's fold scratch.  A later single
    Reduce with a wider unit grows (reallocates) that scratch; the next batch run must notice
    and rebuild, in both the plain and the graph form, and still match the oracle."""
    f = sfgen.zipf_forest(31, 2, 40000, 500, 3)      # heavy roots: multi-block folds use the scratch
    sf = StarForest.from_forest(f).setup().set_mode("deterministic")
    assert sf.info()["rm_chunks"] > sf.info()["multi_roots"]
    root, leaf = make_data(f, "fp32", 1, 1200)
    wroot, wleaf = make_data(f, "fp64", 8, 1201)
    for use_graph in (False, True):
        r, l = to_dev(root, "fp32"), to_dev(leaf, "fp32")
        b = Batch().set_ops([("reduce", sf, "SUM", l, r, 1)])
        b.run(use_graph=use_graph)
        torch.cuda.synchronize()
        want = oracle.reduce(f, "fp32", 1, leaf, root, "SUM")
        assert_bits_equal(to_host(r, "fp32"), want, "first batch run")
        wr, wl = to_dev(wroot, "fp64"), to_dev(wleaf, "fp64")
        sf.reduce(wl, wr, "SUM", bs=8)           # 64-byte units: the scratch is reallocated
        torch.cuda.synchronize()
        assert_bits_equal(to_host(wr, "fp64"), oracle.reduce(f, "fp64", 8, wleaf, wroot, "SUM"), "wide reduce")
        r.copy_(to_dev(root, "fp32"))
        b.run(use_graph=use_graph)
        torch.cuda.synchronize()
        assert_bits_equal(to_host(r, "fp32"), want, f"batch run after the scratch moved (graph={use_graph})")
    assert sf.device_status() == 0


@pytest.mark.parametrize("edges", [64, 512, 4096, 0])
@pytest.mark.parametrize("vec", [4, 0])
def test_tile_edges_and_vector_bytes_keep_results(edges, vec):
    """The launch-shape knobs the tuner turns change no result: Bcast and the deterministic and
    atomic Reduce against the oracle for every tile size and vector cap."""
    f = sfgen.zipf_forest(33, 3, 20000, 6000, 4)
    sf = StarForest.from_forest(f).setup().set_tile_edges(edges).set_vector_bytes(vec)
    t = sf.tuning()
    assert t["vector_bytes"] == vec and t["tile_edges"] == (edges or sf.info()["ts_tile_edges"])
    for dtype, bs in (("fp64", 2), ("fp32", 8), ("int64", 3)):
        root, leaf = make_data(f, dtype, bs, 1220)
        for op in ("REPLACE", "SUM", "MAX"):
            l = to_dev(leaf, dtype)
            sf.bcast(to_dev(root, dtype), l, op, bs=bs)
            assert_bits_equal(to_host(l, dtype), oracle.bcast(f, dtype, bs, root, leaf, op), f"bcast {op} {edges} {vec}")
            want = oracle.reduce(f, dtype, bs, leaf, root, op)
            for mode in ("deterministic", "atomic"):
                r = to_dev(root, dtype)
                sf.set_mode(mode).reduce(to_dev(leaf, dtype), r, op, bs=bs)
                if mode == "atomic" and op == "SUM" and dtype.startswith("fp"):
                    assert_atomic_sum_close(to_host(r, dtype), want, f, dtype, bs, leaf, root, "atomic")
                else:
                    assert_bits_equal(to_host(r, dtype), want, f"reduce {mode} {op} {edges} {vec}")
    sf.set_mode("deterministic")


@pytest.mark.parametrize("use_graph", [False, True])
def test_tuned_batch_matches_oracle_at_each_choice(use_graph):
    """Every forest tuned on its own (path, mode, vector width, tile size), then run as one batch:
    bit-exact where the tuner kept the deterministic Reduce, within the atomic bound where it
    chose atomics.  Retuning one forest afterwards rebuilds the batch's tables."""
    items = build(FORESTS[:16], modes=["auto"])
    fresh(items)
    choices = []
    for it in items:
        sf = it["sf"]
        sf.autotune("bcast", it["r"], it["l"], it["op"], bs=it["bs"])
        sf.autotune("reduce", it["l2"], it["r2"], it["op"], bs=it["bs"])
        choices.append(sf.tuning())
    assert all(c["path"] in ("fused", "root_major", "three_phase") for c in choices)
    b = Batch().set_ops(ops_for(items))
    for run in range(2):
        fresh_inplace(items)
        b.run(use_graph=use_graph)
        torch.cuda.synchronize()
        check_choices(items, choices)
        if run == 0:      # retune one forest: its tile list and vector width change
            items[0]["sf"].set_tile_edges(64).set_vector_bytes(2 if items[0]["dt"] == "bf16" else 0)
            choices[0] = items[0]["sf"].tuning()


def fresh_inplace(items):
    for it in items:
        for k, src in (("r", "root"), ("l", "leaf"), ("r2", "root"), ("l2", "leaf")):
            it[k].copy_(to_dev(it[src], it["dt"]))


def check_choices(items, choices):
    for it, c in zip(items, choices):
        f, dt, bs, op = it["f"], it["dt"], it["bs"], it["op"]
        assert_bits_equal(to_host(it["l"], dt), oracle.bcast(f, dt, bs, it["root"], it["leaf"], op),
                          f"tuned batch bcast {f.name} {c}")
        want = oracle.reduce(f, dt, bs, it["leaf"], it["root"], op)
        got = to_host(it["r2"], dt)
        if c["mode"] == "atomic" and op == "SUM" and dt.startswith("fp"):
            assert_atomic_sum_close(got, want, f, dt, bs, it["leaf"], it["root"], f"tuned batch reduce {f.name}")
        else:
            assert_bits_equal(got, want, f"tuned batch reduce {f.name} {c}")
