"""Multi-forest, Gather / Scatter and embedded forests on the GPU (Sec. III.B-C)."""
import json
import os

import numpy as np
import pytest

import oracle
import sfgen
from tests import npref
from tests.gpu_util import assert_bits_equal, make_data, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import StarForest  # noqa: E402

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig2.json")))


@pytest.mark.parametrize("dtype,bs", [("int32", 1), ("fp32", 2), ("bf16", 3), ("int64", 1)])
def test_gather_scatter_match_oracle(dtype, bs):
    f = sfgen.zipf_forest(12, 3, 30000, 4000, 4)
    sf = StarForest.from_forest(f).setup()
    m = sf.multi_sf()
    root, leaf = make_data(f, dtype, bs, 1402)
    multi0 = sfgen.data(dtype, m.nroots_total * bs, 1402, 3)
    multi = to_dev(multi0, dtype)
    sf.gather(to_dev(leaf, dtype), multi, bs=bs)
    assert_bits_equal(to_host(multi, dtype), oracle.gather(f, dtype, bs, leaf, multi0), f"gather {dtype}x{bs}")
    l = to_dev(leaf, dtype)
    sf.scatter(to_dev(multi0, dtype), l, bs=bs)
    assert_bits_equal(to_host(l, dtype), oracle.scatter(f, dtype, bs, multi0, leaf), f"scatter {dtype}x{bs}")


def test_fig2_multi_forest_sizes_and_gather():
    sf = StarForest.from_forest(sfgen.fig2()).setup()
    m = sf.multi_sf()
    assert m.rootoff.tolist() == [0, 3, 8, 10]          # degrees per rank: 2+0+1, 3+0+1+1, 1+1
    assert np.array_equal(m.leafoff, sf.leafoff)
    leaf = torch.arange(11, dtype=torch.int32, device="cuda") * 10
    multi = torch.full((10,), -1, dtype=torch.int32, device="cuda")
    sf.gather(leaf, multi)
    # leaf unit of each edge and its new root offset: the FetchAndOp leafupdate of Fig. 2
    upd = [v for rank in GOLD["fetch_and_op_sum"]["leafupdate"] for v in rank]
    want = np.full(10, -1)
    lo = sf.leafoff
    ro = m.rootoff
    for q, rank_upd in enumerate(GOLD["fetch_and_op_sum"]["leafupdate"]):
        for l, off in enumerate(rank_upd):
            if off == -7:       # isolated leaf
                continue
            p = sfgen.fig2().iremote_rank[q][list(sfgen.fig2().ilocal[q]).index(l)]
            want[ro[p] + off] = (lo[q] + l) * 10
    assert multi.cpu().numpy().tolist() == want.tolist()


@pytest.mark.parametrize("f", [sfgen.cfg1_plain_tiny(), sfgen.zipf_forest(9, 4, 50000, 2000, 4),
                               sfgen.random_forest(61, 6, 300, 400)], ids=lambda f: f.name)
def test_gather_then_scatter_round_trip(f):
    sf = StarForest.from_forest(f).setup()
    m = sf.multi_sf()
    L, R = npref.edge_arrays(f)
    deg = np.bincount(R, minlength=sf.nroots_total)
    assert m.nroots_total == len(L) and m.nroots_total == int(deg.sum())
    _, leaf = make_data(f, "fp64", 3, 1400)
    multi = torch.zeros(m.nroots_total * 3, dtype=torch.float64, device="cuda")
    sf.gather(to_dev(leaf, "fp64"), multi, bs=3)
    # every new root holds one leaf's unit; as a multiset per original root they are its leaves
    back = to_dev(np.zeros_like(leaf), "fp64")
    sf.scatter(multi, back, bs=3)
    connected = np.zeros(sf.leaf_extent, bool)
    connected[L] = True
    got = to_host(back, "fp64").reshape(-1, 3)
    assert np.array_equal(got[connected], leaf.reshape(-1, 3)[connected])
    assert np.all(got[~connected] == 0)
    # the oracle's Gather and Scatter (Sec. III.B), element by element
    want_multi = oracle.gather(f, "fp64", 3, leaf, np.zeros(m.nroots_total * 3))
    assert_bits_equal(multi.cpu().numpy(), want_multi, f"gather {f.name}")
    leaf0 = sfgen.data("fp64", leaf.size, 1401, 1)
    back2 = to_dev(leaf0, "fp64")
    sf.scatter(to_dev(want_multi, "fp64"), back2, bs=3)
    assert_bits_equal(to_host(back2, "fp64"), oracle.scatter(f, "fp64", 3, want_multi, leaf0), f"scatter {f.name}")


@pytest.mark.parametrize("f", [sfgen.cfg3_spmv(1 << 15, 4), sfgen.random_forest(62, 4, 200, 300)],
                         ids=lambda f: f.name)
def test_embedded_root_forest_moves_only_selected_roots(f):
    sf = StarForest.from_forest(f).setup()
    sel = np.arange(0, sf.nroots_total, 3)
    er = sf.embedded_roots(sel).setup()
    root, leaf = make_data(f, "fp64", 1, 1500)
    full = oracle.bcast(f, "fp64", 1, root, leaf, "REPLACE")
    L, R = npref.edge_arrays(f)
    keep = np.isin(R, sel)
    want = leaf.copy()
    want[L[keep]] = full[L[keep]]
    l = to_dev(leaf, "fp64")
    er.bcast(to_dev(root, "fp64"), l, "REPLACE")
    assert_bits_equal(to_host(l, "fp64"), want, "embedded bcast")
    # Reduce over the embedded forest: unselected roots unchanged
    r = to_dev(root, "fp64")
    er.set_mode("deterministic").reduce(to_dev(leaf, "fp64"), r, "SUM")
    got = to_host(r, "fp64")
    unsel = np.setdiff1d(np.arange(sf.nroots_total), sel)
    assert np.array_equal(got[unsel], root[unsel])


def _roots_for_leaf_space(seed, ext):
    """A forest whose rank q owns ext[q] roots (a leaf space) and whose leaves point at them."""
    nl = [int(x) + 3 for x in ext]
    total = int(np.sum(ext))
    off = np.concatenate([[0], np.cumsum(ext)])
    rr, ri = [], []
    for q, n in enumerate(nl):
        g = sfgen.rng.randint(seed, 50 + q, n, 0, total)
        r = np.searchsorted(off, g, side="right") - 1
        rr.append(r.astype(np.int32))
        ri.append((g - off[r]).astype(np.int64))
    return sfgen.Forest(len(ext), np.array(ext), np.array(nl), [None] * len(ext), rr, ri, name=f"onleaves{seed}")


def test_compose_equals_two_bcasts():
    a = sfgen.random_forest(71, 4, 200, 250, sparse=True)
    sfa = StarForest.from_forest(a)
    ext = np.diff(sfa.leafoff)
    b = _roots_for_leaf_space(72, ext)
    ab = sfa.compose(StarForest.from_forest(b)).setup()
    x, _ = make_data(a, "fp64", 2, 1600)
    mid0 = np.full(int(sfa.leafoff[-1]) * 2, -5.0)
    mid = oracle.bcast(a, "fp64", 2, x, mid0, "REPLACE")
    rob, lob = oracle.layout(b)
    out0 = np.full(int(lob[-1]) * 2, 7.0)
    two_step = oracle.bcast(b, "fp64", 2, mid, out0, "REPLACE")
    got = to_dev(out0, "fp64")
    ab.bcast(to_dev(x, "fp64"), got, "REPLACE", bs=2)
    # B leaves whose B root is an isolated A leaf are not in AB: the two-step result shows -5
    g = to_host(got, "fp64").reshape(-1, 2)
    w = two_step.reshape(-1, 2)
    through = w[:, 0] != -5.0
    assert np.array_equal(g[through], w[through])
    assert np.all(g[~through] == 7.0)


def test_compose_inverse_equals_bcast_then_reduce_replace():
    a = sfgen.random_forest(73, 3, 150, 200, sparse=False)
    sfa = StarForest.from_forest(a)
    ext = np.diff(sfa.leafoff)
    NL = int(ext.sum())
    perm = np.argsort(sfgen.rng.u64(74, 1, NL), kind="stable")     # bijection leaves <-> roots
    lo = np.concatenate([[0], np.cumsum(ext)])
    rr = [(np.searchsorted(lo, perm[lo[q]:lo[q + 1]], side="right") - 1).astype(np.int32) for q in range(3)]
    ri = [(perm[lo[q]:lo[q + 1]] - lo[rr[q]]).astype(np.int64) for q in range(3)]
    b = sfgen.Forest(3, ext, ext, [None] * 3, rr, ri, name="bijection")
    ab = sfa.compose_inverse(StarForest.from_forest(b)).setup()
    x, _ = make_data(a, "fp64", 1, 1700)
    mid = oracle.bcast(a, "fp64", 1, x, np.full(NL, -5.0), "REPLACE")
    want = oracle.reduce(b, "fp64", 1, mid, np.full(NL, 9.0), "REPLACE")
    got = to_dev(np.full(NL, 9.0), "fp64")
    ab.bcast(to_dev(x, "fp64"), got, "REPLACE")
    g = to_host(got, "fp64")
    through = want != -5.0
    assert np.array_equal(g[through], want[through])
    assert np.all(g[~through] == 9.0)
