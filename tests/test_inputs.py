"""The seeded input generators against the recipes they state: the splitmix64 streams
against the generator's published outputs and exact integer arithmetic, and each workload
family against closed forms and structural invariants (sizes, ranges, orderings, the
halo's ghost count, the Zipf and Chung-Lu weight laws).  CPU only."""
import math

import numpy as np
import pytest

import sfgen
from sfgen import rng


# ---- splitmix64 (Steele, Lea & Flood 2014) --------------------------------------------

def test_mix64_reproduces_splitmix64_from_state_zero():
    """A splitmix64 generator started at state 0 returns mix64(k * golden) as its k-th
    output; its first three outputs are the generator's published test values."""
    k = np.arange(1, 4, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out = rng.mix64(rng.GOLDEN * k)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_randint_is_the_exact_multiply_high():
    """randint(lo, hi) = lo + floor(x * span / 2^64) for the raw stream x (Lemire), checked
    with Python's unbounded integers."""
    for span in (1, 7, 1000, 4096, (1 << 40) + 3, (1 << 63) - 25):
        x = rng.u64(123, 9, 257)
        got = rng.randint(123, 9, 257, 5, 5 + span)
        want = [5 + (int(v) * span >> 64) for v in x]
        assert [int(g) for g in got] == want


def test_streams_are_counter_based():
    a = rng.u64(77, 3, 100)
    assert np.array_equal(rng.u64(77, 3, 40, start=60), a[60:])
    assert not np.array_equal(rng.u64(77, 4, 100), a)


@pytest.mark.parametrize("dtype", ["fp64", "fp32", "bf16", "int32", "int64"])
def test_data_values_are_exact_and_in_range(dtype):
    v = sfgen.data(dtype, 20000, 5, 6)
    if dtype == "bf16":
        f = (v.astype(np.uint32) << np.uint32(16)).view(np.float32)
        assert np.all((f >= -1) & (f < 1)) and np.all(f * 64 == np.round(f * 64))
        assert not np.any(v == 0x8000)                       # no negative zero
    elif dtype in ("fp64", "fp32"):
        assert np.all((v >= -1) & (v < 1))
        assert not np.any(np.signbit(v) & (v == 0))
    else:
        assert v.min() >= 0 and v.max() <= 999
    u = sfgen.data("fp64", 20000, 5, 7, "unit")
    assert u.min() >= 0 and u.max() < 1


# ---- plain tiny forest ----------------------------------------------------------------

def test_plain_tiny_shape_and_uniform_roots():
    f = sfgen.cfg1_plain_tiny()
    assert f.nranks == 4 and list(f.nroots) == [4096] * 4 and f.nedges == 16384
    assert all(a is None for a in f.ilocal)
    g = np.concatenate([r.astype(np.int64) * 4096 + i for r, i in zip(f.iremote_rank, f.iremote_index)])
    assert g.min() >= 0 and g.max() < 16384
    # 16384 uniform draws over 16384 roots: E[distinct] = N (1 - (1 - 1/N)^N) ~ N (1 - 1/e)
    N = 16384
    mean = N * (1 - (1 - 1 / N) ** N)
    sd = math.sqrt(N * math.exp(-1) * (1 - 2 * math.exp(-1)))   # occupancy variance, large N
    assert abs(len(np.unique(g)) - mean) < 6 * sd


# ---- 3-D halo exchange ----------------------------------------------------------------

@pytest.mark.parametrize("n,m", [(8, 2), (12, 3), (32, 4), (256, 4)])
def test_halo_ghost_count_closed_form(n, m):
    """The ghosted boxes tile ((n + 2(m-1))^3 points along the three axes) and every rank's
    owned b^3 points are removed: n^3 of them in all; 262^3 - 256^3 at full size."""
    f = sfgen.cfg2_halo(n, m)
    assert f.nedges == (n + 2 * (m - 1)) ** 3 - n ** 3
    if (n, m) == (256, 4):
        assert f.nedges == 1207512


@pytest.mark.parametrize("n,m", [(12, 3), (32, 4)])
def test_halo_ghosts_point_at_their_own_grid_point(n, m):
    """Each leaf of rank p is a point of p's ghosted box owned by a neighbouring rank, and
    its root (owner, owner-local index, x fastest) is that same grid point."""
    f = sfgen.cfg2_halo(n, m)
    b = n // m
    deg = {}
    for p in range(f.nranks):
        c = np.array([p % m, (p // m) % m, p // (m * m)])
        lo = (c > 0).astype(int)
        e = b + lo + (c < m - 1)
        loc = f.ilocal[p]
        box = np.stack([loc % e[0], (loc // e[0]) % e[1], loc // (e[0] * e[1])], 1)
        glob = c * b - lo + box
        owner = f.iremote_rank[p].astype(int)
        oc = np.stack([owner % m, (owner // m) % m, owner // (m * m)], 1)
        assert np.all(owner != p) and np.all(np.abs(oc - c) <= 1)
        oi = f.iremote_index[p]
        oloc = np.stack([oi % b, (oi // b) % b, oi // (b * b)], 1)
        assert np.array_equal(oc * b + oloc, glob)
        assert np.all(np.diff(loc) > 0)                  # increasing local index
        for key in zip(owner.tolist(), oi.tolist()):
            deg[key] = deg.get(key, 0) + 1
    # a block-corner point is a ghost of its 7 surrounding ranks (interior corners)
    assert max(deg.values()) == 7


# ---- unstructured SpMV-style scatter ----------------------------------------------------

def test_spmv_scatter_leaf_order():
    """Rank p lists its owned entries first, in order, then its ghost columns: distinct,
    owned by other ranks, ascending by global column (the lvec order of Sec. IV.A)."""
    f = sfgen.cfg3_spmv(1 << 15, 4)
    per = int(f.nroots[0])
    assert f.nranks == 16 and np.all(f.nroots == per)
    ghosts = 0
    for p in range(f.nranks):
        rr, ri = f.iremote_rank[p].astype(np.int64), f.iremote_index[p]
        assert np.all(rr[:per] == p) and np.array_equal(ri[:per], np.arange(per))
        col = rr[per:] * per + ri[per:]
        assert np.all(rr[per:] != p) and np.all(np.diff(col) > 0)
        assert np.all((ri >= 0) & (ri < per))
        ghosts += len(col)
    assert ghosts == f.meta["ghosts"]
    assert abs(f.meta["degree_sample"] - 14.0) < 1.5


# ---- Zipf batch and Chung-Lu power law --------------------------------------------------

def _in_degrees_descending(f):
    off = np.concatenate([[0], np.cumsum(f.nroots)])
    gid = np.concatenate([off[r] + i for r, i in zip(f.iremote_rank, f.iremote_index)])
    return np.sort(np.bincount(gid, minlength=int(f.nroots.sum())))[::-1]


def test_zipf_forest_follows_the_weight_law():
    """P(root of rank k) = k^-s / H(N, s): the three heaviest roots carry the first three
    weights (within binomial error), and ranks split leaves and roots evenly."""
    N, E, s = 2000, 200000, 1.1
    f = sfgen.zipf_forest(99, 5, E, N, 4, s)
    assert f.nedges == E and int(f.nroots.sum()) == N
    assert f.nleaves.max() - f.nleaves.min() <= 1 and f.nroots.max() - f.nroots.min() <= 1
    cnt = _in_degrees_descending(f)
    H = sum(k ** -s for k in range(1, N + 1))
    for k in range(1, 4):
        p = k ** -s / H
        assert abs(cnt[k - 1] - E * p) < 6 * math.sqrt(E * p * (1 - p)), k


def test_batched_forest_sizes_follow_the_recipe():
    fs = sfgen.cfg4_batched(64)
    for fo in fs:
        assert 100 <= fo.nedges <= 1000000
        assert 0.25 * fo.nedges - 1 <= int(fo.nroots.sum()) <= 4 * fo.nedges + 1
        assert fo.nranks in (1, 2, 4, 8, 16) or fo.nranks == int(fo.nroots.sum())
        assert fo.meta["dtype"] in ("fp32", "fp64", "int64") and fo.meta["bs"] in (1, 2, 3, 8)
        assert fo.meta["op"] in ("SUM", "MAX", "REPLACE")


def test_powerlaw_forest_follows_the_chung_lu_weights():
    """Leaf -> root with probability proportional to (k+1)^(-1/(gamma-1)) for the root of
    weight rank k: the heaviest roots match the first weights within binomial error."""
    N, E, gamma = 1 << 12, 1 << 17, 2.2
    f = sfgen.cfg5_powerlaw(N, E, 8, gamma)
    assert f.nedges == E and int(f.nroots.sum()) == N
    cnt = _in_degrees_descending(f)
    a = 1.0 / (gamma - 1.0)
    Z = sum(k ** -a for k in range(1, N + 1))
    for k in range(1, 4):
        p = k ** -a / Z
        assert abs(cnt[k - 1] - E * p) < 6 * math.sqrt(E * p * (1 - p)), k
