"""Seeded synthetic star forests and data for the five workload families.

A forest is given the way its owner ranks would describe it: per simulated rank p,
``nroots[p]`` roots, ``nleaves[p]`` connected leaves, the leaves' local indices
``ilocal[p]`` (``None`` = contiguous 0..nleaves-1) and their root addresses
``(iremote_rank[p][i], iremote_index[p][i])`` (Sec. III.A, PetscSFSetGraph).

This module builds graphs and draws numbers only.  It computes no Bcast, Reduce or
FetchAndOp, no buffer layout and no index plan: both the oracle and the CUDA path
take these arrays as inputs and derive everything else on their own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import rng


@dataclass
class Forest:
    nranks: int
    nroots: np.ndarray                      # int64 [P]
    nleaves: np.ndarray                     # int64 [P]
    ilocal: List[Optional[np.ndarray]]      # per rank int64 [nleaves[p]] or None
    iremote_rank: List[np.ndarray]          # per rank int32 [nleaves[p]]
    iremote_index: List[np.ndarray]         # per rank int64 [nleaves[p]]
    name: str = ""
    meta: dict = field(default_factory=dict)

    def __post_init__(self):
        self.nroots = np.ascontiguousarray(self.nroots, dtype=np.int64)
        self.nleaves = np.ascontiguousarray(self.nleaves, dtype=np.int64)
        self.ilocal = [None if a is None else np.ascontiguousarray(a, dtype=np.int64) for a in self.ilocal]
        self.iremote_rank = [np.ascontiguousarray(a, dtype=np.int32) for a in self.iremote_rank]
        self.iremote_index = [np.ascontiguousarray(a, dtype=np.int64) for a in self.iremote_index]

    @property
    def nedges(self) -> int:
        return int(self.nleaves.sum())

    def flat(self):
        """Concatenated arrays: has_ilocal[P] int32, ilocal[E] int64 (zeros where a rank
        passes None), iremote rank[E] int32 and index[E] int64."""
        E = self.nedges
        has = np.array([a is not None for a in self.ilocal], dtype=np.int32)
        il = np.zeros(E, dtype=np.int64)
        pos = 0
        for p in range(self.nranks):
            n = int(self.nleaves[p])
            if self.ilocal[p] is not None:
                il[pos:pos + n] = self.ilocal[p]
            pos += n
        rr = np.concatenate(self.iremote_rank) if E else np.zeros(0, np.int32)
        ri = np.concatenate(self.iremote_index) if E else np.zeros(0, np.int64)
        return has, il, np.ascontiguousarray(rr, np.int32), np.ascontiguousarray(ri, np.int64)


def from_lists(nroots, leaves, name="") -> Forest:
    """leaves[p] = list of (local, (rank, index)); local=None for all → ilocal None."""
    P = len(nroots)
    il, rr, ri, nl = [], [], [], []
    for p in range(P):
        L = leaves[p]
        nl.append(len(L))
        if all(l is None for l, _ in L):
            il.append(None)
        else:
            il.append(np.array([l for l, _ in L], dtype=np.int64))
        rr.append(np.array([r for _, (r, _) in L], dtype=np.int32))
        ri.append(np.array([i for _, (_, i) in L], dtype=np.int64))
    return Forest(P, np.array(nroots), np.array(nl), il, rr, ri, name=name)


def fig2() -> Forest:
    """The three-rank forest drawn with its local/remote arrays in Fig. 2."""
    return Forest(
        3,
        np.array([3, 4, 2]),
        np.array([4, 3, 3]),
        [np.array([0, 1, 2, 3]), np.array([0, 1, 3]), np.array([0, 1, 2])],
        [np.array([1, 1, 1, 0]), np.array([2, 0, 2]), np.array([0, 1, 1])],
        [np.array([2, 0, 0, 2]), np.array([0, 0, 1]), np.array([0, 0, 3])],
        name="fig2",
    )


def random_forest(seed: int, nranks: int, max_roots: int, max_leaves: int,
                  sparse: bool = True, allow_empty: bool = True, name: str = "") -> Forest:
    """Small random forest: random per-rank sizes (possibly 0), optional sparse ilocal
    (a random subset of a larger leaf space, unsorted), roots uniform over all roots."""
    lo = 0 if allow_empty else 1
    nroots = rng.randint(seed, 1, nranks, lo, max_roots + 1)
    if nroots.sum() == 0:
        nroots[0] = 1
    nleaves = rng.randint(seed, 2, nranks, lo, max_leaves + 1)
    total_roots = int(nroots.sum())
    rootoff = np.concatenate([[0], np.cumsum(nroots)])
    il, rr, ri = [], [], []
    for p in range(nranks):
        n = int(nleaves[p])
        g = rng.randint(seed, 100 + p, n, 0, total_roots)
        r = np.searchsorted(rootoff, g, side="right") - 1
        rr.append(r.astype(np.int32))
        ri.append((g - rootoff[r]).astype(np.int64))
        use_sparse = sparse and (rng.u64(seed, 200 + p, 1)[0] & np.uint64(1)) == 1
        if use_sparse and n > 0:
            extent = n + int(rng.randint(seed, 300 + p, 1, 0, n + 3)[0])
            keys = rng.u64(seed, 400 + p, extent)
            il.append(np.argsort(keys, kind="stable")[:n].astype(np.int64))
        else:
            il.append(None)
    return Forest(nranks, nroots, nleaves, il, rr, ri, name=name or f"random{seed}")


def one_to_one(seed: int, nranks: int, n_per_rank: int) -> Forest:
    """Every root has exactly one leaf: a random bijection between all roots and all
    leaves (the ping-pong forest of Sec. VI.A is the special case of identity order)."""
    total = nranks * n_per_rank
    perm = np.argsort(rng.u64(seed, 7, total), kind="stable")
    il, rr, ri = [], [], []
    for q in range(nranks):
        g = perm[q * n_per_rank:(q + 1) * n_per_rank]
        rr.append((g // n_per_rank).astype(np.int32))
        ri.append((g % n_per_rank).astype(np.int64))
        il.append(None)
    return Forest(nranks, np.full(nranks, n_per_rank), np.full(nranks, n_per_rank), il, rr, ri,
                  name=f"one_to_one{seed}")


def pingpong(n: int) -> Forest:
    """n roots on rank 0 connected consecutively to n leaves on rank 1 (Sec. VI.A)."""
    return Forest(2, np.array([n, 0]), np.array([0, n]), [None, None],
                  [np.zeros(0, np.int32), np.zeros(n, np.int32)],
                  [np.zeros(0, np.int64), np.arange(n, dtype=np.int64)], name=f"pingpong{n}")


# --------------------------------------------------------------------------------------
# Workload family 1: plain tiny forest
# --------------------------------------------------------------------------------------

def cfg1_plain_tiny(nranks: int = 4, nroots_per: int = 4096, nleaves_per: int = 4096) -> Forest:
    """4 ranks x 4096 roots; 4096 leaves per rank (16384 total), ilocal = identity;
    each leaf's root uniform over (rank, index)."""
    seed = rng.BASE_SEED + 1
    rr, ri = [], []
    for q in range(nranks):
        rr.append(rng.randint(seed, 10 + q, nleaves_per, 0, nranks).astype(np.int32))
        ri.append(rng.randint(seed, 20 + q, nleaves_per, 0, nroots_per))
    return Forest(nranks, np.full(nranks, nroots_per), np.full(nranks, nleaves_per),
                  [None] * nranks, rr, ri, name="plain_tiny")


# --------------------------------------------------------------------------------------
# Workload family 2: 3-D structured halo exchange
# --------------------------------------------------------------------------------------

def cfg2_halo(n: int = 256, m: int = 4, include_owned: bool = False) -> Forest:
    """n^3 grid (x fastest) split into m^3 ranks of b^3 owned points (b = n/m), rank
    order x fastest.  Rank p's leaf space is its ghosted box (width-1 layer toward each
    existing neighbour, non-periodic), numbered x fastest.  Leaves are the ghost points
    of the 27-point box stencil, listed in increasing local index; each points to the
    owner's local index.  With include_owned, the owned points are leaves as well (the
    global-to-local copy of a local vector with ghosts)."""
    assert n % m == 0
    b = n // m
    P = m ** 3
    il, rr, ri, nl = [], [], [], []
    for p in range(P):
        px, py, pz = p % m, (p // m) % m, p // (m * m)
        lo = [(px > 0), (py > 0), (pz > 0)]
        hi = [(px < m - 1), (py < m - 1), (pz < m - 1)]
        ex, ey, ez = (b + lo[0] + hi[0], b + lo[1] + hi[1], b + lo[2] + hi[2])
        # global coordinates of the ghosted box
        gx = np.arange(px * b - lo[0], px * b + b + hi[0])
        gy = np.arange(py * b - lo[1], py * b + b + hi[1])
        gz = np.arange(pz * b - lo[2], pz * b + b + hi[2])
        Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
        X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
        local = np.arange(ex * ey * ez, dtype=np.int64)
        ox, oy, oz = X // b, Y // b, Z // b
        owner = ox + m * (oy + m * oz)
        if not include_owned:
            sel = owner != p
            local, X, Y, Z, owner = local[sel], X[sel], Y[sel], Z[sel], owner[sel]
        oidx = (X - (X // b) * b) + b * ((Y - (Y // b) * b) + b * (Z - (Z // b) * b))
        il.append(local)
        rr.append(owner.astype(np.int32))
        ri.append(oidx.astype(np.int64))
        nl.append(local.size)
    return Forest(P, np.full(P, b ** 3), np.array(nl), il, rr, ri,
                  name=f"halo{n}_{m}x{m}x{m}" + ("_owned" if include_owned else ""),
                  meta={"n": n, "m": m, "b": b})


# --------------------------------------------------------------------------------------
# Workload family 4: batched, Zipf in-degree
# --------------------------------------------------------------------------------------

def owned_plus_ghosts(seed: int, nroots=(1000, 2048, 37, 3001, 700, 96), keep: float = 0.9,
                      ghosts_per_rank: int = 900, heavy: int = 3, shuffled_rank: int = 2) -> Forest:
    """The shape of the SpMV scatter (Sec. IV.A) with its corner cases: every rank q lists
    its owned entries first -- leaf i -> root (q, i), each kept with probability `keep` --
    then ghost leaves pointing at random roots of any rank (in random order, so a root's
    ghosts fall before or after its owned leaf in canonical order), 70 or 30 of them piled on
    each of `heavy` roots per rank so that some roots get more than 64 leaves.  On rank
    `shuffled_rank` the owned leaves are permuted, so they sit at no fixed offset from their
    roots.  Rank sizes that are not multiples of 32 leave chunks of 32 roots straddling two
    ranks.  ilocal is given (owned leaves keep local index i, ghosts follow at n_q + k)."""
    P = len(nroots)
    nroots = np.array(nroots, dtype=np.int64)
    total = int(nroots.sum())
    rootoff = np.concatenate([[0], np.cumsum(nroots)])
    il, rr, ri, nl = [], [], [], []
    for q in range(P):
        n = int(nroots[q])
        own = np.nonzero(rng.uniform01(seed, 10 + q, n) < keep)[0]
        own_root = own.copy()
        if q == shuffled_rank:
            own_root = own[np.argsort(rng.u64(seed, 20 + q, own.size), kind="stable")]
        g = rng.randint(seed, 30 + q, ghosts_per_rank, 0, total)
        hot = rng.randint(seed, 40 + q, heavy, 0, total)
        g = np.concatenate([g, np.repeat(hot, [70] + [30] * (heavy - 1))])
        g = g[np.argsort(rng.u64(seed, 50 + q, g.size), kind="stable")]
        gr = np.searchsorted(rootoff, g, side="right") - 1
        il.append(np.concatenate([own, n + np.arange(g.size)]).astype(np.int64))
        rr.append(np.concatenate([np.full(own.size, q), gr]).astype(np.int32))
        ri.append(np.concatenate([own_root, g - rootoff[gr]]).astype(np.int64))
        nl.append(own.size + g.size)
    return Forest(P, nroots, np.array(nl), il, rr, ri, name=f"owned_plus_ghosts{seed}")


def zipf_forest(seed: int, tag: int, nleaves: int, nroots: int, nranks: int,
                s: float = 1.1) -> Forest:
    """nleaves leaves split evenly over nranks (ilocal None); roots split evenly; each
    leaf's root is Zipf(s) over a random permutation of the roots (inverse-CDF table)."""
    w = np.arange(1, nroots + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.uniform01(seed, tag * 16 + 1, nleaves)
    rankk = np.minimum(np.searchsorted(cdf, u, side="right"), nroots - 1)
    perm = np.argsort(rng.u64(seed, tag * 16 + 2, nroots), kind="stable")
    g = perm[rankk]
    nr = np.full(nranks, nroots // nranks, dtype=np.int64)
    nr[: nroots % nranks] += 1
    rootoff = np.concatenate([[0], np.cumsum(nr)])
    nlv = np.full(nranks, nleaves // nranks, dtype=np.int64)
    nlv[: nleaves % nranks] += 1
    leafoff = np.concatenate([[0], np.cumsum(nlv)])
    r = np.searchsorted(rootoff, g, side="right") - 1
    idx = g - rootoff[r]
    rr = [r[leafoff[q]:leafoff[q + 1]].astype(np.int32) for q in range(nranks)]
    ri = [idx[leafoff[q]:leafoff[q + 1]].astype(np.int64) for q in range(nranks)]
    return Forest(nranks, nr, nlv, [None] * nranks, rr, ri, name=f"zipf{tag}")


BATCH_DTYPES = ("fp32", "fp64", "int64")
BATCH_BS = (1, 2, 3, 8)
BATCH_OPS = ("SUM", "MAX", "REPLACE")


def cfg4_batched(nforests: int = 512, lo: float = 1e2, hi: float = 1e6, scale: float = 1.0):
    """512 independent forests: nleaves log-uniform in [lo, hi] (times scale), nroots =
    ceil(nleaves * U[0.25, 4]), ranks U{1,2,4,8,16}, Zipf(1.1) in-degree; per forest a
    dtype in {fp32, fp64, int64}, bs in {1,2,3,8} and op in {SUM, MAX, REPLACE}."""
    seed = rng.BASE_SEED + 4
    u1 = rng.uniform01(seed, 1, nforests)
    u2 = rng.uniform01(seed, 2, nforests)
    pr = rng.randint(seed, 3, nforests, 0, 5)
    dt = rng.randint(seed, 4, nforests, 0, 3)
    bsi = rng.randint(seed, 5, nforests, 0, 4)
    opi = rng.randint(seed, 6, nforests, 0, 3)
    out = []
    for f in range(nforests):
        nleaves = max(1, int(round(math.exp(math.log(lo) + u1[f] * (math.log(hi) - math.log(lo))) * scale)))
        nroots = max(1, int(math.ceil(nleaves * (0.25 + 3.75 * u2[f]))))
        P = [1, 2, 4, 8, 16][int(pr[f])]
        P = min(P, nroots)
        fo = zipf_forest(seed, 1000 + f, nleaves, nroots, P)
        fo.name = f"batch{f}"
        fo.meta = {"dtype": BATCH_DTYPES[int(dt[f])], "bs": BATCH_BS[int(bsi[f])],
                   "op": BATCH_OPS[int(opi[f])]}
        out.append(fo)
    return out


# --------------------------------------------------------------------------------------
# Workload family 5: differentiable message passing graph (power-law in-degree)
# --------------------------------------------------------------------------------------

def cfg5_powerlaw(nroots: int = 1 << 20, nleaves: int = 1 << 23, nranks: int = 8,
                  exponent: float = 2.2) -> Forest:
    """Chung-Lu in-degree: leaf -> root with probability proportional to
    (pi(r)+1)^(-1/(exponent-1)) over a random permutation pi; ranks split evenly."""
    seed = rng.BASE_SEED + 5
    w = np.arange(1, nroots + 1, dtype=np.float64) ** (-1.0 / (exponent - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.uniform01(seed, 1, nleaves)
    k = np.minimum(np.searchsorted(cdf, u, side="right"), nroots - 1)
    perm = np.argsort(rng.u64(seed, 2, nroots), kind="stable")
    g = perm[k]
    nr = np.full(nranks, nroots // nranks, dtype=np.int64)
    nlv = np.full(nranks, nleaves // nranks, dtype=np.int64)
    assert nr.sum() == nroots and nlv.sum() == nleaves
    per = nroots // nranks
    r = g // per
    idx = g - r * per
    rr = [r[q * (nleaves // nranks):(q + 1) * (nleaves // nranks)].astype(np.int32) for q in range(nranks)]
    ri = [idx[q * (nleaves // nranks):(q + 1) * (nleaves // nranks)].astype(np.int64) for q in range(nranks)]
    return Forest(nranks, nr, nlv, [None] * nranks, rr, ri, name=f"powerlaw{nroots}_{nleaves}")


# --------------------------------------------------------------------------------------
# Data
# --------------------------------------------------------------------------------------

DTYPES = {"int32": np.int32, "int64": np.int64, "fp32": np.float32, "fp64": np.float64,
          "bf16": np.uint16}


def data(dtype: str, n: int, seed: int, tag: int, kind: str = "signed") -> np.ndarray:
    """n values of a dtype.  Floats: uniform in [-1, 1) ("signed") or [0, 1) ("unit"),
    on a 2^-53 / 2^-24 / 2^-7 grid so every value is exact in its type; bf16 is returned
    as raw uint16 bit patterns.  Integers: uniform in {0..999} ("signed"/"unit") or the
    full range ("wide", exercises wraparound).  No NaN and no negative zero."""
    x = rng.u64(seed, tag, n)
    if dtype == "fp64":
        v = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        v = 2.0 * v - 1.0 if kind == "signed" else v
        return np.where(v == 0.0, 0.0, v).astype(np.float64)
    if dtype == "fp32":
        v = (x >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)
        v = 2.0 * v - 1.0 if kind == "signed" else v
        return np.where(v == 0.0, 0.0, v).astype(np.float32)
    if dtype == "bf16":
        k = (x >> np.uint64(57)).astype(np.float64)          # 0..127
        v = k * (2.0 ** -7)
        v = 2.0 * v - 1.0 if kind == "signed" else v         # multiples of 2^-6 in [-1,1)
        f = np.where(v == 0.0, 0.0, v).astype(np.float32)
        return (f.view(np.uint32) >> np.uint32(16)).astype(np.uint16)   # exact: low bits 0
    if dtype in ("int32", "int64"):
        if kind == "wide":
            if dtype == "int32":
                return (x >> np.uint64(32)).astype(np.uint32).view(np.int32)
            return x.view(np.int64)
        return (x % np.uint64(1000)).astype(DTYPES[dtype])
    raise ValueError(dtype)
