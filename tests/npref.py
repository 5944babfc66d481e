"""Independent numpy formulations used to pin the oracle (never the oracle itself).

These restate the star-forest model with different machinery: offsets by cumulative sums,
edges as index arrays, operations as dense incidence-matrix products or numpy scatter
routines (np.add.at, np.maximum.at, ...).  A mistake in the oracle's loops would have to be
repeated here in a different form to go unnoticed.
"""
from __future__ import annotations

import numpy as np


def extents(forest):
    out = []
    for p in range(forest.nranks):
        a = forest.ilocal[p]
        out.append(int(forest.nleaves[p]) if a is None else (int(a.max()) + 1 if a.size else 0))
    return np.array(out, dtype=np.int64)


def offsets(forest):
    rootoff = np.concatenate([[0], np.cumsum(forest.nroots)]).astype(np.int64)
    leafoff = np.concatenate([[0], np.cumsum(extents(forest))]).astype(np.int64)
    return rootoff, leafoff


def edge_arrays(forest):
    """(leaf unit, root unit) of every edge in canonical order."""
    rootoff, leafoff = offsets(forest)
    L, R = [], []
    for q in range(forest.nranks):
        n = int(forest.nleaves[q])
        loc = np.arange(n) if forest.ilocal[q] is None else forest.ilocal[q]
        L.append(leafoff[q] + loc)
        R.append(rootoff[forest.iremote_rank[q].astype(np.int64)] + forest.iremote_index[q])
    if not L:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(L).astype(np.int64), np.concatenate(R).astype(np.int64)


def incidence(forest):
    """Dense leaf x root incidence matrix P (P[l, r] = 1 for each edge)."""
    rootoff, leafoff = offsets(forest)
    L, R = edge_arrays(forest)
    Pm = np.zeros((int(leafoff[-1]), int(rootoff[-1])), dtype=np.float64)
    Pm[L, R] = 1.0
    return Pm, L, R
