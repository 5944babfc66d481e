"""The algorithmic byte counts behind every GB/s and roofline figure of bench.py, against the
forests themselves (CPU): connected roots and edges counted here with numpy, index words from
the setup pass's pattern analysis, and Fig. 2 worked by hand."""
import numpy as np
import pytest

import bench
import sfgen
from paper_2102_13018_gb300 import StarForest


def _counts(f):
    """(edges, connected roots) of a forest, from its arrays."""
    rootoff = np.concatenate([[0], np.cumsum(f.nroots)]).astype(np.int64)
    g = np.concatenate([rootoff[f.iremote_rank[q].astype(np.int64)] + f.iremote_index[q] for q in range(f.nranks)])
    return int(g.size), int(np.unique(g).size)


@pytest.mark.parametrize("f", [sfgen.fig2(), sfgen.random_forest(61, 3, 300, 400), sfgen.cfg1_plain_tiny(),
                               sfgen.zipf_forest(62, 1, 5000, 700, 3)], ids=lambda f: f.name)
@pytest.mark.parametrize("unit", [4, 8, 40, 256])
def test_byte_counts_follow_the_forest(f, unit):
    info = StarForest.from_forest(f).analyze().info()
    E, C = _counts(f)
    assert info["nedges"] == E and info["connected_roots"] == C
    idx = 4 * (info["edges_one_indexed"] + 2 * info["edges_two_indexed"])
    b, r = bench.algorithmic_bytes(info, unit)
    assert b == unit * (C + E) + idx
    assert r == unit * E + 2 * unit * C + idx
    assert bench.op_bytes(info, "bcast", "REPLACE", unit) == b
    assert bench.op_bytes(info, "bcast", "SUM", unit) == b + unit * E      # leaves read too
    assert bench.op_bytes(info, "reduce", "SUM", unit) == r
    assert bench.op_bytes(info, "fetch", "SUM", unit) == r + unit * E      # leafupdate written


def test_fig2_by_hand():
    """Fig. 2: 10 leaves over 3 ranks reaching 7 distinct roots of the 9 (Sec. III.A): rank 0's
    leaves reach (1,2), (1,0) twice and (0,2); rank 1's (2,0), (0,0), (2,1); rank 2's (0,0),
    (1,0), (1,3)."""
    f = sfgen.fig2()
    info = StarForest.from_forest(f).analyze().info()
    assert (info["nedges"], info["connected_roots"]) == (10, 7)
    idx = 4 * (info["edges_one_indexed"] + 2 * info["edges_two_indexed"])
    assert bench.algorithmic_bytes(info, 8) == (8 * 7 + 8 * 10 + idx, 8 * 10 + 16 * 7 + idx)
