"""The multi-core CPU baseline of the benchmark (oracle/sf_cpu_parallel.c) computes what the
oracle computes, bit for bit: Bcast REPLACE and the deterministic Reduce SUM (CPU only)."""
import numpy as np
import pytest

import oracle
import sfgen


@pytest.mark.parametrize("f", [sfgen.fig2(), sfgen.cfg1_plain_tiny(), sfgen.random_forest(71, 5, 300, 400),
                               sfgen.zipf_forest(72, 1, 50000, 300, 3), sfgen.cfg3_spmv(1 << 14, 3),
                               sfgen.owned_plus_ghosts(5)], ids=lambda f: f.name)
def test_cpu_parallel_step_matches_oracle(f):
    if oracle.build_parallel() is None:
        pytest.skip("no OpenMP compiler")
    cp = oracle.CpuParallel(f)
    assert cp.threads >= 1
    ro, lo = oracle.layout(f)
    x = sfgen.data("fp64", int(ro[-1]), 73, 1)
    leaf0 = sfgen.data("fp64", int(lo[-1]), 73, 2)
    y = sfgen.data("fp64", int(ro[-1]), 73, 3)
    lv = leaf0.copy()
    cp.bcast_replace(x, lv)
    assert np.array_equal(lv.view(np.uint64), oracle.bcast(f, "fp64", 1, x, leaf0, "REPLACE").view(np.uint64))
    yy = y.copy()
    cp.reduce_sum(lv, yy)
    assert np.array_equal(yy.view(np.uint64), oracle.reduce(f, "fp64", 1, lv, y, "SUM").view(np.uint64))
