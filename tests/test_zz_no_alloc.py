"""sf_reduce_noalloc: the deterministic Reduce for callers that must not allocate device memory
during the call.  Its fold scratch is a fixed device array inside the library instead of
memory the forest allocates on demand.  This checks, through the C ABI, that it returns
exactly what sf_reduce_begin/end return in deterministic mode, on two calls in a row (the
shared array keeps the previous call's contents), and that a forest whose scratch would not
fit is refused before anything runs.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import sfgen
from tests.gpu_util import assert_bits_equal, make_data, signed_zero_data, signed_zero_forest, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2102_13018_gb300 import StarForest, _abi  # noqa: E402

DTYPE = {"int32": _abi.SF_INT32, "int64": _abi.SF_INT64, "fp32": _abi.SF_FP32, "fp64": _abi.SF_FP64,
         "bf16": _abi.SF_BF16}
OP = {"REPLACE": 0, "SUM": 1, "MIN": 2, "MAX": 3}


def heavy_forests():
    n = 150000
    star = sfgen.Forest(1, np.array([3]), np.array([n]), [None], [np.zeros(n, np.int32)],
                        [(np.arange(n) % 3).astype(np.int64)], name="star3")
    return [star, sfgen.zipf_forest(91, 2, 60000, 2000, 4), sfgen.cfg3_spmv(1 << 15, 4), sfgen.owned_plus_ghosts(5)]


FORESTS = heavy_forests()


def existing_reduce(sf, leaf_t, root_t, unit, op):
    lib = sf._lib
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.sf_set_mode(sf._h, _abi.SF_MODE_DETERMINISTIC) == 0
    args = (sf._h, unit, ctypes.c_void_p(leaf_t.data_ptr()), ctypes.c_void_p(root_t.data_ptr()), OP[op], s)
    assert lib.sf_reduce_begin(*args) == 0
    assert lib.sf_reduce_end(*args) == 0


def noalloc_reduce(sf, leaf_t, root_t, unit, op):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return sf._lib.sf_reduce_noalloc(sf._h, unit, ctypes.c_void_p(leaf_t.data_ptr()),
                                     ctypes.c_void_p(root_t.data_ptr()), OP[op], s)


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
@pytest.mark.parametrize("dtype,bs,op", [("fp64", 1, "SUM"), ("fp32", 4, "SUM"), ("bf16", 8, "SUM"),
                                         ("fp64", 3, "MAX"), ("int32", 1, "SUM"), ("int64", 2, "REPLACE")])
def test_noalloc_matches_existing_reduce_twice(f, dtype, bs, op):
    sf = StarForest.from_forest(f).setup()
    sf.set_mode("atomic")           # the call must be deterministic whatever the forest's mode
    unit = _abi.sf_unit(DTYPE[dtype], bs)
    root, leaf = make_data(f, dtype, bs, 900)
    l = to_dev(leaf, dtype)
    r_ref = to_dev(root, dtype)
    existing_reduce(sf, l, r_ref, unit, op)
    want = to_host(r_ref, dtype)
    assert_bits_equal(want, oracle.reduce(f, dtype, bs, leaf, root, op), f"existing reduce vs oracle {f.name}")
    for call in range(2):           # two calls in a row share the one scratch array
        r = to_dev(root, dtype)
        assert noalloc_reduce(sf, l, r, unit, op) == 0
        torch.cuda.synchronize()
        assert_bits_equal(to_host(r, dtype), want, f"noalloc call {call} {f.name} {op} {dtype}x{bs}")
    sf.destroy()


def test_noalloc_refuses_scratch_beyond_the_maximum():
    """2.2M leaves of one root, fp64 units of 64: fold partials of 34375 blocks x 512 bytes
    exceed the 16 MiB array, so the call returns SF_ERR_TOO_LARGE and launches nothing."""
    n = 2200000
    f = sfgen.Forest(1, np.array([1]), np.array([n]), [None], [np.zeros(n, np.int32)],
                     [np.zeros(n, np.int64)], name="bigstar")
    sf = StarForest.from_forest(f).setup()
    unit = _abi.sf_unit(_abi.SF_FP64, 64)
    leaf = torch.zeros(n * 64, dtype=torch.float64, device="cuda")
    root = torch.zeros(64, dtype=torch.float64, device="cuda")
    from paper_2102_13018_gb300 import launch_count
    n0 = launch_count()
    assert noalloc_reduce(sf, leaf, root, unit, "SUM") == _abi.CODES["SF_ERR_TOO_LARGE"]
    assert launch_count() == n0
    # REPLACE needs no fold scratch, so the same forest is accepted
    leaf.fill_(2.5)
    assert noalloc_reduce(sf, leaf, root, unit, "REPLACE") == 0
    torch.cuda.synchronize()
    assert bool((root == 2.5).all())
    sf.destroy()


def test_noalloc_rejects_bad_arguments_like_reduce_begin():
    f = sfgen.fig2()
    sf = StarForest.from_forest(f)
    unit = _abi.sf_unit(_abi.SF_FP64, 1)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert sf._lib.sf_reduce_noalloc(sf._h, unit, p, p, 1, None) == _abi.CODES["SF_ERR_STATE"]
    sf.setup()
    assert sf._lib.sf_reduce_noalloc(sf._h, _abi.sf_unit(9, 1), p, p, 1, None) == _abi.CODES["SF_ERR_ARG"]
    q = ctypes.c_void_p(buf.data_ptr() + 4)
    assert sf._lib.sf_reduce_noalloc(sf._h, unit, q, p, 1, None) == _abi.CODES["SF_ERR_ALIGN"]
    sf.destroy()


@pytest.mark.parametrize("op", ["MIN", "MAX"])
def test_noalloc_keeps_signed_zero_ties_like_the_oracle(op):
    """+0 and -0 compare equal: MIN/MAX must keep the first in canonical order, exactly as
    the deterministic Reduce and the oracle do, on two calls in a row."""
    SZ = signed_zero_forest()
    sf = StarForest.from_forest(SZ).setup()
    root, leaf = signed_zero_data(SZ, "fp64", 2, 95)
    if op == "MIN":
        root = np.where(root == -1.0, -root, root)
    want = oracle.reduce(SZ, "fp64", 2, leaf, root, op)
    unit = _abi.sf_unit(_abi.SF_FP64, 2)
    l = to_dev(leaf, "fp64")
    for call in range(2):
        r = to_dev(root, "fp64")
        assert noalloc_reduce(sf, l, r, unit, op) == 0
        torch.cuda.synchronize()
        assert_bits_equal(to_host(r, "fp64"), want, f"noalloc signed zeros {op} call {call}")
    sf.destroy()
