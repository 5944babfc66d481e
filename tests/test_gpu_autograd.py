"""Differentiable Bcast / Reduce (SUM, MAX) and MAX-with-location vs the oracle (GB300)."""
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
from paper_2102_13018_gb300 import autograd as sfa  # noqa: E402


def slice_of_powerlaw(nroots_keep=256, nroots=1 << 14, nleaves=1 << 17, nranks=8):
    """The power-law message-passing forest restricted to roots < nroots_keep and the leaves that
    point at them (an embedded-root slice), leaves renumbered compactly per rank."""
    f = sfgen.cfg5_powerlaw(nroots, nleaves, nranks)
    per = nroots // nranks
    rr, ri, nl = [], [], []
    for q in range(nranks):
        g = f.iremote_rank[q].astype(np.int64) * per + f.iremote_index[q]
        k = g < nroots_keep
        rr.append((g[k] // max(per, 1)).astype(np.int32))
        ri.append((g[k] % max(per, 1)).astype(np.int64))
        nl.append(int(k.sum()))
    roots = np.zeros(nranks, np.int64)
    for p in range(nranks):
        roots[p] = max(0, min(per, nroots_keep - p * per))
    return sfgen.Forest(nranks, roots, np.array(nl), [None] * nranks, rr, ri, name=f"powerlaw_slice{nroots_keep}")


SLICE = slice_of_powerlaw()


@pytest.mark.parametrize("f", [sfgen.fig2(), sfgen.cfg1_plain_tiny(), SLICE, sfgen.zipf_forest(5, 3, 300000, 500, 4),
                               sfgen.random_forest(51, 5, 200, 300)], ids=lambda f: f.name)
@pytest.mark.parametrize("dtype,bs", [("fp64", 1), ("fp32", 3), ("bf16", 4), ("int32", 2)])
def test_maxloc_matches_oracle(f, dtype, bs):
    sf = StarForest.from_forest(f).setup()
    _, leaf = make_data(f, dtype, bs, 1200)
    want_v, want_e = oracle.reduce_maxloc(f, dtype, bs, leaf)
    L, R = npref.edge_arrays(f)
    ro, lo = oracle.layout(f)
    root = to_dev(np.zeros(ro[-1] * bs, oracle.NPTYPE[dtype]), dtype)
    arg = torch.full((int(ro[-1]) * bs,), -1, dtype=torch.int32, device="cuda")
    sf.reduce_maxloc(to_dev(leaf, dtype), root, arg, bs=bs)
    assert_bits_equal(to_host(root, dtype), want_v, f"maxloc value {f.name}")
    want_leaf = np.where(want_e >= 0, L[np.maximum(want_e, 0)], -1)
    assert np.array_equal(arg.cpu().numpy().astype(np.int64), want_leaf)


def test_gradcheck_fp64_slice():
    sf = StarForest.from_forest(SLICE).setup().set_mode("deterministic")
    bs = 2
    x = torch.rand(sf.nroots_total, bs, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: sfa.bcast(sf, t), (x,), eps=1e-6, atol=1e-7)
    y = torch.rand(sf.leaf_extent, bs, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: sfa.reduce(sf, t, "SUM"), (y,), eps=1e-6, atol=1e-7)
    assert torch.autograd.gradcheck(lambda t: sfa.reduce(sf, t, "MAX"), (y,), eps=1e-6, atol=1e-7)


@pytest.fixture(scope="module")
def powerlaw_root_slice():
    """The full power-law message-passing forest (2^20 roots, 2^23 leaves) cut to its roots
    below 1024 by sf_create_embedded_root_sf (Sec. III.C: the edges of the selected roots, with
    nothing renumbered, so the slice keeps the full buffer layout).  Returns the slice, the
    leaf and root units of its edges in canonical order, and the layout sizes."""
    f = sfgen.cfg5_powerlaw()
    full = StarForest.from_forest(f)
    sl = full.embedded_roots(np.arange(1024)).setup().set_mode("deterministic")
    L, R = npref.edge_arrays(f)
    keep = R < 1024
    assert sl.info()["nedges"] == int(keep.sum()) > 1024
    return sl, L[keep], R[keep]


def test_gradcheck_fp64_on_embedded_root_slice(powerlaw_root_slice):
    """fp64 gradcheck of Bcast, Reduce SUM and Reduce MAX on the 2^10-root slice of the full
    power-law forest.  The checked function maps the 1024 selected roots' values (or the slice's
    leaf values) through the full-layout operation and back out, so the Jacobian stays small."""
    sl, L, R = powerlaw_root_slice
    bs = 2
    Lt, sel = torch.from_numpy(L).cuda(), torch.arange(1024, device="cuda")

    def bcast_slice(xs):
        x = torch.zeros(sl.nroots_total, bs, dtype=xs.dtype, device="cuda").index_copy(0, sel, xs)
        return sfa.bcast(sl, x).index_select(0, Lt)

    def reduce_slice(ys, op):
        y = torch.zeros(sl.leaf_extent, bs, dtype=ys.dtype, device="cuda").index_copy(0, Lt, ys)
        return sfa.reduce(sl, y, op).index_select(0, sel)

    xs = torch.rand(1024, bs, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(bcast_slice, (xs,), eps=1e-6, atol=1e-7, fast_mode=True)
    ys = torch.rand(len(L), bs, dtype=torch.float64, device="cuda", requires_grad=True)   # no ties
    assert torch.autograd.gradcheck(lambda t: reduce_slice(t, "SUM"), (ys,), eps=1e-6, atol=1e-7, fast_mode=True)
    assert torch.autograd.gradcheck(lambda t: reduce_slice(t, "MAX"), (ys,), eps=1e-6, atol=1e-7, fast_mode=True)


def test_embedded_root_slice_gradients_are_dense_transposes(powerlaw_root_slice):
    """On the slice, Bcast is lvec[L_e] = x[R_e] and its gradient the sum of g[L_e] into R_e;
    integer-valued fp64 data makes every sum exact.  Leaves of other roots stay 0."""
    sl, L, R = powerlaw_root_slice
    bs = 3
    x = torch.randint(-9, 9, (sl.nroots_total, bs), device="cuda").double().requires_grad_(True)
    out = sfa.bcast(sl, x)
    want = np.zeros((sl.leaf_extent, bs))
    xh = x.detach().cpu().numpy()
    want[L] = xh[R]
    assert np.array_equal(out.detach().cpu().numpy(), want)
    g = torch.randint(-50, 50, out.shape, device="cuda").double()
    out.backward(g)
    gh = g.cpu().numpy()
    want_g = np.zeros((sl.nroots_total, bs))
    np.add.at(want_g, R, gh[L])
    assert np.array_equal(x.grad.cpu().numpy(), want_g)


def test_gradients_are_dense_transposes():
    """Bcast backward = P^T g, Reduce SUM backward = P g (fp64, exact for these sums of at most
    a few hundred terms of integer-valued data)."""
    f = SLICE
    Pm, L, R = npref.incidence(f)
    sf = StarForest.from_forest(f).setup().set_mode("deterministic")
    bs = 3
    x = torch.rand(sf.nroots_total, bs, dtype=torch.float64, device="cuda", requires_grad=True)
    out = sfa.bcast(sf, x)
    g = torch.randint(-50, 50, out.shape, device="cuda").double()
    out.backward(g)
    assert np.array_equal(x.grad.cpu().numpy(), Pm.T @ g.cpu().numpy())
    assert np.array_equal(out.detach().cpu().numpy(), Pm @ x.detach().cpu().numpy())
    y = torch.rand(sf.leaf_extent, bs, dtype=torch.float64, device="cuda", requires_grad=True)
    r = sfa.reduce(sf, y, "SUM")
    gr = torch.randint(-50, 50, r.shape, device="cuda").double()
    r.backward(gr)
    assert np.array_equal(y.grad.cpu().numpy(), Pm @ gr.cpu().numpy())


def test_max_gradient_goes_to_first_maximum():
    f = SLICE
    sf = StarForest.from_forest(f).setup()
    bs = 2
    y = torch.randint(0, 4, (sf.leaf_extent, bs), device="cuda").double().requires_grad_(True)   # many ties
    r = sfa.reduce(sf, y, "MAX")
    r.backward(torch.ones_like(r))
    want_v, want_e = oracle.reduce_maxloc(f, "fp64", bs, y.detach().cpu().numpy().ravel())
    L, _ = npref.edge_arrays(f)
    gl = np.zeros(sf.leaf_extent * bs)
    for i, e in enumerate(want_e):
        if e >= 0:
            gl[L[e] * bs + i % bs] = 1.0
    assert np.array_equal(r.detach().cpu().numpy().ravel(), want_v)
    assert np.array_equal(y.grad.cpu().numpy().ravel(), gl)


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_full_size_forward_and_backward_match_oracle(dtype):
    """2^20 roots, 2^23 leaves, bs = 64: forward Bcast and Reduce SUM, and the backward of Bcast
    (a Reduce SUM into zeros), bit-exact against the oracle's deterministic fold."""
    f = sfgen.cfg5_powerlaw()
    sf = StarForest.from_forest(f).setup().set_mode("deterministic")
    bs = 64
    root, leaf = make_data(f, dtype, bs, 1300)
    tdt = torch.float32 if dtype == "fp32" else torch.bfloat16
    x = to_dev(root, dtype).view(-1, bs).requires_grad_(True)
    out = sfa.bcast(sf, x)
    assert_bits_equal(to_host(out.detach().reshape(-1), dtype),
                      oracle.bcast(f, dtype, bs, root, np.zeros_like(leaf), "REPLACE"), "bcast fwd")
    g = to_dev(leaf, dtype).view(-1, bs)
    out.backward(g)
    want = oracle.reduce(f, dtype, bs, leaf, np.zeros_like(root), "SUM")
    assert_bits_equal(to_host(x.grad.reshape(-1), dtype), want, "bcast backward = Reduce SUM")
    assert x.grad.dtype == tdt
