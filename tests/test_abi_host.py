"""C ABI surface and the host setup pass, on the CPU (no CUDA call needs a device here)."""
import ctypes

import numpy as np
import pytest

import oracle
import sfgen
from paper_2102_13018_gb300 import _abi, StarForest, SFError
from tests import npref


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    names = _abi.declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_error_strings_cover_every_code():
    lib = _abi.load()
    for code in _abi.ERRORS:
        s = lib.sf_error_string(code).decode()
        assert s and s != "unknown error code"
    assert lib.sf_error_string(999).decode() == "unknown error code"


def _create_raw(P, nroots, nleaves, ilocal, rr, ri):
    try:
        StarForest(nroots, nleaves, ilocal, rr, ri)
        return 0
    except SFError as e:
        return e.code


@pytest.mark.parametrize("case,code", [
    ("zero_ranks", "SF_ERR_ARG"),
    ("negative_nroots", "SF_ERR_ARG"),
    ("rank_out_of_range", "SF_ERR_RANGE"),
    ("index_out_of_range", "SF_ERR_RANGE"),
    ("negative_index", "SF_ERR_RANGE"),
    ("negative_ilocal", "SF_ERR_RANGE"),
    ("duplicate_ilocal", "SF_ERR_DUP_LEAF"),
    ("ok", "SF_SUCCESS"),
])
def test_create_validation(case, code):
    args = {
        "zero_ranks": ([], [], None, [], []),
        "negative_nroots": ([-1], [0], None, [[]], [[]]),
        "rank_out_of_range": ([2, 2], [1, 0], None, [[2], []], [[0], []]),
        "index_out_of_range": ([2, 2], [1, 0], None, [[1], []], [[2], []]),
        "negative_index": ([2], [1], None, [[0]], [[-1]]),
        "negative_ilocal": ([2], [1], [[-3]], [[0]], [[0]]),
        "duplicate_ilocal": ([2], [2], [[5, 5]], [[0, 0]], [[0, 1]]),
        "ok": ([2], [2], [[5, 1]], [[0, 0]], [[0, 1]]),
    }[case]
    assert _create_raw(len(args[0]), *args) == _abi.CODES[code]


def test_create_null_pointers():
    lib = _abi.load()
    h = ctypes.c_void_p()
    assert lib.sf_create(1, None, None, None, None, ctypes.byref(h)) == _abi.CODES["SF_ERR_NULL"]
    n = (ctypes.c_int64 * 1)(1)
    # nleaves > 0 but no iremote
    assert lib.sf_create(1, n, n, None, None, ctypes.byref(h)) == _abi.CODES["SF_ERR_NULL"]
    assert lib.sf_create(1, n, n, None, None, None) == _abi.CODES["SF_ERR_NULL"]


def test_too_large_leaf_space_is_rejected():
    code = _create_raw(1, [1], [1], [[1 << 40]], [[0]], [[0]])
    assert code == _abi.CODES["SF_ERR_TOO_LARGE"]


FORESTS = [sfgen.fig2(), sfgen.cfg1_plain_tiny()] + [sfgen.random_forest(s, P, 30, 40) for s, P in
                                                       [(31, 1), (32, 4), (33, 9)]]


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
def test_layout_matches_oracle(f):
    sf = StarForest.from_forest(f)
    ro, lo = oracle.layout(f)
    assert np.array_equal(sf.rootoff, ro) and np.array_equal(sf.leafoff, lo)


@pytest.mark.parametrize("f", FORESTS, ids=lambda f: f.name)
def test_analysis_statistics(f):
    info = StarForest.from_forest(f).analyze().info()
    L, R = npref.edge_arrays(f)
    deg = np.bincount(R, minlength=info["nroots_total"])
    assert info["nedges"] == len(L)
    assert info["max_in_degree"] == (deg.max() if len(deg) else 0)
    assert info["connected_roots"] == int((deg > 0).sum())
    assert info["multi_roots"] == int((deg > 1).sum())
    assert info["multi_edges"] == int(deg[deg > 1].sum())
    assert info["has_dup_roots"] == int(deg.max() > 1)
    # every edge lands in exactly one run class and one root-major class
    assert info["edges_both_pattern"] + info["edges_one_indexed"] + info["edges_two_indexed"] == len(L)
    assert info["rm_masked_edges"] + info["rm_pairs"] + info["multi_edges"] == len(L)
    rank_of_leaf = np.concatenate([np.full(int(f.nleaves[q]), q) for q in range(f.nranks)]) if len(L) else []
    rr = np.concatenate(f.iremote_rank) if len(L) else []
    assert info["self_edges"] == int(np.sum(np.asarray(rank_of_leaf) == np.asarray(rr)))
    pairs = {(int(a), int(b)) for a, b in zip(rr, rank_of_leaf)}
    assert info["segments"] == len(pairs)
    assert info["analyzed"] == 1 and info["setup_done"] == 0


def test_fig2_analysis_by_hand():
    info = StarForest.from_forest(sfgen.fig2()).analyze().info()
    assert info["nroots_total"] == 9 and info["leaf_extent_total"] == 11
    assert info["max_in_degree"] == 3 and info["multi_roots"] == 2 and info["multi_edges"] == 5
    # (root rank, leaf rank) pairs: (1,0) (0,0) (2,1) (0,1) (0,2) (1,2)
    assert info["segments"] == 6 and info["self_edges"] == 1


def test_halo_is_index_free():
    """3-D halo (Sec. V.B multi-strided sub-blocks): faces and edges become pattern runs;
    only the 1-point corner groups keep indices."""
    f = sfgen.cfg2_halo(128, 2)          # 64^3 owned points per rank, as at full size
    info = StarForest.from_forest(f).analyze().info()
    assert info["runs_3d"] > 0
    corners = info["edges_two_indexed"] + info["edges_one_indexed"]
    assert corners <= f.nranks             # one corner point per rank
    assert info["edges_both_pattern"] >= 0.97 * info["nedges"]


def test_spmv_scatter_patterns():
    """Owned entries are one contiguous run per rank; ghost columns are contiguous on the
    leaf side and need root indices only."""
    f = sfgen.cfg3_spmv(1 << 15, 4)
    info = StarForest.from_forest(f).analyze().info()
    P = f.nranks
    assert info["self_edges"] == f.nroots.sum()
    assert info["edges_both_pattern"] >= f.nroots.sum()
    assert info["edges_two_indexed"] <= 0.05 * info["nedges"]
    assert info["rm_masked_runs"] >= P


def test_header_constants_match_the_binding():
    import re
    from paper_2102_13018_gb300 import _abi
    text = open(_abi.HEADER).read()
    for name in ("SF_DEVSTAT_STAGE_TIMEOUT", "SF_DEVSTAT_TILE_REFUSED", "SF_MAX_UNIT_BYTES"):
        m = re.search(r"#define\s+" + name + r"\s+\((\d+) << (\d+)\)|#define\s+" + name + r"\s+(\d+)", text)
        assert m, name
        val = int(m.group(1)) << int(m.group(2)) if m.group(1) else int(m.group(3))
        assert getattr(_abi, name) == val, name


def _tile_rule(work, lo, hi, target=4096):
    """Smallest power of two in [lo, hi] giving at most `target` tiles (hi if none does)."""
    s = lo
    while s < hi and -(-work // s) > target:
        s *= 2
    return s


@pytest.mark.parametrize("n_per_rank", [100, 1 << 16, 300_000, 1 << 22])
def test_tile_sizes_follow_the_forest_size(n_per_rank):
    """Tiles shrink with the forest so that a launch has about 4096 of them (powers of two,
    512..4096 edges; 256..1024 fold blocks), keeping small forests spread over every SM."""
    f = sfgen.one_to_one(3, 4, n_per_rank)
    info = StarForest.from_forest(f).analyze().info()
    E = info["nedges"]
    assert info["ts_tile_edges"] == _tile_rule(E, 512, 4096)
    assert info["rm_tile_edges"] == _tile_rule(info["rm_masked_edges"] + info["rm_pairs"], 512, 4096)
    assert info["rm_tile_blocks"] == _tile_rule(info["rm_chunks"], 256, 1024)
    if E >= 4096 * 4096:
        assert info["ts_tile_edges"] == 4096


def test_halo_and_spmv_tile_sizes():
    """The 256^3 halo (1.2M ghost edges) gets 512-edge tiles; the 2^24-root SpMV scatter keeps
    the 4096-edge maximum."""
    halo = StarForest.from_forest(sfgen.cfg2_halo()).analyze().info()
    assert halo["ts_tile_edges"] == 512 and halo["rm_tile_edges"] == 512 and halo["rm_tile_blocks"] == 256


def test_operations_before_setup_fail_cleanly():
    lib = _abi.load()
    sf = StarForest.from_forest(sfgen.fig2())
    u = _abi.sf_unit(_abi.SF_FP64, 1)
    buf = ctypes.c_void_p(64)
    assert lib.sf_bcast_begin(sf._h, u, buf, buf, 0, None) == _abi.CODES["SF_ERR_STATE"]
    assert lib.sf_reduce_begin(sf._h, u, buf, buf, 1, None) == _abi.CODES["SF_ERR_STATE"]
    assert lib.sf_bcast_end(sf._h, u, buf, buf, 0, None) == _abi.CODES["SF_ERR_NO_PENDING"]
    assert lib.sf_set_mode(sf._h, 7) == _abi.CODES["SF_ERR_ARG"]
    assert lib.sf_set_path(sf._h, -1) == _abi.CODES["SF_ERR_ARG"]
    assert lib.sf_destroy(None) == 0


def test_setup_without_a_device_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sf = StarForest.from_forest(sfgen.fig2())
    with pytest.raises(SFError) as ei:
        sf.setup(stream=0)
    assert ei.value.name == "SF_ERR_CUDA"


def test_embedded_root_and_leaf_forests_keep_the_layout():
    """Sec. III.C: removing edges renumbers nothing; Fig. 2 with root (1,0) (unit 3) selected
    keeps edges e1, e2, e8; with leaf units {0, 5} selected keeps e0 and e5."""
    sf = StarForest.from_forest(sfgen.fig2())
    er = sf.embedded_roots([3])
    assert np.array_equal(er.rootoff, sf.rootoff) and np.array_equal(er.leafoff, sf.leafoff)
    info = er.analyze().info()
    assert info["nedges"] == 3 and info["max_in_degree"] == 3 and info["connected_roots"] == 1
    el = sf.embedded_leaves([0, 5])
    assert np.array_equal(el.leafoff, sf.leafoff)
    assert el.analyze().info()["nedges"] == 2
    with pytest.raises(SFError) as e:
        sf.embedded_roots([9])
    assert e.value.name == "SF_ERR_RANGE"
    assert sf.embedded_roots([]).analyze().info()["nedges"] == 0


def test_compose_checks_layouts_and_degrees():
    a = StarForest.from_forest(sfgen.fig2())          # leaf extents 4, 4, 3
    with pytest.raises(SFError) as e:
        a.compose(a)                                   # A's leaf space (4,4,3) is not A's roots (3,4,2)
    assert e.value.name == "SF_ERR_ARG"
    with pytest.raises(SFError) as e:
        a.compose_inverse(a)                           # shared leaves, but A's root (1,0) has 3 leaves
    assert e.value.name == "SF_ERR_ARG"
    # B with roots = A's leaf space: rank q owns extent(q) roots, one leaf per root, identity
    ext = [4, 4, 3]
    b = sfgen.Forest(3, np.array(ext), np.array(ext), [None] * 3,
                     [np.full(n, q, np.int32) for q, n in enumerate(ext)],
                     [np.arange(n, dtype=np.int64) for n in ext])
    ab = a.compose(StarForest.from_forest(b))
    info = ab.analyze().info()
    assert info["nedges"] == 10                       # rank 1's isolated leaf 2 drops out
    assert ab.rootoff.tolist() == a.rootoff.tolist()


def _diagonal_chunks_numpy(f, block=64, min_chunk=8, min_roots=1024):
    """The diagonal-chunk rule restated with numpy: in each chunk of 32 root units, among
    roots of in-degree 1..block, the offset leaf - root shared by the most roots (the smallest
    such offset on a tie) is the chunk's, if at least min_chunk roots share it; those roots
    are covered.  The plan exists when at least min_roots roots, and half of the connected
    roots, are covered.  Returns (covered mask, in-degrees, number of chunks) or None."""
    L, R = npref.edge_arrays(f)
    NR = int(np.sum(f.nroots))
    deg = np.bincount(R, minlength=NR)
    ok = (deg[R] >= 1) & (deg[R] <= block)
    d, r = (L - R)[ok], R[ok]
    covered = np.zeros(NR, bool)
    good_chunks = []
    for c in np.unique(r // 32):
        sel = (r // 32) == c
        vals, counts = np.unique(d[sel], return_counts=True)
        best = int(np.argmax(counts))           # first maximum: the smallest offset
        if counts[best] >= min_chunk:
            covered[r[sel][d[sel] == vals[best]]] = True
            good_chunks.append(c)
    if covered.sum() < min_roots or 2 * covered.sum() < (deg > 0).sum():
        return None
    return covered, deg, good_chunks[-1] - good_chunks[0] + 1


@pytest.mark.parametrize("f", [sfgen.owned_plus_ghosts(5), sfgen.owned_plus_ghosts(6, keep=0.6),
                               sfgen.cfg3_spmv(1 << 15, 4), sfgen.zipf_forest(8, 1, 20000, 3000, 4),
                               sfgen.cfg1_plain_tiny()], ids=lambda f: f.name)
def test_diagonal_chunk_plan_statistics(f):
    info = StarForest.from_forest(f).analyze().info()
    want = _diagonal_chunks_numpy(f)
    if want is None:
        assert info["dg_chunks"] == 0 and info["dg_roots"] == 0 and info["dg_rest_roots"] == 0
        return
    covered, deg, nchunks = want
    assert info["dg_chunks"] == nchunks
    assert info["dg_roots"] == int(covered.sum())
    assert info["dg_extra_leaves"] == int((deg[covered] - 1).sum())
    assert info["dg_list_roots"] == int((deg[covered] >= 3).sum())
    assert info["dg_rest_roots"] == int(((deg > 0) & ~covered).sum())


def test_diagonal_chunks_cover_the_spmv_scatter_and_leave_corner_cases_to_the_rest():
    spmv = StarForest.from_forest(sfgen.cfg3_spmv(1 << 15, 4)).analyze().info()
    assert spmv["dg_roots"] == spmv["connected_roots"] and spmv["dg_rest_roots"] == 0
    mix = StarForest.from_forest(sfgen.owned_plus_ghosts(5)).analyze().info()
    # roots without an owned leaf, roots of the shuffled rank and roots of more than 64 leaves
    assert mix["dg_rest_roots"] > 0 and mix["dg_list_roots"] > 0
    assert 0 < mix["dg_roots"] < mix["connected_roots"]


def test_tuning_knobs_validate_and_report_before_setup():
    """The launch-shape and plan setters check their arguments; before the setup pass builds a
    diagonal-chunk plan a forest reports the root-major Reduce plan whatever is selected."""
    lib = _abi.load()
    sf = StarForest.from_forest(sfgen.fig2())
    for bad in (-1, 4, 99):
        assert lib.sf_set_reduce_plan(sf._h, bad) == _abi.CODES["SF_ERR_ARG"]
    for bad in (1, 3, 32):
        assert lib.sf_set_vector_bytes(sf._h, bad) == _abi.CODES["SF_ERR_ARG"]
    assert lib.sf_set_reduce_plan(None, 0) == _abi.CODES["SF_ERR_NULL"]
    for plan in ("auto", "root_major", "diagonal", "diagonal_staged"):
        t = sf.set_reduce_plan(plan).tuning()
        assert t["reduce_plan"] == "root_major"
        assert t["path"] == "fused" and t["mode"] == "deterministic" and t["vector_bytes"] == 0
    sf.set_vector_bytes(8)
    assert sf.tuning()["vector_bytes"] == 8


def test_header_enums_match_the_binding():
    import re
    text = open(_abi.HEADER).read()
    for prefix in ("SF_PLAN_", "SF_PATH_", "SF_MODE_"):
        found = dict(re.findall(r"\b(" + prefix + r"[A-Z_]+)\s*=\s*(\d+)", text))
        assert found, prefix
        for name, val in found.items():
            assert getattr(_abi, name) == int(val), name
