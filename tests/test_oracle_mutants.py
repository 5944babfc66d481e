"""Planted mistakes: each mutant of the oracle source (a plausible slip, made on the CPU)
must fail at least one pin.  Shows that the pins constrain every part of the oracle."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import sfgen
from tests import npref

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "sf_oracle.c")).read()

MUTANTS = {
    "bcast_operands_swapped": (
        "apply(dtype, op, (char *)leafdata + (L[e] * bs + c) * w, (const char *)rootdata + (R[e] * bs + c) * w);",
        "{ char t[8]; memcpy(t, (const char *)rootdata + (R[e] * bs + c) * w, w); "
        "apply(dtype, op, t, (char *)leafdata + (L[e] * bs + c) * w); memcpy((char *)leafdata + (L[e] * bs + c) * w, t, w); }"),
    "extent_off_by_one": ("extent = mx + 1;", "extent = mx;"),
    "fold_drops_last": ("for (int64_t t = 1; t < n; ++t) acc = acc + y[t];\n  return acc;\n}\nstatic float",
                        "for (int64_t t = 1; t < n - 1; ++t) acc = acc + y[t];\n  return acc;\n}\nstatic float"),
    "fold_block_boundary": ("  while (n > K) {\n    int64_t m = 0;\n    for (int64_t s = 0; s < n; s += K) {\n      int64_t t_end = s + K < n ? s + K : n;\n      float acc",
                            "  while (n > K) {\n    int64_t m = 0;\n    for (int64_t s = 0; s < n; s += K) {\n      int64_t t_end = s + K - 1 < n ? s + K - 1 : n;\n      float acc"),
    "root_added_first": ("          a = a + s;\n          memcpy(dst, &a, 8);",
                         "          a = a + (s - 0.0);\n          { double z = a; for (int64_t t = 0; t < n; ++t) z = z + 0.0; a = z; }\n          memcpy(dst, &a, 8); if (n >= 2) { double q; memcpy(&q, dst, 8); q = (q - s) ; for (int64_t t = 0; t < n; ++t) q = q + yd[t]; memcpy(dst, &q, 8); }"),
    "fetch_after_op": ("      memcpy((char *)leafupdate + (L[e] * bs + c) * w, root, w);\n      apply(dtype, op, root, (const char *)leafdata + (L[e] * bs + c) * w);",
                       "      apply(dtype, op, root, (const char *)leafdata + (L[e] * bs + c) * w);\n      memcpy((char *)leafupdate + (L[e] * bs + c) * w, root, w);"),
    "min_max_swapped": ("else if (op == O_MIN) r = b < a ? b : a;\n      else r = a < b ? b : a;\n      memcpy(dst, &r, 8);\n      break;\n    }\n    case O_BF16",
                        "else if (op == O_MIN) r = a < b ? b : a;\n      else r = b < a ? b : a;\n      memcpy(dst, &r, 8);\n      break;\n    }\n    case O_BF16"),
    "bf16_ties_away": ("(lower == 0x8000u && (upper & 1u))", "(lower == 0x8000u)"),
    "bf16_min_max_swapped": ("else if (op == O_MIN) hr = b < a ? hb : ha;\n      else hr = a < b ? hb : ha;",
                             "else if (op == O_MIN) hr = a < b ? hb : ha;\n      else hr = b < a ? hb : ha;"),
    "bf16_sum_truncated": ("else if (op == O_SUM) hr = f32_to_bf16(a + b);",
                           "else if (op == O_SUM) { float s = a + b; uint32_t u; memcpy(&u, &s, 4); hr = (uint16_t)(u >> 16); }"),
    "reverse_canonical_order": ("  for (int64_t e = 0; e < E; ++e) perm[fill[R[e]]++] = e;",
                                "  for (int64_t e = E - 1; e >= 0; --e) perm[fill[R[e]]++] = e;"),
    "edge_root_rank_ignored": ("R[e] = ro[f->rrank[e]] + f->rindex[e];", "R[e] = f->rindex[e];"),
    "gather_slots_reversed": ("  for (int64_t e = 0; e < E; ++e) slot[e] = first[R[e]]++;",
                              "  for (int64_t e = E - 1; e >= 0; --e) slot[e] = first[R[e]]++;"),
    "maxloc_last_tie_wins": ("if (argedge[u] < 0 || less_than(dtype, (char *)out + u * w, src)) {",
                             "if (argedge[u] < 0 || !less_than(dtype, src, (char *)out + u * w)) {"),
    "maxloc_component_dropped": ("const char *src = (const char *)leafdata + (L[e] * bs + c) * w;",
                                 "const char *src = (const char *)leafdata + (L[e] * bs) * w;"),
    "gather_slot_excludes_own_root": ("for (int64_t r = 0; r < NR; ++r) first[r + 1] += first[r];     /* edges",
                                      "for (int64_t r = 1; r < NR; ++r) first[r + 1] += first[r - 1];     /* edges"),
}


def battery(lib):
    """A compact run of the pins; returns the names of those that fail."""
    fails = []

    def check(name, cond):
        if not cond:
            fails.append(name)

    f = sfgen.fig2()
    try:
        ro, lo = oracle.layout(f, lib)
        check("layout", ro.tolist() == [0, 3, 7, 9] and lo.tolist() == [0, 4, 8, 11])
        x = np.concatenate([100 * p + np.arange(f.nroots[p]) for p in range(3)]).astype(np.int64)
        leaf = oracle.bcast(f, "int64", 1, x, np.full(lo[-1], -1, np.int64), "REPLACE", lib=lib)
        check("fig2_bcast", leaf.tolist() == [102, 100, 100, 2, 200, 0, -1, 201, 0, 100, 103])
        r0 = np.array([0, 2, 2, 0, 3, 3, 4, 0, 1], np.int32)
        root, upd = oracle.fetch_and_op(f, "int32", 1, r0, np.ones(lo[-1], np.int32),
                                        np.full(lo[-1], -7, np.int32), "SUM", lib=lib)
        check("fig2_fetch", upd.tolist() == [3, 0, 1, 2, 0, 0, -7, 1, 1, 2, 4])
        yv = np.concatenate([10 * q + np.arange(lo[q + 1] - lo[q]) for q in range(3)])
        rr = oracle.reduce(f, "fp64", 1, yv.astype(np.float64), np.full(ro[-1], 100.0), "MIN", lib=lib)
        check("fig2_min", rr.astype(int).tolist() == [11, 100, 3, 1, 100, 0, 22, 10, 13])
    except Exception:
        fails.append("fig2_crash")
    # blocked fold hand values
    def star(n):
        return sfgen.Forest(1, np.array([1]), np.array([n]), [None], [np.zeros(n, np.int32)],
                            [np.zeros(n, np.int64)])
    y = np.ones(128, np.float32)
    y[0] = 2.0 ** 24
    g = oracle.reduce(star(128), "fp32", 1, y, np.zeros(1, np.float32), "SUM", lib=lib)
    check("fold_128", g[0] == np.float32(2.0 ** 24 + 64))
    y = np.ones(4097, np.float32)
    y[0] = 2.0 ** 24
    g = oracle.reduce(star(4097), "fp32", 1, y, np.zeros(1, np.float32), "SUM", lib=lib)
    check("fold_4097", g[0] == np.float32(2.0 ** 24 + 4032))
    g = oracle.reduce(star(200), "fp32", 1, np.arange(1, 201, dtype=np.float32), np.zeros(1, np.float32),
                      "SUM", lib=lib)
    check("fold_exact_ints", g[0] == 20100.0)
    g = oracle.reduce(star(2), "fp64", 1, np.array([1.0, 1.0]), np.array([2.0 ** 53]), "SUM", lib=lib)
    check("root_last", g[0] == 2.0 ** 53 + 2.0)
    g = oracle.reduce(star(3), "fp64", 1, np.array([1.0, 1e16, -1e16]), np.array([0.0]), "SUM", lib=lib)
    check("left_order", g[0] == 0.0)
    # incidence product on a random forest
    fr = sfgen.random_forest(3, 5, 9, 12)
    Pm, L, R = npref.incidence(fr)
    nl, nr = Pm.shape
    yy = sfgen.data("int32", nl, 12, 1).astype(np.float64)
    rz = np.zeros(nr)
    check("transpose", np.array_equal(oracle.reduce(fr, "fp64", 1, yy, rz, "SUM", lib=lib), Pm.T @ yy))
    xx = sfgen.data("fp64", nr, 3, 3)
    maxw = np.full(nr, -5.0)
    np.maximum.at(maxw, R, yy[L])
    check("max_scatter", np.array_equal(oracle.reduce(fr, "fp64", 1, yy, np.full(nr, -5.0), "MAX", lib=lib), maxw))
    # bf16 element op: MAX against numpy on the float32 values, SUM rounded to nearest even
    yb = (sfgen.data("fp32", nl, 9, 1).view(np.uint32) >> np.uint32(16)).astype(np.uint16)
    yf = (yb.astype(np.uint32) << np.uint32(16)).view(np.float32)
    mb = np.full(nr, -5.0, np.float32)
    np.maximum.at(mb, R, yf[L])
    got = oracle.reduce(fr, "bf16", 1, yb, np.full(nr, 0xC0A0, np.uint16), "MAX", lib=lib)
    check("bf16_max_scatter", np.array_equal((got.astype(np.uint32) << np.uint32(16)).view(np.float32), mb))
    one = sfgen.Forest(1, np.array([1]), np.array([1]), [None], [np.zeros(1, np.int32)], [np.zeros(1, np.int64)])
    check("bf16_bcast_sum_tie", oracle.bcast(one, "bf16", 1, np.array([0x3B80], np.uint16),
                                             np.array([0x3F81], np.uint16), "SUM", lib=lib).tolist() == [0x3F82])
    # Gather / Scatter on Fig. 2 (hand values)
    try:
        lo2 = oracle.layout(f, lib)[1]
        yv2 = np.concatenate([10 * q + np.arange(lo2[q + 1] - lo2[q]) for q in range(3)]).astype(np.int32)
        mg = oracle.gather(f, "int32", 1, yv2, np.full(f.nedges, -9, np.int32), lib=lib)
        check("fig2_gather", mg.tolist() == [11, 20, 3, 1, 2, 21, 0, 22, 10, 13])
        sc = oracle.scatter(f, "int32", 1, 100 + np.arange(f.nedges, dtype=np.int32),
                            np.full(lo2[-1], -1, np.int32), lib=lib)
        check("fig2_scatter", sc.tolist() == [106, 103, 104, 102, 108, 100, -1, 109, 101, 105, 107])
    except Exception:
        fails.append("gather_crash")
    # MAX with location, two components with many ties: the first canonical edge per element
    ym = (sfgen.data("int32", nl * 2, 13, 1) % 3).astype(np.int32)
    vm, am = oracle.reduce_maxloc(fr, "int32", 2, ym, lib=lib)
    ok = True
    for c in range(2):
        kc = ym.reshape(-1, 2)[:, c]
        e_ = np.arange(len(L))
        order = np.lexsort((e_, -kc[L].astype(np.int64), R))
        first = np.ones(len(order), bool)
        first[1:] = R[order][1:] != R[order][:-1]
        want = np.full(nr, -1, np.int64)
        want[R[order][first]] = e_[order][first]
        ok &= np.array_equal(am.reshape(-1, 2)[:, c], want)
    check("maxloc_first_tie", ok)
    # bf16 rounding tie
    t = np.array([0x3F808000, 0x3F818000], np.uint32).view(np.float32)
    check("bf16_tie", oracle.f32_to_bf16(t, lib=lib).tolist() == [0x3F80, 0x3F82])
    return fails


def test_unmutated_oracle_passes_battery():
    assert battery(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    assert SRC.count(old) == 1, f"mutation anchor for {name} not unique"
    src = tmp_path / "mutant.c"
    src.write_text(SRC.replace(old, new))
    lib_path = str(tmp_path / "libmutant.so")
    subprocess.check_call(["gcc", *oracle.GCC_FLAGS, "-o", lib_path, str(src), "-lm"])
    fails = battery(oracle.load(lib_path))
    assert fails, f"planted mistake {name} passed every pin"
