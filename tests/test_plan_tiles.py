"""The root-major plan's chunk tiles against the shared-memory stages of the kernels that
read them.  The library's own setup pass (sf_setup.cpp, compiled here with g++) builds plans
for varied forests; for both chunk-tile lists -- the general Reduce kernel's and the
one-vector (NV1) kernel's, of every root and of the roots the diagonal chunks leave out --
every tile must fit its kernel's stage (block records and leaf entries, widened as the kernel
widens them), describe exactly the leaf span of its blocks, and the tiles must cover every
fold block exactly once.  The tiles of the staged diagonal-chunk Reduce are checked the same
way: every bulk copy aligned and inside its array and its shared-memory area.  CPU only."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2102_13018_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")

CHECK = r'''
#include <algorithm>
#include <cstdio>
#include <cstdint>
#include <vector>
#include "sf_host.h"
using namespace sfgb;

static uint64_t state = 0x2545F4914F6CDD1Dull;
static uint64_t next64() { state ^= state << 13; state ^= state >> 7; state ^= state << 17; return state; }
static int64_t below(int64_t n) { return int64_t(next64() % uint64_t(n)); }

// check one chunk-tile list against a stage of `stage_leaves` leaf entries
static int check_list(const HostPlan &p, const std::vector<RmTile> &tiles, int stage_leaves, const char *name) {
  const int64_t nblocks = int64_t(p.blocks.size());
  std::vector<std::pair<int64_t, int64_t>> spans;
  for (const RmTile &t : tiles) {
    if (t.kind != T_CHUNKS) continue;
    if (t.cnt < 1 || t.cnt > RM_TILE_CHUNKS || t.a < 0 || t.a + t.cnt > nblocks) {
      std::printf("%s: bad block range a=%d cnt=%d of %lld\n", name, t.a, t.cnt, (long long)nblocks);
      return 1;
    }
    const int64_t r0 = t.a & ~1, r1 = (int64_t(t.a) + t.cnt + 2) & ~int64_t(1);
    const int64_t l0 = t.k0 & ~3, l1 = (t.e1 + 3) & ~int64_t(3);
    if (r1 - r0 > RM_STAGE_RECS || l1 - l0 > stage_leaves) {
      std::printf("%s: tile a=%d cnt=%d stages %lld records / %lld leaves (limits %d / %d)\n", name, t.a, t.cnt,
                  (long long)(r1 - r0), (long long)(l1 - l0), RM_STAGE_RECS, stage_leaves);
      return 1;
    }
    if (t.k0 != p.block_recs[t.a].e0 || t.e1 != p.block_recs[t.a + t.cnt].e0) {
      std::printf("%s: tile a=%d leaf span [%d, %lld) is not its blocks' span\n", name, t.a, t.k0, (long long)t.e1);
      return 1;
    }
    spans.push_back({t.a, t.a + t.cnt});
  }
  std::sort(spans.begin(), spans.end());
  int64_t next = 0;
  for (auto &s : spans) {
    if (s.first != next) { std::printf("%s: blocks [%lld, %lld) not covered once\n", name, (long long)next, (long long)s.first); return 1; }
    next = s.second;
  }
  if (next != nblocks) { std::printf("%s: covers %lld of %lld blocks\n", name, (long long)next, (long long)nblocks); return 1; }
  return 0;
}

// The staged diagonal-chunk kernel's copies for every tile and unit width: the same spans the
// kernel forms (dg_spans), checked to start 16-byte aligned, to stay inside the root, leaf and x
// arrays and inside the stage's areas (leaf and x areas: the span's bytes plus 32 spare); the
// tiles must cover every chunk that has a coded root exactly once, with one delta, at most
// DG_TILE_CHUNKS chunks and DG_TILE_XCAP x entries, and `full` must say whether every root of
// the tile below the last root is coded.
static int64_t dg_tiles_checked = 0;
static int check_dg(const HostPlan &p, int64_t NR, int64_t leaf_units, const char *name) {
  const DiagHost &d = p.dg;
  dg_tiles_checked += int64_t(d.tiles.size());
  const int64_t nch = int64_t(d.chunks.size());
  std::vector<int> seen(nch, 0);
  for (const DgTile &t : d.tiles) {
    if (t.n < 1 || t.n > DG_TILE_CHUNKS || t.c < 0 || t.c + t.n > nch || t.xend - t.xbeg > DG_TILE_XCAP ||
        t.xbeg != d.chunks[t.c].xoff) {
      std::printf("%s: bad tile c=%d n=%d x=[%d,%d)\n", name, t.c, t.n, t.xbeg, t.xend);
      return 1;
    }
    bool full = true;
    for (int32_t k = t.c; k < t.c + t.n; ++k) {
      seen[k]++;
      if (d.chunks[k].delta != t.delta) { std::printf("%s: tile mixes deltas\n", name); return 1; }
      for (int lane = 0; lane < 32; ++lane) {
        const int64_t u = (d.c0 + k) * 32 + lane;
        const uint32_t code = ((lane < 16 ? d.chunks[k].lo : d.chunks[k].hi) >> (2 * (lane & 15))) & 3u;
        if (u < NR && !code) full = false;
        if (u >= NR && code) { std::printf("%s: code beyond the last root\n", name); return 1; }
        if (code && (u + t.delta < 0 || u + t.delta >= leaf_units)) { std::printf("%s: diagonal leaf out of range\n", name); return 1; }
      }
    }
    if (bool(t.full) != full) { std::printf("%s: full flag wrong\n", name); return 1; }
    // every list root's list (a negative header, then its other leaves) inside [lbeg, lend)
    for (int32_t k = t.c, xi = t.xbeg; k < t.c + t.n; ++k)
      for (int lane = 0; lane < 32; ++lane) {
        const uint32_t code = ((lane < 16 ? d.chunks[k].lo : d.chunks[k].hi) >> (2 * (lane & 15))) & 3u;
        if (code < DG_PAIR) continue;
        if (code == DG_LIST) {
          const int32_t o = d.x[xi];
          if (o < t.lbeg || o >= t.lend || d.lists[o] >= 0) { std::printf("%s: list outside its tile\n", name); return 1; }
          const int32_t h = -1 - d.lists[o], n = (h & 0xffff) + (h >> 16);
          if (o + 1 + n > t.lend) { std::printf("%s: list runs past its tile\n", name); return 1; }
          for (int32_t q = 1; q <= n; ++q)
            if (d.lists[o + q] < 0 || d.lists[o + q] >= leaf_units) { std::printf("%s: bad list entry\n", name); return 1; }
        }
        ++xi;
      }
    {
      const int64_t lslo = (int64_t(t.lbeg) * 4) & ~int64_t(15);
      const int64_t lshi = (int64_t(t.lend) * 4 + 15) & ~int64_t(15);
      const bool staged = t.lend > t.lbeg && t.lend - t.lbeg <= DG_TILE_LCAP;
      if (t.lbeg < 0 || t.lend < t.lbeg || t.lend > int64_t(d.lists.size()) ||
          (staged && (lshi > int64_t(d.lists.size()) * 4 + 16 || lshi - lslo > DG_TILE_LCAP * 4 + 32))) {
        std::printf("%s: list span [%d, %d) out of bounds\n", name, t.lbeg, t.lend);
        return 1;
      }
    }
    const int64_t xend_chunks = t.c + t.n < nch ? d.chunks[t.c + t.n].xoff : int64_t(d.x.size());
    if (t.xend != xend_chunks) { std::printf("%s: tile x span is not its chunks' span\n", name); return 1; }
    for (int VB : {2, 4, 8, 16}) {
      const int64_t R = int64_t(DG_TILE_CHUNKS) * 32 * VB;
      const int64_t u0 = (d.c0 + t.c) * 32;
      const int64_t n = std::min<int64_t>(int64_t(t.n) * 32, NR - u0);
      const int64_t rstage = (n * VB) & ~int64_t(15);
      const int64_t L0 = u0 + t.delta, leaf_bytes = leaf_units * VB;
      int64_t llo = std::max<int64_t>(0, (L0 * VB) & ~int64_t(15));
      int64_t lhi = std::min<int64_t>(((L0 + n) * VB + 15) & ~int64_t(15), leaf_bytes & ~int64_t(15));
      if (lhi < llo) lhi = llo;
      const int64_t xlo = (int64_t(t.xbeg) * 4) & ~int64_t(15);
      const int64_t xhi = t.xend == t.xbeg ? xlo : ((int64_t(t.xend) * 4 + 15) & ~int64_t(15));
      const int64_t xbytes = int64_t(d.x.size()) * 4 + 16;   // the plan blob keeps 16 bytes after an array
      const bool ok = n > 0 && rstage >= 0 && rstage <= R && u0 * VB + rstage <= NR * VB && (u0 * VB) % 16 == 0 &&
                      llo % 16 == 0 && lhi % 16 == 0 && llo >= 0 && lhi <= leaf_bytes && lhi - llo <= R + 32 &&
                      xlo % 16 == 0 && xhi % 16 == 0 && xhi <= xbytes && xhi - xlo <= DG_TILE_XCAP * 4 + 32 &&
                      t.n * 16 <= DG_TILE_CHUNKS * 16;
      if (!ok) {
        std::printf("%s: tile c=%d VB=%d spans out of bounds (roots %lld, leaves [%lld,%lld) of %lld, x [%lld,%lld))\n",
                    name, t.c, VB, (long long)rstage, (long long)llo, (long long)lhi, (long long)leaf_bytes,
                    (long long)xlo, (long long)xhi);
        return 1;
      }
    }
  }
  for (int64_t k = 0; k < nch; ++k)
    if (seen[k] != int(bool(d.chunks[k].lo | d.chunks[k].hi))) {
      std::printf("%s: chunk %lld covered %d times\n", name, (long long)k, seen[k]);
      return 1;
    }
  return 0;
}

// forest from per-leaf global roots (ranks split evenly, ilocal identity)
static int run(const char *name, int P, int64_t nroots_total, const std::vector<int64_t> &root_of_leaf) {
  std::vector<int64_t> nroots(P, nroots_total / P), nleaves(P, 0);
  for (int p = 0; p < int(nroots_total % P); ++p) nroots[p]++;
  std::vector<int64_t> rootoff(P + 1, 0);
  for (int p = 0; p < P; ++p) rootoff[p + 1] = rootoff[p] + nroots[p];
  const int64_t E = int64_t(root_of_leaf.size());
  for (int64_t e = 0; e < E; ++e) nleaves[e * P / E]++;
  std::vector<std::vector<sf_node>> rem(P);
  int64_t e = 0;
  for (int q = 0; q < P; ++q)
    for (int64_t i = 0; i < nleaves[q]; ++i, ++e) {
      const int64_t g = root_of_leaf[e];
      const int r = int(std::upper_bound(rootoff.begin(), rootoff.end(), g) - rootoff.begin()) - 1;
      rem[q].push_back(sf_node{r, g - rootoff[r]});
    }
  std::vector<const sf_node *> rp(P);
  std::vector<const int64_t *> il(P, nullptr);
  for (int q = 0; q < P; ++q) rp[q] = rem[q].data();
  Graph g;
  HostPlan plan;
  sf_info info{};
  if (build_graph(P, nroots.data(), nleaves.data(), il.data(), rp.data(), g) || analyze(g, plan, info)) {
    std::printf("%s: setup failed\n", name);
    return 1;
  }
  int bad = check_list(plan, plan.rm_fold_tiles, RM_STAGE_LEAVES, name) +
            check_list(plan, plan.rm_fold_nv1_tiles, RM_STAGE_LEAVES_NV1, name) +
            check_dg(plan, info.nroots_total, info.leaf_extent_total, name);
  if (plan.rest)   // the root-major plan of the roots the diagonal chunks leave out
    bad += check_list(*plan.rest, plan.rest->rm_fold_tiles, RM_STAGE_LEAVES, name) +
           check_list(*plan.rest, plan.rest->rm_fold_nv1_tiles, RM_STAGE_LEAVES_NV1, name);
  return bad;
}

int main() {
  int bad = 0;
  for (int t = 0; t < 12 && !bad; ++t) {   // uniform random forests of many sizes
    const int64_t N = 1 + below(int64_t(1) << (4 + t)), E = below(int64_t(1) << (5 + t));
    std::vector<int64_t> r(E);
    for (auto &x : r) x = below(N);
    bad += run("uniform", 1 + int(below(8)), N, r);
  }
  for (int64_t n : {1, 63, 64, 65, 4095, 4096, 4097, 8192, 8193, 100000, 300000}) {   // one heavy star
    std::vector<int64_t> r(n, 0);
    bad += run("star", 1, 3, r);
  }
  {   // a few heavy roots inside many light ones (Zipf-like skew)
    std::vector<int64_t> r;
    for (int64_t i = 0; i < 400000; ++i) r.push_back(below(5) == 0 ? below(4) : below(200000));
    bad += run("skew", 4, 200000, r);
  }
  {   // degree ladder: root k has (k % 200) + 1 leaves, crossing every block boundary
    std::vector<int64_t> r;
    for (int64_t k = 0; k < 3000; ++k)
      for (int64_t j = 0; j <= k % 200; ++j) r.push_back(k);
    for (int64_t i = int64_t(r.size()) - 1; i > 0; --i) std::swap(r[i], r[below(i + 1)]);
    bad += run("ladder", 3, 3000, r);
  }
  {   // more than 2M fold blocks, so tiles take their largest sizes (1024 blocks, the full
      // leaf caps), plus one heavy root whose tiles reach the leaf cap
    std::vector<int64_t> r;
    const int64_t N = 2100000;
    for (int64_t k = 1; k < N; ++k) { r.push_back(k); r.push_back(k); }
    for (int64_t j = 0; j < 40000; ++j) r.push_back(0);
    for (int64_t i = int64_t(r.size()) - 1; i > 0; --i) std::swap(r[i], r[below(i + 1)]);
    bad += run("large", 8, N, r);
  }
  {   // every root owns the leaf at its own position (diagonal chunks), plus ghosts and heavy
      // roots of up to 9000 leaves left to the root-major plan of the rest
    std::vector<int64_t> r;
    const int64_t N = 600000;
    for (int64_t k = 0; k < N; ++k) r.push_back(k);
    for (int64_t j = 0; j < 200000; ++j) r.push_back(below(N));
    for (int64_t h = 0; h < 30; ++h)
      for (int64_t j = 0; j < 300 * h; ++j) r.push_back(h * 1000);
    bad += run("diagonal", 6, N, r);
  }
  {   // diagonal leaves at a negative offset (leaf = root - 37) on odd-sized ranks, ghosts after
    std::vector<int64_t> r;
    const int64_t N = 100003;
    for (int64_t k = 0; k < 37; ++k) r.push_back(below(N));
    for (int64_t k = 0; k < N; ++k) r.push_back(k);
    for (int64_t j = 0; j < 30001; ++j) r.push_back(below(N));
    bad += run("diagonal_shifted", 7, N, r);
  }
  {   // negative offset (leaf = root - 37): the first roots have no diagonal leaf, so a tile's
      // leaf span would start before the leaf array
    std::vector<int64_t> r;
    const int64_t N = 70001;
    for (int64_t k = 0; k < N; ++k) r.push_back(k + 37 < N ? k + 37 : below(N));
    for (int64_t j = 0; j < 9001; ++j) r.push_back(below(N));
    bad += run("diagonal_negative", 3, N, r);
  }
  {   // one-to-one: no fold blocks at all
    std::vector<int64_t> r(50000);
    for (int64_t i = 0; i < 50000; ++i) r[i] = i;
    bad += run("one_to_one", 5, 50000, r);
  }
  if (dg_tiles_checked < 100) { std::printf("only %lld diagonal tiles\n", (long long)dg_tiles_checked); bad++; }
  std::printf("%s\n", bad ? "FAIL" : "OK");
  return bad != 0;
}
'''


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_chunk_tiles_fit_their_kernels_stages(tmp_path):
    src = tmp_path / "tile_check.cpp"
    src.write_text(CHECK)
    exe = tmp_path / "tile_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", INCLUDE, "-I", CSRC, str(src),
                    os.path.join(CSRC, "sf_setup.cpp"), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout[-2000:]
