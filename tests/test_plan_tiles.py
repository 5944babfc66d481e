"""The root-major plan's chunk tiles against the shared-memory stages of the kernels that
read them.  The library's own setup pass (sf_setup.cpp, compiled here with g++) builds plans
for varied forests; for both chunk-tile lists -- the general Reduce kernel's and the
one-vector (NV1) kernel's -- every tile must fit its kernel's stage (block records and leaf
entries, widened as the kernel widens them), describe exactly the leaf span of its blocks,
and the tiles must cover every fold block exactly once.  CPU only."""
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
  return check_list(plan, plan.rm_fold_tiles, RM_STAGE_LEAVES, name) +
         check_list(plan, plan.rm_fold_nv1_tiles, RM_STAGE_LEAVES_NV1, name);
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
  {   // one-to-one: no fold blocks at all
    std::vector<int64_t> r(50000);
    for (int64_t i = 0; i < 50000; ++i) r[i] = i;
    bad += run("one_to_one", 5, 50000, r);
  }
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
