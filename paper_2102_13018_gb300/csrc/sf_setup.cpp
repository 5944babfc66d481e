// sf_setup.cpp -- the setup pass (PetscSFSetUp, Sec. III.A and V.A-B), host only.
//
// 1. Two-sided information (Sec. V.A): edges grouped by root rank p; inside p by leaf rank q
//    with q == p first ("self moved to the head", Sec. V.B); canonical order inside a group.
//    Root-rank-major order keeps the gathers of one root rank close in time (L2 reuse).
// 2. Pattern detection (Sec. V.B): each (p, q) group is cut into runs.  A run whose root and
//    leaf units both follow a multi-strided sub-block start + X*Y*k + X*j + i (contiguous runs
//    are the 1-D case) carries six numbers instead of two index arrays; a run with one side
//    contiguous keeps only the other side's indices.
// 3. Duplicate detection (Sec. V.C): in-degree of every root; runs touching a root of
//    in-degree > 1 are flagged for atomics.
// 4. Root-major plan: single-leaf roots as masked contiguous runs (or explicit pairs),
//    multi-leaf roots in CSR form with their leaves in canonical order, cut into blocks of
//    FOLD_BLOCK leaves for the deterministic fold.
#include <algorithm>
#include <cstring>
#include <new>

#include "sf_host.h"

namespace sfgb {

namespace {
constexpr int64_t kMaxUnits = (int64_t(1) << 31) - 1;
constexpr int64_t kMinPatternEdges = 64;   // smallest run worth a pattern descriptor
constexpr int64_t kMinMaskedSingles = 64;  // smallest masked run in the root-major plan
constexpr int64_t kMaxMaskGap = 32;        // longest stretch of skipped roots inside one
}  // namespace

int build_graph(int32_t P, const int64_t nroots[], const int64_t nleaves[],
                const int64_t *const ilocal[], const sf_node *const iremote[], Graph &g) {
  if (P < 1) return SF_ERR_ARG;
  if (!nroots || !nleaves) return SF_ERR_NULL;
  g = Graph();
  g.P = P;
  try {
    g.nroots.assign(nroots, nroots + P);
    g.nleaves.assign(nleaves, nleaves + P);
    g.rootoff.assign(P + 1, 0);
    g.leafoff.assign(P + 1, 0);
    g.edgeoff.assign(P + 1, 0);
    for (int32_t p = 0; p < P; ++p) {
      if (nroots[p] < 0 || nleaves[p] < 0) return SF_ERR_ARG;
      g.rootoff[p + 1] = g.rootoff[p] + nroots[p];
      g.edgeoff[p + 1] = g.edgeoff[p] + nleaves[p];
      if (g.rootoff[p + 1] > kMaxUnits || g.edgeoff[p + 1] > kMaxUnits) return SF_ERR_TOO_LARGE;
    }
    g.E = g.edgeoff[P];
    g.has_ilocal.assign(P, 0);
    g.ilocal.assign(g.E, 0);
    g.rrank.assign(g.E, 0);
    g.rindex.assign(g.E, 0);
    std::vector<uint64_t> seen;
    for (int32_t q = 0; q < P; ++q) {
      const int64_t n = nleaves[q], e0 = g.edgeoff[q];
      if (n > 0 && (!iremote || !iremote[q])) return SF_ERR_NULL;
      for (int64_t i = 0; i < n; ++i) {
        const sf_node nd = iremote[q][i];
        if (nd.rank < 0 || nd.rank >= P) return SF_ERR_RANGE;
        if (nd.index < 0 || nd.index >= nroots[nd.rank]) return SF_ERR_RANGE;
        g.rrank[e0 + i] = nd.rank;
        g.rindex[e0 + i] = nd.index;
      }
      int64_t extent = n;
      if (ilocal && ilocal[q] && n > 0) {
        int64_t mx = -1;
        for (int64_t i = 0; i < n; ++i) {
          const int64_t l = ilocal[q][i];
          if (l < 0) return SF_ERR_RANGE;
          mx = std::max(mx, l);
        }
        extent = mx + 1;
        if (extent > kMaxUnits) return SF_ERR_TOO_LARGE;
        seen.assign((extent + 63) / 64, 0);
        for (int64_t i = 0; i < n; ++i) {
          const int64_t l = ilocal[q][i];
          uint64_t &w = seen[l >> 6];
          const uint64_t bit = uint64_t(1) << (l & 63);
          if (w & bit) return SF_ERR_DUP_LEAF;
          w |= bit;
          g.ilocal[e0 + i] = l;
        }
        g.has_ilocal[q] = 1;
      }
      g.leafoff[q + 1] = g.leafoff[q] + extent;
      if (g.leafoff[q + 1] > kMaxUnits) return SF_ERR_TOO_LARGE;
    }
  } catch (const std::bad_alloc &) {
    return SF_ERR_ALLOC;
  }
  return SF_SUCCESS;
}

int build_graph_extents(int32_t P, const int64_t nroots[], const int64_t nleaves[], const int64_t *const ilocal[],
                        const sf_node *const iremote[], const int64_t extents[], Graph &g) {
  const int rc = build_graph(P, nroots, nleaves, ilocal, iremote, g);
  if (rc != SF_SUCCESS || !extents) return rc;
  for (int32_t q = 0; q < P; ++q) {
    const int64_t own = g.leafoff[q + 1] - g.leafoff[q];
    if (extents[q] < own) return SF_ERR_RANGE;
  }
  for (int32_t q = 0; q < P; ++q) {
    g.leafoff[q + 1] = g.leafoff[q] + extents[q];
    if (g.leafoff[q + 1] > kMaxUnits) return SF_ERR_TOO_LARGE;
  }
  return SF_SUCCESS;
}

namespace {

struct RunBuilder {
  HostPlan &plan;
  const int64_t *A;   // root units of the group, in group order
  const int64_t *B;   // leaf units
  int64_t n;
  int32_t base_flags;
  std::vector<int64_t> pending;   // positions of edges waiting for a both-indexed run

  void emit(int64_t k, int32_t cnt, int32_t nx, int32_t ny, int64_t rsy, int64_t rsz,
            int64_t lsy, int64_t lsz, int32_t idx_flags) {
    Run r{};
    r.root0 = A[k];
    r.leaf0 = B[k];
    r.rsy = rsy;
    r.rsz = rsz;
    r.lsy = lsy;
    r.lsz = lsz;
    r.n = cnt;
    r.nx = nx;
    r.ny = ny;
    r.flags = base_flags | idx_flags;
    r.idx0 = int64_t(plan.ts_ridx.size());
    if (idx_flags) {
      for (int64_t t = 0; t < cnt; ++t) {
        plan.ts_ridx.push_back(int32_t(A[k + t]));
        plan.ts_lidx.push_back(int32_t(B[k + t]));
      }
    }
    plan.runs.push_back(r);
  }

  void flush_pending() {
    if (pending.empty()) return;
    // pending positions are consecutive in the group
    const int64_t k = pending.front();
    emit(k, int32_t(pending.size()), int32_t(pending.size()), 1, 0, 0, 0, 0,
         RUN_ROOT_IDX | RUN_LEAF_IDX);
    pending.clear();
  }

  bool rows_match(int64_t r0, int64_t nx, int64_t a0, int64_t b0) const {
    for (int64_t t = 0; t < nx; ++t)
      if (A[r0 + t] != a0 + t || B[r0 + t] != b0 + t) return false;
    return true;
  }

  void run() {
    int64_t k = 0;
    while (k < n) {
      // joint multi-strided sub-block, both sides
      int64_t nx = 1;
      while (k + nx < n && A[k + nx] == A[k + nx - 1] + 1 && B[k + nx] == B[k + nx - 1] + 1) ++nx;
      int64_t ny = 1, nz = 1, rsy = 0, lsy = 0, rsz = 0, lsz = 0;
      if (k + 2 * nx <= n) {
        rsy = A[k + nx] - A[k];
        lsy = B[k + nx] - B[k];
        while (k + (ny + 1) * nx <= n && rows_match(k + ny * nx, nx, A[k] + ny * rsy, B[k] + ny * lsy)) ++ny;
        if (ny == 1) rsy = lsy = 0;
        const int64_t plane = nx * ny;
        if (k + 2 * plane <= n) {
          rsz = A[k + plane] - A[k];
          lsz = B[k + plane] - B[k];
          auto plane_ok = [&](int64_t z) {
            for (int64_t j = 0; j < ny; ++j)
              if (!rows_match(k + z * plane + j * nx, nx, A[k] + z * rsz + j * rsy, B[k] + z * lsz + j * lsy))
                return false;
            return true;
          };
          while (k + (nz + 1) * plane <= n && plane_ok(nz)) ++nz;
          if (nz == 1) rsz = lsz = 0;
        }
      }
      const int64_t total = nx * ny * nz;
      if (total >= kMinPatternEdges) {
        flush_pending();
        emit(k, int32_t(total), int32_t(nx), int32_t(ny), rsy, rsz, lsy, lsz, 0);
        k += total;
        continue;
      }
      // one side contiguous, the other indexed
      int64_t lb = 1, la = 1;
      while (k + lb < n && B[k + lb] == B[k + lb - 1] + 1) ++lb;
      while (k + la < n && A[k + la] == A[k + la - 1] + 1) ++la;
      if (lb >= kMinPatternEdges && lb >= la) {
        flush_pending();
        emit(k, int32_t(lb), int32_t(lb), 1, 0, 0, 0, 0, RUN_ROOT_IDX);
        k += lb;
        continue;
      }
      if (la >= kMinPatternEdges) {
        flush_pending();
        emit(k, int32_t(la), int32_t(la), 1, 0, 0, 0, 0, RUN_LEAF_IDX);
        k += la;
        continue;
      }
      pending.push_back(k);
      ++k;
    }
    flush_pending();
  }
};

void push_ts_tiles(std::vector<TsTile> &out, const Run &r, int64_t per) {
  for (int64_t k0 = 0; k0 < r.n; k0 += per) {
    TsTile t{};
    // every value below is a unit index, a stride between two units or an edge offset: all
    // within (-2^31, 2^31) once sizes passed the kMaxUnits checks
    t.root0 = int32_t(r.root0); t.rsy = int32_t(r.rsy); t.rsz = int32_t(r.rsz);
    t.leaf0 = int32_t(r.leaf0); t.lsy = int32_t(r.lsy); t.lsz = int32_t(r.lsz);
    t.idx0 = int32_t(r.idx0); t.rbuf0 = int32_t(r.rbuf0); t.lbuf0 = int32_t(r.lbuf0);
    t.n = r.n; t.nx = r.nx; t.ny = r.ny; t.flags = r.flags;
    const DivMagic dx = div_magic(uint32_t(std::max(r.nx, 1))), dy = div_magic(uint32_t(std::max(r.ny, 1)));
    t.mx = dx.m; t.sx = dx.s; t.my = dy.m; t.sy = dy.s;
    t.k0 = int32_t(k0);
    t.cnt = int32_t(std::min<int64_t>(per, r.n - k0));
    out.push_back(t);
  }
}

}  // namespace

void cut_ts_tiles(const HostPlan &plan, int32_t per, std::vector<TsTile> &out) {
  out.clear();
  for (const Run &r : plan.runs) push_ts_tiles(out, r, per);
}

namespace {

// Smallest power of two in [lo, hi] that splits `work` into at most TILE_TARGET tiles (hi if
// none does).
int32_t tile_size(int64_t work, int32_t lo, int32_t hi) {
  const int64_t want = (work + TILE_TARGET - 1) / TILE_TARGET;
  int64_t s = lo;
  while (s < want && s < hi) s *= 2;
  return int32_t(std::min<int64_t>(s, hi));
}

RmTile rm_tile(int32_t kind, int32_t a, int32_t k0, int32_t cnt) {
  RmTile t{};
  t.kind = kind; t.a = a; t.k0 = k0; t.cnt = cnt;
  return t;
}

// Root-major plan (Sec. V.B, extended): single-leaf roots as masked contiguous runs or explicit
// pairs, multi-leaf roots in CSR form with their leaves in canonical order, cut into fold blocks,
// and the tile lists of the root-major kernels.  Only edges into roots with deg[r] > 0 take part
// (deg holds the in-degree of every root, or 0 for a root the plan leaves out).
void build_rm(int64_t NR, int64_t E, const std::vector<int64_t> &rootu, const std::vector<int64_t> &leafu,
              const std::vector<int32_t> &deg, HostPlan &plan, int32_t *rm_per_out, int32_t *ch_per_out) {
  // multi roots: CSR of leaves in canonical order
  std::vector<int32_t> mid(NR, -1);
  int32_t M = 0;
  int64_t multi_edges = 0;
  for (int64_t r = 0; r < NR; ++r)
    if (deg[r] >= 2) { mid[r] = M++; multi_edges += deg[r]; }
  plan.m_root.resize(M);
  plan.m_ptr.assign(M + 1, 0);
  for (int64_t r = 0; r < NR; ++r)
    if (mid[r] >= 0) { plan.m_root[mid[r]] = int32_t(r); plan.m_ptr[mid[r] + 1] = deg[r]; }
  for (int32_t m = 0; m < M; ++m) plan.m_ptr[m + 1] += plan.m_ptr[m];
  plan.m_leaf.resize(multi_edges);
  {
    std::vector<int32_t> fill(plan.m_ptr.begin(), plan.m_ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
      const int32_t m = mid[rootu[e]];
      if (m >= 0) plan.m_leaf[fill[m]++] = int32_t(leafu[e]);
    }
  }
  // single-leaf roots
  std::vector<int64_t> sleaf(NR, -1);
  for (int64_t e = 0; e < E; ++e)
    if (deg[rootu[e]] == 1) sleaf[rootu[e]] = leafu[e];
  {
    int64_t r0 = -1, l0 = 0, last = -1;
    std::vector<int64_t> members;
    auto close = [&]() {
      if (members.empty()) return;
      if (int64_t(members.size()) >= kMinMaskedSingles) {
        MaskedRun mr{};
        mr.root0 = r0;
        mr.leaf0 = l0;
        mr.n = int32_t(last - r0 + 1);
        mr.mask0 = int64_t(plan.mask.size()) * 32;
        plan.mask.resize(plan.mask.size() + (mr.n + 31) / 32, 0u);
        for (int64_t r : members) {
          const int64_t bit = mr.mask0 + (r - r0);
          plan.mask[bit >> 5] |= 1u << (bit & 31);
        }
        plan.mruns.push_back(mr);
      } else {
        for (int64_t r : members) {
          plan.pr_root.push_back(int32_t(r));
          plan.pr_leaf.push_back(int32_t(sleaf[r]));
        }
      }
      members.clear();
    };
    for (int64_t r = 0; r < NR; ++r) {
      if (deg[r] != 1) continue;
      const bool extend = !members.empty() && r - last <= kMaxMaskGap && sleaf[r] - l0 == r - r0 &&
                          r - r0 < (int64_t(1) << 30);
      if (!extend) {
        close();
        r0 = r;
        l0 = sleaf[r];
      }
      members.push_back(r);
      last = r;
    }
    close();
  }
  // fold blocks of multi roots
  std::vector<int32_t> blk_m;   // block -> multi root (host only, for tiling)
  std::vector<uint8_t> heavy(M, 0);
  for (int32_t m = 0; m < M; ++m) {
    const int32_t d = plan.m_ptr[m + 1] - plan.m_ptr[m];
    const int32_t nch = (d + FOLD_BLOCK - 1) / FOLD_BLOCK;
    int32_t comb = -1;
    if (nch > 1) {
      comb = int32_t(plan.combs.size());
      const int32_t nsuper = (nch + FOLD_BLOCK - 1) / FOLD_BLOCK;
      plan.combs.push_back(Comb{plan.n_partial_slots, plan.n_partial_slots + nch, plan.n_counters, nch,
                                plan.m_ptr[m], plan.m_root[m]});
      plan.n_partial_slots += nch + nsuper;
      plan.n_counters += nsuper + 1;
    }
    for (int32_t c = 0; c < nch; ++c) {
      const int32_t e0 = plan.m_ptr[m] + c * FOLD_BLOCK;
      plan.blocks.push_back(Block{plan.m_root[m], e0, std::min(FOLD_BLOCK, plan.m_ptr[m + 1] - e0), comb});
      plan.block_recs.push_back(BlockRec{comb < 0 ? plan.m_root[m] : -(comb + 1), e0});
      blk_m.push_back(m);
    }
    heavy[m] = nch >= 16;
  }
  plan.block_recs.push_back(BlockRec{0, int32_t(plan.m_leaf.size())});   // sentinel
  // tiles, ordered by the first root they touch (heavy multi roots first)
  struct Keyed { int64_t key; RmTile t; };
  std::vector<Keyed> common;
  int64_t single_work = int64_t(plan.pr_root.size());
  for (const MaskedRun &mr : plan.mruns) single_work += mr.n;
  const int32_t rm_per = tile_size(single_work, RM_TILE_EDGES_MIN, RM_TILE_EDGES);   // a multiple of 32
  const int32_t ch_per = tile_size(int64_t(plan.blocks.size()), RM_TILE_CHUNKS_MIN, RM_TILE_CHUNKS);
  if (rm_per_out) *rm_per_out = rm_per;
  if (ch_per_out) *ch_per_out = ch_per;
  for (size_t i = 0; i < plan.mruns.size(); ++i)
    for (int64_t k0 = 0; k0 < plan.mruns[i].n; k0 += rm_per) {
      RmTile t = rm_tile(T_MASKED, int32_t(i), int32_t(k0),
                         int32_t(std::min<int64_t>(rm_per, plan.mruns[i].n - k0)));
      t.root0 = plan.mruns[i].root0;
      t.leaf0 = plan.mruns[i].leaf0;
      t.mask0 = plan.mruns[i].mask0;
      common.push_back({plan.mruns[i].root0 + k0, t});
    }
  for (int64_t i = 0; i < int64_t(plan.pr_root.size()); i += rm_per)
    common.push_back({plan.pr_root[i], rm_tile(T_PAIRS, int32_t(i), 0,
                                               int32_t(std::min<int64_t>(rm_per, plan.pr_root.size() - i)))});
  const int64_t heavy_key = -(int64_t(1) << 40);
  auto finish = [&](std::vector<Keyed> extra, std::vector<RmTile> &out) {
    extra.insert(extra.end(), common.begin(), common.end());
    std::stable_sort(extra.begin(), extra.end(), [](const Keyed &a, const Keyed &b) { return a.key < b.key; });
    out.clear();
    for (auto &k : extra) out.push_back(k.t);
  };
  // chunk tiles: at most ch_per blocks and ch_edges leaf entries per tile (the shared-memory
  // stage of the kernel that reads them); one list for the general Reduce kernel, one cut at
  // half the leaves for the one-vector-unit kernel
  auto chunk_tiles = [&](int64_t max_edges, std::vector<RmTile> &out) {
    const int64_t ch_edges = max_edges * ch_per / RM_TILE_CHUNKS;
    std::vector<Keyed> ch;
    const int64_t nblocks = int64_t(plan.blocks.size());
    int64_t c = 0;
    while (c < nblocks) {
      const int32_t m = blk_m[c];
      int64_t c1 = c, edges = 0;
      if (heavy[m]) {   // a heavy root's blocks get tiles of their own, scheduled first
        while (c1 < nblocks && blk_m[c1] == m && c1 - c < ch_per / 4 && edges + plan.blocks[c1].n <= ch_edges)
          edges += plan.blocks[c1++].n;
      } else {
        while (c1 < nblocks && !heavy[blk_m[c1]] && c1 - c < ch_per && edges + plan.blocks[c1].n <= ch_edges)
          edges += plan.blocks[c1++].n;
      }
      RmTile t = rm_tile(T_CHUNKS, int32_t(c), plan.blocks[c].e0, int32_t(c1 - c));
      t.e1 = int64_t(plan.blocks[c].e0) + edges;
      ch.push_back({heavy[m] ? heavy_key + plan.m_root[m] : int64_t(plan.m_root[m]), t});
      c = c1;
    }
    finish(ch, out);
  };
  chunk_tiles(RM_TILE_CHUNK_EDGES, plan.rm_fold_tiles);
  chunk_tiles(RM_TILE_CHUNK_EDGES_NV1, plan.rm_fold_nv1_tiles);
  {
    std::vector<Keyed> w;
    for (int32_t m = 0; m < M; m += RM_TILE_ROOTS)
      w.push_back({plan.m_root[m], rm_tile(T_WINNERS, m, 0, std::min<int32_t>(RM_TILE_ROOTS, M - m))});
    finish(w, plan.rm_winner_tiles);
  }
  {
    std::vector<Keyed> f;
    int32_t m = 0;
    while (m < M) {
      int32_t m1 = m;
      int64_t edges = 0;
      while (m1 < M && m1 - m < RM_TILE_FETCH && (edges < 4096 || m1 == m)) {
        edges += plan.m_ptr[m1 + 1] - plan.m_ptr[m1];
        ++m1;
      }
      f.push_back({plan.m_root[m], rm_tile(T_FETCH, m, 0, m1 - m)});
      m = m1;
    }
    finish(f, plan.rm_fetch_tiles);
  }
}

// Diagonal chunks: a root-streaming plan for the deterministic Reduce of forests in which most
// roots own one leaf at a fixed offset from themselves (leaf unit = root unit + delta) -- the
// owned entries of a rank's local vector in the SpMV scatter of Sec. IV.A, whose ghost columns
// are the other leaves.  Roots are taken 32 at a time (one warp), in root order, so the roots
// and their diagonal leaves stream through fully used sectors; a root's other leaves (at most
// DG_MAX_LEAVES - 1) are listed in canonical order, and the diagonal leaf keeps its canonical
// place in the fold.  Roots that do not fit are left to the root-major plan of the rest.
// Returns false (and builds nothing) when too few roots fit for the plan to pay.
bool build_diag(int64_t NR, int64_t E, const std::vector<int64_t> &rootu, const std::vector<int64_t> &leafu,
                const std::vector<int32_t> &deg, DiagHost &dg, std::vector<uint8_t> &covered) {
  dg = DiagHost();
  if (NR == 0 || E == 0) return false;
  // CSR of every root's leaves, canonical order inside a root (stable counting sort)
  std::vector<int32_t> ptr(NR + 1, 0), eleaf(E);
  for (int64_t r = 0; r < NR; ++r) ptr[r + 1] = ptr[r] + deg[r];
  {
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) eleaf[fill[rootu[e]]++] = int32_t(leafu[e]);
  }
  // per chunk of 32 roots: the offset most of its roots' leaves share, and how many roots have it
  const int64_t NC = (NR + 31) / 32;
  std::vector<int32_t> cdelta(NC, 0), cgood(NC, 0);
  std::vector<int64_t> cand;
  int64_t good = 0, connected = 0;
  for (int64_t c = 0; c < NC; ++c) {
    cand.clear();
    for (int64_t u = c * 32; u < std::min(NR, c * 32 + 32); ++u) {
      connected += deg[u] > 0;
      if (deg[u] < 1 || deg[u] > DG_MAX_LEAVES) continue;
      for (int32_t k = ptr[u]; k < ptr[u + 1]; ++k) cand.push_back(int64_t(eleaf[k]) - u);
    }
    if (cand.empty()) continue;
    std::sort(cand.begin(), cand.end());   // a root's leaves differ, so a value counts roots
    int64_t best = cand[0], best_n = 0;
    for (size_t i = 0; i < cand.size();) {
      size_t j = i;
      while (j < cand.size() && cand[j] == cand[i]) ++j;
      if (int64_t(j - i) > best_n) { best_n = int64_t(j - i); best = cand[i]; }
      i = j;
    }
    if (best_n >= DG_MIN_CHUNK_ROOTS) {
      cdelta[c] = int32_t(best);
      cgood[c] = int32_t(best_n);
      good += best_n;
    }
  }
  if (good < DG_MIN_ROOTS || 2 * good < connected) return false;
  int64_t c_lo = 0, c_hi = NC;
  while (!cgood[c_lo]) ++c_lo;
  while (!cgood[c_hi - 1]) --c_hi;
  covered.assign(NR, 0);
  dg.c0 = c_lo;
  dg.chunks.reserve(c_hi - c_lo);
  for (int64_t c = c_lo; c < c_hi; ++c) {
    DiagChunk rec{0u, 0u, int32_t(dg.x.size()), cdelta[c]};
    if (cgood[c]) {
      for (int32_t lane = 0; lane < 32; ++lane) {
        const int64_t u = c * 32 + lane;
        if (u >= NR) break;
        const int32_t n = deg[u];
        if (n < 1 || n > DG_MAX_LEAVES) continue;
        int32_t k = -1;
        for (int32_t i = 0; i < n; ++i)
          if (int64_t(eleaf[ptr[u] + i]) - u == cdelta[c]) { k = i; break; }
        if (k < 0) continue;
        uint32_t code;
        if (n == 1) {
          code = DG_DIAG;
        } else if (n == 2) {
          // the other leaf, with the top bit set when it comes after the diagonal leaf
          const int32_t other = eleaf[ptr[u] + 1 - k];
          dg.x.push_back(k == 0 ? int32_t(uint32_t(other) | 0x80000000u) : other);
          code = DG_PAIR;
        } else {
          dg.x.push_back(int32_t(dg.lists.size()));
          dg.lists.push_back(-1 - (k | ((n - 1 - k) << 16)));   // leaves before | after the diagonal one
          for (int32_t i = 0; i < n; ++i)
            if (i != k) dg.lists.push_back(eleaf[ptr[u] + i]);
          code = DG_LIST;
          ++dg.list_roots;
        }
        (lane < 16 ? rec.lo : rec.hi) |= code << (2 * (lane & 15));
        covered[u] = 1;
        ++dg.roots;
        dg.extras += n - 1;
      }
    }
    dg.chunks.push_back(rec);
  }
  // tiles: runs of chunks with one delta, at most DG_TILE_CHUNKS chunks, DG_TILE_XCAP x entries
  // and DG_TILE_LCAP list entries each; chunks without any covered root are left out.  A
  // chunk's list entries start at the list of its first DG_LIST root (lists are in root order).
  const int64_t nch = int64_t(dg.chunks.size());
  auto x_end = [&](int64_t k) { return k + 1 < nch ? dg.chunks[k + 1].xoff : int32_t(dg.x.size()); };
  std::vector<int32_t> lfirst(nch + 1, int32_t(dg.lists.size()));   // first list entry of chunk k
  for (int64_t k = nch - 1; k >= 0; --k) {
    lfirst[k] = lfirst[k + 1];
    const DiagChunk &ch = dg.chunks[k];
    for (int32_t lane = 31, xi = x_end(k) - 1; lane >= 0; --lane) {
      const uint32_t code = ((lane < 16 ? ch.lo : ch.hi) >> (2 * (lane & 15))) & 3u;
      if (code == DG_LIST) lfirst[k] = dg.x[xi];
      if (code >= DG_PAIR) --xi;
    }
  }
  for (int64_t k = 0; k < nch;) {
    if (!dg.chunks[k].lo && !dg.chunks[k].hi) { ++k; continue; }
    int64_t k1 = k + 1;
    while (k1 < nch && k1 - k < DG_TILE_CHUNKS && (dg.chunks[k1].lo || dg.chunks[k1].hi) &&
           dg.chunks[k1].delta == dg.chunks[k].delta && x_end(k1) - dg.chunks[k].xoff <= DG_TILE_XCAP &&
           lfirst[k1 + 1] - lfirst[k] <= DG_TILE_LCAP)
      ++k1;
    DgTile t{};
    t.c = int32_t(k);
    t.n = int32_t(k1 - k);
    t.delta = dg.chunks[k].delta;
    t.xbeg = dg.chunks[k].xoff;
    t.xend = x_end(k1 - 1);
    t.lbeg = lfirst[k];
    t.lend = lfirst[k1];
    t.full = 1;
    for (int64_t u = (c_lo + k) * 32; u < std::min(NR, (c_lo + k1) * 32); ++u)
      if (!covered[u]) { t.full = 0; break; }
    dg.tiles.push_back(t);
    k = k1;
  }
  return true;
}

}  // namespace

int analyze(const Graph &g, HostPlan &plan, sf_info &info) {
  try {
    plan = HostPlan();
    const int32_t P = g.P;
    const int64_t E = g.E, NR = g.rootoff[P];
    std::vector<int64_t> leafu(E), rootu(E);
    std::vector<int32_t> lq(E);
    for (int32_t q = 0; q < P; ++q)
      for (int64_t i = 0, e = g.edgeoff[q]; e < g.edgeoff[q + 1]; ++i, ++e) {
        leafu[e] = g.leafoff[q] + (g.has_ilocal[q] ? g.ilocal[e] : i);
        rootu[e] = g.rootoff[g.rrank[e]] + g.rindex[e];
        lq[e] = q;
      }
    std::vector<int32_t> deg(NR, 0);
    for (int64_t e = 0; e < E; ++e) deg[rootu[e]]++;

    // ---- two-sided grouping: key = p*(P+1) + (q == p ? 0 : q + 1), stable counting sort
    const int64_t nkeys = int64_t(P) * (P + 1);
    std::vector<int64_t> cnt(nkeys + 1, 0), order(E);
    auto key_of = [&](int64_t e) {
      const int64_t p = g.rrank[e], q = lq[e];
      return p * (P + 1) + (q == p ? 0 : q + 1);
    };
    for (int64_t e = 0; e < E; ++e) cnt[key_of(e) + 1]++;
    for (int64_t k = 0; k < nkeys; ++k) cnt[k + 1] += cnt[k];
    {
      std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
      for (int64_t e = 0; e < E; ++e) order[fill[key_of(e)]++] = e;
    }
    // leaf-side buffer offsets: segments ordered (q, p) for the receive side
    std::vector<int64_t> lbuf_off(nkeys, -1);
    {
      int64_t off = 0;
      for (int32_t q = 0; q < P; ++q)
        for (int32_t p = 0; p < P; ++p) {
          if (p == q) continue;
          const int64_t key = int64_t(p) * (P + 1) + (q + 1);
          const int64_t n = cnt[key + 1] - cnt[key];
          if (n) { lbuf_off[key] = off; off += n; }
        }
      plan.remote_units = off;
    }
    std::vector<int64_t> A, B;
    int64_t rbuf = 0;
    for (int64_t key = 0; key < nkeys; ++key) {
      const int64_t s = cnt[key], t = cnt[key + 1];
      if (s == t) continue;
      info.segments++;
      const bool self = (key % (P + 1)) == 0;
      A.resize(t - s);
      B.resize(t - s);
      bool dup = false;
      for (int64_t k = s; k < t; ++k) {
        A[k - s] = rootu[order[k]];
        B[k - s] = leafu[order[k]];
        dup |= deg[A[k - s]] > 1;
      }
      const size_t run_first = plan.runs.size();
      RunBuilder rb{plan, A.data(), B.data(), t - s, int32_t((self ? RUN_SELF : 0) | (dup ? RUN_DUP : 0)), {}};
      rb.run();
      if (self) {
        info.self_edges += t - s;
      } else {
        // buffer offsets of each run inside this segment's chunks
        int64_t pos = 0;
        for (size_t r = run_first; r < plan.runs.size(); ++r) {
          plan.runs[r].rbuf0 = rbuf + pos;
          plan.runs[r].lbuf0 = lbuf_off[key] + pos;
          pos += plan.runs[r].n;
        }
        plan.segs.push_back(SegCopy{rbuf, lbuf_off[key], t - s});
        rbuf += t - s;
      }
    }
    const int32_t ts_per = tile_size(E, TS_TILE_EDGES_MIN, TS_TILE_EDGES);
    info.ts_tile_edges = ts_per;
    for (size_t r = 0; r < plan.runs.size(); ++r) {
      const Run &run = plan.runs[r];
      push_ts_tiles(plan.ts_tiles, run, ts_per);
      push_ts_tiles((run.flags & RUN_SELF) ? plan.ts_self_tiles : plan.ts_remote_tiles, run, ts_per);
      info.runs++;
      const int32_t idx = run.flags & (RUN_ROOT_IDX | RUN_LEAF_IDX);
      if (idx == 0) {
        info.runs_pattern++;
        if (run.ny > 1 || run.nx < run.n) info.runs_3d++;
        info.edges_both_pattern += run.n;
      } else if (idx == (RUN_ROOT_IDX | RUN_LEAF_IDX)) {
        info.edges_two_indexed += run.n;
      } else {
        info.edges_one_indexed += run.n;
      }
    }

    for (int64_t r = 0; r < NR; ++r)
      if (deg[r] == 0) plan.z_root.push_back(int32_t(r));

    // ---- root-major plan over every root, then the diagonal chunks and the root-major plan of the
    // roots they leave out
    int32_t rm_per = 0, ch_per = 0;
    build_rm(NR, E, rootu, leafu, deg, plan, &rm_per, &ch_per);
    info.rm_tile_edges = rm_per;
    info.rm_tile_blocks = ch_per;
    {
      std::vector<uint8_t> covered;
      if (build_diag(NR, E, rootu, leafu, deg, plan.dg, covered)) {
        std::vector<int32_t> rest_deg(deg);
        for (int64_t r = 0; r < NR; ++r)
          if (covered[r]) rest_deg[r] = 0;
        plan.rest = std::make_shared<HostPlan>();
        build_rm(NR, E, rootu, leafu, rest_deg, *plan.rest, nullptr, nullptr);
      }
    }

    // ---- statistics
    info.nranks = P;
    info.nroots_total = NR;
    info.leaf_extent_total = g.leafoff[P];
    info.nedges = E;
    for (int64_t r = 0; r < NR; ++r) {
      info.max_in_degree = std::max<int64_t>(info.max_in_degree, deg[r]);
      info.connected_roots += deg[r] > 0;
    }
    info.has_dup_roots = info.max_in_degree > 1;
    info.multi_roots = int64_t(plan.m_root.size());
    info.multi_edges = int64_t(plan.m_leaf.size());
    info.dg_chunks = int64_t(plan.dg.chunks.size());
    info.dg_roots = plan.dg.roots;
    info.dg_extra_leaves = plan.dg.extras;
    info.dg_list_roots = plan.dg.list_roots;
    info.dg_rest_roots = plan.rest ? info.connected_roots - plan.dg.roots : 0;
    info.rm_masked_runs = int64_t(plan.mruns.size());
    for (auto &mr : plan.mruns)
      for (int32_t k = 0; k < mr.n; ++k)
        info.rm_masked_edges += (plan.mask[(mr.mask0 + k) >> 5] >> ((mr.mask0 + k) & 31)) & 1u;
    info.rm_pairs = int64_t(plan.pr_root.size());
    info.rm_chunks = int64_t(plan.blocks.size());
    info.analyzed = 1;
  } catch (const std::bad_alloc &) {
    return SF_ERR_ALLOC;
  }
  return SF_SUCCESS;
}

}  // namespace sfgb
