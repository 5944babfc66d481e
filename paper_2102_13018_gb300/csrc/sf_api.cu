// sf_api.cu -- the C ABI of sf.h: object lifetime, device plans, begin/end bookkeeping and
// dispatch of every operation to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sf_object.h"

using namespace sfgb;

namespace sfgb {

std::atomic<int64_t> &launch_counter() {
  static std::atomic<int64_t> count{0};
  return count;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? SF_SUCCESS : SF_ERR_CUDA; }

// grow-only device buffer; a reallocation waits for the device so no kernel still uses the old one
int ensure(DevBuf &b, size_t bytes, bool zero, cudaStream_t s) {
  if (bytes == 0 || b.bytes >= bytes) return SF_SUCCESS;
  if (b.p) {
    if (cudaDeviceSynchronize() != cudaSuccess) return SF_ERR_CUDA;
    cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_ALLOC;
  }
  b.bytes = bytes;
  if (zero && cudaMemsetAsync(b.p, 0, bytes, s) != cudaSuccess) return SF_ERR_CUDA;
  return SF_SUCCESS;
}

void release(DevBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// Layout of the plan blob: each array 256-byte aligned.
struct BlobBuilder {
  std::vector<char> host;
  template <typename V> size_t add(const std::vector<V> &v) {
    // 256-byte aligned, and followed by at least 16 bytes of the blob: a bulk copy of a span
    // widened to 16-byte boundaries stays inside the allocation
    size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + v.size() * sizeof(V) + 16);
    if (!v.empty()) memcpy(host.data() + off, v.data(), v.size() * sizeof(V));
    return off;
  }
};

// widest vector (bytes) usable for a unit of `ub` bytes with the given pointers
int pick_vb(int w, int ub, bool allow_wide, std::initializer_list<const void *> ptrs, int cap) {
  static const int cand[] = {16, 8, 4, 2};
  for (int vb : cand) {
    if (vb < w || ub % vb || (vb > cap && vb > w)) continue;
    if (vb != w && !allow_wide) continue;
    bool ok = true;
    for (const void *p : ptrs)
      if (p && (reinterpret_cast<uintptr_t>(p) % vb)) ok = false;
    if (ok) return vb;
  }
  return 0;
}

int check_unit(const sf_unit &u, int32_t op) {
  if (elem_size(u.dtype) == 0 || u.bs < 1 || int64_t(u.bs) * elem_size(u.dtype) > SF_MAX_UNIT_BYTES) return SF_ERR_ARG;
  if (op < SF_REPLACE || op > SF_MAX) return SF_ERR_ARG;
  return SF_SUCCESS;
}

int check_ptr(const void *p, int w) {
  if (!p) return SF_ERR_NULL;
  if (reinterpret_cast<uintptr_t>(p) % w) return SF_ERR_ALIGN;
  return SF_SUCCESS;
}

Pending *find_pending(sf_t *sf, int kind, const sf_unit &u, const void *p0, const void *p1, const void *p2,
                      int32_t op, int32_t m0, int32_t m1) {
  for (auto &pd : sf->pending)
    if (pd.kind == kind && pd.unit.dtype == u.dtype && pd.unit.bs == u.bs && pd.p0 == p0 && pd.p1 == p1 &&
        pd.p2 == p2 && pd.op == op && pd.m0 == m0 && pd.m1 == m1)
      return &pd;
  return nullptr;
}

void drop_pending(sf_t *sf, Pending *pd) { sf->pending.erase(sf->pending.begin() + (pd - sf->pending.data())); }

int launched(cudaError_t e) {
  if (e != cudaSuccess) return SF_ERR_CUDA;
  launch_counter().fetch_add(1, std::memory_order_relaxed);
  return SF_SUCCESS;
}

TsArgs ts_args(const sf_t *sf, const TsTile *tiles, int32_t ntiles, const void *src, void *dst, void *upd, int nv,
               int phase) {
  TsArgs a{};
  a.ridx = sf->dp.ts_ridx;
  a.lidx = sf->dp.ts_lidx;
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.src = src;
  a.dst = dst;
  a.upd = upd;
  a.nv = nv;
  const DivMagic dm = div_magic(uint32_t(nv));
  a.nv_m = dm.m;
  a.nv_s = dm.s;
  a.phase = phase;
  return a;
}

RmArgs rm_args(sf_t *sf, const RmTile *tiles, int32_t ntiles, void *root, void *leaf, void *upd, int nv) {
  return rm_args_plan(sf, sf->dp, tiles, ntiles, root, leaf, upd, nv);
}

RmArgs rm_args_plan(sf_t *sf, const DevPlan &d, const RmTile *tiles, int32_t ntiles, void *root, void *leaf, void *upd,
                    int nv) {
  RmArgs a{};
  a.mask = d.mask;
  a.pr_root = d.pr_root;
  a.pr_leaf = d.pr_leaf;
  a.m_root = d.m_root;
  a.m_ptr = d.m_ptr;
  a.m_leaf = d.m_leaf;
  a.blocks = d.blocks;
  a.combs = d.combs;
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.root = root;
  a.leaf = leaf;
  a.upd = upd;
  a.partial = sf->partial.p;
  a.counter = static_cast<int32_t *>(sf->counter.p);
  a.status = static_cast<int32_t *>(sf->status.p);
  a.nv = nv;
  const DivMagic dm = div_magic(uint32_t(nv));
  a.nv_m = dm.m;
  a.nv_s = dm.s;
  return a;
}

// ---- Bcast data paths -------------------------------------------------------------------
int bcast_launch(sf_t *sf, const sf_unit &u, const void *root, void *leaf, int32_t op, cudaStream_t s,
                 int path, int *finish) {
  const int w = elem_size(u.dtype), ub = w * u.bs;
  *finish = 0;
  if (sf->info.nedges == 0) return SF_SUCCESS;
  const bool copy = op == SF_REPLACE;
  if (path == SF_PATH_ROOT_MAJOR) {
    const int vb = pick_vb_sf(sf, w, ub, true, {root, leaf});
    if (!vb) return SF_ERR_ALIGN;
    const int vbo = copy ? vb : (vb == 16 ? 16 : w);
    RmArgs a = rm_args(sf, sf->dp.rm_fold_tiles, sf->dp.n_rm_fold_tiles, const_cast<void *>(root), leaf, nullptr, ub / vbo);
    return launched(launch_rm(u.dtype, op, vbo, RM_BCAST, a, sf->dp.n_rm_fold_tiles, s));
  }
  if (path == SF_PATH_THREE_PHASE && sf->dp.remote_units > 0) {
    const size_t bytes = size_t(sf->dp.remote_units) * ub;
    int rc;
    if ((rc = ensure(sf->rootbuf, bytes, false, s)) || (rc = ensure(sf->leafbuf, bytes, false, s))) return rc;
    const int vb = pick_vb(w, ub, copy, {root, leaf, sf->rootbuf.p, sf->leafbuf.p});
    if (!vb) return SF_ERR_ALIGN;
    const int nv = ub / vb;
    // self edges: direct scatter; remote edges: pack, then move
    TsArgs self = ts_args(sf, sf->dp.ts_self_tiles, sf->dp.n_ts_self_tiles, root, leaf, nullptr, nv, PH_FUSED);
    if ((rc = launched(launch_ts(u.dtype, op, vb, false, false, false, self, sf->dp.n_ts_self_tiles, s)))) return rc;
    const int vbc = pick_vb(w, ub, true, {root, sf->rootbuf.p, sf->leafbuf.p});
    TsArgs pack = ts_args(sf, sf->dp.ts_remote_tiles, sf->dp.n_ts_remote_tiles, root, sf->rootbuf.p, nullptr, ub / vbc,
                          PH_PACK);
    if ((rc = launched(launch_ts(u.dtype, SF_REPLACE, vbc, false, false, false, pack, sf->dp.n_ts_remote_tiles, s))))
      return rc;
    MoveArgs mv{sf->dp.segs, sf->move_tiles, sf->rootbuf.p, sf->leafbuf.p, ub / vbc, 0};
    if ((rc = launched(launch_move(vbc, mv, sf->n_move_tiles, s)))) return rc;
    *finish = 1;
    return SF_SUCCESS;
  }
  const int vb = pick_vb_sf(sf, w, ub, true, {root, leaf});
  if (!vb) return SF_ERR_ALIGN;
  const int vbo = copy ? vb : (vb == 16 ? 16 : w);
  TsArgs a = ts_args(sf, sf->dp.ts_tiles, sf->dp.n_ts_tiles, root, leaf, nullptr, ub / vbo, PH_FUSED);
  return launched(launch_ts(u.dtype, op, vbo, false, false, false, a, sf->dp.n_ts_tiles, s));
}

int bcast_finish(sf_t *sf, const sf_unit &u, const void *root, void *leaf, int32_t op, cudaStream_t s) {
  const int w = elem_size(u.dtype), ub = w * u.bs;
  const int vb = pick_vb(w, ub, op == SF_REPLACE, {leaf, sf->leafbuf.p});
  if (!vb) return SF_ERR_ALIGN;
  const int vbo = op == SF_REPLACE ? vb : (vb == 16 ? 16 : w);
  TsArgs a = ts_args(sf, sf->dp.ts_remote_tiles, sf->dp.n_ts_remote_tiles, sf->leafbuf.p, leaf, nullptr, ub / vbo,
                     PH_UNPACK);
  return launched(launch_ts(u.dtype, op, vbo, false, false, false, a, sf->dp.n_ts_remote_tiles, s));
}

// ---- Reduce -------------------------------------------------------------------------------
DgArgs dg_args(const sf_t *sf, const void *leaf, void *root) {
  DgArgs g{};
  g.chunks = sf->dp.dg_chunks;
  g.x = sf->dp.dg_x;
  g.lists = sf->dp.dg_lists;
  g.c0 = sf->dp.dg_c0;
  g.nchunks = sf->dp.dg_nchunks;
  g.nroots = int32_t(sf->info.nroots_total);
  g.ntiles = (sf->dp.dg_nchunks + DG_TILE_CHUNKS - 1) / DG_TILE_CHUNKS;
  g.root = root;
  g.leaf = leaf;
  return g;
}

int reduce_det_launch(sf_t *sf, const sf_unit &u, const void *leaf, void *root, int32_t op, cudaStream_t s, int vbo,
                      int nv, void *partial, int32_t *counter, bool zero_root) {
  const bool nv1 = reduce_nv1(op, vbo, nv), flat = reduce_flat(op, vbo, nv);
  const DevPlan *d = &sf->dp;
  if (reduce_dg(sf, op, nv)) {
    DgArgs g = dg_args(sf, leaf, root);
    g.zero_root = zero_root;
    int rc;
    // staged by bulk copies (SF_PLAN_DIAGONAL_STAGED, both bases 16-byte aligned), else direct loads
    cudaError_t e = cudaErrorNotSupported;
    if (reduce_plan(sf) == SF_PLAN_DIAGONAL_STAGED && sf->dp.n_dg_tiles > 0 && (reinterpret_cast<uintptr_t>(root) & 15) == 0 &&
        (reinterpret_cast<uintptr_t>(leaf) & 15) == 0) {
      DgBulkArgs b{g, sf->dp.dg_tiles, sf->dp.n_dg_tiles, static_cast<int32_t *>(sf->status.p),
                   sf->info.nroots_total * vbo, sf->info.leaf_extent_total * vbo};
      e = launch_dg_bulk(u.dtype, op, vbo, b, s);
    }
    if (e == cudaErrorNotSupported) e = launch_dg(u.dtype, op, vbo, DgLaunch{&g, nullptr, nullptr, g.ntiles, g.ntiles, s});
    if ((rc = launched(e))) return rc;
    if (!sf->has_rest) return SF_SUCCESS;
    d = &sf->dp_rest;   // the roots the chunks leave out
  }
  const bool nv1_list = nv1 || flat;
  const RmTile *tiles = op == SF_REPLACE ? d->rm_winner_tiles : nv1_list ? d->rm_fold_nv1_tiles : d->rm_fold_tiles;
  const int nt = op == SF_REPLACE ? d->n_rm_winner_tiles : nv1_list ? d->n_rm_fold_nv1_tiles : d->n_rm_fold_tiles;
  if (nt == 0) return SF_SUCCESS;
  RmArgs a = rm_args_plan(sf, *d, tiles, nt, root, const_cast<void *>(leaf), nullptr, nv);
  a.partial = partial;
  a.counter = counter;
  a.zero_root = zero_root;
  return launched(launch_rm(u.dtype, op, vbo, RM_REDUCE, RmLaunch{&a, nullptr, nullptr, nt, s, nv1, flat}));
}

// Zero the roots without leaves (and their argleaf entries, if given) for an operation that
// starts its roots at zero.
int zero_leafless(sf_t *sf, const sf_unit &u, void *root, int32_t *arg, cudaStream_t s) {
  if (sf->dp.n_z_root == 0) return SF_SUCCESS;
  const int w = elem_size(u.dtype), ub = w * u.bs;
  const int vb = pick_vb(w, ub, true, {root});
  if (!vb) return SF_ERR_ALIGN;
  return launched(launch_zero(vb, sf->dp.z_root, sf->dp.n_z_root, root, ub / vb, arg, u.bs, s));
}

int reduce_launch(sf_t *sf, const sf_unit &u, const void *leaf, void *root, int32_t op, cudaStream_t s,
                  bool from_zero = false) {
  const int w = elem_size(u.dtype), ub = w * u.bs;
  if (sf->info.nedges == 0) return from_zero ? zero_leafless(sf, u, root, nullptr, s) : SF_SUCCESS;
  if (reduce_atomic(sf, u.dtype, op)) {
    // atomics combine into the roots in place: start them at zero first
    if (from_zero && (sf->info.nroots_total > 0) &&
        cudaMemsetAsync(root, 0, size_t(sf->info.nroots_total) * ub, s) != cudaSuccess)
      return SF_ERR_CUDA;
    TsArgs a = ts_args(sf, sf->dp.ts_tiles, sf->dp.n_ts_tiles, leaf, root, nullptr, u.bs, PH_FUSED);
    return launched(launch_ts(u.dtype, op, w, true, true, false, a, sf->dp.n_ts_tiles, s));
  }
  int rc;
  if (from_zero && (rc = zero_leafless(sf, u, root, nullptr, s))) return rc;
  const int vb = pick_vb_sf(sf, w, ub, true, {root, leaf});
  if (!vb) return SF_ERR_ALIGN;
  const int vbo = op == SF_REPLACE ? vb : (vb == 16 ? 16 : w);
  const int nv = ub / vbo;
  if (op != SF_REPLACE && sf->dp.n_partial_slots > 0) {
    // the full plan's scratch also serves the plan of the rest (a subset of its multi roots)
    const size_t pbytes = size_t(sf->dp.n_partial_slots) * nv * acc_pack_bytes(u.dtype, op, vbo);
    const size_t cbytes = size_t(sf->dp.n_counters) * nv * sizeof(int32_t);
    if ((rc = ensure(sf->partial, pbytes, false, s)) || (rc = ensure(sf->counter, cbytes, true, s))) return rc;
  }
  return reduce_det_launch(sf, u, leaf, root, op, s, vbo, nv, sf->partial.p, static_cast<int32_t *>(sf->counter.p),
                           from_zero);
}

// ---- FetchAndOp ---------------------------------------------------------------------------
int fetch_launch(sf_t *sf, const sf_unit &u, void *root, const void *leaf, void *upd, int32_t op, cudaStream_t s) {
  const int w = elem_size(u.dtype), ub = w * u.bs;
  if (sf->info.nedges == 0) return SF_SUCCESS;
  if (sf->mode == SF_MODE_ATOMIC) {
    if (u.bs != 1) return SF_ERR_UNSUPPORTED;
    TsArgs a = ts_args(sf, sf->dp.ts_tiles, sf->dp.n_ts_tiles, leaf, root, upd, 1, PH_FUSED);
    return launched(launch_ts(u.dtype, op, w, true, true, true, a, sf->dp.n_ts_tiles, s));
  }
  const int vb = pick_vb(w, ub, true, {root, leaf, upd});
  if (!vb) return SF_ERR_ALIGN;
  const int vbo = op == SF_REPLACE ? vb : (vb == 16 ? 16 : w);
  RmArgs a = rm_args(sf, sf->dp.rm_fetch_tiles, sf->dp.n_rm_fetch_tiles, root, const_cast<void *>(leaf), upd, ub / vbo);
  return launched(launch_rm(u.dtype, op, vbo, RM_FETCH, a, sf->dp.n_rm_fetch_tiles, s));
}

int bcast_path(const sf_t *sf, int64_t unit_bytes) {
  if (sf->path != SF_PATH_AUTO) return sf->path;
  if (sf->path_tuned) return sf->tuned_path;
  return unit_bytes >= kRootMajorUnitBytes && sf->info.nedges >= kRootMajorMeanDegree * sf->info.connected_roots
             ? SF_PATH_ROOT_MAJOR
             : SF_PATH_FUSED;
}
int reduce_mode(const sf_t *sf) { return sf->mode == SF_MODE_AUTO ? sf->tuned_mode : sf->mode; }

bool reduce_atomic(const sf_t *sf, int32_t dtype, int32_t op) {
  if (op == SF_REPLACE || dtype == SF_BF16) return false;
  if (reduce_mode(sf) == SF_MODE_ATOMIC) return true;
  // Only integer results are independent of the arrival order: a floating MIN/MAX keeps the
  // first of two equal values (+0 and -0 compare equal), so it stays on the ordered fold.  A
  // Reduce set to the diagonal chunks runs there.
  const bool integer = dtype == SF_INT32 || dtype == SF_INT64;
  return integer && sf->info.max_in_degree <= kOrderFreeMaxDegree && reduce_plan(sf) == SF_PLAN_ROOT_MAJOR;
}

int ensure_ready(const sf_t *sf) {
  if (!sf) return SF_ERR_NULL;
  if (!sf->setup) return SF_ERR_STATE;
  return SF_SUCCESS;
}

int bcast_all(sf_t *sf, const sf_unit &u, const void *root, void *leaf, int32_t op, cudaStream_t s, int path) {
  int finish = 0;
  int rc = bcast_launch(sf, u, root, leaf, op, s, path, &finish);
  if (!rc && finish) rc = bcast_finish(sf, u, root, leaf, op, s);
  return rc;
}

int reduce_all(sf_t *sf, const sf_unit &u, const void *leaf, void *root, int32_t op, cudaStream_t s, int mode) {
  const int32_t saved = sf->mode;
  sf->mode = mode;
  const int rc = reduce_launch(sf, u, leaf, root, op, s);
  sf->mode = saved;
  return rc;
}

}  // namespace sfgb

extern "C" {

int sf_create(int32_t nranks, const int64_t nroots[], const int64_t nleaves[], const int64_t *const ilocal[],
              const sf_node *const iremote[], sf_t **out) {
  if (!out) return SF_ERR_NULL;
  *out = nullptr;
  sf_t *sf = new (std::nothrow) sf_t();
  if (!sf) return SF_ERR_ALLOC;
  const int rc = build_graph(nranks, nroots, nleaves, ilocal, iremote, sf->g);
  if (rc != SF_SUCCESS) {
    delete sf;
    return rc;
  }
  sf->info.nranks = nranks;
  *out = sf;
  return SF_SUCCESS;
}

int sf_analyze(sf_t *sf) {
  if (!sf) return SF_ERR_NULL;
  if (sf->info.analyzed) return SF_SUCCESS;
  return analyze(sf->g, sf->hp, sf->info);
}

int sf_setup(sf_t *sf, sf_stream_t stream) {
  if (!sf) return SF_ERR_NULL;
  if (sf->setup) return SF_SUCCESS;
  int rc = sf_analyze(sf);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&sf->device) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  HostPlan &h = sf->hp;
  // move tiles: slices of 4096 units of each remote segment
  sf->h_move_tiles.clear();
  for (size_t i = 0; i < h.segs.size(); ++i)
    for (int64_t k0 = 0; k0 < h.segs[i].n; k0 += 4096)
      sf->h_move_tiles.push_back(Tile{T_RUN, int32_t(i), int32_t(k0), int32_t(std::min<int64_t>(4096, h.segs[i].n - k0))});
  BlobBuilder b;
  const size_t o_ridx = b.add(h.ts_ridx), o_lidx = b.add(h.ts_lidx),
               o_tst = b.add(h.ts_tiles), o_tss = b.add(h.ts_self_tiles), o_tsr = b.add(h.ts_remote_tiles),
               o_segs = b.add(h.segs), o_mv = b.add(sf->h_move_tiles), o_mask = b.add(h.mask),
               o_prr = b.add(h.pr_root), o_prl = b.add(h.pr_leaf), o_mro = b.add(h.m_root), o_mpt = b.add(h.m_ptr),
               o_mle = b.add(h.m_leaf), o_blk = b.add(h.block_recs), o_cmb = b.add(h.combs),
               o_rf = b.add(h.rm_fold_tiles), o_rf1 = b.add(h.rm_fold_nv1_tiles), o_rw = b.add(h.rm_winner_tiles),
               o_rfe = b.add(h.rm_fetch_tiles), o_dgc = b.add(h.dg.chunks), o_dgx = b.add(h.dg.x),
               o_dgl = b.add(h.dg.lists), o_z = b.add(h.z_root), o_dgt = b.add(h.dg.tiles);
  // the root-major plan of the roots the diagonal chunks leave out (Reduce only)
  static const HostPlan kNone;
  const HostPlan &hr = h.rest ? *h.rest : kNone;
  const size_t r_mask = b.add(hr.mask), r_prr = b.add(hr.pr_root), r_prl = b.add(hr.pr_leaf),
               r_mro = b.add(hr.m_root), r_mpt = b.add(hr.m_ptr), r_mle = b.add(hr.m_leaf),
               r_blk = b.add(hr.block_recs), r_cmb = b.add(hr.combs), r_rf = b.add(hr.rm_fold_tiles),
               r_rf1 = b.add(hr.rm_fold_nv1_tiles), r_rw = b.add(hr.rm_winner_tiles);
  const size_t bytes = std::max<size_t>(b.host.size(), 256);
  if (cudaMalloc(&sf->blob.p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_ALLOC;
  }
  sf->blob.bytes = bytes;
  if (!b.host.empty() && cudaMemcpyAsync(sf->blob.p, b.host.data(), b.host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SF_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SF_ERR_CUDA;
  char *base = static_cast<char *>(sf->blob.p);
  DevPlan &d = sf->dp;
  d.ts_ridx = reinterpret_cast<const int32_t *>(base + o_ridx);
  d.ts_lidx = reinterpret_cast<const int32_t *>(base + o_lidx);
  d.ts_tiles = reinterpret_cast<const TsTile *>(base + o_tst);
  d.ts_self_tiles = reinterpret_cast<const TsTile *>(base + o_tss);
  d.ts_remote_tiles = reinterpret_cast<const TsTile *>(base + o_tsr);
  d.segs = reinterpret_cast<const SegCopy *>(base + o_segs);
  d.n_ts_tiles = int32_t(h.ts_tiles.size());
  sf->ts_default = d.ts_tiles;
  sf->n_ts_default = d.n_ts_tiles;
  d.n_ts_self_tiles = int32_t(h.ts_self_tiles.size());
  d.n_ts_remote_tiles = int32_t(h.ts_remote_tiles.size());
  d.n_segs = int32_t(h.segs.size());
  d.remote_units = h.remote_units;
  sf->move_tiles = reinterpret_cast<const Tile *>(base + o_mv);
  sf->n_move_tiles = int32_t(sf->h_move_tiles.size());
  d.mask = reinterpret_cast<const uint32_t *>(base + o_mask);
  d.pr_root = reinterpret_cast<const int32_t *>(base + o_prr);
  d.pr_leaf = reinterpret_cast<const int32_t *>(base + o_prl);
  d.m_root = reinterpret_cast<const int32_t *>(base + o_mro);
  d.m_ptr = reinterpret_cast<const int32_t *>(base + o_mpt);
  d.m_leaf = reinterpret_cast<const int32_t *>(base + o_mle);
  d.blocks = reinterpret_cast<const BlockRec *>(base + o_blk);
  d.combs = reinterpret_cast<const Comb *>(base + o_cmb);
  d.rm_fold_tiles = reinterpret_cast<const RmTile *>(base + o_rf);
  d.rm_fold_nv1_tiles = reinterpret_cast<const RmTile *>(base + o_rf1);
  d.rm_winner_tiles = reinterpret_cast<const RmTile *>(base + o_rw);
  d.rm_fetch_tiles = reinterpret_cast<const RmTile *>(base + o_rfe);
  d.n_rm_fold_tiles = int32_t(h.rm_fold_tiles.size());
  d.n_rm_fold_nv1_tiles = int32_t(h.rm_fold_nv1_tiles.size());
  d.n_rm_winner_tiles = int32_t(h.rm_winner_tiles.size());
  d.n_rm_fetch_tiles = int32_t(h.rm_fetch_tiles.size());
  d.n_multi = int32_t(h.m_root.size());
  d.n_partial_slots = h.n_partial_slots;
  d.n_counters = h.n_counters;
  d.dg_chunks = reinterpret_cast<const DiagChunk *>(base + o_dgc);
  d.dg_x = reinterpret_cast<const int32_t *>(base + o_dgx);
  d.dg_lists = reinterpret_cast<const int32_t *>(base + o_dgl);
  d.dg_c0 = int32_t(h.dg.c0);
  d.dg_nchunks = int32_t(h.dg.chunks.size());
  d.z_root = reinterpret_cast<const int32_t *>(base + o_z);
  d.n_z_root = int32_t(h.z_root.size());
  d.dg_tiles = reinterpret_cast<const DgTile *>(base + o_dgt);
  d.n_dg_tiles = int32_t(h.dg.tiles.size());
  sf->has_rest = bool(h.rest);
  {
    DevPlan &r = sf->dp_rest;
    r = DevPlan{};
    r.mask = reinterpret_cast<const uint32_t *>(base + r_mask);
    r.pr_root = reinterpret_cast<const int32_t *>(base + r_prr);
    r.pr_leaf = reinterpret_cast<const int32_t *>(base + r_prl);
    r.m_root = reinterpret_cast<const int32_t *>(base + r_mro);
    r.m_ptr = reinterpret_cast<const int32_t *>(base + r_mpt);
    r.m_leaf = reinterpret_cast<const int32_t *>(base + r_mle);
    r.blocks = reinterpret_cast<const BlockRec *>(base + r_blk);
    r.combs = reinterpret_cast<const Comb *>(base + r_cmb);
    r.rm_fold_tiles = reinterpret_cast<const RmTile *>(base + r_rf);
    r.rm_fold_nv1_tiles = reinterpret_cast<const RmTile *>(base + r_rf1);
    r.rm_winner_tiles = reinterpret_cast<const RmTile *>(base + r_rw);
    r.n_rm_fold_tiles = int32_t(hr.rm_fold_tiles.size());
    r.n_rm_fold_nv1_tiles = int32_t(hr.rm_fold_nv1_tiles.size());
    r.n_rm_winner_tiles = int32_t(hr.rm_winner_tiles.size());
    r.n_multi = int32_t(hr.m_root.size());
    r.n_partial_slots = hr.n_partial_slots;
    r.n_counters = hr.n_counters;
  }
  // fold scratch for units up to 16 bytes, so common operations allocate nothing later
  if ((rc = ensure(sf->partial, size_t(h.n_partial_slots) * 16, false, s)) ||
      (rc = ensure(sf->counter, size_t(h.n_counters) * 4 * 8, true, s)) || (rc = ensure(sf->status, 16, true, s)))
    return rc;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SF_ERR_CUDA;
  sf->info.device_plan_bytes = int64_t(bytes);
  sf->info.setup_done = 1;
  sf->setup = true;
  return SF_SUCCESS;
}

int sf_get_layout(const sf_t *sf, int64_t *rootoff, int64_t *leafoff) {
  if (!sf || !rootoff || !leafoff) return SF_ERR_NULL;
  for (int32_t p = 0; p <= sf->g.P; ++p) {
    rootoff[p] = sf->g.rootoff[p];
    leafoff[p] = sf->g.leafoff[p];
  }
  return SF_SUCCESS;
}

int sf_get_info(const sf_t *sf, sf_info *info) {
  if (!sf || !info) return SF_ERR_NULL;
  *info = sf->info;
  return SF_SUCCESS;
}

int sf_set_mode(sf_t *sf, int32_t mode) {
  if (!sf) return SF_ERR_NULL;
  if (mode < SF_MODE_AUTO || mode > SF_MODE_DETERMINISTIC) return SF_ERR_ARG;
  sf->mode = mode;
  return SF_SUCCESS;
}

int sf_set_path(sf_t *sf, int32_t path) {
  if (!sf) return SF_ERR_NULL;
  if (path < SF_PATH_AUTO || path > SF_PATH_ROOT_MAJOR) return SF_ERR_ARG;
  sf->path = path;
  return SF_SUCCESS;
}

int sf_set_reduce_plan(sf_t *sf, int32_t plan) {
  if (!sf) return SF_ERR_NULL;
  if (plan < SF_PLAN_AUTO || plan > SF_PLAN_DIAGONAL_STAGED) return SF_ERR_ARG;
  sf->plan = plan;
  return SF_SUCCESS;
}

int sf_set_vector_bytes(sf_t *sf, int32_t bytes) {
  if (!sf) return SF_ERR_NULL;
  if (bytes != 0 && bytes != 2 && bytes != 4 && bytes != 8 && bytes != 16) return SF_ERR_ARG;
  sf->vec_bytes = bytes;
  return SF_SUCCESS;
}

int sf_set_tile_edges(sf_t *sf, int32_t edges) {
  if (!sf) return SF_ERR_NULL;
  if (!sf->setup) return SF_ERR_STATE;
  if (!sf->pending.empty()) return SF_ERR_PENDING;
  if (edges != 0 && (edges < 64 || edges > (1 << 16) || (edges & (edges - 1)))) return SF_ERR_ARG;
  if (edges == sf->tile_edges) return SF_SUCCESS;
  // work already enqueued may still read the current list
  if (cudaDeviceSynchronize() != cudaSuccess) return SF_ERR_CUDA;
  release(sf->ts_tuned);
  sf->dp.ts_tiles = sf->ts_default;
  sf->dp.n_ts_tiles = sf->n_ts_default;
  sf->tile_edges = 0;
  if (edges == 0) return SF_SUCCESS;
  std::vector<TsTile> tiles;
  cut_ts_tiles(sf->hp, edges, tiles);
  const size_t bytes = std::max<size_t>(tiles.size() * sizeof(TsTile), 256);
  int rc;
  if ((rc = ensure(sf->ts_tuned, bytes, false, nullptr))) return rc;
  if (!tiles.empty() &&
      cudaMemcpy(sf->ts_tuned.p, tiles.data(), tiles.size() * sizeof(TsTile), cudaMemcpyHostToDevice) != cudaSuccess)
    return SF_ERR_CUDA;
  sf->dp.ts_tiles = static_cast<const TsTile *>(sf->ts_tuned.p);
  sf->dp.n_ts_tiles = int32_t(tiles.size());
  sf->tile_edges = edges;
  return SF_SUCCESS;
}

int sf_get_tuning(const sf_t *sf, sf_tuning *out) {
  if (!sf || !out) return SF_ERR_NULL;
  out->path = bcast_path(sf, 0);
  out->mode = reduce_mode(sf);
  out->vector_bytes = sf->vec_bytes;
  out->tile_edges = sf->tile_edges ? sf->tile_edges : int32_t(sf->info.ts_tile_edges);
  out->reduce_plan = reduce_plan(sf);
  return SF_SUCCESS;
}

int sf_bcast_begin(sf_t *sf, sf_unit unit, const void *rootdata, void *leafdata, int32_t op, sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  const int w = elem_size(unit.dtype);
  if ((sf->info.nroots_total && (rc = check_ptr(rootdata, w))) ||
      (sf->info.leaf_extent_total && (rc = check_ptr(leafdata, w))))
    return rc;
  if (find_pending(sf, K_BCAST, unit, rootdata, leafdata, nullptr, op, 0, 0)) return SF_ERR_PENDING;
  int finish = 0;
  if ((rc = bcast_launch(sf, unit, rootdata, leafdata, op, static_cast<cudaStream_t>(stream),
                         bcast_path(sf, int64_t(w) * unit.bs), &finish)))
    return rc;
  sf->pending.push_back(Pending{K_BCAST, unit, rootdata, leafdata, nullptr, op, 0, 0, finish});
  return SF_SUCCESS;
}

int sf_bcast_end(sf_t *sf, sf_unit unit, const void *rootdata, void *leafdata, int32_t op, sf_stream_t stream) {
  if (!sf) return SF_ERR_NULL;
  Pending *pd = find_pending(sf, K_BCAST, unit, rootdata, leafdata, nullptr, op, 0, 0);
  if (!pd) return SF_ERR_NO_PENDING;
  const int finish = pd->finish;
  drop_pending(sf, pd);
  if (finish) return bcast_finish(sf, unit, rootdata, leafdata, op, static_cast<cudaStream_t>(stream));
  return SF_SUCCESS;
}

int sf_reduce_begin(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op, sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  const int w = elem_size(unit.dtype);
  if ((sf->info.nroots_total && (rc = check_ptr(rootdata, w))) ||
      (sf->info.leaf_extent_total && (rc = check_ptr(leafdata, w))))
    return rc;
  if (find_pending(sf, K_REDUCE, unit, leafdata, rootdata, nullptr, op, 0, 0)) return SF_ERR_PENDING;
  if ((rc = reduce_launch(sf, unit, leafdata, rootdata, op, static_cast<cudaStream_t>(stream)))) return rc;
  sf->pending.push_back(Pending{K_REDUCE, unit, leafdata, rootdata, nullptr, op, 0, 0, 0});
  return SF_SUCCESS;
}

int sf_reduce_end(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op, sf_stream_t stream) {
  (void)stream;
  if (!sf) return SF_ERR_NULL;
  Pending *pd = find_pending(sf, K_REDUCE, unit, leafdata, rootdata, nullptr, op, 0, 0);
  if (!pd) return SF_ERR_NO_PENDING;
  drop_pending(sf, pd);
  return SF_SUCCESS;
}

int sf_reduce_from_zero_begin(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                              sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  const int w = elem_size(unit.dtype);
  if ((sf->info.nroots_total && (rc = check_ptr(rootdata, w))) ||
      (sf->info.leaf_extent_total && (rc = check_ptr(leafdata, w))))
    return rc;
  if (find_pending(sf, K_REDUCE_Z, unit, leafdata, rootdata, nullptr, op, 0, 0)) return SF_ERR_PENDING;
  if ((rc = reduce_launch(sf, unit, leafdata, rootdata, op, static_cast<cudaStream_t>(stream), true))) return rc;
  sf->pending.push_back(Pending{K_REDUCE_Z, unit, leafdata, rootdata, nullptr, op, 0, 0, 0});
  return SF_SUCCESS;
}

int sf_reduce_from_zero_end(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                            sf_stream_t stream) {
  (void)stream;
  if (!sf) return SF_ERR_NULL;
  Pending *pd = find_pending(sf, K_REDUCE_Z, unit, leafdata, rootdata, nullptr, op, 0, 0);
  if (!pd) return SF_ERR_NO_PENDING;
  drop_pending(sf, pd);
  return SF_SUCCESS;
}

int sf_zero_leafless_roots(sf_t *sf, sf_unit unit, void *rootdata, int32_t *argleaf, sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, SF_REPLACE))) return rc;
  if (sf->info.nroots_total && ((rc = check_ptr(rootdata, elem_size(unit.dtype))) ||
                                (argleaf && (rc = check_ptr(argleaf, 4)))))
    return rc;
  return zero_leafless(sf, unit, rootdata, argleaf, static_cast<cudaStream_t>(stream));
}

int sf_fetch_and_op_begin(sf_t *sf, sf_unit unit, void *rootdata, const void *leafdata, void *leafupdate, int32_t op,
                          sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  const int w = elem_size(unit.dtype);
  if (sf->info.nroots_total && (rc = check_ptr(rootdata, w))) return rc;
  if (sf->info.leaf_extent_total && ((rc = check_ptr(leafdata, w)) || (rc = check_ptr(leafupdate, w)))) return rc;
  if (sf->mode == SF_MODE_ATOMIC && unit.bs != 1) return SF_ERR_UNSUPPORTED;
  if (find_pending(sf, K_FETCH, unit, rootdata, leafdata, leafupdate, op, 0, 0)) return SF_ERR_PENDING;
  if ((rc = fetch_launch(sf, unit, rootdata, leafdata, leafupdate, op, static_cast<cudaStream_t>(stream)))) return rc;
  sf->pending.push_back(Pending{K_FETCH, unit, rootdata, leafdata, leafupdate, op, 0, 0, 0});
  return SF_SUCCESS;
}

int sf_fetch_and_op_end(sf_t *sf, sf_unit unit, void *rootdata, const void *leafdata, void *leafupdate, int32_t op,
                        sf_stream_t stream) {
  (void)stream;
  if (!sf) return SF_ERR_NULL;
  Pending *pd = find_pending(sf, K_FETCH, unit, rootdata, leafdata, leafupdate, op, 0, 0);
  if (!pd) return SF_ERR_NO_PENDING;
  drop_pending(sf, pd);
  return SF_SUCCESS;
}

// ---- memtype variants: host buffers staged through library-owned device buffers ----------
int sf_bcast_with_memtype_begin(sf_t *sf, sf_unit unit, int32_t rootmtype, const void *rootdata, int32_t leafmtype,
                                void *leafdata, int32_t op, sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  if ((rootmtype != SF_MEM_HOST && rootmtype != SF_MEM_DEVICE) || (leafmtype != SF_MEM_HOST && leafmtype != SF_MEM_DEVICE))
    return SF_ERR_ARG;
  if (find_pending(sf, K_BCAST_MT, unit, rootdata, leafdata, nullptr, op, rootmtype, leafmtype)) return SF_ERR_PENDING;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ub = size_t(elem_size(unit.dtype)) * unit.bs;
  const size_t rb = size_t(sf->info.nroots_total) * ub, lb = size_t(sf->info.leaf_extent_total) * ub;
  const void *droot = rootdata;
  void *dleaf = leafdata;
  if (rootmtype == SF_MEM_HOST) {
    if ((rc = ensure(sf->stage_root, rb, false, s))) return rc;
    if (rb && (rc = cuda_err(cudaMemcpyAsync(sf->stage_root.p, rootdata, rb, cudaMemcpyHostToDevice, s)))) return rc;
    droot = sf->stage_root.p;
  }
  if (leafmtype == SF_MEM_HOST) {
    if ((rc = ensure(sf->stage_leaf, lb, false, s))) return rc;
    // the whole leaf array goes back out, so it must come in unless REPLACE writes every slot
    const bool all_written = op == SF_REPLACE && sf->info.nedges == sf->info.leaf_extent_total;
    if (lb && !all_written &&
        (rc = cuda_err(cudaMemcpyAsync(sf->stage_leaf.p, leafdata, lb, cudaMemcpyHostToDevice, s))))
      return rc;
    dleaf = sf->stage_leaf.p;
  }
  int finish = 0;
  if ((rc = bcast_launch(sf, unit, droot, dleaf, op, s, bcast_path(sf, int64_t(elem_size(unit.dtype)) * unit.bs),
                         &finish)))
    return rc;
  sf->pending.push_back(Pending{K_BCAST_MT, unit, rootdata, leafdata, nullptr, op, rootmtype, leafmtype, finish});
  return SF_SUCCESS;
}

int sf_bcast_with_memtype_end(sf_t *sf, sf_unit unit, int32_t rootmtype, const void *rootdata, int32_t leafmtype,
                              void *leafdata, int32_t op, sf_stream_t stream) {
  if (!sf) return SF_ERR_NULL;
  Pending *pd = find_pending(sf, K_BCAST_MT, unit, rootdata, leafdata, nullptr, op, rootmtype, leafmtype);
  if (!pd) return SF_ERR_NO_PENDING;
  const int finish = pd->finish;
  drop_pending(sf, pd);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const void *droot = rootmtype == SF_MEM_HOST ? sf->stage_root.p : rootdata;
  void *dleaf = leafmtype == SF_MEM_HOST ? sf->stage_leaf.p : leafdata;
  int rc;
  if (finish && (rc = bcast_finish(sf, unit, droot, dleaf, op, s))) return rc;
  if (leafmtype == SF_MEM_HOST) {
    const size_t lb = size_t(sf->info.leaf_extent_total) * elem_size(unit.dtype) * unit.bs;
    if (lb && (rc = cuda_err(cudaMemcpyAsync(leafdata, sf->stage_leaf.p, lb, cudaMemcpyDeviceToHost, s)))) return rc;
  }
  return SF_SUCCESS;
}

int sf_reduce_with_memtype_begin(sf_t *sf, sf_unit unit, int32_t leafmtype, const void *leafdata, int32_t rootmtype,
                                 void *rootdata, int32_t op, sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  if ((rootmtype != SF_MEM_HOST && rootmtype != SF_MEM_DEVICE) || (leafmtype != SF_MEM_HOST && leafmtype != SF_MEM_DEVICE))
    return SF_ERR_ARG;
  if (find_pending(sf, K_REDUCE_MT, unit, leafdata, rootdata, nullptr, op, leafmtype, rootmtype)) return SF_ERR_PENDING;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ub = size_t(elem_size(unit.dtype)) * unit.bs;
  const size_t rb = size_t(sf->info.nroots_total) * ub, lb = size_t(sf->info.leaf_extent_total) * ub;
  const void *dleaf = leafdata;
  void *droot = rootdata;
  if (leafmtype == SF_MEM_HOST) {
    if ((rc = ensure(sf->stage_leaf, lb, false, s))) return rc;
    if (lb && (rc = cuda_err(cudaMemcpyAsync(sf->stage_leaf.p, leafdata, lb, cudaMemcpyHostToDevice, s)))) return rc;
    dleaf = sf->stage_leaf.p;
  }
  if (rootmtype == SF_MEM_HOST) {
    if ((rc = ensure(sf->stage_root, rb, false, s))) return rc;
    if (rb && (rc = cuda_err(cudaMemcpyAsync(sf->stage_root.p, rootdata, rb, cudaMemcpyHostToDevice, s)))) return rc;
    droot = sf->stage_root.p;
  }
  if ((rc = reduce_launch(sf, unit, dleaf, droot, op, s))) return rc;
  sf->pending.push_back(Pending{K_REDUCE_MT, unit, leafdata, rootdata, nullptr, op, leafmtype, rootmtype, 0});
  return SF_SUCCESS;
}

int sf_reduce_with_memtype_end(sf_t *sf, sf_unit unit, int32_t leafmtype, const void *leafdata, int32_t rootmtype,
                               void *rootdata, int32_t op, sf_stream_t stream) {
  if (!sf) return SF_ERR_NULL;
  Pending *pd = find_pending(sf, K_REDUCE_MT, unit, leafdata, rootdata, nullptr, op, leafmtype, rootmtype);
  if (!pd) return SF_ERR_NO_PENDING;
  drop_pending(sf, pd);
  if (rootmtype == SF_MEM_HOST) {
    const size_t rb = size_t(sf->info.nroots_total) * elem_size(unit.dtype) * unit.bs;
    if (rb) return cuda_err(cudaMemcpyAsync(rootdata, sf->stage_root.p, rb, cudaMemcpyDeviceToHost,
                                            static_cast<cudaStream_t>(stream)));
  }
  return SF_SUCCESS;
}

int sf_destroy(sf_t *sf) {
  if (!sf) return SF_SUCCESS;
  if (!sf->pending.empty()) return SF_ERR_PENDING;
  if (sf->multi) {
    const int rc = sf_destroy(sf->multi);
    if (rc) return rc;
    sf->multi = nullptr;
  }
  if (sf->setup) {
    release(sf->blob);
    release(sf->partial);
    release(sf->counter);
    release(sf->partial_arg);
    release(sf->rootbuf);
    release(sf->leafbuf);
    release(sf->stage_root);
    release(sf->stage_leaf);
    release(sf->status);
    release(sf->ts_tuned);
  }
  delete sf;
  return SF_SUCCESS;
}

static_assert(SF_DEVSTAT_STAGE_TIMEOUT == DEVSTAT_STAGE_TIMEOUT, "status bits agree");

int sf_get_device_status(sf_t *sf, sf_stream_t stream, int32_t *status) {
  int rc;
  if ((rc = ensure_ready(sf))) return rc;
  if (!status) return SF_ERR_NULL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t v = 0;
  if (cudaMemcpyAsync(&v, sf->status.p, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaMemsetAsync(sf->status.p, 0, sizeof v, s) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  *status = v;
  return SF_SUCCESS;
}

int sf_reduce_maxloc(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t *argleaf,
                     sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, SF_MAX))) return rc;
  const int w = elem_size(unit.dtype);
  if (sf->info.nroots_total && ((rc = check_ptr(rootdata, w)) || (rc = check_ptr(argleaf, 4)))) return rc;
  if (sf->info.leaf_extent_total && (rc = check_ptr(leafdata, w))) return rc;
  if (sf->info.nedges == 0) return SF_SUCCESS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (sf->dp.n_partial_slots > 0) {
    const size_t slots = size_t(sf->dp.n_partial_slots) * unit.bs;
    if ((rc = ensure(sf->partial, slots * w, false, s)) || (rc = ensure(sf->partial_arg, slots * 4, false, s)) ||
        (rc = ensure(sf->counter, size_t(sf->dp.n_counters) * unit.bs * 4, true, s)))
      return rc;
  }
  MaxlocArgs a{};
  a.mask = sf->dp.mask;
  a.pr_root = sf->dp.pr_root;
  a.pr_leaf = sf->dp.pr_leaf;
  a.m_leaf = sf->dp.m_leaf;
  a.blocks = sf->dp.blocks;
  a.combs = sf->dp.combs;
  a.tiles = sf->dp.rm_fold_tiles;
  a.out = rootdata;
  a.leaf = leafdata;
  a.arg = argleaf;
  a.partial = sf->partial.p;
  a.partial_arg = static_cast<int32_t *>(sf->partial_arg.p);
  a.counter = static_cast<int32_t *>(sf->counter.p);
  a.bs = unit.bs;
  a.status = static_cast<int32_t *>(sf->status.p);
  // gather-then-fold when the unit is vectors of 4, 8 or 16 bytes, no more than the kernel's
  // items per CTA (a round of the 22 KB buffer holds a whole unit), else the general kernel
  const int ub = w * unit.bs;
  const int pv = pick_vb(w, ub, true, {leafdata, rootdata});
  const int vb = pv == 16 ? 16 : w >= 4 ? w : 0;   // the vector widths the kernel is built for
  const int nv = vb ? ub / vb : 0;
  MaxlocFlat f{};
  const int max_nv = vb >= 16 ? (w < 4 ? 256 : 512) : 1024;   // the kernel's items per CTA
  if (vb >= 4 && nv >= 1 && nv <= max_nv && nv * vb <= RM_FLAT_BYTES) {
    const DivMagic dm = div_magic(uint32_t(nv));
    f = MaxlocFlat{nv, dm.m, dm.s};
    a.tiles = sf->dp.rm_fold_nv1_tiles;
    return launched(launch_maxloc(unit.dtype, a, sf->dp.n_rm_fold_nv1_tiles, vb, f, s));
  }
  return launched(launch_maxloc(unit.dtype, a, sf->dp.n_rm_fold_tiles, 0, f, s));
}

int sf_maxloc_grad(sf_t *sf, sf_unit unit, const int32_t *argleaf, const void *rootgrad, void *leafgrad,
                   sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, SF_MAX))) return rc;
  const int w = elem_size(unit.dtype);
  if (sf->info.nroots_total && ((rc = check_ptr(argleaf, 4)) || (rc = check_ptr(rootgrad, w)))) return rc;
  if (sf->info.leaf_extent_total && (rc = check_ptr(leafgrad, w))) return rc;
  if (sf->info.nedges == 0) return SF_SUCCESS;
  const int ub = w * unit.bs;
  const int vb = pick_vb(w, ub, true, {rootgrad, leafgrad}) == 16 ? 16 : w;
  MaxlocArgs a{};
  a.mask = sf->dp.mask;
  a.pr_root = sf->dp.pr_root;
  a.pr_leaf = sf->dp.pr_leaf;
  a.m_leaf = sf->dp.m_leaf;
  a.blocks = sf->dp.blocks;
  a.combs = sf->dp.combs;
  a.tiles = sf->dp.rm_fold_tiles;
  a.arg = const_cast<int32_t *>(argleaf);
  a.bs = unit.bs;
  return launched(launch_maxloc_grad(unit.dtype, a, sf->dp.n_rm_fold_tiles, vb, ub / vb, rootgrad, leafgrad,
                                     static_cast<cudaStream_t>(stream)));
}

int sf_maxloc_scatter(sf_t *sf, sf_unit unit, const int32_t *argleaf, const void *rootgrad, void *leafgrad,
                      sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, SF_MAX))) return rc;
  const int w = elem_size(unit.dtype);
  if (sf->info.nroots_total && ((rc = check_ptr(argleaf, 4)) || (rc = check_ptr(rootgrad, w)))) return rc;
  if (sf->info.leaf_extent_total && (rc = check_ptr(leafgrad, w))) return rc;
  const int64_t n = sf->info.nroots_total * int64_t(unit.bs);
  return launched(launch_maxloc_scatter(unit.dtype, argleaf, rootgrad, leafgrad, n, unit.bs,
                                        static_cast<cudaStream_t>(stream)));
}

const char *sf_error_string(int code) {
  switch (code) {
    case SF_SUCCESS: return "success";
    case SF_ERR_ARG: return "invalid argument";
    case SF_ERR_NULL: return "required pointer is NULL";
    case SF_ERR_RANGE: return "root address or leaf index out of range";
    case SF_ERR_DUP_LEAF: return "a rank lists the same leaf twice";
    case SF_ERR_STATE: return "call out of order (sf_setup not done)";
    case SF_ERR_NO_PENDING: return "End without a matching Begin";
    case SF_ERR_PENDING: return "a Begin with these arguments is still pending";
    case SF_ERR_UNSUPPORTED: return "combination not supported";
    case SF_ERR_ALLOC: return "allocation failed";
    case SF_ERR_CUDA: return "CUDA runtime error";
    case SF_ERR_ALIGN: return "data pointer not aligned to the element size";
    case SF_ERR_TOO_LARGE: return "sizes beyond 2^31-1 units";
  }
  return "unknown error code";
}

int64_t sf_launch_count(void) { return launch_counter().load(std::memory_order_relaxed); }

}  // extern "C"

// ---- deterministic Reduce without allocation ----------------------------------------------
// The fold partials and arrival counters of sf_reduce_noalloc live in this fixed array instead
// of the forest's cudaMalloc'd scratch.  Host code never uses the symbol itself (on the host it
// is only a stand-in, not a device address): the device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SF_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return SF_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SF_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SF_SUCCESS;
}
}  // namespace

extern "C" int sf_reduce_noalloc(sf_t *sf, sf_unit unit, const void *leafdata, void *rootdata, int32_t op,
                                 sf_stream_t stream) {
  int rc;
  if ((rc = ensure_ready(sf)) || (rc = check_unit(unit, op))) return rc;
  const int w = elem_size(unit.dtype), ub = w * unit.bs;
  if ((sf->info.nroots_total && (rc = check_ptr(rootdata, w))) ||
      (sf->info.leaf_extent_total && (rc = check_ptr(leafdata, w))))
    return rc;
  if (sf->info.nedges == 0) return SF_SUCCESS;
  const int vb = pick_vb(w, ub, true, {rootdata, leafdata});
  if (!vb) return SF_ERR_ALIGN;
  const int vbo = op == SF_REPLACE ? vb : (vb == 16 ? 16 : w);
  const int nv = ub / vbo;
  // counters first (256-byte rounded), then the partials
  size_t cbytes = 0, pbytes = 0;
  if (op != SF_REPLACE) {
    cbytes = size_t(sf->dp.n_counters) * nv * sizeof(int32_t);
    pbytes = size_t(sf->dp.n_partial_slots) * nv * acc_pack_bytes(unit.dtype, op, vbo);
  }
  const size_t coff = 0, poff = (cbytes + 255) & ~size_t(255);
  if (poff + pbytes > SF_NOALLOC_SCRATCH_BYTES) return SF_ERR_TOO_LARGE;
  void *scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char *base = static_cast<char *>(scratch);
  if (cbytes && (rc = cuda_err(cudaMemsetAsync(base + coff, 0, cbytes, s)))) return rc;
  return reduce_det_launch(sf, unit, leafdata, rootdata, op, s, vbo, nv, base + poff,
                           reinterpret_cast<int32_t *>(base + coff));
}
