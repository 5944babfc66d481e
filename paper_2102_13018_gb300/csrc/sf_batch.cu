// sf_batch.cu -- many forests' operations in few launches, optionally replayed as one CUDA
// graph, and the per-forest autotuner that picks the data path and Reduce mode.
//
// The paper counts about 10 us per kernel launch and shows how host synchronisation breaks the
// pipelining of launches (Sec. V.D, Fig. "pipelined vs interrupted launches"); its conclusion
// names CUDA graphs as future work.  A batch therefore groups its operations by kernel variant
// (element type, op, vector width, path) and launches each group once over a combined tile
// table of (operation, tile) pairs; with use_graph the launches of a run are captured once and
// replayed with a single cudaGraphLaunch.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "sf_object.h"

using namespace sfgb;

namespace {

struct Group {
  int stage;
  int family;   // 0 two-sided kernel, 1 root-major kernel, 2 diagonal-chunk Reduce
  int dtype, op, vb, mode;
  bool l2r, atomic;   // two-sided kernel
  int rm_form;        // root-major Reduce kernel: 0 general, 1 one vector per unit, 2 gather-then-fold
  size_t tiles_off;   // BatchTile offset in the tile table
  int ntiles;
};

bool same_ops(const std::vector<sf_batch_op> &a, const sf_batch_op *b, int32_t n) {
  if (int32_t(a.size()) != n) return false;
  for (int32_t i = 0; i < n; ++i)
    if (memcmp(&a[i], &b[i], sizeof(sf_batch_op)) != 0) return false;
  return true;
}

}  // namespace

struct sf_batch_s {
  std::vector<sf_batch_op> ops;    // the list the device tables were built for
  std::vector<int32_t> modes, paths;   // forests' resolved choices at build time
  // what the tables captured of every forest -- fold scratch (a later operation may reallocate
  // it), two-sided tile list, vector width and Reduce plan (sf_set_tile_edges,
  // sf_set_vector_bytes, sf_set_reduce_plan): a change rebuilds the tables
  struct Captured {
    const void *partial, *counter, *ts_tiles;
    int32_t vec_bytes, plan;
  };
  std::vector<Captured> scratch;
  DevBuf tables;
  const TsArgs *ts_ops = nullptr;
  const RmArgs *rm_ops = nullptr;
  const DgArgs *dg_ops = nullptr;
  const BatchTile *tiles = nullptr;
  std::vector<Group> groups;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  // the variant groups of a stage are independent: they run side by side on these streams,
  // forked from and joined back into the caller's stream (parallel branches in the graph)
  static constexpr int kLanes = 8;
  cudaStream_t lanes[kLanes] = {};
  cudaEvent_t fork = nullptr, join[kLanes] = {};
};

namespace {

void drop_graph(sf_batch_t *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Decide each operation's kernel variant and arguments, group them, upload the tables.
int build(sf_batch_t *b, const sf_batch_op *ops, int32_t n, cudaStream_t s) {
  std::vector<TsArgs> ts;
  std::vector<RmArgs> rm;
  std::vector<int32_t> rm_src;   // the operation each RmArgs belongs to
  std::vector<DgArgs> dg;
  std::vector<BatchTile> tiles;
  std::map<std::tuple<int, int, int, int, int, int, int, int>, std::vector<BatchTile>> grouped;
  std::vector<int32_t> modes(n, 0), paths(n, 0);
  int stage = 0;
  std::vector<std::pair<int, const sf_t *>> reduce_seen;   // (stage, forest) with fold scratch in use
  for (int32_t i = 0; i < n; ++i) {
    const sf_batch_op &o = ops[i];
    if (o.kind == SF_OP_BARRIER) {
      ++stage;
      continue;
    }
    sf_t *sf = o.sf;
    int rc;
    if (!sf) return SF_ERR_NULL;
    if (!sf->setup) return SF_ERR_STATE;
    if ((rc = check_unit(o.unit, o.op))) return rc;
    if (o.kind != SF_OP_BCAST && o.kind != SF_OP_REDUCE) return SF_ERR_ARG;
    const int w = elem_size(o.unit.dtype), ub = w * o.unit.bs;
    const void *root = o.kind == SF_OP_BCAST ? o.src : o.dst;
    const void *leaf = o.kind == SF_OP_BCAST ? o.dst : o.src;
    if ((sf->info.nroots_total && (rc = check_ptr(root, w))) || (sf->info.leaf_extent_total && (rc = check_ptr(leaf, w))))
      return rc;
    if (sf->info.nedges == 0) continue;
    if (o.kind == SF_OP_BCAST) {
      const int path = bcast_path(sf, ub);
      paths[i] = path;
      const int vb = pick_vb_sf(sf, w, ub, true, {root, leaf});
      if (!vb) return SF_ERR_ALIGN;
      const int vbo = o.op == SF_REPLACE ? vb : (vb == 16 ? 16 : w);
      if (path == SF_PATH_ROOT_MAJOR) {
        const int idx = int(rm.size());
        rm.push_back(rm_args(sf, sf->dp.rm_fold_tiles, sf->dp.n_rm_fold_tiles, const_cast<void *>(root),
                             const_cast<void *>(leaf), nullptr, ub / vbo));
        rm_src.push_back(i);
        auto &g = grouped[{stage, 1, o.unit.dtype, o.op, vbo, RM_BCAST, 0, 0}];
        for (int32_t t = 0; t < sf->dp.n_rm_fold_tiles; ++t) g.push_back(BatchTile{idx, 0, sf->dp.rm_fold_tiles + t});
      } else {   // fused (the three-phase path is not batched)
        const int idx = int(ts.size());
        ts.push_back(ts_args(sf, sf->dp.ts_tiles, sf->dp.n_ts_tiles, root, const_cast<void *>(leaf), nullptr, ub / vbo,
                             PH_FUSED));
        auto &g = grouped[{stage, 0, o.unit.dtype, o.op, vbo, 0, 0, 0}];
        for (int32_t t = 0; t < sf->dp.n_ts_tiles; ++t) g.push_back(BatchTile{idx, 0, sf->dp.ts_tiles + t});
      }
    } else {
      const int mode = reduce_mode(sf);
      modes[i] = mode;
      if (reduce_atomic(sf, o.unit.dtype, o.op)) {
        const int idx = int(ts.size());
        ts.push_back(ts_args(sf, sf->dp.ts_tiles, sf->dp.n_ts_tiles, leaf, const_cast<void *>(root), nullptr, o.unit.bs,
                             PH_FUSED));
        auto &g = grouped[{stage, 0, o.unit.dtype, o.op, w, 0, 1, 1}];
        for (int32_t t = 0; t < sf->dp.n_ts_tiles; ++t) g.push_back(BatchTile{idx, 0, sf->dp.ts_tiles + t});
      } else {
        const int vb = pick_vb_sf(sf, w, ub, true, {root, leaf});
        if (!vb) return SF_ERR_ALIGN;
        const int vbo = o.op == SF_REPLACE ? vb : (vb == 16 ? 16 : w);
        const int nv = ub / vbo;
        if (o.op != SF_REPLACE && sf->dp.n_partial_slots > 0) {
          for (auto &p : reduce_seen)
            if (p.first == stage && p.second == sf) return SF_ERR_ARG;   // one fold scratch per forest
          reduce_seen.push_back({stage, sf});
          const size_t pbytes = size_t(sf->dp.n_partial_slots) * nv * acc_pack_bytes(o.unit.dtype, o.op, vbo);
          const size_t cbytes = size_t(sf->dp.n_counters) * nv * sizeof(int32_t);
          if ((rc = ensure(sf->partial, pbytes, false, s)) || (rc = ensure(sf->counter, cbytes, true, s))) return rc;
        }
        // diagonal chunks first (their tiles by index), then the root-major plan of the rest
        const DevPlan *d = &sf->dp;
        if (reduce_dg(sf, o.op, nv)) {
          const int idx = int(dg.size());
          dg.push_back(dg_args(sf, leaf, const_cast<void *>(root)));
          auto &g = grouped[{stage, 2, o.unit.dtype, o.op, vbo, 0, 0, 0}];
          for (int32_t t = 0; t < dg.back().ntiles; ++t) g.push_back(BatchTile{idx, t, nullptr});
          d = sf->has_rest ? &sf->dp_rest : nullptr;
        }
        // one vector per unit, or a few (gather-then-fold): the group runs the Reduce kernel of
        // that form, on the forest's chunk tiles cut for it
        const bool nv1 = reduce_nv1(o.op, vbo, nv), flat = reduce_flat(o.op, vbo, nv), l1 = nv1 || flat;
        const int nt = !d ? 0 : o.op == SF_REPLACE ? d->n_rm_winner_tiles
                                                   : l1 ? d->n_rm_fold_nv1_tiles : d->n_rm_fold_tiles;
        if (nt > 0) {
          const RmTile *rt = o.op == SF_REPLACE ? d->rm_winner_tiles : l1 ? d->rm_fold_nv1_tiles : d->rm_fold_tiles;
          const int idx = int(rm.size());
          rm.push_back(rm_args_plan(sf, *d, rt, nt, const_cast<void *>(root), const_cast<void *>(leaf), nullptr, nv));
          rm_src.push_back(i);
          auto &g = grouped[{stage, 1, o.unit.dtype, o.op, vbo, RM_REDUCE, nv1 ? 1 : flat ? 2 : 0, 0}];
          for (int32_t t = 0; t < nt; ++t) g.push_back(BatchTile{idx, 0, rt + t});
        }
      }
    }
  }
  // rm_args captured the forests' scratch pointers before any ensure() above could move them:
  // refresh them now that every scratch buffer has its final size
  for (size_t r = 0; r < rm.size(); ++r) {
    const sf_t *sf = ops[rm_src[r]].sf;
    rm[r].partial = sf->partial.p;
    rm[r].counter = static_cast<int32_t *>(sf->counter.p);
  }
  b->groups.clear();
  for (auto &kv : grouped) {
    const auto &k = kv.first;
    Group g{};
    g.stage = std::get<0>(k);
    g.family = std::get<1>(k);
    g.dtype = std::get<2>(k);
    g.op = std::get<3>(k);
    g.vb = std::get<4>(k);
    g.mode = std::get<5>(k);
    g.l2r = g.family == 0 && std::get<6>(k) != 0;
    g.rm_form = g.family == 1 ? std::get<6>(k) : 0;
    g.atomic = std::get<7>(k);
    g.tiles_off = tiles.size();
    g.ntiles = int(kv.second.size());
    tiles.insert(tiles.end(), kv.second.begin(), kv.second.end());
    b->groups.push_back(g);
  }
  // upload: [TsArgs][RmArgs][DgArgs][BatchTile], 256-byte aligned pieces
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t o_ts = 0, o_rm = al(ts.size() * sizeof(TsArgs)), o_dg = o_rm + al(rm.size() * sizeof(RmArgs)),
               o_t = o_dg + al(dg.size() * sizeof(DgArgs));
  const size_t bytes = std::max<size_t>(o_t + tiles.size() * sizeof(BatchTile), 256);
  std::vector<char> host(bytes, 0);
  if (!ts.empty()) memcpy(host.data() + o_ts, ts.data(), ts.size() * sizeof(TsArgs));
  if (!rm.empty()) memcpy(host.data() + o_rm, rm.data(), rm.size() * sizeof(RmArgs));
  if (!dg.empty()) memcpy(host.data() + o_dg, dg.data(), dg.size() * sizeof(DgArgs));
  if (!tiles.empty()) memcpy(host.data() + o_t, tiles.data(), tiles.size() * sizeof(BatchTile));
  int rc;
  if (b->tables.bytes < bytes) {
    if ((rc = cuda_err(cudaStreamSynchronize(s)))) return rc;
    release(b->tables);
    if ((rc = ensure(b->tables, bytes, false, s))) return rc;
  }
  if ((rc = cuda_err(cudaMemcpyAsync(b->tables.p, host.data(), bytes, cudaMemcpyHostToDevice, s)))) return rc;
  if ((rc = cuda_err(cudaStreamSynchronize(s)))) return rc;   // `host` dies at return
  char *base = static_cast<char *>(b->tables.p);
  b->ts_ops = reinterpret_cast<const TsArgs *>(base + o_ts);
  b->rm_ops = reinterpret_cast<const RmArgs *>(base + o_rm);
  b->dg_ops = reinterpret_cast<const DgArgs *>(base + o_dg);
  b->tiles = reinterpret_cast<const BatchTile *>(base + o_t);
  b->ops.assign(ops, ops + n);
  b->modes = modes;
  b->paths = paths;
  b->scratch.assign(n, {nullptr, nullptr, nullptr, 0, 0});
  for (int32_t i = 0; i < n; ++i)
    if (ops[i].kind != SF_OP_BARRIER) {
      const sf_t *sf = ops[i].sf;
      b->scratch[i] = {sf->partial.p, sf->counter.p, sf->dp.ts_tiles, sf->vec_bytes, reduce_plan(sf)};
    }
  return SF_SUCCESS;
}

int launch_group(const sf_batch_t *b, const Group &g, cudaStream_t s) {
  cudaError_t e;
  if (g.family == 0)
    e = launch_ts(g.dtype, g.op, g.vb, g.l2r, g.atomic, false, TsLaunch{nullptr, b->ts_ops, b->tiles + g.tiles_off, g.ntiles, s});
  else if (g.family == 2)
    e = launch_dg(g.dtype, g.op, g.vb, DgLaunch{nullptr, b->dg_ops, b->tiles + g.tiles_off, g.ntiles, g.ntiles, s});
  else
    e = launch_rm(g.dtype, g.op, g.vb, g.mode,
                  RmLaunch{nullptr, b->rm_ops, b->tiles + g.tiles_off, g.ntiles, s, g.rm_form == 1, g.rm_form == 2});
  return launched(e);
}

int ensure_lanes(sf_batch_t *b) {
  if (b->fork) return SF_SUCCESS;
  int rc;
  for (int l = 0; l < sf_batch_t::kLanes; ++l) {
    if ((rc = cuda_err(cudaStreamCreateWithFlags(&b->lanes[l], cudaStreamNonBlocking)))) return rc;
    if ((rc = cuda_err(cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming)))) return rc;
  }
  return cuda_err(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
}

// Stage by stage (the groups are sorted by stage): a stage of one group runs on `s`; the groups
// of a larger stage go to the lanes, largest first onto the least loaded lane (by tiles), and
// `s` waits for every lane used before the next stage.  On the 512-forest batch 8 lanes replay
// 3% faster than 4, and 4 were 21% faster than one stream.
int launch_groups(sf_batch_t *b, cudaStream_t s) {
  int rc;
  const size_t ng = b->groups.size();
  for (size_t i0 = 0; i0 < ng;) {
    size_t i1 = i0;
    while (i1 < ng && b->groups[i1].stage == b->groups[i0].stage) ++i1;
    if (i1 - i0 == 1) {
      if ((rc = launch_group(b, b->groups[i0], s))) return rc;
      i0 = i1;
      continue;
    }
    if ((rc = ensure_lanes(b)) || (rc = cuda_err(cudaEventRecord(b->fork, s)))) return rc;
    std::vector<size_t> order;
    for (size_t i = i0; i < i1; ++i) order.push_back(i);
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return b->groups[x].ntiles > b->groups[y].ntiles; });
    int64_t load[sf_batch_t::kLanes] = {};
    bool used[sf_batch_t::kLanes] = {};
    for (size_t i : order) {
      int l = 0;
      for (int k = 1; k < sf_batch_t::kLanes; ++k)
        if (load[k] < load[l]) l = k;
      if (!used[l] && (rc = cuda_err(cudaStreamWaitEvent(b->lanes[l], b->fork, 0)))) return rc;
      used[l] = true;
      load[l] += b->groups[i].ntiles;
      if ((rc = launch_group(b, b->groups[i], b->lanes[l]))) return rc;
    }
    for (int l = 0; l < sf_batch_t::kLanes; ++l)
      if (used[l] && ((rc = cuda_err(cudaEventRecord(b->join[l], b->lanes[l]))) ||
                      (rc = cuda_err(cudaStreamWaitEvent(s, b->join[l], 0)))))
        return rc;
    i0 = i1;
  }
  return SF_SUCCESS;
}

// the forests' current choices or fold scratch differ from those the tables were built with
bool choices_changed(const sf_batch_t *b) {
  for (size_t i = 0; i < b->ops.size(); ++i) {
    const sf_batch_op &o = b->ops[i];
    if (o.kind == SF_OP_BARRIER) continue;
    if (o.kind == SF_OP_BCAST && bcast_path(o.sf, int64_t(elem_size(o.unit.dtype)) * o.unit.bs) != b->paths[i])
      return true;
    if (o.kind == SF_OP_REDUCE && reduce_mode(o.sf) != b->modes[i]) return true;
    const auto &c = b->scratch[i];
    if (c.partial != o.sf->partial.p || c.counter != o.sf->counter.p || c.ts_tiles != o.sf->dp.ts_tiles ||
        c.vec_bytes != o.sf->vec_bytes || c.plan != reduce_plan(o.sf))
      return true;
  }
  return false;
}

}  // namespace

extern "C" {

int sf_batch_create(sf_batch_t **out) {
  if (!out) return SF_ERR_NULL;
  *out = new (std::nothrow) sf_batch_t();
  return *out ? SF_SUCCESS : SF_ERR_ALLOC;
}

int sf_batch_run(sf_batch_t *b, const sf_batch_op ops[], int32_t n, int32_t use_graph, sf_stream_t stream) {
  if (!b || (n > 0 && !ops)) return SF_ERR_NULL;
  if (n < 0) return SF_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  if (!same_ops(b->ops, ops, n) || choices_changed(b)) {
    drop_graph(b);
    if ((rc = build(b, ops, n, s))) {
      b->ops.clear();
      return rc;
    }
  }
  if (!use_graph) return launch_groups(b, s);
  if (!b->exec) {
    if (!b->capture_stream && (rc = cuda_err(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking))))
      return rc;
    if ((rc = cuda_err(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal)))) return rc;
    const int lrc = launch_groups(b, b->capture_stream);
    // captured launches run only when the graph is launched: count them there
    launch_counter().fetch_sub(int64_t(b->groups.size()), std::memory_order_relaxed);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->capture_stream, &graph);
    if (lrc) {
      if (graph) cudaGraphDestroy(graph);
      return lrc;
    }
    if ((rc = cuda_err(ec))) return rc;
    b->graph = graph;
    if ((rc = cuda_err(cudaGraphInstantiate(&b->exec, b->graph, 0)))) {
      drop_graph(b);
      return rc;
    }
  }
  if ((rc = cuda_err(cudaGraphLaunch(b->exec, s)))) return rc;
  launch_counter().fetch_add(int64_t(b->groups.size()), std::memory_order_relaxed);
  return SF_SUCCESS;
}

int sf_batch_launches(const sf_batch_t *b, int32_t *launches) {
  if (!b || !launches) return SF_ERR_NULL;
  *launches = int32_t(b->groups.size());
  return SF_SUCCESS;
}

int sf_batch_destroy(sf_batch_t *b) {
  if (!b) return SF_SUCCESS;
  drop_graph(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (int l = 0; l < sf_batch_t::kLanes; ++l) {
    if (b->lanes[l]) cudaStreamDestroy(b->lanes[l]);
    if (b->join[l]) cudaEventDestroy(b->join[l]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  release(b->tables);
  delete b;
  return SF_SUCCESS;
}

// Time the candidate variants of Bcast or Reduce on a scratch copy of the output and keep the
// fastest: path or mode (what AUTO means), vector width and two-sided tile size.
int sf_autotune(sf_t *sf, sf_unit unit, int32_t kind, const void *src, void *dst, int32_t op, int32_t reps,
                sf_stream_t stream, int32_t *choice) {
  int rc;
  if (!sf) return SF_ERR_NULL;
  if (!sf->setup) return SF_ERR_STATE;
  if ((rc = check_unit(unit, op))) return rc;
  if (kind != SF_OP_BCAST && kind != SF_OP_REDUCE) return SF_ERR_ARG;
  if (reps < 1) reps = 3;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int w = elem_size(unit.dtype);
  const size_t ub = size_t(w) * unit.bs;
  const size_t bytes = ub * size_t(kind == SF_OP_BCAST ? sf->info.leaf_extent_total : sf->info.nroots_total);
  struct Cand {
    int32_t c, vec, edges;   // path or mode, vector bytes, tile edges (0: setup's)
    int32_t plan;            // deterministic Reduce plan
  };
  std::vector<Cand> cands;
  std::vector<int32_t> vecs = {0};
  if (ub % 16 == 0 && w < 16) vecs.push_back(w);           // 16-byte vectors or single elements
  else if (ub % 8 == 0 && w < 8) vecs.push_back(w);
  const int32_t sizes[] = {0, 512, 1024, 2048, 4096};
  const int32_t plan0 = sf->plan;
  if (kind == SF_OP_BCAST) {
    for (int32_t v : vecs) {
      for (int32_t e : sizes) cands.push_back({SF_PATH_FUSED, v, e, plan0});
      cands.push_back({SF_PATH_ROOT_MAJOR, v, 0, plan0});
      cands.push_back({SF_PATH_THREE_PHASE, v, 0, plan0});
    }
  } else {
    const bool fixed = sf->mode == SF_MODE_DETERMINISTIC || op == SF_REPLACE || unit.dtype == SF_BF16;
    // the diagonal plans serve one-vector units of SUM/MIN/MAX on forests with diagonal chunks
    std::vector<int32_t> plans = {plan0};
    if (plan0 == SF_PLAN_AUTO && sf->dp.dg_nchunks > 0 && op != SF_REPLACE)
      plans = {SF_PLAN_ROOT_MAJOR, SF_PLAN_DIAGONAL, SF_PLAN_DIAGONAL_STAGED};
    for (int32_t v : vecs)
      for (int32_t p : plans) cands.push_back({SF_MODE_DETERMINISTIC, v, sf->tile_edges, p});
    if (!fixed)
      for (int32_t e : sizes) cands.push_back({SF_MODE_ATOMIC, 0, e, plan0});
  }
  DevBuf scratch;
  if ((rc = ensure(scratch, std::max<size_t>(bytes, 256), false, s))) return rc;
  cudaEvent_t e0, e1;
  if ((rc = cuda_err(cudaEventCreate(&e0)))) { release(scratch); return rc; }
  if ((rc = cuda_err(cudaEventCreate(&e1)))) { cudaEventDestroy(e0); release(scratch); return rc; }
  const int32_t vec0 = sf->vec_bytes, edges0 = sf->tile_edges;
  float best = 1e30f;
  Cand best_c = cands[0];
  for (const Cand &c : cands) {
    sf->vec_bytes = c.vec;
    sf->plan = c.plan;
    if ((rc = sf_set_tile_edges(sf, c.edges))) break;
    float total = 0.f;
    for (int r = 0; r <= reps && !rc; ++r) {   // first round warms up
      if (bytes) rc = cuda_err(cudaMemcpyAsync(scratch.p, dst, bytes, cudaMemcpyDeviceToDevice, s));
      if (!rc) rc = cuda_err(cudaEventRecord(e0, s));
      if (!rc) rc = kind == SF_OP_BCAST ? bcast_all(sf, unit, src, scratch.p, op, s, c.c)
                                        : reduce_all(sf, unit, src, scratch.p, op, s, c.c);
      if (!rc) rc = cuda_err(cudaEventRecord(e1, s));
      if (!rc) rc = cuda_err(cudaEventSynchronize(e1));
      float ms = 0.f;
      if (!rc) rc = cuda_err(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) total += ms;
    }
    if (rc) break;
    if (total < best) {
      best = total;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release(scratch);
  sf->vec_bytes = vec0;
  sf->plan = plan0;
  if (rc) {
    sf_set_tile_edges(sf, edges0);
    return rc;
  }
  sf->vec_bytes = best_c.vec;
  if ((rc = sf_set_tile_edges(sf, best_c.edges))) return rc;
  if (kind == SF_OP_BCAST) {
    sf->tuned_path = best_c.c;
    sf->path_tuned = true;
  }
  else sf->tuned_mode = best_c.c;
  if (kind == SF_OP_REDUCE && best_c.c == SF_MODE_DETERMINISTIC && plan0 == SF_PLAN_AUTO && best_c.plan != SF_PLAN_AUTO)
    sf->tuned_plan = best_c.plan;
  if (choice) *choice = best_c.c;
  return SF_SUCCESS;
}

}  // extern "C"
