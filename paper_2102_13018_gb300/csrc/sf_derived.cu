// sf_derived.cu -- forests derived from forests (Sec. III.B-C):
//  * composition: AB connects A's roots to B's leaves through A's leaves = B's roots; the
//    inverse composition connects A's roots to B's roots through their shared leaves;
//  * embedded root / leaf forests: the edges of selected roots or leaves only, with the same
//    root and leaf numbering, so the original data buffers serve the new forest;
//  * the multi-forest: every root split into as many roots as it has leaves, leaf i of a root
//    connected to its own new root; built with FetchAndOp SUM (roots start at their rank's
//    degree prefix sums, leaves add 1, each leaf fetches its new root's offset) exactly as the
//    paper describes, then Gather / Scatter are Reduce / Bcast REPLACE over it.
#include <algorithm>
#include <vector>

#include "sf_object.h"

using namespace sfgb;

namespace {

// New forest from a subset of the edges of `sf` (keep[e] in canonical order), same layout.
int subset(const sf_t *sf, const std::vector<uint8_t> &keep, sf_t **out) {
  const Graph &g = sf->g;
  const int32_t P = g.P;
  std::vector<int64_t> nleaves(P, 0), extents(P);
  std::vector<std::vector<int64_t>> il(P);
  std::vector<std::vector<sf_node>> ir(P);
  for (int32_t q = 0; q < P; ++q) {
    extents[q] = g.leafoff[q + 1] - g.leafoff[q];
    for (int64_t i = 0, e = g.edgeoff[q]; e < g.edgeoff[q + 1]; ++i, ++e) {
      if (!keep[e]) continue;
      il[q].push_back(g.has_ilocal[q] ? g.ilocal[e] : i);
      ir[q].push_back(sf_node{g.rrank[e], g.rindex[e]});
      nleaves[q]++;
    }
  }
  std::vector<const int64_t *> ilp(P);
  std::vector<const sf_node *> irp(P);
  for (int32_t q = 0; q < P; ++q) {
    ilp[q] = il[q].empty() ? nullptr : il[q].data();
    irp[q] = ir[q].empty() ? nullptr : ir[q].data();
  }
  sf_t *n = new (std::nothrow) sf_t();
  if (!n) return SF_ERR_ALLOC;
  const int rc = build_graph_extents(P, g.nroots.data(), nleaves.data(), ilp.data(), irp.data(), extents.data(), n->g);
  if (rc) {
    delete n;
    return rc;
  }
  n->info.nranks = P;
  n->mode = sf->mode;
  n->path = sf->path;
  *out = n;
  return SF_SUCCESS;
}

int to_device(DevBuf &b, const void *host, size_t bytes, cudaStream_t s) {
  int rc;
  if ((rc = ensure(b, std::max<size_t>(bytes, 16), false, s))) return rc;
  if (bytes && (rc = cuda_err(cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, s)))) return rc;
  return cuda_err(cudaStreamSynchronize(s));
}

// The multi-forest of `sf` (Sec. III.B), built on the device with Reduce and FetchAndOp.
int build_multi(sf_t *sf, cudaStream_t s, sf_t **out) {
  const Graph &g = sf->g;
  const int32_t P = g.P;
  const int64_t NR = sf->info.nroots_total, NL = sf->info.leaf_extent_total;
  const sf_unit u{SF_INT32, 1};
  int rc;
  DevBuf ones, deg, upd;
  std::vector<int32_t> h_ones(NL, 1), h_deg(NR, 0), h_off(NR, 0), h_upd(NL, -1);
  auto cleanup = [&]() { release(ones); release(deg); release(upd); };
  // 1. in-degrees: Reduce SUM of ones into zeros
  if ((rc = to_device(ones, h_ones.data(), NL * 4, s)) || (rc = to_device(deg, h_deg.data(), NR * 4, s)) ||
      (rc = to_device(upd, h_upd.data(), NL * 4, s))) {
    cleanup();
    return rc;
  }
  if ((rc = reduce_all(sf, u, ones.p, deg.p, SF_SUM, s, SF_MODE_DETERMINISTIC)) ||
      (rc = cuda_err(cudaMemcpyAsync(h_deg.data(), deg.p, NR * 4, cudaMemcpyDeviceToHost, s))) ||
      (rc = cuda_err(cudaStreamSynchronize(s)))) {
    cleanup();
    return rc;
  }
  // 2. roots start at their rank's degree prefix sums
  std::vector<int64_t> mroots(P, 0);
  for (int32_t p = 0; p < P; ++p) {
    int64_t acc = 0;
    for (int64_t r = g.rootoff[p]; r < g.rootoff[p + 1]; ++r) {
      h_off[r] = int32_t(acc);
      acc += h_deg[r];
    }
    mroots[p] = acc;
  }
  // 3. FetchAndOp SUM with leaves = 1: each leaf fetches its new root (canonical order per root)
  if ((rc = to_device(deg, h_off.data(), NR * 4, s))) {
    cleanup();
    return rc;
  }
  const int32_t saved = sf->mode;
  sf->mode = SF_MODE_DETERMINISTIC;
  rc = sf_fetch_and_op_begin(sf, u, deg.p, ones.p, upd.p, SF_SUM, s);
  if (!rc) rc = sf_fetch_and_op_end(sf, u, deg.p, ones.p, upd.p, SF_SUM, s);
  sf->mode = saved;
  if (rc || (rc = cuda_err(cudaMemcpyAsync(h_upd.data(), upd.p, NL * 4, cudaMemcpyDeviceToHost, s))) ||
      (rc = cuda_err(cudaStreamSynchronize(s)))) {
    cleanup();
    return rc;
  }
  cleanup();
  // 4. the multi-forest: same leaves, leaf -> (root rank, fetched offset)
  std::vector<int64_t> nleaves(P), extents(P);
  std::vector<std::vector<int64_t>> il(P);
  std::vector<std::vector<sf_node>> ir(P);
  for (int32_t q = 0; q < P; ++q) {
    nleaves[q] = g.nleaves[q];
    extents[q] = g.leafoff[q + 1] - g.leafoff[q];
    for (int64_t i = 0, e = g.edgeoff[q]; e < g.edgeoff[q + 1]; ++i, ++e) {
      const int64_t l = g.has_ilocal[q] ? g.ilocal[e] : i;
      il[q].push_back(l);
      ir[q].push_back(sf_node{g.rrank[e], int64_t(h_upd[g.leafoff[q] + l])});
    }
  }
  std::vector<const int64_t *> ilp(P);
  std::vector<const sf_node *> irp(P);
  for (int32_t q = 0; q < P; ++q) {
    ilp[q] = il[q].empty() ? nullptr : il[q].data();
    irp[q] = ir[q].empty() ? nullptr : ir[q].data();
  }
  sf_t *m = new (std::nothrow) sf_t();
  if (!m) return SF_ERR_ALLOC;
  if ((rc = build_graph_extents(P, mroots.data(), nleaves.data(), ilp.data(), irp.data(), extents.data(), m->g))) {
    delete m;
    return rc;
  }
  m->info.nranks = P;
  if ((rc = sf_setup(m, s))) {
    sf_destroy(m);
    return rc;
  }
  *out = m;
  return SF_SUCCESS;
}

// AB from per-rank leaf lists: leaves[q] = (local index, root rank, root index), layout of the
// leaf space given by extents, roots by nroots.
int from_edges(int32_t P, const std::vector<int64_t> &nroots, const std::vector<int64_t> &extents,
               const std::vector<std::vector<std::pair<int64_t, sf_node>>> &leaves, sf_t **out) {
  std::vector<int64_t> nleaves(P);
  std::vector<std::vector<int64_t>> il(P);
  std::vector<std::vector<sf_node>> ir(P);
  for (int32_t q = 0; q < P; ++q) {
    nleaves[q] = int64_t(leaves[q].size());
    for (const auto &lv : leaves[q]) {
      il[q].push_back(lv.first);
      ir[q].push_back(lv.second);
    }
  }
  std::vector<const int64_t *> ilp(P);
  std::vector<const sf_node *> irp(P);
  for (int32_t q = 0; q < P; ++q) {
    ilp[q] = il[q].empty() ? nullptr : il[q].data();
    irp[q] = ir[q].empty() ? nullptr : ir[q].data();
  }
  sf_t *n = new (std::nothrow) sf_t();
  if (!n) return SF_ERR_ALLOC;
  const int rc = build_graph_extents(P, nroots.data(), nleaves.data(), ilp.data(), irp.data(), extents.data(), n->g);
  if (rc) {
    delete n;
    return rc;
  }
  n->info.nranks = P;
  *out = n;
  return SF_SUCCESS;
}

// root of the edge leaving global leaf unit l of `g`, or {-1, -1} when l is isolated
std::vector<sf_node> leaf_to_root(const Graph &g) {
  std::vector<sf_node> m(g.leafoff[g.P], sf_node{-1, -1});
  for (int32_t q = 0; q < g.P; ++q)
    for (int64_t i = 0, e = g.edgeoff[q]; e < g.edgeoff[q + 1]; ++i, ++e)
      m[g.leafoff[q] + (g.has_ilocal[q] ? g.ilocal[e] : i)] = sf_node{g.rrank[e], g.rindex[e]};
  return m;
}

}  // namespace

extern "C" {

int sf_compose(const sf_t *A, const sf_t *B, sf_t **AB) {
  if (!A || !B || !AB) return SF_ERR_NULL;
  const Graph &a = A->g, &b = B->g;
  if (a.P != b.P) return SF_ERR_ARG;
  for (int32_t p = 0; p < a.P; ++p)   // A's leaf space is B's root space
    if (a.leafoff[p + 1] - a.leafoff[p] != b.nroots[p]) return SF_ERR_ARG;
  const std::vector<sf_node> aroot = leaf_to_root(a);
  std::vector<std::vector<std::pair<int64_t, sf_node>>> leaves(b.P);
  std::vector<int64_t> extents(b.P);
  for (int32_t q = 0; q < b.P; ++q) {
    extents[q] = b.leafoff[q + 1] - b.leafoff[q];
    for (int64_t i = 0, e = b.edgeoff[q]; e < b.edgeoff[q + 1]; ++i, ++e) {
      const sf_node r = aroot[a.leafoff[b.rrank[e]] + b.rindex[e]];   // B's root = A's leaf
      if (r.rank >= 0) leaves[q].push_back({b.has_ilocal[q] ? b.ilocal[e] : i, r});
    }
  }
  return from_edges(a.P, a.nroots, extents, leaves, AB);
}

int sf_compose_inverse(const sf_t *A, const sf_t *B, sf_t **AB) {
  if (!A || !B || !AB) return SF_ERR_NULL;
  const Graph &a = A->g, &b = B->g;
  if (a.P != b.P) return SF_ERR_ARG;
  for (int32_t p = 0; p <= a.P; ++p)   // A and B share the leaf space
    if (a.leafoff[p] != b.leafoff[p]) return SF_ERR_ARG;
  const std::vector<sf_node> aroot = leaf_to_root(a);
  std::vector<uint8_t> seen(b.rootoff[b.P], 0);
  std::vector<std::vector<std::pair<int64_t, sf_node>>> leaves(b.P);
  for (int32_t q = 0; q < b.P; ++q)
    for (int64_t i = 0, e = b.edgeoff[q]; e < b.edgeoff[q + 1]; ++i, ++e) {
      const int64_t broot = b.rootoff[b.rrank[e]] + b.rindex[e];
      if (seen[broot]++) return SF_ERR_ARG;   // B's roots must have degree at most one
      const sf_node r = aroot[b.leafoff[q] + (b.has_ilocal[q] ? b.ilocal[e] : i)];
      if (r.rank >= 0) leaves[b.rrank[e]].push_back({b.rindex[e], r});   // leaf = B's root
    }
  for (auto &l : leaves) std::sort(l.begin(), l.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
  return from_edges(a.P, a.nroots, b.nroots, leaves, AB);
}


int sf_create_embedded_root_sf(const sf_t *sf, int64_t n, const int64_t selected_roots[], sf_t **out) {
  if (!sf || !out || (n > 0 && !selected_roots)) return SF_ERR_NULL;
  if (n < 0) return SF_ERR_ARG;
  const int64_t NR = sf->g.rootoff[sf->g.P];
  std::vector<uint8_t> sel(NR, 0), keep(sf->g.E, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (selected_roots[i] < 0 || selected_roots[i] >= NR) return SF_ERR_RANGE;
    sel[selected_roots[i]] = 1;
  }
  for (int64_t e = 0; e < sf->g.E; ++e) keep[e] = sel[sf->g.rootoff[sf->g.rrank[e]] + sf->g.rindex[e]];
  return subset(sf, keep, out);
}

int sf_create_embedded_leaf_sf(const sf_t *sf, int64_t n, const int64_t selected_leaves[], sf_t **out) {
  if (!sf || !out || (n > 0 && !selected_leaves)) return SF_ERR_NULL;
  if (n < 0) return SF_ERR_ARG;
  const Graph &g = sf->g;
  const int64_t NL = g.leafoff[g.P];
  std::vector<uint8_t> sel(NL, 0), keep(g.E, 0);
  for (int64_t i = 0; i < n; ++i) {
    if (selected_leaves[i] < 0 || selected_leaves[i] >= NL) return SF_ERR_RANGE;
    sel[selected_leaves[i]] = 1;
  }
  for (int32_t q = 0; q < g.P; ++q)
    for (int64_t i = 0, e = g.edgeoff[q]; e < g.edgeoff[q + 1]; ++i, ++e)
      keep[e] = sel[g.leafoff[q] + (g.has_ilocal[q] ? g.ilocal[e] : i)];
  return subset(sf, keep, out);
}

int sf_get_multi_sf(sf_t *sf, sf_stream_t stream, sf_t **multi) {
  int rc;
  if (!sf || !multi) return SF_ERR_NULL;
  if (!sf->setup) return SF_ERR_STATE;
  if (!sf->multi && (rc = build_multi(sf, static_cast<cudaStream_t>(stream), &sf->multi))) return rc;
  *multi = sf->multi;
  return SF_SUCCESS;
}

int sf_gather_begin(sf_t *sf, sf_unit unit, const void *leafdata, void *multirootdata, sf_stream_t stream) {
  sf_t *m;
  int rc;
  if ((rc = sf_get_multi_sf(sf, stream, &m))) return rc;
  return sf_reduce_begin(m, unit, leafdata, multirootdata, SF_REPLACE, stream);
}

int sf_gather_end(sf_t *sf, sf_unit unit, const void *leafdata, void *multirootdata, sf_stream_t stream) {
  if (!sf) return SF_ERR_NULL;
  if (!sf->multi) return SF_ERR_NO_PENDING;
  return sf_reduce_end(sf->multi, unit, leafdata, multirootdata, SF_REPLACE, stream);
}

int sf_scatter_begin(sf_t *sf, sf_unit unit, const void *multirootdata, void *leafdata, sf_stream_t stream) {
  sf_t *m;
  int rc;
  if ((rc = sf_get_multi_sf(sf, stream, &m))) return rc;
  return sf_bcast_begin(m, unit, multirootdata, leafdata, SF_REPLACE, stream);
}

int sf_scatter_end(sf_t *sf, sf_unit unit, const void *multirootdata, void *leafdata, sf_stream_t stream) {
  if (!sf) return SF_ERR_NULL;
  if (!sf->multi) return SF_ERR_NO_PENDING;
  return sf_bcast_end(sf->multi, unit, multirootdata, leafdata, SF_REPLACE, stream);
}

}  // extern "C"
