// sf_launch.h -- host-side launchers of the kernels (runtime dtype/op/width -> template).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sf_kernels.cuh"

namespace sfgb {

// A launch of one kernel variant: either one forest (`single`, passed by value) or a batch
// (`ops` and `tiles` are device tables, one CTA per (operation, tile) pair).
struct TsLaunch {
  const TsArgs *single;
  const TsArgs *ops;
  const BatchTile *tiles;
  int ntiles;
  cudaStream_t s;
};
struct RmLaunch {
  const RmArgs *single;
  const RmArgs *ops;
  const BatchTile *tiles;
  int ntiles;
  cudaStream_t s;
  bool nv1 = false;   // the one-vector-unit Reduce kernel (reduce_nv1); its tiles come from rm_fold_nv1_tiles
  bool flat = false;  // the gather-then-fold Reduce kernel of multi-vector units (reduce_flat); same tiles
};

// The diagonal-chunk Reduce: one forest (`single`, with `grid` CTAs looping over its tiles) or
// a batch (one CTA per (operation, tile) pair of `tiles`, the tile index in BatchTile::pad).
struct DgLaunch {
  const DgArgs *single;
  const DgArgs *ops;
  const BatchTile *tiles;
  int ntiles;
  int grid;
  cudaStream_t s;
};

// dtype codes are the SF_* codes of sf.h
// Two-sided kernel: REPLACE copies (any dtype, vector width vb in {2,4,8,16}), plain ops for
// Bcast (l2r = false), atomics for Reduce / FetchAndOp (l2r = true, vb = element size).
cudaError_t launch_ts(int dtype, int op, int vb, bool l2r, bool atomic, bool fetch, const TsLaunch &L);
cudaError_t launch_rm(int dtype, int op, int vb, int mode, const RmLaunch &L);
cudaError_t launch_move(int vb, const MoveArgs &a, int ntiles, cudaStream_t s);
// Zero n listed units of nv vectors of vb bytes (and their bs entries of arg, if given, to -1).
cudaError_t launch_zero(int vb, const int32_t *units, int32_t n, void *data, int32_t nv, int32_t *arg, int32_t bs,
                        cudaStream_t s);
// Deterministic Reduce over diagonal chunks: op SUM/MIN/MAX, one vector of vb bytes per unit.
cudaError_t launch_dg(int dtype, int op, int vb, const DgLaunch &L);
// The same, staged by bulk copies (one forest; root and leaf bases 16-byte aligned).
// cudaErrorNotSupported when the kernel cannot be configured (the caller uses launch_dg).
cudaError_t launch_dg_bulk(int dtype, int op, int vb, const DgBulkArgs &b, cudaStream_t s);

inline cudaError_t launch_ts(int dtype, int op, int vb, bool l2r, bool atomic, bool fetch, const TsArgs &a,
                             int ntiles, cudaStream_t s) {
  return launch_ts(dtype, op, vb, l2r, atomic, fetch, TsLaunch{&a, nullptr, nullptr, ntiles, s});
}
inline cudaError_t launch_rm(int dtype, int op, int vb, int mode, const RmArgs &a, int ntiles, cudaStream_t s) {
  return launch_rm(dtype, op, vb, mode, RmLaunch{&a, nullptr, nullptr, ntiles, s});
}

// per-dtype instantiations (one translation unit each)
template <typename T> cudaError_t launch_rm_t(int op, int vb, int mode, const RmLaunch &L);
template <typename T> cudaError_t launch_ts_ops_t(int op, int vb, bool atomic, bool fetch, const TsLaunch &L);
template <typename T> cudaError_t launch_dg_t(int op, int vb, const DgLaunch &L);
template <typename T> cudaError_t launch_dg_bulk_t(int op, int vb, const DgBulkArgs &b, cudaStream_t s);

// MAX with location and its gradient scatter (per dtype)
cudaError_t launch_maxloc(int dtype, const MaxlocArgs &a, int ntiles, int vb, const MaxlocFlat &f, cudaStream_t s);
cudaError_t launch_maxloc_scatter(int dtype, const int32_t *arg, const void *grad_root, void *grad_leaf, int64_t n,
                                  int32_t bs, cudaStream_t s);
template <typename T>
cudaError_t launch_maxloc_t(const MaxlocArgs &a, int ntiles, int vb, const MaxlocFlat &f, cudaStream_t s);
cudaError_t launch_maxloc_grad(int dtype, const MaxlocArgs &a, int ntiles, int vb, int32_t nv, const void *grad_root,
                               void *grad_leaf, cudaStream_t s);
template <typename T>
cudaError_t launch_maxloc_grad_t(const MaxlocArgs &a, int ntiles, int vb, int32_t nv, const void *grad_root,
                                 void *grad_leaf, cudaStream_t s);
template <typename T>
cudaError_t launch_maxloc_scatter_t(const int32_t *arg, const void *grad_root, void *grad_leaf, int64_t n, int32_t bs,
                                    cudaStream_t s);

// accumulator pack bytes of the fold for (dtype, op, vb): scratch sizing
int acc_pack_bytes(int dtype, int op, int vb);

}  // namespace sfgb
