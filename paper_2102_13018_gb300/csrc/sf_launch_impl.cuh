// sf_launch_impl.cuh -- template bodies of the per-dtype launchers.
#pragma once
#include "sf_launch.h"

namespace sfgb {

template <typename T, int VB, int OP, bool L2R, bool ATOMIC, bool FETCH>
cudaError_t go_ts(const TsLaunch &L) {
  if (L.ntiles <= 0) return cudaSuccess;
  if (L.tiles) ts_batch_kernel<T, VB, OP, L2R, ATOMIC, FETCH><<<L.ntiles, kThreads, 0, L.s>>>(L.ops, L.tiles);
  else ts_kernel<T, VB, OP, L2R, ATOMIC, FETCH><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
  return cudaGetLastError();
}

template <typename T, int VB, int OP, int MODE>
cudaError_t go_rm(const RmLaunch &L) {
  if (L.ntiles <= 0) return cudaSuccess;
  // A single forest's Reduce from zero runs the ZR instantiation; REPLACE reads no root, and
  // the batch tables never start roots at zero.
  constexpr bool kZr = MODE == RM_REDUCE && OP != OP_REPLACE;
  const bool zr = kZr && !L.tiles && L.single->zero_root;
  if (L.nv1) {   // the one-vector-unit kernel; the caller passed tiles of rm_fold_nv1_tiles
    if constexpr (MODE == RM_REDUCE && OP != OP_REPLACE && VB >= 4) {
      if (L.tiles) {
        rm_batch_kernel<T, VB, OP, MODE, true><<<L.ntiles, kThreads, 0, L.s>>>(L.ops, L.tiles);
      } else {
        if (L.single->nv != 1) return cudaErrorInvalidValue;
        if (zr) rm_kernel<T, VB, OP, MODE, true, true><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
        else rm_kernel<T, VB, OP, MODE, true><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
      }
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (L.flat) {   // multi-vector units, gather-then-fold, on rm_fold_nv1_tiles
    if constexpr (MODE == RM_REDUCE && OP != OP_REPLACE && VB >= 4) {
      if (L.tiles) {   // the batch builder checked every operation's unit (reduce_flat)
        rm_batch_kernel<T, VB, OP, MODE, false, true><<<L.ntiles, kThreads, 0, L.s>>>(L.ops, L.tiles);
        return cudaGetLastError();
      }
      if (L.single->nv < 2 || L.single->nv > RM_FLAT_MAX_NV || L.single->nv * VB > RM_FLAT_BYTES)
        return cudaErrorInvalidValue;
      if (zr) rm_kernel<T, VB, OP, MODE, false, true, true><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
      else rm_kernel<T, VB, OP, MODE, false, false, true><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (L.tiles) {
    rm_batch_kernel<T, VB, OP, MODE><<<L.ntiles, kThreads, 0, L.s>>>(L.ops, L.tiles);
    return cudaGetLastError();
  }
  if constexpr (kZr) {
    if (zr) {
      rm_kernel<T, VB, OP, MODE, false, true><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
      return cudaGetLastError();
    }
  }
  rm_kernel<T, VB, OP, MODE><<<L.ntiles, kThreads, 0, L.s>>>(*L.single);
  return cudaGetLastError();
}

template <typename T, int VB, int OP>
static cudaError_t rm_mode(int mode, const RmLaunch &L) {
  switch (mode) {
    case RM_REDUCE: return go_rm<T, VB, OP, RM_REDUCE>(L);
    case RM_BCAST: return go_rm<T, VB, OP, RM_BCAST>(L);
    case RM_FETCH: return go_rm<T, VB, OP, RM_FETCH>(L);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int VB>
static cudaError_t rm_op(int op, int mode, const RmLaunch &L) {
  switch (op) {
    case OP_REPLACE: return rm_mode<T, VB, OP_REPLACE>(mode, L);
    case OP_SUM: return rm_mode<T, VB, OP_SUM>(mode, L);
    case OP_MIN: return rm_mode<T, VB, OP_MIN>(mode, L);
    case OP_MAX: return rm_mode<T, VB, OP_MAX>(mode, L);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_rm_t(int op, int vb, int mode, const RmLaunch &L) {
  if (vb == int(sizeof(T))) return rm_op<T, int(sizeof(T))>(op, mode, L);
  if (vb == 16) return rm_op<T, 16>(op, mode, L);
  return cudaErrorInvalidValue;
}

template <typename T, int VB, int OP>
static cudaError_t ts_go(bool atomic, bool fetch, const TsLaunch &L) {
  if (!atomic) return go_ts<T, VB, OP, false, false, false>(L);
  if constexpr (VB == int(sizeof(T))) {
    if (fetch) return go_ts<T, VB, OP, true, true, true>(L);
    return go_ts<T, VB, OP, true, true, false>(L);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int VB>
static cudaError_t ts_op(int op, bool atomic, bool fetch, const TsLaunch &L) {
  switch (op) {
    case OP_REPLACE:
      if (!atomic) return cudaErrorInvalidValue;   // plain REPLACE uses the raw copy kernels
      if constexpr (VB == int(sizeof(T))) {
        if (fetch) return go_ts<T, VB, OP_REPLACE, true, true, true>(L);
        return go_ts<T, VB, OP_REPLACE, true, true, false>(L);
      }
      return cudaErrorInvalidValue;
    case OP_SUM: return ts_go<T, VB, OP_SUM>(atomic, fetch, L);
    case OP_MIN: return ts_go<T, VB, OP_MIN>(atomic, fetch, L);
    case OP_MAX: return ts_go<T, VB, OP_MAX>(atomic, fetch, L);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_ts_ops_t(int op, int vb, bool atomic, bool fetch, const TsLaunch &L) {
  if (vb == int(sizeof(T))) return ts_op<T, int(sizeof(T))>(op, atomic, fetch, L);
  if (vb == 16 && !atomic) return ts_op<T, 16>(op, atomic, fetch, L);
  return cudaErrorInvalidValue;
}

template <typename T, int VB, int OP>
cudaError_t go_dg(const DgLaunch &L) {
  if (L.ntiles <= 0) return cudaSuccess;
  if (L.tiles) dg_batch_kernel<T, VB, OP><<<L.ntiles, kThreads, 0, L.s>>>(L.ops, L.tiles);
  else dg_kernel<T, VB, OP><<<L.grid, kThreads, 0, L.s>>>(*L.single);
  return cudaGetLastError();
}

// The staged kernel: a persistent grid of as many CTAs as fit the GPU (DG_STAGES stages of
// DgStage<VB> in dynamic shared memory each).  cudaErrorNotSupported when it cannot be set up.
template <typename T, int VB, int OP>
cudaError_t go_dg_bulk(const DgBulkArgs &b, cudaStream_t s) {
  if (b.ntiles <= 0) return cudaSuccess;
  constexpr int smem = DgStage<VB>::NSTAGE * DgStage<VB>::BYTES;
  static const int per_sm = [] {
    int n = 0;
    if (cudaFuncSetAttribute(dg_bulk_kernel<T, VB, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dg_bulk_kernel<T, VB, OP>, DG_BULK_THREADS, smem) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  }();
  int dev = 0, sms = 0;
  if (per_sm <= 0 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorNotSupported;
  }
  const int grid = b.ntiles < per_sm * sms ? b.ntiles : per_sm * sms;
  dg_bulk_kernel<T, VB, OP><<<grid, DG_BULK_THREADS, smem, s>>>(b);
  return cudaGetLastError();
}

template <typename T, int VB>
static cudaError_t dg_bulk_op(int op, const DgBulkArgs &b, cudaStream_t s) {
  switch (op) {
    case OP_SUM: return go_dg_bulk<T, VB, OP_SUM>(b, s);
    case OP_MIN: return go_dg_bulk<T, VB, OP_MIN>(b, s);
    case OP_MAX: return go_dg_bulk<T, VB, OP_MAX>(b, s);
  }
  return cudaErrorInvalidValue;
}

// 4-, 8- and 16-byte units (its list gathers are cp.async copies); others: cudaErrorNotSupported
template <typename T>
cudaError_t launch_dg_bulk_t(int op, int vb, const DgBulkArgs &b, cudaStream_t s) {
  if constexpr (sizeof(T) >= 4)
    if (vb == int(sizeof(T))) return dg_bulk_op<T, int(sizeof(T))>(op, b, s);
  if (vb == 16) return dg_bulk_op<T, 16>(op, b, s);
  return cudaErrorNotSupported;
}

template <typename T, int VB>
static cudaError_t dg_op(int op, const DgLaunch &L) {
  switch (op) {
    case OP_SUM: return go_dg<T, VB, OP_SUM>(L);
    case OP_MIN: return go_dg<T, VB, OP_MIN>(L);
    case OP_MAX: return go_dg<T, VB, OP_MAX>(L);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_dg_t(int op, int vb, const DgLaunch &L) {
  if (vb == int(sizeof(T))) return dg_op<T, int(sizeof(T))>(op, L);
  if (vb == 16) return dg_op<T, 16>(op, L);
  return cudaErrorInvalidValue;
}

// vb == 0: the general kernel (any unit, a.tiles = rm_fold_tiles); vb = 4, 8 or 16 (at least the
// element size): the gather-then-fold kernel on f.nv vectors of vb bytes (a.tiles =
// rm_fold_nv1_tiles).
template <typename T>
cudaError_t launch_maxloc_t(const MaxlocArgs &a, int ntiles, int vb, const MaxlocFlat &f, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (vb == 0) {
    maxloc_kernel<T><<<ntiles, kThreads, 0, s>>>(a);
  } else if (vb == 16) {
    maxloc_flat_kernel<T, 16><<<ntiles, kThreads, 0, s>>>(a, f);
  } else if constexpr (sizeof(T) >= 4) {
    if (vb != int(sizeof(T))) return cudaErrorInvalidValue;
    maxloc_flat_kernel<T, int(sizeof(T))><<<ntiles, kThreads, 0, s>>>(a, f);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_maxloc_grad_t(const MaxlocArgs &a, int ntiles, int vb, int32_t nv, const void *grad_root,
                                 void *grad_leaf, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  const DivMagic dm = div_magic(uint32_t(nv));
  if (vb == 16)
    maxloc_grad_kernel<T, 16><<<ntiles, kThreads, 0, s>>>(a, nv, dm.m, dm.s, grad_root, grad_leaf);
  else if (vb == int(sizeof(T)))
    maxloc_grad_kernel<T, int(sizeof(T))><<<ntiles, kThreads, 0, s>>>(a, nv, dm.m, dm.s, grad_root, grad_leaf);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_maxloc_scatter_t(const int32_t *arg, const void *grad_root, void *grad_leaf, int64_t n, int32_t bs,
                                    cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + kThreads - 1) / kThreads;
  const int grid = int(blocks < 152 * 16 ? blocks : 152 * 16);
  maxloc_scatter_kernel<T><<<grid, kThreads, 0, s>>>(arg, static_cast<const T *>(grad_root),
                                                     static_cast<T *>(grad_leaf), n, bs);
  return cudaGetLastError();
}

#define SFGB_INSTANTIATE(T)                                                                            \
  template cudaError_t launch_rm_t<T>(int, int, int, const RmLaunch &);                                \
  template cudaError_t launch_ts_ops_t<T>(int, int, bool, bool, const TsLaunch &);                     \
  template cudaError_t launch_dg_t<T>(int, int, const DgLaunch &);                                     \
  template cudaError_t launch_dg_bulk_t<T>(int, int, const DgBulkArgs &, cudaStream_t);                \
  template cudaError_t launch_maxloc_t<T>(const MaxlocArgs &, int, int, const MaxlocFlat &, cudaStream_t);  \
  template cudaError_t launch_maxloc_grad_t<T>(const MaxlocArgs &, int, int, int32_t, const void *, void *,    \
                                               cudaStream_t);                                                 \
  template cudaError_t launch_maxloc_scatter_t<T>(const int32_t *, const void *, void *, int64_t, int32_t, \
                                                  cudaStream_t);

}  // namespace sfgb
