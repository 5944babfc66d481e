// sf_launch_impl.cuh -- template bodies of the per-dtype launchers.
#pragma once
#include "sf_launch.h"

namespace sfgb {

template <typename T, int VB, int OP, int MODE>
static cudaError_t rm_go(const RmArgs &a, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  rm_kernel<T, VB, OP, MODE><<<ntiles, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int VB, int OP>
static cudaError_t rm_mode(int mode, const RmArgs &a, int ntiles, cudaStream_t s) {
  switch (mode) {
    case RM_REDUCE: return rm_go<T, VB, OP, RM_REDUCE>(a, ntiles, s);
    case RM_BCAST: return rm_go<T, VB, OP, RM_BCAST>(a, ntiles, s);
    case RM_FETCH: return rm_go<T, VB, OP, RM_FETCH>(a, ntiles, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int VB>
static cudaError_t rm_op(int op, int mode, const RmArgs &a, int ntiles, cudaStream_t s) {
  switch (op) {
    case OP_REPLACE: return rm_mode<T, VB, OP_REPLACE>(mode, a, ntiles, s);
    case OP_SUM: return rm_mode<T, VB, OP_SUM>(mode, a, ntiles, s);
    case OP_MIN: return rm_mode<T, VB, OP_MIN>(mode, a, ntiles, s);
    case OP_MAX: return rm_mode<T, VB, OP_MAX>(mode, a, ntiles, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_rm_t(int op, int vb, int mode, const RmArgs &a, int ntiles, cudaStream_t s) {
  if (vb == int(sizeof(T))) return rm_op<T, int(sizeof(T))>(op, mode, a, ntiles, s);
  if (vb == 16) return rm_op<T, 16>(op, mode, a, ntiles, s);
  return cudaErrorInvalidValue;
}

template <typename T, int VB, int OP>
static cudaError_t ts_go(bool atomic, bool fetch, const TsArgs &a, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (!atomic) {
    ts_kernel<T, VB, OP, false, false, false><<<ntiles, kThreads, 0, s>>>(a);
  } else {
    if constexpr (VB == int(sizeof(T))) {
      if (fetch) ts_kernel<T, VB, OP, true, true, true><<<ntiles, kThreads, 0, s>>>(a);
      else ts_kernel<T, VB, OP, true, true, false><<<ntiles, kThreads, 0, s>>>(a);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

template <typename T, int VB>
static cudaError_t ts_op(int op, bool atomic, bool fetch, const TsArgs &a, int ntiles, cudaStream_t s) {
  switch (op) {
    case OP_REPLACE:
      if (!atomic) return cudaErrorInvalidValue;   // plain REPLACE uses the raw copy kernels
      if constexpr (VB == int(sizeof(T))) {
        if (ntiles <= 0) return cudaSuccess;
        if (fetch) ts_kernel<T, VB, OP_REPLACE, true, true, true><<<ntiles, kThreads, 0, s>>>(a);
        else ts_kernel<T, VB, OP_REPLACE, true, true, false><<<ntiles, kThreads, 0, s>>>(a);
        return cudaGetLastError();
      }
      return cudaErrorInvalidValue;
    case OP_SUM: return ts_go<T, VB, OP_SUM>(atomic, fetch, a, ntiles, s);
    case OP_MIN: return ts_go<T, VB, OP_MIN>(atomic, fetch, a, ntiles, s);
    case OP_MAX: return ts_go<T, VB, OP_MAX>(atomic, fetch, a, ntiles, s);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_ts_ops_t(int op, int vb, bool atomic, bool fetch, const TsArgs &a, int ntiles, cudaStream_t s) {
  if (vb == int(sizeof(T))) return ts_op<T, int(sizeof(T))>(op, atomic, fetch, a, ntiles, s);
  if (vb == 16 && !atomic) return ts_op<T, 16>(op, atomic, fetch, a, ntiles, s);
  return cudaErrorInvalidValue;
}

#define SFGB_INSTANTIATE(T)                                                                          \
  template cudaError_t launch_rm_t<T>(int, int, int, const RmArgs &, int, cudaStream_t);             \
  template cudaError_t launch_ts_ops_t<T>(int, int, bool, bool, const TsArgs &, int, cudaStream_t);

}  // namespace sfgb
