// sf_launch.cu -- runtime dispatch to the kernel instantiations; raw-copy (REPLACE) kernels.
#include "sf.h"
#include "sf_launch_impl.cuh"

namespace sfgb {

namespace {
template <int VB, bool L2R>
cudaError_t ts_copy(const TsArgs &a, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  using T = typename std::conditional<VB == 2, unsigned short, unsigned int>::type;
  ts_kernel<T, VB, OP_REPLACE, L2R, false, false><<<ntiles, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}
template <int VB>
cudaError_t rm_copy(int mode, const RmArgs &a, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  using T = typename std::conditional<VB == 2, unsigned short, unsigned int>::type;
  switch (mode) {
    case RM_REDUCE: rm_kernel<T, VB, OP_REPLACE, RM_REDUCE><<<ntiles, kThreads, 0, s>>>(a); break;
    case RM_BCAST: rm_kernel<T, VB, OP_REPLACE, RM_BCAST><<<ntiles, kThreads, 0, s>>>(a); break;
    case RM_FETCH: rm_kernel<T, VB, OP_REPLACE, RM_FETCH><<<ntiles, kThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_ts(int dtype, int op, int vb, bool l2r, bool atomic, bool fetch, const TsArgs &a, int ntiles,
                      cudaStream_t s) {
  if (op == OP_REPLACE && !atomic) {   // a copy: independent of the dtype
    switch (vb) {
      case 2: return l2r ? ts_copy<2, true>(a, ntiles, s) : ts_copy<2, false>(a, ntiles, s);
      case 4: return l2r ? ts_copy<4, true>(a, ntiles, s) : ts_copy<4, false>(a, ntiles, s);
      case 8: return l2r ? ts_copy<8, true>(a, ntiles, s) : ts_copy<8, false>(a, ntiles, s);
      case 16: return l2r ? ts_copy<16, true>(a, ntiles, s) : ts_copy<16, false>(a, ntiles, s);
    }
    return cudaErrorInvalidValue;
  }
  if (!atomic && l2r) return cudaErrorInvalidValue;   // leaf->root with an op needs atomics
  switch (dtype) {
    case SF_INT32: return launch_ts_ops_t<int32_t>(op, vb, atomic, fetch, a, ntiles, s);
    case SF_INT64: return launch_ts_ops_t<int64_t>(op, vb, atomic, fetch, a, ntiles, s);
    case SF_FP32: return launch_ts_ops_t<float>(op, vb, atomic, fetch, a, ntiles, s);
    case SF_FP64: return launch_ts_ops_t<double>(op, vb, atomic, fetch, a, ntiles, s);
    case SF_BF16: return launch_ts_ops_t<bf16>(op, vb, atomic, fetch, a, ntiles, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_move(int vb, const MoveArgs &a, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  switch (vb) {
    case 2: move_kernel<2><<<ntiles, kThreads, 0, s>>>(a); break;
    case 4: move_kernel<4><<<ntiles, kThreads, 0, s>>>(a); break;
    case 8: move_kernel<8><<<ntiles, kThreads, 0, s>>>(a); break;
    case 16: move_kernel<16><<<ntiles, kThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rm(int dtype, int op, int vb, int mode, const RmArgs &a, int ntiles, cudaStream_t s) {
  if (op == OP_REPLACE) {
    switch (vb) {
      case 2: return rm_copy<2>(mode, a, ntiles, s);
      case 4: return rm_copy<4>(mode, a, ntiles, s);
      case 8: return rm_copy<8>(mode, a, ntiles, s);
      case 16: return rm_copy<16>(mode, a, ntiles, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (dtype) {
    case SF_INT32: return launch_rm_t<int32_t>(op, vb, mode, a, ntiles, s);
    case SF_INT64: return launch_rm_t<int64_t>(op, vb, mode, a, ntiles, s);
    case SF_FP32: return launch_rm_t<float>(op, vb, mode, a, ntiles, s);
    case SF_FP64: return launch_rm_t<double>(op, vb, mode, a, ntiles, s);
    case SF_BF16: return launch_rm_t<bf16>(op, vb, mode, a, ntiles, s);
  }
  return cudaErrorInvalidValue;
}

int acc_pack_bytes(int dtype, int op, int vb) {
  const int w = (dtype == SF_INT32 || dtype == SF_FP32) ? 4 : (dtype == SF_BF16 ? 2 : 8);
  const int lanes = vb / w;
  const int aw = (dtype == SF_BF16 && op == OP_SUM) ? 4 : w;
  return lanes * aw;
}

}  // namespace sfgb
