// sf_launch.cu -- runtime dispatch to the kernel instantiations; raw-copy (REPLACE) kernels.
#include <algorithm>

#include "sf.h"
#include "sf_launch_impl.cuh"

namespace sfgb {

namespace {
template <int VB, bool L2R>
cudaError_t ts_copy(const TsLaunch &L) {
  using T = typename std::conditional<VB == 2, unsigned short, unsigned int>::type;
  return go_ts<T, VB, OP_REPLACE, L2R, false, false>(L);
}
template <int VB>
cudaError_t rm_copy(int mode, const RmLaunch &L) {
  using T = typename std::conditional<VB == 2, unsigned short, unsigned int>::type;
  switch (mode) {
    case RM_REDUCE: return go_rm<T, VB, OP_REPLACE, RM_REDUCE>(L);
    case RM_BCAST: return go_rm<T, VB, OP_REPLACE, RM_BCAST>(L);
    case RM_FETCH: return go_rm<T, VB, OP_REPLACE, RM_FETCH>(L);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_ts(int dtype, int op, int vb, bool l2r, bool atomic, bool fetch, const TsLaunch &L) {
  if (op == OP_REPLACE && !atomic) {   // a copy: independent of the dtype
    switch (vb) {
      case 2: return l2r ? ts_copy<2, true>(L) : ts_copy<2, false>(L);
      case 4: return l2r ? ts_copy<4, true>(L) : ts_copy<4, false>(L);
      case 8: return l2r ? ts_copy<8, true>(L) : ts_copy<8, false>(L);
      case 16: return l2r ? ts_copy<16, true>(L) : ts_copy<16, false>(L);
    }
    return cudaErrorInvalidValue;
  }
  if (!atomic && l2r) return cudaErrorInvalidValue;   // leaf->root with an op needs atomics
  switch (dtype) {
    case SF_INT32: return launch_ts_ops_t<int32_t>(op, vb, atomic, fetch, L);
    case SF_INT64: return launch_ts_ops_t<int64_t>(op, vb, atomic, fetch, L);
    case SF_FP32: return launch_ts_ops_t<float>(op, vb, atomic, fetch, L);
    case SF_FP64: return launch_ts_ops_t<double>(op, vb, atomic, fetch, L);
    case SF_BF16: return launch_ts_ops_t<bf16>(op, vb, atomic, fetch, L);
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

cudaError_t launch_rm(int dtype, int op, int vb, int mode, const RmLaunch &L) {
  if (op == OP_REPLACE) {
    switch (vb) {
      case 2: return rm_copy<2>(mode, L);
      case 4: return rm_copy<4>(mode, L);
      case 8: return rm_copy<8>(mode, L);
      case 16: return rm_copy<16>(mode, L);
    }
    return cudaErrorInvalidValue;
  }
  switch (dtype) {
    case SF_INT32: return launch_rm_t<int32_t>(op, vb, mode, L);
    case SF_INT64: return launch_rm_t<int64_t>(op, vb, mode, L);
    case SF_FP32: return launch_rm_t<float>(op, vb, mode, L);
    case SF_FP64: return launch_rm_t<double>(op, vb, mode, L);
    case SF_BF16: return launch_rm_t<bf16>(op, vb, mode, L);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_zero(int vb, const int32_t *units, int32_t n, void *data, int32_t nv, int32_t *arg, int32_t bs,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t work = int64_t(n) * (nv > bs ? nv : bs);
  const int grid = int(std::min<int64_t>((work + kThreads - 1) / kThreads, 152 * 16));
  switch (vb) {
    case 2: zero_units_kernel<2><<<grid, kThreads, 0, s>>>(units, n, data, nv, arg, bs); break;
    case 4: zero_units_kernel<4><<<grid, kThreads, 0, s>>>(units, n, data, nv, arg, bs); break;
    case 8: zero_units_kernel<8><<<grid, kThreads, 0, s>>>(units, n, data, nv, arg, bs); break;
    case 16: zero_units_kernel<16><<<grid, kThreads, 0, s>>>(units, n, data, nv, arg, bs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_dg(int dtype, int op, int vb, const DgLaunch &L) {
  switch (dtype) {
    case SF_INT32: return launch_dg_t<int32_t>(op, vb, L);
    case SF_INT64: return launch_dg_t<int64_t>(op, vb, L);
    case SF_FP32: return launch_dg_t<float>(op, vb, L);
    case SF_FP64: return launch_dg_t<double>(op, vb, L);
    case SF_BF16: return launch_dg_t<bf16>(op, vb, L);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dg_bulk(int dtype, int op, int vb, const DgBulkArgs &b, cudaStream_t s) {
  switch (dtype) {
    case SF_INT32: return launch_dg_bulk_t<int32_t>(op, vb, b, s);
    case SF_INT64: return launch_dg_bulk_t<int64_t>(op, vb, b, s);
    case SF_FP32: return launch_dg_bulk_t<float>(op, vb, b, s);
    case SF_FP64: return launch_dg_bulk_t<double>(op, vb, b, s);
    case SF_BF16: return launch_dg_bulk_t<bf16>(op, vb, b, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_maxloc(int dtype, const MaxlocArgs &a, int ntiles, int vb, const MaxlocFlat &f, cudaStream_t s) {
  switch (dtype) {
    case SF_INT32: return launch_maxloc_t<int32_t>(a, ntiles, vb, f, s);
    case SF_INT64: return launch_maxloc_t<int64_t>(a, ntiles, vb, f, s);
    case SF_FP32: return launch_maxloc_t<float>(a, ntiles, vb, f, s);
    case SF_FP64: return launch_maxloc_t<double>(a, ntiles, vb, f, s);
    case SF_BF16: return launch_maxloc_t<bf16>(a, ntiles, vb, f, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_maxloc_grad(int dtype, const MaxlocArgs &a, int ntiles, int vb, int32_t nv, const void *grad_root,
                               void *grad_leaf, cudaStream_t s) {
  switch (dtype) {
    case SF_INT32: return launch_maxloc_grad_t<int32_t>(a, ntiles, vb, nv, grad_root, grad_leaf, s);
    case SF_INT64: return launch_maxloc_grad_t<int64_t>(a, ntiles, vb, nv, grad_root, grad_leaf, s);
    case SF_FP32: return launch_maxloc_grad_t<float>(a, ntiles, vb, nv, grad_root, grad_leaf, s);
    case SF_FP64: return launch_maxloc_grad_t<double>(a, ntiles, vb, nv, grad_root, grad_leaf, s);
    case SF_BF16: return launch_maxloc_grad_t<bf16>(a, ntiles, vb, nv, grad_root, grad_leaf, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_maxloc_scatter(int dtype, const int32_t *arg, const void *grad_root, void *grad_leaf, int64_t n,
                                  int32_t bs, cudaStream_t s) {
  switch (dtype) {
    case SF_INT32: return launch_maxloc_scatter_t<int32_t>(arg, grad_root, grad_leaf, n, bs, s);
    case SF_INT64: return launch_maxloc_scatter_t<int64_t>(arg, grad_root, grad_leaf, n, bs, s);
    case SF_FP32: return launch_maxloc_scatter_t<float>(arg, grad_root, grad_leaf, n, bs, s);
    case SF_FP64: return launch_maxloc_scatter_t<double>(arg, grad_root, grad_leaf, n, bs, s);
    case SF_BF16: return launch_maxloc_scatter_t<bf16>(arg, grad_root, grad_leaf, n, bs, s);
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
