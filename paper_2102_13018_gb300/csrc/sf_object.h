// sf_object.h -- the forest object behind sf_t and helpers shared by the ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "sf.h"
#include "sf_host.h"
#include "sf_launch.h"

namespace sfgb {

enum { K_BCAST = 1, K_REDUCE = 2, K_FETCH = 3, K_BCAST_MT = 4, K_REDUCE_MT = 5, K_REDUCE_Z = 6 };

struct Pending {
  int kind;
  sf_unit unit;
  const void *p0, *p1, *p2;
  int32_t op;
  int32_t m0, m1;      // memtypes (memtype calls)
  int32_t finish;      // work left for End: 0 none, 1 three-phase unpack
};

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};

inline int elem_size(int dtype) {
  switch (dtype) {
    case SF_INT32: case SF_FP32: return 4;
    case SF_INT64: case SF_FP64: return 8;
    case SF_BF16: return 2;
  }
  return 0;
}

}  // namespace sfgb

struct sf_s {
  sfgb::Graph g;
  sfgb::HostPlan hp;
  sf_info info{};
  bool setup = false;
  int device = -1;
  sfgb::DevBuf blob;                 // all plan arrays
  sfgb::DevPlan dp{};
  sfgb::DevPlan dp_rest{};           // root-major plan of the roots the diagonal chunks leave out
  bool has_rest = false;
  std::vector<sfgb::Tile> h_move_tiles;
  const sfgb::Tile *move_tiles = nullptr;
  int32_t n_move_tiles = 0;
  sfgb::DevBuf partial, counter;     // fold scratch
  sfgb::DevBuf partial_arg;          // MAX-with-location scratch (leaf units of block maxima)
  sfgb::DevBuf rootbuf, leafbuf;     // three-phase buffers
  sfgb::DevBuf stage_root, stage_leaf;   // memtype staging
  sfgb::DevBuf status;               // device status word (DEVSTAT_* bits), zero when all is well
  int32_t mode = SF_MODE_AUTO, path = SF_PATH_AUTO;
  int32_t tuned_mode = SF_MODE_DETERMINISTIC;   // what AUTO means (sf_autotune may change it)
  int32_t tuned_path = SF_PATH_FUSED;
  bool path_tuned = false;           // sf_autotune chose tuned_path (else AUTO follows bcast_path's rule)
  int32_t plan = SF_PLAN_AUTO;       // deterministic Reduce plan (SF_PLAN_*)
  int32_t tuned_plan = SF_PLAN_ROOT_MAJOR;   // what SF_PLAN_AUTO means (sf_autotune may change it)
  int32_t vec_bytes = 0;             // widest vector of the Bcast / Reduce kernels (0: 16 bytes)
  int32_t tile_edges = 0;            // edges per two-sided tile (0: the setup pass's choice)
  sfgb::DevBuf ts_tuned;             // the two-sided tile list cut at tile_edges
  const sfgb::TsTile *ts_default = nullptr;
  int32_t n_ts_default = 0;
  std::vector<sfgb::Pending> pending;
  sf_t *multi = nullptr;             // multi-forest, built on first use (Gather / Scatter)
};

namespace sfgb {

std::atomic<int64_t> &launch_counter();
int cuda_err(cudaError_t e);
int ensure(DevBuf &b, size_t bytes, bool zero, cudaStream_t s);
void release(DevBuf &b);
int pick_vb(int w, int ub, bool allow_wide, std::initializer_list<const void *> ptrs, int cap = 16);
// pick_vb under the forest's vector-width setting (sf_set_vector_bytes)
inline int pick_vb_sf(const sf_t *sf, int w, int ub, bool allow_wide, std::initializer_list<const void *> ptrs) {
  return pick_vb(w, ub, allow_wide, ptrs, sf->vec_bytes > 0 ? sf->vec_bytes : 16);
}
int check_unit(const sf_unit &u, int32_t op);
int check_ptr(const void *p, int w);
int launched(cudaError_t e);
TsArgs ts_args(const sf_t *sf, const TsTile *tiles, int32_t ntiles, const void *src, void *dst, void *upd, int nv,
               int phase);
RmArgs rm_args(sf_t *sf, const RmTile *tiles, int32_t ntiles, void *root, void *leaf, void *upd, int nv);
RmArgs rm_args_plan(sf_t *sf, const DevPlan &d, const RmTile *tiles, int32_t ntiles, void *root, void *leaf, void *upd,
                    int nv);
// SF_PLAN_ROOT_MAJOR, SF_PLAN_DIAGONAL or SF_PLAN_DIAGONAL_STAGED after resolving AUTO; a forest
// without diagonal chunks always answers SF_PLAN_ROOT_MAJOR.
inline int32_t reduce_plan(const sf_t *sf) {
  if (sf->dp.dg_nchunks == 0) return SF_PLAN_ROOT_MAJOR;
  return sf->plan == SF_PLAN_AUTO ? sf->tuned_plan : sf->plan;
}
// Whether a deterministic Reduce with `op` and nv vectors per unit runs on the diagonal chunks
// (then on the root-major plan of the rest).
inline bool reduce_dg(const sf_t *sf, int32_t op, int nv) {
  return op != SF_REPLACE && nv == 1 && reduce_plan(sf) != SF_PLAN_ROOT_MAJOR;
}
DgArgs dg_args(const sf_t *sf, const void *leaf, void *root);
// Enqueue the deterministic (root-major or diagonal-chunk) Reduce with its fold scratch.
// With zero_root the roots count as 0 before the operation and are not read.
int reduce_det_launch(sf_t *sf, const sf_unit &u, const void *leaf, void *root, int32_t op, cudaStream_t s, int vbo,
                      int nv, void *partial, int32_t *counter, bool zero_root = false);
int reduce_mode(const sf_t *sf);   // SF_MODE_ATOMIC or SF_MODE_DETERMINISTIC after resolving AUTO
// Whether Reduce with `op` on `dtype` runs on the atomic two-sided kernels: in atomic mode
// (floating SUM rounds in arrival order there), and in deterministic mode for operations whose
// result does not depend on the order (integer SUM/MIN/MAX) while no root has more than
// kOrderFreeMaxDegree leaves (same-address atomics serialise) and the Reduce does not run on
// the diagonal chunks.
constexpr int64_t kOrderFreeMaxDegree = 1024;
bool reduce_atomic(const sf_t *sf, int32_t dtype, int32_t op);
// SF_PATH_* after resolving AUTO for units of unit_bytes: the tuned path, else ROOT_MAJOR for
// units of kRootMajorUnitBytes or more on forests whose connected roots average
// kRootMajorMeanDegree leaves or more (each root unit read once, whole-sector leaf writes), else
// FUSED.  Measured on the 2^20-root power-law forest (8.8 leaves per root), bs = 64 fp32: 0.39 ms
// root-major against 0.54 ms fused.
constexpr int64_t kRootMajorUnitBytes = 64;
constexpr int64_t kRootMajorMeanDegree = 4;
int bcast_path(const sf_t *sf, int64_t unit_bytes);
// Whether a root-major Reduce with `op`, vector width vbo and nv vectors per unit runs the
// one-vector-unit kernel (NV1), which reads the rm_fold_nv1_tiles list; every caller takes the
// tile list and the launch flag from this one test.
inline bool reduce_nv1(int32_t op, int vbo, int nv) { return op != SF_REPLACE && nv == 1 && vbo >= 4; }
// Whether a root-major Reduce of multi-vector units runs the gather-then-fold kernel (FLAT),
// which reads rm_fold_nv1_tiles as NV1 does: SUM/MIN/MAX, vectors of 4 bytes or more, at most
// RM_FLAT_MAX_NV vectors and RM_FLAT_BYTES per unit.
inline bool reduce_flat(int32_t op, int vbo, int nv) {
  return op != SF_REPLACE && vbo >= 4 && nv >= 2 && nv <= RM_FLAT_MAX_NV && nv * vbo <= RM_FLAT_BYTES;
}
// Enqueue a whole operation (begin and end) on `s`; used by sf_autotune.
int bcast_all(sf_t *sf, const sf_unit &u, const void *root, void *leaf, int32_t op, cudaStream_t s, int path);
int reduce_all(sf_t *sf, const sf_unit &u, const void *leaf, void *root, int32_t op, cudaStream_t s, int mode);

}  // namespace sfgb
