// sf_kernels.cuh -- sm_103a kernels of the star-forest data path.
//
// Everything here is HBM- or L2-bound index-driven data movement (Sec. V.B-C): no
// contraction, so no tensor cores.  The design rules are coalesced 16-byte accesses where the
// unit allows it, index-free addressing on detected patterns, several independent loads in
// flight per thread, and one CTA per fixed-size tile of a plan so that grids are many waves
// of the 152 SMs.
//
// Kernels:
//  ts_kernel   -- edges of the two-sided plan: fused scatter (Bcast, and atomic Reduce /
//                 FetchAndOp), or the pack / unpack halves of the three-phase form.
//  move_kernel -- the buffer move of the three-phase form (per (root rank, leaf rank) chunk).
//  rm_kernel   -- the root-major plan: masked single-leaf runs, explicit pairs, blocks of
//                 multi-leaf roots (deterministic fold with a last-arriver combine), last-leaf
//                 winners (Reduce REPLACE) and serial per-root FetchAndOp.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sf_plan.h"

namespace sfgb {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

enum : int { OP_REPLACE = 0, OP_SUM = 1, OP_MIN = 2, OP_MAX = 3 };
enum : int { PH_FUSED = 0, PH_PACK = 1, PH_UNPACK = 2 };
enum : int { RM_REDUCE = 0, RM_BCAST = 1, RM_FETCH = 2 };

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ raw vectors
template <int VB> struct Raw;
template <> struct Raw<2> { using type = unsigned short; };
template <> struct Raw<4> { using type = unsigned int; };
template <> struct Raw<8> { using type = uint2; };
template <> struct Raw<16> { using type = uint4; };

// L lanes of T packed in VB bytes
template <typename T, int VB> struct Pack {
  static constexpr int L = VB / int(sizeof(T));
  T v[L];
};

template <typename T, int VB>
__device__ __forceinline__ Pack<T, VB> ld(const void *base, int64_t vec_index) {
  using R = typename Raw<VB>::type;
  R r = reinterpret_cast<const R *>(base)[vec_index];
  Pack<T, VB> p;
  memcpy(&p, &r, VB);
  return p;
}
template <typename T, int VB>
__device__ __forceinline__ void st(void *base, int64_t vec_index, const Pack<T, VB> &p) {
  using R = typename Raw<VB>::type;
  R r;
  memcpy(&r, &p, VB);
  reinterpret_cast<R *>(base)[vec_index] = r;
}
// L2-coherent variants for the scratch partials
template <typename T, int VB>
__device__ __forceinline__ Pack<T, VB> ld_cg(const void *base, int64_t i) {
  Pack<T, VB> p;
  const T *src = reinterpret_cast<const T *>(base) + i * Pack<T, VB>::L;
#pragma unroll
  for (int l = 0; l < Pack<T, VB>::L; ++l) p.v[l] = __ldcg(src + l);
  return p;
}
template <typename T, int VB>
__device__ __forceinline__ void st_cg(void *base, int64_t i, const Pack<T, VB> &p) {
  T *dst = reinterpret_cast<T *>(base) + i * Pack<T, VB>::L;
#pragma unroll
  for (int l = 0; l < Pack<T, VB>::L; ++l) __stcg(dst + l, p.v[l]);
}

// ------------------------------------------------------------------ element arithmetic
// combine<OP>(a, b): REPLACE b, SUM a+b (integers wrap), MIN (b<a?b:a), MAX (a<b?b:a)
template <int OP, typename T> __device__ __forceinline__ T combine(T a, T b) {
  if constexpr (OP == OP_REPLACE) return b;
  else if constexpr (OP == OP_SUM) return a + b;
  else if constexpr (OP == OP_MIN) return b < a ? b : a;
  else return a < b ? b : a;
}
template <> __device__ __forceinline__ int32_t combine<OP_SUM, int32_t>(int32_t a, int32_t b) {
  return int32_t(uint32_t(a) + uint32_t(b));
}
template <> __device__ __forceinline__ int64_t combine<OP_SUM, int64_t>(int64_t a, int64_t b) {
  return int64_t(uint64_t(a) + uint64_t(b));
}
template <int OP> __device__ __forceinline__ bf16 combine_bf16(bf16 a, bf16 b) {
  if constexpr (OP == OP_REPLACE) return b;
  float fa = __bfloat162float(a), fb = __bfloat162float(b);
  if constexpr (OP == OP_SUM) return __float2bfloat16_rn(fa + fb);
  else if constexpr (OP == OP_MIN) return fb < fa ? b : a;
  else return fa < fb ? b : a;
}
template <> __device__ __forceinline__ bf16 combine<OP_REPLACE, bf16>(bf16 a, bf16 b) { return b; }
template <> __device__ __forceinline__ bf16 combine<OP_SUM, bf16>(bf16 a, bf16 b) { return combine_bf16<OP_SUM>(a, b); }
template <> __device__ __forceinline__ bf16 combine<OP_MIN, bf16>(bf16 a, bf16 b) { return combine_bf16<OP_MIN>(a, b); }
template <> __device__ __forceinline__ bf16 combine<OP_MAX, bf16>(bf16 a, bf16 b) { return combine_bf16<OP_MAX>(a, b); }

template <int OP, typename T, int VB>
__device__ __forceinline__ Pack<T, VB> combine(const Pack<T, VB> &a, const Pack<T, VB> &b) {
  Pack<T, VB> r;
#pragma unroll
  for (int l = 0; l < Pack<T, VB>::L; ++l) r.v[l] = combine<OP, T>(a.v[l], b.v[l]);
  return r;
}

// Fold accumulator: SUM of fp32/bf16 accumulates in fp32, everything else in its own type.
template <typename T, int OP> struct Acc { using type = T; };
template <> struct Acc<bf16, OP_SUM> { using type = float; };

template <typename A, typename T> __device__ __forceinline__ A to_acc(T x) { return A(x); }
template <> __device__ __forceinline__ float to_acc<float, bf16>(bf16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ bf16 to_acc<bf16, bf16>(bf16 x) { return x; }

// root op= S where S is a folded accumulator
template <int OP, typename T, typename A> __device__ __forceinline__ T apply_acc(T root, A s) {
  return combine<OP, T>(root, T(s));
}
template <> __device__ __forceinline__ bf16 apply_acc<OP_SUM, bf16, float>(bf16 root, float s) {
  return __float2bfloat16_rn(__bfloat162float(root) + s);
}

// ------------------------------------------------------------------ atomics (element-wise)
template <int OP> __device__ __forceinline__ int32_t atomic_apply(int32_t *p, int32_t v) {
  if constexpr (OP == OP_SUM) return atomicAdd(p, v);
  else if constexpr (OP == OP_MIN) return atomicMin(p, v);
  else if constexpr (OP == OP_MAX) return atomicMax(p, v);
  else return atomicExch(p, v);
}
template <int OP> __device__ __forceinline__ int64_t atomic_apply(int64_t *p, int64_t v) {
  if constexpr (OP == OP_SUM)
    return int64_t(atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v));
  else if constexpr (OP == OP_MIN) return atomicMin(reinterpret_cast<long long *>(p), (long long)v);
  else if constexpr (OP == OP_MAX) return atomicMax(reinterpret_cast<long long *>(p), (long long)v);
  else return int64_t(atomicExch(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v));
}
template <int OP> __device__ __forceinline__ float atomic_apply(float *p, float v) {
  if constexpr (OP == OP_SUM) return atomicAdd(p, v);
  else if constexpr (OP == OP_REPLACE) return atomicExch(p, v);
  else {
    unsigned int *u = reinterpret_cast<unsigned int *>(p);
    unsigned int old = *u, assumed;
    do {
      assumed = old;
      const float cur = __uint_as_float(assumed);
      const float nv = combine<OP, float>(cur, v);
      if (__float_as_uint(nv) == assumed) break;
      old = atomicCAS(u, assumed, __float_as_uint(nv));
    } while (old != assumed);
    return __uint_as_float(old);
  }
}
template <int OP> __device__ __forceinline__ double atomic_apply(double *p, double v) {
  if constexpr (OP == OP_SUM) return atomicAdd(p, v);
  else {
    unsigned long long *u = reinterpret_cast<unsigned long long *>(p);
    unsigned long long old = *u, assumed;
    do {
      assumed = old;
      const double cur = __longlong_as_double((long long)assumed);
      const double nv = combine<OP, double>(cur, v);
      const unsigned long long nb = (unsigned long long)__double_as_longlong(nv);
      if (nb == assumed) break;
      old = atomicCAS(u, assumed, nb);
    } while (old != assumed);
    return __longlong_as_double((long long)old);
  }
}
template <int OP> __device__ __forceinline__ bf16 atomic_apply(bf16 *p, bf16 v) {
  unsigned short *u = reinterpret_cast<unsigned short *>(p);
  unsigned short old = *u, assumed;
  do {
    assumed = old;
    bf16 cur;
    memcpy(&cur, &assumed, 2);
    const bf16 nv = combine<OP, bf16>(cur, v);
    unsigned short nb;
    memcpy(&nb, &nv, 2);
    if (nb == assumed) break;
    old = atomicCAS(u, assumed, nb);
  } while (old != assumed);
  bf16 r;
  memcpy(&r, &old, 2);
  return r;
}

// ------------------------------------------------------------------ run addressing
__device__ __forceinline__ int64_t pattern_unit(int64_t base, int64_t sy, int64_t sz, int32_t k, int32_t nx,
                                                int32_t ny, bool flat) {
  if (flat) return base + k;
  const int32_t i = k % nx, jz = k / nx, j = jz % ny, z = jz / ny;
  return base + i + int64_t(j) * sy + int64_t(z) * sz;
}

struct TsArgs {
  const Run *runs;
  const int32_t *ridx, *lidx;
  const Tile *tiles;
  const void *src;      // Bcast: rootdata (fused/pack) or leaf buffer (unpack); Reduce: leafdata / root buffer
  void *dst;            // Bcast: leafdata (fused/unpack) or root buffer (pack); Reduce: rootdata / leaf buffer
  void *upd;            // FetchAndOp: leafupdate
  int32_t nv;           // vectors per unit
  int32_t phase;        // PH_*
};

// One CTA per tile of a TS run.  L2R = leaf -> root (Reduce / FetchAndOp), else root -> leaf.
template <typename T, int VB, int OP, bool L2R, bool ATOMIC, bool FETCH>
__global__ void __launch_bounds__(kThreads) ts_kernel(TsArgs a) {
  const Tile t = a.tiles[blockIdx.x];
  const Run r = a.runs[t.a];
  const bool flat = r.nx >= r.n;
  const int32_t nv = a.nv;
  const int64_t work = int64_t(t.cnt) * nv;
  for (int64_t base = threadIdx.x; base < work; base += int64_t(kThreads) * kUnroll) {
    int64_t su[kUnroll], du[kUnroll], lu[kUnroll];
    int32_t vv[kUnroll];
    bool ok[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t w = base + int64_t(u) * kThreads;
      ok[u] = w < work;
      const int32_t kl = ok[u] ? int32_t(w / nv) : 0;
      vv[u] = ok[u] ? int32_t(w - int64_t(kl) * nv) : 0;
      const int32_t k = t.k0 + kl;
      const int64_t ru = (r.flags & RUN_ROOT_IDX) ? int64_t(a.ridx[r.idx0 + k])
                                                  : pattern_unit(r.root0, r.rsy, r.rsz, k, r.nx, r.ny, flat);
      const int64_t leafu = (r.flags & RUN_LEAF_IDX) ? int64_t(a.lidx[r.idx0 + k])
                                                     : pattern_unit(r.leaf0, r.lsy, r.lsz, k, r.nx, r.ny, flat);
      int64_t s = L2R ? leafu : ru, d = L2R ? ru : leafu;
      if (a.phase == PH_PACK) d = (L2R ? r.lbuf0 : r.rbuf0) + k;
      if (a.phase == PH_UNPACK) s = (L2R ? r.rbuf0 : r.lbuf0) + k;
      su[u] = s;
      du[u] = d;
      lu[u] = leafu;
    }
    Pack<T, VB> x[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (ok[u]) x[u] = ld<T, VB>(a.src, su[u] * nv + vv[u]);
    if constexpr (ATOMIC) {
      static_assert(VB == sizeof(T), "atomics are element-wise");
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (ok[u]) {
          T *p = reinterpret_cast<T *>(a.dst) + du[u] * nv + vv[u];
          const T old = atomic_apply<OP>(p, x[u].v[0]);
          if constexpr (FETCH) reinterpret_cast<T *>(a.upd)[lu[u] * nv + vv[u]] = old;
        }
    } else {
      if constexpr (OP == OP_REPLACE) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
          if (ok[u]) st<T, VB>(a.dst, du[u] * nv + vv[u], x[u]);
      } else {
        Pack<T, VB> y[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
          if (ok[u]) y[u] = ld<T, VB>(a.dst, du[u] * nv + vv[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
          if (ok[u]) st<T, VB>(a.dst, du[u] * nv + vv[u], combine<OP, T, VB>(y[u], x[u]));
      }
    }
  }
}

// Buffer move: one CTA per slice of a (root rank -> leaf rank) chunk.
struct MoveArgs {
  const SegCopy *segs;
  const Tile *tiles;   // a = segment, k0 = first unit, cnt = units
  const void *src;
  void *dst;
  int32_t nv;
  int32_t reverse;     // copy dst0 -> src0 (Reduce direction)
};
template <int VB>
__global__ void __launch_bounds__(kThreads) move_kernel(MoveArgs a) {
  const Tile t = a.tiles[blockIdx.x];
  const SegCopy s = a.segs[t.a];
  const int64_t from = (a.reverse ? s.dst0 : s.src0) + t.k0, to = (a.reverse ? s.src0 : s.dst0) + t.k0;
  const int64_t work = int64_t(t.cnt) * a.nv;
  using R = typename Raw<VB>::type;
  const R *src = reinterpret_cast<const R *>(a.src) + from * a.nv;
  R *dst = reinterpret_cast<R *>(a.dst) + to * a.nv;
  for (int64_t base = threadIdx.x; base < work; base += int64_t(kThreads) * kUnroll) {
    R x[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t w = base + int64_t(u) * kThreads;
      if (w < work) x[u] = src[w];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t w = base + int64_t(u) * kThreads;
      if (w < work) dst[w] = x[u];
    }
  }
}

// ------------------------------------------------------------------ root-major kernel
struct RmArgs {
  const MaskedRun *mruns;
  const uint32_t *mask;
  const int32_t *pr_root, *pr_leaf;
  const int32_t *m_root, *m_ptr, *m_leaf, *m_slot, *m_ctr, *ch_m, *ch_e0;
  const Tile *tiles;
  void *root;           // rootdata (read for Bcast, read-modify-write otherwise)
  void *leaf;           // leafdata (read for Reduce / FetchAndOp, read-modify-write for Bcast)
  void *upd;            // leafupdate (FetchAndOp)
  void *partial;        // scratch: fold partials of multi-block roots
  int32_t *counter;     // scratch: arrivals per (multi-block root, vector); zero between calls
  int32_t nv;
};

// Deterministic fold D over n partials (stride nv) of one (root, vector), in place, L2 only.
template <typename A, int VB, int OP>
__device__ Pack<A, VB> fold_partials(void *partial, int64_t slot, int32_t nv, int32_t v, int32_t n) {
  while (n > FOLD_BLOCK) {
    int32_t m = 0;
    for (int32_t s = 0; s < n; s += FOLD_BLOCK) {
      const int32_t e = min(s + FOLD_BLOCK, n);
      Pack<A, VB> acc = ld_cg<A, VB>(partial, (slot + s) * nv + v);
      for (int32_t i = s + 1; i < e; ++i) acc = combine<OP, A, VB>(acc, ld_cg<A, VB>(partial, (slot + i) * nv + v));
      st_cg<A, VB>(partial, (slot + m) * nv + v, acc);   // m <= s: its block was already read
      ++m;
    }
    n = m;
  }
  Pack<A, VB> acc = ld_cg<A, VB>(partial, slot * nv + v);
  for (int32_t i = 1; i < n; ++i) acc = combine<OP, A, VB>(acc, ld_cg<A, VB>(partial, (slot + i) * nv + v));
  return acc;
}

template <typename T, int VB, int OP, int MODE>
__device__ __forceinline__ void single_edge(const RmArgs &a, int64_t ru, int64_t leafu, int32_t v) {
  const int64_t ri = ru * a.nv + v, li = leafu * a.nv + v;
  if constexpr (MODE == RM_BCAST) {
    const Pack<T, VB> x = ld<T, VB>(a.root, ri);
    if constexpr (OP == OP_REPLACE) st<T, VB>(a.leaf, li, x);
    else st<T, VB>(a.leaf, li, combine<OP, T, VB>(ld<T, VB>(a.leaf, li), x));
  } else if constexpr (MODE == RM_REDUCE) {
    const Pack<T, VB> y = ld<T, VB>(a.leaf, li);
    if constexpr (OP == OP_REPLACE) st<T, VB>(a.root, ri, y);
    else st<T, VB>(a.root, ri, combine<OP, T, VB>(ld<T, VB>(a.root, ri), y));
  } else {
    const Pack<T, VB> y = ld<T, VB>(a.leaf, li);
    const Pack<T, VB> x = ld<T, VB>(a.root, ri);
    st<T, VB>(a.upd, li, x);
    st<T, VB>(a.root, ri, combine<OP, T, VB>(x, y));
  }
}

template <typename T, int VB, int OP, int MODE>
__global__ void __launch_bounds__(kThreads) rm_kernel(RmArgs a) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;   // accumulator pack bytes
  const Tile t = a.tiles[blockIdx.x];
  const int32_t nv = a.nv;
  const int64_t work = int64_t(t.cnt) * nv;
  if (t.kind == T_MASKED) {
    const MaskedRun mr = a.mruns[t.a];
    for (int64_t w = threadIdx.x; w < work; w += kThreads) {
      const int32_t kl = int32_t(w / nv), v = int32_t(w - int64_t(kl) * nv), k = t.k0 + kl;
      const int64_t bit = mr.mask0 + k;
      if ((a.mask[bit >> 5] >> (bit & 31)) & 1u) single_edge<T, VB, OP, MODE>(a, mr.root0 + k, mr.leaf0 + k, v);
    }
  } else if (t.kind == T_PAIRS) {
    for (int64_t w = threadIdx.x; w < work; w += kThreads) {
      const int32_t kl = int32_t(w / nv), v = int32_t(w - int64_t(kl) * nv), i = t.a + kl;
      single_edge<T, VB, OP, MODE>(a, a.pr_root[i], a.pr_leaf[i], v);
    }
  } else if (t.kind == T_WINNERS) {
    if constexpr (MODE == RM_REDUCE && OP == OP_REPLACE) {
      for (int64_t w = threadIdx.x; w < work; w += kThreads) {
        const int32_t kl = int32_t(w / nv), v = int32_t(w - int64_t(kl) * nv), m = t.a + kl;
        const int64_t last = a.m_leaf[a.m_ptr[m + 1] - 1];
        st<T, VB>(a.root, int64_t(a.m_root[m]) * nv + v, ld<T, VB>(a.leaf, last * nv + v));
      }
    }
  } else if (t.kind == T_FETCH) {
    if constexpr (MODE == RM_FETCH) {
      for (int64_t w = threadIdx.x; w < work; w += kThreads) {
        const int32_t kl = int32_t(w / nv), v = int32_t(w - int64_t(kl) * nv), m = t.a + kl;
        const int64_t ri = int64_t(a.m_root[m]) * nv + v;
        Pack<T, VB> x = ld<T, VB>(a.root, ri);
        const int32_t e1 = a.m_ptr[m + 1];
        for (int32_t e = a.m_ptr[m]; e < e1; ++e) {
          const int64_t li = int64_t(a.m_leaf[e]) * nv + v;
          const Pack<T, VB> y = ld<T, VB>(a.leaf, li);
          st<T, VB>(a.upd, li, x);
          x = combine<OP, T, VB>(x, y);
        }
        st<T, VB>(a.root, ri, x);
      }
    }
  } else if (t.kind == T_CHUNKS) {
    for (int64_t w = threadIdx.x; w < work; w += kThreads) {
      const int32_t cl = int32_t(w / nv), v = int32_t(w - int64_t(cl) * nv), c = t.a + cl;
      const int32_t m = a.ch_m[c], e0 = a.ch_e0[c], mp0 = a.m_ptr[m], mp1 = a.m_ptr[m + 1];
      const int32_t e1 = min(e0 + FOLD_BLOCK, mp1);
      const int64_t ri = int64_t(a.m_root[m]) * nv + v;
      if constexpr (MODE == RM_BCAST) {
        const Pack<T, VB> x = ld<T, VB>(a.root, ri);
        for (int32_t e = e0; e < e1; ++e) {
          const int64_t li = int64_t(a.m_leaf[e]) * nv + v;
          if constexpr (OP == OP_REPLACE) st<T, VB>(a.leaf, li, x);
          else st<T, VB>(a.leaf, li, combine<OP, T, VB>(ld<T, VB>(a.leaf, li), x));
        }
      } else if constexpr (MODE == RM_REDUCE && OP != OP_REPLACE) {
        // left fold of this block in canonical order, 4 leaves in flight
        Pack<A, AVB> acc;
        {
          const Pack<T, VB> y = ld<T, VB>(a.leaf, int64_t(a.m_leaf[e0]) * nv + v);
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l) acc.v[l] = to_acc<A, T>(y.v[l]);
        }
        int32_t e = e0 + 1;
        for (; e + 4 <= e1; e += 4) {
          Pack<T, VB> y[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) y[u] = ld<T, VB>(a.leaf, int64_t(a.m_leaf[e + u]) * nv + v);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int l = 0; l < Pack<T, VB>::L; ++l) acc.v[l] = combine<OP, A>(acc.v[l], to_acc<A, T>(y[u].v[l]));
        }
        for (; e < e1; ++e) {
          const Pack<T, VB> y = ld<T, VB>(a.leaf, int64_t(a.m_leaf[e]) * nv + v);
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l) acc.v[l] = combine<OP, A>(acc.v[l], to_acc<A, T>(y.v[l]));
        }
        const int32_t nch = (mp1 - mp0 + FOLD_BLOCK - 1) / FOLD_BLOCK;
        bool finish = nch == 1;
        if (!finish) {
          const int64_t slot = a.m_slot[m];
          const int32_t ci = (e0 - mp0) / FOLD_BLOCK;
          st_cg<A, AVB>(a.partial, (slot + ci) * nv + v, acc);
          __threadfence();
          int32_t *ctr = a.counter + int64_t(a.m_ctr[m]) * nv + v;
          if (atomicAdd(ctr, 1) == nch - 1) {
            __threadfence();
            acc = fold_partials<A, AVB, OP>(a.partial, slot, nv, v, nch);
            *ctr = 0;   // ready for the next operation
            finish = true;
          }
        }
        if (finish) {
          Pack<T, VB> x = ld<T, VB>(a.root, ri);
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l) x.v[l] = apply_acc<OP, T, A>(x.v[l], acc.v[l]);
          st<T, VB>(a.root, ri, x);
        }
      }
    }
  }
}

}  // namespace sfgb
