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
// floor(n / d) for 0 <= n < 2^31 from d's DivMagic (m, s): one wide multiply and a shift.
__device__ __forceinline__ int32_t div_by(int32_t n, uint32_t m, int32_t s) {
  return int32_t((uint64_t(uint32_t(n)) * m) >> s);
}

struct TsArgs {
  const int32_t *ridx, *lidx;
  const TsTile *tiles;
  int32_t ntiles;
  const void *src;      // Bcast: rootdata (fused/pack) or leaf buffer (unpack); Reduce: leafdata / root buffer
  void *dst;            // Bcast: leafdata (fused/unpack) or root buffer (pack); Reduce: rootdata / leaf buffer
  void *upd;            // FetchAndOp: leafupdate
  int32_t nv;           // vectors per unit
  int32_t phase;        // PH_*
  uint32_t nv_m;        // DivMagic of nv
  int32_t nv_s;
};

// Contiguous tile, copy: n bytes from s to d.  Both are aligned to `gran` bytes; 16-byte
// vectors carry the body whenever s and d share their offset modulo 16.
template <int GRAN>
__device__ __forceinline__ void copy_contiguous(const char *s, char *d, int64_t n) {
  using G = typename Raw<GRAN>::type;
  const bool v16 = GRAN == 16 || ((reinterpret_cast<uintptr_t>(s) ^ reinterpret_cast<uintptr_t>(d)) & 15) == 0;
  if (!v16) {
    // s and d disagree modulo 16: GRAN-sized accesses, 8 in flight per thread
    constexpr int UG = 8;
    const G *sg = reinterpret_cast<const G *>(s);
    G *dg = reinterpret_cast<G *>(d);
    const int64_t ng = n / GRAN;
    for (int64_t base = threadIdx.x; base < ng; base += int64_t(kThreads) * UG) {
      G x[UG];
#pragma unroll
      for (int u = 0; u < UG; ++u)
        if (base + u * kThreads < ng) x[u] = sg[base + u * kThreads];
#pragma unroll
      for (int u = 0; u < UG; ++u)
        if (base + u * kThreads < ng) dg[base + u * kThreads] = x[u];
    }
    return;
  }
  // head up to the first 16-byte boundary of d, 16-byte body, tail: head and tail in GRAN units
  const int64_t align_gap = int64_t((16 - (reinterpret_cast<uintptr_t>(d) & 15)) & 15);
  const int64_t head = GRAN == 16 ? 0 : (n < align_gap ? n : align_gap);
  const int64_t body = ((n - head) / 16) * 16;
  for (int64_t i = threadIdx.x; i < head / GRAN; i += kThreads)
    reinterpret_cast<G *>(d)[i] = reinterpret_cast<const G *>(s)[i];
  for (int64_t i = (head + body) / GRAN + threadIdx.x; i < n / GRAN; i += kThreads)
    reinterpret_cast<G *>(d)[i] = reinterpret_cast<const G *>(s)[i];
  constexpr int U = 4;
  const uint4 *sv = reinterpret_cast<const uint4 *>(s + head);
  uint4 *dv = reinterpret_cast<uint4 *>(d + head);
  const int64_t nb = body / 16;
  for (int64_t base = threadIdx.x; base < nb; base += int64_t(kThreads) * U) {
    uint4 x[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * kThreads < nb) x[u] = sv[base + u * kThreads];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * kThreads < nb) dv[base + u * kThreads] = x[u];
  }
}

// One CTA per tile of a TS run.  L2R = leaf -> root (Reduce / FetchAndOp), else root -> leaf.
// Tile-uniform paths: contiguous on both sides (a copy or an element-wise op), each side
// contiguous or indexed (gathers and scatters), and the general multi-strided / indexed case.
// Unit indices, run offsets and strides are below 2^31 (the library's size limit), so they are
// carried in 32 bits; only unit * nv + v, the vector index, is formed in 64 bits.
template <typename T, int VB, int OP, bool L2R, bool ATOMIC, bool FETCH>
__device__ __forceinline__ void ts_tile(const TsArgs &a, const TsTile &t) {
  const bool flat = t.nx >= t.n;
  const int32_t nv = a.nv;
  const bool ridx = t.flags & RUN_ROOT_IDX, lidx = t.flags & RUN_LEAF_IDX;
  // source / destination side descriptions
  bool s_idx = L2R ? lidx : ridx, d_idx = L2R ? ridx : lidx;
  bool s_flat = flat && !s_idx, d_flat = flat && !d_idx;
  int32_t s0 = L2R ? t.leaf0 : t.root0, d0 = L2R ? t.root0 : t.leaf0;
  if (a.phase == PH_PACK) { d_flat = true; d_idx = false; d0 = L2R ? t.lbuf0 : t.rbuf0; }
  if (a.phase == PH_UNPACK) { s_flat = true; s_idx = false; s0 = L2R ? t.rbuf0 : t.lbuf0; }
  const int32_t work = t.cnt * nv;   // < 2^31: units are at most SF_MAX_UNIT_BYTES
  if constexpr (!ATOMIC) {
    if (s_flat && d_flat) {
      const int64_t sb = int64_t(s0 + t.k0) * nv, db = int64_t(d0 + t.k0) * nv;
      if constexpr (OP == OP_REPLACE) {
        copy_contiguous<VB>(static_cast<const char *>(a.src) + sb * VB, static_cast<char *>(a.dst) + db * VB,
                            int64_t(work) * VB);
      } else {
        for (int32_t base = threadIdx.x; base < work; base += kThreads * kUnroll) {
          Pack<T, VB> x[kUnroll], y[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u)
            if (base + u * kThreads < work) {
              x[u] = ld<T, VB>(a.src, sb + base + u * kThreads);
              y[u] = ld<T, VB>(a.dst, db + base + u * kThreads);
            }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u)
            if (base + u * kThreads < work) st<T, VB>(a.dst, db + base + u * kThreads, combine<OP, T, VB>(y[u], x[u]));
        }
      }
      return;
    }
  }
  if ((s_flat || s_idx) && (d_flat || d_idx)) {
    // each side contiguous or indexed: gathers, scatters, both indexed, atomics
    const int32_t *sidx = (L2R ? a.lidx : a.ridx) + t.idx0 + t.k0;
    const int32_t *didx = (L2R ? a.ridx : a.lidx) + t.idx0 + t.k0;
    const int32_t sb = s0 + t.k0, db = d0 + t.k0;
    constexpr int UG = 4;   // 16-byte kernels run 2 CTAs per SM: registers for 4 in flight
    for (int32_t base = threadIdx.x; base < work; base += kThreads * UG) {
      int32_t su[UG], du[UG], vv[UG];
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        const int32_t w = base + u * kThreads;
        const int32_t k = w < work ? (nv == 1 ? w : div_by(w, a.nv_m, a.nv_s)) : 0;
        vv[u] = w - k * nv;
        su[u] = s_idx ? __ldg(sidx + k) : sb + k;
        du[u] = d_idx ? __ldg(didx + k) : db + k;
      }
      Pack<T, VB> x[UG];
#pragma unroll
      for (int u = 0; u < UG; ++u)
        if (base + u * kThreads < work) x[u] = ld<T, VB>(a.src, int64_t(su[u]) * nv + vv[u]);
      if constexpr (ATOMIC) {
        static_assert(VB == sizeof(T), "atomics are element-wise");
#pragma unroll
        for (int u = 0; u < UG; ++u)
          if (base + u * kThreads < work) {
            const T old = atomic_apply<OP>(reinterpret_cast<T *>(a.dst) + int64_t(du[u]) * nv + vv[u], x[u].v[0]);
            if constexpr (FETCH) reinterpret_cast<T *>(a.upd)[int64_t(su[u]) * nv + vv[u]] = old;   // source = leaf
          }
      } else if constexpr (OP == OP_REPLACE) {
#pragma unroll
        for (int u = 0; u < UG; ++u)
          if (base + u * kThreads < work) st<T, VB>(a.dst, int64_t(du[u]) * nv + vv[u], x[u]);
      } else {
        Pack<T, VB> y[UG];
#pragma unroll
        for (int u = 0; u < UG; ++u)
          if (base + u * kThreads < work) y[u] = ld<T, VB>(a.dst, int64_t(du[u]) * nv + vv[u]);
#pragma unroll
        for (int u = 0; u < UG; ++u)
          if (base + u * kThreads < work) st<T, VB>(a.dst, int64_t(du[u]) * nv + vv[u], combine<OP, T, VB>(y[u], x[u]));
      }
    }
    return;
  }
  // general: pattern or index on either side.  Edge k of the run sits at (i, j, z) of its
  // nx x ny x nz box, decomposed once for both sides with multiply-shift divisions; a pattern
  // address is formed modulo 2^32 (exact, since the result is a unit index below 2^31).
  constexpr int UP = (OP == OP_REPLACE && !ATOMIC && VB < 16) ? 2 : kUnroll;
  for (int32_t base = threadIdx.x; base < work; base += kThreads * UP) {
    int32_t su[UP], du[UP], lu[UP], vv[UP];
#pragma unroll
    for (int u = 0; u < UP; ++u) {
      const int32_t w = base + u * kThreads;
      const int32_t kl = w >= work ? 0 : nv == 1 ? w : div_by(w, a.nv_m, a.nv_s);
      vv[u] = w - kl * nv;
      const int32_t k = t.k0 + kl;
      uint32_t i = uint32_t(k), j = 0, z = 0;
      if (!flat) {
        const int32_t jz = div_by(k, t.mx, t.sx);
        i = uint32_t(k - jz * t.nx);
        z = uint32_t(div_by(jz, t.my, t.sy));
        j = uint32_t(jz) - z * uint32_t(t.ny);
      }
      const int32_t ru = ridx ? __ldg(a.ridx + t.idx0 + k)
                              : int32_t(uint32_t(t.root0) + i + j * uint32_t(t.rsy) + z * uint32_t(t.rsz));
      const int32_t leafu = lidx ? __ldg(a.lidx + t.idx0 + k)
                                 : int32_t(uint32_t(t.leaf0) + i + j * uint32_t(t.lsy) + z * uint32_t(t.lsz));
      int32_t s = L2R ? leafu : ru, d = L2R ? ru : leafu;
      if (a.phase == PH_PACK) d = (L2R ? t.lbuf0 : t.rbuf0) + k;
      if (a.phase == PH_UNPACK) s = (L2R ? t.rbuf0 : t.lbuf0) + k;
      su[u] = s;
      du[u] = d;
      lu[u] = leafu;
    }
    Pack<T, VB> x[UP];
#pragma unroll
    for (int u = 0; u < UP; ++u)
      if (base + u * kThreads < work) x[u] = ld<T, VB>(a.src, int64_t(su[u]) * nv + vv[u]);
    if constexpr (ATOMIC) {
      static_assert(VB == sizeof(T), "atomics are element-wise");
#pragma unroll
      for (int u = 0; u < UP; ++u)
        if (base + u * kThreads < work) {
          T *p = reinterpret_cast<T *>(a.dst) + int64_t(du[u]) * nv + vv[u];
          const T old = atomic_apply<OP>(p, x[u].v[0]);
          if constexpr (FETCH) reinterpret_cast<T *>(a.upd)[int64_t(lu[u]) * nv + vv[u]] = old;
        }
    } else {
      if constexpr (OP == OP_REPLACE) {
#pragma unroll
        for (int u = 0; u < UP; ++u)
          if (base + u * kThreads < work) st<T, VB>(a.dst, int64_t(du[u]) * nv + vv[u], x[u]);
      } else {
        Pack<T, VB> y[UP];
#pragma unroll
        for (int u = 0; u < UP; ++u)
          if (base + u * kThreads < work) y[u] = ld<T, VB>(a.dst, int64_t(du[u]) * nv + vv[u]);
#pragma unroll
        for (int u = 0; u < UP; ++u)
          if (base + u * kThreads < work) st<T, VB>(a.dst, int64_t(du[u]) * nv + vv[u], combine<OP, T, VB>(y[u], x[u]));
      }
    }
  }
}

// Resident CTAs per SM the register budget must allow: copies are lean, op kernels carry
// arithmetic and more live state.  Measured on the 2^24-root Reduce SUM: 4 CTAs of 64
// registers (a small spill in the rare multi-block combine) beat 3 of 80 (none) and 5 of 48.
template <int OP, int VB, bool ATOMIC = false> struct MinBlocks {
  static constexpr int value = ATOMIC ? 4 : OP == OP_REPLACE ? (VB >= 16 ? 4 : 6) : (VB >= 16 ? 2 : 4);
};
// Resident CTAs per SM of the one-vector-unit Reduce kernel (rm_kernel / rm_batch_kernel with
// NV1): 4 CTAs of 64 registers, no spills; 5 of 48 or 6 of 40 (with smaller gather buffers)
// measured 16-17% slower on the 2^24-root Reduce SUM.
constexpr int RM_NV1_BLOCKS = 4;

// One CTA per tile (the hardware balances uneven tiles); the tile carries its run inline so a
// single descriptor load precedes the data.
template <typename T, int VB, int OP, bool L2R, bool ATOMIC, bool FETCH>
__global__ void __launch_bounds__(kThreads, (MinBlocks<OP, VB, ATOMIC>::value)) ts_kernel(TsArgs a) {
  const TsTile t = a.tiles[blockIdx.x];
  ts_tile<T, VB, OP, L2R, ATOMIC, FETCH>(a, t);
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
  const uint32_t *mask;
  const int32_t *pr_root, *pr_leaf;
  const int32_t *m_root, *m_ptr, *m_leaf;
  const BlockRec *blocks;
  const Comb *combs;
  const RmTile *tiles;
  int32_t ntiles;
  void *root;           // rootdata (read for Bcast, read-modify-write otherwise)
  void *leaf;           // leafdata (read for Reduce / FetchAndOp, read-modify-write for Bcast)
  void *upd;            // leafupdate (FetchAndOp)
  void *partial;        // scratch: fold partials of multi-block roots
  int32_t *counter;     // scratch: arrivals per (multi-block root, vector); zero between calls
  int32_t *status;      // device status word of the forest (DEVSTAT_* bits)
  int32_t zero_root;    // Reduce from zero: every root counts as 0 before the operation (never read)
  int32_t nv;
  uint32_t nv_m;        // DivMagic of nv
  int32_t nv_s;
};

// ------------------------------------------------------------------ bulk staging into shared memory
constexpr long long kWaitCycles = 1ll << 31;   // about 1 s at 2 GHz: the bound of every barrier wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Wait until phase `parity` of the mbarrier at shared address `bar` completes, at most `limit`
// clock cycles; false if it did not.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Two bulk copies global -> shared (cp.async.bulk: 16-byte aligned addresses, sizes multiples
// of 16) issued by thread 0, completion counted in bytes on one mbarrier.  Every thread of the
// CTA calls this and waits; true once the data is in shared memory.  If the wait runs out, the
// forest's status word gets DEVSTAT_STAGE_TIMEOUT, the copies get one more bounded wait, and
// the result is false (the caller skips the tile).
__device__ __forceinline__ bool stage2(void *dst0, const void *src0, uint32_t bytes0, void *dst1, const void *src1,
                                       uint32_t bytes1, uint64_t *bar, int32_t *status) {
  const uint32_t b = smem_addr(bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes0 + bytes1) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst0)), "l"(src0), "r"(bytes0), "r"(b) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst1)), "l"(src1), "r"(bytes1), "r"(b) : "memory");
  }
  if (mbar_wait(b, 0, kWaitCycles)) return true;
  if (threadIdx.x == 0 && status) atomicOr(status, DEVSTAT_STAGE_TIMEOUT);
  mbar_wait(b, 0, kWaitCycles);
  return false;
}

// The current value of root vector i for a Reduce: zero, without a load, when the operation
// starts its roots at zero (sf_reduce_from_zero).
template <typename T, int VB> __device__ __forceinline__ Pack<T, VB> ld_root(const void *root, int64_t i, bool zr) {
  Pack<T, VB> z;
  if (zr) {
    memset(&z, 0, sizeof z);
    return z;
  }
  return ld<T, VB>(root, i);
}

// Index load: read-only global path, or a plain load when the indices were staged in shared memory.
template <bool SM> __device__ __forceinline__ int32_t ld_idx(const int32_t *p) {
  if constexpr (SM) return *p;
  else return __ldg(p);
}

// Expand stored block c (8-byte record plus the next record's first edge) into a Block.
__device__ __forceinline__ Block load_block(const BlockRec *recs, const Comb *combs, int32_t c) {
  const BlockRec r = recs[c];
  const int32_t e1 = recs[c + 1].e0;
  Block b;
  b.e0 = r.e0;
  b.n = e1 - r.e0;
  if (r.who >= 0) {
    b.root = r.who;
    b.comb = -1;
  } else {
    b.comb = -r.who - 1;
    b.root = combs[b.comb].root;
  }
  return b;
}

// Left fold of n partials (stride nv) starting at slot, 8 loads in flight, L2 only.
template <typename A, int VB, int OP>
__device__ Pack<A, VB> fold_range(const void *partial, int64_t slot, int32_t nv, int32_t v, int32_t n) {
  constexpr int U = 8;
  Pack<A, VB> acc = ld_cg<A, VB>(partial, slot * nv + v);
  int32_t i = 1;
  for (; i + U <= n; i += U) {
    Pack<A, VB> y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) y[u] = ld_cg<A, VB>(partial, (slot + i + u) * nv + v);
#pragma unroll
    for (int u = 0; u < U; ++u) acc = combine<OP, A, VB>(acc, y[u]);
  }
  for (; i < n; ++i) acc = combine<OP, A, VB>(acc, ld_cg<A, VB>(partial, (slot + i) * nv + v));
  return acc;
}

// Deterministic fold D over n partials (stride nv) of one (root, vector), in place, L2 only.
template <typename A, int VB, int OP>
__device__ Pack<A, VB> fold_partials(void *partial, int64_t slot, int32_t nv, int32_t v, int32_t n) {
  while (n > FOLD_BLOCK) {
    int32_t m = 0;
    for (int32_t s = 0; s < n; s += FOLD_BLOCK) {
      const Pack<A, VB> acc = fold_range<A, VB, OP>(partial, slot + s, nv, v, min(FOLD_BLOCK, n - s));
      st_cg<A, VB>(partial, (slot + m) * nv + v, acc);   // m <= s: its block was already read
      ++m;
    }
    n = m;
  }
  return fold_range<A, VB, OP>(partial, slot, nv, v, n);
}

// One single-leaf edge (root unit ru, leaf unit lu), vector v, all loads issued by the caller.
template <typename T, int VB, int OP, int MODE>
__device__ __forceinline__ void single_store(const RmArgs &a, int64_t ri, int64_t li, const Pack<T, VB> &x,
                                             const Pack<T, VB> &y) {
  // x = root vector, y = leaf vector (as loaded; unused ones are ignored)
  if constexpr (MODE == RM_BCAST) {
    if constexpr (OP == OP_REPLACE) st<T, VB>(a.leaf, li, x);
    else st<T, VB>(a.leaf, li, combine<OP, T, VB>(y, x));
  } else if constexpr (MODE == RM_REDUCE) {
    if constexpr (OP == OP_REPLACE) st<T, VB>(a.root, ri, y);
    else st<T, VB>(a.root, ri, combine<OP, T, VB>(x, y));
  } else {
    st<T, VB>(a.upd, li, x);
    st<T, VB>(a.root, ri, combine<OP, T, VB>(x, y));
  }
}

// Which vectors a single-leaf edge must read: the root unless Reduce REPLACE, the leaf unless
// Bcast REPLACE.
template <int OP, int MODE> struct SingleReads {
  static constexpr bool root = !(MODE == RM_REDUCE && OP == OP_REPLACE);
  static constexpr bool leaf = !(MODE == RM_BCAST && OP == OP_REPLACE);
};

// The end of a Reduce fold block whose leaves folded to `acc`: a single-block root gets
// root op= acc (xr holds the root vector, loaded by the caller); a block of a multi-block root
// leaves acc as its partial, and the last arriving block of each super-block of FOLD_BLOCK
// blocks folds that super-block's partials, the last super-block folds those by D and applies
// the result to the root.
template <typename T, int VB, int OP>
__device__ __forceinline__ void fold_finish(void *root, const Comb *combs, void *partial, int32_t *counter,
                                            int32_t nv, const Block &b, int32_t v,
                                            Pack<typename Acc<T, OP>::type, int(sizeof(typename Acc<T, OP>::type)) * Pack<T, VB>::L> acc,
                                            Pack<T, VB> xr, bool zr) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  const int64_t ri = int64_t(b.root) * nv + v;
  bool finish = b.comb < 0;
  if (!finish) {
    const Comb cb = combs[b.comb];
    const int32_t ci = (b.e0 - cb.e_first) / FOLD_BLOCK;       // block index in the root
    const int32_t sb = ci / FOLD_BLOCK;                         // super-block
    const int32_t nsb = (cb.nch + FOLD_BLOCK - 1) / FOLD_BLOCK;
    const int32_t in_sb = min(FOLD_BLOCK, cb.nch - sb * FOLD_BLOCK);
    st_cg<A, AVB>(partial, (int64_t(cb.slot) + ci) * nv + v, acc);
    __threadfence();
    int32_t *ctr = counter + int64_t(cb.ctr + sb) * nv + v;
    if (atomicAdd(ctr, 1) == in_sb - 1) {
      // last block of its super-block: left fold of the super-block's partials
      __threadfence();
      acc = fold_range<A, AVB, OP>(partial, int64_t(cb.slot) + sb * FOLD_BLOCK, nv, v, in_sb);
      *ctr = 0;   // ready for the next operation
      if (nsb == 1) {
        finish = true;
      } else {
        st_cg<A, AVB>(partial, (int64_t(cb.slot1) + sb) * nv + v, acc);
        __threadfence();
        int32_t *rctr = counter + int64_t(cb.ctr + nsb) * nv + v;
        if (atomicAdd(rctr, 1) == nsb - 1) {
          __threadfence();
          acc = fold_partials<A, AVB, OP>(partial, cb.slot1, nv, v, nsb);
          *rctr = 0;
          finish = true;
        }
      }
      if (finish) xr = ld_root<T, VB>(root, ri, zr);
    }
  }
  if (finish) {
#pragma unroll
    for (int l = 0; l < Pack<T, VB>::L; ++l) xr.v[l] = apply_acc<OP, T, A>(xr.v[l], acc.v[l]);
    st<T, VB>(root, ri, xr);
  }
}

// One fold block of a multi-leaf root, vector v: Bcast writes the root to the block's leaves;
// Reduce folds the block's leaves in canonical order and either applies the result to the
// root (single-block root) or leaves a partial whose last arriver folds all partials by D.
template <typename T, int VB, int OP, int MODE, bool SM = false>
__device__ __forceinline__ void fold_block(void *root, void *leaf, const int32_t *m_leaf, int32_t lofs,
                                           const Comb *combs, void *partial, int32_t *counter, int32_t nv,
                                           const Block b, int32_t v, bool zr = false) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  constexpr int U = 4;   // 16-byte kernels run 2 CTAs per SM: registers for 4 leaves in flight
  const int64_t ri = int64_t(b.root) * nv + v;
  const int32_t *lidx = m_leaf + (b.e0 - lofs);   // m_leaf holds entries from lofs on
  if constexpr (MODE == RM_BCAST) {
    const Pack<T, VB> x = ld<T, VB>(root, ri);
    for (int32_t e = 0; e < b.n; e += U) {
      int64_t li[U];
#pragma unroll
      for (int u = 0; u < U; ++u) li[u] = e + u < b.n ? int64_t(ld_idx<SM>(lidx + e + u)) * nv + v : 0;
      if constexpr (OP == OP_REPLACE) {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e + u < b.n) st<T, VB>(leaf, li[u], x);
      } else {
        Pack<T, VB> y[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e + u < b.n) y[u] = ld<T, VB>(leaf, li[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (e + u < b.n) st<T, VB>(leaf, li[u], combine<OP, T, VB>(y[u], x));
      }
    }
  } else if constexpr (MODE == RM_REDUCE && OP != OP_REPLACE) {
    // left fold of this block in canonical order, U leaves in flight
    Pack<T, VB> xr;
    if (b.comb < 0) xr = ld_root<T, VB>(root, ri, zr);   // issued early: independent of the fold
    Pack<A, AVB> acc;
    int32_t e = 0;
    {
      Pack<T, VB> y[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (u < b.n) y[u] = ld<T, VB>(leaf, int64_t(ld_idx<SM>(lidx + u)) * nv + v);
#pragma unroll
      for (int l = 0; l < Pack<T, VB>::L; ++l) acc.v[l] = to_acc<A, T>(y[0].v[l]);
#pragma unroll
      for (int u = 1; u < U; ++u)
        if (u < b.n)
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l) acc.v[l] = combine<OP, A>(acc.v[l], to_acc<A, T>(y[u].v[l]));
      e = U;
    }
    for (; e < b.n; e += U) {
      Pack<T, VB> y[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e + u < b.n) y[u] = ld<T, VB>(leaf, int64_t(ld_idx<SM>(lidx + e + u)) * nv + v);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e + u < b.n)
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l) acc.v[l] = combine<OP, A>(acc.v[l], to_acc<A, T>(y[u].v[l]));
    }
    fold_finish<T, VB, OP>(root, combs, partial, counter, nv, b, v, acc, xr, zr);
  }
}

// Asynchronous global -> shared copy of one VB-byte vector (cp.async: the data goes to shared
// memory without passing through registers, so a thread can keep many in flight).  Both
// addresses are VB-aligned; completion is awaited with cp_async_wait_all.
// The copy itself needs no compiler memory barrier: nothing may read its destination before
// the cp.async.wait that follows it, and that wait is one.
template <int VB> __device__ __forceinline__ void cp_async_vec(void *dst_smem, const void *src) {
  static_assert(VB == 4 || VB == 8 || VB == 16, "cp.async copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst_smem)), "l"(src), "n"(VB));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// A Reduce fold tile of one-vector units (nv == 1), gather-then-fold: with the tile's block
// records (s_rec, from record r0 on) and leaf entries (s_leaf, from entry l0 on) in shared
// memory, every thread first issues the root loads of its blocks, then the CTA copies the
// leaf vectors of the tile's entries into s_val by cp.async -- all of them in flight at once,
// RM_FLAT_BYTES at a time -- and each thread folds its blocks from shared memory, entry by
// entry in canonical order (the same left fold as fold_block), carrying the accumulators
// across rounds.  Every thread of the CTA calls this.
template <typename T, int VB, int OP, bool ZR>
__device__ __forceinline__ void fold_tile_flat(const RmArgs &a, const RmTile &t, const BlockRec *s_rec, int32_t r0,
                                               const int32_t *s_leaf, int32_t l0, Pack<T, VB> *s_val) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  constexpr int R = RM_FLAT_BYTES / VB;                 // leaf vectors per round
  constexpr int NBT = RM_TILE_CHUNKS / kThreads;        // blocks per thread (a tile has <= RM_TILE_CHUNKS)
  const int32_t nE = int32_t(t.e1 - t.k0);              // leaf entries of the tile
  const int32_t *idx = s_leaf + (t.k0 - l0);            // idx[i]: leaf unit of entry k0 + i
  const BlockRec *rec = s_rec + (t.a - r0);             // rec[w]: block a + w (rec[cnt]: the next one)
  Pack<T, VB> xr[NBT];
  Pack<A, AVB> acc[NBT];
#pragma unroll
  for (int j = 0; j < NBT; ++j) {
    const int32_t w = threadIdx.x + j * kThreads;
    if (w < t.cnt && rec[w].who >= 0) xr[j] = ld_root<T, VB>(a.root, rec[w].who, ZR);   // single-block root
  }
  for (int32_t q0 = 0; q0 < nE; q0 += R) {
    const int32_t nq = min(R, nE - q0);
    if (q0 > 0) __syncthreads();   // the previous round's vectors are folded
    for (int32_t k = threadIdx.x; k < nq; k += kThreads)
      cp_async_vec<VB>(s_val + k, static_cast<const char *>(a.leaf) + int64_t(idx[q0 + k]) * VB);
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NBT; ++j) {
      const int32_t w = threadIdx.x + j * kThreads;
      if (w >= t.cnt) continue;
      const int32_t b0 = rec[w].e0 - t.k0, b1 = rec[w + 1].e0 - t.k0;   // the block's entries
      const int32_t lo = max(b0, q0), hi = min(b1, q0 + nq);
      for (int32_t i = lo; i < hi; ++i) {
        const Pack<T, VB> y = s_val[i - q0];
#pragma unroll
        for (int l = 0; l < Pack<T, VB>::L; ++l)
          acc[j].v[l] = i == b0 ? to_acc<A, T>(y.v[l]) : combine<OP, A>(acc[j].v[l], to_acc<A, T>(y.v[l]));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NBT; ++j) {
    const int32_t w = threadIdx.x + j * kThreads;
    if (w < t.cnt) {
      const Block b = load_block(rec, a.combs, w);
      fold_finish<T, VB, OP>(a.root, a.combs, a.partial, a.counter, 1, b, 0, acc[j], xr[j], ZR);
    }
  }
}

// Gather-then-fold for units of nv > 1 vectors (FLAT kernels; Reduce SUM/MIN/MAX): the tile's
// blocks are taken in groups of at most NIT * kThreads (block, vector) items, a thread holding up
// to NIT of them (4, or 2 for 16-byte vectors, whose packs would spill at four).  For each group the CTA copies the leaf vectors of the
// group's entries into s_val by cp.async -- R / nv whole leaf units per round, every vector of
// the round in flight at once whatever the blocks' lengths -- and each item folds its block's
// entries of the round from shared memory in canonical order, carrying its accumulator across
// rounds (the same left fold as fold_block).  Every thread of the CTA calls this.
template <typename T, int VB, int OP, bool ZR>
__device__ __forceinline__ void fold_tile_flat_nv(const RmArgs &a, const RmTile &t, const BlockRec *s_rec, int32_t r0,
                                                  const int32_t *s_leaf, int32_t l0, Pack<T, VB> *s_val) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  constexpr int NIT = VB >= 16 ? 2 : 4;                  // items per thread
  static_assert(NIT * kThreads >= RM_FLAT_MAX_NV, "a group holds at least one block");
  constexpr int R = RM_FLAT_BYTES / VB;                  // leaf vectors per round
  const int32_t nv = a.nv;                               // 1 < nv <= min(R, RM_FLAT_MAX_NV)
  const int32_t gb = NIT * kThreads / nv;                // blocks per group
  const int32_t rl = R / nv;                             // leaf units per round
  const int32_t *idx = s_leaf + (t.k0 - l0);             // idx[i]: leaf unit of entry k0 + i
  const BlockRec *rec = s_rec + (t.a - r0);              // rec[w]: block a + w (rec[cnt]: the next one)
  const char *leaf = static_cast<const char *>(a.leaf);
  for (int32_t g0 = 0; g0 < t.cnt; g0 += gb) {
    const int32_t g1 = min(t.cnt, g0 + gb), nitems = (g1 - g0) * nv;
    int32_t bw[NIT], vv[NIT];
    Pack<T, VB> xr[NIT];
    Pack<A, AVB> acc[NIT];
#pragma unroll
    for (int j = 0; j < NIT; ++j) {
      const int32_t it = threadIdx.x + j * kThreads;
      bw[j] = -1;
      if (it < nitems) {
        const int32_t q = div_by(it, a.nv_m, a.nv_s);
        bw[j] = g0 + q;
        vv[j] = it - q * nv;
        if (rec[bw[j]].who >= 0) xr[j] = ld_root<T, VB>(a.root, int64_t(rec[bw[j]].who) * nv + vv[j], ZR);
      }
    }
    const int32_t e0 = int32_t(rec[g0].e0 - t.k0), e1 = int32_t(rec[g1].e0 - t.k0);   // the group's entries
    for (int32_t q0 = e0; q0 < e1; q0 += rl) {
      const int32_t nq = min(rl, e1 - q0), nvec = nq * nv;
      if (q0 > e0) __syncthreads();   // the previous round's vectors are folded
      for (int32_t k = threadIdx.x; k < nvec; k += kThreads) {
        const int32_t e = div_by(k, a.nv_m, a.nv_s), v = k - e * nv;
        cp_async_vec<VB>(s_val + k, leaf + (int64_t(idx[q0 + e]) * nv + v) * VB);
      }
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NIT; ++j) {
        if (bw[j] < 0) continue;
        const int32_t b0 = int32_t(rec[bw[j]].e0 - t.k0), b1 = int32_t(rec[bw[j] + 1].e0 - t.k0);
        const int32_t lo = max(b0, q0), hi = min(b1, q0 + nq);
        for (int32_t i = lo; i < hi; ++i) {
          const Pack<T, VB> y = s_val[(i - q0) * nv + vv[j]];
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l)
            acc[j].v[l] = i == b0 ? to_acc<A, T>(y.v[l]) : combine<OP, A>(acc[j].v[l], to_acc<A, T>(y.v[l]));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NIT; ++j)
      if (bw[j] >= 0)
        fold_finish<T, VB, OP>(a.root, a.combs, a.partial, a.counter, nv, load_block(rec, a.combs, bw[j]), vv[j], acc[j],
                               xr[j], ZR);
    __syncthreads();   // s_val is free for the next group
  }
}

// NB single-block roots folded together (Reduce SUM/MIN/MAX): NB descriptors, then U leaf
// indices per root, then U leaf values per root are in flight at once, so each thread keeps NB
// independent load chains going; each root still folds its leaves in canonical order.
template <typename T, int VB, int OP, int NB, bool SM = false>
__device__ __forceinline__ void fold_many(void *root, void *leaf, const int32_t *m_leaf, int32_t lofs, int32_t nv,
                                          const Block (&b)[NB], const int32_t (&v)[NB], bool zr) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  constexpr int U = VB >= 16 ? 1 : 2;
  Pack<T, VB> x[NB];
  Pack<A, AVB> acc[NB];
  int32_t nmax = 0;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    x[j] = ld_root<T, VB>(root, int64_t(b[j].root) * nv + v[j], zr);
    nmax = b[j].n > nmax ? b[j].n : nmax;
  }
  for (int32_t e = 0; e < nmax; e += U) {
    int32_t li[NB][U];   // leaf units (< 2^31); -1 past the block's end
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int u = 0; u < U; ++u) li[j][u] = e + u < b[j].n ? ld_idx<SM>(m_leaf + (b[j].e0 - lofs) + e + u) : -1;
    Pack<T, VB> y[NB][U];
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (li[j][u] >= 0) y[j][u] = ld<T, VB>(leaf, int64_t(li[j][u]) * nv + v[j]);
#pragma unroll
    for (int j = 0; j < NB; ++j)
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (li[j][u] >= 0)
#pragma unroll
          for (int l = 0; l < Pack<T, VB>::L; ++l)
            acc[j].v[l] = (e + u == 0) ? to_acc<A, T>(y[j][u].v[l]) : combine<OP, A>(acc[j].v[l], to_acc<A, T>(y[j][u].v[l]));
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    Pack<T, VB> r = x[j];
#pragma unroll
    for (int l = 0; l < Pack<T, VB>::L; ++l) r.v[l] = apply_acc<OP, T, A>(x[j].v[l], acc[j].v[l]);
    st<T, VB>(root, int64_t(b[j].root) * nv + v[j], r);
  }
}

// NV1: the launch has one vector per unit (a.nv == 1; Reduce SUM/MIN/MAX with VB >= 4 only),
// so the multi-vector fold code is left out and the kernel fits a smaller register budget.
// ZR: a Reduce from zero (RmArgs.zero_root set; the roots count as 0 and are never read) --
// a template parameter, so the plain Reduce's unrolled root loads carry no branch.
// FLAT: units of several vectors whose chunk tiles fold by gather-then-fold (fold_tile_flat_nv);
// it reads the tiles of rm_fold_nv1_tiles, as NV1 does.
template <typename T, int VB, int OP, int MODE, bool NV1 = false, bool ZR = false, bool FLAT = false>
__device__ __forceinline__ void rm_tile(const RmArgs &a, const RmTile &t) {
  static_assert(!NV1 || (MODE == RM_REDUCE && OP != OP_REPLACE && VB >= 4), "NV1 is a Reduce-op form");
  static_assert(!ZR || (MODE == RM_REDUCE && OP != OP_REPLACE), "ZR is a Reduce-op form");
  static_assert(!FLAT || (MODE == RM_REDUCE && OP != OP_REPLACE && VB >= 4 && !NV1), "FLAT is a Reduce-op form");
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;   // accumulator pack bytes
  constexpr int U = VB >= 16 ? 2 : 4;
  const int32_t nv = NV1 ? 1 : a.nv;
  const int32_t work = t.cnt * nv;
  if (t.kind == T_MASKED && nv == 1) {
    // Scalar units: root, leaf and mask word of an edge are independent loads (every unit in
    // the run's span is valid memory; only the store waits for the mask bit), 8 edges in
    // flight per thread for copies, 4 for ops (whose kernels run 4 CTAs per SM), 32-bit
    // offsets from the tile's base pointers.
    constexpr int UM = VB >= 16 ? 4 : (OP == OP_REPLACE ? 8 : 4);
    constexpr bool need_root = SingleReads<OP, MODE>::root, need_leaf = SingleReads<OP, MODE>::leaf;
    T *rbase = static_cast<T *>(a.root) + (t.root0 + t.k0) * Pack<T, VB>::L;
    T *lbase = static_cast<T *>(a.leaf) + (t.leaf0 + t.k0) * Pack<T, VB>::L;
    T *ubase = MODE == RM_FETCH ? static_cast<T *>(a.upd) + (t.leaf0 + t.k0) * Pack<T, VB>::L : nullptr;
    const uint32_t *mw = a.mask + ((t.mask0 + t.k0) >> 5);   // mask0 and k0 are multiples of 32
    for (int32_t base = threadIdx.x; base < t.cnt; base += kThreads * UM) {
      uint32_t mk[UM];
      Pack<T, VB> x[UM], y[UM];
#pragma unroll
      for (int u = 0; u < UM; ++u) {
        const int32_t k = base + u * kThreads;
        mk[u] = 0;
        if (k < t.cnt) {
          mk[u] = (__ldg(mw + (k >> 5)) >> (k & 31)) & 1u;
          if constexpr (need_root) x[u] = ld_root<T, VB>(rbase, k, ZR);
          if constexpr (need_leaf) y[u] = ld<T, VB>(lbase, k);
        }
      }
#pragma unroll
      for (int u = 0; u < UM; ++u) {
        const int32_t k = base + u * kThreads;
        if (!mk[u]) continue;
        if constexpr (MODE == RM_BCAST) {
          if constexpr (OP == OP_REPLACE) st<T, VB>(lbase, k, x[u]);
          else st<T, VB>(lbase, k, combine<OP, T, VB>(y[u], x[u]));
        } else if constexpr (MODE == RM_REDUCE) {
          if constexpr (OP == OP_REPLACE) st<T, VB>(rbase, k, y[u]);
          else st<T, VB>(rbase, k, combine<OP, T, VB>(x[u], y[u]));
        } else {
          st<T, VB>(ubase, k, x[u]);
          st<T, VB>(rbase, k, combine<OP, T, VB>(x[u], y[u]));
        }
      }
    }
  } else if (t.kind == T_MASKED || t.kind == T_PAIRS) {
    const RmTile &mr = t;
    for (int32_t base = threadIdx.x; base < work; base += kThreads * U) {
      int64_t ri[U], li[U];
      bool on[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t w = base + u * kThreads;
        const int32_t kl = nv == 1 ? w : div_by(w, a.nv_m, a.nv_s), v = w - kl * nv;
        on[u] = w < work;
        int64_t ru = 0, lu = 0;
        if (on[u]) {
          if (t.kind == T_MASKED) {
            const int64_t bit = mr.mask0 + t.k0 + kl;
            on[u] = (__ldg(a.mask + (bit >> 5)) >> (bit & 31)) & 1u;
            ru = mr.root0 + t.k0 + kl;
            lu = mr.leaf0 + t.k0 + kl;
          } else {
            ru = __ldg(a.pr_root + t.a + kl);
            lu = __ldg(a.pr_leaf + t.a + kl);
          }
        }
        ri[u] = ru * nv + v;
        li[u] = lu * nv + v;
      }
      Pack<T, VB> x[U], y[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (on[u]) {
          if constexpr (SingleReads<OP, MODE>::root) x[u] = ld_root<T, VB>(a.root, ri[u], ZR);
          if constexpr (SingleReads<OP, MODE>::leaf) y[u] = ld<T, VB>(a.leaf, li[u]);
        }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (on[u]) single_store<T, VB, OP, MODE>(a, ri[u], li[u], x[u], y[u]);
    }
  } else if (t.kind == T_WINNERS) {
    if constexpr (MODE == RM_REDUCE && OP == OP_REPLACE) {
      for (int32_t w = threadIdx.x; w < work; w += kThreads) {
        const int32_t kl = div_by(w, a.nv_m, a.nv_s), v = w - kl * nv, m = t.a + kl;
        const int64_t last = a.m_leaf[a.m_ptr[m + 1] - 1];
        st<T, VB>(a.root, int64_t(a.m_root[m]) * nv + v, ld<T, VB>(a.leaf, last * nv + v));
      }
    }
  } else if (t.kind == T_FETCH) {
    if constexpr (MODE == RM_FETCH) {
      for (int32_t w = threadIdx.x; w < work; w += kThreads) {
        const int32_t kl = div_by(w, a.nv_m, a.nv_s), v = w - kl * nv, m = t.a + kl;
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
    if constexpr (MODE == RM_REDUCE && OP != OP_REPLACE) {
      // The tile's block records [a, a + cnt] and leaf entries [k0, e1) are staged in shared
      // memory by two bulk copies (spans widened to 16-byte boundaries), so each fold issues
      // only its data loads.  NB work items per thread, folded together when all are
      // single-block roots.
      constexpr int kStageLeaves = NV1 || FLAT ? RM_STAGE_LEAVES_NV1 : RM_STAGE_LEAVES;
      __shared__ alignas(16) BlockRec s_rec[RM_STAGE_RECS];
      __shared__ alignas(16) int32_t s_leaf[kStageLeaves];
      __shared__ alignas(8) uint64_t s_bar;
      const int32_t r0 = t.a & ~1, r1 = (t.a + t.cnt + 2) & ~1;
      const int32_t l0 = t.k0 & ~3, l1 = int32_t((t.e1 + 3) & ~int64_t(3));
      if (t.cnt > RM_TILE_CHUNKS || r1 - r0 > RM_STAGE_RECS || l1 - l0 > kStageLeaves) {
        // not a tile of this kernel's list (the NV1 form reads rm_fold_nv1_tiles): skip it
        if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEVSTAT_TILE_REFUSED);
        return;
      }
      const bool staged = stage2(s_rec, a.blocks + r0, uint32_t(r1 - r0) * uint32_t(sizeof(BlockRec)), s_leaf,
                                 a.m_leaf + l0, uint32_t(l1 - l0) * 4u, &s_bar, a.status);
      if constexpr (NV1 || FLAT) {   // gather-then-fold (the CTA agrees on the stage first)
        __shared__ alignas(16) unsigned char s_val[RM_FLAT_BYTES];
        if (__syncthreads_and(staged)) {
          if constexpr (NV1)
            fold_tile_flat<T, VB, OP, ZR>(a, t, s_rec, r0, s_leaf, l0, reinterpret_cast<Pack<T, VB> *>(s_val));
          else
            fold_tile_flat_nv<T, VB, OP, ZR>(a, t, s_rec, r0, s_leaf, l0, reinterpret_cast<Pack<T, VB> *>(s_val));
        }
        return;
      } else {
        if (!staged) return;
        constexpr int NB = 2;
        int32_t w = threadIdx.x;
        for (; w + (NB - 1) * kThreads < work; w += NB * kThreads) {
          Block b[NB];
          int32_t v[NB];
          bool simple = true;
  #pragma unroll
          for (int j = 0; j < NB; ++j) {
            const int32_t wj = w + j * kThreads, cj = nv == 1 ? wj : div_by(wj, a.nv_m, a.nv_s);
            v[j] = wj - cj * nv;
            b[j] = load_block(s_rec, a.combs, t.a + cj - r0);
            simple &= b[j].comb < 0;
          }
          if (simple) {
            fold_many<T, VB, OP, NB, true>(a.root, a.leaf, s_leaf, l0, nv, b, v, ZR);
          } else {
  #pragma unroll
            for (int j = 0; j < NB; ++j)
              fold_block<T, VB, OP, MODE, true>(a.root, a.leaf, s_leaf, l0, a.combs, a.partial, a.counter, nv, b[j],
                                                v[j], ZR);
          }
        }
        for (; w < work; w += kThreads) {
          const int32_t cl = nv == 1 ? w : div_by(w, a.nv_m, a.nv_s), v = w - cl * nv;
          fold_block<T, VB, OP, MODE, true>(a.root, a.leaf, s_leaf, l0, a.combs, a.partial, a.counter, nv,
                                            load_block(s_rec, a.combs, t.a + cl - r0), v, ZR);
        }
      }
    } else {
      for (int32_t w = threadIdx.x; w < work; w += kThreads) {
        const int32_t cl = nv == 1 ? w : div_by(w, a.nv_m, a.nv_s), v = w - cl * nv;
        fold_block<T, VB, OP, MODE>(a.root, a.leaf, a.m_leaf, 0, a.combs, a.partial, a.counter, nv,
                                    load_block(a.blocks, a.combs, t.a + cl), v, ZR);
      }
    }
  }
}

template <typename T, int VB, int OP, int MODE, bool NV1 = false, bool ZR = false, bool FLAT = false>
__global__ void __launch_bounds__(kThreads, (NV1 || FLAT ? RM_NV1_BLOCKS : MinBlocks<OP, VB, MODE == RM_FETCH>::value))
    rm_kernel(RmArgs a) {
  const RmTile t = a.tiles[blockIdx.x];
  rm_tile<T, VB, OP, MODE, NV1, ZR, FLAT>(a, t);
}

// ------------------------------------------------------------------ diagonal-chunk Reduce
// Deterministic Reduce (SUM/MIN/MAX) of one-vector units over the diagonal chunks (sf_plan.h):
// a warp takes 32 consecutive roots, lane l root 32 (c0 + c) + l, and U chunks at a time.  Per
// chunk the loads come in three dependent rounds, each a coalesced or broadcast access:
//   1. the 16-byte chunk record (every lane the same address) and the root vectors;
//   2. the diagonal leaves (root + delta) and, for roots with other leaves, their x entries
//      (the i-th such root of the chunk reads x[xoff + i]: a ballot and a popcount);
//   3. the other leaf of DG_PAIR roots.
// Each root then folds its leaves in canonical order (the diagonal leaf in its place) and
// stores root op= fold: with at most DG_MAX_LEAVES leaves, D is the plain left fold.  DG_LIST
// roots (three or more leaves) are rare and read their list one lane at a time.
struct DgArgs {
  const DiagChunk *chunks;
  const int32_t *x, *lists;
  int32_t c0, nchunks;   // chunk c of the plan covers root units 32 (c0 + c) .. + 31
  int32_t nroots;        // root units of the forest (a last chunk may run past them)
  int32_t ntiles;        // DG_TILE_CHUNKS chunks per tile
  int32_t zero_root;     // Reduce from zero: roots count as 0 (never read)
  void *root;
  const void *leaf;
};
constexpr int DG_WARP_CHUNKS = 4;                         // chunks per warp per tile
static_assert(DG_WARP_CHUNKS * (kThreads / 32) == DG_TILE_CHUNKS, "a tile is one chunk group per warp");
// chunks in flight per warp: four, one for 16-byte units (their packs fill 64 registers)
template <int VB> struct DgUnroll { static constexpr int value = VB >= 16 ? 1 : 4; };

// A DG_LIST root u (rare): its list at lists[o] -- header -1 - (leaves before | after << 16),
// then the other leaves -- folded with the diagonal leaf u + delta in its canonical place.
template <typename T, int VB, int OP>
__device__ __forceinline__ void dg_list_root(const DgArgs &a, int64_t u, int32_t o, int32_t delta) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  const int32_t h = -1 - __ldg(a.lists + o);
  const int32_t nb = h & 0xffff, n = nb + 1 + (h >> 16);
  Pack<A, AVB> acc;
  for (int32_t i = 0; i < n; ++i) {
    const int64_t lu = i == nb ? u + delta : int64_t(__ldg(a.lists + o + 1 + (i < nb ? i : i - 1)));
    const Pack<T, VB> y = ld<T, VB>(a.leaf, lu);
#pragma unroll
    for (int l = 0; l < Pack<T, VB>::L; ++l)
      acc.v[l] = i == 0 ? to_acc<A, T>(y.v[l]) : combine<OP, A>(acc.v[l], to_acc<A, T>(y.v[l]));
  }
  Pack<T, VB> xr = ld_root<T, VB>(a.root, u, a.zero_root);
#pragma unroll
  for (int l = 0; l < Pack<T, VB>::L; ++l) xr.v[l] = apply_acc<OP, T, A>(xr.v[l], acc.v[l]);
  st<T, VB>(a.root, u, xr);
}

template <typename T, int VB, int OP>
__device__ __forceinline__ void dg_tile(const DgArgs &a, int32_t tile) {
  using A = typename Acc<T, OP>::type;
  constexpr int AVB = int(sizeof(A)) * Pack<T, VB>::L;
  const int lane = threadIdx.x & 31;
  const uint32_t below = (1u << lane) - 1u;
  constexpr int DG_U = DgUnroll<VB>::value;
  const int32_t cw = tile * DG_TILE_CHUNKS + (threadIdx.x >> 5) * DG_WARP_CHUNKS;
  for (int32_t cb = cw; cb < cw + DG_WARP_CHUNKS && cb < a.nchunks; cb += DG_U) {
    uint32_t code[DG_U];
    int32_t xo[DG_U], dl[DG_U];
    Pack<T, VB> xr[DG_U], yd[DG_U], yo[DG_U];
#pragma unroll
    for (int j = 0; j < DG_U; ++j) {   // round 1: chunk records and roots
      code[j] = 0;
      const int32_t c = cb + j;
      if (c < a.nchunks) {
        const uint4 rec = __ldg(reinterpret_cast<const uint4 *>(a.chunks) + c);
        code[j] = ((lane < 16 ? rec.x : rec.y) >> (2 * (lane & 15))) & 3u;
        xo[j] = int32_t(rec.z);
        dl[j] = int32_t(rec.w);
        const int64_t u = int64_t(a.c0 + c) * 32 + lane;
        if (u < a.nroots) xr[j] = ld_root<T, VB>(a.root, u, a.zero_root);
      }
    }
    int32_t xe[DG_U];
#pragma unroll
    for (int j = 0; j < DG_U; ++j) {   // round 2: diagonal leaves and x entries
      const int64_t u = int64_t(a.c0 + cb + j) * 32 + lane;
      const uint32_t more = __ballot_sync(0xffffffffu, code[j] >= DG_PAIR);
      xe[j] = 0;
      if (code[j] != DG_SKIP) yd[j] = ld<T, VB>(a.leaf, u + dl[j]);
      if (code[j] >= DG_PAIR) xe[j] = __ldg(a.x + xo[j] + __popc(more & below));
    }
#pragma unroll
    for (int j = 0; j < DG_U; ++j)     // round 3: the other leaf of two-leaf roots
      if (code[j] == DG_PAIR) yo[j] = ld<T, VB>(a.leaf, xe[j] & 0x7fffffff);
#pragma unroll
    for (int j = 0; j < DG_U; ++j) {
      const int64_t u = int64_t(a.c0 + cb + j) * 32 + lane;
      if (code[j] == DG_DIAG || code[j] == DG_PAIR) {
        // canonical order: the other leaf first unless its entry has the top bit (after)
        const bool pair = code[j] == DG_PAIR, after = xe[j] < 0;
        const Pack<T, VB> &y0 = pair && !after ? yo[j] : yd[j];
        Pack<T, VB> r = xr[j];
#pragma unroll
        for (int l = 0; l < Pack<T, VB>::L; ++l) {
          A acc = to_acc<A, T>(y0.v[l]);
          if (pair) acc = combine<OP, A>(acc, to_acc<A, T>(after ? yo[j].v[l] : yd[j].v[l]));
          r.v[l] = apply_acc<OP, T, A>(xr[j].v[l], acc);
        }
        st<T, VB>(a.root, u, r);
      }
    }
    // roots of three or more leaves, after the others (their root and diagonal leaf are
    // read again, from L1 or L2, so that little stays live here)
#pragma unroll
    for (int j = 0; j < DG_U; ++j)
      if (code[j] == DG_LIST) dg_list_root<T, VB, OP>(a, int64_t(a.c0 + cb + j) * 32 + lane, xe[j], dl[j]);
  }
}

template <typename T, int VB, int OP>
__global__ void __launch_bounds__(kThreads, 4) dg_kernel(DgArgs a) {
  for (int32_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) dg_tile<T, VB, OP>(a, t);
}

// ------------------------------------------------------------------ staged diagonal-chunk Reduce
// The same Reduce as dg_kernel, for one forest, as a warp-specialised pipeline: a persistent CTA
// per SM of one producer warp and DG_CONSUMERS consumer warps loops over the plan's tiles
// (DgTile: up to 32 chunks of one delta) through DgStage<VB>::NSTAGE shared-memory stages.
//  - The producer fills a stage with up to five cp.async.bulk copies on the stage's "full"
//    mbarrier -- the roots (unless the Reduce starts from zero), the diagonal leaves (the span
//    widened to 16-byte boundaries inside the leaf array), the chunk records, the x entries and
//    the list entries -- and refills it once the consumers have released it on its "empty"
//    mbarrier.  Its warp fetches tile descriptors 32 at a time, so issuing waits on nothing.
//  - A consumer warp owns DGB_WARP_CHUNKS chunks of every tile.  Before folding tile k it issues,
//    for tile k + 1 (already landed or landing), the cp.async gathers of its roots' other leaves
//    into the stage (the only reads that depend on staged data), so their latency hides behind
//    a whole tile of work; each thread later reads only the slots it gathered itself, so no
//    CTA-wide barrier is needed.  The fold then runs from shared memory alone, and each warp
//    stores its 32 consecutive roots per chunk with coalesced global stores.
// Waits are bounded (DEVSTAT_STAGE_TIMEOUT); units outside a copied span (the ends of the
// arrays) are read and written directly.  Base pointers must be 16-byte aligned.
struct DgBulkArgs {
  DgArgs a;
  const DgTile *tiles;
  int32_t ntiles;
  int32_t *status;        // forest status word (a wait that ran out)
  int64_t root_bytes;     // bytes of the root and leaf arrays (spans are clamped inside them)
  int64_t leaf_bytes;
};

constexpr int DG_CONSUMERS = 16;                                  // consumer warps of a CTA
constexpr int DGB_WARP_CHUNKS = DG_TILE_CHUNKS / DG_CONSUMERS;    // chunks of a tile per consumer warp
constexpr int DG_BULK_THREADS = (DG_CONSUMERS + 1) * 32;
static_assert(DGB_WARP_CHUNKS * DG_CONSUMERS == DG_TILE_CHUNKS, "the consumers share a tile evenly");

// Shared-memory stage of one tile of VB-byte units: roots, diagonal leaves, chunk records, x
// entries, list entries, the gathered list leaf values and the gathered other leaves of
// two-leaf roots (one slot per x entry).  Widening a span to 16-byte boundaries adds less than
// 16 bytes at each end, so the leaf, x and list areas have 32 bytes to spare.
template <int VB> struct DgStage {
  static constexpr int R = DG_TILE_CHUNKS * 32 * VB;
  static constexpr int O_LEAF = R;
  static constexpr int O_REC = O_LEAF + R + 32;
  static constexpr int O_X = O_REC + DG_TILE_CHUNKS * 16;
  static constexpr int O_L = O_X + DG_TILE_XCAP * 4 + 32;
  static constexpr int O_LV = O_L + DG_TILE_LCAP * 4 + 32;
  static constexpr int O_PV = O_LV + DG_TILE_LCAP * VB;
  static constexpr int BYTES = (O_PV + DG_TILE_XCAP * VB + 127) / 128 * 128;
  // as many stages as fit one CTA per SM (about 200 KB), at most 8: tiles in flight keep the
  // loads of an SM deep enough to cover DRAM latency
  static constexpr int NSTAGE = (200 * 1024) / BYTES < 8 ? (200 * 1024) / BYTES : 8;
};
constexpr int DG_MAX_STAGES = 8;

// One bulk copy global -> shared on mbarrier `bar` (sizes multiples of 16, both addresses
// 16-byte aligned); the copy is counted in the barrier's expected bytes by the caller.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Wait for phase `parity` of mbarrier `bar`, the thread suspended between tries (no spinning),
// at most `limit` clock cycles; false if it did not complete.
__device__ __forceinline__ bool mbar_sleep_wait(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity), "r"(1000000u) : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// The spans a tile stages (bytes, relative to each array's base), computed once per tile by the
// producer and kept in the stage's header for the consumers.
struct DgSpans {
  int64_t u0, L0;          // first root unit, its diagonal leaf unit
  int64_t llo, lhi;        // leaf bytes [llo, lhi) staged
  int64_t xlo, lslo;       // first staged x-entry and list-entry bytes
  int32_t n;               // roots of the tile (below the forest's last root)
  int32_t rstage;          // root bytes staged, a multiple of 16
  int32_t xb, sb;          // staged x-entry and list-entry bytes (sb 0: lists read from global)
  int32_t lofs;            // stage offset of diagonal leaf 0 (fast tiles)
  int32_t fast;            // roots and diagonal leaves staged whole
  int32_t c, tn, xbeg, lbeg, full, pad;   // the tile's fields
};
template <int VB>
__device__ __forceinline__ DgSpans dg_spans(const DgBulkArgs &b, const DgTile &t) {
  DgSpans p;
  p.u0 = int64_t(b.a.c0 + t.c) * 32;
  p.n = int32_t(min(int64_t(t.n) * 32, int64_t(b.a.nroots) - p.u0));
  p.rstage = (p.n * VB) & ~15;
  p.L0 = p.u0 + t.delta;
  p.llo = max(int64_t(0), (p.L0 * VB) & ~int64_t(15));   // inside the leaf array: the tile's first
                                                            // root need not have its diagonal leaf
  p.lhi = min(((p.L0 + p.n) * VB + 15) & ~int64_t(15), b.leaf_bytes & ~int64_t(15));
  if (p.lhi < p.llo) p.lhi = p.llo;
  p.xlo = (int64_t(t.xbeg) * 4) & ~int64_t(15);
  p.xb = t.xend == t.xbeg ? 0 : int32_t(((int64_t(t.xend) * 4 + 15) & ~int64_t(15)) - p.xlo);
  p.lslo = (int64_t(t.lbeg) * 4) & ~int64_t(15);
  p.sb = t.lend == t.lbeg || t.lend - t.lbeg > DG_TILE_LCAP
             ? 0 : int32_t(((int64_t(t.lend) * 4 + 15) & ~int64_t(15)) - p.lslo);
  p.lofs = int32_t(DgStage<VB>::O_LEAF + (p.L0 * VB - p.llo));
  p.fast = p.rstage == p.n * VB && p.llo <= p.L0 * VB && p.lhi >= (p.L0 + p.n) * VB;
  p.c = t.c;
  p.tn = t.n;
  p.xbeg = t.xbeg;
  p.lbeg = t.lbeg;
  p.full = t.full;
  p.pad = 0;
  return p;
}

// Producer: the stage's header, then up to five bulk copies on its "full" mbarrier.
template <int VB>
__device__ __forceinline__ void dg_issue(const DgBulkArgs &b, unsigned char *sg, DgSpans *hdr, uint32_t bar,
                                         const DgTile &tl) {
  using S = DgStage<VB>;
  const DgSpans p = dg_spans<VB>(b, tl);
  *hdr = p;   // published to the consumers by the barrier's completion
  const uint32_t rb = b.a.zero_root ? 0u : uint32_t(p.rstage);
  const uint32_t lb = uint32_t(p.lhi - p.llo), cb = uint32_t(tl.n) * 16u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(rb + lb + cb + uint32_t(p.xb) + uint32_t(p.sb)) : "memory");
  if (rb) bulk_load(sg, static_cast<const char *>(b.a.root) + p.u0 * VB, rb, bar);
  if (lb) bulk_load(sg + S::O_LEAF, static_cast<const char *>(b.a.leaf) + p.llo, lb, bar);
  bulk_load(sg + S::O_REC, b.a.chunks + tl.c, cb, bar);
  if (p.xb) bulk_load(sg + S::O_X, reinterpret_cast<const char *>(b.a.x) + p.xlo, uint32_t(p.xb), bar);
  if (p.sb) bulk_load(sg + S::O_L, reinterpret_cast<const char *>(b.a.lists) + p.lslo, uint32_t(p.sb), bar);
}

// What a consumer lane keeps of a tile between its gathers and its fold: per chunk the root's
// code and its x entry's index relative to the tile (or -1).
struct DgLane {
  uint32_t code[DGB_WARP_CHUNKS];
  int32_t xi[DGB_WARP_CHUNKS];
};

// A consumer's gathers for a landed tile: for each of its chunks, the other leaf of every
// two-leaf root into its x entry's slot, and the list leaves of every list root into theirs
// (staged lists only), by cp.async; then one commit group.
template <int VB>
__device__ __forceinline__ DgLane dg_gather(const DgBulkArgs &b, unsigned char *sg, const DgSpans p) {
  using S = DgStage<VB>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t below = (1u << lane) - 1u;
  const int32_t *xs = reinterpret_cast<const int32_t *>(sg + S::O_X) + (p.xbeg - int32_t(p.xlo / 4));   // by tile index
  const int32_t *sl = reinterpret_cast<const int32_t *>(sg + S::O_L) - int32_t(p.lslo / 4);
  const char *leaf = static_cast<const char *>(b.a.leaf);
  DgLane d;
#pragma unroll
  for (int j = 0; j < DGB_WARP_CHUNKS; ++j) {
    const int32_t cc = warp * DGB_WARP_CHUNKS + j;
    d.code[j] = DG_SKIP;
    d.xi[j] = -1;
    if (cc >= p.tn) continue;
    const uint4 rec = *reinterpret_cast<const uint4 *>(sg + S::O_REC + cc * 16);
    const uint32_t code = ((lane >= 16 ? rec.y : rec.x) >> (2 * (lane & 15))) & 3u;
    const uint32_t more = __ballot_sync(0xffffffffu, code >= DG_PAIR);
    const int32_t xi = int32_t(rec.z) - p.xbeg + __popc(more & below);
    d.code[j] = code;
    if (code == DG_PAIR) {
      d.xi[j] = xi;
      cp_async_vec<VB>(sg + S::O_PV + xi * VB, leaf + int64_t(xs[xi] & 0x7fffffff) * VB);
    } else if (code == DG_LIST) {
      d.xi[j] = xi;
      if (p.sb) {
        const int32_t o = xs[xi], h = -1 - sl[o], n = (h & 0xffff) + (h >> 16);
        for (int32_t k = 1; k <= n; ++k)
          cp_async_vec<VB>(sg + S::O_LV + (o + k - p.lbeg) * VB, leaf + int64_t(sl[o + k]) * VB);
      }
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  return d;
}

// A consumer's fold of its chunks of a staged tile (its gathers have landed); the results of a
// full tile go back into the stage's root area, others straight to the root array.  FAST: the
// tile's roots and diagonal leaves are staged whole, so both are read at fixed offsets.
template <typename T, int VB, int OP, bool FAST>
__device__ __forceinline__ void dg_fold_stage(const DgBulkArgs &b, unsigned char *sg, const DgSpans p,
                                              const DgLane &d) {
  using A = typename Acc<T, OP>::type;
  using S = DgStage<VB>;
  using P = Pack<T, VB>;
  const DgArgs &a = b.a;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t *xs = reinterpret_cast<const int32_t *>(sg + S::O_X) + (p.xbeg - int32_t(p.xlo / 4));
  const int32_t *sl = reinterpret_cast<const int32_t *>(sg + S::O_L) - int32_t(p.lslo / 4);
  const bool zr = a.zero_root;
#pragma unroll
  for (int j = 0; j < DGB_WARP_CHUNKS; ++j) {
    const uint32_t code = d.code[j];
    if (code == DG_SKIP) continue;
    const int32_t i = (warp * DGB_WARP_CHUNKS + j) * 32 + lane;
    P xr, yd;
    if (FAST) {
      xr = zr ? ld_root<T, VB>(nullptr, 0, true) : *reinterpret_cast<const P *>(sg + i * VB);
      yd = *reinterpret_cast<const P *>(sg + p.lofs + i * VB);
    } else {
      xr = !zr && i * VB < p.rstage ? *reinterpret_cast<const P *>(sg + i * VB) : ld_root<T, VB>(a.root, p.u0 + i, zr);
      const int64_t gb = (p.L0 + i) * VB;
      yd = gb >= p.llo && gb + VB <= p.lhi ? *reinterpret_cast<const P *>(sg + S::O_LEAF + (gb - p.llo))
                                           : ld<T, VB>(a.leaf, p.L0 + i);
    }
    Pack<A, int(sizeof(A)) * P::L> acc;
    if (code == DG_DIAG) {
#pragma unroll
      for (int l = 0; l < P::L; ++l) acc.v[l] = to_acc<A, T>(yd.v[l]);
    } else if (code == DG_PAIR) {
      // canonical order: the other leaf first unless its entry has the top bit (after)
      const bool after = xs[d.xi[j]] < 0;
      const P yo = *reinterpret_cast<const P *>(sg + S::O_PV + d.xi[j] * VB);
      const P &y0 = after ? yd : yo, &y1 = after ? yo : yd;
#pragma unroll
      for (int l = 0; l < P::L; ++l) acc.v[l] = combine<OP, A>(to_acc<A, T>(y0.v[l]), to_acc<A, T>(y1.v[l]));
    } else {
      // three or more leaves: the list (header, then the other leaves) and its gathered values
      // in shared memory, or from global memory for a tile whose lists did not fit the stage
      const int32_t o = xs[d.xi[j]], h = -1 - (p.sb ? sl[o] : __ldg(a.lists + o));
      const int32_t nb = h & 0xffff, nl = nb + 1 + (h >> 16);
      for (int32_t k = 0; k < nl; ++k) {
        const int32_t ok = o + 1 + (k < nb ? k : k - 1);
        const P y = k == nb ? yd
                            : p.sb ? *reinterpret_cast<const P *>(sg + S::O_LV + (ok - p.lbeg) * VB)
                                   : ld<T, VB>(a.leaf, __ldg(a.lists + ok));
#pragma unroll
        for (int l = 0; l < P::L; ++l)
          acc.v[l] = k == 0 ? to_acc<A, T>(y.v[l]) : combine<OP, A>(acc.v[l], to_acc<A, T>(y.v[l]));
      }
    }
    P r;
#pragma unroll
    for (int l = 0; l < P::L; ++l) r.v[l] = apply_acc<OP, T, A>(xr.v[l], acc.v[l]);
    st<T, VB>(a.root, p.u0 + i, r);   // coalesced: a warp's lanes hold consecutive roots
  }
}

// A tile at an end of the root or leaf array (rare): out of line, so that the common path keeps
// its registers.
template <typename T, int VB, int OP>
__device__ __noinline__ void dg_fold_edge(const DgBulkArgs &b, unsigned char *sg, const DgSpans &p, const DgLane &d) {
  dg_fold_stage<T, VB, OP, false>(b, sg, p, d);
}

template <typename T, int VB, int OP>
__global__ void __launch_bounds__(DG_BULK_THREADS, 1) dg_bulk_kernel(DgBulkArgs b) {
  using S = DgStage<VB>;
  constexpr int DG_STAGES = S::NSTAGE;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ alignas(8) uint64_t full[DG_MAX_STAGES], empty[DG_MAX_STAGES];
  __shared__ DgSpans hdr[DG_MAX_STAGES];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < DG_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&empty[s])), "r"(DG_CONSUMERS) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int32_t G = gridDim.x;
  const int32_t nk = b.ntiles > int32_t(blockIdx.x) ? (b.ntiles - int32_t(blockIdx.x) + G - 1) / G : 0;   // tiles of this CTA
  if (warp == DG_CONSUMERS) {
    // producer: fill stage k % S with tile k once its previous tile (k - S) is folded.  The warp
    // fetches the descriptors of 32 tiles at a time, one per lane, and lane 0 takes each by
    // shuffle, so no issue waits on a descriptor load.
    int4 d0 = make_int4(0, 0, 0, 0), d1 = d0;
    bool stop = false;
    for (int32_t k = 0; k < nk; ++k) {
      if ((k & 31) == 0 && k + lane < nk) {
        const int4 *src = reinterpret_cast<const int4 *>(b.tiles + blockIdx.x + (k + lane) * G);
        d0 = __ldg(src);
        d1 = __ldg(src + 1);
      }
      const int src_lane = k & 31;
      DgTile tl;
      tl.c = __shfl_sync(0xffffffffu, d0.x, src_lane);
      tl.n = __shfl_sync(0xffffffffu, d0.y, src_lane);
      tl.delta = __shfl_sync(0xffffffffu, d0.z, src_lane);
      tl.xbeg = __shfl_sync(0xffffffffu, d0.w, src_lane);
      tl.xend = __shfl_sync(0xffffffffu, d1.x, src_lane);
      tl.full = __shfl_sync(0xffffffffu, d1.y, src_lane);
      tl.lbeg = __shfl_sync(0xffffffffu, d1.z, src_lane);
      tl.lend = __shfl_sync(0xffffffffu, d1.w, src_lane);
      const int s = k % DG_STAGES;
      if (lane == 0) {
        if (k >= DG_STAGES &&
            !mbar_sleep_wait(smem_addr(&empty[s]), uint32_t((k - DG_STAGES) / DG_STAGES) & 1u, kWaitCycles)) {
          // the consumers stopped: record it, let the loads still in flight land (bounded), stop
          if (b.status) atomicOr(b.status, DEVSTAT_STAGE_TIMEOUT);
          for (int32_t kk = k - DG_STAGES; kk < k; ++kk)
            mbar_sleep_wait(smem_addr(&full[kk % DG_STAGES]), uint32_t(kk / DG_STAGES) & 1u, kWaitCycles);
          stop = true;
        } else {
          dg_issue<VB>(b, dsm + s * S::BYTES, &hdr[s], smem_addr(&full[s]), tl);
        }
      }
      if (__shfl_sync(0xffffffffu, int(stop), 0)) break;
    }
    return;
  }
  // consumers: gathers of tile k + 1 before the fold of tile k
  auto landed = [&](int32_t k) {
    return mbar_sleep_wait(smem_addr(&full[k % DG_STAGES]), uint32_t(k / DG_STAGES) & 1u, kWaitCycles);
  };
  bool ok = nk == 0 || landed(0);
  DgLane cur{};
  if (ok && nk > 0) cur = dg_gather<VB>(b, dsm, hdr[0]);
  for (int32_t k = 0; ok && k < nk; ++k) {
    const int s = k % DG_STAGES;
    unsigned char *sg = dsm + s * S::BYTES;
    DgLane nxt{};
    if (k + 1 < nk) {
      if (!(ok = landed(k + 1))) break;
      const int sn = (k + 1) % DG_STAGES;
      nxt = dg_gather<VB>(b, dsm + sn * S::BYTES, hdr[sn]);
      asm volatile("cp.async.wait_group 1;" ::: "memory");   // tile k's gathers
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    const DgSpans p = hdr[s];   // read once: the header lives in shared memory
    if (p.fast) dg_fold_stage<T, VB, OP, true>(b, sg, p, cur);
    else dg_fold_edge<T, VB, OP>(b, sg, p, cur);
    cur = nxt;
    __syncwarp();   // every lane is done with the stage: release it
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[s])) : "memory");
  }
  if (!ok && lane == 0 && b.status) atomicOr(b.status, DEVSTAT_STAGE_TIMEOUT);
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// ------------------------------------------------------------------ roots without leaves
// Zero the listed units (roots without leaves, for the operations that start their roots at
// zero): `units` holds unit indices, each nv vectors of VB bytes; with `arg`, the unit's bs
// entries of arg are set to -1 as well.
template <int VB>
__global__ void __launch_bounds__(kThreads) zero_units_kernel(const int32_t *units, int32_t n, void *data, int32_t nv,
                                                              int32_t *arg, int32_t bs) {
  using R = typename Raw<VB>::type;
  const int64_t work = int64_t(n) * nv;
  for (int64_t w = blockIdx.x * int64_t(kThreads) + threadIdx.x; w < work; w += int64_t(gridDim.x) * kThreads) {
    const int64_t k = w / nv, v = w - k * nv;
    R z;
    memset(&z, 0, sizeof z);
    reinterpret_cast<R *>(data)[int64_t(units[k]) * nv + v] = z;
  }
  if (arg) {
    const int64_t na = int64_t(n) * bs;
    for (int64_t w = blockIdx.x * int64_t(kThreads) + threadIdx.x; w < na; w += int64_t(gridDim.x) * kThreads) {
      const int64_t k = w / bs;
      arg[int64_t(units[k]) * bs + (w - k * bs)] = -1;
    }
  }
}

// ------------------------------------------------------------------ MAX with location
// out[root] = max over the root's leaves (not combined with out's old value) and arg[root] =
// the leaf unit of the first leaf in canonical order that reaches it, per component; roots
// without leaves are left alone.  Ties keep the earlier leaf: strict "greater" inside a block,
// and blocks of one root are combined in block order by the last arriver.
struct MaxlocArgs {
  const uint32_t *mask;
  const int32_t *pr_root, *pr_leaf;
  const int32_t *m_leaf;
  const BlockRec *blocks;
  const Comb *combs;
  const RmTile *tiles;
  void *out;            // max values, units of bs elements
  const void *leaf;
  int32_t *arg;         // leaf unit per (root, component)
  void *partial;        // scratch values of multi-block roots
  int32_t *partial_arg; // scratch leaf units of multi-block roots
  int32_t *counter;
  int32_t bs;
  int32_t *status;      // the forest's device status word (a refused or timed-out stage)
};

template <typename T> __device__ __forceinline__ bool greater(T a, T b) { return a > b; }
template <> __device__ __forceinline__ bool greater<bf16>(bf16 a, bf16 b) {
  return __bfloat162float(a) > __bfloat162float(b);
}

// Single-leaf roots of a masked or pairs tile: the root element is its leaf's, and so is the
// location.
template <typename T> __device__ __forceinline__ void maxloc_single_tile(const MaxlocArgs &a, const RmTile &t) {
  const T *leaf = static_cast<const T *>(a.leaf);
  T *out = static_cast<T *>(a.out);
  const int32_t bs = a.bs;
  const int32_t work = t.cnt * bs;
  for (int32_t w = threadIdx.x; w < work; w += kThreads) {
    const int32_t k = w / bs, c = w - k * bs;
    int64_t ru, lu;
    if (t.kind == T_MASKED) {
      const int64_t bit = t.mask0 + t.k0 + k;
      if (!((a.mask[bit >> 5] >> (bit & 31)) & 1u)) continue;
      ru = t.root0 + t.k0 + k;
      lu = t.leaf0 + t.k0 + k;
    } else {
      ru = a.pr_root[t.a + k];
      lu = a.pr_leaf[t.a + k];
    }
    out[ru * bs + c] = leaf[lu * bs + c];
    a.arg[ru * bs + c] = int32_t(lu);
  }
}

// The general form (any unit): one thread per (block, element), walking the block's entries.
template <typename T>
__global__ void __launch_bounds__(kThreads) maxloc_kernel(MaxlocArgs a) {
  const RmTile t = a.tiles[blockIdx.x];
  const T *leaf = static_cast<const T *>(a.leaf);
  T *out = static_cast<T *>(a.out);
  const int32_t bs = a.bs;
  const int32_t work = t.cnt * bs;
  if (t.kind == T_MASKED || t.kind == T_PAIRS) {
    maxloc_single_tile<T>(a, t);
  } else if (t.kind == T_CHUNKS) {
    for (int32_t w = threadIdx.x; w < work; w += kThreads) {
      const int32_t cl = w / bs, c = w - cl * bs;
      const Block b = load_block(a.blocks, a.combs, t.a + cl);
      int32_t best_l = a.m_leaf[b.e0];
      T best = leaf[int64_t(best_l) * bs + c];
      for (int32_t e = 1; e < b.n; ++e) {
        const int32_t l = a.m_leaf[b.e0 + e];
        const T y = leaf[int64_t(l) * bs + c];
        if (greater(y, best)) { best = y; best_l = l; }
      }
      const int64_t ri = int64_t(b.root) * bs + c;
      if (b.comb < 0) {
        out[ri] = best;
        a.arg[ri] = best_l;
        continue;
      }
      const Comb cb = a.combs[b.comb];
      const int32_t ci = (b.e0 - cb.e_first) / FOLD_BLOCK;
      const int64_t slot = (int64_t(cb.slot) + ci) * bs + c;
      __stcg(static_cast<T *>(a.partial) + slot, best);
      __stcg(a.partial_arg + slot, best_l);
      __threadfence();
      int32_t *ctr = a.counter + int64_t(cb.ctr) * bs + c;
      if (atomicAdd(ctr, 1) == cb.nch - 1) {
        __threadfence();
        T v = __ldcg(static_cast<const T *>(a.partial) + int64_t(cb.slot) * bs + c);
        int32_t l = __ldcg(a.partial_arg + int64_t(cb.slot) * bs + c);
        for (int32_t i = 1; i < cb.nch; ++i) {
          const int64_t si = (int64_t(cb.slot) + i) * bs + c;
          const T y = __ldcg(static_cast<const T *>(a.partial) + si);
          if (greater(y, v)) { v = y; l = __ldcg(a.partial_arg + si); }
        }
        out[ri] = v;
        a.arg[ri] = l;
        *ctr = 0;
      }
    }
  }
}

// MAX with location, gather-then-fold (the one-vector-unit kernel's tile list and stage): a
// fold tile's records and leaf entries come into shared memory by bulk copies, and its blocks go
// in groups of (block, vector) items.  For each group the CTA copies rounds of whole leaf units
// into shared memory by cp.async; each item keeps, per element of its vector, the running
// maximum and the leaf unit of its first occurrence in canonical order (a strictly greater value
// replaces it), carried across rounds.  A single-block root takes the item's result; the blocks
// of a multi-block root leave partials (values and locations) whose last arrivers combine them
// in two levels in block order -- super-blocks of FOLD_BLOCK blocks, then the root -- with the
// same strict comparison, which keeps the earliest maximum: the serial definition's result.
// MaxlocFlat::nv vectors of VB bytes make a unit of bs elements.
struct MaxlocFlat {
  int32_t nv;
  uint32_t nv_m;   // DivMagic of nv
  int32_t nv_s;
};

template <typename T, int VB>
__device__ __forceinline__ void maxloc_store(const MaxlocArgs &a, int64_t e0, const Pack<T, VB> &v,
                                             const int32_t (&loc)[Pack<T, VB>::L]) {
  st<T, VB>(a.out, e0 / Pack<T, VB>::L, v);
#pragma unroll
  for (int l = 0; l < Pack<T, VB>::L; ++l) a.arg[e0 + l] = loc[l];
}

// Fold n partials (values and locations, stride bs elements) from slot `slot` into (v, loc)
// in order, strictly greater replacing.
template <typename T, int VB>
__device__ __forceinline__ void maxloc_fold_partials(const MaxlocArgs &a, int64_t slot, int32_t n, int32_t c0,
                                                     Pack<T, VB> &v, int32_t (&loc)[Pack<T, VB>::L]) {
  constexpr int L = Pack<T, VB>::L;
  const T *pv = static_cast<const T *>(a.partial);
  for (int32_t i = 0; i < n; ++i) {
    const int64_t e = (slot + i) * a.bs + c0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      const T y = __ldcg(pv + e + l);
      if (i == 0 || greater(y, v.v[l])) {
        v.v[l] = y;
        loc[l] = __ldcg(a.partial_arg + e + l);
      }
    }
  }
}

template <typename T, int VB>
__device__ __forceinline__ void maxloc_finish(const MaxlocArgs &a, const MaxlocFlat &f, const Block &b, int32_t vv,
                                              Pack<T, VB> v, int32_t (&loc)[Pack<T, VB>::L]) {
  constexpr int L = Pack<T, VB>::L;
  const int32_t c0 = vv * L;                                  // the vector's first element in the unit
  if (b.comb < 0) {
    maxloc_store<T, VB>(a, int64_t(b.root) * a.bs + c0, v, loc);
    return;
  }
  const Comb cb = a.combs[b.comb];
  const int32_t ci = (b.e0 - cb.e_first) / FOLD_BLOCK;       // block index in the root
  const int32_t sb = ci / FOLD_BLOCK;                         // super-block
  const int32_t nsb = (cb.nch + FOLD_BLOCK - 1) / FOLD_BLOCK;
  const int32_t in_sb = min(FOLD_BLOCK, cb.nch - sb * FOLD_BLOCK);
  T *pv = static_cast<T *>(a.partial);
  {
    const int64_t e = (int64_t(cb.slot) + ci) * a.bs + c0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      __stcg(pv + e + l, v.v[l]);
      __stcg(a.partial_arg + e + l, loc[l]);
    }
  }
  __threadfence();
  int32_t *ctr = a.counter + int64_t(cb.ctr + sb) * f.nv + vv;
  if (atomicAdd(ctr, 1) != in_sb - 1) return;
  __threadfence();
  maxloc_fold_partials<T, VB>(a, int64_t(cb.slot) + sb * FOLD_BLOCK, in_sb, c0, v, loc);
  *ctr = 0;   // ready for the next operation
  if (nsb > 1) {
    const int64_t e = (int64_t(cb.slot1) + sb) * a.bs + c0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      __stcg(pv + e + l, v.v[l]);
      __stcg(a.partial_arg + e + l, loc[l]);
    }
    __threadfence();
    int32_t *rctr = a.counter + int64_t(cb.ctr + nsb) * f.nv + vv;
    if (atomicAdd(rctr, 1) != nsb - 1) return;
    __threadfence();
    maxloc_fold_partials<T, VB>(a, cb.slot1, nsb, c0, v, loc);
    *rctr = 0;
  }
  maxloc_store<T, VB>(a, int64_t(cb.root) * a.bs + c0, v, loc);
}

template <typename T, int VB>
__global__ void __launch_bounds__(kThreads, RM_NV1_BLOCKS) maxloc_flat_kernel(MaxlocArgs a, MaxlocFlat f) {
  constexpr int L = Pack<T, VB>::L;
  const RmTile t = a.tiles[blockIdx.x];
  if (t.kind == T_MASKED || t.kind == T_PAIRS) {
    maxloc_single_tile<T>(a, t);
    return;
  }
  if (t.kind != T_CHUNKS) return;
  __shared__ alignas(16) BlockRec s_rec[RM_STAGE_RECS];
  __shared__ alignas(16) int32_t s_leaf[RM_STAGE_LEAVES_NV1];
  __shared__ alignas(16) unsigned char s_raw[RM_FLAT_BYTES];
  __shared__ alignas(8) uint64_t s_bar;
  const int32_t r0 = t.a & ~1, r1 = (t.a + t.cnt + 2) & ~1;
  const int32_t l0 = t.k0 & ~3, l1 = int32_t((t.e1 + 3) & ~int64_t(3));
  if (t.cnt > RM_TILE_CHUNKS || r1 - r0 > RM_STAGE_RECS || l1 - l0 > RM_STAGE_LEAVES_NV1) {
    if (threadIdx.x == 0 && a.status) atomicOr(a.status, DEVSTAT_TILE_REFUSED);
    return;
  }
  const bool staged = stage2(s_rec, a.blocks + r0, uint32_t(r1 - r0) * uint32_t(sizeof(BlockRec)), s_leaf,
                             a.m_leaf + l0, uint32_t(l1 - l0) * 4u, &s_bar, a.status);
  if (!__syncthreads_and(staged)) return;
  // (block, vector) items per thread: a 16-byte vector of 2-byte elements keeps eight
  // locations, so one item
  constexpr int NIT = VB >= 16 ? (L > 4 ? 1 : 2) : 4;
  constexpr int R = RM_FLAT_BYTES / VB;                  // leaf vectors per round
  const int32_t nv = f.nv;                               // 1 <= nv <= min(R, NIT * kThreads)
  const int32_t gb = NIT * kThreads / nv, rl = R / nv;   // blocks per group, leaf units per round
  const int32_t *idx = s_leaf + (t.k0 - l0);             // idx[i]: leaf unit of entry k0 + i
  const BlockRec *rec = s_rec + (t.a - r0);
  Pack<T, VB> *s_val = reinterpret_cast<Pack<T, VB> *>(s_raw);
  const char *leaf = static_cast<const char *>(a.leaf);
  for (int32_t g0 = 0; g0 < t.cnt; g0 += gb) {
    const int32_t g1 = min(t.cnt, g0 + gb), nitems = (g1 - g0) * nv;
    int32_t bw[NIT], vv[NIT];
    Pack<T, VB> best[NIT];
    int32_t loc[NIT][L];
#pragma unroll
    for (int j = 0; j < NIT; ++j) {
      const int32_t it = threadIdx.x + j * kThreads;
      bw[j] = -1;
      if (it < nitems) {
        const int32_t q = nv == 1 ? it : div_by(it, f.nv_m, f.nv_s);
        bw[j] = g0 + q;
        vv[j] = it - q * nv;
      }
    }
    const int32_t e0 = int32_t(rec[g0].e0 - t.k0), e1 = int32_t(rec[g1].e0 - t.k0);
    for (int32_t q0 = e0; q0 < e1; q0 += rl) {
      const int32_t nq = min(rl, e1 - q0), nvec = nq * nv;
      if (q0 > e0) __syncthreads();   // the previous round's vectors are folded
      for (int32_t k = threadIdx.x; k < nvec; k += kThreads) {
        const int32_t e = nv == 1 ? k : div_by(k, f.nv_m, f.nv_s), v = k - e * nv;
        cp_async_vec<VB>(s_val + k, leaf + (int64_t(idx[q0 + e]) * nv + v) * VB);
      }
      cp_async_wait_all();
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NIT; ++j) {
        if (bw[j] < 0) continue;
        const int32_t b0 = int32_t(rec[bw[j]].e0 - t.k0), b1 = int32_t(rec[bw[j] + 1].e0 - t.k0);
        const int32_t lo = max(b0, q0), hi = min(b1, q0 + nq);
        for (int32_t i = lo; i < hi; ++i) {
          const Pack<T, VB> y = s_val[(i - q0) * nv + vv[j]];
          const int32_t lu = idx[i];
#pragma unroll
          for (int l = 0; l < L; ++l)
            if (i == b0 || greater(y.v[l], best[j].v[l])) {
              best[j].v[l] = y.v[l];
              loc[j][l] = lu;
            }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NIT; ++j)
      if (bw[j] >= 0) maxloc_finish<T, VB>(a, f, load_block(rec, a.combs, bw[j]), vv[j], best[j], loc[j]);
    __syncthreads();   // s_val is free for the next group
  }
}

// The gradient of MAX with location, written leaf by leaf in root-major order: every connected
// leaf l of root r gets, per element c, grad_root[r, c] if arg[r, c] == l and 0 otherwise (whole
// units, no read of the leaves, no combine across blocks).  Single-leaf roots are their leaf's
// maximum, so their leaves get grad_root[r] whole.  Leaves without a root are not written.
// nv vectors of VB bytes make a unit of bs elements; a.tiles is rm_fold_tiles.
template <typename T, int VB>
__global__ void __launch_bounds__(kThreads) maxloc_grad_kernel(MaxlocArgs a, int32_t nv, uint32_t nv_m, int32_t nv_s,
                                                               const void *grad_root, void *grad_leaf) {
  constexpr int L = Pack<T, VB>::L;
  const RmTile t = a.tiles[blockIdx.x];
  const int32_t work = t.cnt * nv;
  for (int32_t w = threadIdx.x; w < work; w += kThreads) {
    const int32_t k = nv == 1 ? w : div_by(w, nv_m, nv_s), v = w - k * nv;
    if (t.kind == T_MASKED || t.kind == T_PAIRS) {
      int64_t ru, lu;
      if (t.kind == T_MASKED) {
        const int64_t bit = t.mask0 + t.k0 + k;
        if (!((__ldg(a.mask + (bit >> 5)) >> (bit & 31)) & 1u)) continue;
        ru = t.root0 + t.k0 + k;
        lu = t.leaf0 + t.k0 + k;
      } else {
        ru = __ldg(a.pr_root + t.a + k);
        lu = __ldg(a.pr_leaf + t.a + k);
      }
      st<T, VB>(grad_leaf, lu * nv + v, ld<T, VB>(grad_root, ru * nv + v));
    } else if (t.kind == T_CHUNKS) {
      const Block b = load_block(a.blocks, a.combs, t.a + k);
      const Pack<T, VB> g = ld<T, VB>(grad_root, int64_t(b.root) * nv + v);
      int32_t loc[L];
#pragma unroll
      for (int l = 0; l < L; ++l) loc[l] = __ldg(a.arg + int64_t(b.root) * a.bs + v * L + l);
      for (int32_t e = 0; e < b.n; ++e) {
        const int32_t lu = __ldg(a.m_leaf + b.e0 + e);
        Pack<T, VB> o;
        memset(&o, 0, sizeof o);
#pragma unroll
        for (int l = 0; l < L; ++l)
          if (loc[l] == lu) o.v[l] = g.v[l];
        st<T, VB>(grad_leaf, int64_t(lu) * nv + v, o);
      }
    }
  }
}

// grad_leaf[arg[i] * bs + c] = grad_root[i] for every root element i = r * bs + c with arg >= 0
// (each leaf belongs to one root, so no two elements write the same place).
template <typename T>
__global__ void __launch_bounds__(kThreads) maxloc_scatter_kernel(const int32_t *arg, const T *grad_root,
                                                                  T *grad_leaf, int64_t n, int32_t bs) {
  for (int64_t i = blockIdx.x * int64_t(kThreads) + threadIdx.x; i < n; i += int64_t(gridDim.x) * kThreads) {
    const int32_t l = arg[i];
    if (l >= 0) grad_leaf[int64_t(l) * bs + (i % bs)] = grad_root[i];
  }
}

// ------------------------------------------------------------------ batched launches
// Many forests' operations of one kernel variant in one launch: each CTA takes one
// (operation, tile) pair and runs that forest's tile with that operation's arguments.  The
// entry points at the tile itself, so the arguments and the tile load side by side.
struct BatchTile {
  int32_t op;          // index into the operation table
  int32_t pad;         // the tile index of a diagonal-chunk operation (its `tile` is unused)
  const void *tile;    // TsTile or RmTile of that operation's forest (device address)
};

template <typename T, int VB, int OP, bool L2R, bool ATOMIC, bool FETCH>
__global__ void __launch_bounds__(kThreads, (MinBlocks<OP, VB, ATOMIC>::value))
    ts_batch_kernel(const TsArgs *ops, const BatchTile *tiles) {
  const BatchTile bt = tiles[blockIdx.x];
  const TsArgs a = ops[bt.op];
  const TsTile t = *static_cast<const TsTile *>(bt.tile);
  ts_tile<T, VB, OP, L2R, ATOMIC, FETCH>(a, t);
}

template <typename T, int VB, int OP, int MODE, bool NV1 = false, bool FLAT = false>
__global__ void __launch_bounds__(kThreads, (NV1 || FLAT ? RM_NV1_BLOCKS : MinBlocks<OP, VB, MODE == RM_FETCH>::value))
    rm_batch_kernel(const RmArgs *ops, const BatchTile *tiles) {
  const BatchTile bt = tiles[blockIdx.x];
  const RmArgs a = ops[bt.op];
  const RmTile t = *static_cast<const RmTile *>(bt.tile);
  rm_tile<T, VB, OP, MODE, NV1, false, FLAT>(a, t);
}

template <typename T, int VB, int OP>
__global__ void __launch_bounds__(kThreads, 4) dg_batch_kernel(const DgArgs *ops, const BatchTile *tiles) {
  const BatchTile bt = tiles[blockIdx.x];
  dg_tile<T, VB, OP>(ops[bt.op], bt.pad);
}

}  // namespace sfgb
