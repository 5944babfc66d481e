/* sf_oracle.c -- reference semantics of the star-forest operations, for testing only.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load this file's library.  The CUDA library never calls it, includes it or shares
 * a helper with it.  It is plain, single-threaded and slow on purpose: every operation is a
 * loop over the edges in canonical order, the definition itself.
 *
 * Model (Sec. III.A): P ranks; rank p owns nroots[p] roots and describes nleaves[p]
 * connected leaves by their local index ilocal (or 0..nleaves-1 when absent) and the root
 * address (rank, index) of each.  Buffers hold all ranks back to back, rank-major:
 *   root (p, r)  -> unit rootoff[p] + r,  rootoff[p] = sum of nroots over ranks < p
 *   leaf (q, l)  -> unit leafoff[q] + l,  leafoff[q] = sum of leaf extents over ranks < q
 * where a rank's leaf extent is max(ilocal)+1, or nleaves when ilocal is absent.  A unit
 * is bs consecutive elements of one dtype.  Edge e = (q, i) is the i-th leaf that rank q
 * describes; the canonical edge order is ascending (q, i).
 *
 * Operations (Sec. III.B):
 *   Bcast(op):   for each edge in canonical order, leaf = op(leaf, root)
 *   Reduce(op):  for each edge in canonical order, root = op(root, leaf); for a floating
 *                point SUM the leaves of one root are first combined by the blocked fold D
 *                below and then added to the root once (the paper leaves the order open)
 *   FetchAndOp:  for each edge in canonical order, leafupdate = root; root = op(root, leaf)
 * REPLACE(a,b)=b, SUM=a+b, MIN=(b<a?b:a), MAX=(a<b?b:a).  Integers wrap (two's complement).
 * bf16 values are combined in fp32 and rounded to bf16 to nearest even once per result.
 *
 * Blocked fold D(y_0..y_{n-1}) with block K: if n <= K, the left fold ((y_0+y_1)+...)+y_{n-1};
 * otherwise D applied to the list of left folds of consecutive blocks of K values.
 * Reduce SUM sets root = root + D(values of the root's leaves in canonical order).
 *
 * Compiled with -ffp-contract=off: no fused multiply-add, every sum rounded once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_INT32 = 0, O_INT64 = 1, O_FP32 = 2, O_FP64 = 3, O_BF16 = 4 };
enum { O_REPLACE = 0, O_SUM = 1, O_MIN = 2, O_MAX = 3 };

typedef struct {
  int32_t P;
  const int64_t *nroots;     /* [P] */
  const int64_t *nleaves;    /* [P] */
  const int32_t *has_ilocal; /* [P] */
  const int64_t *ilocal;     /* [E], rank-major; entries of ranks without ilocal unused */
  const int32_t *rrank;      /* [E] */
  const int64_t *rindex;     /* [E] */
} of_forest;

static size_t dsize(int dtype) {
  switch (dtype) {
    case O_INT32: case O_FP32: return 4;
    case O_INT64: case O_FP64: return 8;
    case O_BF16: return 2;
  }
  return 0;
}

/* ---- bf16: round to nearest, ties to even, from the bit patterns (IEEE definition) ---- */
static float bf16_to_f32(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
static uint16_t f32_to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu)) return (uint16_t)((u >> 16) | 0x40u); /* NaN */
  uint32_t upper = u >> 16, lower = u & 0xFFFFu;
  if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1u; /* carries into exponent */
  return (uint16_t)upper;
}

/* ---- layout and canonical edges ---- */
int64_t oracle_layout(const of_forest *f, int64_t *rootoff, int64_t *leafoff) {
  int64_t e = 0;
  rootoff[0] = 0;
  leafoff[0] = 0;
  for (int32_t p = 0; p < f->P; ++p) {
    int64_t extent;
    if (f->has_ilocal[p]) {
      int64_t mx = -1;
      for (int64_t i = 0; i < f->nleaves[p]; ++i)
        if (f->ilocal[e + i] > mx) mx = f->ilocal[e + i];
      extent = mx + 1;
    } else {
      extent = f->nleaves[p];
    }
    rootoff[p + 1] = rootoff[p] + f->nroots[p];
    leafoff[p + 1] = leafoff[p] + extent;
    e += f->nleaves[p];
  }
  return e;
}

/* global leaf unit and global root unit of every edge, canonical order */
static int64_t edges(const of_forest *f, int64_t **leafu, int64_t **rootu, int64_t *nroot_total) {
  int64_t *ro = malloc(sizeof(int64_t) * (f->P + 1)), *lo = malloc(sizeof(int64_t) * (f->P + 1));
  int64_t E = oracle_layout(f, ro, lo);
  int64_t *L = malloc(sizeof(int64_t) * (E ? E : 1)), *R = malloc(sizeof(int64_t) * (E ? E : 1));
  int64_t e = 0;
  for (int32_t q = 0; q < f->P; ++q)
    for (int64_t i = 0; i < f->nleaves[q]; ++i, ++e) {
      L[e] = lo[q] + (f->has_ilocal[q] ? f->ilocal[e] : i);
      R[e] = ro[f->rrank[e]] + f->rindex[e];
    }
  *nroot_total = ro[f->P];
  free(ro);
  free(lo);
  *leafu = L;
  *rootu = R;
  return E;
}

/* ---- elementwise op: *dst = op(*dst, *src) in the dtype ---- */
static void apply(int dtype, int op, void *dst, const void *src) {
  switch (dtype) {
    case O_INT32: {
      int32_t a, b, r;
      memcpy(&a, dst, 4);
      memcpy(&b, src, 4);
      if (op == O_REPLACE) r = b;
      else if (op == O_SUM) r = (int32_t)((uint32_t)a + (uint32_t)b);
      else if (op == O_MIN) r = b < a ? b : a;
      else r = a < b ? b : a;
      memcpy(dst, &r, 4);
      break;
    }
    case O_INT64: {
      int64_t a, b, r;
      memcpy(&a, dst, 8);
      memcpy(&b, src, 8);
      if (op == O_REPLACE) r = b;
      else if (op == O_SUM) r = (int64_t)((uint64_t)a + (uint64_t)b);
      else if (op == O_MIN) r = b < a ? b : a;
      else r = a < b ? b : a;
      memcpy(dst, &r, 8);
      break;
    }
    case O_FP32: {
      float a, b, r;
      memcpy(&a, dst, 4);
      memcpy(&b, src, 4);
      if (op == O_REPLACE) r = b;
      else if (op == O_SUM) r = a + b;
      else if (op == O_MIN) r = b < a ? b : a;
      else r = a < b ? b : a;
      memcpy(dst, &r, 4);
      break;
    }
    case O_FP64: {
      double a, b, r;
      memcpy(&a, dst, 8);
      memcpy(&b, src, 8);
      if (op == O_REPLACE) r = b;
      else if (op == O_SUM) r = a + b;
      else if (op == O_MIN) r = b < a ? b : a;
      else r = a < b ? b : a;
      memcpy(dst, &r, 8);
      break;
    }
    case O_BF16: {
      uint16_t ha, hb, hr;
      memcpy(&ha, dst, 2);
      memcpy(&hb, src, 2);
      float a = bf16_to_f32(ha), b = bf16_to_f32(hb);
      if (op == O_REPLACE) hr = hb;
      else if (op == O_SUM) hr = f32_to_bf16(a + b);
      else if (op == O_MIN) hr = b < a ? hb : ha;
      else hr = a < b ? hb : ha;
      memcpy(dst, &hr, 2);
      break;
    }
  }
}

static int valid(int dtype, int bs, int op) {
  return dsize(dtype) > 0 && bs >= 1 && op >= O_REPLACE && op <= O_MAX;
}

/* ---- Bcast: leaf = op(leaf, root), edges in canonical order ---- */
int oracle_bcast(const of_forest *f, int dtype, int bs, const void *rootdata, void *leafdata, int op) {
  if (!valid(dtype, bs, op)) return 1;
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  size_t w = dsize(dtype);
  for (int64_t e = 0; e < E; ++e)
    for (int c = 0; c < bs; ++c)
      apply(dtype, op, (char *)leafdata + (L[e] * bs + c) * w, (const char *)rootdata + (R[e] * bs + c) * w);
  free(L);
  free(R);
  return 0;
}

/* ---- blocked fold D ---- */
static double fold_d(double *y, int64_t n, int64_t K) {
  while (n > K) {
    int64_t m = 0;
    for (int64_t s = 0; s < n; s += K) {
      int64_t t_end = s + K < n ? s + K : n;
      double acc = y[s];
      for (int64_t t = s + 1; t < t_end; ++t) acc = acc + y[t];
      y[m++] = acc; /* m <= s: the block that held index m was already read */
    }
    n = m;
  }
  double acc = y[0];
  for (int64_t t = 1; t < n; ++t) acc = acc + y[t];
  return acc;
}
static float fold_f(float *y, int64_t n, int64_t K) {
  while (n > K) {
    int64_t m = 0;
    for (int64_t s = 0; s < n; s += K) {
      int64_t t_end = s + K < n ? s + K : n;
      float acc = y[s];
      for (int64_t t = s + 1; t < t_end; ++t) acc = acc + y[t];
      y[m++] = acc;
    }
    n = m;
  }
  float acc = y[0];
  for (int64_t t = 1; t < n; ++t) acc = acc + y[t];
  return acc;
}

/* edges grouped by root, canonical order inside each root (stable counting sort) */
static void by_root(int64_t E, int64_t NR, const int64_t *R, int64_t **ptr_out, int64_t **perm_out) {
  int64_t *ptr = calloc((size_t)NR + 1, sizeof(int64_t)), *perm = malloc(sizeof(int64_t) * (E ? E : 1));
  for (int64_t e = 0; e < E; ++e) ptr[R[e] + 1]++;
  for (int64_t r = 0; r < NR; ++r) ptr[r + 1] += ptr[r];
  int64_t *fill = malloc(sizeof(int64_t) * (NR ? NR : 1));
  memcpy(fill, ptr, sizeof(int64_t) * NR);
  for (int64_t e = 0; e < E; ++e) perm[fill[R[e]]++] = e;
  free(fill);
  *ptr_out = ptr;
  *perm_out = perm;
}

/* ---- Reduce: root = op(root, leaf) per edge; floating SUM = root + D(leaf values) ---- */
int oracle_reduce(const of_forest *f, int dtype, int bs, const void *leafdata, void *rootdata, int op, int64_t K) {
  if (!valid(dtype, bs, op) || K < 2) return 1;
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  size_t w = dsize(dtype);
  int fp_sum = op == O_SUM && (dtype == O_FP32 || dtype == O_FP64 || dtype == O_BF16);
  if (!fp_sum) {
    for (int64_t e = 0; e < E; ++e)
      for (int c = 0; c < bs; ++c)
        apply(dtype, op, (char *)rootdata + (R[e] * bs + c) * w, (const char *)leafdata + (L[e] * bs + c) * w);
  } else {
    int64_t *ptr, *perm;
    by_root(E, NR, R, &ptr, &perm);
    int64_t maxdeg = 0;
    for (int64_t r = 0; r < NR; ++r)
      if (ptr[r + 1] - ptr[r] > maxdeg) maxdeg = ptr[r + 1] - ptr[r];
    double *yd = malloc(sizeof(double) * (maxdeg ? maxdeg : 1));
    float *yf = malloc(sizeof(float) * (maxdeg ? maxdeg : 1));
    for (int64_t r = 0; r < NR; ++r) {
      int64_t n = ptr[r + 1] - ptr[r];
      if (n == 0) continue;
      for (int c = 0; c < bs; ++c) {
        char *dst = (char *)rootdata + (r * bs + c) * w;
        for (int64_t t = 0; t < n; ++t) {
          const char *src = (const char *)leafdata + (L[perm[ptr[r] + t]] * bs + c) * w;
          if (dtype == O_FP64) memcpy(&yd[t], src, 8);
          else if (dtype == O_FP32) memcpy(&yf[t], src, 4);
          else { uint16_t h; memcpy(&h, src, 2); yf[t] = bf16_to_f32(h); }
        }
        if (dtype == O_FP64) {
          double a, s = fold_d(yd, n, K);
          memcpy(&a, dst, 8);
          a = a + s;
          memcpy(dst, &a, 8);
        } else if (dtype == O_FP32) {
          float a, s = fold_f(yf, n, K);
          memcpy(&a, dst, 4);
          a = a + s;
          memcpy(dst, &a, 4);
        } else {
          uint16_t h;
          float s = fold_f(yf, n, K);
          memcpy(&h, dst, 2);
          h = f32_to_bf16(bf16_to_f32(h) + s);
          memcpy(dst, &h, 2);
        }
      }
    }
    free(yd);
    free(yf);
    free(ptr);
    free(perm);
  }
  free(L);
  free(R);
  return 0;
}

/* ---- FetchAndOp: leafupdate = root; root = op(root, leaf), edges in canonical order ---- */
int oracle_fetch_and_op(const of_forest *f, int dtype, int bs, void *rootdata, const void *leafdata,
                        void *leafupdate, int op) {
  if (!valid(dtype, bs, op)) return 1;
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  size_t w = dsize(dtype);
  for (int64_t e = 0; e < E; ++e)
    for (int c = 0; c < bs; ++c) {
      char *root = (char *)rootdata + (R[e] * bs + c) * w;
      memcpy((char *)leafupdate + (L[e] * bs + c) * w, root, w);
      apply(dtype, op, root, (const char *)leafdata + (L[e] * bs + c) * w);
    }
  free(L);
  free(R);
  return 0;
}

/* ---- accurate reference for stating SUM errors: r0 + sum of leaves, Neumaier-compensated
 * in double (Neumaier 1974), and |r0| + sum |leaf|, per root element ---- */
static double as_double(int dtype, const void *p) {
  switch (dtype) {
    case O_INT32: { int32_t v; memcpy(&v, p, 4); return (double)v; }
    case O_INT64: { int64_t v; memcpy(&v, p, 8); return (double)v; }
    case O_FP32: { float v; memcpy(&v, p, 4); return (double)v; }
    case O_FP64: { double v; memcpy(&v, p, 8); return v; }
    case O_BF16: { uint16_t v; memcpy(&v, p, 2); return (double)bf16_to_f32(v); }
  }
  return 0.0;
}

int oracle_sum_reference(const of_forest *f, int dtype, int bs, const void *leafdata, const void *rootdata,
                         double *sum_out, double *abs_out) {
  if (!valid(dtype, bs, O_SUM)) return 1;
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  size_t w = dsize(dtype);
  double *comp = calloc((size_t)(NR * bs ? NR * bs : 1), sizeof(double));
  for (int64_t u = 0; u < NR * bs; ++u) {
    double v = as_double(dtype, (const char *)rootdata + u * w);
    sum_out[u] = v;
    abs_out[u] = fabs(v);
  }
  for (int64_t e = 0; e < E; ++e)
    for (int c = 0; c < bs; ++c) {
      int64_t u = R[e] * bs + c;
      double y = as_double(dtype, (const char *)leafdata + (L[e] * bs + c) * w);
      double s = sum_out[u], t = s + y;
      if (fabs(s) >= fabs(y)) comp[u] += (s - t) + y;
      else comp[u] += (y - t) + s;
      sum_out[u] = t;
      abs_out[u] += fabs(y);
    }
  for (int64_t u = 0; u < NR * bs; ++u) sum_out[u] += comp[u];
  free(comp);
  free(L);
  free(R);
  return 0;
}

/* a < b in the dtype (no NaN) */
static int less_than(int dtype, const void *a, const void *b) {
  switch (dtype) {
    case O_INT32: { int32_t x, y; memcpy(&x, a, 4); memcpy(&y, b, 4); return x < y; }
    case O_INT64: { int64_t x, y; memcpy(&x, a, 8); memcpy(&y, b, 8); return x < y; }
    case O_FP32: { float x, y; memcpy(&x, a, 4); memcpy(&y, b, 4); return x < y; }
    case O_FP64: { double x, y; memcpy(&x, a, 8); memcpy(&y, b, 8); return x < y; }
    case O_BF16: { uint16_t x, y; memcpy(&x, a, 2); memcpy(&y, b, 2); return bf16_to_f32(x) < bf16_to_f32(y); }
  }
  return 0;
}

/* ---- functional MAX with location: out = max over the root's leaves (0 for a root with
 * no leaves); argedge = canonical id of the first edge reaching it (-1 when none) ---- */
int oracle_reduce_maxloc(const of_forest *f, int dtype, int bs, const void *leafdata, void *out,
                         int64_t *argedge) {
  if (!valid(dtype, bs, O_MAX)) return 1;
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  size_t w = dsize(dtype);
  memset(out, 0, (size_t)(NR * bs) * w);
  for (int64_t u = 0; u < NR * bs; ++u) argedge[u] = -1;
  for (int64_t e = 0; e < E; ++e)
    for (int c = 0; c < bs; ++c) {
      int64_t u = R[e] * bs + c;
      const char *src = (const char *)leafdata + (L[e] * bs + c) * w;
      if (argedge[u] < 0 || less_than(dtype, (char *)out + u * w, src)) {
        memcpy((char *)out + u * w, src, w);
        argedge[u] = e;
      }
    }
  free(L);
  free(R);
  return 0;
}

/* ---- in-degree of every root ---- */
int oracle_in_degree(const of_forest *f, int64_t *deg) {
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  memset(deg, 0, sizeof(int64_t) * (size_t)NR);
  for (int64_t e = 0; e < E; ++e) deg[R[e]]++;
  free(L);
  free(R);
  return 0;
}

/* ---- bf16 rounding, exported so its pin can test it against an independent library ---- */
void oracle_f32_to_bf16(const float *x, uint16_t *y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = f32_to_bf16(x[i]);
}

/* ---- Gather / Scatter through the multi-forest (Sec. III.B): every root of degree d owns d
 * consecutive multi-roots, rank-major like the roots (so the multi-root of root unit u is
 * the number of edges into roots below u, plus k); the k-th leaf of a root in canonical order
 * goes to its k-th multi-root.  Gather copies leaf units into multirootdata, Scatter copies
 * them back.  nmulti receives the multi-root count (= edges). ---- */
static int64_t multi_slots(const of_forest *f, int64_t **slot_out, int64_t **leafu_out) {
  int64_t *L, *R, NR;
  int64_t E = edges(f, &L, &R, &NR);
  int64_t *first = calloc((size_t)NR + 1, sizeof(int64_t)), *slot = malloc(sizeof(int64_t) * (E ? E : 1));
  for (int64_t e = 0; e < E; ++e) first[R[e] + 1]++;
  for (int64_t r = 0; r < NR; ++r) first[r + 1] += first[r];     /* edges into roots below r */
  for (int64_t e = 0; e < E; ++e) slot[e] = first[R[e]]++;       /* canonical order inside a root */
  free(first);
  free(R);
  *slot_out = slot;
  *leafu_out = L;
  return E;
}

int oracle_gather(const of_forest *f, int dtype, int bs, const void *leafdata, void *multirootdata, int64_t *nmulti) {
  if (!valid(dtype, bs, O_REPLACE)) return 1;
  int64_t *slot, *L;
  int64_t E = multi_slots(f, &slot, &L);
  size_t unit = dsize(dtype) * (size_t)bs;
  for (int64_t e = 0; e < E; ++e)
    memcpy((char *)multirootdata + slot[e] * unit, (const char *)leafdata + L[e] * unit, unit);
  *nmulti = E;
  free(slot);
  free(L);
  return 0;
}

int oracle_scatter(const of_forest *f, int dtype, int bs, const void *multirootdata, void *leafdata) {
  if (!valid(dtype, bs, O_REPLACE)) return 1;
  int64_t *slot, *L;
  int64_t E = multi_slots(f, &slot, &L);
  size_t unit = dsize(dtype) * (size_t)bs;
  for (int64_t e = 0; e < E; ++e)
    memcpy((char *)leafdata + L[e] * unit, (const char *)multirootdata + slot[e] * unit, unit);
  free(slot);
  free(L);
  return 0;
}
