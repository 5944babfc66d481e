/* sf_cpu_parallel.c -- multi-core CPU baseline of the benchmark step, for bench.py only.
 *
 * TEST INFRASTRUCTURE, like the oracle beside it: bench.py's CPU-baseline leg times it and
 * tests/ check it against the oracle; the CUDA library never calls it.  It is not the oracle
 * (which stays single-threaded and literal) and no result of the library is checked against
 * it.  It computes the benchmark step of the SpMV scatter (Sec. IV.A) on all host cores with
 * OpenMP: Bcast REPLACE (leaf = root for every edge, leaves are unique so the edges are
 * independent) and Reduce SUM in the deterministic reading (root = root + D(values of the
 * root's leaves in canonical order), D the blocked left fold of block 64), parallel over
 * roots.  fp64 units of bs = 1.  The per-root edge lists are built once (not timed).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {   /* the same forest description as the oracle's (rank-major arrays) */
  int32_t P;
  const int64_t *nroots, *nleaves;
  const int32_t *has_ilocal;
  const int64_t *ilocal;
  const int32_t *rrank;
  const int64_t *rindex;
} cp_forest;

typedef struct {
  int64_t E, NR;
  int64_t *leafu, *rootu;   /* [E], canonical order */
  int64_t *ptr;             /* [NR + 1]: edges of root r are by_root[ptr[r] .. ptr[r+1]) */
  int64_t *by_root;         /* leaf units grouped by root, canonical order inside */
} cp_plan;

cp_plan *cp_plan_create(const cp_forest *f) {
  cp_plan *p = calloc(1, sizeof(cp_plan));
  int64_t *ro = malloc(sizeof(int64_t) * (f->P + 1)), *lo = malloc(sizeof(int64_t) * (f->P + 1));
  ro[0] = lo[0] = 0;
  int64_t e = 0;
  for (int32_t q = 0; q < f->P; ++q) {
    int64_t ext = f->nleaves[q];
    if (f->has_ilocal[q]) {
      int64_t mx = -1;
      for (int64_t i = 0; i < f->nleaves[q]; ++i)
        if (f->ilocal[e + i] > mx) mx = f->ilocal[e + i];
      ext = mx + 1;
    }
    ro[q + 1] = ro[q] + f->nroots[q];
    lo[q + 1] = lo[q] + ext;
    e += f->nleaves[q];
  }
  p->E = e;
  p->NR = ro[f->P];
  p->leafu = malloc(sizeof(int64_t) * (e ? e : 1));
  p->rootu = malloc(sizeof(int64_t) * (e ? e : 1));
  e = 0;
  for (int32_t q = 0; q < f->P; ++q)
    for (int64_t i = 0; i < f->nleaves[q]; ++i, ++e) {
      p->leafu[e] = lo[q] + (f->has_ilocal[q] ? f->ilocal[e] : i);
      p->rootu[e] = ro[f->rrank[e]] + f->rindex[e];
    }
  p->ptr = calloc((size_t)p->NR + 1, sizeof(int64_t));
  p->by_root = malloc(sizeof(int64_t) * (p->E ? p->E : 1));
  for (int64_t k = 0; k < p->E; ++k) p->ptr[p->rootu[k] + 1]++;
  for (int64_t r = 0; r < p->NR; ++r) p->ptr[r + 1] += p->ptr[r];
  int64_t *fill = malloc(sizeof(int64_t) * (p->NR ? p->NR : 1));
  memcpy(fill, p->ptr, sizeof(int64_t) * p->NR);
  for (int64_t k = 0; k < p->E; ++k) p->by_root[fill[p->rootu[k]]++] = p->leafu[k];
  free(fill);
  free(ro);
  free(lo);
  return p;
}

void cp_plan_destroy(cp_plan *p) {
  if (!p) return;
  free(p->leafu);
  free(p->rootu);
  free(p->ptr);
  free(p->by_root);
  free(p);
}

int cp_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void cp_bcast_replace_f64(const cp_plan *p, const double *root, double *leaf) {
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < p->E; ++e) leaf[p->leafu[e]] = root[p->rootu[e]];
}

/* left fold of y[0..n) */
static double lfold(const double *y, int64_t n) {
  double a = y[0];
  for (int64_t t = 1; t < n; ++t) a = a + y[t];
  return a;
}

void cp_reduce_sum_f64(const cp_plan *p, const double *leaf, double *root) {
#pragma omp parallel
  {
    double buf[64];
    double *big = NULL;
    int64_t big_n = 0;
#pragma omp for schedule(dynamic, 4096)
    for (int64_t r = 0; r < p->NR; ++r) {
      const int64_t n = p->ptr[r + 1] - p->ptr[r];
      if (n == 0) continue;
      const int64_t *ls = p->by_root + p->ptr[r];
      double s;
      if (n <= 64) {
        for (int64_t t = 0; t < n; ++t) buf[t] = leaf[ls[t]];
        s = lfold(buf, n);
      } else {   /* D: fold blocks of 64, then D of the block folds */
        if (big_n < n) {
          free(big);
          big = malloc(sizeof(double) * (size_t)n);
          big_n = n;
        }
        for (int64_t t = 0; t < n; ++t) big[t] = leaf[ls[t]];
        int64_t m = n;
        while (m > 64) {
          int64_t k = 0;
          for (int64_t s0 = 0; s0 < m; s0 += 64) big[k++] = lfold(big + s0, s0 + 64 < m ? 64 : m - s0);
          m = k;
        }
        s = lfold(big, m);
      }
      root[r] = root[r] + s;
    }
    free(big);
  }
}
