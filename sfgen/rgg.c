/* Input generator for the unstructured SpMV-style scatter workload (Sec. IV.A shape).
 *
 * N points uniform in the unit torus; random geometric graph with radius r chosen so the
 * expected degree is `deg` (4/3 pi r^3 N = deg); recursive coordinate bisection at the
 * median along the longest axis of each part's bounding box, `levels` times, giving
 * P = 2^levels ranks of N/P points; points renumbered rank-major and, inside a rank, by
 * (cell z, cell y, cell x, original id).  For each rank p the leaves are its owned
 * entries 0..n_p-1 pointing at (p, i), followed by its ghost columns (distinct neighbours
 * owned by other ranks) in increasing global column order, like PETSc's lvec.
 *
 * This file draws points and builds a graph; it computes no star-forest operation.
 * Built with -ffp-contract=off so the graph is the same on every host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t P, N, E, G;   /* ranks, points (roots), edges (leaves), ghost leaves */
  int64_t *nleaves;     /* [P] */
  int32_t *rrank;       /* [E] root rank per leaf, rank-major */
  int64_t *rindex;      /* [E] root local index per leaf */
  double r;             /* radius */
  int64_t ncell;        /* cells per dimension */
  double deg_sample;    /* mean degree over a sample of points */
} rgg_result;

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline uint64_t salt(uint64_t seed, uint64_t tag) {
  return seed ^ mix64(tag ^ 0xD1B54A32D192ED03ULL);
}
static inline double unif(uint64_t base, uint64_t i) {
  return (double)(mix64(base + 0x9E3779B97F4A7C15ULL * (i + 1)) >> 11) * (1.0 / 9007199254740992.0);
}

static double cube_root(double c) { /* Newton on x^3 = c, IEEE +,*,/ only */
  double x = 0.01;
  for (int it = 0; it < 200; ++it) x = (2.0 * x + c / (x * x)) / 3.0;
  return x;
}

static const double *g_coord[3];

/* strict weak order on (coordinate along axis, id) */
static inline int less_on(int axis, int64_t a, int64_t b) {
  double ca = g_coord[axis][a], cb = g_coord[axis][b];
  return (ca < cb) || (ca == cb && a < b);
}

/* place the k-th smallest of v[0..n) (by less_on) at v[k], smaller ones before it */
static void select_kth(int64_t *v, int64_t n, int64_t k, int axis) {
  int64_t lo = 0, hi = n - 1;
  while (hi > lo) {
    int64_t mid = lo + (hi - lo) / 2;
    /* median of three by position as pivot */
    int64_t a = v[lo], b = v[mid], c = v[hi], piv;
    if (less_on(axis, a, b)) {
      if (less_on(axis, b, c)) piv = b; else if (less_on(axis, a, c)) piv = c; else piv = a;
    } else {
      if (less_on(axis, a, c)) piv = a; else if (less_on(axis, b, c)) piv = c; else piv = b;
    }
    int64_t i = lo, j = hi;
    while (i <= j) {
      while (less_on(axis, v[i], piv)) ++i;
      while (less_on(axis, piv, v[j])) --j;
      if (i <= j) { int64_t t = v[i]; v[i] = v[j]; v[j] = t; ++i; --j; }
    }
    if (k <= j) hi = j; else if (k >= i) lo = i; else return;
  }
}

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

static inline double tdist(double a, double b) {
  double d = a > b ? a - b : b - a;
  return d > 0.5 ? 1.0 - d : d;
}

void rgg_free(rgg_result *res) {
  if (!res) return;
  free(res->nleaves); free(res->rrank); free(res->rindex); free(res);
}

rgg_result *rgg_generate(int64_t N, int32_t levels, double deg, uint64_t seed) {
  const int64_t P = (int64_t)1 << levels;
  if (N <= 0 || N % P != 0) return NULL;
  const int64_t np = N / P;
  double *x = malloc(sizeof(double) * N * 3);
  if (!x) return NULL;
  double *cx[3] = {x, x + N, x + 2 * N};
  for (int d = 0; d < 3; ++d) {
    uint64_t base = salt(seed, (uint64_t)(d + 1));
    for (int64_t i = 0; i < N; ++i) cx[d][i] = unif(base, (uint64_t)i);
  }
  const double pi = 3.141592653589793;
  const double r = cube_root(3.0 * deg / (4.0 * pi * (double)N));
  const double r2 = r * r;
  int64_t nc = (int64_t)(1.0 / r);
  if (nc < 3) nc = 1;
  const int64_t ncell = nc * nc * nc;

  /* cell lists (counting sort, stable in id) */
  int32_t *cell = malloc(sizeof(int32_t) * N);
  int64_t *cstart = calloc((size_t)ncell + 1, sizeof(int64_t));
  int64_t *cpts = malloc(sizeof(int64_t) * N);
  for (int64_t i = 0; i < N; ++i) {
    int64_t a = (int64_t)(cx[0][i] * (double)nc), b = (int64_t)(cx[1][i] * (double)nc),
            c = (int64_t)(cx[2][i] * (double)nc);
    if (a >= nc) a = nc - 1;
    if (b >= nc) b = nc - 1;
    if (c >= nc) c = nc - 1;
    cell[i] = (int32_t)((c * nc + b) * nc + a);
    cstart[cell[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, cstart, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < N; ++i) cpts[fill[cell[i]]++] = i;
    free(fill);
  }

  /* recursive coordinate bisection */
  int64_t *perm = malloc(sizeof(int64_t) * N);
  double *box = malloc(sizeof(double) * 6 * P); /* per part: lo[3], hi[3] */
  for (int64_t i = 0; i < N; ++i) perm[i] = i;
  g_coord[0] = cx[0]; g_coord[1] = cx[1]; g_coord[2] = cx[2];
  for (int d = 0; d < 3; ++d) { box[d] = 0.0; box[3 + d] = 1.0; }
  for (int lev = 0; lev < levels; ++lev) {
    int64_t parts = (int64_t)1 << lev, psize = N / parts;
    for (int64_t q = parts - 1; q >= 0; --q) { /* children 2q, 2q+1 from parent q */
      int64_t *v = perm + q * psize;
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int64_t t = 0; t < psize; ++t)
        for (int d = 0; d < 3; ++d) {
          double c = cx[d][v[t]];
          if (c < lo[d]) lo[d] = c;
          if (c > hi[d]) hi[d] = c;
        }
      int axis = 0;
      for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
      int64_t k = psize / 2;
      select_kth(v, psize, k, axis);
      double split = cx[axis][v[k]];
      double pb[6];
      memcpy(pb, box + 6 * q, sizeof(pb));
      memcpy(box + 6 * (2 * q), pb, sizeof(pb));
      memcpy(box + 6 * (2 * q + 1), pb, sizeof(pb));
      box[6 * (2 * q) + 3 + axis] = split;
      box[6 * (2 * q + 1) + axis] = split;
    }
  }
  uint32_t *part = malloc(sizeof(uint32_t) * N);
  for (int64_t p = 0; p < P; ++p)
    for (int64_t t = 0; t < np; ++t) part[perm[p * np + t]] = (uint32_t)p;

  /* renumber: rank-major, by (cell, id) inside a rank */
  int64_t *newid = malloc(sizeof(int64_t) * N), *oldof = perm; /* reuse perm as inverse */
  {
    int64_t *cnt = calloc((size_t)P, sizeof(int64_t));
    for (int64_t t = 0; t < N; ++t) {
      int64_t i = cpts[t];
      int64_t p = part[i];
      newid[i] = p * np + cnt[p]++;
    }
    free(cnt);
    for (int64_t i = 0; i < N; ++i) oldof[newid[i]] = i;
  }

  /* ghost columns per rank */
  int32_t *stamp = malloc(sizeof(int32_t) * N);
  for (int64_t i = 0; i < N; ++i) stamp[i] = -1;
  int64_t gcap = N / 4 + 1024, G = 0;
  int64_t *gcol = malloc(sizeof(int64_t) * gcap); /* global new ids, rank-major lists */
  int64_t *goff = calloc((size_t)P + 1, sizeof(int64_t));
  for (int64_t p = 0; p < P; ++p) {
    const double *bx = box + 6 * p;
    int64_t g0 = G;
    for (int64_t t = 0; t < np; ++t) {
      int64_t i = oldof[p * np + t];
      int interior = 1;
      for (int d = 0; d < 3; ++d)
        if (cx[d][i] - bx[d] < r || bx[3 + d] - cx[d][i] < r) interior = 0;
      if (interior) continue;
      int64_t ci = cell[i], a = ci % nc, b = (ci / nc) % nc, c = ci / (nc * nc);
      int span = nc >= 3 ? 1 : 0;
      for (int dz = -span; dz <= span; ++dz)
        for (int dy = -span; dy <= span; ++dy)
          for (int dx = -span; dx <= span; ++dx) {
            int64_t aa = (a + dx + nc) % nc, bb = (b + dy + nc) % nc, cc = (c + dz + nc) % nc;
            int64_t cl = (cc * nc + bb) * nc + aa;
            for (int64_t s = cstart[cl]; s < cstart[cl + 1]; ++s) {
              int64_t j = cpts[s];
              if (j == i || part[j] == (uint32_t)p || stamp[j] == (int32_t)p) continue;
              double ddx = tdist(cx[0][i], cx[0][j]), ddy = tdist(cx[1][i], cx[1][j]),
                     ddz = tdist(cx[2][i], cx[2][j]);
              double d2 = ddx * ddx + ddy * ddy + ddz * ddz;
              if (d2 < r2) {
                stamp[j] = (int32_t)p;
                if (G == gcap) { gcap *= 2; gcol = realloc(gcol, sizeof(int64_t) * gcap); }
                gcol[G++] = newid[j];
              }
            }
          }
    }
    qsort(gcol + g0, (size_t)(G - g0), sizeof(int64_t), cmp_i64);
    goff[p + 1] = G;
  }

  /* mean degree over a sample of points */
  int64_t ns = N < 65536 ? N : 65536, dsum = 0;
  for (int64_t i = 0; i < ns; ++i) {
    int64_t ci = cell[i], a = ci % nc, b = (ci / nc) % nc, c = ci / (nc * nc);
    int span = nc >= 3 ? 1 : 0;
    for (int dz = -span; dz <= span; ++dz)
      for (int dy = -span; dy <= span; ++dy)
        for (int dx = -span; dx <= span; ++dx) {
          int64_t aa = (a + dx + nc) % nc, bb = (b + dy + nc) % nc, cc = (c + dz + nc) % nc;
          int64_t cl = (cc * nc + bb) * nc + aa;
          for (int64_t s = cstart[cl]; s < cstart[cl + 1]; ++s) {
            int64_t j = cpts[s];
            if (j == i) continue;
            double ddx = tdist(cx[0][i], cx[0][j]), ddy = tdist(cx[1][i], cx[1][j]),
                   ddz = tdist(cx[2][i], cx[2][j]);
            if (ddx * ddx + ddy * ddy + ddz * ddz < r2) dsum++;
          }
        }
  }

  rgg_result *res = calloc(1, sizeof(rgg_result));
  res->P = P; res->N = N; res->G = G; res->E = N + G; res->r = r; res->ncell = nc;
  res->deg_sample = (double)dsum / (double)ns;
  res->nleaves = malloc(sizeof(int64_t) * P);
  res->rrank = malloc(sizeof(int32_t) * (size_t)res->E);
  res->rindex = malloc(sizeof(int64_t) * (size_t)res->E);
  int64_t e = 0;
  for (int64_t p = 0; p < P; ++p) {
    res->nleaves[p] = np + (goff[p + 1] - goff[p]);
    for (int64_t t = 0; t < np; ++t, ++e) { res->rrank[e] = (int32_t)p; res->rindex[e] = t; }
    for (int64_t s = goff[p]; s < goff[p + 1]; ++s, ++e) {
      int64_t gid = gcol[s];
      res->rrank[e] = (int32_t)(gid / np);
      res->rindex[e] = gid % np;
    }
  }
  free(x); free(cell); free(cstart); free(cpts); free(perm); free(box); free(part);
  free(newid); free(stamp); free(gcol); free(goff);
  return res;
}
