/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Shared helpers of the oracle's C files (neighbour search, switch function).
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load the
 * oracle; the GPU library never includes or links anything from here.
 *
 * Compile with -ffp-contract=off: distance comparisons that decide which
 * neighbours are kept must be plain IEEE products and sums.
 */
#ifndef ORACLE_COMMON_H
#define ORACLE_COMMON_H

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* One neighbour of a centre atom: atom index j, periodic image n (in box
 * lengths), separation r = (w_j - w_i) + n*L with w the wrapped positions,
 * and its squared length. */
typedef struct {
  int j;
  int n[3];
  double r[3];
  double d2;
} onbr;

/* Wrapped position w = x - L*floor(x/L), one product and one difference. */
static inline double owrap(double x, double L) {
  double f = floor(x / L);
  double p = L * f;
  return x - p;
}

/* Neighbour order: squared distance, then atom index, then image (x, y, z). */
static int onbr_cmp(const void* pa, const void* pb) {
  const onbr* a = (const onbr*)pa;
  const onbr* b = (const onbr*)pb;
  if (a->d2 < b->d2) return -1;
  if (a->d2 > b->d2) return 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  for (int k = 0; k < 3; ++k)
    if (a->n[k] != b->n[k]) return a->n[k] < b->n[k] ? -1 : 1;
  return 0;
}

/* Separation vector and squared length for image n of atom j seen from i. */
static inline void osep(const double* wi, const double* wj, const int* n, const double* L,
                        double* r, double* d2) {
  for (int a = 0; a < 3; ++a) {
    double t = wj[a] - wi[a];
    double u = (double)n[a] * L[a];
    r[a] = t + u;
  }
  double xx = r[0] * r[0];
  double yy = r[1] * r[1];
  double zz = r[2] * r[2];
  *d2 = (xx + yy) + zz;
}

/* Every (j, n) with 0 < |r| < rc seen from atom i (brute force over atoms and
 * images), sorted by onbr_cmp.  Returns the count; *out is malloc'ed. */
static int onbrs_brute(int i, int n, const double* w, const double* L, double rc, onbr** out) {
  int nimg[3];
  for (int a = 0; a < 3; ++a) nimg[a] = (int)ceil(rc / L[a]) + 1;
  int cap = 64, cnt = 0;
  onbr* v = (onbr*)malloc(sizeof(onbr) * cap);
  double rc2 = rc * rc;
  for (int j = 0; j < n; ++j)
    for (int nx = -nimg[0]; nx <= nimg[0]; ++nx)
      for (int ny = -nimg[1]; ny <= nimg[1]; ++ny)
        for (int nz = -nimg[2]; nz <= nimg[2]; ++nz) {
          if (j == i && nx == 0 && ny == 0 && nz == 0) continue;
          int nn[3] = {nx, ny, nz};
          double r[3], d2;
          osep(w + 3 * i, w + 3 * j, nn, L, r, &d2);
          if (!(d2 < rc2) || d2 == 0.0) continue;
          if (cnt == cap) {
            cap *= 2;
            v = (onbr*)realloc(v, sizeof(onbr) * cap);
          }
          v[cnt].j = j;
          memcpy(v[cnt].n, nn, sizeof nn);
          memcpy(v[cnt].r, r, sizeof r);
          v[cnt].d2 = d2;
          ++cnt;
        }
  qsort(v, cnt, sizeof(onbr), onbr_cmp);
  *out = v;
  return cnt;
}

/* Cell list over wrapped positions: cells of edge L/nc >= rc with nc >= 3 in
 * every direction, so each of the 27 neighbouring cells is a distinct
 * (cell, image) pair.  Returns 0 when the box is too small (caller then uses
 * brute force). */
typedef struct {
  int nc[3];
  double cs[3];
  int* start; /* ncell + 1 */
  int* idx;   /* n */
} ocells;

static int ocells_build(ocells* c, int n, const double* w, const double* L, double rc) {
  for (int a = 0; a < 3; ++a) {
    c->nc[a] = (int)floor(L[a] / rc);
    if (c->nc[a] < 3) return 0;
    c->cs[a] = L[a] / c->nc[a];
  }
  int ncell = c->nc[0] * c->nc[1] * c->nc[2];
  int* cell_of = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  c->start = (int*)calloc(ncell + 1, sizeof(int));
  c->idx = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    int k[3];
    for (int a = 0; a < 3; ++a) {
      k[a] = (int)floor(w[3 * i + a] / c->cs[a]);
      if (k[a] < 0) k[a] = 0;
      if (k[a] >= c->nc[a]) k[a] = c->nc[a] - 1;
    }
    cell_of[i] = (k[0] * c->nc[1] + k[1]) * c->nc[2] + k[2];
    c->start[cell_of[i] + 1]++;
  }
  for (int q = 0; q < ncell; ++q) c->start[q + 1] += c->start[q];
  int* fill = (int*)malloc(sizeof(int) * (ncell > 0 ? ncell : 1));
  memcpy(fill, c->start, sizeof(int) * ncell);
  for (int i = 0; i < n; ++i) c->idx[fill[cell_of[i]]++] = i;
  free(fill);
  free(cell_of);
  return 1;
}

static void ocells_free(ocells* c) {
  free(c->start);
  free(c->idx);
}

static int onbrs_cells(const ocells* c, int i, const double* w, const double* L, double rc,
                       onbr** out) {
  int k[3];
  for (int a = 0; a < 3; ++a) {
    k[a] = (int)floor(w[3 * i + a] / c->cs[a]);
    if (k[a] < 0) k[a] = 0;
    if (k[a] >= c->nc[a]) k[a] = c->nc[a] - 1;
  }
  int cap = 128, cnt = 0;
  onbr* v = (onbr*)malloc(sizeof(onbr) * cap);
  double rc2 = rc * rc;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        int q[3] = {k[0] + dx, k[1] + dy, k[2] + dz};
        int nn[3];
        for (int a = 0; a < 3; ++a) {
          nn[a] = 0;
          if (q[a] < 0) { q[a] += c->nc[a]; nn[a] = -1; }
          if (q[a] >= c->nc[a]) { q[a] -= c->nc[a]; nn[a] = 1; }
        }
        int cell = (q[0] * c->nc[1] + q[1]) * c->nc[2] + q[2];
        for (int s = c->start[cell]; s < c->start[cell + 1]; ++s) {
          int j = c->idx[s];
          if (j == i && nn[0] == 0 && nn[1] == 0 && nn[2] == 0) continue;
          double r[3], d2;
          osep(w + 3 * i, w + 3 * j, nn, L, r, &d2);
          if (!(d2 < rc2) || d2 == 0.0) continue;
          if (cnt == cap) {
            cap *= 2;
            v = (onbr*)realloc(v, sizeof(onbr) * cap);
          }
          v[cnt].j = j;
          memcpy(v[cnt].n, nn, sizeof nn);
          memcpy(v[cnt].r, r, sizeof r);
          v[cnt].d2 = d2;
          ++cnt;
        }
      }
  qsort(v, cnt, sizeof(onbr), onbr_cmp);
  *out = v;
  return cnt;
}

/* Smooth switch: 1 below rs, 0 from rc on, and between them
 * u^3 (-6u^2 + 15u - 10) + 1 with u = (r - rs)/(rc - rs); value and d/dr. */
static inline void oswitch(double r, double rs, double rc, double* sw, double* dsw) {
  if (r < rs) {
    *sw = 1.0;
    *dsw = 0.0;
  } else if (r < rc) {
    double u = (r - rs) / (rc - rs);
    double u2 = u * u, u3 = u2 * u;
    *sw = u3 * (-6.0 * u2 + 15.0 * u - 10.0) + 1.0;
    *dsw = -30.0 * u2 * (u - 1.0) * (u - 1.0) / (rc - rs);
  } else {
    *sw = 0.0;
    *dsw = 0.0;
  }
}

#endif
