/*
 * mcc_oracle.c -- CPU oracle of the multi-component unstructured-mesh
 * compressor of Gong et al. (Sec. III-IV, Algorithms 3 and 4).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, single-threaded restatement of what
 * the compressor computes, step by step, used to check the CUDA library. It
 * shares no code, header or table with the library. Build with
 * -ffp-contract=off: every floating-point expression below is evaluated
 * operation by operation in the written order, and fused multiply-adds appear
 * only where fmaf() is written out.
 *
 * Steps (the paper's notation: x on mesh vertices, x1 on grid nodes,
 * x2 = x - g(x1') residuals, tau = tau1 + tau2):
 *   plan       grid corners from the mesh bounding box (Sec. IV-C); every grid
 *              point located in a simplex (minimum simplex id wins);
 *              barycentric weights; per vertex the grid cell and local
 *              coordinates.
 *   f          x1 = barycentric interpolation of the vertex values (Sec. IV-D,
 *              "linear interpolation" operator), evaluated on the prequantised
 *              vertex codes.
 *   C(x1)      dual quantisation: q1 = round(x1 / (2 tau1)), N-D Lorenzo
 *              difference, canonical Huffman.
 *   g          bilinear / trilinear interpolation of the decompressed grid at
 *              each vertex (piecewise linear, sum |a_j| = 1, Sec. III).
 *   C(x2)      linear quantisation with bin 2 tau2 in dual form: vertex code
 *              Q = round(x / (2 tau2)), residual code q2 = Q - P with
 *              P = round(g(x1') / (2 tau2)); canonical Huffman.
 *   D          the inverse (Algorithm 4): x' = 2 tau2 (P + q2).
 * Parity pins: see the tests; every function here is pinned there.
 */
#include "mcc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define HEADER_BYTES 384u
#define MAGIC 0x3143434Du /* bytes 'M' 'C' 'C' '1' */
#define VERSION 1u
#define LAM_ONE 32768.0   /* u16 fixed point: value * 2^15 */
#define TOL64 1e-12       /* barycentric tolerance of the FP64 inside test */
#define TOL32 0.05f       /* FP32 pre-filter rejects lambda < -0.05 */
#define MARGIN32 0.01f    /* candidate range margin in grid cells */
#define BIN_SHRINK (1.0 - 1.0 / 1048576.0) /* bins are 2 tau (1 - 2^-20) */

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */
/* ------------------------------------------------------------------------ */
static int32_t wrap_sub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }
static int32_t wrap_add(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }

static void put_u32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }
static void put_u64(uint8_t *p, uint64_t v) { memcpy(p, &v, 8); }
static void put_f64(uint8_t *p, double v) { memcpy(p, &v, 8); }
static uint32_t get_u32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t get_u64(const uint8_t *p) { uint64_t v; memcpy(&v, p, 8); return v; }
static double get_f64(const uint8_t *p) { double v; memcpy(&v, p, 8); return v; }
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static double load_value(const void *x, int dtype, int64_t i) {
  return dtype == 0 ? ((const double *)x)[i] : (double)((const float *)x)[i];
}

/* ------------------------------------------------------------------------ */
/* grid (Sec. IV-C: corners from the vertices' min / max per axis)           */
/* ------------------------------------------------------------------------ */
int orc_grid_resolve(int dim, int64_t n_v, const double *coords, const int32_t n[3],
                     const double lo[3], const double hi[3], orc_grid *g) {
  if (dim != 2 && dim != 3) return ORC_ERR_INVALID_ARG;
  if (n_v <= 0 || !coords) return ORC_ERR_INVALID_ARG;
  memset(g, 0, sizeof(*g));
  g->dim = dim;
  int64_t ng = 1;
  int use_bbox = 0;
  for (int d = 0; d < dim; d++) {
    if (n[d] < 2 || n[d] > 32768) return ORC_ERR_INVALID_ARG;
    ng *= n[d];
    if (!(lo[d] < hi[d])) use_bbox = 1;
  }
  if (ng > ((int64_t)1 << 31)) return ORC_ERR_INVALID_ARG;
  double blo[3] = {0, 0, 0}, bhi[3] = {0, 0, 0};
  for (int d = 0; d < dim; d++) {
    if (use_bbox) {
      blo[d] = coords[d];
      bhi[d] = coords[d];
      for (int64_t i = 1; i < n_v; i++) {
        double c = coords[i * dim + d];
        if (c < blo[d]) blo[d] = c;
        if (c > bhi[d]) bhi[d] = c;
      }
    } else {
      blo[d] = lo[d];
      bhi[d] = hi[d];
    }
    if (!(blo[d] < bhi[d]) || !isfinite(blo[d]) || !isfinite(bhi[d])) return ORC_ERR_INVALID_ARG;
  }
  for (int d = 0; d < 3; d++) {
    if (d < dim) {
      g->n[d] = n[d];
      g->lo[d] = blo[d];
      g->h[d] = (bhi[d] - blo[d]) / (double)(n[d] - 1);
      g->inv_h[d] = 1.0 / g->h[d];
    } else {
      g->n[d] = 1;
      g->lo[d] = 0.0;
      g->h[d] = 1.0;
      g->inv_h[d] = 1.0;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* point location (plan)                                                     */
/* ------------------------------------------------------------------------ */
/* Barycentric coordinates of P in the simplex with vertices a, b, c (, d):
 * Cramer's rule on the edge vectors from a. Written once for double and once
 * for float (the pre-filter) with the identical operation order. */
#define BARY2(T, ax, ay, bx, by, cx, cy, px, py, lam, den_out)                   \
  do {                                                                           \
    T v0x = bx - ax, v0y = by - ay, v1x = cx - ax, v1y = cy - ay;                \
    T v2x = px - ax, v2y = py - ay;                                              \
    T t1 = v0x * v1y, t2 = v1x * v0y;                                            \
    T den_ = t1 - t2;                                                             \
    T nb1 = v2x * v1y, nb2 = v1x * v2y;                                          \
    T nc1 = v0x * v2y, nc2 = v2x * v0y;                                          \
    T lb = (nb1 - nb2) / den_;                                                    \
    T lc = (nc1 - nc2) / den_;                                                    \
    T la = ((T)1 - lb) - lc;                                                     \
    lam[0] = la; lam[1] = lb; lam[2] = lc;                                       \
    den_out = den_;                                                              \
  } while (0)

#define CROSS(T, ux, uy, uz, wx, wy, wz, rx, ry, rz)                             \
  do {                                                                           \
    T p1, p2;                                                                    \
    p1 = uy * wz; p2 = uz * wy; rx = p1 - p2;                                    \
    p1 = uz * wx; p2 = ux * wz; ry = p1 - p2;                                    \
    p1 = ux * wy; p2 = uy * wx; rz = p1 - p2;                                    \
  } while (0)

#define DOT(T, ux, uy, uz, wx, wy, wz, r)                                        \
  do {                                                                           \
    T q1 = ux * wx, q2 = uy * wy, q3 = uz * wz;                                  \
    r = (q1 + q2) + q3;                                                          \
  } while (0)

#define BARY3(T, A, B, Cc, Dd, P, lam, den_out)                                  \
  do {                                                                           \
    T v0x = B[0] - A[0], v0y = B[1] - A[1], v0z = B[2] - A[2];                   \
    T v1x = Cc[0] - A[0], v1y = Cc[1] - A[1], v1z = Cc[2] - A[2];                \
    T v2x = Dd[0] - A[0], v2y = Dd[1] - A[1], v2z = Dd[2] - A[2];                \
    T vpx = P[0] - A[0], vpy = P[1] - A[1], vpz = P[2] - A[2];                   \
    T cx, cy, cz, den_, nb, nc, nd;                                               \
    CROSS(T, v1x, v1y, v1z, v2x, v2y, v2z, cx, cy, cz);                          \
    DOT(T, v0x, v0y, v0z, cx, cy, cz, den_);                                      \
    DOT(T, vpx, vpy, vpz, cx, cy, cz, nb);                                       \
    CROSS(T, vpx, vpy, vpz, v2x, v2y, v2z, cx, cy, cz);                          \
    DOT(T, v0x, v0y, v0z, cx, cy, cz, nc);                                       \
    CROSS(T, v1x, v1y, v1z, vpx, vpy, vpz, cx, cy, cz);                          \
    DOT(T, v0x, v0y, v0z, cx, cy, cz, nd);                                       \
    T lb = nb / den_, lc = nc / den_, ld = nd / den_;                               \
    T la = (((T)1 - lb) - lc) - ld;                                              \
    lam[0] = la; lam[1] = lb; lam[2] = lc; lam[3] = ld;                          \
    den_out = den_;                                                               \
  } while (0)

/* FP32 coordinates relative to the grid origin: (float)(c - lo). */
static void rel32(const orc_grid *g, const double *coords, int32_t v, float out[3]) {
  for (int d = 0; d < 3; d++)
    out[d] = d < g->dim ? (float)(coords[(int64_t)v * g->dim + d] - g->lo[d]) : 0.0f;
}

int orc_point_in_simplex(const orc_grid *g, const double *coords, const int32_t *cell,
                         const int32_t idx[3], double lam[4]) {
  const int dim = g->dim;
  /* FP32 pre-filter: reject points that are clearly outside. */
  float hf[3], pf[3], vf[4][3], l32[4], den32;
  for (int d = 0; d < 3; d++) {
    hf[d] = (float)g->h[d];
    pf[d] = (float)idx[d] * hf[d];
  }
  for (int k = 0; k <= dim; k++) rel32(g, coords, cell[k], vf[k]);
  if (dim == 2) {
    BARY2(float, vf[0][0], vf[0][1], vf[1][0], vf[1][1], vf[2][0], vf[2][1], pf[0], pf[1],
          l32, den32);
    if (den32 != 0.0f && (l32[0] < -TOL32 || l32[1] < -TOL32 || l32[2] < -TOL32)) return 0;
  } else {
    BARY3(float, vf[0], vf[1], vf[2], vf[3], pf, l32, den32);
    if (den32 != 0.0f &&
        (l32[0] < -TOL32 || l32[1] < -TOL32 || l32[2] < -TOL32 || l32[3] < -TOL32))
      return 0;
  }
  /* FP64 barycentric test on the grid point lo + i h. */
  double P[3], V[4][3], den;
  for (int d = 0; d < 3; d++) {
    double ih = (double)idx[d] * g->h[d];
    P[d] = g->lo[d] + ih;
  }
  for (int k = 0; k <= dim; k++)
    for (int d = 0; d < 3; d++) V[k][d] = d < dim ? coords[(int64_t)cell[k] * dim + d] : 0.0;
  if (dim == 2) {
    BARY2(double, V[0][0], V[0][1], V[1][0], V[1][1], V[2][0], V[2][1], P[0], P[1], lam, den);
    lam[3] = 0.0;
    if (den == 0.0) return 0;
    return lam[0] >= -TOL64 && lam[1] >= -TOL64 && lam[2] >= -TOL64;
  }
  BARY3(double, V[0], V[1], V[2], V[3], P, lam, den);
  if (den == 0.0) return 0;
  return lam[0] >= -TOL64 && lam[1] >= -TOL64 && lam[2] >= -TOL64 && lam[3] >= -TOL64;
}

/* Grid-index range of a simplex's bounding box, from FP32 relative
 * coordinates with a margin of MARGIN32 cells. Returns 0 if empty. */
static int candidate_range(const orc_grid *g, const double *coords, const int32_t *cell,
                           int32_t ilo[3], int32_t ihi[3]) {
  float vf[4][3];
  for (int k = 0; k <= g->dim; k++) rel32(g, coords, cell[k], vf[k]);
  for (int d = 0; d < 3; d++) {
    if (d >= g->dim) { ilo[d] = 0; ihi[d] = 0; continue; }
    float mn = vf[0][d], mx = vf[0][d];
    for (int k = 1; k <= g->dim; k++) {
      if (vf[k][d] < mn) mn = vf[k][d];
      if (vf[k][d] > mx) mx = vf[k][d];
    }
    float hf = (float)g->h[d];
    float a = mn / hf - MARGIN32;
    float b = mx / hf + MARGIN32;
    float top = (float)(g->n[d] - 1);
    if (!(a <= top) || !(b >= 0.0f)) return 0; /* also rejects NaN */
    a = ceilf(a);
    b = floorf(b);
    if (a < 0.0f) a = 0.0f;
    if (b > top) b = top;
    if (a > b) return 0;
    ilo[d] = (int32_t)a;
    ihi[d] = (int32_t)b;
  }
  return 1;
}

int orc_locate(const orc_grid *g, int64_t n_v, const double *coords, int64_t n_c,
               const int32_t *cells, int brute, int32_t *owner) {
  const int dim = g->dim, k1 = dim + 1;
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int64_t ng = nx * ny * nz;
  for (int64_t t = 0; t < n_c * k1; t++)
    if (cells[t] < 0 || cells[t] >= n_v) return ORC_ERR_INVALID_ARG;
  for (int64_t j = 0; j < ng; j++) owner[j] = -1;
  double lam[4];
  if (brute) {
    for (int64_t j = 0; j < ng; j++) {
      int32_t idx[3] = {(int32_t)(j % nx), (int32_t)((j / nx) % ny), (int32_t)(j / (nx * ny))};
      for (int64_t t = 0; t < n_c; t++) {
        if (orc_point_in_simplex(g, coords, cells + t * k1, idx, lam)) {
          owner[j] = (int32_t)t;
          break; /* simplices are visited in increasing id: the first is the minimum */
        }
      }
    }
    return ORC_OK;
  }
  for (int64_t t = 0; t < n_c; t++) {
    int32_t ilo[3], ihi[3];
    if (!candidate_range(g, coords, cells + t * k1, ilo, ihi)) continue;
    for (int32_t z = ilo[2]; z <= ihi[2]; z++)
      for (int32_t y = ilo[1]; y <= ihi[1]; y++)
        for (int32_t x = ilo[0]; x <= ihi[0]; x++) {
          int64_t j = x + nx * (y + ny * (int64_t)z);
          if (owner[j] >= 0) continue; /* an earlier (smaller) simplex owns it */
          int32_t idx[3] = {x, y, z};
          if (orc_point_in_simplex(g, coords, cells + t * k1, idx, lam)) owner[j] = (int32_t)t;
        }
  }
  return ORC_OK;
}

static uint16_t to_u16_unit(double v) {
  /* clamp to [0, 1] and round to 2^-15 units */
  if (!(v > 0.0)) return 0;
  if (v >= 1.0) return 32768;
  return (uint16_t)rint(v * LAM_ONE);
}

int orc_plan_tables(const orc_grid *g, int64_t n_v, const double *coords, const int32_t *cells,
                    const int32_t *owner, int32_t *vid, uint16_t *lam, double *lam64,
                    uint32_t *cell, uint16_t *frac) {
  const int dim = g->dim, k1 = dim + 1;
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int64_t ng = nx * ny * nz;
  double l[4];
  for (int64_t j = 0; j < ng; j++) {
    int32_t t = owner[j];
    if (t < 0) {
      vid[j] = -1;
      for (int k = 1; k < k1; k++) vid[k * ng + j] = 0;
      for (int k = 0; k < dim; k++) lam[k * ng + j] = 0;
      if (lam64)
        for (int k = 0; k < k1; k++) lam64[k * ng + j] = 0.0;
      continue;
    }
    int32_t idx[3] = {(int32_t)(j % nx), (int32_t)((j / nx) % ny), (int32_t)(j / (nx * ny))};
    orc_point_in_simplex(g, coords, cells + (int64_t)t * k1, idx, l);
    for (int k = 0; k < k1; k++) vid[k * ng + j] = cells[(int64_t)t * k1 + k];
    for (int k = 0; k < dim; k++) lam[k * ng + j] = to_u16_unit(l[k + 1]);
    if (lam64)
      for (int k = 0; k < k1; k++) lam64[k * ng + j] = l[k];
  }
  /* per vertex: lower-corner cell index and local coordinates in the cell */
  for (int64_t i = 0; i < n_v; i++) {
    int64_t ci[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) {
      double dd = coords[i * dim + d] - g->lo[d];
      double t = dd * g->inv_h[d];
      double fl = floor(t);
      int64_t c;
      if (!(fl >= 0.0)) c = 0;
      else if (fl > (double)(g->n[d] - 2)) c = g->n[d] - 2;
      else c = (int64_t)fl;
      double f = t - (double)c;
      ci[d] = c;
      frac[(int64_t)d * n_v + i] = to_u16_unit(f);
    }
    cell[i] = (uint32_t)(ci[0] + nx * (ci[1] + ny * ci[2]));
  }
  (void)nz;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* per-field parameters (Sec. III: tau = tau1 + tau2)                        */
/* ------------------------------------------------------------------------ */
int orc_field_params(const orc_params *p, int64_t n_v, const void *x, orc_field *f) {
  memset(f, 0, sizeof(*f));
  if (n_v <= 0 || !x) return ORC_ERR_INVALID_ARG;
  if (p->dtype != 0 && p->dtype != 1) return ORC_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return ORC_ERR_INVALID_ARG;
  if (!(p->grid_fraction >= 1e-3 && p->grid_fraction <= 1.0 - 1e-3)) return ORC_ERR_INVALID_ARG;
  double lo = load_value(x, p->dtype, 0), hi = lo;
  for (int64_t i = 0; i < n_v; i++) {
    double v = load_value(x, p->dtype, i);
    if (!isfinite(v)) return ORC_ERR_INVALID_ARG;
    if (v < lo) lo = v;
    if (v > hi) hi = v;
  }
  f->lo = lo;
  f->hi = hi;
  f->M = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
  double tau = p->eb;
  if (p->eb_mode == 1 && hi > lo) tau = p->eb * (hi - lo);
  f->tau = tau;
  f->tau1 = p->grid_fraction * tau;
  f->tau2 = (1.0 - p->grid_fraction) * tau;
  if (!isfinite(tau) || !(f->tau1 >= 1e-290) || !(f->tau2 >= 1e-290)) return ORC_ERR_RANGE;
  f->s1 = (2.0 * f->tau1) * BIN_SHRINK;
  f->s2 = (2.0 * f->tau2) * BIN_SHRINK;
  if (!isfinite(f->s1) || !isfinite(f->s2)) return ORC_ERR_RANGE;
  f->inv2 = 1.0 / f->s2;
  double kd = rint(lo * f->inv2);
  double hd = rint(hi * f->inv2);
  if (!(fabs(kd) < 4611686018427387904.0) || !(fabs(hd) < 4611686018427387904.0))
    return ORC_ERR_RANGE; /* |.| < 2^62 */
  f->K = (int64_t)kd;
  f->Qhi = (int64_t)hd - f->K;
  if (f->Qhi >= ((int64_t)1 << 29)) return ORC_ERR_RANGE;
  /* outside-the-mesh grid value: zero, clamped to the field's range */
  f->fill_u = -f->K;
  if (f->fill_u < 0) f->fill_u = 0;
  if (f->fill_u > f->Qhi) f->fill_u = f->Qhi;
  /* bin-width ratios in 2^-40 fixed point, below 2^10 */
  double r21 = rint((f->s2 / f->s1) * 1099511627776.0);
  double r12 = rint((f->s1 / f->s2) * 1099511627776.0);
  if (!(r21 >= 1.0 && r21 < 1125899906842624.0) || !(r12 >= 1.0 && r12 < 1125899906842624.0))
    return ORC_ERR_INVALID_ARG;
  f->rho21_q = (int64_t)r21;
  f->rho12_q = (int64_t)r12;
  f->rho21_f = (float)f->rho21_q * 0x1p-40f;
  f->rho12_f = (float)f->rho12_q * 0x1p-40f;
  f->guard = (p->dtype == 1) || !(f->M <= f->tau2 * 268435456.0); /* 2^28 */
  return ORC_OK;
}

/* round(rho * (a + acc)) with rho = rq 2^-40: the integer part of a*rho from
 * the exact 128-bit product, the 40-bit fraction and the small FP32
 * correction acc*rho in float (one fused multiply-add, then round to even). */
#define RHO_BITS 40
static int64_t rescale(int64_t a, float acc, int64_t rq, float rf) {
  const uint64_t mask = ((uint64_t)1 << RHO_BITS) - 1;
  unsigned __int128 U = (unsigned __int128)(uint64_t)(a < 0 ? -a : a) * (uint64_t)rq;
  uint64_t q = (uint64_t)(U >> RHO_BITS), r = (uint64_t)U & mask;
  int64_t hi;
  uint64_t lo;
  if (a >= 0) { hi = (int64_t)q; lo = r; }
  else if (r == 0) { hi = -(int64_t)q; lo = 0; }
  else { hi = -(int64_t)q - 1; lo = ((uint64_t)1 << RHO_BITS) - r; }
  float base = (float)lo * 0x1p-40f;
  float t = fmaf(acc, rf, base);
  return hi + (int64_t)rintf(t);
}

/* ------------------------------------------------------------------------ */
/* Lorenzo prediction on the grid codes (zero outside the grid)              */
/* ------------------------------------------------------------------------ */
static int32_t qat(const int32_t *q, const int32_t n[3], int64_t x, int64_t y, int64_t z) {
  if (x < 0 || y < 0 || z < 0) return 0;
  return q[x + n[0] * (y + (int64_t)n[1] * z)];
}

void orc_lorenzo(int dim, const int32_t n[3], const int32_t *q, int32_t *delta) {
  for (int64_t z = 0; z < (dim == 3 ? n[2] : 1); z++)
    for (int64_t y = 0; y < n[1]; y++)
      for (int64_t x = 0; x < n[0]; x++) {
        int32_t d;
        if (dim == 2) {
          d = wrap_add(wrap_sub(wrap_sub(qat(q, n, x, y, 0), qat(q, n, x - 1, y, 0)),
                                qat(q, n, x, y - 1, 0)),
                       qat(q, n, x - 1, y - 1, 0));
        } else {
          int32_t s = qat(q, n, x, y, z);
          s = wrap_sub(s, qat(q, n, x - 1, y, z));
          s = wrap_sub(s, qat(q, n, x, y - 1, z));
          s = wrap_sub(s, qat(q, n, x, y, z - 1));
          s = wrap_add(s, qat(q, n, x - 1, y - 1, z));
          s = wrap_add(s, qat(q, n, x - 1, y, z - 1));
          s = wrap_add(s, qat(q, n, x, y - 1, z - 1));
          s = wrap_sub(s, qat(q, n, x - 1, y - 1, z - 1));
          d = s;
        }
        delta[x + n[0] * (y + (int64_t)n[1] * z)] = d;
      }
}

/* inverse: inclusive prefix sums along x, then y, then z */
void orc_lorenzo_inverse(int dim, const int32_t n[3], const int32_t *delta, int32_t *q) {
  const int64_t nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
  const int64_t ng = nx * ny * nz;
  memcpy(q, delta, (size_t)ng * sizeof(int32_t));
  for (int64_t z = 0; z < nz; z++)
    for (int64_t y = 0; y < ny; y++)
      for (int64_t x = 1; x < nx; x++) {
        int64_t j = x + nx * (y + ny * z);
        q[j] = wrap_add(q[j], q[j - 1]);
      }
  for (int64_t z = 0; z < nz; z++)
    for (int64_t y = 1; y < ny; y++)
      for (int64_t x = 0; x < nx; x++) {
        int64_t j = x + nx * (y + ny * z);
        q[j] = wrap_add(q[j], q[j - nx]);
      }
  for (int64_t z = 1; z < nz; z++)
    for (int64_t y = 0; y < ny; y++)
      for (int64_t x = 0; x < nx; x++) {
        int64_t j = x + nx * (y + ny * z);
        q[j] = wrap_add(q[j], q[j - nx * ny]);
      }
}

/* ------------------------------------------------------------------------ */
/* Huffman: two-queue construction on the sorted leaves, length limit by     */
/* halving the counts, canonical codes                                       */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t w; int32_t sym; } leaf_t;

static int leaf_cmp(const void *a, const void *b) {
  const leaf_t *x = (const leaf_t *)a, *y = (const leaf_t *)b;
  if (x->w != y->w) return x->w < y->w ? -1 : 1;
  return x->sym < y->sym ? -1 : (x->sym > y->sym);
}

int orc_huffman_lengths(const uint64_t *count, int nsym, int lmax, uint8_t *len) {
  memset(len, 0, (size_t)nsym);
  int m = 0;
  for (int s = 0; s < nsym; s++) m += count[s] != 0;
  if (m == 0) return ORC_OK;
  if (m == 1) {
    for (int s = 0; s < nsym; s++)
      if (count[s]) len[s] = 1;
    return ORC_OK;
  }
  uint64_t *c = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nsym);
  leaf_t *L = (leaf_t *)malloc(sizeof(leaf_t) * (size_t)m);
  uint64_t *Iw = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
  int32_t *parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m));
  int32_t *depth = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m));
  if (!c || !L || !Iw || !parent || !depth) {
    free(c); free(L); free(Iw); free(parent); free(depth);
    return ORC_ERR_OOM;
  }
  memcpy(c, count, sizeof(uint64_t) * (size_t)nsym);
  for (;;) {
    int k = 0;
    for (int s = 0; s < nsym; s++)
      if (c[s]) { L[k].w = c[s]; L[k].sym = s; k++; }
    qsort(L, (size_t)m, sizeof(leaf_t), leaf_cmp);
    /* node ids: leaves 0..m-1 (sorted position), internal m..2m-2 */
    int a = 0, b = 0, created = 0;
    while (created < m - 1) {
      int pick[2];
      uint64_t pw[2];
      for (int r = 0; r < 2; r++) {
        int take_leaf;
        if (a >= m) take_leaf = 0;
        else if (b >= created) take_leaf = 1;
        else take_leaf = L[a].w <= Iw[b]; /* tie: the leaf goes first */
        if (take_leaf) { pick[r] = a; pw[r] = L[a].w; a++; }
        else { pick[r] = m + b; pw[r] = Iw[b]; b++; }
      }
      Iw[created] = pw[0] + pw[1];
      parent[pick[0]] = m + created;
      parent[pick[1]] = m + created;
      created++;
    }
    int root = m + created - 1;
    depth[root] = 0;
    for (int node = root - 1; node >= 0; node--) depth[node] = depth[parent[node]] + 1;
    int maxlen = 0;
    for (int i = 0; i < m; i++)
      if (depth[i] > maxlen) maxlen = depth[i];
    if (maxlen <= lmax) {
      for (int i = 0; i < m; i++) len[L[i].sym] = (uint8_t)depth[i];
      break;
    }
    for (int s = 0; s < nsym; s++)
      if (c[s]) { c[s] >>= 1; if (c[s] == 0) c[s] = 1; }
  }
  free(c); free(L); free(Iw); free(parent); free(depth);
  return ORC_OK;
}

/* code_{k+1} = (code_k + 1) << (len_{k+1} - len_k) over symbols sorted by
 * (length, symbol); the first code is 0. */
int orc_canonical_codes(const uint8_t *len, int nsym, uint32_t *code) {
  uint32_t cur = 0;
  int prev = -1;
  for (int l = 1; l <= 32; l++)
    for (int s = 0; s < nsym; s++) {
      if (len[s] != l) continue;
      if (prev < 0) cur = 0;
      else cur = (cur + 1) << (l - prev);
      code[s] = cur;
      prev = l;
    }
  for (int s = 0; s < nsym; s++)
    if (!len[s]) code[s] = 0;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* stream layout                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
  size_t lens1, lens2, gtab1, gtab2, etab1, etab2, rtab2, ltab1, ltab2, out1, out2, raw, bits1,
      bits2, total;
} layout_t;

static int64_t ngroups(int64_t n, int C) { return n == 0 ? 0 : (n + 32 * (int64_t)C - 1) / (32 * (int64_t)C); }

/* Section order: header | code lengths 1, 2 | group word offsets 1, 2 |
 * group escape-count prefixes 1, 2 | group raw-count prefix 2 | lane bit
 * lengths 1, 2 | escape values 1, 2 (int32) | raw values (dtype) |
 * bitstream 1, 2 (u32 words). */
static void make_layout(int R1, int R2, int64_t ng1, int64_t ng2, uint64_t nout1, uint64_t nout2,
                        uint64_t nraw, size_t vsz, uint64_t words1, uint64_t words2, layout_t *L) {
  size_t o = HEADER_BYTES;
  L->lens1 = o; o += 2 * (size_t)R1;
  L->lens2 = o; o += 2 * (size_t)R2;
  o = align_up(o, 4);
  L->gtab1 = o; o += 4 * (size_t)(ng1 + 1);
  L->gtab2 = o; o += 4 * (size_t)(ng2 + 1);
  L->etab1 = o; o += 4 * (size_t)(ng1 + 1);
  L->etab2 = o; o += 4 * (size_t)(ng2 + 1);
  L->rtab2 = o; o += 4 * (size_t)(ng2 + 1);
  L->ltab1 = o; o += 64 * (size_t)ng1;
  L->ltab2 = o; o += 64 * (size_t)ng2;
  L->out1 = o; o += 4 * (size_t)nout1;
  L->out2 = o; o += 4 * (size_t)nout2;
  o = align_up(o, 8);
  L->raw = o; o += vsz * (size_t)nraw;
  o = align_up(o, 4);
  L->bits1 = o; o += 4 * (size_t)words1;
  L->bits2 = o; o += 4 * (size_t)words2;
  L->total = o;
}

static int check_params(const orc_params *p) {
  if (p->R1 < 4 || p->R1 > 32768 || p->R2 < 4 || p->R2 > 32768) return ORC_ERR_INVALID_ARG;
  if (p->C1 < 1 || p->C1 > 2048 || p->C2 < 1 || p->C2 > 2048) return ORC_ERR_INVALID_ARG;
  if (p->lmax < 1 || p->lmax > 24) return ORC_ERR_INVALID_ARG;
  return ORC_OK;
}

size_t orc_compress_bound(const orc_grid *g, int64_t n_v, const orc_params *p) {
  int64_t ng = (int64_t)g->n[0] * g->n[1] * g->n[2];
  size_t vsz = p->dtype == 0 ? 8 : 4;
  int64_t g1 = ngroups(ng, p->C1), g2 = ngroups(n_v, p->C2);
  uint64_t w1 = (uint64_t)((ng * p->lmax + 31) / 32 + g1);
  uint64_t w2 = (uint64_t)((n_v * p->lmax + 31) / 32 + g2);
  layout_t L;
  make_layout(p->R1, p->R2, g1, g2, (uint64_t)ng, 0, (uint64_t)n_v, vsz, w1, w2, &L);
  return L.total + 16;
}

/* Pack one component: symbols in lane-chunk order. Lane l of group g owns the
 * symbols g*32C + 32k + l (k = 0..C-1); each lane's codes are concatenated
 * MSB-first, the 32 lanes of a group follow each other without gaps, and
 * each group starts on a 32-bit word. Bit b of a group is bit 31 - b%32 of
 * its word b/32. Writes gtab (word offsets) and ltab (lane bit lengths). */
static uint64_t pack_component(const uint16_t *sym, int64_t n, int C, const uint8_t *len,
                               const uint32_t *code, uint32_t *gtab, uint16_t *ltab,
                               uint32_t *etab, uint32_t *rtab, uint16_t raw_sym,
                               uint32_t *words /* may be NULL: count only */) {
  int64_t G = 32 * (int64_t)C, ng = ngroups(n, C);
  uint64_t w = 0, ne = 0, nr = 0;
  for (int64_t g = 0; g < ng; g++) {
    if (gtab) gtab[g] = (uint32_t)w;
    if (etab) etab[g] = (uint32_t)ne;
    if (rtab) rtab[g] = (uint32_t)nr;
    for (int64_t p = g * G; p < n && p < (g + 1) * G; p++) {
      ne += sym[p] == 0;
      nr += sym[p] == raw_sym;
    }
    uint64_t bit = 0;
    for (int l = 0; l < 32; l++) {
      uint64_t lane_bits = 0;
      for (int64_t k = 0; k < C; k++) {
        int64_t p = g * G + 32 * k + l;
        if (p >= n) break;
        uint16_t s = sym[p];
        for (int b = len[s] - 1; b >= 0; b--) {
          if (words && ((code[s] >> b) & 1u)) {
            uint64_t pos = bit;
            words[w + pos / 32] |= 1u << (31 - (pos % 32));
          }
          bit++;
        }
        lane_bits += len[s];
      }
      if (ltab) ltab[g * 32 + l] = (uint16_t)lane_bits;
    }
    w += (bit + 31) / 32;
  }
  if (gtab) gtab[ng] = (uint32_t)w;
  if (etab) etab[ng] = (uint32_t)ne;
  if (rtab) rtab[ng] = (uint32_t)nr;
  return w;
}

/* ------------------------------------------------------------------------ */
/* compression (Algorithm 3, closed loop)                                    */
/* ------------------------------------------------------------------------ */
int orc_compress(const orc_grid *g, int64_t n_v, const int32_t *vid, const uint16_t *lam,
                 const uint32_t *cell, const uint16_t *frac, const void *x, const orc_params *p,
                 uint8_t *out, size_t capacity, size_t *out_size, int32_t *Q_dbg,
                 int32_t *q1_dbg, uint16_t *sym1_dbg, uint16_t *sym2_dbg) {
  int st = check_params(p);
  if (st) return st;
  orc_field f;
  st = orc_field_params(p, n_v, x, &f);
  if (st) return st;
  const int dim = g->dim;
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int64_t ng = nx * ny * nz;
  const size_t vsz = p->dtype == 0 ? 8 : 4;
  const int R1 = p->R1, R2 = p->R2;

  int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_v);
  int32_t *q1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  int32_t *dl = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  uint16_t *sym1 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)ng);
  uint16_t *sym2 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n_v);
  int32_t *val2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_v);
  uint64_t *h1 = (uint64_t *)calloc((size_t)2 * R1, sizeof(uint64_t));
  uint64_t *h2 = (uint64_t *)calloc((size_t)2 * R2, sizeof(uint64_t));
  uint8_t *len1 = (uint8_t *)calloc((size_t)2 * R1, 1), *len2 = (uint8_t *)calloc((size_t)2 * R2, 1);
  uint32_t *code1 = (uint32_t *)calloc((size_t)2 * R1, 4), *code2 = (uint32_t *)calloc((size_t)2 * R2, 4);
  st = ORC_OK;
  if (!Q || !q1 || !dl || !sym1 || !sym2 || !val2 || !h1 || !h2 || !len1 || !len2 || !code1 ||
      !code2) {
    st = ORC_ERR_OOM;
    goto done;
  }

  /* 1. vertex codes: Q = round(x / s2) - K (FP64 product, ties to even) */
  for (int64_t i = 0; i < n_v; i++) {
    double v = load_value(x, p->dtype, i);
    double u = v * f.inv2;
    Q[i] = (int32_t)((int64_t)rint(u) - f.K);
  }

  /* 2. f: barycentric interpolation of the vertex codes onto the grid, then
   *    rescaled to grid bins: q1 = round((s2 / s1) * x1) */
  for (int64_t j = 0; j < ng; j++) {
    int64_t a;
    float acc = 0.0f;
    if (vid[j] < 0) {
      a = f.fill_u;
    } else {
      a = Q[vid[j]];
      for (int k = 1; k <= dim; k++) {
        int32_t dk = wrap_sub(Q[vid[k * ng + j]], (int32_t)a);
        float lf = (float)lam[(k - 1) * ng + j] * 0x1p-15f;
        if (k == 1) acc = (float)dk * lf;
        else acc = fmaf((float)dk, lf, acc);
      }
    }
    int64_t q = rescale(a, acc, f.rho21_q, f.rho21_f);
    if (q <= -((int64_t)1 << 27) || q >= ((int64_t)1 << 27)) { st = ORC_ERR_RANGE; goto done; }
    q1[j] = (int32_t)q;
  }

  /* 3. C(x1): Lorenzo difference and symbols */
  int32_t nn[3] = {g->n[0], g->n[1], g->n[2]};
  orc_lorenzo(dim, nn, q1, dl);
  uint64_t nout1 = 0;
  for (int64_t j = 0; j < ng; j++) {
    int32_t d = dl[j];
    if (d >= -(R1 - 1) && d <= R1 - 2) sym1[j] = (uint16_t)(d + R1);
    else { sym1[j] = 0; nout1++; }
    h1[sym1[j]]++;
  }

  /* 4. g(x1') at every vertex, residual code q2 = Q - P, bound guard */
  uint64_t nout2 = 0, nraw = 0;
  for (int64_t i = 0; i < n_v; i++) {
    uint32_t c = cell[i];
    float fx = (float)frac[i] * 0x1p-15f;
    float fy = (float)frac[n_v + i] * 0x1p-15f;
    int32_t c000 = q1[c], c100 = q1[c + 1], c010 = q1[c + nx], c110 = q1[c + nx + 1];
    int32_t d100 = wrap_sub(c100, c000), d010 = wrap_sub(c010, c000);
    float acc;
    if (dim == 2) {
      int32_t d110 = wrap_add(wrap_sub(wrap_sub(c110, c100), c010), c000);
      acc = fx * (float)d100;
      acc = fmaf(fy, (float)d010, acc);
      float fxy = fx * fy;
      acc = fmaf(fxy, (float)d110, acc);
    } else {
      float fz = (float)frac[2 * n_v + i] * 0x1p-15f;
      int64_t sxy = nx * ny;
      int32_t c001 = q1[c + sxy], c101 = q1[c + sxy + 1], c011 = q1[c + sxy + nx],
              c111 = q1[c + sxy + nx + 1];
      int32_t d001 = wrap_sub(c001, c000);
      int32_t d110 = wrap_add(wrap_sub(wrap_sub(c110, c100), c010), c000);
      int32_t d101 = wrap_add(wrap_sub(wrap_sub(c101, c100), c001), c000);
      int32_t d011 = wrap_add(wrap_sub(wrap_sub(c011, c010), c001), c000);
      int32_t d111 = wrap_sub(c111, c110);
      d111 = wrap_sub(d111, c101);
      d111 = wrap_sub(d111, c011);
      d111 = wrap_add(d111, c100);
      d111 = wrap_add(d111, c010);
      d111 = wrap_add(d111, c001);
      d111 = wrap_sub(d111, c000);
      acc = fx * (float)d100;
      acc = fmaf(fy, (float)d010, acc);
      acc = fmaf(fz, (float)d001, acc);
      float fxy = fx * fy, fxz = fx * fz, fyz = fy * fz;
      float fxyz = fxy * fz;
      acc = fmaf(fxy, (float)d110, acc);
      acc = fmaf(fxz, (float)d101, acc);
      acc = fmaf(fyz, (float)d011, acc);
      acc = fmaf(fxyz, (float)d111, acc);
    }
    int64_t P = rescale(c000, acc, f.rho12_q, f.rho12_f);
    int64_t q2 = (int64_t)Q[i] - P;
    /* guard: reconstruct exactly as the decompressor will, check |x - x'| */
    double v = load_value(x, p->dtype, i);
    double xr = f.s2 * (double)((int64_t)Q[i] + f.K);
    double xo = p->dtype == 0 ? xr : (double)(float)xr;
    if (fabs(v - xo) > f.tau2 || q2 <= INT32_MIN || q2 > INT32_MAX) {
      sym2[i] = (uint16_t)(2 * R2 - 1);
      nraw++;
    } else if (q2 >= -(R2 - 1) && q2 <= R2 - 2) {
      sym2[i] = (uint16_t)(q2 + R2);
    } else {
      sym2[i] = 0;
      val2[i] = (int32_t)q2;
      nout2++;
    }
    h2[sym2[i]]++;
  }

  /* 5. canonical Huffman code books */
  if ((st = orc_huffman_lengths(h1, 2 * R1, p->lmax, len1))) goto done;
  if ((st = orc_huffman_lengths(h2, 2 * R2, p->lmax, len2))) goto done;
  orc_canonical_codes(len1, 2 * R1, code1);
  orc_canonical_codes(len2, 2 * R2, code2);

  /* 6. layout, then write */
  {
    int64_t g1 = ngroups(ng, p->C1), g2 = ngroups(n_v, p->C2);
    uint64_t w1 = pack_component(sym1, ng, p->C1, len1, code1, NULL, NULL, NULL, NULL, 0xFFFF, NULL);
    uint64_t w2 = pack_component(sym2, n_v, p->C2, len2, code2, NULL, NULL, NULL, NULL, 0xFFFF, NULL);
    layout_t L;
    make_layout(R1, R2, g1, g2, nout1, nout2, nraw, vsz, w1, w2, &L);
    *out_size = L.total;
    if (L.total > capacity || !out) { st = ORC_ERR_CAPACITY; goto done; }
    memset(out, 0, L.total);
    uint8_t *h = out;
    put_u32(h + 0, MAGIC);
    put_u32(h + 4, VERSION);
    put_u32(h + 8, HEADER_BYTES);
    put_u32(h + 12, (uint32_t)p->dtype);
    put_u32(h + 16, (uint32_t)dim);
    put_u32(h + 20, (uint32_t)(f.guard ? 1 : 0));
    put_u32(h + 24, (uint32_t)R1);
    put_u32(h + 28, (uint32_t)R2);
    put_u32(h + 32, (uint32_t)p->C1);
    put_u32(h + 36, (uint32_t)p->C2);
    put_u32(h + 40, (uint32_t)p->lmax);
    put_u32(h + 44, (uint32_t)nx);
    put_u32(h + 48, (uint32_t)ny);
    put_u32(h + 52, (uint32_t)nz);
    put_u64(h + 56, (uint64_t)n_v);
    put_u64(h + 64, (uint64_t)ng);
    put_f64(h + 72, f.tau);
    put_f64(h + 80, f.tau1);
    put_f64(h + 88, f.tau2);
    put_f64(h + 96, f.s1);
    put_f64(h + 104, f.s2);
    put_u64(h + 112, (uint64_t)f.K);
    put_u64(h + 120, (uint64_t)f.rho21_q);
    put_u64(h + 128, (uint64_t)f.rho12_q);
    put_u64(h + 136, (uint64_t)f.fill_u);
    put_u64(h + 144, nout1);
    put_u64(h + 152, nout2);
    put_u64(h + 160, nraw);
    put_u64(h + 168, w1);
    put_u64(h + 176, w2);
    put_u64(h + 184, (uint64_t)L.total);
    memcpy(out + L.lens1, len1, (size_t)2 * R1);
    memcpy(out + L.lens2, len2, (size_t)2 * R2);
    pack_component(sym1, ng, p->C1, len1, code1, (uint32_t *)(out + L.gtab1),
                   (uint16_t *)(out + L.ltab1), (uint32_t *)(out + L.etab1), NULL, 0xFFFF,
                   (uint32_t *)(out + L.bits1));
    pack_component(sym2, n_v, p->C2, len2, code2, (uint32_t *)(out + L.gtab2),
                   (uint16_t *)(out + L.ltab2), (uint32_t *)(out + L.etab2),
                   (uint32_t *)(out + L.rtab2), (uint16_t)(2 * R2 - 1), (uint32_t *)(out + L.bits2));
    /* escape values and raw values in increasing index order */
    uint64_t k1 = 0, k2 = 0, kr = 0;
    for (int64_t j = 0; j < ng; j++)
      if (sym1[j] == 0) put_u32(out + L.out1 + 4 * k1++, (uint32_t)dl[j]);
    for (int64_t i = 0; i < n_v; i++) {
      if (sym2[i] == 0) put_u32(out + L.out2 + 4 * k2++, (uint32_t)val2[i]);
      else if (sym2[i] == 2 * R2 - 1)
        memcpy(out + L.raw + vsz * kr++, (const uint8_t *)x + vsz * (size_t)i, vsz);
    }
  }
  if (Q_dbg) memcpy(Q_dbg, Q, sizeof(int32_t) * (size_t)n_v);
  if (q1_dbg) memcpy(q1_dbg, q1, sizeof(int32_t) * (size_t)ng);
  if (sym1_dbg) memcpy(sym1_dbg, sym1, sizeof(uint16_t) * (size_t)ng);
  if (sym2_dbg) memcpy(sym2_dbg, sym2, sizeof(uint16_t) * (size_t)n_v);
done:
  free(Q); free(q1); free(dl); free(sym1); free(sym2); free(val2); free(h1); free(h2);
  free(len1); free(len2); free(code1); free(code2);
  return st;
}

/* ------------------------------------------------------------------------ */
/* decompression (Algorithm 4)                                               */
/* ------------------------------------------------------------------------ */
/* canonical decoder: read one bit at a time until the prefix is a code */
typedef struct {
  uint32_t first[26];  /* first code of each length */
  uint32_t count[26];  /* number of codes of each length */
  uint32_t offset[26]; /* index of the first symbol of each length in sorted[] */
  uint16_t *sorted;    /* symbols in (length, symbol) order */
} decoder_t;

static int decoder_init(const uint8_t *len, int nsym, int lmax, decoder_t *D) {
  memset(D, 0, sizeof(*D));
  D->sorted = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)nsym);
  if (!D->sorted) return ORC_ERR_OOM;
  for (int s = 0; s < nsym; s++) {
    if (len[s] > lmax) return ORC_ERR_CORRUPT;
    D->count[len[s]]++;
  }
  /* Kraft inequality: sum 2^-len <= 1 */
  uint64_t kraft = 0;
  for (int l = 1; l <= 24; l++) kraft += (uint64_t)D->count[l] << (24 - l);
  if (kraft > ((uint64_t)1 << 24)) return ORC_ERR_CORRUPT;
  uint32_t code = 0, off = 0;
  for (int l = 1; l <= 24; l++) {
    D->first[l] = code;
    D->offset[l] = off;
    off += D->count[l];
    code = (code + D->count[l]) << 1;
  }
  uint32_t pos[26];
  memcpy(pos, D->offset, sizeof(pos));
  for (int l = 1; l <= 24; l++)
    for (int s = 0; s < nsym; s++)
      if (len[s] == l) D->sorted[pos[l]++] = (uint16_t)s;
  return ORC_OK;
}

typedef struct { const uint32_t *w; uint64_t nwords; uint64_t bit; } bitreader_t;

static int read_bit(bitreader_t *r, uint32_t *b) {
  uint64_t wi = r->bit / 32;
  if (wi >= r->nwords) return ORC_ERR_CORRUPT;
  *b = (r->w[wi] >> (31 - r->bit % 32)) & 1u;
  r->bit++;
  return ORC_OK;
}

static int decode_symbol(const decoder_t *D, int lmax, bitreader_t *r, uint16_t *sym) {
  uint32_t code = 0;
  for (int l = 1; l <= lmax; l++) {
    uint32_t b;
    if (read_bit(r, &b)) return ORC_ERR_CORRUPT;
    code = (code << 1) | b;
    if (D->count[l] && code - D->first[l] < D->count[l]) {
      *sym = D->sorted[D->offset[l] + (code - D->first[l])];
      return ORC_OK;
    }
  }
  return ORC_ERR_CORRUPT;
}

static int unpack_component(const uint8_t *in, size_t size, const layout_t *L, int which,
                            int64_t n, int C, int nsym, int lmax, uint64_t words, uint16_t *sym) {
  size_t off_len = which == 1 ? L->lens1 : L->lens2;
  size_t off_g = which == 1 ? L->gtab1 : L->gtab2;
  size_t off_l = which == 1 ? L->ltab1 : L->ltab2;
  size_t off_b = which == 1 ? L->bits1 : L->bits2;
  (void)size;
  decoder_t D;
  int st = decoder_init(in + off_len, nsym, lmax, &D);
  if (st) { free(D.sorted); return st; }
  int64_t G = 32 * (int64_t)C, ng = ngroups(n, C);
  if (get_u32(in + off_g) != 0 || get_u32(in + off_g + 4 * (size_t)ng) != words) {
    free(D.sorted);
    return ORC_ERR_CORRUPT;
  }
  for (int64_t g = 0; g < ng; g++) {
    uint64_t w0 = get_u32(in + off_g + 4 * (size_t)g), w1 = get_u32(in + off_g + 4 * (size_t)(g + 1));
    if (w1 < w0 || w1 > words) { free(D.sorted); return ORC_ERR_CORRUPT; }
    bitreader_t r;
    r.w = (const uint32_t *)(in + off_b);
    r.nwords = w1; /* a group may not read past its own words */
    uint64_t start = w0 * 32;
    for (int l = 0; l < 32; l++) {
      uint16_t lb;
      memcpy(&lb, in + off_l + 2 * (size_t)(g * 32 + l), 2);
      r.bit = start;
      for (int64_t k = 0; k < C; k++) {
        int64_t p = g * G + 32 * k + l;
        if (p >= n) break;
        if (decode_symbol(&D, lmax, &r, &sym[p])) { free(D.sorted); return ORC_ERR_CORRUPT; }
      }
      if (r.bit - start != lb) { free(D.sorted); return ORC_ERR_CORRUPT; }
      start += lb;
    }
  }
  free(D.sorted);
  return ORC_OK;
}

/* A group prefix table must start at 0, end at the total, and step by the
 * number of symbols equal to `target` in each group. */
static int check_prefix(const uint8_t *tab, int64_t ng, uint64_t total, const uint16_t *sym,
                        int64_t n, int C, uint16_t target) {
  int64_t G = 32 * (int64_t)C;
  uint64_t acc = 0;
  for (int64_t g = 0; g < ng; g++) {
    if (get_u32(tab + 4 * g) != acc) return ORC_ERR_CORRUPT;
    for (int64_t p = g * G; p < n && p < (g + 1) * G; p++) acc += sym[p] == target;
  }
  if (acc != total || get_u32(tab + 4 * ng) != total) return ORC_ERR_CORRUPT;
  return ORC_OK;
}

int orc_decompress(const orc_grid *g, int64_t n_v, const uint32_t *cell, const uint16_t *frac,
                   const uint8_t *in, size_t size, void *xout, int32_t *q1_dbg) {
  if (!in || size < HEADER_BYTES) return ORC_ERR_CORRUPT;
  if (get_u32(in) != MAGIC || get_u32(in + 4) != VERSION || get_u32(in + 8) != HEADER_BYTES)
    return ORC_ERR_CORRUPT;
  const int dtype = (int)get_u32(in + 12), dim = (int)get_u32(in + 16);
  const int R1 = (int)get_u32(in + 24), R2 = (int)get_u32(in + 28);
  const int C1 = (int)get_u32(in + 32), C2 = (int)get_u32(in + 36), lmax = (int)get_u32(in + 40);
  const int64_t nx = get_u32(in + 44), ny = get_u32(in + 48), nz = get_u32(in + 52);
  if (dtype != 0 && dtype != 1) return ORC_ERR_CORRUPT;
  if (dim != g->dim || nx != g->n[0] || ny != g->n[1] || nz != g->n[2]) return ORC_ERR_CORRUPT;
  if ((int64_t)get_u64(in + 56) != n_v || (int64_t)get_u64(in + 64) != nx * ny * nz)
    return ORC_ERR_CORRUPT;
  orc_params chk = {dtype, 0, 1.0, 0.5, R1, R2, C1, C2, lmax};
  if (check_params(&chk)) return ORC_ERR_CORRUPT;
  const int64_t ng = nx * ny * nz;
  const double s2 = get_f64(in + 104);
  const int64_t K = (int64_t)get_u64(in + 112);
  const int64_t rho12_q = (int64_t)get_u64(in + 128);
  if (!(rho12_q >= 1 && rho12_q < 1125899906842624LL)) return ORC_ERR_CORRUPT;
  const float rho12_f = (float)rho12_q * 0x1p-40f;
  const uint64_t nout1 = get_u64(in + 144), nout2 = get_u64(in + 152), nraw = get_u64(in + 160);
  const uint64_t w1 = get_u64(in + 168), w2 = get_u64(in + 176), total = get_u64(in + 184);
  if (nout1 > (uint64_t)ng || nout2 > (uint64_t)n_v || nraw > (uint64_t)n_v) return ORC_ERR_CORRUPT;
  if (w1 > (uint64_t)ng * 24 + 64 || w2 > (uint64_t)n_v * 24 + 64) return ORC_ERR_CORRUPT;
  const size_t vsz = dtype == 0 ? 8 : 4;
  layout_t L;
  make_layout(R1, R2, ngroups(ng, C1), ngroups(n_v, C2), nout1, nout2, nraw, vsz, w1, w2, &L);
  if (L.total != total || total > size) return ORC_ERR_CORRUPT;

  int st = ORC_OK;
  uint16_t *sym1 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)ng);
  uint16_t *sym2 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n_v);
  int32_t *dl = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  int32_t *q1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  if (!sym1 || !sym2 || !dl || !q1) { st = ORC_ERR_OOM; goto done; }
  if ((st = unpack_component(in, size, &L, 1, ng, C1, 2 * R1, lmax, w1, sym1))) goto done;
  if ((st = unpack_component(in, size, &L, 2, n_v, C2, 2 * R2, lmax, w2, sym2))) goto done;

  /* grid: symbols -> Lorenzo differences; escapes take the next value */
  if ((st = check_prefix(in + L.etab1, ngroups(ng, C1), nout1, sym1, ng, C1, 0))) goto done;
  {
    uint64_t k = 0;
    for (int64_t j = 0; j < ng; j++) {
      uint16_t s = sym1[j];
      if (s == 0) dl[j] = (int32_t)get_u32(in + L.out1 + 4 * k++);
      else if (s == 2 * R1 - 1) { st = ORC_ERR_CORRUPT; goto done; }
      else dl[j] = (int32_t)s - R1;
    }
  }
  if ((st = check_prefix(in + L.etab2, ngroups(n_v, C2), nout2, sym2, n_v, C2, 0))) goto done;
  if ((st = check_prefix(in + L.rtab2, ngroups(n_v, C2), nraw, sym2, n_v, C2, 2 * R2 - 1))) goto done;
  int32_t nn[3] = {(int32_t)nx, (int32_t)ny, (int32_t)nz};
  orc_lorenzo_inverse(dim, nn, dl, q1);

  /* vertices: x' = s2 (K + P + q2), raw values for guarded vertices */
  {
    uint64_t k = 0, kr = 0;
    for (int64_t i = 0; i < n_v; i++) {
      uint16_t s = sym2[i];
      if (s == 2 * R2 - 1) {
        memcpy((uint8_t *)xout + vsz * (size_t)i, in + L.raw + vsz * kr++, vsz);
        continue;
      }
      int64_t q2;
      if (s == 0) {
        q2 = (int32_t)get_u32(in + L.out2 + 4 * k++);
      } else {
        q2 = (int64_t)s - R2;
      }
      uint32_t c = cell[i];
      float fx = (float)frac[i] * 0x1p-15f;
      float fy = (float)frac[n_v + i] * 0x1p-15f;
      int32_t c000 = q1[c], c100 = q1[c + 1], c010 = q1[c + nx], c110 = q1[c + nx + 1];
      int32_t d100 = wrap_sub(c100, c000), d010 = wrap_sub(c010, c000);
      float acc;
      if (dim == 2) {
        int32_t d110 = wrap_add(wrap_sub(wrap_sub(c110, c100), c010), c000);
        acc = fx * (float)d100;
        acc = fmaf(fy, (float)d010, acc);
        float fxy = fx * fy;
        acc = fmaf(fxy, (float)d110, acc);
      } else {
        float fz = (float)frac[2 * n_v + i] * 0x1p-15f;
        int64_t sxy = nx * ny;
        int32_t c001 = q1[c + sxy], c101 = q1[c + sxy + 1], c011 = q1[c + sxy + nx],
                c111 = q1[c + sxy + nx + 1];
        int32_t d001 = wrap_sub(c001, c000);
        int32_t d110 = wrap_add(wrap_sub(wrap_sub(c110, c100), c010), c000);
        int32_t d101 = wrap_add(wrap_sub(wrap_sub(c101, c100), c001), c000);
        int32_t d011 = wrap_add(wrap_sub(wrap_sub(c011, c010), c001), c000);
        int32_t d111 = wrap_sub(c111, c110);
        d111 = wrap_sub(d111, c101);
        d111 = wrap_sub(d111, c011);
        d111 = wrap_add(d111, c100);
        d111 = wrap_add(d111, c010);
        d111 = wrap_add(d111, c001);
        d111 = wrap_sub(d111, c000);
        acc = fx * (float)d100;
        acc = fmaf(fy, (float)d010, acc);
        acc = fmaf(fz, (float)d001, acc);
        float fxy = fx * fy, fxz = fx * fz, fyz = fy * fz;
        float fxyz = fxy * fz;
        acc = fmaf(fxy, (float)d110, acc);
        acc = fmaf(fxz, (float)d101, acc);
        acc = fmaf(fyz, (float)d011, acc);
        acc = fmaf(fxyz, (float)d111, acc);
      }
      int64_t P = rescale(c000, acc, rho12_q, rho12_f);
      double xr = s2 * (double)(K + P + q2);
      if (dtype == 0) ((double *)xout)[i] = xr;
      else ((float *)xout)[i] = (float)xr;
    }
    if (k != nout2 || kr != nraw) { st = ORC_ERR_CORRUPT; goto done; }
  }
  if (q1_dbg) memcpy(q1_dbg, q1, sizeof(int32_t) * (size_t)ng);
done:
  free(sym1); free(sym2); free(dl); free(q1);
  return st;
}
