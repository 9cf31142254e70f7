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
#define VERSION 2u
/* Lane table of a group (LTAB_BYTES): u16 base, then one u8 per lane; lane l
 * occupies base + delta_l bits. base = max(min lane bits, max lane bits -
 * 255): a lane shorter than base is padded with zero bits to base (delta 0),
 * so every delta fits a byte. */
#define LTAB_BYTES 34
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
/* Grid_Init (Algorithm 1): spacing per axis from the mesh                   */
/* ------------------------------------------------------------------------ */
static int cmp_f64(const void *a, const void *b) {
  const double x = *(const double *)a, y = *(const double *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Traverse the cells, take |p_a,d - p_b,d| for every edge of every cell (an
 * edge shared by several cells counts once per cell, as the traversal meets
 * it); gs_d is the bottom k-th percentile of these extents (nearest rank:
 * the ceil(k/100 N)-th smallest); while (max_d - min_d) / gs_d reaches gmax,
 * k grows by delta (k is not reset between axes, as Algorithm 1 prints it).
 * Output: n_d = ceil((max_d - min_d) / gs_d) + 1 points per axis (spacing at
 * most gs_d) and the corners min_d, max_d. ORC_ERR_RANGE when even k = 100
 * leaves gmax or more nodes. */
int orc_grid_init(int dim, int64_t n_v, const double *coords, int64_t n_c, const int32_t *cells,
                  double k_pct, double delta_pct, int32_t gmax, int32_t n_out[3], double lo[3],
                  double hi[3], double gs_out[3]) {
  if (dim != 2 && dim != 3) return ORC_ERR_INVALID_ARG;
  if (n_v < 1 || n_c < 1 || !coords || !cells) return ORC_ERR_INVALID_ARG;
  if (!(k_pct > 0.0 && k_pct <= 100.0) || !(delta_pct > 0.0) || gmax < 2 || gmax > 32767)
    return ORC_ERR_INVALID_ARG;
  const int nvc = dim + 1, npair = dim == 2 ? 3 : 6;
  for (int64_t i = 0; i < n_c * nvc; i++)
    if (cells[i] < 0 || cells[i] >= n_v) return ORC_ERR_INVALID_ARG;
  const int64_t N = n_c * npair;
  double *ext = (double *)malloc(sizeof(double) * (size_t)N);
  if (!ext) return ORC_ERR_OOM;
  double k = k_pct;
  for (int d = 0; d < 3; d++) { n_out[d] = 1; lo[d] = hi[d] = gs_out[d] = 0.0; }
  for (int d = 0; d < dim; d++) {
    double mn = coords[d], mx = coords[d];
    for (int64_t i = 1; i < n_v; i++) {
      const double c = coords[i * dim + d];
      if (c < mn) mn = c;
      if (c > mx) mx = c;
    }
    if (!(mn < mx)) { free(ext); return ORC_ERR_INVALID_ARG; }
    int64_t e = 0;
    for (int64_t c = 0; c < n_c; c++)
      for (int a = 0; a < nvc; a++)
        for (int b = a + 1; b < nvc; b++)
          ext[e++] = fabs(coords[(int64_t)cells[c * nvc + a] * dim + d] -
                          coords[(int64_t)cells[c * nvc + b] * dim + d]);
    qsort(ext, (size_t)N, sizeof(double), cmp_f64);
    double gs, gn;
    for (;;) {
      int64_t r = (int64_t)ceil(k / 100.0 * (double)N);
      if (r < 1) r = 1;
      if (r > N) r = N;
      gs = ext[r - 1];
      gn = gs > 0.0 ? (mx - mn) / gs : INFINITY;
      if (gn < (double)gmax) break;
      if (k >= 100.0) { free(ext); return ORC_ERR_RANGE; }
      k = k + delta_pct;
      if (k > 100.0) k = 100.0;
    }
    n_out[d] = (int32_t)ceil(gn) + 1;
    lo[d] = mn;
    hi[d] = mx;
    gs_out[d] = gs;
  }
  free(ext);
  return ORC_OK;
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
  /* the point's index on the base grid (Grid_Coarsen keeps a subset of its
   * planes; the point lies where it lies on the base grid) */
  int32_t bi[3];
  for (int d = 0; d < 3; d++) bi[d] = d < dim && g->keep[d] ? g->keep[d][idx[d]] : idx[d];
  /* FP32 pre-filter: reject points that are clearly outside. */
  float hf[3], pf[3], vf[4][3], l32[4], den32;
  for (int d = 0; d < 3; d++) {
    hf[d] = (float)g->h[d];
    pf[d] = (float)bi[d] * hf[d];
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
    double ih = (double)bi[d] * g->h[d];
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
 * coordinates with a margin of MARGIN32 cells (base-grid cells; with kept
 * planes, the kept indices inside that base range). Returns 0 if empty. */
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
    const int32_t *kp = g->keep[d];
    float hf = (float)g->h[d];
    float a = mn / hf - MARGIN32;
    float b = mx / hf + MARGIN32;
    float top = (float)(kp ? kp[g->n[d] - 1] : g->n[d] - 1);
    if (!(a <= top) || !(b >= 0.0f)) return 0; /* also rejects NaN */
    a = ceilf(a);
    b = floorf(b);
    if (a < 0.0f) a = 0.0f;
    if (b > top) b = top;
    if (a > b) return 0;
    if (!kp) {
      ilo[d] = (int32_t)a;
      ihi[d] = (int32_t)b;
      continue;
    }
    /* the kept planes with base index in [a, b]: the first at or above a,
     * the last at or below b (binary searches over the increasing list) */
    int32_t lo_k = 0, hi_k = g->n[d];
    while (lo_k < hi_k) {
      const int32_t md = (lo_k + hi_k) / 2;
      if ((float)kp[md] < a) lo_k = md + 1;
      else hi_k = md;
    }
    const int32_t i0 = lo_k;
    lo_k = 0;
    hi_k = g->n[d];
    while (lo_k < hi_k) {
      const int32_t md = (lo_k + hi_k) / 2;
      if ((float)kp[md] <= b) lo_k = md + 1;
      else hi_k = md;
    }
    const int32_t i1 = lo_k - 1;
    if (i0 > i1) return 0;
    ilo[d] = i0;
    ihi[d] = i1;
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
      double t = dd * g->inv_h[d];  /* in base-grid spacings */
      int64_t c;
      double f;
      const int32_t *kp = g->keep[d];
      if (!kp) {
        double fl = floor(t);
        if (!(fl >= 0.0)) c = 0;
        else if (fl > (double)(g->n[d] - 2)) c = g->n[d] - 2;
        else c = (int64_t)fl;
        f = t - (double)c;
      } else {
        /* kept planes: the last interval [kp[c], kp[c + 1]] starting at or
         * below t (the first one below kp[0]); f in that interval */
        c = 0;
        int64_t lo_k = 0, hi_k = g->n[d] - 2;  /* binary search in [0, n - 2] */
        while (lo_k <= hi_k) {
          const int64_t md = (lo_k + hi_k) / 2;
          if ((double)kp[md] <= t) {
            c = md;
            lo_k = md + 1;
          } else {
            hi_k = md - 1;
          }
        }
        f = (t - (double)kp[c]) / (double)(kp[c + 1] - kp[c]);
      }
      ci[d] = c;
      frac[(int64_t)d * n_v + i] = to_u16_unit(f);
    }
    cell[i] = (uint32_t)(ci[0] + nx * (ci[1] + ny * ci[2]));
  }
  (void)nz;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid_Coarsen (Algorithm 2)                                                */
/* ------------------------------------------------------------------------ */
/* Every vertex marks the nodes its g uses: the nearest node (the corner of
 * its cell on the near side of every midplane, from the u16 local
 * coordinates, half going up) or all corners of its cell. A node marks the
 * planes through it, one per axis; the unmarked planes go (every node on
 * them is unvisited), and the grid keeps the others in order. Removing a
 * plane leaves the other planes' marks as they were, so the axes and
 * planes may be taken in any order. */
int orc_grid_coarsen(const orc_grid *g, int64_t n_v, const uint32_t *cell, const uint16_t *frac,
                     int g_op, int32_t *keep_out[3], int32_t n_out[3]) {
  const int dim = g->dim;
  if (g_op != 0 && g_op != 1) return ORC_ERR_INVALID_ARG;
  if (n_v < 1 || !cell || !frac) return ORC_ERR_INVALID_ARG;
  for (int d = 0; d < dim; d++)
    if (g->keep[d] || !keep_out[d]) return ORC_ERR_INVALID_ARG;  /* a uniform grid */
  const int64_t nx = g->n[0], ny = g->n[1];
  uint8_t *mark[3] = {NULL, NULL, NULL};
  int st = ORC_OK;
  for (int d = 0; d < dim; d++)
    if (!(mark[d] = (uint8_t *)calloc((size_t)g->n[d], 1))) { st = ORC_ERR_OOM; goto done; }
  for (int64_t i = 0; i < n_v; i++) {
    const int64_t c = cell[i];
    const int64_t ci[3] = {c % nx, (c / nx) % ny, c / (nx * ny)};
    for (int d = 0; d < dim; d++) {
      if (ci[d] < 0 || ci[d] + 1 >= g->n[d]) { st = ORC_ERR_INVALID_ARG; goto done; }
      if (g_op == 1) {
        mark[d][ci[d] + (frac[(int64_t)d * n_v + i] >= 16384 ? 1 : 0)] = 1;
      } else {
        mark[d][ci[d]] = 1;
        mark[d][ci[d] + 1] = 1;
      }
    }
  }
  for (int d = 0; d < 3; d++) {
    if (d >= dim) { n_out[d] = 1; continue; }
    int32_t m = 0;
    for (int32_t k = 0; k < g->n[d]; k++) m += mark[d][k];
    const int all = m < 2;  /* fewer than two planes cannot make a grid */
    m = 0;
    for (int32_t k = 0; k < g->n[d]; k++)
      if (all || mark[d][k]) keep_out[d][m++] = k;
    n_out[d] = m;
  }
done:
  for (int d = 0; d < 3; d++) free(mark[d]);
  return st;
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

/* g at a vertex: the corner codes of its cell (order 000, 100, 010, 110, 001,
 * 101, 011, 111; x fastest) and the multilinear interpolation written on the
 * integer differences from corner 000, in FP32 with the fused multiply-adds
 * written out. Returns acc (the interpolation minus c000, in grid bins). */
static float vertex_interp(int dim, const int32_t *q1, int64_t nx, int64_t ny, uint32_t c, float fx,
                           float fy, float fz, int32_t cor[8]) {
  cor[0] = q1[c];
  cor[1] = q1[c + 1];
  cor[2] = q1[c + nx];
  cor[3] = q1[c + nx + 1];
  int32_t c000 = cor[0], c100 = cor[1], c010 = cor[2], c110 = cor[3];
  int32_t d100 = wrap_sub(c100, c000), d010 = wrap_sub(c010, c000);
  int32_t d110 = wrap_add(wrap_sub(wrap_sub(c110, c100), c010), c000);
  float acc;
  if (dim == 2) {
    acc = fx * (float)d100;
    acc = fmaf(fy, (float)d010, acc);
    float fxy = fx * fy;
    acc = fmaf(fxy, (float)d110, acc);
    return acc;
  }
  int64_t sxy = nx * ny;
  cor[4] = q1[c + sxy];
  cor[5] = q1[c + sxy + 1];
  cor[6] = q1[c + sxy + nx];
  cor[7] = q1[c + sxy + nx + 1];
  int32_t c001 = cor[4], c101 = cor[5], c011 = cor[6], c111 = cor[7];
  int32_t d001 = wrap_sub(c001, c000);
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
  return acc;
}

/* Nearest grid node m_k of vertex k (Sec. III-B): the corner of its cell on
 * the near side of the midpoint along every axis, read from the local
 * coordinates (2^-15 units; exactly half goes to the upper node). */
static int64_t nearest_node(int dim, int64_t nx, int64_t ny, uint32_t c, const uint16_t *frac,
                            int64_t n_v, int64_t i) {
  int64_t m = c;
  if (frac[i] >= 16384) m += 1;
  if (frac[n_v + i] >= 16384) m += nx;
  if (dim == 3 && frac[2 * n_v + i] >= 16384) m += nx * ny;
  return m;
}

/* Open loop: g on real corner values (vertex bins) in FP64, the same
 * difference form and order as vertex_interp, products and sums rounded one
 * at a time. */
static double vertex_interp64(int dim, const double c[8], float fx, float fy, float fz) {
  const double x = fx, y = fy, z = fz;
  const double d100 = c[1] - c[0], d010 = c[2] - c[0];
  const double d110 = ((c[3] - c[1]) - c[2]) + c[0];
  double acc = x * d100;
  acc = acc + y * d010;
  if (dim == 2) {
    const double xy = x * y;
    acc = acc + xy * d110;
    return c[0] + acc;
  }
  const double d001 = c[4] - c[0];
  const double d101 = ((c[5] - c[1]) - c[4]) + c[0];
  const double d011 = ((c[6] - c[2]) - c[4]) + c[0];
  const double d111 = ((((((c[7] - c[3]) - c[5]) - c[6]) + c[1]) + c[2]) + c[4]) - c[0];
  acc = acc + z * d001;
  const double xy = x * y, xz = x * z, yz = y * z, xyz = xy * z;
  acc = acc + xy * d110;
  acc = acc + xz * d101;
  acc = acc + yz * d011;
  acc = acc + xyz * d111;
  return c[0] + acc;
}

static void corner_values(int dim, const double *arr, int64_t nx, int64_t ny, uint32_t c,
                          double out[8]) {
  out[0] = arr[c];
  out[1] = arr[c + 1];
  out[2] = arr[c + nx];
  out[3] = arr[c + nx + 1];
  if (dim == 3) {
    const int64_t sxy = nx * ny;
    out[4] = arr[c + sxy];
    out[5] = arr[c + sxy + 1];
    out[6] = arr[c + sxy + nx];
    out[7] = arr[c + sxy + nx + 1];
  }
}

/* ------------------------------------------------------------------------ */
/* learned residual predictor: an integer-exact MLP                         */
/* ------------------------------------------------------------------------ */
/* Inputs: the corner codes' differences from corner 000 in vertex bins,
 * e_k = (c_k - c_000) * (s1/s2), scaled by 2^-sx and rounded to [-127, 127],
 * the local coordinates rounded to 0..127, and the level of corner 000 as a
 * fraction of the value range, L = c_000 (s1/s2) / Qhi rounded to 0..127
 * (Qhi the largest vertex code), so the network sees the corner values
 * themselves, not only their differences. Two hidden layers of 64 ReLU
 * units with 8-bit activations (right shifts s1, s2 with rounding, clamped to
 * 0..255), int8 weights, int32 biases, output p = acc3 * 2^e3 in vertex bins.
 * Every sum is an integer below 2^24 in magnitude, so it is exact in any
 * order and in FP32 as well as in integers. */
#define MLP_H 64
#define MLP_K 16
#define MODEL_MAGIC 0x4D43434Du /* 'M' 'C' 'C' 'M' */
#define MODEL_BYTES 5736u

typedef struct {
  int dim, n_in, sx, s1, s2, e3;
  int8_t W1[MLP_H][MLP_K], W2[MLP_H][MLP_H], W3[MLP_H];
  int32_t b1[MLP_H], b2[MLP_H], b3;
} mlp_t;

static int model_parse(const uint8_t *b, size_t n, int dim, mlp_t *m) {
  if (!b || n != MODEL_BYTES) return ORC_ERR_INVALID_ARG;
  if (get_u32(b) != MODEL_MAGIC || get_u32(b + 4) != 1) return ORC_ERR_INVALID_ARG;
  m->dim = (int)get_u32(b + 8);
  m->n_in = (int)get_u32(b + 12);
  memcpy(&m->sx, b + 16, 4);
  memcpy(&m->s1, b + 20, 4);
  memcpy(&m->s2, b + 24, 4);
  memcpy(&m->e3, b + 28, 4);
  if (m->dim != dim || m->n_in != (1 << dim) + dim) return ORC_ERR_INVALID_ARG;
  if (m->sx < -60 || m->sx > 60 || m->s1 < 1 || m->s1 > 30 || m->s2 < 1 || m->s2 > 30 ||
      m->e3 < -100 || m->e3 > 60)
    return ORC_ERR_INVALID_ARG;
  memcpy(m->W1, b + 32, sizeof(m->W1));
  memcpy(m->W2, b + 1056, sizeof(m->W2));
  memcpy(m->W3, b + 5152, sizeof(m->W3));
  memcpy(m->b1, b + 5216, sizeof(m->b1));
  memcpy(m->b2, b + 5472, sizeof(m->b2));
  memcpy(&m->b3, b + 5728, 4);
  for (int j = 0; j < MLP_H; j++) {
    for (int i = 0; i < MLP_K; i++)
      if (m->W1[j][i] < -127 || (i >= m->n_in && m->W1[j][i] != 0)) return ORC_ERR_INVALID_ARG;
    for (int i = 0; i < MLP_H; i++)
      if (m->W2[j][i] < -127) return ORC_ERR_INVALID_ARG;
    if (m->W3[j] < -127) return ORC_ERR_INVALID_ARG;
    if (m->b1[j] < -(1 << 22) || m->b1[j] > (1 << 22) || m->b2[j] < -(1 << 22) ||
        m->b2[j] > (1 << 22))
      return ORC_ERR_INVALID_ARG;
  }
  if (m->b3 < -(1 << 22) || m->b3 > (1 << 22)) return ORC_ERR_INVALID_ARG;
  return ORC_OK;
}

static void mlp_features(int dim, int sx, const int32_t cor[8], float fx, float fy, float fz,
                         float rho12_f, int64_t Qhi, int32_t xq[MLP_K]) {
  const int nc = 1 << dim;
  const float scale = ldexpf(1.0f, -sx);
  memset(xq, 0, sizeof(int32_t) * MLP_K);
  for (int k = 1; k < nc; k++) {
    float e = (float)wrap_sub(cor[k], cor[0]) * rho12_f;
    e = e * scale;
    float r = rintf(e);
    if (r > 127.0f) r = 127.0f;
    if (r < -127.0f) r = -127.0f;
    xq[k - 1] = (int32_t)r;
  }
  const float f3[3] = {fx, fy, fz};
  for (int d = 0; d < dim; d++) xq[nc - 1 + d] = (int32_t)rintf(f3[d] * 127.0f);
  float lv = 0.0f;
  if (Qhi > 0) {
    const float inv = 127.0f / (float)Qhi;
    lv = rintf(((float)cor[0] * rho12_f) * inv);
    if (lv > 127.0f) lv = 127.0f;
    if (lv < 0.0f) lv = 0.0f;
  }
  xq[nc - 1 + dim] = (int32_t)lv;
}

static int32_t act8(int32_t a, int s) {
  /* round(a / 2^s) half up, clamped to 0..255 (negative sums give 0) */
  int64_t t = (int64_t)a + ((int64_t)1 << (s - 1));
  if (t < 0) return 0;
  int64_t v = t >> s;
  return v > 255 ? 255 : (int32_t)v;
}

static float mlp_forward(const mlp_t *m, const int32_t xq[MLP_K]) {
  int32_t h1[MLP_H], h2[MLP_H];
  for (int j = 0; j < MLP_H; j++) {
    int32_t a = m->b1[j];
    for (int i = 0; i < MLP_K; i++) a += (int32_t)m->W1[j][i] * xq[i];
    h1[j] = act8(a, m->s1);
  }
  for (int j = 0; j < MLP_H; j++) {
    int32_t a = m->b2[j];
    for (int i = 0; i < MLP_H; i++) a += (int32_t)m->W2[j][i] * h1[i];
    h2[j] = act8(a, m->s2);
  }
  int32_t a = m->b3;
  for (int i = 0; i < MLP_H; i++) a += (int32_t)m->W3[i] * h2[i];
  return ldexpf((float)a, m->e3);
}

/* P = round((s1/s2) g + p): the fixed-point rescale of the interpolation with
 * the network's correction added in FP32 before rounding. The rounded
 * fraction is clamped to +-2^50 (a larger correction makes the residual code
 * leave the int32 range, so the vertex is stored raw either way). */
static int64_t rescale_p(int64_t a, float acc, int64_t rq, float rf, float p) {
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
  t = t + p;
  if (t > 0x1p50f) t = 0x1p50f;
  if (t < -0x1p50f) t = -0x1p50f;
  return hi + (int64_t)rintf(t);
}

int orc_mlp_predict(int dim, const uint8_t *model, size_t model_bytes, const int32_t *corners,
                    const float *fr, float rho12_f, int64_t Qhi, int64_t n, int32_t *features,
                    float *p) {
  mlp_t m;
  int st = model_parse(model, model_bytes, dim, &m);
  if (st) return st;
  for (int64_t i = 0; i < n; i++) {
    int32_t xq[MLP_K];
    const int32_t *cor = corners + 8 * i;
    mlp_features(dim, m.sx, cor, fr[3 * i], fr[3 * i + 1], fr[3 * i + 2], rho12_f, Qhi, xq);
    if (features) memcpy(features + MLP_K * i, xq, sizeof(xq));
    p[i] = mlp_forward(&m, xq);
  }
  return ORC_OK;
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
  /* m codes fit in lmax bits only if m <= 2^lmax; then halving the counts
   * ends (at worst with all counts 1, a tree of depth ceil(log2 m)) */
  if (lmax < 1 || lmax > 32 || (lmax < 31 && (uint64_t)m > ((uint64_t)1 << lmax)))
    return ORC_ERR_INVALID_ARG;
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
      bits2, model, total;
} layout_t;

static int64_t ngroups(int64_t n, int C) { return n == 0 ? 0 : (n + 32 * (int64_t)C - 1) / (32 * (int64_t)C); }

/* Section order: header | code lengths 1, 2 | group word offsets 1, 2 |
 * group escape-count prefixes 1, 2 | group raw-count prefix 2 | lane bit
 * lengths 1, 2 | escape values 1, 2 (int32) | raw values (dtype) |
 * bitstream 1, 2 (u32 words) | predictor model (when used, 8-byte aligned). */
static void make_layout(int R1, int R2, int64_t ng1, int64_t ng2, uint64_t nout1, uint64_t nout2,
                        uint64_t nraw, size_t vsz, uint64_t words1, uint64_t words2,
                        size_t model_bytes, layout_t *L) {
  size_t o = HEADER_BYTES;
  L->lens1 = o; o += 2 * (size_t)R1;
  L->lens2 = o; o += 2 * (size_t)R2;
  o = align_up(o, 4);
  L->gtab1 = o; o += 4 * (size_t)(ng1 + 1);
  L->gtab2 = o; o += 4 * (size_t)(ng2 + 1);
  L->etab1 = o; o += 4 * (size_t)(ng1 + 1);
  L->etab2 = o; o += 4 * (size_t)(ng2 + 1);
  L->rtab2 = o; o += 4 * (size_t)(ng2 + 1);
  L->ltab1 = o; o += LTAB_BYTES * (size_t)ng1;
  L->ltab2 = o; o += LTAB_BYTES * (size_t)ng2;
  o = align_up(o, 4);
  L->out1 = o; o += 4 * (size_t)nout1;
  L->out2 = o; o += 4 * (size_t)nout2;
  o = align_up(o, 8);
  L->raw = o; o += vsz * (size_t)nraw;
  o = align_up(o, 4);
  L->bits1 = o; o += 4 * (size_t)words1;
  L->bits2 = o; o += 4 * (size_t)words2;
  o = align_up(o, 8);
  L->model = o; o += model_bytes;
  L->total = o;
}

static int check_params(const orc_params *p) {
  if (p->R1 < 4 || p->R1 > 32768 || p->R2 < 4 || p->R2 > 32768) return ORC_ERR_INVALID_ARG;
  if (p->C1 < 1 || p->C1 > 2048 || p->C2 < 1 || p->C2 > 2048) return ORC_ERR_INVALID_ARG;
  if (p->lmax < 1 || p->lmax > 24) return ORC_ERR_INVALID_ARG;
  /* every symbol of an alphabet must fit in lmax bits */
  if (2 * p->R1 > (1 << p->lmax) || 2 * p->R2 > (1 << p->lmax)) return ORC_ERR_INVALID_ARG;
  if (p->open_loop != 0 && p->open_loop != 1) return ORC_ERR_INVALID_ARG;
  if (p->open_loop && p->model) return ORC_ERR_INVALID_ARG;  /* the predictor is closed loop */
  if (p->f_op != 0 && p->f_op != 1) return ORC_ERR_INVALID_ARG;
  if (p->g_op != 0 && p->g_op != 1) return ORC_ERR_INVALID_ARG;
  if (p->g_op && p->model) return ORC_ERR_INVALID_ARG;  /* it corrects the interpolation */
  if (p->zero_run != 0 && p->zero_run != 1) return ORC_ERR_INVALID_ARG;
  /* the two run tokens extend each alphabet to 2R + 2 symbols */
  if (p->zero_run && (p->R1 > 32767 || p->R2 > 32767 || 2 * p->R1 + 2 > (1 << p->lmax) ||
                      2 * p->R2 + 2 > (1 << p->lmax)))
    return ORC_ERR_INVALID_ARG;
  return ORC_OK;
}

size_t orc_compress_bound(const orc_grid *g, int64_t n_v, const orc_params *p) {
  int64_t ng = (int64_t)g->n[0] * g->n[1] * g->n[2];
  size_t vsz = p->dtype == 0 ? 8 : 4;
  int64_t g1 = ngroups(ng, p->C1), g2 = ngroups(n_v, p->C2);
  uint64_t w1 = (uint64_t)((ng * p->lmax + 31) / 32 + g1);
  uint64_t w2 = (uint64_t)((n_v * p->lmax + 31) / 32 + g2);
  layout_t L;
  make_layout(p->R1, p->R2, g1, g2, (uint64_t)ng, 0, (uint64_t)n_v, vsz, w1, w2, MODEL_BYTES, &L);
  return L.total + 16;
}

/* Zero-run stage (an option; not in the paper). The symbols of one lane, in
 * lane order, become tokens: with zr, every maximal run of r >= 1 zero
 * symbols z = R (a Lorenzo difference or residual of 0) becomes the digits
 * d_i in {1, 2} of r = sum_i d_i 2^i (bijective base 2), least significant
 * digit first, as token 2R for a digit 1 and token 2R + 1 for a digit 2;
 * every other symbol is its own token. Without zr the tokens are the
 * symbols. A lane of c symbols gives at most c tokens. */
static int put_run(int64_t r, int R, uint16_t *tok, int nt) {
  while (r > 0) {
    const int64_t d = r % 2 == 1 ? 1 : 2;
    tok[nt++] = (uint16_t)(2 * R + d - 1);
    r = (r - d) / 2;
  }
  return nt;
}

static int lane_tokens(const uint16_t *sym, int64_t n, int C, int64_t g, int l, int R, int zr,
                       uint16_t *tok) {
  int nt = 0;
  int64_t run = 0;
  for (int64_t k = 0; k < C; k++) {
    const int64_t p = g * 32 * (int64_t)C + 32 * k + l;
    if (p >= n) break;
    if (zr && sym[p] == R) {
      run++;
      continue;
    }
    nt = put_run(run, R, tok, nt);
    run = 0;
    tok[nt++] = sym[p];
  }
  return put_run(run, R, tok, nt);
}

/* Token counts of one component over all its lanes (h has 2R + 2 entries,
 * zeroed by the caller). */
static void token_hist(const uint16_t *sym, int64_t n, int C, int R, int zr, uint64_t *h) {
  uint16_t tok[2048];
  for (int64_t g = 0; g < ngroups(n, C); g++)
    for (int l = 0; l < 32; l++) {
      const int nt = lane_tokens(sym, n, C, g, l, R, zr, tok);
      for (int t = 0; t < nt; t++) h[tok[t]]++;
    }
}

/* Pack one component: tokens in lane-chunk order. Lane l of group g owns the
 * symbols g*32C + 32k + l (k = 0..C-1); each lane's token codes are
 * concatenated MSB-first (then its padding), the 32 lanes of a group follow
 * each other without gaps, and each group starts on a 32-bit word. Bit b of a
 * group is bit 31 - b%32 of its word b/32. Writes gtab (word offsets) and
 * ltab (lane table); escape and raw counts are taken over the symbols. */
static uint64_t pack_component(const uint16_t *sym, int64_t n, int C, int R, int zr,
                               const uint8_t *len, const uint32_t *code, uint32_t *gtab,
                               uint8_t *ltab, uint32_t *etab, uint32_t *rtab, uint16_t raw_sym,
                               uint32_t *words /* may be NULL: count only */) {
  int64_t G = 32 * (int64_t)C, ng = ngroups(n, C);
  uint64_t w = 0, ne = 0, nr = 0;
  uint16_t tok[2048];
  for (int64_t g = 0; g < ng; g++) {
    if (gtab) gtab[g] = (uint32_t)w;
    if (etab) etab[g] = (uint32_t)ne;
    if (rtab) rtab[g] = (uint32_t)nr;
    for (int64_t p = g * G; p < n && p < (g + 1) * G; p++) {
      ne += sym[p] == 0;
      nr += sym[p] == raw_sym;
    }
    uint64_t lane_bits[32], mn = ~(uint64_t)0, mx = 0;
    for (int l = 0; l < 32; l++) {
      lane_bits[l] = 0;
      const int nt = lane_tokens(sym, n, C, g, l, R, zr, tok);
      for (int t = 0; t < nt; t++) lane_bits[l] += len[tok[t]];
      if (lane_bits[l] < mn) mn = lane_bits[l];
      if (lane_bits[l] > mx) mx = lane_bits[l];
    }
    const uint64_t base = mx > 255 && mx - 255 > mn ? mx - 255 : mn;
    if (ltab) {
      ltab[(size_t)g * LTAB_BYTES] = (uint8_t)(base & 0xFF);
      ltab[(size_t)g * LTAB_BYTES + 1] = (uint8_t)(base >> 8);
    }
    uint64_t bit = 0;
    for (int l = 0; l < 32; l++) {
      const uint64_t padded = lane_bits[l] < base ? base : lane_bits[l];
      uint64_t b0 = bit;
      const int nt = lane_tokens(sym, n, C, g, l, R, zr, tok);
      for (int t = 0; t < nt; t++) {
        const uint16_t s = tok[t];
        for (int b = len[s] - 1; b >= 0; b--) {
          if (words && ((code[s] >> b) & 1u)) {
            uint64_t pos = bit;
            words[w + pos / 32] |= 1u << (31 - (pos % 32));
          }
          bit++;
        }
      }
      bit = b0 + padded;  /* padding bits stay zero */
      if (ltab) ltab[(size_t)g * LTAB_BYTES + 2 + l] = (uint8_t)(padded - base);
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
  mlp_t model;
  int use_model = p->model != NULL;
  if (use_model && (st = model_parse(p->model, p->model_bytes, dim, &model))) return st;
  /* with auto_select both predictors run and the smaller encoding is kept */
  const int passes = use_model && p->auto_select ? 2 : 1;

  int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_v);
  int32_t *q1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  int32_t *dl = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  const int open = p->open_loop;
  double *x1v = open ? (double *)malloc(sizeof(double) * (size_t)ng) : NULL;
  int64_t *csum = NULL, *ccnt = NULL;  /* cluster sums and sizes (cluster-mean f) */
  uint16_t *sym1 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)ng);
  uint16_t *sym2 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n_v);
  int32_t *val2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_v);
  uint16_t *sym2b = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n_v);
  int32_t *val2b = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_v);
  /* code books over 2R symbols plus the zero-run stage's two run tokens
   * (which keep count 0, hence no code, without the stage) */
  const int nsym1 = 2 * R1 + 2, nsym2 = 2 * R2 + 2;
  uint64_t *h1 = (uint64_t *)calloc((size_t)nsym1, sizeof(uint64_t));
  uint64_t *h2 = (uint64_t *)calloc((size_t)nsym2, sizeof(uint64_t));
  uint64_t *h2b = (uint64_t *)calloc((size_t)nsym2, sizeof(uint64_t));
  uint8_t *len2b = (uint8_t *)calloc((size_t)nsym2, 1);
  uint8_t *len1 = (uint8_t *)calloc((size_t)nsym1, 1), *len2 = (uint8_t *)calloc((size_t)nsym2, 1);
  uint32_t *code1 = (uint32_t *)calloc((size_t)nsym1, 4), *code2 = (uint32_t *)calloc((size_t)nsym2, 4);
  st = ORC_OK;
  if (!Q || !q1 || !dl || !sym1 || !sym2 || !val2 || !h1 || !h2 || !len1 || !len2 || !code1 ||
      !code2 || !sym2b || !val2b || !h2b || !len2b || (open && !x1v)) {
    st = ORC_ERR_OOM;
    goto done;
  }

  /* 1. vertex codes: Q = round(x / s2) - K (FP64 product, ties to even) */
  for (int64_t i = 0; i < n_v; i++) {
    double v = load_value(x, p->dtype, i);
    double u = v * f.inv2;
    Q[i] = (int32_t)((int64_t)rint(u) - f.K);
  }

  /* 2. f: barycentric interpolation of the vertex codes onto the grid, or
   *    the cluster mean (the mean of the codes of the vertices whose nearest
   *    node is j: integer part S / n, fraction (S mod n) / n in FP32; a node
   *    no vertex is nearest to keeps the fill value, the paper's x1 = 0),
   *    then rescaled to grid bins: q1 = round((s2 / s1) * x1) */
  if (p->f_op) {
    csum = (int64_t *)calloc((size_t)ng, sizeof(int64_t));
    ccnt = (int64_t *)calloc((size_t)ng, sizeof(int64_t));
    if (!csum || !ccnt) { st = ORC_ERR_OOM; goto done; }
    for (int64_t i = 0; i < n_v; i++) {
      const int64_t m = nearest_node(dim, nx, ny, cell[i], frac, n_v, i);
      csum[m] += Q[i];
      ccnt[m] += 1;
    }
  }
  for (int64_t j = 0; j < ng; j++) {
    int64_t a;
    float acc = 0.0f;
    if (p->f_op) {
      if (ccnt[j] == 0) {
        a = f.fill_u;
      } else {
        a = csum[j] / ccnt[j];
        acc = (float)(csum[j] - a * ccnt[j]) / (float)ccnt[j];
      }
    } else if (vid[j] < 0) {
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
    if (open) x1v[j] = (double)a + (double)acc;  /* x1 itself, in vertex bins */
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

  /* 4. g(x1') at every vertex (plus the learned correction when a model is
   *    given), residual code q2 = Q - P, bound guard. With auto_select, pass
   *    0 is the plain predictor and pass 1 the learned one. */
  uint64_t nout2 = 0, nraw = 0, nout2b = 0, nrawb = 0;
  for (int pass = 0; pass < passes; pass++) {
    const int um = passes == 2 ? pass : use_model;
    uint16_t *s2 = pass ? sym2b : sym2;
    int32_t *v2 = pass ? val2b : val2;
    uint64_t *hh = pass ? h2b : h2;
    uint64_t *no = pass ? &nout2b : &nout2, *nr = pass ? &nrawb : &nraw;
    for (int64_t i = 0; i < n_v; i++) {
      float fx = (float)frac[i] * 0x1p-15f;
      float fy = (float)frac[n_v + i] * 0x1p-15f;
      float fz = dim == 3 ? (float)frac[2 * n_v + i] * 0x1p-15f : 0.0f;
      int32_t cor[8];
      float acc = vertex_interp(dim, q1, nx, ny, cell[i], fx, fy, fz, cor);
      if (open) {
        /* Algorithm 3 as printed: x2 = x - g(x1) with the unquantised x1, its
         * code q2 = round(x2 / s2) (vertex bins: u - K - g(x1), u = x / s2,
         * taken as (Q - g) + (u - rint(u))); reconstruction s2 (K + q2 +
         * g(x1')), bound tau1 + tau2, every vertex checked */
        double gv, gq;
        const double rho12 = (double)f.rho12_q * 0x1p-40;
        if (p->g_op) {  /* nearest node */
          const int64_t m = nearest_node(dim, nx, ny, cell[i], frac, n_v, i);
          gv = x1v[m];
          gq = (double)q1[m] * rho12;
        } else {
          double c[8], cq[8];
          corner_values(dim, x1v, nx, ny, cell[i], c);
          gv = vertex_interp64(dim, c, fx, fy, fz);
          for (int k = 0; k < (1 << dim); k++) cq[k] = (double)cor[k] * rho12;
          gq = vertex_interp64(dim, cq, fx, fy, fz);
        }
        double v = load_value(x, p->dtype, i);
        const double u = v * f.inv2;
        const double r = ((double)Q[i] - gv) + (u - rint(u));
        const double q2d = rint(r);
        int raw = !(fabs(q2d) < 2147483647.0);
        const int64_t q2 = raw ? 0 : (int64_t)q2d;
        if (!raw) {
          const double xr = f.s2 * ((double)(f.K + q2) + gq);
          const double xo = p->dtype == 0 ? xr : (double)(float)xr;
          raw = !(fabs(v - xo) <= f.tau1 + f.tau2);
        }
        if (raw) {
          s2[i] = (uint16_t)(2 * R2 - 1);
          (*nr)++;
        } else if (q2 >= -(R2 - 1) && q2 <= R2 - 2) {
          s2[i] = (uint16_t)(q2 + R2);
        } else {
          s2[i] = 0;
          v2[i] = (int32_t)q2;
          (*no)++;
        }
        hh[s2[i]]++;
        continue;
      }
      int64_t P;
      if (p->g_op) {  /* nearest node: P = round((s1/s2) q1[m]) */
        P = rescale(q1[nearest_node(dim, nx, ny, cell[i], frac, n_v, i)], 0.0f, f.rho12_q,
                    f.rho12_f);
      } else if (um) {
        int32_t xq[MLP_K];
        mlp_features(dim, model.sx, cor, fx, fy, fz, f.rho12_f, f.Qhi, xq);
        P = rescale_p(cor[0], acc, f.rho12_q, f.rho12_f, mlp_forward(&model, xq));
      } else {
        P = rescale(cor[0], acc, f.rho12_q, f.rho12_f);
      }
      int64_t q2 = (int64_t)Q[i] - P;
      /* guard: reconstruct exactly as the decompressor will, check |x - x'| */
      double v = load_value(x, p->dtype, i);
      double xr = f.s2 * (double)((int64_t)Q[i] + f.K);
      double xo = p->dtype == 0 ? xr : (double)(float)xr;
      if (fabs(v - xo) > f.tau2 || q2 <= INT32_MIN || q2 > INT32_MAX) {
        s2[i] = (uint16_t)(2 * R2 - 1);
        (*nr)++;
      } else if (q2 >= -(R2 - 1) && q2 <= R2 - 2) {
        s2[i] = (uint16_t)(q2 + R2);
      } else {
        s2[i] = 0;
        v2[i] = (int32_t)q2;
        (*no)++;
      }
      hh[s2[i]]++;
    }
  }
  /* 4b. zero-run stage: the code books count tokens (runs of zero symbols
   *     as their digits) instead of symbols; escape and raw counts stay */
  if (p->zero_run) {
    memset(h1, 0, sizeof(uint64_t) * (size_t)nsym1);
    memset(h2, 0, sizeof(uint64_t) * (size_t)nsym2);
    token_hist(sym1, ng, p->C1, R1, 1, h1);
    token_hist(sym2, n_v, p->C2, R2, 1, h2);
    if (passes == 2) {
      memset(h2b, 0, sizeof(uint64_t) * (size_t)nsym2);
      token_hist(sym2b, n_v, p->C2, R2, 1, h2b);
    }
  }
  if (passes == 2) {
    /* the exact encoded size of each choice: code bits plus escape and raw
     * values, plus the model for the learned one; a tie keeps the plain */
    if ((st = orc_huffman_lengths(h2, nsym2, p->lmax, len2))) goto done;
    if ((st = orc_huffman_lengths(h2b, nsym2, p->lmax, len2b))) goto done;
    uint64_t bz = 0, bl = 0;
    for (int k = 0; k < nsym2; k++) {
      bz += h2[k] * len2[k];
      bl += h2b[k] * len2b[k];
    }
    bz += 32 * h2[0] + 8 * vsz * h2[2 * R2 - 1];
    bl += 32 * h2b[0] + 8 * vsz * h2b[2 * R2 - 1] + 8 * (uint64_t)MODEL_BYTES;
    if (bl < bz) {
      uint16_t *ts = sym2; sym2 = sym2b; sym2b = ts;
      int32_t *tv = val2; val2 = val2b; val2b = tv;
      uint64_t *th = h2; h2 = h2b; h2b = th;
      nout2 = nout2b;
      nraw = nrawb;
    } else {
      use_model = 0;
    }
  }

  /* 5. canonical Huffman code books */
  if ((st = orc_huffman_lengths(h1, nsym1, p->lmax, len1))) goto done;
  if ((st = orc_huffman_lengths(h2, nsym2, p->lmax, len2))) goto done;
  orc_canonical_codes(len1, nsym1, code1);
  orc_canonical_codes(len2, nsym2, code2);

  /* 6. layout, then write */
  {
    int64_t g1 = ngroups(ng, p->C1), g2 = ngroups(n_v, p->C2);
    const int zr = p->zero_run;
    uint64_t w1 = pack_component(sym1, ng, p->C1, R1, zr, len1, code1, NULL, NULL, NULL, NULL,
                                 0xFFFF, NULL);
    uint64_t w2 = pack_component(sym2, n_v, p->C2, R2, zr, len2, code2, NULL, NULL, NULL, NULL,
                                 0xFFFF, NULL);
    layout_t L;
    make_layout(R1, R2, g1, g2, nout1, nout2, nraw, vsz, w1, w2, use_model ? MODEL_BYTES : 0, &L);
    *out_size = L.total;
    if (L.total > capacity || !out) { st = ORC_ERR_CAPACITY; goto done; }
    memset(out, 0, L.total);
    uint8_t *h = out;
    put_u32(h + 0, MAGIC);
    put_u32(h + 4, VERSION);
    put_u32(h + 8, HEADER_BYTES);
    put_u32(h + 12, (uint32_t)p->dtype);
    put_u32(h + 16, (uint32_t)dim);
    put_u32(h + 20, (uint32_t)((f.guard || open ? 1 : 0) | (use_model ? 2 : 0) | (open ? 4 : 0) |
                               (p->g_op ? 8 : 0) | (p->f_op ? 16 : 0) | (zr ? 64 : 0)));
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
    put_u64(h + 192, (uint64_t)(use_model ? MODEL_BYTES : 0));
    put_u64(h + 200, (uint64_t)f.Qhi);
    if (use_model) memcpy(out + L.model, p->model, MODEL_BYTES);
    memcpy(out + L.lens1, len1, (size_t)2 * R1);
    memcpy(out + L.lens2, len2, (size_t)2 * R2);
    /* the run tokens' code lengths (zero without the stage) */
    out[208] = len1[2 * R1];
    out[209] = len1[2 * R1 + 1];
    out[210] = len2[2 * R2];
    out[211] = len2[2 * R2 + 1];
    pack_component(sym1, ng, p->C1, R1, zr, len1, code1, (uint32_t *)(out + L.gtab1),
                   out + L.ltab1, (uint32_t *)(out + L.etab1), NULL, 0xFFFF,
                   (uint32_t *)(out + L.bits1));
    pack_component(sym2, n_v, p->C2, R2, zr, len2, code2, (uint32_t *)(out + L.gtab2),
                   out + L.ltab2, (uint32_t *)(out + L.etab2),
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
  free(sym2b); free(val2b); free(h2b); free(len2b); free(x1v); free(csum); free(ccnt);
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

/* Decode one component into symbols. With zr the code book also holds the
 * two run tokens (lengths from header bytes 208 + 2 (which - 1) and the next)
 * and each lane's tokens expand back: a digit d at digit position i (counted
 * from the last symbol that was not a digit) stands for d 2^i zero symbols. */
static int unpack_component(const uint8_t *in, size_t size, const layout_t *L, int which,
                            int64_t n, int C, int R, int zr, int lmax, uint64_t words,
                            uint16_t *sym) {
  size_t off_len = which == 1 ? L->lens1 : L->lens2;
  size_t off_g = which == 1 ? L->gtab1 : L->gtab2;
  size_t off_l = which == 1 ? L->ltab1 : L->ltab2;
  size_t off_b = which == 1 ? L->bits1 : L->bits2;
  (void)size;
  const int nsym = 2 * R + 2;
  uint8_t *len = (uint8_t *)calloc((size_t)nsym, 1);
  if (!len) return ORC_ERR_OOM;
  memcpy(len, in + off_len, (size_t)2 * R);
  if (zr) {
    len[2 * R] = in[208 + 2 * (which - 1)];
    len[2 * R + 1] = in[209 + 2 * (which - 1)];
  }
  decoder_t D;
  int st = decoder_init(len, nsym, lmax, &D);
  free(len);
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
    const uint8_t *lt = in + off_l + (size_t)g * LTAB_BYTES;
    const uint64_t base = (uint64_t)lt[0] | ((uint64_t)lt[1] << 8);
    for (int l = 0; l < 32; l++) {
      const uint64_t lb = base + lt[2 + l];
      r.bit = start;
      int64_t cnt = 0;  /* the lane's symbols: positions g G + 32 k + l < n */
      while (cnt < C && g * G + 32 * cnt + l < n) cnt++;
      int64_t k = 0;
      int digit = 0;
      while (k < cnt) {
        uint16_t t;
        if (decode_symbol(&D, lmax, &r, &t)) { free(D.sorted); return ORC_ERR_CORRUPT; }
        if (t >= 2 * R) {  /* a run digit (only in the zero-run stage's code book) */
          const int64_t z = (int64_t)(t - 2 * R + 1) << digit;
          if (digit > 40 || z > cnt - k) { free(D.sorted); return ORC_ERR_CORRUPT; }
          for (int64_t e = 0; e < z; e++) sym[g * G + 32 * (k + e) + l] = (uint16_t)R;
          k += z;
          digit++;
        } else {
          sym[g * G + 32 * k + l] = t;
          k++;
          digit = 0;
        }
      }
      /* the codes fill the lane, or a padded lane (delta 0) ends early */
      const uint64_t used = r.bit - start;
      if (used > lb || (used < lb && lt[2 + l] != 0)) { free(D.sorted); return ORC_ERR_CORRUPT; }
      start += lb;
    }
    if (start > w1 * 32) { free(D.sorted); return ORC_ERR_CORRUPT; }
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
  const uint32_t flags = get_u32(in + 20);
  const int zr = (flags & 64) != 0;  /* bit 6: zero-run stage */
  orc_params chk = {dtype, 0, 1.0, 0.5, R1, R2, C1, C2, lmax, NULL, 0};
  chk.zero_run = zr;
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
  const uint64_t mbytes = get_u64(in + 192);
  const int64_t Qhi = (int64_t)get_u64(in + 200);
  if (Qhi < 0 || Qhi >= ((int64_t)1 << 29)) return ORC_ERR_CORRUPT;
  const int use_model = (flags & 2) != 0;
  const int open = (flags & 4) != 0;
  const int g_near = (flags & 8) != 0;  /* bit 4: cluster-mean f (compression only) */
  if (flags & ~(31u | 64u)) return ORC_ERR_CORRUPT;
  if ((open || g_near) && use_model) return ORC_ERR_CORRUPT;
  if (mbytes != (use_model ? MODEL_BYTES : 0)) return ORC_ERR_CORRUPT;
  layout_t L;
  make_layout(R1, R2, ngroups(ng, C1), ngroups(n_v, C2), nout1, nout2, nraw, vsz, w1, w2,
              (size_t)mbytes, &L);
  if (L.total != total || total > size) return ORC_ERR_CORRUPT;
  mlp_t model;
  if (use_model && model_parse(in + L.model, MODEL_BYTES, dim, &model)) return ORC_ERR_CORRUPT;

  int st = ORC_OK;
  uint16_t *sym1 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)ng);
  uint16_t *sym2 = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n_v);
  int32_t *dl = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  int32_t *q1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)ng);
  if (!sym1 || !sym2 || !dl || !q1) { st = ORC_ERR_OOM; goto done; }
  if ((st = unpack_component(in, size, &L, 1, ng, C1, R1, zr, lmax, w1, sym1))) goto done;
  if ((st = unpack_component(in, size, &L, 2, n_v, C2, R2, zr, lmax, w2, sym2))) goto done;

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
      float fx = (float)frac[i] * 0x1p-15f;
      float fy = (float)frac[n_v + i] * 0x1p-15f;
      float fz = dim == 3 ? (float)frac[2 * n_v + i] * 0x1p-15f : 0.0f;
      int32_t cor[8];
      float acc = vertex_interp(dim, q1, nx, ny, cell[i], fx, fy, fz, cor);
      const int64_t m = g_near ? nearest_node(dim, nx, ny, cell[i], frac, n_v, i) : 0;
      if (open) {
        const double rho12 = (double)rho12_q * 0x1p-40;
        double gq;
        if (g_near) {
          gq = (double)q1[m] * rho12;
        } else {
          double cq[8];
          for (int k = 0; k < (1 << dim); k++) cq[k] = (double)cor[k] * rho12;
          gq = vertex_interp64(dim, cq, fx, fy, fz);
        }
        const double xr = s2 * ((double)(K + q2) + gq);
        if (dtype == 0) ((double *)xout)[i] = xr;
        else ((float *)xout)[i] = (float)xr;
        continue;
      }
      int64_t P;
      if (g_near) {
        P = rescale(q1[m], 0.0f, rho12_q, rho12_f);
      } else if (use_model) {
        int32_t xq[MLP_K];
        mlp_features(dim, model.sx, cor, fx, fy, fz, rho12_f, Qhi, xq);
        P = rescale_p(cor[0], acc, rho12_q, rho12_f, mlp_forward(&model, xq));
      } else {
        P = rescale(cor[0], acc, rho12_q, rho12_f);
      }
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

/* ------------------------------------------------------------------------ */
/* training network (the float form the predictor is trained in)            */
/* ------------------------------------------------------------------------ */
/* Round a float to bfloat16 (nearest, ties to even) and back. */
static double bf16(float v) {
  uint32_t b;
  memcpy(&b, &v, 4);
  if ((b & 0x7F800000u) == 0x7F800000u) return (double)v; /* inf / nan unchanged */
  uint32_t lsb = (b >> 16) & 1u;
  b = (b + 0x7FFFu + lsb) & 0xFFFF0000u;
  float r;
  memcpy(&r, &b, 4);
  return (double)r;
}

/* Loss and gradient of the float training network p = W3 a2 + b3,
 * a2 = relu(W2 a1 + b2), a1 = relu(W1 x + b1), over a batch of B samples:
 * mean absolute error (loss_kind 1) or mean squared error (loss_kind 0).
 * Layout: W1 [64][16], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]; grad
 * in the same layout (5313 values).
 *
 * rounding 0: the network in FP64 as written (the definition).
 * rounding 1: every operand of a tensor-core product rounded to bfloat16 as
 * the GPU rounds it: the weights, the inputs, a1 and a2 in the forward pass;
 * da2 (the gradient at the second hidden layer) where it multiplies a1 (for
 * dW2) and W2 (for da1), and da1 where it multiplies x (for dW1). The bias
 * gradients, dW3 and everything else stay unrounded. Sums are in FP64. */
int orc_mlp_grad(const float *W1, const float *b1, const float *W2, const float *b2,
                 const float *W3, const float *b3, const float *X, const float *Y, int64_t B,
                 int loss_kind, int rounding, double *grad, double *loss) {
  if (B <= 0 || (loss_kind != 0 && loss_kind != 1) || (rounding != 0 && rounding != 1))
    return ORC_ERR_INVALID_ARG;
  double w1[MLP_H][MLP_K], w2[MLP_H][MLP_H], w3[MLP_H];
#define RND(v) (rounding ? bf16((float)(v)) : (double)(v))
  for (int j = 0; j < MLP_H; j++) {
    for (int i = 0; i < MLP_K; i++) w1[j][i] = RND(W1[j * MLP_K + i]);
    for (int i = 0; i < MLP_H; i++) w2[j][i] = RND(W2[j * MLP_H + i]);
    w3[j] = RND(W3[j]);
  }
  const size_t ng = (size_t)MLP_H * MLP_K + MLP_H + (size_t)MLP_H * MLP_H + MLP_H + MLP_H + 1;
  memset(grad, 0, sizeof(double) * ng);
  double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_K, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H,
         *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_H;
  double L = 0.0;
  for (int64_t n = 0; n < B; n++) {
    double x[MLP_K], z1[MLP_H], a1[MLP_H], z2[MLP_H], a2[MLP_H];
    for (int i = 0; i < MLP_K; i++) x[i] = RND(X[n * MLP_K + i]);
    for (int j = 0; j < MLP_H; j++) {
      double z = b1[j];
      for (int i = 0; i < MLP_K; i++) z += w1[j][i] * x[i];
      z1[j] = z;
      a1[j] = RND(z > 0.0 ? z : 0.0);
    }
    for (int j = 0; j < MLP_H; j++) {
      double z = b2[j];
      for (int i = 0; i < MLP_H; i++) z += w2[j][i] * a1[i];
      z2[j] = z;
      a2[j] = RND(z > 0.0 ? z : 0.0);
    }
    double pr = b3[0];
    for (int i = 0; i < MLP_H; i++) pr += w3[i] * a2[i];
    const double e = pr - (double)Y[n];
    double dp;
    if (loss_kind == 0) {
      L += e * e;
      dp = 2.0 * e / (double)B;
    } else {
      L += fabs(e);
      dp = (e > 0.0 ? 1.0 : e < 0.0 ? -1.0 : 0.0) / (double)B;
    }
    gb3[0] += dp;
    double da2[MLP_H], da2r[MLP_H], da1[MLP_H];
    for (int i = 0; i < MLP_H; i++) {
      gW3[i] += dp * a2[i];
      da2[i] = z2[i] > 0.0 ? dp * w3[i] : 0.0;
      da2r[i] = RND(da2[i]);
    }
    for (int j = 0; j < MLP_H; j++) {
      gb2[j] += da2[j];
      for (int i = 0; i < MLP_H; i++) gW2[j * MLP_H + i] += da2r[j] * a1[i];
    }
    for (int i = 0; i < MLP_H; i++) {
      double t = 0.0;
      for (int j = 0; j < MLP_H; j++) t += w2[j][i] * da2r[j];
      da1[i] = z1[i] > 0.0 ? t : 0.0;
    }
    for (int j = 0; j < MLP_H; j++) {
      gb1[j] += da1[j];
      const double d = RND(da1[j]);
      for (int i = 0; i < MLP_K; i++) gW1[j * MLP_K + i] += d * x[i];
    }
  }
#undef RND
  *loss = L / (double)B;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* post-training quantisation of the float network                          */
/* ------------------------------------------------------------------------ */
/* Largest a in [-40, 40] with maxw 2^a <= 127 (0 for a zero matrix). */
static int weight_exp(double maxw) {
  if (maxw == 0.0) return 0;
  int a = -40;
  while (a < 40 && ldexp(maxw, a + 1) <= 127.0) a++;
  return a;
}

/* Smallest t in [-60, 60] with maxz 2^-t <= 255. */
static int act_exp(double maxz) {
  int t = -60;
  while (t < 60 && ldexp(maxz, -t) > 255.0) t++;
  return t;
}

static int32_t qbias(float b, int k) {
  double v = rint(ldexp((double)b, k));
  if (v > (double)(1 << 22)) v = (double)(1 << 22);
  if (v < -(double)(1 << 22)) v = -(double)(1 << 22);
  return (int32_t)v;
}

/* The float network takes x = X 2^-7 (X the integer features). With weight
 * exponents a_l (W_l 2^a_l rounded to int8) and activation exponents t_l
 * (the hidden values are relu(z_l) 2^-t_l on 0..255, t_l the smallest that
 * fits the calibration maximum max_z_l), the integer accumulators are
 * 2^(a1+7) z1, 2^(a2-t1) z2 and 2^(a3-t2) p, so s1 = t1 + a1 + 7,
 * s2 = t2 + a2 - t1 and e3 = t2 - a3. A shift above 30 lowers the weight
 * exponent, one below 1 raises the activation exponent. */
int orc_mlp_quantize(int dim, int sx, const float *params, float max_z1, float max_z2,
                     uint8_t *model) {
  if ((dim != 2 && dim != 3) || sx < -60 || sx > 60 || !params || !model) return ORC_ERR_INVALID_ARG;
  if (!(max_z1 >= 0.0f) || !(max_z2 >= 0.0f) || isinf(max_z1) || isinf(max_z2))
    return ORC_ERR_INVALID_ARG;
  const int n_in = (1 << dim) + dim;
  const float *W1 = params, *b1 = W1 + MLP_H * MLP_K, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
              *W3 = b2 + MLP_H, *b3 = W3 + MLP_H;
  for (int k = 0; k < MLP_H * MLP_K + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1; k++)
    if (!isfinite(params[k])) return ORC_ERR_INVALID_ARG;
  double m1 = 0.0, m2 = 0.0, m3 = 0.0;
  for (int j = 0; j < MLP_H; j++) {
    for (int i = 0; i < n_in; i++) m1 = fmax(m1, fabs((double)W1[j * MLP_K + i]));
    for (int i = 0; i < MLP_H; i++) m2 = fmax(m2, fabs((double)W2[j * MLP_H + i]));
    m3 = fmax(m3, fabs((double)W3[j]));
  }
  if (!(m1 <= 1e30 && m2 <= 1e30 && m3 <= 1e30)) return ORC_ERR_INVALID_ARG;
  int a1 = weight_exp(m1), t1 = act_exp(max_z1);
  int s1 = t1 + a1 + 7;
  if (s1 > 30) { a1 -= s1 - 30; s1 = 30; }
  if (s1 < 1) { t1 += 1 - s1; s1 = 1; }
  int a2 = weight_exp(m2), t2 = act_exp(max_z2);
  int s2 = t2 + a2 - t1;
  if (s2 > 30) { a2 -= s2 - 30; s2 = 30; }
  if (s2 < 1) { t2 += 1 - s2; s2 = 1; }
  const int a3 = weight_exp(m3);
  const int e3 = t2 - a3;
  if (e3 < -100 || e3 > 60) return ORC_ERR_RANGE;

  memset(model, 0, MODEL_BYTES);
  put_u32(model + 0, MODEL_MAGIC);
  put_u32(model + 4, 1);
  put_u32(model + 8, (uint32_t)dim);
  put_u32(model + 12, (uint32_t)n_in);
  put_u32(model + 16, (uint32_t)sx);
  put_u32(model + 20, (uint32_t)s1);
  put_u32(model + 24, (uint32_t)s2);
  put_u32(model + 28, (uint32_t)e3);
  for (int j = 0; j < MLP_H; j++) {
    for (int i = 0; i < n_in; i++)
      model[32 + j * MLP_K + i] = (uint8_t)(int8_t)rint(ldexp((double)W1[j * MLP_K + i], a1));
    for (int i = 0; i < MLP_H; i++)
      model[1056 + j * MLP_H + i] = (uint8_t)(int8_t)rint(ldexp((double)W2[j * MLP_H + i], a2));
    model[5152 + j] = (uint8_t)(int8_t)rint(ldexp((double)W3[j], a3));
    put_u32(model + 5216 + 4 * j, (uint32_t)qbias(b1[j], a1 + 7));
    put_u32(model + 5472 + 4 * j, (uint32_t)qbias(b2[j], a2 - t1));
  }
  put_u32(model + 5728, (uint32_t)qbias(b3[0], a3 - t2));
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* the paper's "default": the same coder on the vertex array (Sec. V)        */
/* ------------------------------------------------------------------------ */
/* Spacing of the value type at magnitude M (at least the smallest
 * subnormal): 2^(e - p) with M in [2^e, 2^(e+1)), p = 52 (FP64) or 23. */
static double spacing_at(double M, int dtype) {
  const int p = dtype == 0 ? 52 : 23;
  const double tiny = dtype == 0 ? 0x1p-1074 : 0x1p-149;
  if (!(M > 0.0)) return tiny;
  int e;
  frexp(M, &e); /* M = f 2^e, f in [0.5, 1): leading exponent e - 1 */
  double u = ldexp(1.0, e - 1 - p);
  return u > tiny ? u : tiny;
}

/* Per-field parameters of the 1D coder: tau as for the method, the bin
 * s = 2 (tau - m) (1 - 2^-20) with the margin m = 4 u64(M) (+ 2 u32(M) for
 * FP32 values), u the spacings at M = max |x|. The FP64 rounding of x / s
 * and of s (K + Q) moves x' by at most about 3 u64(M) and the cast to FP32
 * by at most u32(M), so |x - x'| <= tau at every value without a check and
 * no value is stored raw (which would break the chain of differences). */
static int field_params_1d(const orc_params *p, int64_t n, const void *x, orc_field *f) {
  memset(f, 0, sizeof(*f));
  if (n <= 0 || !x) return ORC_ERR_INVALID_ARG;
  if (p->dtype != 0 && p->dtype != 1) return ORC_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return ORC_ERR_INVALID_ARG;
  double lo = load_value(x, p->dtype, 0), hi = lo;
  for (int64_t i = 0; i < n; i++) {
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
  double m = 4.0 * spacing_at(f->M, 0);
  if (p->dtype == 1) m = m + 2.0 * spacing_at(f->M, 1);
  const double t = tau - m;
  if (!isfinite(tau) || !(t >= 1e-290)) return ORC_ERR_RANGE;
  f->tau1 = t;
  f->tau2 = t;
  f->s1 = (2.0 * t) * BIN_SHRINK;
  f->s2 = f->s1;
  if (!isfinite(f->s2)) return ORC_ERR_RANGE;
  f->inv2 = 1.0 / f->s2;
  double kd = rint(lo * f->inv2);
  double hd = rint(hi * f->inv2);
  if (!(fabs(kd) < 4611686018427387904.0) || !(fabs(hd) < 4611686018427387904.0))
    return ORC_ERR_RANGE;
  f->K = (int64_t)kd;
  f->Qhi = (int64_t)hd - f->K;
  if (f->Qhi >= ((int64_t)1 << 29)) return ORC_ERR_RANGE;
  f->rho21_q = f->rho12_q = (int64_t)1 << 40; /* one bin: ratio 1 */
  f->rho21_f = f->rho12_f = 1.0f;
  return ORC_OK;
}

size_t orc_compress_bound_1d(int64_t n, const orc_params *p) {
  size_t vsz = p->dtype == 0 ? 8 : 4;
  int64_t g1 = ngroups(n, p->C1);
  uint64_t w1 = (uint64_t)((n * p->lmax + 31) / 32 + g1);
  layout_t L;
  make_layout(p->R1, p->R2, g1, 0, (uint64_t)n, 0, 0, vsz, w1, 0, 0, &L);
  (void)vsz;
  return L.total + 16;
}

/* Q = round(x / s) - K; delta_i = Q_i - Q_(i-1) (delta_0 = Q_0); symbols
 * delta + R1 or an escape; canonical Huffman (of tokens with the zero-run
 * stage); the grid component's lane-group stream with the residual
 * component empty. Header: dim 1, n_x = n, flags bit 5 (and bit 6 with the
 * zero-run stage). */
int orc_compress_1d(int64_t n, const void *x, const orc_params *p, uint8_t *out, size_t capacity,
                    size_t *out_size, int32_t *Q_dbg) {
  if (!out_size) return ORC_ERR_INVALID_ARG;
  *out_size = 0;
  int st = check_params(p);
  if (st) return st;
  if (p->model || p->open_loop || p->f_op || p->g_op) return ORC_ERR_INVALID_ARG;
  if (n >= ((int64_t)1 << 31)) return ORC_ERR_INVALID_ARG;
  orc_field f;
  if ((st = field_params_1d(p, n, x, &f))) return st;
  const int R1 = p->R1, R2 = p->R2;
  const size_t vsz = p->dtype == 0 ? 8 : 4;
  int32_t *Q = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *dl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  uint16_t *sym = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
  const int nsym1 = 2 * R1 + 2, zr = p->zero_run;  /* 2R symbols and the two run tokens */
  uint64_t *h1 = (uint64_t *)calloc((size_t)nsym1, sizeof(uint64_t));
  uint8_t *len1 = (uint8_t *)calloc((size_t)nsym1, 1), *len2 = (uint8_t *)calloc((size_t)2 * R2, 1);
  uint32_t *code1 = (uint32_t *)calloc((size_t)nsym1, 4);
  if (!Q || !dl || !sym || !h1 || !len1 || !len2 || !code1) { st = ORC_ERR_OOM; goto done; }
  for (int64_t i = 0; i < n; i++)
    Q[i] = (int32_t)((int64_t)rint(load_value(x, p->dtype, i) * f.inv2) - f.K);
  uint64_t nout1 = 0;
  for (int64_t i = 0; i < n; i++) {
    const int32_t d = wrap_sub(Q[i], i ? Q[i - 1] : 0);
    dl[i] = d;
    if (d >= -(R1 - 1) && d <= R1 - 2) sym[i] = (uint16_t)(d + R1);
    else { sym[i] = 0; nout1++; }
    h1[sym[i]]++;
  }
  if (zr) {  /* the zero-run stage: count tokens */
    memset(h1, 0, sizeof(uint64_t) * (size_t)nsym1);
    token_hist(sym, n, p->C1, R1, 1, h1);
  }
  if ((st = orc_huffman_lengths(h1, nsym1, p->lmax, len1))) goto done;
  orc_canonical_codes(len1, nsym1, code1);
  {
    const int64_t g1 = ngroups(n, p->C1);
    const uint64_t w1 = pack_component(sym, n, p->C1, R1, zr, len1, code1, NULL, NULL, NULL, NULL,
                                       0xFFFF, NULL);
    layout_t L;
    make_layout(R1, R2, g1, 0, nout1, 0, 0, vsz, w1, 0, 0, &L);
    *out_size = L.total;
    if (L.total > capacity || !out) { st = ORC_ERR_CAPACITY; goto done; }
    memset(out, 0, L.total);
    uint8_t *h = out;
    put_u32(h + 0, MAGIC);
    put_u32(h + 4, VERSION);
    put_u32(h + 8, HEADER_BYTES);
    put_u32(h + 12, (uint32_t)p->dtype);
    put_u32(h + 16, 1u);
    put_u32(h + 20, zr ? 32u | 64u : 32u);
    put_u32(h + 24, (uint32_t)R1);
    put_u32(h + 28, (uint32_t)R2);
    put_u32(h + 32, (uint32_t)p->C1);
    put_u32(h + 36, (uint32_t)p->C2);
    put_u32(h + 40, (uint32_t)p->lmax);
    put_u32(h + 44, (uint32_t)n);
    put_u32(h + 48, 1u);
    put_u32(h + 52, 1u);
    put_u64(h + 56, (uint64_t)n);
    put_u64(h + 64, (uint64_t)n);
    put_f64(h + 72, f.tau);
    put_f64(h + 80, f.tau1);
    put_f64(h + 88, f.tau2);
    put_f64(h + 96, f.s1);
    put_f64(h + 104, f.s2);
    put_u64(h + 112, (uint64_t)f.K);
    put_u64(h + 120, (uint64_t)f.rho21_q);
    put_u64(h + 128, (uint64_t)f.rho12_q);
    put_u64(h + 136, 0);
    put_u64(h + 144, nout1);
    put_u64(h + 152, 0);
    put_u64(h + 160, 0);
    put_u64(h + 168, w1);
    put_u64(h + 176, 0);
    put_u64(h + 184, (uint64_t)L.total);
    put_u64(h + 192, 0);
    put_u64(h + 200, (uint64_t)f.Qhi);
    memcpy(out + L.lens1, len1, (size_t)2 * R1);
    memcpy(out + L.lens2, len2, (size_t)2 * R2);
    out[208] = len1[2 * R1];  /* the run tokens' code lengths */
    out[209] = len1[2 * R1 + 1];
    pack_component(sym, n, p->C1, R1, zr, len1, code1, (uint32_t *)(out + L.gtab1), out + L.ltab1,
                   (uint32_t *)(out + L.etab1), NULL, 0xFFFF, (uint32_t *)(out + L.bits1));
    put_u32(out + L.gtab2, 0);  /* the empty residual component: one zero entry per table */
    put_u32(out + L.etab2, 0);
    put_u32(out + L.rtab2, 0);
    uint64_t k1 = 0;
    for (int64_t i = 0; i < n; i++)
      if (sym[i] == 0) put_u32(out + L.out1 + 4 * k1++, (uint32_t)dl[i]);
  }
  if (Q_dbg) memcpy(Q_dbg, Q, sizeof(int32_t) * (size_t)n);
done:
  free(Q); free(dl); free(sym); free(h1); free(len1); free(len2); free(code1);
  return st;
}

/* Inverse: decode the differences, prefix sums (wrapping int32) give Q,
 * x' = cast(s (K + Q)). */
int orc_decompress_1d(int64_t n, const uint8_t *in, size_t size, void *xout) {
  if (!in || size < HEADER_BYTES) return ORC_ERR_CORRUPT;
  if (get_u32(in) != MAGIC || get_u32(in + 4) != VERSION || get_u32(in + 8) != HEADER_BYTES)
    return ORC_ERR_CORRUPT;
  const int dtype = (int)get_u32(in + 12);
  const int R1 = (int)get_u32(in + 24), R2 = (int)get_u32(in + 28);
  const int C1 = (int)get_u32(in + 32), C2 = (int)get_u32(in + 36), lmax = (int)get_u32(in + 40);
  if (dtype != 0 && dtype != 1) return ORC_ERR_CORRUPT;
  const uint32_t flags = get_u32(in + 20);  /* bit 5 alone, or with bit 6 (zero-run stage) */
  if (get_u32(in + 16) != 1u || (flags != 32u && flags != (32u | 64u))) return ORC_ERR_CORRUPT;
  const int zr = flags == (32u | 64u);
  if (get_u32(in + 44) != (uint32_t)n || get_u32(in + 48) != 1u || get_u32(in + 52) != 1u ||
      (int64_t)get_u64(in + 56) != n || (int64_t)get_u64(in + 64) != n)
    return ORC_ERR_CORRUPT;
  orc_params chk = {dtype, 0, 1.0, 0.5, R1, R2, C1, C2, lmax, NULL, 0};
  chk.zero_run = zr;
  if (check_params(&chk)) return ORC_ERR_CORRUPT;
  const double s = get_f64(in + 104);
  const int64_t K = (int64_t)get_u64(in + 112);
  const uint64_t nout1 = get_u64(in + 144), w1 = get_u64(in + 168), total = get_u64(in + 184);
  if (get_u64(in + 152) || get_u64(in + 160) || get_u64(in + 176) || get_u64(in + 192))
    return ORC_ERR_CORRUPT;
  if (nout1 > (uint64_t)n || w1 > (uint64_t)n * 24 + 64) return ORC_ERR_CORRUPT;
  if (!(s > 0.0) || !isfinite(s)) return ORC_ERR_CORRUPT;
  const size_t vsz = dtype == 0 ? 8 : 4;
  layout_t L;
  make_layout(R1, R2, ngroups(n, C1), 0, nout1, 0, 0, vsz, w1, 0, 0, &L);
  if (L.total != total || total > size) return ORC_ERR_CORRUPT;
  uint16_t *sym = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)n);
  int st = ORC_OK;
  if (!sym) return ORC_ERR_OOM;
  if ((st = unpack_component(in, size, &L, 1, n, C1, R1, zr, lmax, w1, sym))) goto done;
  {
    uint64_t k = 0;
    uint32_t q = 0;
    for (int64_t i = 0; i < n; i++) {
      int32_t d;
      if (sym[i] == 0) {
        if (k >= nout1) { st = ORC_ERR_CORRUPT; goto done; }
        d = (int32_t)get_u32(in + L.out1 + 4 * k++);
      } else if (sym[i] == 2 * R1 - 1) {
        st = ORC_ERR_CORRUPT;
        goto done;
      } else {
        d = (int32_t)sym[i] - R1;
      }
      q += (uint32_t)d;
      const double xr = s * (double)(K + (int64_t)(int32_t)q);
      if (dtype == 0) ((double *)xout)[i] = xr;
      else ((float *)xout)[i] = (float)xr;
    }
    if (k != nout1) st = ORC_ERR_CORRUPT;
  }
done:
  free(sym);
  return st;
}
