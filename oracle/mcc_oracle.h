/*
 * mcc_oracle.h -- CPU oracle of the multi-component unstructured-mesh
 * compressor (Gong et al., Sec. III-IV, Algorithms 3 and 4).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, single-threaded C; slow on purpose. It
 * shares no code, header or table with the CUDA library; only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg may call it.
 * All arrays are host memory owned by the caller.
 */
#ifndef MCC_ORACLE_H
#define MCC_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (numerically equal to the library's, compared in tests) */
enum {
  ORC_OK = 0, ORC_ERR_INVALID_ARG = 1, ORC_ERR_CUDA = 2, ORC_ERR_OOM = 3,
  ORC_ERR_RANGE = 4, ORC_ERR_CORRUPT = 5, ORC_ERR_CAPACITY = 6,
  ORC_ERR_TIMEOUT = 7, ORC_ERR_UNSUPPORTED = 8
};

/* ---- plan (mesh -> grid mapping) ---------------------------------------- */
typedef struct {
  int dim;                 /* 2 or 3 */
  int32_t n[3];            /* grid points per axis (n[2] = 1 in 2D) */
  double lo[3], h[3], inv_h[3];
  /* Grid_Coarsen (Algorithm 2): the kept planes of a uniform base grid with
   * corner lo and spacing h, as increasing base indices keep[d][0 .. n[d]);
   * NULL keeps every plane (the uniform grid itself). Point i along axis d
   * lies at lo[d] + keep[d][i] * h[d]. */
  const int32_t *keep[3];
} orc_grid;

/* Grid_Init (Algorithm 1): points per axis from the bottom k-th percentile
 * of the cells' edge extents along the axis, k raised by delta while the
 * axis would have gmax or more intervals; corners from the vertices'
 * min / max (see the definition in mcc_oracle.c). */
int orc_grid_init(int dim, int64_t n_v, const double *coords, int64_t n_c, const int32_t *cells,
                  double k_pct, double delta_pct, int32_t gmax, int32_t n_out[3], double lo[3],
                  double hi[3], double gs_out[3]);

/* Grid_Coarsen (Algorithm 2) on a uniform grid g and its vertex tables
 * (cell, frac from orc_plan_tables): every vertex marks the grid nodes its
 * g uses (g_op 1, nearest node: the cell corner on the near side of every
 * midplane; g_op 0, multilinear: all 2^dim corners of its cell); a plane
 * (line in 2D) of the grid normal to axis d at index k is kept when one of
 * its nodes is marked. keep_out[d] (n[d] entries each) receives the kept
 * indices, n_out[d] their count. An axis that would keep fewer than two
 * planes keeps them all. */
int orc_grid_coarsen(const orc_grid *g, int64_t n_v, const uint32_t *cell, const uint16_t *frac,
                     int g_op, int32_t *keep_out[3], int32_t n_out[3]);

/* Resolve the grid: lo/hi given, or the mesh bounding box when lo >= hi on
 * any axis (Sec. IV-C: corners from the vertex min / max). */
int orc_grid_resolve(int dim, int64_t n_v, const double *coords,
                     const int32_t n[3], const double lo[3], const double hi[3],
                     orc_grid *g);

/* Inside test of one grid point against one simplex; returns 1 when the point
 * lies in the simplex (FP32 pre-filter, then FP64 barycentric test) and writes
 * the FP64 barycentric coordinates lam[0..dim]. */
int orc_point_in_simplex(const orc_grid *g, const double *coords, const int32_t *cell,
                         const int32_t idx[3], double lam[4]);

/* Owner (minimum simplex id containing the point, -1 if none) of every grid
 * point. brute = 1: every simplex against every point; brute = 0: each
 * simplex against the grid points of its bounding box. */
int orc_locate(const orc_grid *g, int64_t n_v, const double *coords, int64_t n_c,
               const int32_t *cells, int brute, int32_t *owner);

/* Plan tables from owners: per grid point vid[(dim+1)][n_g] (vid[0] = -1 for
 * points outside the mesh) and lam[dim][n_g] (u16, 2^-15 units); per vertex
 * cell[n_v] and frac[dim][n_v] (u16, 2^-15 units). lam64 (optional, may be
 * NULL) receives the FP64 barycentric coordinates [(dim+1)][n_g]. */
int orc_plan_tables(const orc_grid *g, int64_t n_v, const double *coords,
                    const int32_t *cells, const int32_t *owner,
                    int32_t *vid, uint16_t *lam, double *lam64,
                    uint32_t *cell, uint16_t *frac);

/* ---- compression --------------------------------------------------------- */
typedef struct {
  int dtype;          /* 0 = float64, 1 = float32 */
  int eb_mode;        /* 0 = absolute, 1 = relative to the value range */
  double eb;
  double grid_fraction; /* tau1 = f tau, tau2 = (1 - f) tau */
  int R1, R2;         /* quantisation radii (alphabet 2R) */
  int C1, C2;         /* symbols per lane chunk */
  int lmax;           /* Huffman length limit */
  const uint8_t *model; /* learned predictor (integer MLP blob) or NULL */
  size_t model_bytes;
  int auto_select;    /* with a model: keep the predictor whose encoding is smaller */
  int open_loop;      /* 1: residual against g(x1) with the unquantised x1 (Algorithm 3
                         as printed), bound tau1 + tau2; 0: against g(x1'), bound tau2 */
  int f_op;           /* mesh -> grid: 0 barycentric interpolation, 1 cluster mean
                         (mean of the vertices whose nearest node is j, Sec. III-C) */
  int g_op;           /* grid -> mesh: 0 bi/trilinear interpolation, 1 nearest node
                         (x2[k] = x[k] - x1[m_k], Sec. III-B) */
  int zero_run;       /* 1: lossless zero-run stage before the Huffman coder (not in
                         the paper): within each lane chunk a run of r zero symbols
                         becomes the digits of r in bijective base 2 */
} orc_params;

/* Per-field scalars derived from the values (Sec. III bound split). */
typedef struct {
  double lo, hi, M, tau, tau1, tau2, s1, s2, inv2;
  int64_t K, Qhi, fill_u, rho21_q, rho12_q;
  float rho21_f, rho12_f;
  int guard;
} orc_field;

int orc_field_params(const orc_params *p, int64_t n_v, const void *x, orc_field *f);

size_t orc_compress_bound(const orc_grid *g, int64_t n_v, const orc_params *p);

/* Compress x (n_v values of p->dtype) into out (capacity bytes).
 * Intermediate arrays are optional debug outputs (NULL to skip):
 * Q[n_v] node codes, q1[n_g] grid codes, sym1[n_g], sym2[n_v]. */
int orc_compress(const orc_grid *g, int64_t n_v, const int32_t *vid, const uint16_t *lam,
                 const uint32_t *cell, const uint16_t *frac, const void *x,
                 const orc_params *p, uint8_t *out, size_t capacity, size_t *out_size,
                 int32_t *Q, int32_t *q1, uint16_t *sym1, uint16_t *sym2);

/* Decompress a stream into x (n_v values of the stream's dtype). q1 optional. */
int orc_decompress(const orc_grid *g, int64_t n_v, const uint32_t *cell,
                   const uint16_t *frac, const uint8_t *in, size_t size, void *x,
                   int32_t *q1);

/* ---- building blocks exposed for the pin tests -------------------------- */
int orc_huffman_lengths(const uint64_t *count, int nsym, int lmax, uint8_t *len);
int orc_canonical_codes(const uint8_t *len, int nsym, uint32_t *code);
void orc_lorenzo(int dim, const int32_t n[3], const int32_t *q, int32_t *delta);
void orc_lorenzo_inverse(int dim, const int32_t n[3], const int32_t *delta, int32_t *q);

/* Learned predictor: for n vertices given their 8 corner codes (corners,
 * [n][8], order 000,100,010,110,001,101,011,111) and local coordinates (fr,
 * [n][3]), with s1/s2 (rho12_f) and the largest vertex code Qhi of the
 * field, the integer features ([n][16], may be NULL) and the correction p in
 * vertex bins. */
int orc_mlp_predict(int dim, const uint8_t *model, size_t model_bytes, const int32_t *corners,
                    const float *fr, float rho12_f, int64_t Qhi, int64_t n, int32_t *features,
                    float *p);

/* Loss (loss_kind 0: mean squared, 1: mean absolute error) and FP64
 * gradient of the float training network on a batch; rounding 1 rounds the
 * tensor-core operands to bfloat16 (see the definition in mcc_oracle.c). */
int orc_mlp_grad(const float *W1, const float *b1, const float *W2, const float *b2,
                 const float *W3, const float *b3, const float *X, const float *Y, int64_t B,
                 int loss_kind, int rounding, double *grad, double *loss);

/* Post-training quantisation of the float network (params in the gradient's
 * layout, trained on the features times 2^-7) into a model blob of
 * 5736 bytes, given the feature exponent sx and the calibration maxima of
 * relu(z1) and relu(z2). */
int orc_mlp_quantize(int dim, int sx, const float *params, float max_z1, float max_z2,
                     uint8_t *model);

/* ---- the paper's default: the same coder on the vertex array ----------- */
/* The vertex values in storage order as one 1D array (the paper's "default"
 * serialisation, Sec. V): Q = round(x / s) - K, 1D Lorenzo differences,
 * the grid component's coder; the bin keeps a margin for the rounding so
 * that no value is stored raw (see mcc_oracle.c). Header dim 1, flag bit 5. */
size_t orc_compress_bound_1d(int64_t n, const orc_params *p);
int orc_compress_1d(int64_t n, const void *x, const orc_params *p, uint8_t *out, size_t capacity,
                    size_t *out_size, int32_t *Q_dbg);
int orc_decompress_1d(int64_t n, const uint8_t *in, size_t size, void *xout);

#ifdef __cplusplus
}
#endif
#endif
