/*
 * mcc.h -- C ABI of the GB300 (sm_103a) multi-component compressor for data on
 * unstructured triangle / tetrahedral meshes, after Gong et al., "A General
 * Framework for Error-controlled Unstructured Scientific Data Compression".
 *
 * The method (Sec. III-IV): vertex values x are approximated on a rectilinear
 * grid, x1 = f(x) (barycentric interpolation, Sec. IV-D); the residual
 * x2 = x - g(x1') at every vertex uses the decompressed grid x1' and the
 * bilinear / trilinear operator g (Sec. III: piecewise-linear g has
 * sum |a_j| = 1, so the bound splits as tau = tau1 + tau2); both components
 * are compressed by an error-bounded compressor C (here: dual quantisation,
 * N-D Lorenzo prediction for the grid, canonical Huffman for both;
 * Algorithm 3) and reconstructed as x' = g(x1') + x2' (Algorithm 4).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers (current device), owned by the
 *     caller; the library never frees or retains them past the call. Host
 *     pointers are plain C pointers, also caller owned.
 *   - Work is enqueued on the given stream; calls return after enqueueing
 *     unless documented to synchronise. No call allocates device memory
 *     except mcc_plan_create (the plan owns its tables until
 *     mcc_plan_destroy).
 *   - No exception, exit, abort or device trap crosses this boundary. Errors
 *     found on the host are returned at once; errors found on the device
 *     (range overflow, corrupt stream, capacity) are recorded in the
 *     workspace's status word and returned by the synchronising calls.
 *   - One call may use a workspace at a time: two calls in flight on the same
 *     workspace race.
 */
#ifndef MCC_H
#define MCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mcc_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  MCC_OK = 0,
  MCC_ERR_INVALID_ARG = 1, /* bad pointer, size, mesh index or parameter */
  MCC_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
  MCC_ERR_OOM = 3,         /* plan tables could not be allocated */
  MCC_ERR_RANGE = 4,       /* bound too small for the value range: a code would
                              overflow (node codes need range/(2 tau2) < 2^29,
                              grid codes |q1| < 2^27) */
  MCC_ERR_CORRUPT = 5,     /* stream fails validation (magic, version, sizes,
                              tables, codes); nothing read out of bounds */
  MCC_ERR_CAPACITY = 6,    /* output or workspace buffer too small */
  MCC_ERR_TIMEOUT = 7,     /* a bounded device wait gave up */
  MCC_ERR_UNSUPPORTED = 8  /* parameter outside what this build supports */
} mcc_status;

enum { MCC_F64 = 0, MCC_F32 = 1 };   /* value types */
enum { MCC_ABS = 0, MCC_REL = 1 };   /* bound modes: absolute, or x (max - min) */
enum { MCC_PRED_ZERO = 0, MCC_PRED_LEARNED = 1, MCC_PRED_AUTO = 2 };  /* residual predictor */
enum { MCC_LOOP_CLOSED = 0, MCC_LOOP_OPEN = 1 };  /* residual against g(x1') or g(x1) */
enum { MCC_F_BARYCENTRIC = 0, MCC_F_CLUSTER = 1 };   /* mesh -> grid operator f */
enum { MCC_G_MULTILINEAR = 0, MCC_G_NEAREST = 1 };   /* grid -> mesh operator g */
#define MCC_MODEL_BYTES 5736   /* learned-predictor blob */
#define MCC_MLP_PARAMS 5313    /* float parameters of the training network */

/* Unstructured mesh (Sec. IV-C input: vertex coordinates {p_i} and
 * connectivity {c_j}). Triangles for dim 2, tetrahedra for dim 3. */
typedef struct {
  int dim;                /* 2 or 3 */
  int64_t n_vertices;     /* >= 1 */
  const double *coords;   /* device, [n_vertices][dim], row major */
  int64_t n_cells;        /* >= 1 */
  const int32_t *cells;   /* device, [n_cells][dim + 1] vertex ids in [0, n_vertices) */
} mcc_mesh;

/* Rectilinear grid layout S (Sec. IV-C): n[d] points per axis (2..32768;
 * n[2] ignored for dim 2), corners lo/hi. If lo[d] >= hi[d] on any axis the
 * corners are the mesh bounding box (Grid_Init, Algorithm 1: min/max of the
 * vertex coordinates). */
typedef struct {
  int32_t n[3];
  double lo[3], hi[3];
} mcc_grid_spec;

/* Compression parameters. The error bound tau (absolute, or relative to the
 * value range max(x) - min(x); a constant field uses eb itself) splits into
 * tau1 = grid_fraction * tau for the grid component and tau2 = (1 -
 * grid_fraction) * tau for the residuals (Sec. III, tau1 + tau2 <= tau). */
typedef struct {
  int dtype;             /* MCC_F64 or MCC_F32 */
  int eb_mode;           /* MCC_ABS or MCC_REL */
  double eb;             /* > 0 */
  double grid_fraction;  /* in [0.001, 0.999] */
  int R1, R2;            /* quantisation radii: alphabets of 2R symbols, 4..2048 */
  int C1, C2;            /* symbols per lane chunk (32 lanes per group), 1..256 */
  int lmax;              /* Huffman code length limit, 1..24 */
  /* Residual predictor. MCC_PRED_ZERO: the method as published, the vertex
   * prediction is the interpolation g(x1'). MCC_PRED_LEARNED: a learned
   * correction p(corner codes, local coordinates) is added to g before the
   * vertex rounding (P = round(rho12 g + p), so the bound holds as before);
   * d_model is a device pointer (4-byte aligned) to an MCC_MODEL_BYTES blob
   * (see mcc_model_train), copied into every stream that uses it. An invalid
   * blob records MCC_ERR_INVALID_ARG on the device. MCC_PRED_AUTO: both
   * predictors run and the field keeps the one whose encoding is smaller:
   * code bits (sum over symbols of count x code length, each predictor with
   * the code book of its own histogram) plus 32 bits per escape, the raw
   * values and, for the learned one, the model; a tie keeps the plain one. */
  int predictor;
  const void *d_model;
  /* Residual reference (Algorithm 3). MCC_LOOP_CLOSED: x2 = x - g(x1'), the
   * interpolation of the decompressed grid, so the vertex error is the
   * residual's alone, |x - x'| <= tau2, and tau1 only trades rate between the
   * components. MCC_LOOP_OPEN: x2 = x - g(x1) with the grid component before
   * quantisation, as Algorithm 3 prints it; the grid's error reaches the
   * vertices and the bound is |x - x'| <= tau1 + tau2 <= tau (Sec. III),
   * checked at every vertex (violators are stored raw). The vertex code is
   * q2 = round(x / s2 - g(x1)) in FP64 and the reconstruction s2 (q2 +
   * g(x1')). Open loop takes MCC_PRED_ZERO only. */
  int loop;
  /* Operators (Sec. III-B, III-C). f, mesh -> grid: MCC_F_BARYCENTRIC, the
   * barycentric interpolation of the vertex codes in the simplex holding the
   * node; MCC_F_CLUSTER, the paper's cluster mean: the mean of the codes of
   * the vertices whose nearest node is the node (integer part, then the
   * remainder / count in FP32), a node no vertex is nearest to keeping the
   * fill value (the paper initialises x1 to 0). g, grid -> mesh:
   * MCC_G_MULTILINEAR, bilinear / trilinear interpolation over the vertex's
   * cell; MCC_G_NEAREST, the paper's nearest node m_k (the cell corner on the
   * near side of every midplane of the cell, half going up), P =
   * round((s1/s2) q1[m_k]). Both gs are linear with weights summing to 1, so
   * the bound holds for every combination. The nearest-node g takes
   * MCC_PRED_ZERO only (the learned predictor corrects the interpolation). */
  int f_op;
  int g_op;
  /* Zero-run stage (not in the paper; 0 off, 1 on): before the Huffman
   * coder, every maximal run of r zero symbols in a lane chunk (a Lorenzo
   * difference or residual of 0, symbol R) becomes the digits of r in
   * bijective base 2, least significant first (r = sum d_i 2^i, d_i in
   * {1, 2}; token 2R for a digit 1, 2R + 1 for a digit 2), and each code
   * book covers these 2R + 2 tokens. Lossless; it lifts the one bit per
   * symbol floor of a Huffman code where zeros dominate (loose bounds).
   * Stream flags bit 6; the two run tokens' code lengths sit at header
   * bytes 208..209 (grid component) and 210..211 (residual component).
   * Requires R <= 2047 (MCC_ERR_UNSUPPORTED) and 2R + 2 <= 2^lmax. */
  int zero_run;
} mcc_params;

typedef struct mcc_plan_s *mcc_plan;

typedef struct {
  int dim;
  int32_t n[3];
  double lo[3], h[3];
  int64_t n_vertices, n_grid;
  int64_t n_outside;     /* grid points in no simplex (filled with zero) */
} mcc_plan_info;

/* Defaults: F64, REL, eb 1e-4, grid_fraction 0.5, R1 = R2 = 512,
 * C1 = C2 = 128, lmax 24, MCC_PRED_ZERO, MCC_LOOP_CLOSED, MCC_F_BARYCENTRIC,
 * MCC_G_MULTILINEAR, zero_run 0. */
void mcc_params_default(mcc_params *p);

/* Build the mesh -> grid mapping once per mesh (Sec. IV-B: reused across
 * variables and timesteps; excluded from the compression ratio, Sec. IV-A).
 * Per grid point: the minimum-id simplex containing it and its barycentric
 * weights (points in no simplex take the value zero, as the hollow regions
 * of Fig. 1); per vertex: its grid cell and local coordinates. Synchronises
 * the stream. The plan allocates and owns its device tables. */
mcc_status mcc_plan_create(const mcc_mesh *mesh, const mcc_grid_spec *grid, mcc_stream stream,
                           mcc_plan *out);

/* Grid_Coarsen (Algorithm 2) on a plan of a uniform grid: every vertex
 * marks the grid nodes its g uses (g_op MCC_G_NEAREST: the nearest node, the
 * cell corner on the near side of every midplane from the plan's local
 * coordinates, half going up; MCC_G_MULTILINEAR: all 2^dim corners of its
 * cell), and a plane of the grid normal to axis d (a line in 2D) stays when
 * one of its nodes is marked. keep_out (HOST, n[0] + n[1] (+ n[2]) entries)
 * receives the kept indices of axis 0, then axis 1 (then axis 2), n_out[d]
 * their counts (n_out[2] = 1 in 2D). An axis that would keep fewer than two
 * planes keeps all of them. Synchronises the stream. MCC_ERR_INVALID_ARG
 * for a plan made with mcc_plan_create_kept or an unknown g_op. */
mcc_status mcc_grid_coarsen(mcc_plan plan, int g_op, int32_t *keep_out, int32_t n_out[3],
                            mcc_stream stream);

/* The plan of the kept planes of a uniform grid (Algorithm 2's updated
 * layout S): grid as for mcc_plan_create (the uniform base grid), keep a
 * HOST array of n_keep[0] + n_keep[1] (+ n_keep[2]) increasing base indices,
 * at least two per axis (mcc_grid_coarsen's output). Point i of axis d
 * lies at lo[d] + keep_d[i] h[d]: every grid point is a base grid point,
 * located and weighted as there; a vertex's cell lies between the kept
 * planes around it and its local coordinate is (t - k_c) / (k_(c+1) - k_c),
 * t = (p - lo) / h in base spacings. The compressor takes the plan like
 * any other (n_keep[d] points per axis); the stream records those counts,
 * so decompression takes the same plan. mcc_plan_get_info reports the kept
 * counts with the base corner and spacing. */
mcc_status mcc_plan_create_kept(const mcc_mesh *mesh, const mcc_grid_spec *grid,
                                const int32_t *keep, const int32_t n_keep[3], mcc_stream stream,
                                mcc_plan *out);

/* Grid_Init (Algorithm 1): a grid layout for the mesh. For each axis d the
 * spacing gs_d is the bottom k-th percentile, nearest rank (the
 * ceil(k/100 N)-th smallest), of |p_a,d - p_b,d| over every edge of every
 * cell (N = 3 n_cells edges in 2D, 6 n_cells in 3D; an edge shared by cells
 * counts once per cell); while (max_d - min_d) / gs_d >= gmax, k grows by
 * delta_pct (k carries over to the next axis, as the algorithm prints it).
 * Writes n[d] = ceil((max_d - min_d) / gs_d) + 1 points and the corners
 * lo = min, hi = max of the vertex coordinates to *out, ready for
 * mcc_plan_create. k_pct in (0, 100], delta_pct > 0, gmax in [2, 32767].
 * Synchronises the stream (the selection is host-driven, 8 passes per axis
 * over the edges). MCC_ERR_RANGE when even k = 100 leaves gmax or more
 * intervals; MCC_ERR_INVALID_ARG for invalid cells or a flat axis. */
mcc_status mcc_grid_init(const mcc_mesh *mesh, double k_pct, double delta_pct, int32_t gmax,
                         mcc_grid_spec *out, mcc_stream stream);
void mcc_plan_destroy(mcc_plan plan);
mcc_status mcc_plan_get_info(mcc_plan plan, mcc_plan_info *info);

/* Launch configuration of a plan's kernels (no counterpart in the paper;
 * chosen by timing, see the package's autotuner): the tile of the 2D grid
 * kernel (MCC_TILE_64x16 by default, MCC_TILE_32x32, MCC_TILE_128x8), the
 * blocks per SM and field of the vertex-streaming kernels (quantisation,
 * the 3D grid codes, residuals, reconstruction: 2 .. 32, or 0, the
 * default: one full wave of as many blocks as fit on the SMs at once), and
 * the fields per launch chain of the batched calls (1 .. 64; 0, the
 * default: as many as keep their gathered codes, 4 (n_grid + n_vertices)
 * bytes each, within half the L2 cache, at least 1; the workspace may limit
 * it further), and the tensor-core path of the learned predictor's network
 * (MCC_NET_MMA_SYNC, the default: warp-level mma.sync, each warp's 32
 * vertices kept in registers from layer to layer; MCC_NET_TCGEN05: one
 * 128-vertex tile per 128-thread CTA, tcgen05.mma with BF16 operands in
 * shared memory and FP32 accumulators in tensor memory, at most four CTAs
 * per SM; measured slower, kept selectable). Streams and decoded values
 * never depend on it (the network is integer-exact in any accumulation
 * order). Set it between calls (it is read when a call launches);
 * MCC_ERR_INVALID_ARG outside the ranges. */
typedef struct {
  int tile2d;
  int vertex_blocks_per_sm;
  int batch_fields;
  int net_path;
} mcc_tuning;
enum { MCC_TILE_64x16 = 0, MCC_TILE_32x32 = 1, MCC_TILE_128x8 = 2 };
enum { MCC_NET_MMA_SYNC = 0, MCC_NET_TCGEN05 = 1 };
mcc_status mcc_plan_set_tuning(mcc_plan plan, const mcc_tuning *tuning);
mcc_status mcc_plan_get_tuning(mcc_plan plan, mcc_tuning *tuning);

/* Copy the plan tables to caller buffers (device pointers, any may be NULL):
 * vid [(dim+1)][n_grid] int32 (vid[0][j] = -1 outside the mesh), lam
 * [dim][n_grid] u16 (weights of vertices 1..dim in 2^-15 units), cell
 * [n_vertices] u32 (linear index of the cell's lower corner), frac
 * [dim][n_vertices] u16 (local coordinates in 2^-15 units). */
mcc_status mcc_plan_copy_tables(mcc_plan plan, int32_t *d_vid, uint16_t *d_lam, uint32_t *d_cell,
                                uint16_t *d_frac, mcc_stream stream);

/* Workspace bytes needed by mcc_compress / mcc_decompress for this plan. */
mcc_status mcc_workspace_size(mcc_plan plan, const mcc_params *p, size_t *compress_bytes,
                              size_t *decompress_bytes);

/* Upper bound of the compressed size for any field on this plan. */
mcc_status mcc_compress_bound(mcc_plan plan, const mcc_params *p, size_t *max_bytes);

/* Algorithm 3 (closed loop): compress n_vertices values of p->dtype at
 * d_values into d_out (capacity bytes, 8-byte aligned). The stream's size
 * is written to its header (bytes 184..191, u64) and to the workspace. If
 * out_size is non-NULL the call synchronises the stream and returns the size
 * together with any device-side error; otherwise it returns after enqueueing
 * (read the result later with mcc_workspace_result). */
mcc_status mcc_compress(mcc_plan plan, const void *d_values, const mcc_params *p,
                        void *d_workspace, size_t workspace_bytes, void *d_out, size_t capacity,
                        size_t *out_size, mcc_stream stream);

/* Algorithm 4: reconstruct x' = g(x1') + x2' at every vertex into d_values
 * (n_vertices values of type dtype, which must equal the stream's). The
 * stream (in_bytes at d_in, 4-byte aligned) is validated on the device: a
 * corrupt or mismatched stream records MCC_ERR_CORRUPT and nothing is read
 * or written out of bounds. If sync is nonzero the call synchronises and
 * returns device-side errors. */
mcc_status mcc_decompress(mcc_plan plan, const void *d_in, size_t in_bytes, void *d_values,
                          int dtype, void *d_workspace, size_t workspace_bytes, int sync,
                          mcc_stream stream);

/* Batched form of Algorithms 3 and 4 for many variables / timesteps on one
 * mesh (Sec. IV-B: the mapping is computed once and reused across variables
 * and timesteps). Field f is compressed from d_values[f] (a HOST array of n
 * device pointers) with per_field[f] (a host array; eb_mode, eb,
 * grid_fraction, predictor, d_model, loop, f_op, g_op and zero_run may differ per
 * field; dtype, R1, R2, C1, C2 and lmax must equal per_field[0]'s) into the
 * slot d_out + f * slot_bytes (slot_bytes a multiple of 8 and >=
 * mcc_compress_bound). Fields run in launch chains of up to 64 whose kernels
 * carry a field dimension, so latency-bound stages (code books, decode
 * tables, Huffman decoding) of different fields overlap and the fields share
 * plan tiles in L2. The workspace holds one compression workspace
 * (mcc_workspace_size) per field of a chain: workspace_bytes / that size
 * fields per chain, at least one. If out_sizes (host, n entries) is
 * non-NULL the call synchronises and fills it; device-side errors are then
 * returned (the first one found). */
mcc_status mcc_compress_batch(mcc_plan plan, int n, const void *const *d_values,
                              const mcc_params *per_field, void *d_workspace,
                              size_t workspace_bytes, void *d_out, size_t slot_bytes,
                              size_t *out_sizes, mcc_stream stream);

/* Batched Algorithm 4: field f decodes in_bytes[f] (host array) bytes at
 * d_in + f * slot_bytes into d_values[f] (host array of n device pointers,
 * n_vertices values of dtype each). The workspace holds one decompression
 * workspace per field of a chain of up to 64. If sync is nonzero the call
 * synchronises and returns the first device-side error. */
mcc_status mcc_decompress_batch(mcc_plan plan, int n, const void *d_in, size_t slot_bytes,
                                const size_t *in_bytes, void *const *d_values, int dtype,
                                void *d_workspace, size_t workspace_bytes, int sync,
                                mcc_stream stream);

/* ---- the paper's default baseline: the 1D coder on the vertex array ------
 * The paper compares the multi-component method with its "default": the
 * vertex values serialised in storage order into a 1D array and compressed
 * by the same compressor (Sec. V). Here: the grid component's coder in one
 * dimension, with no plan and no residual component: Q = round(x / s) - K,
 * differences delta_i = Q_i - Q_(i-1) (delta_0 = Q_0) coded as symbols
 * delta + R1 or escapes, canonical Huffman, the same lane-group stream
 * (header dim 1, n_x = n, flags = 32, or 32 | 64 with the zero-run stage).
 * The bin is s = 2 (tau - m)(1 - 2^-20)
 * with the margin m = 4 u64(M) (+ 2 u32(M) for FP32 values), u the value
 * type's spacing at M = max |x|: the roundings of x / s, of s (K + Q) and of
 * the cast stay inside it, so |x - x'| <= tau at every value and no value is
 * stored raw. MCC_ERR_RANGE when tau <= m or the codes exceed 2^29 bins.
 * Parameters as for the method (R1, C1, lmax, dtype, eb_mode, eb; R2 and C2
 * are recorded; zero_run applies); predictor, loop and operators must be the defaults. The
 * buffers follow the rules of mcc_compress / mcc_decompress. */
mcc_status mcc_workspace_size_1d(int64_t n, const mcc_params *p, size_t *compress_bytes,
                                 size_t *decompress_bytes);
mcc_status mcc_compress_bound_1d(int64_t n, const mcc_params *p, size_t *max_bytes);
mcc_status mcc_compress_1d(const void *d_values, int64_t n, const mcc_params *p,
                           void *d_workspace, size_t workspace_bytes, void *d_out,
                           size_t capacity, size_t *out_size, mcc_stream stream);
mcc_status mcc_decompress_1d(const void *d_in, size_t in_bytes, void *d_values, int64_t n,
                             int dtype, void *d_workspace, size_t workspace_bytes, int sync,
                             mcc_stream stream);

/* Decompression without any device allocation (the paper has no counterpart;
 * this serves callers that cannot call cudaMalloc, e.g. code that must stay
 * inside a memory budget owned by another allocator, or a plugin handed only
 * its input and output buffers). Same result as mcc_decompress; the scratch
 * memory is a fixed array inside this library's device image of
 * mcc_static_scratch_bytes() bytes (32 MiB) per device, held by every GPU
 * that loads the library until the process exits. Plans whose decompression
 * workspace (mcc_workspace_size) exceeds it get MCC_ERR_CAPACITY. Every call
 * looks up the array's device address in the current context (so a reset
 * device never sees a stale one); the first call on a device may load the
 * library's device code: make it before any stream capture. All calls on a
 * device share the array and leave its contents behind: calls whose GPU work
 * overlaps race. */
mcc_status mcc_decompress_static(mcc_plan plan, const void *d_in, size_t in_bytes, void *d_values,
                                 int dtype, int sync, mcc_stream stream);
size_t mcc_static_scratch_bytes(void);

/* Synchronise the stream and read the status (and, after a compression, the
 * stream size; may be NULL) that the last call recorded in the workspace. */
mcc_status mcc_workspace_result(const void *d_workspace, mcc_stream stream, size_t *out_size);

/* ---- executable graphs of asynchronous calls ----------------------------
 * No counterpart in the paper: the batching of many variables and timesteps
 * on one plan (each a fixed sequence of launches) replayed as one CUDA graph.
 * mcc_graph_begin starts recording the calls made on a NON-default stream
 * (captured in this thread only); every call in between must be
 * asynchronous (sync = 0, out_sizes = NULL; a synchronising call invalidates
 * the recording and mcc_graph_end returns MCC_ERR_CUDA). mcc_graph_end
 * instantiates the recorded work into *out (owned by the caller, released
 * with mcc_graph_destroy); mcc_graph_launch replays it on a stream, with the
 * same device pointers, parameters and workspaces as recorded. Make one
 * uncaptured call of each kind first (the library sets kernel attributes on
 * first use). Errors: MCC_ERR_INVALID_ARG for the default stream, a nested
 * begin or an end without a begin; MCC_ERR_CUDA from the CUDA runtime. */
typedef struct mcc_graph_s *mcc_graph;
mcc_status mcc_graph_begin(mcc_stream stream);
mcc_status mcc_graph_end(mcc_stream stream, mcc_graph *out);
mcc_status mcc_graph_launch(mcc_graph graph, mcc_stream stream);
void mcc_graph_destroy(mcc_graph graph);

const char *mcc_status_string(mcc_status s);

/* ---- learned residual predictor: training ------------------------------
 * No counterpart in the paper (its predictor for the residual component is
 * the interpolation g alone). The correction network takes, per vertex, the
 * corner codes of its grid cell (differences from corner 000 in vertex bins,
 * scaled by 2^-sx and rounded to [-127, 127]; the level of corner 000 as a
 * fraction of the value range, rounded to 0..127) and its local coordinates
 * (rounded to 0..127), and runs two hidden layers of 64 ReLU units. The
 * stored model is integer (int8 weights, 8-bit activations, power-of-two
 * scales), so compressor and decompressor evaluate it bit for bit; it is
 * trained in floating point on the residuals the method itself generates:
 * target y = Q - rho12 g (the vertex code minus the interpolated prediction,
 * in vertex bins), so that the corrected prediction round(rho12 g + p)
 * leaves residual codes near zero. */
enum { MCC_LOSS_L2 = 0, MCC_LOSS_L1 = 1 };

typedef struct {
  int steps;                 /* Adam steps, 1..1e6 (default 1500) */
  int batch;                 /* samples per step, multiple of 128, <= 65536 (4096) */
  float lr, beta1, beta2, eps; /* Adam (2e-3, 0.9, 0.999, 1e-8) */
  int loss;                  /* MCC_LOSS_L1 (default) or MCC_LOSS_L2 */
  int64_t samples_per_field; /* vertices drawn (with replacement) per field (65536) */
  uint64_t seed;             /* sampling, minibatch and initialisation seed (1) */
} mcc_train_cfg;

void mcc_train_cfg_default(mcc_train_cfg *cfg);

/* Device workspace bytes for mcc_model_train with n training fields. */
mcc_status mcc_train_workspace_size(mcc_plan plan, const mcc_params *p, const mcc_train_cfg *cfg,
                                    int n, size_t *bytes);

/* Train a model on n fields of this plan (d_fields: a HOST array of n device
 * pointers to n_vertices values of p->dtype; the bound parameters of p apply
 * to every field, its predictor and loop fields are ignored: the model serves
 * the closed loop). Steps: for each field
 * the front of the compression chain (bound split, vertex and grid codes),
 * then cfg->samples_per_field vertices drawn by a counter-based hash with
 * their features and targets; the feature exponent sx from the 99.9th
 * percentile of the corner differences; cfg->steps Adam steps on minibatches
 * of cfg->batch samples (tensor-core forward and backward passes, per-CTA
 * partial gradients summed in a fixed order: the run is deterministic);
 * calibration of the hidden-layer ranges over all samples; quantisation into
 * the MCC_MODEL_BYTES blob at d_model_out (device, 4-byte aligned). The
 * workspace (device, 256-byte aligned) must hold mcc_train_workspace_size
 * bytes. h_loss (host, cfg->steps floats, may be NULL) receives the
 * minibatch loss of every step. Synchronises the stream; returns the first
 * field's device-side error (e.g. MCC_ERR_RANGE) if any. */
mcc_status mcc_model_train(mcc_plan plan, int n, const void *const *d_fields, const mcc_params *p,
                           const mcc_train_cfg *cfg, void *d_workspace, size_t workspace_bytes,
                           void *d_model_out, float *h_loss, mcc_stream stream);

/* One evaluation of the training network's loss and gradient, the kernels
 * every training step runs (exposed for gradient checks). d_params: the
 * MCC_MLP_PARAMS float parameters, layout W1 [64][16], b1 [64], W2 [64][64],
 * b2 [64], W3 [64], b3 [1]; d_x: [B][16] inputs (16-byte aligned); d_y: [B]
 * targets; loss MCC_LOSS_L1 (mean absolute) or MCC_LOSS_L2 (mean squared
 * error). Writes d_grad (MCC_MLP_PARAMS floats, same layout) and *d_loss.
 * Tensor-core operands are rounded to bf16 (weights, inputs, hidden
 * activations, and the hidden-layer gradients where they multiply), sums are
 * FP32. Workspace: mcc_mlp_grad_workspace_size(B) bytes (device). */
size_t mcc_mlp_grad_workspace_size(int64_t B);
mcc_status mcc_mlp_grad(const float *d_params, const float *d_x, const float *d_y, int64_t B,
                        int loss, void *d_workspace, size_t workspace_bytes, float *d_grad,
                        float *d_loss, mcc_stream stream);

/* Post-training quantisation of the float parameters (the network trained on
 * the features times 2^-7) into a model blob at d_model (device,
 * MCC_MODEL_BYTES, 4-byte aligned): weight exponents a_l (largest with
 * |W_l| 2^a_l <= 127), activation exponents t_l (smallest with
 * max_z_l 2^-t_l <= 255), shifts s1 = t1 + a1 + 7, s2 = t2 + a2 - t1 (a shift
 * above 30 lowers the weight exponent, one below 1 raises the activation
 * exponent), e3 = t2 - a3; weights and biases rounded to nearest even. The
 * outcome (an mcc_status) is written to *d_status (device int). */
mcc_status mcc_mlp_quantize(int dim, int sx, const float *d_params, float max_z1, float max_z2,
                            void *d_model, int *d_status, mcc_stream stream);

/* Diagnostics (no counterpart in the paper): per-kernel device timing. While
 * enabled, every kernel that mcc_compress / mcc_decompress launches is
 * bracketed by a pair of CUDA events recorded on its stream; pairs stay
 * registered until mcc_profile_reset. mcc_profile_read synchronises on the
 * pairs and fills up to max_entries rows of (kernel name, milliseconds,
 * launches) summed over each pair's latest recording, sorted by name, and
 * returns the number of rows. When the bracketed launches were captured into
 * a CUDA graph, each replay re-records the captured pairs, so a read after a
 * replay returns that replay's times. Host-side state is process wide and
 * guarded by a mutex. */
void mcc_profile_enable(int on);
void mcc_profile_reset(void);
int mcc_profile_read(char (*names)[32], double *ms, long long *launches, int max_entries);

#ifdef __cplusplus
}
#endif
#endif /* MCC_H */
