// plan.cu -- mesh -> grid mapping, built once per mesh and reused for every
// field (Gong et al., Sec. IV-B: "the mesh-grid mapping can be pre-computed";
// Sec. IV-C grid construction; excluded from the ratio, Sec. IV-A).
//
// Per grid point j: the minimum-id simplex that contains it (FP32 pre-filter,
// then the FP64 barycentric test with tolerance 1e-12) and its barycentric
// weights, stored as vertex ids + u16 weights of vertices 1..dim (the weight
// of vertex 0 is implied). Points in no simplex take the value zero (the
// hollow regions of Fig. 1). Per vertex: the lower corner of its grid cell and
// its local coordinates (u16, 2^-15 units).
//
// Point location rasterises every simplex over the grid points of its
// bounding box (thread per simplex) and keeps the minimum id with atomicMin,
// so the result does not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>

#include "common.cuh"

using namespace mcc;

struct mcc_plan_s {
  int dim;
  int kept;  // on kept planes of a uniform grid (Grid_Coarsen)
  int32_t n[3];
  double lo[3], h[3], inv_h[3];
  int64_t n_v, n_g, n_outside;
  int4 *vid;      // [n_g] vertex ids of the owning simplex (x = -1 outside)
  ushort4 *lam;   // [n_g] u16 weights of vertices 1..dim
  uint32_t *cell;
  uint16_t *frac;
  void *vrec;  // per vertex {cell, local coordinates} as one 8- (2D) or 16-byte (3D) record
  // a second stream for the component that does not wait on the other (the
  // grid coder beside the residual stage), its fork / join events, and the
  // mutex that keeps one call's fork and join together
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  std::mutex mu;
  int tile2d = MCC_TILE_64x16;  // launch configuration (mcc_plan_set_tuning)
  int vbps = 0;  // 0: one full wave of resident blocks
  int batch_fields = 0;
  int net_path = MCC_NET_MMA_SYNC;
};

namespace {

constexpr double kTol64 = 1e-12;
constexpr float kTol32 = 0.05f;
constexpr float kMargin32 = 0.01f;

// The grid of a plan: n[d] points per axis at lo + i h, or, with kept planes
// (Grid_Coarsen), at lo + keep[d][i] h on the uniform base grid (device
// arrays, increasing); top[d] is the largest base index.
struct GridDev {
  int dim;
  int32_t n[3];
  double lo[3], h[3], inv_h[3];
  float hf[3];
  const int32_t *keep[3];
  int32_t top[3];
};

// base-grid index of point i along axis d
__device__ __forceinline__ int32_t base_index(const GridDev &g, int d, int32_t i) {
  return g.keep[d] ? __ldg(g.keep[d] + i) : i;
}

// ---- barycentric coordinates (same operation order as the definition) ----
__device__ __forceinline__ void bary2_f(const float *a, const float *b, const float *c,
                                        const float *p, float *lam, float &den) {
  const float v0x = __fsub_rn(b[0], a[0]), v0y = __fsub_rn(b[1], a[1]);
  const float v1x = __fsub_rn(c[0], a[0]), v1y = __fsub_rn(c[1], a[1]);
  const float v2x = __fsub_rn(p[0], a[0]), v2y = __fsub_rn(p[1], a[1]);
  const float t1 = __fmul_rn(v0x, v1y), t2 = __fmul_rn(v1x, v0y);
  den = __fsub_rn(t1, t2);
  const float nb1 = __fmul_rn(v2x, v1y), nb2 = __fmul_rn(v1x, v2y);
  const float nc1 = __fmul_rn(v0x, v2y), nc2 = __fmul_rn(v2x, v0y);
  const float lb = __fdiv_rn(__fsub_rn(nb1, nb2), den);
  const float lc = __fdiv_rn(__fsub_rn(nc1, nc2), den);
  lam[0] = __fsub_rn(__fsub_rn(1.0f, lb), lc);
  lam[1] = lb;
  lam[2] = lc;
}

__device__ __forceinline__ void bary2_d(const double *a, const double *b, const double *c,
                                        const double *p, double *lam, double &den) {
  const double v0x = __dsub_rn(b[0], a[0]), v0y = __dsub_rn(b[1], a[1]);
  const double v1x = __dsub_rn(c[0], a[0]), v1y = __dsub_rn(c[1], a[1]);
  const double v2x = __dsub_rn(p[0], a[0]), v2y = __dsub_rn(p[1], a[1]);
  const double t1 = __dmul_rn(v0x, v1y), t2 = __dmul_rn(v1x, v0y);
  den = __dsub_rn(t1, t2);
  const double nb1 = __dmul_rn(v2x, v1y), nb2 = __dmul_rn(v1x, v2y);
  const double nc1 = __dmul_rn(v0x, v2y), nc2 = __dmul_rn(v2x, v0y);
  const double lb = __ddiv_rn(__dsub_rn(nb1, nb2), den);
  const double lc = __ddiv_rn(__dsub_rn(nc1, nc2), den);
  lam[0] = __dsub_rn(__dsub_rn(1.0, lb), lc);
  lam[1] = lb;
  lam[2] = lc;
}

template <typename T>
struct Ar;
template <>
struct Ar<float> {
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};
template <>
struct Ar<double> {
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

template <typename T>
__device__ __forceinline__ void cross3(T ux, T uy, T uz, T wx, T wy, T wz, T &rx, T &ry, T &rz) {
  using A = Ar<T>;
  rx = A::sub(A::mul(uy, wz), A::mul(uz, wy));
  ry = A::sub(A::mul(uz, wx), A::mul(ux, wz));
  rz = A::sub(A::mul(ux, wy), A::mul(uy, wx));
}
template <typename T>
__device__ __forceinline__ T dot3(T ux, T uy, T uz, T wx, T wy, T wz) {
  using A = Ar<T>;
  return A::add(A::add(A::mul(ux, wx), A::mul(uy, wy)), A::mul(uz, wz));
}

template <typename T>
__device__ __forceinline__ void bary3(const T *A_, const T *B, const T *C, const T *D, const T *P,
                                      T *lam, T &den) {
  using A = Ar<T>;
  const T v0x = A::sub(B[0], A_[0]), v0y = A::sub(B[1], A_[1]), v0z = A::sub(B[2], A_[2]);
  const T v1x = A::sub(C[0], A_[0]), v1y = A::sub(C[1], A_[1]), v1z = A::sub(C[2], A_[2]);
  const T v2x = A::sub(D[0], A_[0]), v2y = A::sub(D[1], A_[1]), v2z = A::sub(D[2], A_[2]);
  const T vpx = A::sub(P[0], A_[0]), vpy = A::sub(P[1], A_[1]), vpz = A::sub(P[2], A_[2]);
  T cx, cy, cz;
  cross3<T>(v1x, v1y, v1z, v2x, v2y, v2z, cx, cy, cz);
  den = dot3<T>(v0x, v0y, v0z, cx, cy, cz);
  const T nb = dot3<T>(vpx, vpy, vpz, cx, cy, cz);
  cross3<T>(vpx, vpy, vpz, v2x, v2y, v2z, cx, cy, cz);
  const T nc = dot3<T>(v0x, v0y, v0z, cx, cy, cz);
  cross3<T>(v1x, v1y, v1z, vpx, vpy, vpz, cx, cy, cz);
  const T nd = dot3<T>(v0x, v0y, v0z, cx, cy, cz);
  const T lb = A::div(nb, den), lc = A::div(nc, den), ld = A::div(nd, den);
  lam[0] = A::sub(A::sub(A::sub((T)1, lb), lc), ld);
  lam[1] = lb;
  lam[2] = lc;
  lam[3] = ld;
}

// FP32 pre-filter: 0 when the point is clearly outside the simplex.
template <int DIM>
__device__ __forceinline__ bool prefilter(const float (*vf)[3], const float *pf) {
  float l[4], den;
  if (DIM == 2) {
    bary2_f(vf[0], vf[1], vf[2], pf, l, den);
    if (den != 0.0f && (l[0] < -kTol32 || l[1] < -kTol32 || l[2] < -kTol32)) return false;
  } else {
    bary3<float>(vf[0], vf[1], vf[2], vf[3], pf, l, den);
    if (den != 0.0f &&
        (l[0] < -kTol32 || l[1] < -kTol32 || l[2] < -kTol32 || l[3] < -kTol32))
      return false;
  }
  return true;
}

template <int DIM>
__device__ __forceinline__ bool inside64(const double (*V)[3], const double *P, double *lam) {
  double den;
  if (DIM == 2) {
    bary2_d(V[0], V[1], V[2], P, lam, den);
    if (den == 0.0) return false;
    return lam[0] >= -kTol64 && lam[1] >= -kTol64 && lam[2] >= -kTol64;
  }
  bary3<double>(V[0], V[1], V[2], V[3], P, lam, den);
  if (den == 0.0) return false;
  return lam[0] >= -kTol64 && lam[1] >= -kTol64 && lam[2] >= -kTol64 && lam[3] >= -kTol64;
}

__device__ __forceinline__ uint16_t to_u16_unit(double v) {
  if (!(v > 0.0)) return 0;
  if (v >= 1.0) return 32768;
  return (uint16_t)rint(__dmul_rn(v, 32768.0));
}

// ---- kernels ---------------------------------------------------------------
__global__ void k_check_cells(const int32_t *cells, int64_t n, int64_t n_v, int *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = cells[i];
    if (v < 0 || v >= n_v) atomicExch(bad, 1);
  }
}

__global__ void k_bbox(const double *coords, int64_t n_v, int dim, unsigned long long *keys) {
  // keys[2d] = max of ~key (so ~result is the min key), keys[2d+1] = max key
  unsigned long long mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_v;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < dim; d++) {
      const unsigned long long k = order_key(coords[i * dim + d]);
      mn[d] = max(mn[d], ~k);
      mx[d] = max(mx[d], k);
    }
  for (int d = 0; d < dim; d++) {
    for (int o = 16; o; o >>= 1) {
      mn[d] = max(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
      mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&keys[2 * d], mn[d]);
      atomicMax(&keys[2 * d + 1], mx[d]);
    }
  }
}

// FP32 coordinates relative to the grid origin, 4 floats per vertex.
__global__ void k_rel32(const double *coords, int64_t n_v, GridDev g, float4 *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_v;
       i += (int64_t)gridDim.x * blockDim.x) {
    float r[3] = {0.f, 0.f, 0.f};
    for (int d = 0; d < g.dim; d++) r[d] = __double2float_rn(__dsub_rn(coords[i * g.dim + d], g.lo[d]));
    out[i] = make_float4(r[0], r[1], r[2], 0.f);
  }
}

// Binning of the simplices for the rasterisation: the grid tile (kBinTile^D
// base-grid cells) of each simplex's centroid, counts per tile, their
// exclusive prefix sums, and a scatter of the simplex ids (any order inside
// a tile). Tiles are numbered in Morton (Z) order of their coordinates, so
// consecutive bins, and the rasterising CTAs that take them in turn, cover
// compact blocks of the grid; x-fastest numbering when the Morton range of
// the tile counts would exceed kMortonMaxBins counters.
constexpr int kBinTile = 8;
constexpr int64_t kMortonMaxBins = (int64_t)1 << 24;

// bit interleaving: bits 0, 1, 2 .. of x to bits 0, 2, 4 .. (2D) or 0, 3, 6 .. (3D)
__host__ __device__ inline uint32_t spread2(uint32_t x) {
  x &= 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__host__ __device__ inline uint32_t spread3(uint32_t x) {
  x &= 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFu;
  x = (x | (x << 8)) & 0x0300F00Fu;
  x = (x | (x << 4)) & 0x030C30C3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}

template <int DIM>
__device__ __forceinline__ uint32_t centroid_tile(const int32_t *__restrict__ cells, int64_t t,
                                                  const float4 *__restrict__ rel, const GridDev &g,
                                                  const uint32_t (&nt)[3], bool morton) {
  float c[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k <= DIM; k++) {
    const float4 r = rel[cells[t * (DIM + 1) + k]];
    c[0] += r.x; c[1] += r.y; c[2] += r.z;
  }
  uint32_t ti[3] = {0, 0, 0};
  for (int d = 0; d < DIM; d++) {
    float u = c[d] / (float)(DIM + 1) / g.hf[d] / (float)kBinTile;
    if (!(u >= 0.f)) u = 0.f;  // also NaN
    ti[d] = u >= (float)(nt[d] - 1) ? nt[d] - 1 : (uint32_t)u;
  }
  if (morton)
    return DIM == 2 ? spread2(ti[0]) | (spread2(ti[1]) << 1)
                    : spread3(ti[0]) | (spread3(ti[1]) << 1) | (spread3(ti[2]) << 2);
  return ti[0] + nt[0] * (ti[1] + nt[1] * ti[2]);
}

template <int DIM>
__global__ void k_bin_count(const int32_t *__restrict__ cells, int64_t n_c,
                            const float4 *__restrict__ rel, GridDev g, uint32_t ntx, uint32_t nty,
                            uint32_t ntz, int morton, uint32_t *tile_of, unsigned int *count) {
  const uint32_t nt[3] = {ntx, nty, ntz};
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_c;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t tile = centroid_tile<DIM>(cells, t, rel, g, nt, morton != 0);
    tile_of[t] = tile;
    atomicAdd(count + tile, 1u);
  }
}

// Exclusive prefix sums of n counts in place, one block of 1024 threads
// (plan time; a few million tiles at most).
__global__ void __launch_bounds__(1024) k_bin_scan(unsigned int *count, int64_t n) {
  __shared__ unsigned int wsum[32];
  __shared__ unsigned int carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const unsigned int v = i < n ? count[i] : 0u;
    unsigned int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      const unsigned int sv = wsum[lane];
      unsigned int si = sv;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, si, o);
        if (lane >= o) si += t;
      }
      wsum[lane] = si - sv;  // exclusive over the warps
    }
    __syncthreads();
    const unsigned int c0 = carry;
    if (i < n) count[i] = c0 + wsum[w] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c0 + wsum[w] + incl;
    __syncthreads();
  }
}

__global__ void k_bin_scatter(const uint32_t *__restrict__ tile_of, int64_t n_c, unsigned int *cursor,
                              uint32_t *order) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_c;
       t += (int64_t)gridDim.x * blockDim.x)
    order[atomicAdd(cursor + tile_of[t], 1u)] = (uint32_t)t;
}

// Simplices in the order of `order` (binned by the grid tile of their
// centroid, so a warp rasterises neighbouring simplices: coherent loops and
// nearby atomics); the owner is the minimum id whatever the order.
template <int DIM>
__global__ void k_raster(const double *__restrict__ coords, const int32_t *__restrict__ cells,
                         int64_t n_c, const float4 *__restrict__ rel, GridDev g,
                         const uint32_t *__restrict__ order, unsigned int *owner) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n_c) return;
  const int64_t t = order[q];
  int32_t v[DIM + 1];
  float vf[4][3];
  for (int k = 0; k <= DIM; k++) {
    v[k] = cells[t * (DIM + 1) + k];
    const float4 r = rel[v[k]];
    vf[k][0] = r.x; vf[k][1] = r.y; vf[k][2] = r.z;
  }
  int32_t ilo[3] = {0, 0, 0}, ihi[3] = {0, 0, 0};
  for (int d = 0; d < DIM; d++) {
    float mn = vf[0][d], mx = vf[0][d];
    for (int k = 1; k <= DIM; k++) {
      mn = fminf(mn, vf[k][d]);
      mx = fmaxf(mx, vf[k][d]);
    }
    float a = __fsub_rn(__fdiv_rn(mn, g.hf[d]), kMargin32);
    float b = __fadd_rn(__fdiv_rn(mx, g.hf[d]), kMargin32);
    const float top = (float)g.top[d];
    if (!(a <= top) || !(b >= 0.0f)) return;
    a = ceilf(a);
    b = floorf(b);
    if (a < 0.0f) a = 0.0f;
    if (b > top) b = top;
    if (a > b) return;
    if (!g.keep[d]) {
      ilo[d] = (int32_t)a;
      ihi[d] = (int32_t)b;
      continue;
    }
    // kept planes with base index in [a, b]: the first at or above a, the
    // last at or below b
    const int32_t *kp = g.keep[d];
    int32_t lo_k = 0, hi_k = g.n[d];
    while (lo_k < hi_k) {
      const int32_t md = (lo_k + hi_k) >> 1;
      if (__int2float_rn(__ldg(kp + md)) < a) lo_k = md + 1;
      else hi_k = md;
    }
    const int32_t i0 = lo_k;
    lo_k = 0;
    hi_k = g.n[d];
    while (lo_k < hi_k) {
      const int32_t md = (lo_k + hi_k) >> 1;
      if (__int2float_rn(__ldg(kp + md)) <= b) lo_k = md + 1;
      else hi_k = md;
    }
    if (i0 > lo_k - 1) return;
    ilo[d] = i0;
    ihi[d] = lo_k - 1;
  }
  bool have64 = false;
  double V[4][3];
  const int64_t nx = g.n[0], ny = g.n[1];
  for (int32_t z = ilo[2]; z <= ihi[2]; z++)
    for (int32_t y = ilo[1]; y <= ihi[1]; y++)
      for (int32_t x = ilo[0]; x <= ihi[0]; x++) {
        const int64_t j = x + nx * (y + ny * (int64_t)z);
        if (owner[j] <= (unsigned int)t) continue;  // a smaller id already owns it
        const int32_t idx[3] = {x, y, z};
        int32_t bi[3] = {0, 0, 0};  // the point's index on the base grid
        for (int d = 0; d < DIM; d++) bi[d] = base_index(g, d, idx[d]);
        float pf[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < DIM; d++) pf[d] = __fmul_rn(__int2float_rn(bi[d]), g.hf[d]);
        if (!prefilter<DIM>(vf, pf)) continue;
        if (!have64) {
          for (int k = 0; k <= DIM; k++)
            for (int d = 0; d < 3; d++) V[k][d] = d < DIM ? coords[(int64_t)v[k] * DIM + d] : 0.0;
          have64 = true;
        }
        double P[3] = {0.0, 0.0, 0.0}, lam[4];
        for (int d = 0; d < DIM; d++) P[d] = __dadd_rn(g.lo[d], __dmul_rn((double)bi[d], g.h[d]));
        if (inside64<DIM>(V, P, lam)) atomicMin(owner + j, (unsigned int)t);
      }
}

template <int DIM>
__global__ void k_grid_tables(const double *__restrict__ coords, const int32_t *__restrict__ cells,
                              const unsigned int *__restrict__ owner, GridDev g, int64_t n_g,
                              int4 *vid, ushort4 *lam, unsigned long long *n_out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n_g) return;
  const unsigned int t = owner[j];
  if (t == 0xFFFFFFFFu) {
    vid[j] = make_int4(-1, 0, 0, 0);
    if (DIM == 3) lam[j] = make_ushort4(0, 0, 0, 0);
    atomicAdd(n_out, 1ull);
    return;
  }
  const int64_t nx = g.n[0], ny = g.n[1];
  const int32_t idx[3] = {(int32_t)(j % nx), (int32_t)((j / nx) % ny), (int32_t)(j / (nx * ny))};
  double V[4][3], P[3] = {0.0, 0.0, 0.0}, l[4];
  int32_t v4[4] = {0, 0, 0, 0};
  for (int k = 0; k <= DIM; k++) {
    const int32_t v = cells[(int64_t)t * (DIM + 1) + k];
    v4[k] = v;
    for (int d = 0; d < 3; d++) V[k][d] = d < DIM ? coords[(int64_t)v * DIM + d] : 0.0;
  }
  for (int d = 0; d < DIM; d++)
    P[d] = __dadd_rn(g.lo[d], __dmul_rn((double)base_index(g, d, idx[d]), g.h[d]));
  inside64<DIM>(V, P, l);
  unsigned short w[3] = {0, 0, 0};
  for (int k = 0; k < DIM; k++) w[k] = to_u16_unit(l[k + 1]);
  if (DIM == 2) {  // both weights in the record's fourth word
    vid[j] = make_int4(v4[0], v4[1], v4[2], (int)((unsigned int)w[0] | ((unsigned int)w[1] << 16)));
  } else {
    vid[j] = make_int4(v4[0], v4[1], v4[2], v4[3]);
    lam[j] = make_ushort4(w[0], w[1], w[2], 0);
  }
}

template <int DIM>
__global__ void k_node_tables(const double *__restrict__ coords, int64_t n_v, GridDev g,
                              uint32_t *cell, uint16_t *frac) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  int64_t ci[3] = {0, 0, 0};
  for (int d = 0; d < DIM; d++) {
    const double dd = __dsub_rn(coords[i * DIM + d], g.lo[d]);
    const double t = __dmul_rn(dd, g.inv_h[d]);  // in base-grid spacings
    int64_t c;
    double f;
    if (!g.keep[d]) {
      const double fl = floor(t);
      if (!(fl >= 0.0)) c = 0;
      else if (fl > (double)(g.n[d] - 2)) c = g.n[d] - 2;
      else c = (int64_t)fl;
      f = __dsub_rn(t, (double)c);
    } else {
      // kept planes: the last interval [k_c, k_(c+1)] starting at or below t
      // (the first one below k_0), f in that interval
      const int32_t *kp = g.keep[d];
      c = 0;
      int32_t lo_k = 0, hi_k = g.n[d] - 2;
      while (lo_k <= hi_k) {
        const int32_t md = (lo_k + hi_k) >> 1;
        if ((double)__ldg(kp + md) <= t) {
          c = md;
          lo_k = md + 1;
        } else {
          hi_k = md - 1;
        }
      }
      const int32_t k0 = __ldg(kp + c), k1 = __ldg(kp + c + 1);
      f = __ddiv_rn(__dsub_rn(t, (double)k0), (double)(k1 - k0));
    }
    ci[d] = c;
    frac[(int64_t)d * n_v + i] = to_u16_unit(f);
  }
  cell[i] = (uint32_t)(ci[0] + (int64_t)g.n[0] * (ci[1] + (int64_t)g.n[1] * ci[2]));
}

// One record per vertex of its cell and u16 local coordinates (the vertex
// kernels read it with one vector load).
template <int DIM>
__global__ void k_vertex_records(const uint32_t *__restrict__ cell, const uint16_t *__restrict__ frac,
                                 int64_t n_v, void *vrec) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_v;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned int fx = frac[i], fy = frac[n_v + i];
    if (DIM == 2) ((uint2 *)vrec)[i] = make_uint2(cell[i], fx | (fy << 16));
    else ((uint4 *)vrec)[i] = make_uint4(cell[i], fx | (fy << 16), frac[2 * n_v + i], 0u);
  }
}

// Grid_Coarsen (Algorithm 2): every vertex marks, per axis, the planes of
// the nodes its g uses (the nearest node, half going up; or both corners of
// its cell). mark holds n[0] + n[1] + n[2] bytes, axis by axis.
template <int DIM>
__global__ void k_coarsen_mark(const uint32_t *__restrict__ cell, const uint16_t *__restrict__ frac,
                               int64_t n_v, int32_t nx, int32_t ny, int32_t nz, int nearest,
                               unsigned char *mark) {
  const int64_t off[3] = {0, nx, (int64_t)nx + ny};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_v;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cell[i];
    const int64_t ci[3] = {c % nx, (c / nx) % ny, c / ((int64_t)nx * ny)};
    for (int d = 0; d < DIM; d++) {
      if (nearest) {
        mark[off[d] + ci[d] + (frac[(int64_t)d * n_v + i] >= 16384 ? 1 : 0)] = 1;
      } else {
        mark[off[d] + ci[d]] = 1;
        mark[off[d] + ci[d] + 1] = 1;
      }
    }
  }
  (void)nz;
}

inline unsigned int nblocks(int64_t n, int bs) {
  int64_t b = (n + bs - 1) / bs;
  return (unsigned int)(b < 1 ? 1 : b);
}

}  // namespace

// ---------------------------------------------------------------------------
// The plan of a uniform grid (keep == nullptr) or of kept planes of it
// (keep: host array of n_keep[0] + n_keep[1] (+ n_keep[2]) base indices).
static mcc_status plan_create(const mcc_mesh *mesh, const mcc_grid_spec *grid, const int32_t *keep,
                              const int32_t *n_keep, cudaStream_t stream, mcc_plan *out) {
  if (!out) return MCC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !grid) return MCC_ERR_INVALID_ARG;
  const int dim = mesh->dim;
  if (dim != 2 && dim != 3) return MCC_ERR_INVALID_ARG;
  if (mesh->n_vertices < 1 || mesh->n_vertices >= (int64_t)1 << 31 || mesh->n_cells < 1 ||
      mesh->n_cells >= (int64_t)1 << 31 || !mesh->coords || !mesh->cells)
    return MCC_ERR_INVALID_ARG;
  int64_t n_g = 1, n_keep_all = 0;
  bool use_bbox = false;
  for (int d = 0; d < dim; d++) {
    if (grid->n[d] < 2 || grid->n[d] > 32768) return MCC_ERR_INVALID_ARG;
    if (keep) {  // increasing base indices, at least two per axis
      if (!n_keep || n_keep[d] < 2 || n_keep[d] > grid->n[d]) return MCC_ERR_INVALID_ARG;
      const int32_t *k = keep + n_keep_all;
      if (k[0] < 0 || k[n_keep[d] - 1] >= grid->n[d]) return MCC_ERR_INVALID_ARG;
      for (int32_t i = 1; i < n_keep[d]; i++)
        if (k[i] <= k[i - 1]) return MCC_ERR_INVALID_ARG;
      n_keep_all += n_keep[d];
    }
    n_g *= keep ? n_keep[d] : grid->n[d];
    if (!(grid->lo[d] < grid->hi[d])) use_bbox = true;
  }
  if (n_g > ((int64_t)1 << 31)) return MCC_ERR_INVALID_ARG;
  const int64_t n_v = mesh->n_vertices, n_c = mesh->n_cells;

  mcc_plan_s *P = new (std::nothrow) mcc_plan_s();
  if (!P) return MCC_ERR_OOM;
  int *d_flag = nullptr;
  unsigned long long *d_keys = nullptr;
  unsigned int *d_owner = nullptr;
  float4 *d_rel = nullptr;
  int32_t *d_keep = nullptr;
  unsigned int *d_bins = nullptr;
  uint32_t *d_tile_of = nullptr, *d_order = nullptr;
  mcc_status st = MCC_OK;
  auto fail = [&](mcc_status s) {
    cudaFree(d_flag); cudaFree(d_keys); cudaFree(d_owner); cudaFree(d_rel); cudaFree(d_keep);
    cudaFree(d_bins); cudaFree(d_tile_of); cudaFree(d_order);
    if (P) {
      cudaFree(P->vid); cudaFree(P->lam); cudaFree(P->cell); cudaFree(P->frac);
      cudaFree(P->vrec);
      delete P;
    }
    return s;
  };
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&d_keys, 6 * sizeof(unsigned long long)) != cudaSuccess)
    return fail(MCC_ERR_OOM);
  if (keep && (cudaMalloc(&d_keep, sizeof(int32_t) * n_keep_all) != cudaSuccess ||
               cudaMemcpyAsync(d_keep, keep, sizeof(int32_t) * n_keep_all, cudaMemcpyHostToDevice,
                               stream) != cudaSuccess))
    return fail(MCC_ERR_OOM);
  cudaMemsetAsync(d_flag, 0, sizeof(int), stream);
  cudaMemsetAsync(d_keys, 0, 6 * sizeof(unsigned long long), stream);
  k_check_cells<<<1216, 256, 0, stream>>>(mesh->cells, n_c * (dim + 1), n_v, d_flag);
  if (use_bbox) k_bbox<<<608, 256, 0, stream>>>(mesh->coords, n_v, dim, d_keys);
  int h_flag = 0;
  unsigned long long h_keys[6] = {0, 0, 0, 0, 0, 0};
  if (cudaMemcpyAsync(&h_flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemcpyAsync(h_keys, d_keys, sizeof(h_keys), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return fail(MCC_ERR_CUDA);
  if (h_flag) return fail(MCC_ERR_INVALID_ARG);

  // grid corners and spacing: h = (hi - lo) / (n - 1), inv_h = 1 / h
  GridDev g;
  memset(&g, 0, sizeof(g));
  g.dim = dim;
  for (int d = 0; d < 3; d++) {
    if (d < dim) {
      double lo = grid->lo[d], hi = grid->hi[d];
      if (use_bbox) { lo = key_value(~h_keys[2 * d]); hi = key_value(h_keys[2 * d + 1]); }
      if (!(lo < hi) || !std::isfinite(lo) || !std::isfinite(hi)) return fail(MCC_ERR_INVALID_ARG);
      g.n[d] = grid->n[d];
      g.lo[d] = lo;
      g.h[d] = (hi - lo) / (double)(grid->n[d] - 1);
      g.inv_h[d] = 1.0 / g.h[d];
      g.top[d] = grid->n[d] - 1;
    } else {
      g.n[d] = 1; g.lo[d] = 0.0; g.h[d] = 1.0; g.inv_h[d] = 1.0;
    }
    g.hf[d] = (float)g.h[d];
  }
  if (keep) {  // the kept planes of the base grid just resolved
    int64_t o = 0;
    for (int d = 0; d < dim; d++) {
      g.keep[d] = d_keep + o;
      g.n[d] = n_keep[d];
      g.top[d] = keep[o + n_keep[d] - 1];
      o += n_keep[d];
    }
  }

  P->dim = dim;
  P->kept = keep ? 1 : 0;
  for (int d = 0; d < 3; d++) {
    P->n[d] = g.n[d]; P->lo[d] = g.lo[d]; P->h[d] = g.h[d]; P->inv_h[d] = g.inv_h[d];
  }
  P->n_v = n_v;
  P->n_g = n_g;
  if (cudaMalloc(&P->vid, sizeof(int4) * n_g) != cudaSuccess ||
      (dim == 3 && cudaMalloc(&P->lam, sizeof(ushort4) * n_g) != cudaSuccess) ||
      cudaMalloc(&P->cell, sizeof(uint32_t) * n_v) != cudaSuccess ||
      cudaMalloc(&P->frac, sizeof(uint16_t) * dim * n_v) != cudaSuccess ||
      cudaMalloc(&P->vrec, (dim == 2 ? sizeof(uint2) : sizeof(uint4)) * n_v) != cudaSuccess ||
      cudaMalloc(&d_owner, sizeof(unsigned int) * n_g) != cudaSuccess ||
      cudaMalloc(&d_rel, sizeof(float4) * n_v) != cudaSuccess)
    return fail(MCC_ERR_OOM);
  cudaMemsetAsync(d_owner, 0xFF, sizeof(unsigned int) * n_g, stream);
  cudaMemsetAsync(d_keys, 0, sizeof(unsigned long long), stream);
  k_rel32<<<nblocks(n_v, 256), 256, 0, stream>>>(mesh->coords, n_v, g, d_rel);
  // simplices binned by the base-grid tile of their centroid
  uint32_t ntb[3] = {1, 1, 1};
  for (int d = 0; d < dim; d++) ntb[d] = (uint32_t)((g.top[d] + kBinTile) / kBinTile);
  // Morton numbering: the bins span the next power of two of the largest
  // tile count in every dimension
  uint32_t p2 = 1;
  while (p2 < std::max(ntb[0], std::max(ntb[1], ntb[2]))) p2 <<= 1;
  const int64_t mbins = dim == 2 ? (int64_t)p2 * p2 : (int64_t)p2 * p2 * p2;
  const int morton = (dim == 2 ? p2 <= 65536u : p2 <= 1024u) && mbins <= kMortonMaxBins ? 1 : 0;
  const int64_t nbins = morton ? mbins : (int64_t)ntb[0] * ntb[1] * ntb[2];
  if (cudaMalloc(&d_bins, sizeof(unsigned int) * nbins) != cudaSuccess ||
      cudaMalloc(&d_tile_of, sizeof(uint32_t) * n_c) != cudaSuccess ||
      cudaMalloc(&d_order, sizeof(uint32_t) * n_c) != cudaSuccess)
    return fail(MCC_ERR_OOM);
  cudaMemsetAsync(d_bins, 0, sizeof(unsigned int) * nbins, stream);
  {
    const unsigned int nb = (unsigned int)std::min<int64_t>(nblocks(n_c, 256), 152 * 16);
    if (dim == 2)
      k_bin_count<2><<<nb, 256, 0, stream>>>(mesh->cells, n_c, d_rel, g, ntb[0], ntb[1], ntb[2],
                                            morton, d_tile_of, d_bins);
    else
      k_bin_count<3><<<nb, 256, 0, stream>>>(mesh->cells, n_c, d_rel, g, ntb[0], ntb[1], ntb[2],
                                            morton, d_tile_of, d_bins);
    k_bin_scan<<<1, 1024, 0, stream>>>(d_bins, nbins);
    k_bin_scatter<<<nb, 256, 0, stream>>>(d_tile_of, n_c, d_bins, d_order);
  }
  if (dim == 2) {
    k_raster<2><<<nblocks(n_c, 128), 128, 0, stream>>>(mesh->coords, mesh->cells, n_c, d_rel, g, d_order, d_owner);
    k_grid_tables<2><<<nblocks(n_g, 256), 256, 0, stream>>>(mesh->coords, mesh->cells, d_owner, g, n_g,
                                                          P->vid, P->lam, d_keys);
    k_node_tables<2><<<nblocks(n_v, 256), 256, 0, stream>>>(mesh->coords, n_v, g, P->cell, P->frac);
    k_vertex_records<2><<<nblocks(n_v, 256), 256, 0, stream>>>(P->cell, P->frac, n_v, P->vrec);
  } else {
    k_raster<3><<<nblocks(n_c, 128), 128, 0, stream>>>(mesh->coords, mesh->cells, n_c, d_rel, g, d_order, d_owner);
    k_grid_tables<3><<<nblocks(n_g, 256), 256, 0, stream>>>(mesh->coords, mesh->cells, d_owner, g, n_g,
                                                          P->vid, P->lam, d_keys);
    k_node_tables<3><<<nblocks(n_v, 256), 256, 0, stream>>>(mesh->coords, n_v, g, P->cell, P->frac);
    k_vertex_records<3><<<nblocks(n_v, 256), 256, 0, stream>>>(P->cell, P->frac, n_v, P->vrec);
  }
  unsigned long long n_out = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&n_out, d_keys, sizeof(n_out), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return fail(MCC_ERR_CUDA);
  P->n_outside = (int64_t)n_out;
  cudaFree(d_flag); cudaFree(d_keys); cudaFree(d_owner); cudaFree(d_rel); cudaFree(d_keep);
  cudaFree(d_bins); cudaFree(d_tile_of); cudaFree(d_order);
  // the second stream (without it every launch stays on the caller's stream)
  if (cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    if (P->side) cudaStreamDestroy(P->side);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    P->side = nullptr;
    P->ev_fork = P->ev_join = nullptr;
    cudaGetLastError();
  }
  *out = P;
  (void)st;
  return MCC_OK;
}

extern "C" mcc_status mcc_plan_create(const mcc_mesh *mesh, const mcc_grid_spec *grid,
                                      mcc_stream stream, mcc_plan *out) {
  return plan_create(mesh, grid, nullptr, nullptr, (cudaStream_t)stream, out);
}

extern "C" mcc_status mcc_plan_create_kept(const mcc_mesh *mesh, const mcc_grid_spec *grid,
                                           const int32_t *keep, const int32_t n_keep[3],
                                           mcc_stream stream, mcc_plan *out) {
  if (!keep) {
    if (out) *out = nullptr;
    return MCC_ERR_INVALID_ARG;
  }
  return plan_create(mesh, grid, keep, n_keep, (cudaStream_t)stream, out);
}

extern "C" mcc_status mcc_grid_coarsen(mcc_plan P, int g_op, int32_t *keep_out, int32_t n_out[3],
                                       mcc_stream stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!P || !keep_out || !n_out || P->kept) return MCC_ERR_INVALID_ARG;
  if (g_op != MCC_G_MULTILINEAR && g_op != MCC_G_NEAREST) return MCC_ERR_INVALID_ARG;
  const int dim = P->dim;
  const int64_t nm = (int64_t)P->n[0] + P->n[1] + (dim == 3 ? P->n[2] : 0);
  unsigned char *d_mark = nullptr;
  unsigned char *h_mark = new (std::nothrow) unsigned char[nm];
  if (!h_mark) return MCC_ERR_OOM;
  if (cudaMalloc(&d_mark, nm) != cudaSuccess) {
    delete[] h_mark;
    return MCC_ERR_OOM;
  }
  cudaMemsetAsync(d_mark, 0, nm, stream);
  const unsigned int nb = (unsigned int)std::min<int64_t>((P->n_v + 255) / 256, 152 * 8);
  const int nearest = g_op == MCC_G_NEAREST ? 1 : 0;
  if (dim == 2)
    k_coarsen_mark<2><<<nb, 256, 0, stream>>>(P->cell, P->frac, P->n_v, P->n[0], P->n[1], P->n[2],
                                             nearest, d_mark);
  else
    k_coarsen_mark<3><<<nb, 256, 0, stream>>>(P->cell, P->frac, P->n_v, P->n[0], P->n[1], P->n[2],
                                             nearest, d_mark);
  mcc_status st = MCC_OK;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h_mark, d_mark, nm, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    st = MCC_ERR_CUDA;
  if (st == MCC_OK) {
    int64_t o = 0, w = 0;
    for (int d = 0; d < 3; d++) {
      if (d >= dim) { n_out[d] = 1; continue; }
      int32_t m = 0;
      for (int32_t k = 0; k < P->n[d]; k++) m += h_mark[o + k];
      const bool all = m < 2;  // fewer than two planes cannot make a grid
      m = 0;
      for (int32_t k = 0; k < P->n[d]; k++)
        if (all || h_mark[o + k]) keep_out[w + m++] = k;
      n_out[d] = m;
      o += P->n[d];
      w += m;
    }
  }
  cudaFree(d_mark);
  delete[] h_mark;
  return st;
}

extern "C" void mcc_plan_destroy(mcc_plan P) {
  if (!P) return;
  cudaFree(P->vid); cudaFree(P->lam); cudaFree(P->cell); cudaFree(P->frac);
  cudaFree(P->vrec);
  if (P->side) cudaStreamDestroy(P->side);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  delete P;
}

extern "C" mcc_status mcc_plan_set_tuning(mcc_plan P, const mcc_tuning *t) {
  if (!P || !t) return MCC_ERR_INVALID_ARG;
  if (t->tile2d < MCC_TILE_64x16 || t->tile2d > MCC_TILE_128x8) return MCC_ERR_INVALID_ARG;
  if (t->vertex_blocks_per_sm != 0 && (t->vertex_blocks_per_sm < 2 || t->vertex_blocks_per_sm > 32))
    return MCC_ERR_INVALID_ARG;
  if (t->batch_fields < 0 || t->batch_fields > kMaxBatch) return MCC_ERR_INVALID_ARG;
  if (t->net_path != MCC_NET_MMA_SYNC && t->net_path != MCC_NET_TCGEN05) return MCC_ERR_INVALID_ARG;
  P->tile2d = t->tile2d;
  P->vbps = t->vertex_blocks_per_sm;
  P->batch_fields = t->batch_fields;
  P->net_path = t->net_path;
  return MCC_OK;
}

extern "C" mcc_status mcc_plan_get_tuning(mcc_plan P, mcc_tuning *t) {
  if (!P || !t) return MCC_ERR_INVALID_ARG;
  t->tile2d = P->tile2d;
  t->vertex_blocks_per_sm = P->vbps;
  t->batch_fields = P->batch_fields;
  t->net_path = P->net_path;
  return MCC_OK;
}

extern "C" mcc_status mcc_plan_get_info(mcc_plan P, mcc_plan_info *info) {
  if (!P || !info) return MCC_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->dim = P->dim;
  for (int d = 0; d < 3; d++) { info->n[d] = P->n[d]; info->lo[d] = P->lo[d]; info->h[d] = P->h[d]; }
  info->n_vertices = P->n_v;
  info->n_grid = P->n_g;
  info->n_outside = P->n_outside;
  return MCC_OK;
}

namespace {
// The grid tables in the ABI's layout, vid [(dim+1)][n_g] and lam [dim][n_g].
__global__ void k_tables_soa(const int4 *__restrict__ vid4, const ushort4 *__restrict__ lam4,
                             int64_t n_g, int dim, int32_t *vid, uint16_t *lam) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_g;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = vid4[j];
    const ushort4 l = dim == 3 ? lam4[j]
                               : make_ushort4((unsigned short)(v.w & 0xFFFF),
                                              (unsigned short)((unsigned int)v.w >> 16), 0, 0);
    const int32_t vv[4] = {v.x, v.y, v.z, v.w};
    const uint16_t ll[3] = {l.x, l.y, l.z};
    if (vid)
      for (int k = 0; k <= dim; k++) vid[k * n_g + j] = vv[k];
    if (lam)
      for (int k = 0; k < dim; k++) lam[k * n_g + j] = ll[k];
  }
}
}  // namespace

extern "C" mcc_status mcc_plan_copy_tables(mcc_plan P, int32_t *d_vid, uint16_t *d_lam,
                                           uint32_t *d_cell, uint16_t *d_frac, mcc_stream s) {
  if (!P) return MCC_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)s;
  const int dim = P->dim;
  cudaError_t e = cudaSuccess;
  if (d_vid || d_lam) {
    k_tables_soa<<<(unsigned int)std::min<int64_t>((P->n_g + 255) / 256, 152 * 16), 256, 0, stream>>>(
        P->vid, P->lam, P->n_g, dim, d_vid, d_lam);
    e = cudaGetLastError();
  }
  if (d_cell && e == cudaSuccess)
    e = cudaMemcpyAsync(d_cell, P->cell, sizeof(uint32_t) * P->n_v, cudaMemcpyDeviceToDevice, stream);
  if (d_frac && e == cudaSuccess)
    e = cudaMemcpyAsync(d_frac, P->frac, sizeof(uint16_t) * dim * P->n_v, cudaMemcpyDeviceToDevice, stream);
  return e == cudaSuccess ? MCC_OK : MCC_ERR_CUDA;
}

// internal accessor for the other translation units
PlanView mcc_plan_view(mcc_plan P) {
  PlanView v;
  v.dim = P->dim;
  v.nx = P->n[0]; v.ny = P->n[1]; v.nz = P->n[2];
  v.n_v = P->n_v; v.n_g = P->n_g;
  v.vid4 = P->vid; v.lam4 = P->lam; v.cell = P->cell; v.frac = P->frac; v.vrec = P->vrec;
  v.side = P->side;
  v.ev_fork = P->ev_fork;
  v.ev_join = P->ev_join;
  v.mu = P->side ? &P->mu : nullptr;
  v.tile2d = P->tile2d;
  v.vbps = P->vbps;
  v.batch_fields = P->batch_fields;
  v.net_path = P->net_path;
  return v;
}
