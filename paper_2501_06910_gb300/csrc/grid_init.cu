// grid_init.cu -- Grid_Init (Algorithm 1): the grid's points per axis from
// the mesh. Per axis d the spacing is the bottom k-th percentile (nearest
// rank) of |p_a,d - p_b,d| over every edge of every cell; k grows by delta
// while the axis would need gmax or more intervals. The percentile is an
// exact selection: the extents are non-negative doubles, so their bit
// patterns order like the values, and eight passes of 8-bit histograms over
// the edges (recomputed from the cells each pass, nothing stored) pin the
// rank's bit pattern from the top byte down.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"

using namespace mcc;

namespace {

__global__ void k_gi_check(const int32_t *cells, int64_t n, int64_t n_v, int *bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = cells[i];
    if (v < 0 || v >= n_v) atomicExch(bad, 1);
  }
}

// min / max per axis as ordered 64-bit keys (keys[2d] holds ~min key)
__global__ void k_gi_bbox(const double *coords, int64_t n_v, int dim, unsigned long long *keys) {
  unsigned long long mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_v;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < dim; d++) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(coords[i * dim + d]);
      const unsigned long long k = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
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

// Histogram of the byte at `shift` of the extents along axis d whose bits
// above it equal `prefix` (under `mask`).
template <int DIM>
__global__ void __launch_bounds__(256) k_gi_hist(const double *__restrict__ coords,
                                                 const int32_t *__restrict__ cells, int64_t n_c,
                                                 int d, int shift, unsigned long long mask,
                                                 unsigned long long prefix, unsigned int *hist) {
  __shared__ unsigned int sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  constexpr int NV = DIM + 1;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_c;
       c += (int64_t)gridDim.x * blockDim.x) {
    double p[NV];
#pragma unroll
    for (int a = 0; a < NV; a++) p[a] = __ldg(coords + (int64_t)__ldg(cells + c * NV + a) * DIM + d);
#pragma unroll
    for (int a = 0; a < NV; a++)
#pragma unroll
      for (int b = a + 1; b < NV; b++) {
        const unsigned long long key =
            (unsigned long long)__double_as_longlong(fabs(__dsub_rn(p[a], p[b])));
        if ((key & mask) == prefix) atomicAdd(&sh[(key >> shift) & 255u], 1u);
      }
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(hist + threadIdx.x, sh[threadIdx.x]);
}

double key_to_double(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double v;
  memcpy(&v, &b, 8);
  return v;
}

}  // namespace

extern "C" mcc_status mcc_grid_init(const mcc_mesh *mesh, double k_pct, double delta_pct,
                                    int32_t gmax, mcc_grid_spec *out, mcc_stream stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!mesh || !out) return MCC_ERR_INVALID_ARG;
  const int dim = mesh->dim;
  if (dim != 2 && dim != 3) return MCC_ERR_INVALID_ARG;
  if (mesh->n_vertices < 1 || mesh->n_vertices >= (int64_t)1 << 31 || mesh->n_cells < 1 ||
      mesh->n_cells >= (int64_t)1 << 31 || !mesh->coords || !mesh->cells)
    return MCC_ERR_INVALID_ARG;
  if (!(k_pct > 0.0 && k_pct <= 100.0) || !(delta_pct > 0.0) || gmax < 2 || gmax > 32767)
    return MCC_ERR_INVALID_ARG;
  const int64_t n_v = mesh->n_vertices, n_c = mesh->n_cells;
  const int64_t npair = dim == 2 ? 3 : 6, N = n_c * npair;
  int *d_bad = nullptr;
  unsigned long long *d_keys = nullptr;
  unsigned int *d_hist = nullptr;
  auto fail = [&](mcc_status s) {
    cudaFree(d_bad); cudaFree(d_keys); cudaFree(d_hist);
    return s;
  };
  if (cudaMalloc(&d_bad, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&d_keys, 6 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&d_hist, 256 * sizeof(unsigned int)) != cudaSuccess)
    return fail(MCC_ERR_OOM);
  cudaMemsetAsync(d_bad, 0, sizeof(int), stream);
  cudaMemsetAsync(d_keys, 0, 6 * sizeof(unsigned long long), stream);
  k_gi_check<<<1216, 256, 0, stream>>>(mesh->cells, n_c * (dim + 1), n_v, d_bad);
  k_gi_bbox<<<608, 256, 0, stream>>>(mesh->coords, n_v, dim, d_keys);
  int h_bad = 0;
  unsigned long long h_keys[6];
  if (cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemcpyAsync(h_keys, d_keys, sizeof(h_keys), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return fail(MCC_ERR_CUDA);
  if (h_bad) return fail(MCC_ERR_INVALID_ARG);
  mcc_grid_spec g;
  memset(&g, 0, sizeof(g));
  double k = k_pct;  // shared by the axes, as Algorithm 1 prints it
  const unsigned int blocks = (unsigned int)std::min<int64_t>((n_c + 255) / 256, 152 * 16);
  for (int d = 0; d < dim; d++) {
    const double mn = key_to_double(~h_keys[2 * d]), mx = key_to_double(h_keys[2 * d + 1]);
    if (!(mn < mx) || !std::isfinite(mn) || !std::isfinite(mx)) return fail(MCC_ERR_INVALID_ARG);
    double gs = 0.0, gn = 0.0;
    for (;;) {
      int64_t r = (int64_t)std::ceil(k / 100.0 * (double)N);  // rank (1-based) of the percentile
      if (r < 1) r = 1;
      if (r > N) r = N;
      unsigned long long prefix = 0, mask = 0, rem = (unsigned long long)r;
      for (int shift = 56; shift >= 0; shift -= 8) {
        unsigned int h[256];
        cudaMemsetAsync(d_hist, 0, sizeof(h), stream);
        if (dim == 2)
          k_gi_hist<2><<<blocks, 256, 0, stream>>>(mesh->coords, mesh->cells, n_c, d, shift, mask,
                                                    prefix, d_hist);
        else
          k_gi_hist<3><<<blocks, 256, 0, stream>>>(mesh->coords, mesh->cells, n_c, d, shift, mask,
                                                    prefix, d_hist);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h, d_hist, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
          return fail(MCC_ERR_CUDA);
        int b = 0;
        while (b < 255 && rem > h[b]) rem -= h[b++];
        if (rem > h[b]) return fail(MCC_ERR_CUDA);  // counts lost: cannot happen
        prefix |= (unsigned long long)b << shift;
        mask |= 0xFFull << shift;
      }
      double v;
      memcpy(&v, &prefix, 8);
      gs = v;
      gn = gs > 0.0 ? (mx - mn) / gs : INFINITY;
      if (gn < (double)gmax) break;
      if (k >= 100.0) return fail(MCC_ERR_RANGE);
      k = k + delta_pct;
      if (k > 100.0) k = 100.0;
    }
    g.n[d] = (int32_t)std::ceil(gn) + 1;
    g.lo[d] = mn;
    g.hi[d] = mx;
  }
  if (dim == 2) g.n[2] = 1;
  cudaFree(d_bad); cudaFree(d_keys); cudaFree(d_hist);
  *out = g;
  return MCC_OK;
}
