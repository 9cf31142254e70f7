// train.cu -- training of the learned residual predictor on the GPU.
//
// The residuals the method itself generates are the training data: for every
// training field the front of the compression chain (bound split, vertex
// codes Q, grid codes q1) runs as usual, then k_sample draws vertices with a
// counter-based hash and records their features (corner-code differences in
// vertex bins, local coordinates, level of corner 000) and their target
// y = Q - rho12 g, the residual in vertex bins that the network's output is
// added against. The feature exponent sx puts the 99.9th percentile of the
// corner differences at the top of the 8-bit input range.
//
// The float network (inputs x = X 2^-7, X the integer features; 64-64 ReLU;
// one output) trains with Adam on FP32 master weights. k_grad evaluates one
// minibatch on the tensor cores (bf16 mma.sync m16n8k16, FP32 accumulation):
// the forward pass, the backward pass through both hidden layers, and the
// weight gradients as products over the batch (gW2 = da2^T a1, gW1 = da1^T x);
// every CTA writes its partial gradient, and k_adam sums the partials in CTA
// order, so a run is deterministic. Operands of every product are rounded to
// bf16 (weights, x, a1, a2, da2, da1), the bias gradients and gW3 are FP32
// sums of unrounded values -- the rounding the oracle's gradient models.
//
// After training, k_grad in calibration mode takes the maxima of relu(z1) and
// relu(z2) over the samples and k_quantize turns the float network into the
// integer model (power-of-two scales, int8 weights, 8-bit activations).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "predictor.cuh"
#include "workspace.cuh"

using namespace mcc;

namespace {

// float parameter layout (the oracle's gradient layout)
constexpr int oW1 = 0, oB1 = 1024, oW2 = 1088, oB2 = 5184, oW3 = 5248, oB3 = 5312, kNP = 5313;
constexpr int kPartial = kNP + 1;  // + loss
constexpr int kRows = 128;         // samples per k_grad CTA (4 warps x 32)

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t hash3(uint64_t seed, uint64_t a, uint64_t b) {
  return mix64(mix64(mix64(seed) ^ a) ^ b);
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }
__device__ __forceinline__ double pow2d(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// ---------------------------------------------------------------------------
// sampling
// ---------------------------------------------------------------------------
struct SampleArgs {
  PlanView pv;
  const int *Q, *q1;
  const Status *st;
  float *X;  // [S][16]: raw features (corner differences unscaled)
  float *Y;  // [S]
  int64_t S;
  uint64_t seed;
  int field;
};

template <int DIM>
__global__ void __launch_bounds__(256) k_sample(const __grid_constant__ SampleArgs A) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= A.S) return;
  const PlanView &pv = A.pv;
  float *x = A.X + s * kK;
  if (A.st->err) {  // a field the front stage rejected contributes nothing
#pragma unroll
    for (int k = 0; k < kK; k++) x[k] = 0.0f;
    A.Y[s] = 0.0f;
    return;
  }
  const FieldParams &f = A.st->f;
  const int64_t n = pv.n_v;
  const int64_t i = (int64_t)(hash3(A.seed, (uint64_t)A.field, (uint64_t)s) % (uint64_t)n);
  const uint32_t c = pv.cell[i];
  const float fx = __fmul_rn(__uint2float_rn(pv.frac[i]), 0x1p-15f);
  const float fy = __fmul_rn(__uint2float_rn(pv.frac[n + i]), 0x1p-15f);
  const float fz = DIM == 3 ? __fmul_rn(__uint2float_rn(pv.frac[2 * n + i]), 0x1p-15f) : 0.0f;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  float acc;
  const int c000 = interp_vertex<DIM>(A.q1, c, fx, fy, fz, nx, sxy, acc);
  long long hi;
  float t0;
  rescale_split(c000, acc, f.rho12_q, f.rho12_f, hi, t0);
  // target: the correction that makes the residual code zero
  float y = (float)__dsub_rn((double)((long long)A.Q[i] - hi), (double)t0);
  y = fminf(fmaxf(y, -1048576.0f), 1048576.0f);
  A.Y[s] = y;
  const int offs[8] = {0, 1, nx, nx + 1, (int)sxy, (int)sxy + 1, (int)sxy + nx, (int)sxy + nx + 1};
  const float rf = f.rho12_f;
#pragma unroll
  for (int k = 1; k < (1 << DIM); k++)
    x[k - 1] = __fmul_rn(__int2float_rn(wsub(A.q1[c + offs[k]], c000)), rf);
  const float fr[3] = {fx, fy, fz};
#pragma unroll
  for (int d = 0; d < DIM; d++) x[(1 << DIM) - 1 + d] = rintf(__fmul_rn(fr[d], 127.0f));
  const float linv = f.Qhi > 0 ? __fdiv_rn(127.0f, __ll2float_rn(f.Qhi)) : 0.0f;
  const float lv = rintf(__fmul_rn(__fmul_rn(__int2float_rn(c000), rf), linv));
  x[(1 << DIM) + DIM - 1] = fminf(fmaxf(lv, 0.0f), 127.0f);
#pragma unroll
  for (int k = (1 << DIM) + DIM; k < kK; k++) x[k] = 0.0f;
}

// histogram of the binary exponents of the nonzero corner differences
__global__ void k_exp_hist(const float *X, int64_t S, int ncd, unsigned int *hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < S * ncd;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = X[(e / ncd) * kK + e % ncd];
    if (v != 0.0f) atomicAdd(&h[(__float_as_uint(v) >> 23) & 255], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(hist + i, h[i]);
}

// sx: the 99.9th percentile exponent E maps to [2^6, 2^7)
__global__ void k_pick_sx(const unsigned int *hist, int *sx_out) {
  if (threadIdx.x | blockIdx.x) return;
  unsigned long long tot = 0;
  for (int i = 0; i < 256; i++) tot += hist[i];
  int sx = 0;
  if (tot) {
    const unsigned long long want = tot - tot / 1000;
    unsigned long long run = 0;
    int b = 0;
    for (; b < 256; b++) {
      run += hist[b];
      if (run >= want) break;
    }
    sx = (b - 127) - 6;
    sx = sx < -60 ? -60 : (sx > 60 ? 60 : sx);
  }
  *sx_out = sx;
}

// integer features (the inference's rounding) scaled by 2^-7
__global__ void k_finalize(float *X, int64_t S, int ncd, const int *sx_p) {
  const float sc = pow2f(-*sx_p);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < S * kK;
       e += (int64_t)gridDim.x * blockDim.x) {
    float v = X[e];
    if ((int)(e % kK) < ncd) v = fminf(fmaxf(rintf(__fmul_rn(v, sc)), -127.0f), 127.0f);
    X[e] = __fmul_rn(v, 0x1p-7f);
  }
}

// He-uniform initialisation from a counter-based hash; biases and the
// padding inputs start at zero; Adam moments zero
__global__ void k_init(float *w, float *m, float *v, int n_in, uint64_t seed) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kNP) return;
  float lim = 0.0f;
  if (k < oB1) lim = (k % kK) < n_in ? sqrtf(6.0f / (float)n_in) : 0.0f;
  else if (k >= oW2 && k < oB2) lim = sqrtf(6.0f / 64.0f);
  else if (k >= oW3 && k < oB3) lim = sqrtf(6.0f / 64.0f) * 0.25f;
  const float u = (float)(hash3(seed, 7u, (uint64_t)k) >> 40) * 0x1p-24f;
  w[k] = (2.0f * u - 1.0f) * lim;
  m[k] = 0.0f;
  v[k] = 0.0f;
}

// ---------------------------------------------------------------------------
// k_grad: one minibatch through the network and back (or, in calibration
// mode, the forward maxima) on the tensor cores
// ---------------------------------------------------------------------------
struct GradArgs {
  const float *w;      // [kNP] float parameters
  const float *X, *Y;  // samples [S][16] (already scaled by 2^-7), [S]
  int64_t S;
  int64_t B;           // rows of this evaluation
  int random;          // 1: row b is sample hash(seed, step, b) % S; 0: sample b
  int step;
  uint64_t seed;
  int loss;            // 0: squared, 1: absolute error
  float inv_b;         // 1 / B
  float *partial;      // [gridDim.x][kPartial] (gradient mode)
  int calib;           // 1: maxima of relu(z1), relu(z2) into zmax[2]
  unsigned int *zmax;
};

struct GradSmem {
  float w3[64], b1[64], b2[64];
  float cs[4][3][64];  // per-warp column sums: gb1, gb2, gW3
  float wsum[4][2];    // per-warp gb3 and loss
  float b3;
  uint16_t W1[64][24];   // [unit][input]
  uint16_t W2[64][72];   // [unit j][input i]
  uint16_t W2T[64][72];  // [input i][unit j]
  uint16_t W3[8][72];    // row 0 = W3
  uint16_t xs[4][32][24];
  uint16_t xT[16][136];
  uint16_t a1T[64][136];
  uint16_t da2T[64][136];
  uint16_t da1T[64][136];
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// round to bf16, nearest even (bit pattern)
__device__ __forceinline__ uint16_t bf(float v) {
  uint32_t b = __float_as_uint(v);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}
__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
  return (uint32_t)bf(lo) | ((uint32_t)bf(hi) << 16);
}
__device__ __forceinline__ float unbf(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }
__device__ __forceinline__ uint32_t ld32s(const uint16_t *p) { return *(const uint32_t *)p; }

__global__ void __launch_bounds__(128) k_grad(const __grid_constant__ GradArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GradSmem &S = *reinterpret_cast<GradSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, tq = lane & 3;
  // ---- parameters: bf16 operands, FP32 biases
  for (int e = tid; e < 64 * 16; e += 128) S.W1[e / 16][e % 16] = bf(A.w[oW1 + e]);
  for (int e = tid; e < 64 * 64; e += 128) {
    const uint16_t v = bf(A.w[oW2 + e]);
    S.W2[e / 64][e % 64] = v;
    S.W2T[e % 64][e / 64] = v;
  }
  for (int e = tid; e < 8 * 64; e += 128) S.W3[e / 64][e % 64] = e < 64 ? bf(A.w[oW3 + e]) : 0;
  if (tid < 64) {
    S.w3[tid] = unbf(bf(A.w[oW3 + tid]));
    S.b1[tid] = A.w[oB1 + tid];
    S.b2[tid] = A.w[oB2 + tid];
  }
  if (tid == 0) S.b3 = A.w[oB3];
  __syncthreads();

  float zm1 = 0.0f, zm2 = 0.0f;  // calibration maxima
  const int64_t ntiles = (A.B + kRows - 1) / kRows;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncwarp();  // the warp's staging rows are reused
    // ---- this lane's sample
    const int64_t b = tile * kRows + 32 * w + lane;
    const bool valid = b < A.B;
    float yl = 0.0f;
    {
      float xv[kK];
#pragma unroll
      for (int k = 0; k < kK; k++) xv[k] = 0.0f;
      if (valid) {
        const int64_t row = A.random ? (int64_t)(hash3(A.seed, (uint64_t)A.step, (uint64_t)b) %
                                                 (uint64_t)A.S)
                                     : b;
        const float4 *src = reinterpret_cast<const float4 *>(A.X + row * kK);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const float4 v = src[q];
          xv[4 * q] = v.x; xv[4 * q + 1] = v.y; xv[4 * q + 2] = v.z; xv[4 * q + 3] = v.w;
        }
        yl = A.Y[row];
      }
#pragma unroll
      for (int k = 0; k < kK; k += 2) {
        const uint32_t pr = bf2(xv[k], xv[k + 1]);
        *(uint32_t *)&S.xs[w][lane][k] = pr;
        S.xT[k][32 * w + lane] = (uint16_t)pr;
        S.xT[k + 1][32 * w + lane] = (uint16_t)(pr >> 16);
      }
    }
    __syncwarp();
    float csum[3][8][2];
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
      for (int nt = 0; nt < 8; nt++) csum[q][nt][0] = csum[q][nt][1] = 0.0f;
    float gb3 = 0.0f, lsum = 0.0f;
#pragma unroll 1
    for (int t = 0; t < 2; t++) {
      const int r0 = 16 * t + g, r1 = r0 + 8;      // rows within the warp
      const int R0 = 32 * w + r0, R1 = R0 + 8;     // rows within the CTA
      uint32_t a[4];
      a[0] = ld32s(&S.xs[w][r0][2 * tq]);
      a[1] = ld32s(&S.xs[w][r1][2 * tq]);
      a[2] = ld32s(&S.xs[w][r0][2 * tq + 8]);
      a[3] = ld32s(&S.xs[w][r1][2 * tq + 8]);
      const bool v0 = __shfl_sync(0xffffffffu, valid, r0), v1 = __shfl_sync(0xffffffffu, valid, r1);
      // layer 1
      float z[8][4];
      uint32_t m1 = 0, m2 = 0;
      uint32_t a2[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        z[nt][0] = z[nt][1] = z[nt][2] = z[nt][3] = 0.0f;
        mma_bf16(z[nt], a, ld32s(&S.W1[8 * nt + g][2 * tq]), ld32s(&S.W1[8 * nt + g][2 * tq + 8]));
        const int c0 = 8 * nt + 2 * tq;
        z[nt][0] += S.b1[c0]; z[nt][1] += S.b1[c0 + 1];
        z[nt][2] += S.b1[c0]; z[nt][3] += S.b1[c0 + 1];
        float r[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          if (z[nt][e] > 0.0f) m1 |= 1u << (4 * nt + e);
          r[e] = fmaxf(z[nt][e], 0.0f);
        }
        if (v0) zm1 = fmaxf(zm1, fmaxf(r[0], r[1]));
        if (v1) zm1 = fmaxf(zm1, fmaxf(r[2], r[3]));
        const uint32_t p01 = bf2(r[0], r[1]), p23 = bf2(r[2], r[3]);
        a2[nt >> 1][(nt & 1) ? 2 : 0] = p01;
        a2[nt >> 1][(nt & 1) ? 3 : 1] = p23;
        S.a1T[c0][R0] = (uint16_t)p01;
        S.a1T[c0 + 1][R0] = (uint16_t)(p01 >> 16);
        S.a1T[c0][R1] = (uint16_t)p23;
        S.a1T[c0 + 1][R1] = (uint16_t)(p23 >> 16);
      }
      // layer 2
      uint32_t a3[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        z[nt][0] = z[nt][1] = z[nt][2] = z[nt][3] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 4; kt++)
          mma_bf16(z[nt], a2[kt], ld32s(&S.W2[8 * nt + g][16 * kt + 2 * tq]),
                   ld32s(&S.W2[8 * nt + g][16 * kt + 2 * tq + 8]));
        const int c0 = 8 * nt + 2 * tq;
        z[nt][0] += S.b2[c0]; z[nt][1] += S.b2[c0 + 1];
        z[nt][2] += S.b2[c0]; z[nt][3] += S.b2[c0 + 1];
        float r[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
          if (z[nt][e] > 0.0f) m2 |= 1u << (4 * nt + e);
          r[e] = fmaxf(z[nt][e], 0.0f);
        }
        if (v0) zm2 = fmaxf(zm2, fmaxf(r[0], r[1]));
        if (v1) zm2 = fmaxf(zm2, fmaxf(r[2], r[3]));
        a3[nt >> 1][(nt & 1) ? 2 : 0] = bf2(r[0], r[1]);
        a3[nt >> 1][(nt & 1) ? 3 : 1] = bf2(r[2], r[3]);
      }
      if (A.calib) continue;
      // output and loss
      float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kt = 0; kt < 4; kt++)
        mma_bf16(o, a3[kt], ld32s(&S.W3[g][16 * kt + 2 * tq]), ld32s(&S.W3[g][16 * kt + 2 * tq + 8]));
      const int src = lane & ~3;
      const float p0 = __shfl_sync(0xffffffffu, o[0], src) + S.b3;
      const float p1 = __shfl_sync(0xffffffffu, o[2], src) + S.b3;
      const float e0 = p0 - __shfl_sync(0xffffffffu, yl, r0);
      const float e1 = p1 - __shfl_sync(0xffffffffu, yl, r1);
      float dp0, dp1;
      if (A.loss == 1) {
        dp0 = e0 > 0.0f ? A.inv_b : (e0 < 0.0f ? -A.inv_b : 0.0f);
        dp1 = e1 > 0.0f ? A.inv_b : (e1 < 0.0f ? -A.inv_b : 0.0f);
      } else {
        dp0 = 2.0f * e0 * A.inv_b;
        dp1 = 2.0f * e1 * A.inv_b;
      }
      if (!v0) dp0 = 0.0f;
      if (!v1) dp1 = 0.0f;
      if (tq == 0) {
        gb3 += dp0 + dp1;
        const float l0 = A.loss == 1 ? fabsf(e0) : e0 * e0, l1 = A.loss == 1 ? fabsf(e1) : e1 * e1;
        lsum += (v0 ? l0 : 0.0f) + (v1 ? l1 : 0.0f);
      }
      // back through layer 3 and the second ReLU
      uint32_t ad[4][4];
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        const int c0 = 8 * nt + 2 * tq;
        const float wa = S.w3[c0], wb = S.w3[c0 + 1];
        const float d00 = (m2 >> (4 * nt)) & 1 ? dp0 * wa : 0.0f;
        const float d01 = (m2 >> (4 * nt + 1)) & 1 ? dp0 * wb : 0.0f;
        const float d10 = (m2 >> (4 * nt + 2)) & 1 ? dp1 * wa : 0.0f;
        const float d11 = (m2 >> (4 * nt + 3)) & 1 ? dp1 * wb : 0.0f;
        csum[1][nt][0] += d00 + d10;
        csum[1][nt][1] += d01 + d11;
        const uint32_t h01 = a3[nt >> 1][(nt & 1) ? 2 : 0], h23 = a3[nt >> 1][(nt & 1) ? 3 : 1];
        csum[2][nt][0] += dp0 * unbf((uint16_t)h01) + dp1 * unbf((uint16_t)h23);
        csum[2][nt][1] += dp0 * unbf((uint16_t)(h01 >> 16)) + dp1 * unbf((uint16_t)(h23 >> 16));
        const uint32_t q01 = bf2(d00, d01), q23 = bf2(d10, d11);
        ad[nt >> 1][(nt & 1) ? 2 : 0] = q01;
        ad[nt >> 1][(nt & 1) ? 3 : 1] = q23;
        S.da2T[c0][R0] = (uint16_t)q01;
        S.da2T[c0 + 1][R0] = (uint16_t)(q01 >> 16);
        S.da2T[c0][R1] = (uint16_t)q23;
        S.da2T[c0 + 1][R1] = (uint16_t)(q23 >> 16);
      }
      // da1 = (da2 W2) * [z1 > 0]
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int kt = 0; kt < 4; kt++)
          mma_bf16(d, ad[kt], ld32s(&S.W2T[8 * nt + g][16 * kt + 2 * tq]),
                   ld32s(&S.W2T[8 * nt + g][16 * kt + 2 * tq + 8]));
#pragma unroll
        for (int e = 0; e < 4; e++)
          if (!((m1 >> (4 * nt + e)) & 1)) d[e] = 0.0f;
        const int c0 = 8 * nt + 2 * tq;
        csum[0][nt][0] += d[0] + d[2];
        csum[0][nt][1] += d[1] + d[3];
        S.da1T[c0][R0] = bf(d[0]);
        S.da1T[c0 + 1][R0] = bf(d[1]);
        S.da1T[c0][R1] = bf(d[2]);
        S.da1T[c0 + 1][R1] = bf(d[3]);
      }
    }
    if (A.calib) continue;
    // ---- per-warp column sums (reduced over the 8 row groups)
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
      for (int nt = 0; nt < 8; nt++)
#pragma unroll
        for (int e = 0; e < 2; e++) {
          float v = csum[q][nt][e];
          v += __shfl_xor_sync(0xffffffffu, v, 4);
          v += __shfl_xor_sync(0xffffffffu, v, 8);
          v += __shfl_xor_sync(0xffffffffu, v, 16);
          if (g == 0) S.cs[w][q][8 * nt + 2 * tq + e] = v;
        }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      gb3 += __shfl_xor_sync(0xffffffffu, gb3, o);
      lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if (lane == 0) { S.wsum[w][0] = gb3; S.wsum[w][1] = lsum; }
    __syncthreads();
    // ---- weight gradients over the CTA's 128 rows: warp w owns units 16w..16w+15
    float *P = A.partial + (int64_t)blockIdx.x * kPartial;
    {
      float acc[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
      float acc1[2][4];
#pragma unroll
      for (int nt = 0; nt < 2; nt++) acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.0f;
      const int j0 = 16 * w + g;
#pragma unroll 2
      for (int kt = 0; kt < kRows / 16; kt++) {
        const int k0 = 16 * kt + 2 * tq;
        uint32_t fa[4];
        fa[0] = ld32s(&S.da2T[j0][k0]);
        fa[1] = ld32s(&S.da2T[j0 + 8][k0]);
        fa[2] = ld32s(&S.da2T[j0][k0 + 8]);
        fa[3] = ld32s(&S.da2T[j0 + 8][k0 + 8]);
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
          mma_bf16(acc[nt], fa, ld32s(&S.a1T[8 * nt + g][k0]), ld32s(&S.a1T[8 * nt + g][k0 + 8]));
        uint32_t fb[4];
        fb[0] = ld32s(&S.da1T[j0][k0]);
        fb[1] = ld32s(&S.da1T[j0 + 8][k0]);
        fb[2] = ld32s(&S.da1T[j0][k0 + 8]);
        fb[3] = ld32s(&S.da1T[j0 + 8][k0 + 8]);
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
          mma_bf16(acc1[nt], fb, ld32s(&S.xT[8 * nt + g][k0]), ld32s(&S.xT[8 * nt + g][k0 + 8]));
      }
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        const int i0 = 8 * nt + 2 * tq;
        P[oW2 + j0 * 64 + i0] = acc[nt][0];
        P[oW2 + j0 * 64 + i0 + 1] = acc[nt][1];
        P[oW2 + (j0 + 8) * 64 + i0] = acc[nt][2];
        P[oW2 + (j0 + 8) * 64 + i0 + 1] = acc[nt][3];
      }
#pragma unroll
      for (int nt = 0; nt < 2; nt++) {
        const int i0 = 8 * nt + 2 * tq;
        P[oW1 + j0 * 16 + i0] = acc1[nt][0];
        P[oW1 + j0 * 16 + i0 + 1] = acc1[nt][1];
        P[oW1 + (j0 + 8) * 16 + i0] = acc1[nt][2];
        P[oW1 + (j0 + 8) * 16 + i0 + 1] = acc1[nt][3];
      }
    }
    if (tid < 64) {
      P[oB1 + tid] = ((S.cs[0][0][tid] + S.cs[1][0][tid]) + S.cs[2][0][tid]) + S.cs[3][0][tid];
      P[oB2 + tid] = ((S.cs[0][1][tid] + S.cs[1][1][tid]) + S.cs[2][1][tid]) + S.cs[3][1][tid];
      P[oW3 + tid] = ((S.cs[0][2][tid] + S.cs[1][2][tid]) + S.cs[2][2][tid]) + S.cs[3][2][tid];
    } else if (tid == 64) {
      P[oB3] = ((S.wsum[0][0] + S.wsum[1][0]) + S.wsum[2][0]) + S.wsum[3][0];
      P[kNP] = ((S.wsum[0][1] + S.wsum[1][1]) + S.wsum[2][1]) + S.wsum[3][1];
    }
    __syncthreads();  // the next tile reuses the shared arrays
  }
  if (A.calib) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      zm1 = fmaxf(zm1, __shfl_xor_sync(0xffffffffu, zm1, o));
      zm2 = fmaxf(zm2, __shfl_xor_sync(0xffffffffu, zm2, o));
    }
    if (lane == 0) {
      atomicMax(A.zmax, __float_as_uint(zm1));
      atomicMax(A.zmax + 1, __float_as_uint(zm2));
    }
  }
}

// ---------------------------------------------------------------------------
// Adam on the FP32 master weights; gradient = partials summed in CTA order
// ---------------------------------------------------------------------------
struct AdamArgs {
  const float *partial;
  int nblocks;
  float *w, *m, *v;
  float lr, beta1, beta2, eps, c1, c2;  // c1 = 1 - beta1^t, c2 = 1 - beta2^t
  float inv_b;
  float *loss;  // this step's slot
};

__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamArgs A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kNP) return;
  float gsum = 0.0f;
  for (int b = 0; b < A.nblocks; b++) gsum += A.partial[(int64_t)b * kPartial + k];
  if (k == kNP) {
    *A.loss = gsum * A.inv_b;
    return;
  }
  const float m = A.beta1 * A.m[k] + (1.0f - A.beta1) * gsum;
  const float v = A.beta2 * A.v[k] + (1.0f - A.beta2) * gsum * gsum;
  A.m[k] = m;
  A.v[k] = v;
  const float mh = m / A.c1, vh = v / A.c2;
  A.w[k] -= A.lr * mh / (sqrtf(vh) + A.eps);
}

// gradient and loss of one evaluation (partials summed in CTA order)
__global__ void __launch_bounds__(256) k_reduce_grad(const float *partial, int nblocks, float inv_b,
                                                     float *grad, float *loss) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kNP) return;
  float gsum = 0.0f;
  for (int b = 0; b < nblocks; b++) gsum += partial[(int64_t)b * kPartial + k];
  if (k == kNP) *loss = gsum * inv_b;
  else grad[k] = gsum;
}

// ---------------------------------------------------------------------------
// post-training quantisation (one thread; a few thousand weights)
// ---------------------------------------------------------------------------
// largest a in [-40, 40] with maxw 2^a <= 127 (0 for a zero matrix)
__device__ int weight_exp(double maxw) {
  if (maxw == 0.0) return 0;
  int a = -40;
  while (a < 40 && maxw * pow2d(a + 1) <= 127.0) a++;
  return a;
}
// smallest t in [-60, 60] with maxz 2^-t <= 255
__device__ int act_exp(double maxz) {
  int t = -60;
  while (t < 60 && maxz * pow2d(-t) > 255.0) t++;
  return t;
}
__device__ int qbias(float b, int k) {
  double v = rint((double)b * pow2d(k));
  v = fmin(fmax(v, -4194304.0), 4194304.0);
  return (int)v;
}

struct QuantArgs {
  int dim;
  int sx;
  float max_z1, max_z2;
  const int *sx_p;             // device overrides (training) or NULL
  const unsigned int *zmax_p;
  const float *w;
  unsigned char *model;
  int *status;                 // 0 = ok, else an mcc_status
};

__global__ void k_quantize(const __grid_constant__ QuantArgs A) {
  if (threadIdx.x | blockIdx.x) return;
  const int sx = A.sx_p ? *A.sx_p : A.sx;
  const float mz1 = A.zmax_p ? __uint_as_float(A.zmax_p[0]) : A.max_z1;
  const float mz2 = A.zmax_p ? __uint_as_float(A.zmax_p[1]) : A.max_z2;
  const int n_in = (1 << A.dim) + A.dim;
  const float *W1 = A.w + oW1, *b1 = A.w + oB1, *W2 = A.w + oW2, *b2 = A.w + oB2, *W3 = A.w + oW3;
  double m1 = 0.0, m2 = 0.0, m3 = 0.0;
  bool finite = true;
  for (int k = 0; k < kNP; k++) finite = finite && isfinite(A.w[k]);
  for (int j = 0; j < 64; j++) {
    for (int i = 0; i < n_in; i++) m1 = fmax(m1, fabs((double)W1[j * 16 + i]));
    for (int i = 0; i < 64; i++) m2 = fmax(m2, fabs((double)W2[j * 64 + i]));
    m3 = fmax(m3, fabs((double)W3[j]));
  }
  if (!finite || !(mz1 >= 0.0f) || !(mz2 >= 0.0f) || isinf(mz1) || isinf(mz2) || sx < -60 ||
      sx > 60 || !(m1 <= 1e30 && m2 <= 1e30 && m3 <= 1e30)) {
    *A.status = MCC_ERR_INVALID_ARG;
    return;
  }
  int a1 = weight_exp(m1), t1 = act_exp(mz1);
  int s1 = t1 + a1 + 7;
  if (s1 > 30) { a1 -= s1 - 30; s1 = 30; }
  if (s1 < 1) { t1 += 1 - s1; s1 = 1; }
  int a2 = weight_exp(m2), t2 = act_exp(mz2);
  int s2 = t2 + a2 - t1;
  if (s2 > 30) { a2 -= s2 - 30; s2 = 30; }
  if (s2 < 1) { t2 += 1 - s2; s2 = 1; }
  const int a3 = weight_exp(m3);
  const int e3 = t2 - a3;
  if (e3 < -100 || e3 > 60) {
    *A.status = MCC_ERR_RANGE;
    return;
  }
  unsigned char *o = A.model;
  int *hdr = (int *)o;
  hdr[M_MAGIC / 4] = (int)kModelMagic;
  hdr[M_VERSION / 4] = 1;
  hdr[M_DIM / 4] = A.dim;
  hdr[M_NIN / 4] = n_in;
  hdr[M_SX / 4] = sx;
  hdr[M_S1 / 4] = s1;
  hdr[M_S2 / 4] = s2;
  hdr[M_E3 / 4] = e3;
  const double f1 = pow2d(a1), f2 = pow2d(a2), f3 = pow2d(a3);
  for (int j = 0; j < 64; j++) {
    for (int i = 0; i < 16; i++)
      o[M_W1 + j * 16 + i] = i < n_in ? (unsigned char)(signed char)(int)rint((double)W1[j * 16 + i] * f1) : 0;
    for (int i = 0; i < 64; i++)
      o[M_W2 + j * 64 + i] = (unsigned char)(signed char)(int)rint((double)W2[j * 64 + i] * f2);
    o[M_W3 + j] = (unsigned char)(signed char)(int)rint((double)W3[j] * f3);
    ((int *)(o + M_B1))[j] = qbias(b1[j], a1 + 7);
    ((int *)(o + M_B2))[j] = qbias(b2[j], a2 - t1);
  }
  ((int *)(o + M_B3))[0] = qbias(A.w[oB3], a3 - t2);
  ((int *)(o + M_B3))[1] = 0;
  *A.status = MCC_OK;
}

__global__ void k_keep_err(const Status *st, unsigned int *out) {
  if (threadIdx.x | blockIdx.x) return;
  *out = st->err;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct TrainWs {
  size_t comp, X, Y, w, m, v, partial, loss, hist, sx, zmax, errs, qstat, total;
  int64_t S;  // samples in all
  int G;      // k_grad CTAs per step
};

TrainWs train_ws_layout(const PlanView &pv, const mcc_params *p, const mcc_train_cfg *c, int n) {
  TrainWs t;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  t.S = (int64_t)n * c->samples_per_field;
  t.G = c->batch / kRows;
  t.comp = take(compress_ws_layout(pv, p).total);
  t.X = take(sizeof(float) * kK * (size_t)t.S);
  t.Y = take(sizeof(float) * (size_t)t.S);
  t.w = take(sizeof(float) * kNP);
  t.m = take(sizeof(float) * kNP);
  t.v = take(sizeof(float) * kNP);
  t.partial = take(sizeof(float) * kPartial * (size_t)t.G);
  t.loss = take(sizeof(float) * (size_t)c->steps);
  t.hist = take(sizeof(unsigned int) * 256);
  t.sx = take(sizeof(int));
  t.zmax = take(2 * sizeof(unsigned int));
  t.errs = take(sizeof(unsigned int) * (size_t)n);
  t.qstat = take(sizeof(int));
  t.total = o;
  return t;
}

mcc_status check_cfg(const mcc_train_cfg *c) {
  if (!c) return MCC_ERR_INVALID_ARG;
  if (c->steps < 1 || c->steps > 1000000) return MCC_ERR_INVALID_ARG;
  if (c->batch < kRows || c->batch > 65536 || c->batch % kRows) return MCC_ERR_INVALID_ARG;
  if (!(c->lr > 0.0f) || !(c->lr < 1.0f) || !(c->beta1 >= 0.0f && c->beta1 < 1.0f) ||
      !(c->beta2 >= 0.0f && c->beta2 < 1.0f) || !(c->eps > 0.0f))
    return MCC_ERR_INVALID_ARG;
  if (c->loss != MCC_LOSS_L2 && c->loss != MCC_LOSS_L1) return MCC_ERR_INVALID_ARG;
  if (c->samples_per_field < 1 || c->samples_per_field > (1ll << 26)) return MCC_ERR_INVALID_ARG;
  return MCC_OK;
}

bool grad_attr_set = false;

void set_grad_attr() {
  if (!grad_attr_set) {
    cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GradSmem));
    grad_attr_set = true;
  }
}

int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

extern "C" void mcc_train_cfg_default(mcc_train_cfg *c) {
  if (!c) return;
  c->steps = 1500;
  c->batch = 4096;
  c->lr = 2e-3f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-8f;
  c->loss = MCC_LOSS_L1;
  c->samples_per_field = 65536;
  c->seed = 1;
}

extern "C" mcc_status mcc_train_workspace_size(mcc_plan plan, const mcc_params *p,
                                               const mcc_train_cfg *cfg, int n, size_t *bytes) {
  if (!plan || !p || !bytes || n < 1 || n > 4096) return MCC_ERR_INVALID_ARG;
  mcc_status s = check_params(p);
  if (s) return s;
  if ((s = check_cfg(cfg))) return s;
  *bytes = train_ws_layout(mcc_plan_view(plan), p, cfg, n).total;
  return MCC_OK;
}

extern "C" mcc_status mcc_model_train(mcc_plan plan, int n, const void *const *d_fields,
                                      const mcc_params *p, const mcc_train_cfg *cfg,
                                      void *d_workspace, size_t workspace_bytes,
                                      void *d_model_out, float *h_loss, mcc_stream stream_) {
  if (!plan || !d_fields || !p || !d_workspace || !d_model_out || n < 1 || n > 4096)
    return MCC_ERR_INVALID_ARG;
  if ((uintptr_t)d_model_out & 3 || (uintptr_t)d_workspace & 255) return MCC_ERR_INVALID_ARG;
  mcc_status s = check_params(p);
  if (s) return s;
  if ((s = check_cfg(cfg))) return s;
  mcc_params pz = *p;  // the residuals of the method without a predictor
  pz.predictor = MCC_PRED_ZERO;
  pz.d_model = nullptr;
  pz.loop = MCC_LOOP_CLOSED;  // the predictor serves the closed loop only
  pz.zero_run = 0;            // (the coder does not run in training)
  const PlanView pv = mcc_plan_view(plan);
  const TrainWs T = train_ws_layout(pv, &pz, cfg, n);
  if (workspace_bytes < T.total) return MCC_ERR_CAPACITY;
  for (int f = 0; f < n; f++)
    if (!d_fields[f] || ((uintptr_t)d_fields[f] & (p->dtype == MCC_F64 ? 7 : 3)))
      return MCC_ERR_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)stream_;
  unsigned char *ws = (unsigned char *)d_workspace;
  float *X = (float *)(ws + T.X), *Y = (float *)(ws + T.Y);
  float *w = (float *)(ws + T.w), *m = (float *)(ws + T.m), *v = (float *)(ws + T.v);
  float *partial = (float *)(ws + T.partial), *loss = (float *)(ws + T.loss);
  unsigned int *hist = (unsigned int *)(ws + T.hist), *zmax = (unsigned int *)(ws + T.zmax);
  unsigned int *errs = (unsigned int *)(ws + T.errs);
  int *sx = (int *)(ws + T.sx), *qstat = (int *)(ws + T.qstat);
  const int64_t Sf = cfg->samples_per_field;
  const int ncd = (1 << pv.dim) - 1;
  const int sms = sm_count();
  const size_t cwss = compress_ws_layout(pv, &pz).total;
  // 1. samples of every training field
  for (int f = 0; f < n; f++) {
    const void *xs[1] = {d_fields[f]};
    s = launch_compress_batch(pv, 1, xs, &pz, ws + T.comp, (int64_t)cwss, nullptr, 0, 0, stream,
                              true);
    if (s) return s;
    SampleArgs A;
    A.pv = pv;
    A.Q = (const int *)(ws + T.comp + compress_ws_layout(pv, &pz).Q);
    A.q1 = (const int *)(ws + T.comp + compress_ws_layout(pv, &pz).q1);
    A.st = (const Status *)(ws + T.comp);
    A.X = X + (int64_t)f * Sf * kK;
    A.Y = Y + (int64_t)f * Sf;
    A.S = Sf;
    A.seed = cfg->seed;
    A.field = f;
    const unsigned int nb = (unsigned int)((Sf + 255) / 256);
    if (pv.dim == 2) k_sample<2><<<nb, 256, 0, stream>>>(A);
    else k_sample<3><<<nb, 256, 0, stream>>>(A);
    k_keep_err<<<1, 32, 0, stream>>>(A.st, errs + f);
  }
  // 2. feature exponent and integer features
  if (cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), stream) != cudaSuccess) return MCC_ERR_CUDA;
  k_exp_hist<<<sms * 2, 256, 0, stream>>>(X, T.S, ncd, hist);
  k_pick_sx<<<1, 32, 0, stream>>>(hist, sx);
  k_finalize<<<sms * 4, 256, 0, stream>>>(X, T.S, ncd, sx);
  // 3. training
  const int n_in = (1 << pv.dim) + pv.dim;
  k_init<<<(kNP + 255) / 256, 256, 0, stream>>>(w, m, v, n_in, cfg->seed);
  set_grad_attr();
  GradArgs G;
  memset(&G, 0, sizeof(G));
  G.w = w;
  G.X = X;
  G.Y = Y;
  G.S = T.S;
  G.B = cfg->batch;
  G.random = 1;
  G.seed = cfg->seed ^ 0x5DEECE66Dull;
  G.loss = cfg->loss;
  G.inv_b = 1.0f / (float)cfg->batch;
  G.partial = partial;
  AdamArgs D;
  D.partial = partial;
  D.nblocks = T.G;
  D.w = w;
  D.m = m;
  D.v = v;
  D.lr = cfg->lr;
  D.beta1 = cfg->beta1;
  D.beta2 = cfg->beta2;
  D.eps = cfg->eps;
  D.inv_b = G.inv_b;
  double p1 = 1.0, p2 = 1.0;
  for (int t = 0; t < cfg->steps; t++) {
    G.step = t;
    k_grad<<<T.G, 128, sizeof(GradSmem), stream>>>(G);
    p1 *= cfg->beta1;
    p2 *= cfg->beta2;
    D.c1 = (float)(1.0 - p1);
    D.c2 = (float)(1.0 - p2);
    D.loss = loss + t;
    k_adam<<<(kNP + 1 + 255) / 256, 256, 0, stream>>>(D);
  }
  // 4. calibration maxima over all samples, then quantisation
  if (cudaMemsetAsync(zmax, 0, 2 * sizeof(unsigned int), stream) != cudaSuccess) return MCC_ERR_CUDA;
  G.random = 0;
  G.B = T.S;
  G.calib = 1;
  G.zmax = zmax;
  const int64_t tiles = (T.S + kRows - 1) / kRows;
  k_grad<<<(unsigned int)(tiles < sms * 2 ? tiles : sms * 2), 128, sizeof(GradSmem), stream>>>(G);
  QuantArgs Q;
  memset(&Q, 0, sizeof(Q));
  Q.dim = pv.dim;
  Q.sx_p = sx;
  Q.zmax_p = zmax;
  Q.w = w;
  Q.model = (unsigned char *)d_model_out;
  Q.status = qstat;
  k_quantize<<<1, 32, 0, stream>>>(Q);
  if (cudaGetLastError() != cudaSuccess) return MCC_ERR_CUDA;
  std::vector<unsigned int> herr((size_t)n);
  int hq = 0;
  if (cudaMemcpyAsync(herr.data(), errs, sizeof(unsigned int) * (size_t)n, cudaMemcpyDeviceToHost,
                      stream) != cudaSuccess ||
      cudaMemcpyAsync(&hq, qstat, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  if (h_loss && cudaMemcpyAsync(h_loss, loss, sizeof(float) * (size_t)cfg->steps,
                                cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return MCC_ERR_CUDA;
  for (int f = 0; f < n; f++)
    if (herr[(size_t)f]) return (mcc_status)herr[(size_t)f];
  return (mcc_status)hq;
}

extern "C" size_t mcc_mlp_grad_workspace_size(int64_t B) {
  if (B < 1) return 0;
  return sizeof(float) * kPartial * (size_t)((B + kRows - 1) / kRows);
}

extern "C" mcc_status mcc_mlp_grad(const float *d_params, const float *d_x, const float *d_y,
                                   int64_t B, int loss, void *d_workspace, size_t workspace_bytes,
                                   float *d_grad, float *d_loss, mcc_stream stream_) {
  if (!d_params || !d_x || !d_y || !d_workspace || !d_grad || !d_loss || B < 1 ||
      B > (1ll << 30) || (loss != MCC_LOSS_L2 && loss != MCC_LOSS_L1))
    return MCC_ERR_INVALID_ARG;
  if ((uintptr_t)d_x & 15 || (uintptr_t)d_workspace & 3) return MCC_ERR_INVALID_ARG;
  if (workspace_bytes < mcc_mlp_grad_workspace_size(B)) return MCC_ERR_CAPACITY;
  cudaStream_t stream = (cudaStream_t)stream_;
  const int64_t tiles = (B + kRows - 1) / kRows;
  if (tiles > 0x7fffffff) return MCC_ERR_INVALID_ARG;
  set_grad_attr();
  GradArgs G;
  memset(&G, 0, sizeof(G));
  G.w = d_params;
  G.X = d_x;
  G.Y = d_y;
  G.S = B;
  G.B = B;
  G.loss = loss;
  G.inv_b = 1.0f / (float)B;
  G.partial = (float *)d_workspace;
  k_grad<<<(unsigned int)tiles, 128, sizeof(GradSmem), stream>>>(G);
  k_reduce_grad<<<(kNP + 1 + 255) / 256, 256, 0, stream>>>((const float *)d_workspace, (int)tiles,
                                                          G.inv_b, d_grad, d_loss);
  return cudaGetLastError() == cudaSuccess ? MCC_OK : MCC_ERR_CUDA;
}

extern "C" mcc_status mcc_mlp_quantize(int dim, int sx, const float *d_params, float max_z1,
                                       float max_z2, void *d_model, int *d_status,
                                       mcc_stream stream_) {
  if ((dim != 2 && dim != 3) || !d_params || !d_model || !d_status || ((uintptr_t)d_model & 3))
    return MCC_ERR_INVALID_ARG;
  QuantArgs Q;
  memset(&Q, 0, sizeof(Q));
  Q.dim = dim;
  Q.sx = sx;
  Q.max_z1 = max_z1;
  Q.max_z2 = max_z2;
  Q.w = d_params;
  Q.model = (unsigned char *)d_model;
  Q.status = d_status;
  k_quantize<<<1, 32, 0, (cudaStream_t)stream_>>>(Q);
  return cudaGetLastError() == cudaSuccess ? MCC_OK : MCC_ERR_CUDA;
}
