// predictor.cu -- inference of the learned residual predictor on the tensor
// cores (bf16 mma.sync m16n8k16, FP32 accumulation).
//
// Each warp takes 32 consecutive vertices: lanes compute the integer features
// of their vertex (corner-code differences in vertex bins, local coordinates
// and the level of corner 000), then the warp runs two 16-row tiles through the network:
// layer 1 (16 -> 64) is 8 MMAs, layer 2 (64 -> 64) 32 MMAs, layer 3 (64 -> 1,
// padded to 8 columns) 4 MMAs. Accumulator fragments of one layer become the
// A fragments of the next in registers (columns 16k .. 16k+15 of the output
// are tiles 2k and 2k+1). Every product and partial sum is an integer below
// 2^24 in magnitude, so the FP32 accumulation is exact and the result equals
// the integer arithmetic of the definition.
//
// The activation round(a / 2^s) half up, clamped to 0..255, is taken in FP32
// without conversions: (a + 2^(s-1)) 2^-s is one exact fused multiply-add for
// s <= 23 (|a| < 2^23), and adding 2^23 rounding down leaves floor() in the
// low bits; for s >= 24 the result is 0. Integers of magnitude <= 256 are
// exact in bf16 and their FP32 bit pattern ends in 16 zero bits, so a pair
// packs into a bf16x2 register with one byte permutation.
#include <cuda_runtime.h>
#include <stdint.h>

#include "predictor.cuh"
#include "workspace.cuh"

using namespace mcc;

namespace {

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two small integers held in FP32 -> bf16x2 (lo in the low half)
__device__ __forceinline__ uint32_t pack_int2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// act(h + b, s) with bb = (b + 2^(s-1)) 2^-s precomputed: one fused
// multiply-add gives (h + b + 2^(s-1)) 2^-s exactly (an integer below 2^24
// times a power of two), then floor and clamp.
__device__ __forceinline__ float act8(float h, float inv, float bb) {
  const float x = __fmaf_rn(h, inv, bb);
  const float f = __fsub_rn(__fadd_rd(x, 0x1p23f), 0x1p23f);
  return fminf(fmaxf(f, 0.0f), 255.0f);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Model in shared memory: bf16 weights with rows padded by 8 elements
// (row strides of 12 and 36 words put the 8 rows of a fragment load on
// distinct banks), biases as exact floats.
struct SModel {
  uint16_t W1[kH][kK + 8];
  uint16_t W2[kH][kH + 8];
  uint16_t W3[8][kH + 8];  // row 0 = W3, rows 1..7 = 0
  float bb1[kH], bb2[kH];  // (b + 2^(s-1)) 2^-s per unit
  float b3, half1, inv1, half2, inv2, out_scale, sxs;
  int ok;
};

__device__ __forceinline__ uint16_t bf16_of_int8(int v) {
  return (uint16_t)(__float_as_uint((float)v) >> 16);
}

// Parse and validate the blob (the same checks as the format's definition);
// every thread returns the same verdict.
__device__ bool load_model(const unsigned char *blob, int dim, SModel &m) {
  const int tid = threadIdx.x;
  const int nin = (1 << dim) + dim;
  if (tid == 0) {
    const int *w = (const int *)blob;
    const int sx = w[M_SX / 4], s1 = w[M_S1 / 4], s2 = w[M_S2 / 4], e3 = w[M_E3 / 4];
    const int b3 = w[M_B3 / 4];
    int ok = (uint32_t)w[M_MAGIC / 4] == kModelMagic && w[M_VERSION / 4] == 1 &&
             w[M_DIM / 4] == dim && w[M_NIN / 4] == nin;
    ok = ok && sx >= -60 && sx <= 60 && s1 >= 1 && s1 <= 30 && s2 >= 1 && s2 <= 30 && e3 >= -100 &&
         e3 <= 60 && b3 >= -(1 << 22) && b3 <= (1 << 22);
    m.ok = ok;
    if (ok) {
      m.b3 = (float)b3;
      // s >= 24: every activation is 0 (|a| < 2^23); half = inv = 0 gives that
      m.half1 = s1 <= 23 ? pow2f(s1 - 1) : 0.0f;
      m.inv1 = s1 <= 23 ? pow2f(-s1) : 0.0f;
      m.half2 = s2 <= 23 ? pow2f(s2 - 1) : 0.0f;
      m.inv2 = s2 <= 23 ? pow2f(-s2) : 0.0f;
      m.out_scale = pow2f(e3);
      m.sxs = pow2f(-sx);
    }
  }
  __syncthreads();
  int bad = 0;
  const signed char *W1 = (const signed char *)(blob + M_W1);
  const signed char *W2 = (const signed char *)(blob + M_W2);
  const signed char *W3 = (const signed char *)(blob + M_W3);
  for (int e = tid; e < kH * kK; e += blockDim.x) {
    const int v = W1[e], i = e % kK;
    bad |= v < -127 || (i >= nin && v != 0);
    m.W1[e / kK][i] = bf16_of_int8(v);
  }
  for (int e = tid; e < kH * kH; e += blockDim.x) {
    const int v = W2[e];
    bad |= v < -127;
    m.W2[e / kH][e % kH] = bf16_of_int8(v);
  }
  for (int e = tid; e < 8 * kH; e += blockDim.x) {
    const int v = e < kH ? (int)W3[e] : 0;
    bad |= v < -127;
    m.W3[e / kH][e % kH] = bf16_of_int8(v);
  }
  for (int j = tid; j < kH; j += blockDim.x) {
    const int c1 = ((const int *)(blob + M_B1))[j], c2 = ((const int *)(blob + M_B2))[j];
    bad |= c1 < -(1 << 22) || c1 > (1 << 22) || c2 < -(1 << 22) || c2 > (1 << 22);
    // |b| <= 2^22 and 2^(s-1) <= 2^22: the sums and their scaling are exact
    m.bb1[j] = __fmul_rn(__fadd_rn((float)c1, m.half1), m.inv1);
    m.bb2[j] = __fmul_rn(__fadd_rn((float)c2, m.half2), m.inv2);
  }
  if (bad) atomicAnd(&m.ok, 0);
  __syncthreads();
  return m.ok != 0;
}

// Layer output fragments (8 n-tiles of 16x8, C layout) -> activations as the
// A fragments of the next layer (4 k-tiles of 16x16).
__device__ __forceinline__ void act_to_frag(const float (&h)[8][4], const float *bb, float inv,
                                            int tq, uint32_t (&a)[4][4]) {
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    const int c0 = 8 * nt + 2 * tq;
    const float bl = bb[c0], bh = bb[c0 + 1];
    const float v0 = act8(h[nt][0], inv, bl);
    const float v1 = act8(h[nt][1], inv, bh);
    const float v2 = act8(h[nt][2], inv, bl);
    const float v3 = act8(h[nt][3], inv, bh);
    a[nt >> 1][(nt & 1) ? 2 : 0] = pack_int2(v0, v1);
    a[nt >> 1][(nt & 1) ? 3 : 1] = pack_int2(v2, v3);
  }
}

template <int DIM>
__global__ void __launch_bounds__(256, 4) k_predict(const __grid_constant__ PredArgs A) {
  pdl_wait();
  __shared__ SModel m;
  __shared__ __align__(16) uint16_t xs[8][32][kK + 8];
  __shared__ float ps[8][32];
  __shared__ int skip;
  const int f = blockIdx.x;
  Status *st = A.st[f];
  if (threadIdx.x == 0)  // fields without a model (or a plain stream) have nothing to do
    skip = A.model[f] == nullptr || *(volatile unsigned int *)&st->err != 0 ||
           (A.use[f] && *A.use[f] == 0);
  __syncthreads();
  if (skip) return;
  const unsigned char *blob = A.model[f] + (A.model_off[f] ? *A.model_off[f] : 0);
  if (!load_model(blob, DIM, m)) {
    if (threadIdx.x == 0) set_error(st, A.bad_model_err);
    return;
  }
  const PlanView &pv = A.pv;
  const int *__restrict__ q1 = A.q1[f];
  float *__restrict__ pout = A.p[f];
  const float rf = *A.rho12_f[f];
  const long long Qhi = *A.qhi[f];
  const float linv = Qhi > 0 ? __fdiv_rn(127.0f, __ll2float_rn(Qhi)) : 0.0f;
  const float sxs = m.sxs;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, tq = lane & 3;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const int64_t step = (int64_t)gridDim.y * 256;
  for (int64_t base = ((int64_t)blockIdx.y * 8 + w) * 32; base < n; base += step) {
    // ---- features of this lane's vertex
    const int64_t i = base + lane;
    float feat[kK];
#pragma unroll
    for (int k = 0; k < kK; k++) feat[k] = 0.0f;
    if (i < n) {
      const uint32_t c = __ldg(pv.cell + i);
      int cor[8];
      corner_codes<DIM>(q1, c, nx, sxy, cor);
#pragma unroll
      for (int k = 1; k < (1 << DIM); k++) {
        float e = __fmul_rn(__int2float_rn(wsub(cor[k], cor[0])), rf);
        e = __fmul_rn(e, sxs);
        feat[k - 1] = fminf(fmaxf(rintf(e), -127.0f), 127.0f);
      }
#pragma unroll
      for (int d = 0; d < DIM; d++) {
        const float fr = __fmul_rn(__uint2float_rn(__ldg(pv.frac + (int64_t)d * n + i)), 0x1p-15f);
        feat[(1 << DIM) - 1 + d] = rintf(__fmul_rn(fr, 127.0f));
      }
      const float lv = rintf(__fmul_rn(__fmul_rn(__int2float_rn(cor[0]), rf), linv));
      feat[(1 << DIM) + DIM - 1] = fminf(fmaxf(lv, 0.0f), 127.0f);
    }
#pragma unroll
    for (int k = 0; k < kK; k += 2)
      *reinterpret_cast<uint32_t *>(&xs[w][lane][k]) = pack_int2(feat[k], feat[k + 1]);
    __syncwarp();
    // ---- two 16-row tiles through the network
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const int r0 = 16 * t + g, r1 = r0 + 8;
      uint32_t a[4];
      a[0] = *reinterpret_cast<const uint32_t *>(&xs[w][r0][2 * tq]);
      a[1] = *reinterpret_cast<const uint32_t *>(&xs[w][r1][2 * tq]);
      a[2] = *reinterpret_cast<const uint32_t *>(&xs[w][r0][2 * tq + 8]);
      a[3] = *reinterpret_cast<const uint32_t *>(&xs[w][r1][2 * tq + 8]);
      float h[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        h[nt][0] = h[nt][1] = h[nt][2] = h[nt][3] = 0.0f;
        const int col = 8 * nt + g;
        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&m.W1[col][2 * tq]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&m.W1[col][2 * tq + 8]);
        mma_bf16(h[nt], a, b0, b1);
      }
      uint32_t a2[4][4];
      act_to_frag(h, m.bb1, m.inv1, tq, a2);
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        h[nt][0] = h[nt][1] = h[nt][2] = h[nt][3] = 0.0f;
        const int col = 8 * nt + g;
#pragma unroll
        for (int kt = 0; kt < 4; kt++) {
          const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&m.W2[col][16 * kt + 2 * tq]);
          const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&m.W2[col][16 * kt + 2 * tq + 8]);
          mma_bf16(h[nt], a2[kt], b0, b1);
        }
      }
      uint32_t a3[4][4];
      act_to_frag(h, m.bb2, m.inv2, tq, a3);
      float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kt = 0; kt < 4; kt++) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&m.W3[g][16 * kt + 2 * tq]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t *>(&m.W3[g][16 * kt + 2 * tq + 8]);
        mma_bf16(o, a3[kt], b0, b1);
      }
      if (tq == 0) {  // column 0 holds the outputs of rows g and g + 8
        ps[w][r0] = __fmul_rn(__fadd_rn(o[0], m.b3), m.out_scale);
        ps[w][r1] = __fmul_rn(__fadd_rn(o[2], m.b3), m.out_scale);
      }
    }
    __syncwarp();
    if (i < n) pout[i] = ps[w][lane];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// tcgen05 inference: one CTA of 128 threads takes tiles of 128 vertices (one
// row per thread). Layer 1 (16 -> 64) and layer 2 (64 -> 64) run as
// tcgen05.mma kind::f16 (BF16 operands in shared memory, FP32 accumulators in
// TMEM, issued by one thread, completion through an mbarrier); the
// accumulator rows come back with tcgen05.ld (TMEM lane = row), take the
// activation and become the next layer's A tile; layer 3 (64 -> 1) is a
// 64-term FP32 sum per thread. All values are the integers of the
// definition, so the result is the mma.sync kernel's bit for bit.
//
// Operands are K-major without swizzle: core matrices of 8 rows x 8 bf16
// (128 bytes, rows of 16 bytes), core matrix (row group r8, column group k8)
// at (r8 (K / 8) + k8) 128 bytes: the descriptor's leading-dimension offset
// is 128 bytes (the next 8 columns), its stride offset (K / 8) 128 bytes (the
// next 8 rows).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (in 16-byte units), descriptor version 1, no swizzle, base offset 0
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: D F32, A and B BF16, both K-major, dense,
// M = 128, N = 64
constexpr uint32_t kIdescM128N64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                                   ((128u >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(kIdescM128N64), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

// bounded wait for the mbarrier phase (false: the limit ran out)
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 24) && !done; it++)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(phase));
  return done != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_sync() {  // thread sync ordered with the tensor-core work
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// byte offset of element (row r, column k) of a K-major operand with K columns
__device__ __forceinline__ uint32_t kmaj(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct TcModel {
  __align__(128) uint16_t W1[kH * kK];  // B of layer 1: 64 rows (units) x 16 (inputs)
  __align__(128) uint16_t W2[kH * kH];  // B of layer 2
  __align__(128) uint16_t A1[128 * kK]; // this tile's features
  __align__(128) uint16_t A2[128 * kH]; // this tile's first-layer activations
  float W3[kH], bb1[kH], bb2[kH];
  float b3, inv1, inv2, out_scale, sxs;
  uint64_t mbar;
  uint32_t tmem;
};

template <int DIM>
__global__ void __launch_bounds__(128) k_predict_tc(const __grid_constant__ PredArgs A) {
  pdl_wait();
  __shared__ TcModel m;
  __shared__ SModel sm;  // the blob's validation and scalars (shared with the mma.sync layout)
  const int tid = threadIdx.x;
  const int f = blockIdx.x;
  Status *st = A.st[f];
  __shared__ int skip;
  if (tid == 0)
    skip = A.model[f] == nullptr || *(volatile unsigned int *)&st->err != 0 ||
           (A.use[f] && *A.use[f] == 0);
  __syncthreads();
  if (skip) return;
  const unsigned char *blob = A.model[f] + (A.model_off[f] ? *A.model_off[f] : 0);
  if (!load_model(blob, DIM, sm)) {
    if (tid == 0) set_error(st, A.bad_model_err);
    return;
  }
  // the weights in the K-major core-matrix layout, biases and scalars
  for (int e = tid; e < kH * kK; e += blockDim.x) {
    const int r = e / kK, k = e % kK;
    *(uint16_t *)((unsigned char *)m.W1 + kmaj(r, k, kK)) = sm.W1[r][k];
  }
  for (int e = tid; e < kH * kH; e += blockDim.x) {
    const int r = e / kH, k = e % kH;
    *(uint16_t *)((unsigned char *)m.W2 + kmaj(r, k, kH)) = sm.W2[r][k];
  }
  for (int j = tid; j < kH; j += blockDim.x) {
    m.W3[j] = __uint_as_float((uint32_t)sm.W3[0][j] << 16);  // the int8 weight (exact in bf16)
    m.bb1[j] = sm.bb1[j];
    m.bb2[j] = sm.bb2[j];
  }
  if (tid == 0) {
    m.b3 = sm.b3;
    m.inv1 = sm.inv1;
    m.inv2 = sm.inv2;
    m.out_scale = sm.out_scale;
    m.sxs = sm.sxs;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&m.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid < 32) {  // warp 0 holds 128 TMEM columns: layer 1 in 0..63, layer 2 in 64..127
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&m.tmem)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_sync();
  const uint32_t tm = m.tmem;
  const PlanView &pv = A.pv;
  const int *__restrict__ q1 = A.q1[f];
  float *__restrict__ pout = A.p[f];
  const float rf = *A.rho12_f[f];
  const long long Qhi = *A.qhi[f];
  const float linv = Qhi > 0 ? __fdiv_rn(127.0f, __ll2float_rn(Qhi)) : 0.0f;
  const float sxs = m.sxs;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const int w = tid >> 5;
  const uint32_t lane_base = (uint32_t)(32 * w) << 16;  // this warp's TMEM lanes (rows)
  const uint32_t a1 = smem_u32(m.A1), a2 = smem_u32(m.A2);
  const uint32_t b1 = smem_u32(m.W1), b2 = smem_u32(m.W2);
  uint32_t phase = 0;
  bool ok = true;
  for (int64_t base = (int64_t)blockIdx.y * 128; base < n; base += (int64_t)gridDim.y * 128) {
    // ---- features of this thread's vertex (row tid of the tile)
    const int64_t i = base + tid;
    float feat[kK];
#pragma unroll
    for (int k = 0; k < kK; k++) feat[k] = 0.0f;
    if (i < n) {
      const uint32_t c = __ldg(pv.cell + i);
      int cor[8];
      corner_codes<DIM>(q1, c, nx, sxy, cor);
#pragma unroll
      for (int k = 1; k < (1 << DIM); k++) {
        float e = __fmul_rn(__int2float_rn(wsub(cor[k], cor[0])), rf);
        e = __fmul_rn(e, sxs);
        feat[k - 1] = fminf(fmaxf(rintf(e), -127.0f), 127.0f);
      }
#pragma unroll
      for (int d = 0; d < DIM; d++) {
        const float fr = __fmul_rn(__uint2float_rn(__ldg(pv.frac + (int64_t)d * n + i)), 0x1p-15f);
        feat[(1 << DIM) - 1 + d] = rintf(__fmul_rn(fr, 127.0f));
      }
      const float lv = rintf(__fmul_rn(__fmul_rn(__int2float_rn(cor[0]), rf), linv));
      feat[(1 << DIM) + DIM - 1] = fminf(fmaxf(lv, 0.0f), 127.0f);
    }
#pragma unroll
    for (int k8 = 0; k8 < kK / 8; k8++) {
      uint4 v;
      v.x = pack_int2(feat[8 * k8 + 0], feat[8 * k8 + 1]);
      v.y = pack_int2(feat[8 * k8 + 2], feat[8 * k8 + 3]);
      v.z = pack_int2(feat[8 * k8 + 4], feat[8 * k8 + 5]);
      v.w = pack_int2(feat[8 * k8 + 6], feat[8 * k8 + 7]);
      *(uint4 *)((unsigned char *)m.A1 + kmaj(tid, 8 * k8, kK)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    // ---- layer 1: [128 x 16] x [16 x 64] -> TMEM columns 0..63
    if (tid == 0) {
      umma_f16(tm, umma_desc(a1, 128, (kK / 8) * 128), umma_desc(b1, 128, (kK / 8) * 128), 0u);
      umma_commit(&m.mbar);
    }
    // every thread waits; the verdict is taken by the whole block (a wait that
    // ran out stops the block, uniformly)
    if (!__syncthreads_and(mbar_wait(&m.mbar, phase) ? 1 : 0)) { ok = false; break; }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float h[16];
      tmem_ld16(tm + lane_base + (uint32_t)c0, h);
#pragma unroll
      for (int q = 0; q < 2; q++) {
        uint4 v;
        const int c = c0 + 8 * q;
        v.x = pack_int2(act8(h[8 * q + 0], m.inv1, m.bb1[c + 0]), act8(h[8 * q + 1], m.inv1, m.bb1[c + 1]));
        v.y = pack_int2(act8(h[8 * q + 2], m.inv1, m.bb1[c + 2]), act8(h[8 * q + 3], m.inv1, m.bb1[c + 3]));
        v.z = pack_int2(act8(h[8 * q + 4], m.inv1, m.bb1[c + 4]), act8(h[8 * q + 5], m.inv1, m.bb1[c + 5]));
        v.w = pack_int2(act8(h[8 * q + 6], m.inv1, m.bb1[c + 6]), act8(h[8 * q + 7], m.inv1, m.bb1[c + 7]));
        *(uint4 *)((unsigned char *)m.A2 + kmaj(tid, c, kH)) = v;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    // ---- layer 2: [128 x 64] x [64 x 64] -> TMEM columns 64..127 (4 K steps)
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < kH / 16; s++)
        umma_f16(tm + 64, umma_desc(a2 + 256 * s, 128, (kH / 8) * 128),
                 umma_desc(b2 + 256 * s, 128, (kH / 8) * 128), s > 0 ? 1u : 0u);
      umma_commit(&m.mbar);
    }
    if (!__syncthreads_and(mbar_wait(&m.mbar, phase) ? 1 : 0)) { ok = false; break; }
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- layer 3 on the CUDA cores
    float acc = 0.0f;
#pragma unroll
    for (int c0 = 0; c0 < kH; c0 += 16) {
      float h[16];
      tmem_ld16(tm + lane_base + 64u + (uint32_t)c0, h);
#pragma unroll
      for (int j = 0; j < 16; j++) acc = __fmaf_rn(act8(h[j], m.inv2, m.bb2[c0 + j]), m.W3[c0 + j], acc);
    }
    if (i < n) pout[i] = __fmul_rn(__fadd_rn(acc, m.b3), m.out_scale);
  }
  if (!ok) {  // a wait ran out: give the tensor core a bounded while to finish
    mbar_wait(&m.mbar, phase);
    if (tid == 0) set_error(st, MCC_ERR_TIMEOUT);
  }
  tc_sync();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tm));
}

}  // namespace

cudaError_t launch_predict(const PredArgs &A, cudaStream_t stream, bool pdl) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t warps = (A.pv.n_v + 31) / 32;
  // one full wave of resident blocks (every block has the same share)
  int64_t chunks = A.pv.dim == 2 ? wave_blocks(k_predict<2>, 256, 0, 0, sms, A.nf)
                                 : wave_blocks(k_predict<3>, 256, 0, 0, sms, A.nf);
  if (chunks > (warps + 7) / 8) chunks = (warps + 7) / 8;
  if (chunks < 1) chunks = 1;
  if (chunks > 65535) chunks = 65535;
  const dim3 grid(A.nf, (unsigned int)chunks);
  if (A.pv.net_path == MCC_NET_TCGEN05) {
    // at most 4 resident CTAs per SM: each holds 128 of the SM's 512 TMEM
    // columns (a fifth would wait in tcgen05.alloc until one finishes).
    // Shared memory sets the residency: the CTA's static share plus the
    // driver's reserve per block, padded with dynamic shared memory when a
    // fifth CTA would fit.
    void (*kern)(PredArgs) = A.pv.dim == 2 ? k_predict_tc<2> : k_predict_tc<3>;
    cudaFuncAttributes fa;
    int smem_sm = 0, reserve = 0;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
      return cudaErrorInvalidConfiguration;
    const size_t per_block = fa.sharedSizeBytes + (size_t)reserve;
    size_t pad = 0;
    if ((size_t)smem_sm / per_block > 4) pad = ((size_t)smem_sm / 5 + 1 - per_block + 127) / 128 * 128;
    if (pad && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pad) !=
                   cudaSuccess)
      return cudaErrorInvalidConfiguration;
    const int64_t per_sm = (int64_t)smem_sm / (int64_t)(per_block + pad);
    if (per_sm < 1 || per_sm > 4) return cudaErrorInvalidConfiguration;
    const int64_t tiles = (A.pv.n_v + 127) / 128;
    int64_t tch = ((int64_t)sms * per_sm + A.nf - 1) / A.nf;
    if (tch > tiles) tch = tiles;
    if (tch < 1) tch = 1;
    const dim3 tgrid(A.nf, (unsigned int)tch);
    if (pdl) return launch_pdl(kern, tgrid, dim3(128), pad, stream, A);
    kern<<<tgrid, 128, pad, stream>>>(A);
    return cudaGetLastError();
  }
  if (A.pv.dim == 2) {
    if (pdl) return launch_pdl(k_predict<2>, grid, dim3(256), 0, stream, A);
    k_predict<2><<<grid, 256, 0, stream>>>(A);
  } else {
    if (pdl) return launch_pdl(k_predict<3>, grid, dim3(256), 0, stream, A);
    k_predict<3><<<grid, 256, 0, stream>>>(A);
  }
  return cudaGetLastError();
}
