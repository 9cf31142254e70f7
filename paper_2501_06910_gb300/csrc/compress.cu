// compress.cu -- Algorithm 3 of Gong et al. (multi-component compression),
// closed loop, as a chain of kernels (for a large single field the grid
// component's Lorenzo stage, code book and group lengths run on the plan's
// second stream beside k_node and the residual's code book, joined before
// k_pack):
//
//   k_reduce     min / max / finiteness of x; the last block derives the
//                bound split tau = tau1 + tau2 (Sec. III) and the bin widths
//   k_prequant   vertex codes Q = round(x / s2) - K            (FP64, 2 ops)
//   k_grid2d / k_grid_codes3d + k_grid3d
//                x1 = f(x): barycentric interpolation of Q at every grid
//                point (Sec. IV-D), grid codes q1, N-D Lorenzo difference,
//                symbols + histogram (C(x1))
//   k_predict    (learned predictor only) the network's correction p at
//                every vertex, from the corner codes of its cell
//   k_node       g(x1'): multilinear interpolation of q1 at every vertex,
//                residual code q2 = Q - P, bound guard, symbols + histogram
//                (C(x2), residuals serialised 1-D, Sec. IV-B)
//   k_codebook   canonical Huffman code books (one CTA per component)
//   k_group_len  bit length of every lane chunk, escapes per group
//                (its last block per field: group offsets, section
//                layout, header)
//   k_pack       bit packing through shared memory, escape / raw values
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <mutex>

#include "common.cuh"
#include "predictor.cuh"
#include "workspace.cuh"
#include "prof.cuh"

using namespace mcc;

namespace {

constexpr int kRawNone = 0xFFFF;

struct RParams {
  int dtype, eb_mode;
  double eb, frac;
  int one_d;  // the 1D coder (the paper's default baseline)
};

// Arguments shared by every compression kernel of one launch chain: the plan,
// the workspace layout (one region of wss bytes per field), the output slots
// (oss bytes per field) and the per-field inputs and bound parameters.
struct CompArgs {
  PlanView pv;
  CompressWs W;
  Layout F;  // fixed-size part of every stream (lens .. ltab2)
  unsigned char *ws0, *out0;
  int64_t wss, oss;
  uint64_t capacity;  // per-field output bytes
  int nf, dtype, R1, R2, C1, C2, lmax, nsym1, nsym2;
  int64_t ng1, ng2;
  const void *x[kMaxBatch];
  RParams rp[kMaxBatch];
  const unsigned char *model[kMaxBatch];  // learned-predictor blob or NULL
  unsigned char mode[kMaxBatch];          // MCC_PRED_* per field
  unsigned char open[kMaxBatch];          // MCC_LOOP_OPEN per field
  unsigned char fop[kMaxBatch], gop[kMaxBatch];  // MCC_F_* / MCC_G_* per field
  unsigned char zr[kMaxBatch];            // zero-run stage per field
  int any_auto, any_zr;
  int one_d;  // the 1D coder: component 1 holds the vertex codes' differences
  // logical index of the launch's first block along x (k_runs, k_codebook,
  // k_group_len): the grid and residual components' blocks may come in
  // separate launches (on two streams)
  int bx0;
};

// Per-field pointers into the workspace and the output slot.
struct Ctx {
  Status *st;
  unsigned int *hist1, *hist2, *code1, *code2, *gw, *ge, *gr, *pe, *pr;
  unsigned char *len1, *len2, *out;
  int *Q, *q1, *val1, *val2;
  unsigned short *sym1, *sym2, *pb, *rs;
  float *p;
  const void *x;
};

// The residual component's arrays of field f: the learned side when the
// field's auto choice kept the learned predictor (read from its status block).
__device__ __forceinline__ Ctx ctx_of(const CompArgs &A, int f, bool chosen = false) {
  Ctx c;
  unsigned char *ws = A.ws0 + (int64_t)f * A.wss;
  const bool b = chosen && A.any_auto && A.mode[f] == MCC_PRED_AUTO &&
                 *(volatile const unsigned int *)&((const Status *)ws)->pick;
  c.st = (Status *)ws;
  c.hist1 = (unsigned int *)(ws + A.W.hist1);
  c.hist2 = (unsigned int *)(ws + (b ? A.W.hist2b : A.W.hist2));
  c.code1 = (unsigned int *)(ws + A.W.code1);
  c.code2 = (unsigned int *)(ws + (b ? A.W.code2b : A.W.code2));
  c.len1 = ws + A.W.len1;
  c.len2 = ws + (b ? A.W.len2b : A.W.len2);
  c.Q = (int *)(ws + A.W.Q);
  c.q1 = (int *)(ws + A.W.q1);
  c.sym1 = (unsigned short *)(ws + A.W.sym1);
  c.sym2 = (unsigned short *)(ws + (b ? A.W.sym2b : A.W.sym2));
  c.val1 = (int *)(ws + A.W.val1);
  c.val2 = (int *)(ws + (b ? A.W.val2b : A.W.val2));
  c.gw = (unsigned int *)(ws + A.W.gw);
  c.ge = (unsigned int *)(ws + A.W.ge);
  c.gr = (unsigned int *)(ws + A.W.gr);
  c.pb = (unsigned short *)(ws + A.W.pb);
  c.rs = (unsigned short *)(ws + (b ? A.W.rsb : A.W.rs));
  c.pe = (unsigned int *)(ws + A.W.pe);
  c.pr = (unsigned int *)(ws + A.W.pr);
  c.p = (float *)(ws + A.W.p);
  c.out = A.out0 + (int64_t)f * A.oss;
  c.x = A.x[f];
  return c;
}

// Error check taken once per block, so every thread of the block agrees
// (an error may be recorded concurrently by another block).
__device__ __forceinline__ bool block_failed(const Status *st) {
  __shared__ int failed;
  if (threadIdx.x == 0) failed = *(volatile const unsigned int *)&st->err != 0;
  __syncthreads();
  return failed != 0;
}

__device__ __forceinline__ unsigned long long value_bits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

// ---------------------------------------------------------------------------
// k_reduce: min / max of x (ordered integer keys, no FP64 compares), finite
// check, and -- in the last block to finish -- the per-field parameters.
// ---------------------------------------------------------------------------
// Spacing of the value type at magnitude M (at least the smallest
// subnormal): 2^(e - p) with M in [2^e, 2^(e+1)), p = 52 (FP64) or 23.
__device__ double spacing_at(double M, int dtype) {
  const int p = dtype == MCC_F64 ? 52 : 23;
  const double tiny = dtype == MCC_F64 ? 0x1p-1074 : 0x1p-149;
  if (!(M > 0.0)) return tiny;
  int e;
  frexp(M, &e);  // M = f 2^e, f in [0.5, 1)
  const double u = ldexp(1.0, e - 1 - p);
  return u > tiny ? u : tiny;
}

// The 1D coder's parameters: bin s = 2 (tau - m) (1 - 2^-20), m = 4 u64(M)
// (+ 2 u32(M) for FP32 values): the FP64 roundings of x / s and s (K + Q)
// and the cast stay inside the margin, so every value holds the bound and
// none is stored raw.
__device__ void field_params_1d(Status *st, FieldParams &f, double tau, int dtype) {
  double m = __dmul_rn(4.0, spacing_at(f.M, MCC_F64));
  if (dtype == MCC_F32) m = __dadd_rn(m, __dmul_rn(2.0, spacing_at(f.M, MCC_F32)));
  const double t = __dsub_rn(tau, m);
  if (!isfinite(tau) || !(t >= 1e-290)) { set_error(st, MCC_ERR_RANGE); return; }
  f.tau1 = t;
  f.tau2 = t;
  f.s1 = __dmul_rn(__dmul_rn(2.0, t), kBinShrink);
  f.s2 = f.s1;
  if (!isfinite(f.s2)) { set_error(st, MCC_ERR_RANGE); return; }
  f.inv2 = __ddiv_rn(1.0, f.s2);
  const double kd = rint(__dmul_rn(f.lo, f.inv2));
  const double hd = rint(__dmul_rn(f.hi, f.inv2));
  if (!(fabs(kd) < 4611686018427387904.0) || !(fabs(hd) < 4611686018427387904.0)) {
    set_error(st, MCC_ERR_RANGE);
    return;
  }
  f.K = (long long)kd;
  f.Qhi = (long long)hd - f.K;
  if (f.Qhi >= (1ll << 29)) { set_error(st, MCC_ERR_RANGE); return; }
  f.fill_u = 0;
  f.rho21_q = f.rho12_q = 1ll << kRhoBits;  // one bin: ratio 1
  f.rho21_f = f.rho12_f = 1.0f;
  f.guard = 0;
  st->f = f;
}

__device__ void field_params(Status *st, RParams rp) {
  FieldParams f;
  memset(&f, 0, sizeof(f));
  const unsigned long long klo = ~atomicAdd(&st->key_lo, 0ull);
  const unsigned long long khi = atomicAdd(&st->key_hi, 0ull);
  const double lo = key_value(klo), hi = key_value(khi);
  f.lo = lo;
  f.hi = hi;
  f.M = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
  double tau = rp.eb;
  if (rp.eb_mode == 1 && hi > lo) tau = __dmul_rn(rp.eb, __dsub_rn(hi, lo));
  f.tau = tau;
  if (rp.one_d) {
    field_params_1d(st, f, tau, rp.dtype);
    return;
  }
  f.tau1 = __dmul_rn(rp.frac, tau);
  f.tau2 = __dmul_rn(__dsub_rn(1.0, rp.frac), tau);
  if (!isfinite(tau) || !(f.tau1 >= 1e-290) || !(f.tau2 >= 1e-290)) { set_error(st, MCC_ERR_RANGE); return; }
  f.s1 = __dmul_rn(__dmul_rn(2.0, f.tau1), kBinShrink);
  f.s2 = __dmul_rn(__dmul_rn(2.0, f.tau2), kBinShrink);
  if (!isfinite(f.s1) || !isfinite(f.s2)) { set_error(st, MCC_ERR_RANGE); return; }
  f.inv2 = __ddiv_rn(1.0, f.s2);
  const double kd = rint(__dmul_rn(lo, f.inv2));
  const double hd = rint(__dmul_rn(hi, f.inv2));
  if (!(fabs(kd) < 4611686018427387904.0) || !(fabs(hd) < 4611686018427387904.0)) {
    set_error(st, MCC_ERR_RANGE);
    return;
  }
  f.K = (long long)kd;
  f.Qhi = (long long)hd - f.K;
  if (f.Qhi >= (1ll << 29)) { set_error(st, MCC_ERR_RANGE); return; }
  f.fill_u = -f.K;
  if (f.fill_u < 0) f.fill_u = 0;
  if (f.fill_u > f.Qhi) f.fill_u = f.Qhi;
  const double r21 = rint(__dmul_rn(__ddiv_rn(f.s2, f.s1), 1099511627776.0));
  const double r12 = rint(__dmul_rn(__ddiv_rn(f.s1, f.s2), 1099511627776.0));
  if (!(r21 >= 1.0 && r21 < 1125899906842624.0) || !(r12 >= 1.0 && r12 < 1125899906842624.0)) {
    set_error(st, MCC_ERR_INVALID_ARG);
    return;
  }
  f.rho21_q = (long long)r21;
  f.rho12_q = (long long)r12;
  f.rho21_f = __fmul_rn(__ll2float_rn(f.rho21_q), 0x1p-40f);
  f.rho12_f = __fmul_rn(__ll2float_rn(f.rho12_q), 0x1p-40f);
  f.guard = (rp.dtype == MCC_F32) || !(f.M <= __dmul_rn(f.tau2, 268435456.0));
  st->f = f;
}

template <typename T>
__global__ void __launch_bounds__(256) k_reduce(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.y);
  const T *__restrict__ x = (const T *)c.x;
  const int64_t n = A.pv.n_v;
  Status *st = c.st;
  const RParams rp = A.rp[blockIdx.y];
  unsigned int *hist = c.hist1;
  const int nhist = (int)((A.W.hist2 - A.W.hist1) / 4 + A.nsym2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nhist; i += gridDim.x * blockDim.x)
    hist[i] = 0;
  if (A.mode[blockIdx.y] == MCC_PRED_AUTO) {
    unsigned int *hb = (unsigned int *)(A.ws0 + (int64_t)blockIdx.y * A.wss + A.W.hist2b);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.nsym2; i += gridDim.x * blockDim.x)
      hb[i] = 0;
  }
  unsigned long long mn = 0, mx = 0;  // mn holds ~key (max of ~key = min key)
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // x is read with the default caching: k_prequant reads it again from L2
  if (sizeof(T) == 8) {
    auto key = [&](double v) {
      const unsigned long long b = value_bits(v);
      bad |= ((b >> 52) & 0x7FF) == 0x7FF;
      const unsigned long long k = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
      mn = max(mn, ~k);
      mx = max(mx, k);
    };
    if (((uintptr_t)x & 15) == 0) {
      // pairs as 16-byte loads, four pairs in flight per thread
      const double2 *x2 = (const double2 *)x;
      const int64_t n2 = n / 2;
      int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
      for (; j + 3 * stride < n2; j += 4 * stride) {
        double2 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = __ldg(x2 + j + u * stride);
#pragma unroll
        for (int u = 0; u < 4; u++) { key(v[u].x); key(v[u].y); }
      }
      for (; j < n2; j += stride) {
        const double2 v = __ldg(x2 + j);
        key(v.x);
        key(v.y);
      }
      if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) key((double)__ldg(x + n - 1));
    } else {
      for (; i < n; i += stride) key((double)__ldg(x + i));
    }
  } else {
    // FP32: ordered 32-bit keys (no float -> double conversion per value,
    // a slow operation on this GPU); the extremes are widened once below
    unsigned int mn32 = 0, mx32 = 0;
    for (; i < n; i += stride) {
      const unsigned int b = __float_as_uint((float)__ldg(x + i));
      bad |= ((b >> 23) & 0xFF) == 0xFF;
      const unsigned int k = (b >> 31) ? ~b : (b | 0x80000000u);
      mn32 = max(mn32, ~k);
      mx32 = max(mx32, k);
    }
    if (mx32 != 0) {  // this thread saw a value: keys of the same values as doubles
      const unsigned int klo = ~mn32, khi = mx32;
      const float flo = __uint_as_float((klo >> 31) ? (klo & 0x7FFFFFFFu) : ~klo);
      const float fhi = __uint_as_float((khi >> 31) ? (khi & 0x7FFFFFFFu) : ~khi);
      const unsigned long long blo = value_bits((double)flo), bhi = value_bits((double)fhi);
      const unsigned long long kl = (blo >> 63) ? ~blo : (blo | 0x8000000000000000ull);
      const unsigned long long kh = (bhi >> 63) ? ~bhi : (bhi | 0x8000000000000000ull);
      mn = ~kl;
      mx = kh;
    }
  }
  for (int o = 16; o; o >>= 1) {
    mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  __shared__ unsigned long long smn[8], smx[8];
  __shared__ int sbad;
  if (threadIdx.x == 0) sbad = 0;
  __syncthreads();
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    smn[w] = mn;
    smx[w] = mx;
    if (bad) sbad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
      mn = max(mn, smn[k]);
      mx = max(mx, smx[k]);
    }
    if (sbad) set_error(st, MCC_ERR_INVALID_ARG);
    atomicMax(&st->key_lo, mn);
    atomicMax(&st->key_hi, mx);
    __threadfence();
    const unsigned int ticket = atomicAdd(&st->done_blocks, 1u);
    if (ticket == gridDim.x - 1) {
      __threadfence();
      if (atomicAdd(&st->err, 0u) == 0) field_params(st, rp);
    }
  }
}

// ---------------------------------------------------------------------------
// k_prequant: Q = round(x * (1 / s2)) - K
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_prequant(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.y);
  const T *__restrict__ x = (const T *)c.x;
  const int64_t n = A.pv.n_v;
  const Status *st = c.st;
  int *__restrict__ Q = c.Q;
  if (st->err) return;
  const double inv2 = st->f.inv2;
  const long long K = st->f.K;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (A.fop[blockIdx.y] == MCC_F_CLUSTER) {
    // cluster-mean f: every vertex adds its code to the sum and count of its
    // nearest node (integer atomics: the totals do not depend on the order)
    unsigned char *ws = A.ws0 + (int64_t)blockIdx.y * A.wss;
    unsigned long long *csum = (unsigned long long *)(ws + A.W.csum);
    unsigned int *ccnt = (unsigned int *)(ws + A.W.ccnt);
    const PlanView &pv = A.pv;
    const int64_t sxy = (int64_t)pv.nx * pv.ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      const double v = (double)__ldg(x + i);
      const int q = (int)(rint_ll64(__dmul_rn(v, inv2)) - K);
      Q[i] = q;
      const uint32_t c = __ldg(pv.cell + i);
      const unsigned fx = __ldg(pv.frac + i), fy = __ldg(pv.frac + n + i);
      const uint32_t m = pv.dim == 3 ? nearest_node<3>(c, fx, fy, __ldg(pv.frac + 2 * n + i), pv.nx, sxy)
                                     : nearest_node<2>(c, fx, fy, 0u, pv.nx, sxy);
      atomicAdd(csum + m, (unsigned long long)q);  // q >= 0: the codes start at the minimum
      atomicAdd(ccnt + m, 1u);
    }
    return;
  }
  if (sizeof(T) == 8 && ((uintptr_t)x & 15) == 0) {  // pairs: 16-byte loads, 8-byte stores
    const double2 *x2 = (const double2 *)x;
    int2 *Q2 = (int2 *)Q;  // the workspace's Q is 256-byte aligned
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n / 2; j += stride) {
      const double2 v = __ldg(x2 + j);
      Q2[j] = make_int2((int)(rint_ll64(__dmul_rn(v.x, inv2)) - K),
                        (int)(rint_ll64(__dmul_rn(v.y, inv2)) - K));
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0)
      Q[n - 1] = (int)(rint_ll64(__dmul_rn((double)__ldg(x + n - 1), inv2)) - K);
    return;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const double v = (double)__ldg(x + i);
    Q[i] = (int)(rint_ll64(__dmul_rn(v, inv2)) - K);
  }
}

// ---------------------------------------------------------------------------
// k_delta1d: the 1D coder's symbols, delta_i = Q_i - Q_(i-1) (delta_0 = Q_0),
// in component 1 (symbol delta + R1 or an escape), with its histogram
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hist_add(unsigned int *sh, int sym, bool valid);

__global__ void __launch_bounds__(256) k_delta1d(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.y);
  Status *st = c.st;
  extern __shared__ unsigned int shist[];
  if (block_failed(st)) return;
  const int R1 = A.R1, nsym = 2 * R1;
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) shist[i] = 0;
  __syncthreads();
  const int64_t n = A.pv.n_g;
  const int *__restrict__ Q = c.Q;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nloop = (n + stride - 1) / stride * stride;  // uniform trip count per warp
  unsigned int nesc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nloop; i += stride) {
    const bool valid = i < n;
    int sym = 0;
    if (valid) {
      const int d = wsub(__ldg(Q + i), i ? __ldg(Q + i - 1) : 0);
      if (d >= -(R1 - 1) && d <= R1 - 2) {
        sym = d + R1;
      } else {
        c.val1[i] = d;
        nesc++;
      }
      c.sym1[i] = (unsigned short)sym;
    }
    hist_add(shist, sym, valid);
  }
  if (nesc) atomicAdd(&st->nout1, nesc);
  __syncthreads();
  for (int i = threadIdx.x; i < nsym; i += blockDim.x)
    if (shist[i]) atomicAdd(c.hist1 + i, shist[i]);
}

// ---------------------------------------------------------------------------
// grid codes: x1 = f(x) on the vertex codes, rescaled to grid bins
// ---------------------------------------------------------------------------
// Grid codes of U points at once: every point's plan entries, then every
// vertex code, are loaded before any is used (the gathers overlap).
// Open loop: x1v (or NULL) receives, at the points flagged in own, the grid
// value before quantisation (vertex bins, a + acc; FP64 work, done only then).
template <int DIM, int U>
__device__ __forceinline__ void grid_codes(const int64_t (&j)[U], const bool (&ok)[U],
                                           const PlanView &pv, const int *__restrict__ Q,
                                           const FieldParams &f, Status *st, int (&out)[U],
                                           double *__restrict__ x1v, const bool (&own)[U]) {
  int v[U][DIM + 1];
  float lf[U][DIM];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const int64_t jj = ok[u] ? j[u] : 0;
    // the plan records are streamed once per call (evict-first: the gathered
    // vertex codes stay in L2)
    const int4 vv = __ldcs(pv.vid4 + jj);
    unsigned int lk[3];
    if (DIM == 2) {  // the weights share the record (lam1 | lam2 << 16)
      lk[0] = (unsigned int)vv.w & 0xFFFFu;
      lk[1] = (unsigned int)vv.w >> 16;
      lk[2] = 0;
    } else {
      const ushort4 ll = __ldcs(pv.lam4 + jj);
      lk[0] = ll.x;
      lk[1] = ll.y;
      lk[2] = ll.z;
    }
    const int vk[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
    for (int k = 0; k <= DIM; k++) v[u][k] = vk[k];
#pragma unroll
    for (int k = 0; k < DIM; k++) lf[u][k] = __fmul_rn(__uint2float_rn(lk[k]), 0x1p-15f);
    if (!ok[u]) v[u][0] = -1;
  }
  int qv[U][DIM + 1];
#pragma unroll
  for (int u = 0; u < U; u++)
#pragma unroll
    for (int k = 0; k <= DIM; k++) qv[u][k] = v[u][0] >= 0 ? __ldg(Q + v[u][k]) : 0;
#pragma unroll
  for (int u = 0; u < U; u++) {
    int a;  // a vertex code or the fill value: both in [0, Qhi], Qhi < 2^29
    float acc = 0.0f;
    if (v[u][0] < 0) {
      a = (int)f.fill_u;
    } else {
      const int qa = qv[u][0];
      a = qa;
#pragma unroll
      for (int k = 1; k <= DIM; k++) {
        const int dk = wsub(qv[u][k], qa);
        acc = k == 1 ? __fmul_rn(__int2float_rn(dk), lf[u][0])
                     : __fmaf_rn(__int2float_rn(dk), lf[u][k - 1], acc);
      }
    }
    const long long q = rescale(a, acc, f.rho21_q, f.rho21_f);
    if (x1v && own[u]) x1v[j[u]] = __dadd_rn((double)a, (double)acc);
    out[u] = 0;
    if (!ok[u]) continue;
    if (q <= -(1ll << 27) || q >= (1ll << 27)) set_error(st, MCC_ERR_RANGE);
    else out[u] = (int)q;
  }
}

// Cluster-mean f (Sec. III-C) at U grid points: the mean of the codes of the
// vertices whose nearest node is the point, as integer part a = S / n and
// fraction (S - a n) / n in FP32, rescaled to grid bins; a point no vertex is
// nearest to takes the fill value.
template <int U>
__device__ __forceinline__ void grid_codes_cluster(const int64_t (&j)[U], const bool (&ok)[U],
                                                   const unsigned long long *__restrict__ csum,
                                                   const unsigned int *__restrict__ ccnt,
                                                   const FieldParams &f, Status *st, int (&out)[U],
                                                   double *__restrict__ x1v,
                                                   const bool (&own)[U]) {
  unsigned long long S[U];
  unsigned int cnt[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    S[u] = ok[u] ? __ldg(csum + j[u]) : 0ull;
    cnt[u] = ok[u] ? __ldg(ccnt + j[u]) : 0u;
  }
#pragma unroll
  for (int u = 0; u < U; u++) {
    int a;
    float acc = 0.0f;
    if (cnt[u] == 0) {
      a = (int)f.fill_u;
    } else {
      const unsigned long long a64 = S[u] / cnt[u];
      a = (int)a64;
      acc = __fdiv_rn(__uint2float_rn((unsigned int)(S[u] - a64 * cnt[u])), __uint2float_rn(cnt[u]));
    }
    const long long q = rescale(a, acc, f.rho21_q, f.rho21_f);
    if (x1v && own[u]) x1v[j[u]] = __dadd_rn((double)a, (double)acc);
    out[u] = 0;
    if (!ok[u]) continue;
    if (q <= -(1ll << 27) || q >= (1ll << 27)) set_error(st, MCC_ERR_RANGE);
    else out[u] = (int)q;
  }
}

// Shared-memory histogram add, aggregated over lanes holding the same symbol.
__device__ __forceinline__ void hist_add(unsigned int *sh, int sym, bool valid) {
  const int key = valid ? sym : -1;
  const unsigned same = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (valid && (__ffs(same) - 1) == lane) atomicAdd(sh + sym, (unsigned)__popc(same));
}

template <int TX, int TY>
__global__ void __launch_bounds__(256) k_grid2d(const __grid_constant__ CompArgs A) {
  pdl_wait();
  // blocks are field-fastest so that the fields of a batch share plan tiles in L2
  const Ctx c = ctx_of(A, blockIdx.x);
  const PlanView &pv = A.pv;
  const int *__restrict__ Q = c.Q;
  Status *st = c.st;
  const int R1 = A.R1;
  int *__restrict__ q1 = c.q1;
  double *__restrict__ x1v =
      A.open[blockIdx.x] ? (double *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.x1v) : nullptr;
  const bool cluster = A.fop[blockIdx.x] == MCC_F_CLUSTER;
  const unsigned long long *csum =
      (const unsigned long long *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.csum);
  const unsigned int *ccnt = (const unsigned int *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.ccnt);
  unsigned short *__restrict__ sym1 = c.sym1;
  int *__restrict__ val1 = c.val1;
  unsigned int *hist1 = c.hist1;
  extern __shared__ unsigned int shist[];
  __shared__ int s[TY + 1][TX + 1];
  if (block_failed(st)) return;
  const int nsym = 2 * R1;
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) shist[i] = 0;
  const FieldParams f = st->f;
  const int nx = pv.nx, ny = pv.ny;
  const int x0 = blockIdx.y * TX, y0 = blockIdx.z * TY;
  {  // the tile with its halo row and column: every thread's points at once
    constexpr int NP = (TY + 1) * (TX + 1), U = (NP + 255) / 256;
    int64_t j[U];
    bool ok[U];
    int q[U];
    bool own[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int idx = threadIdx.x + 256 * u;
      const int ly = idx / (TX + 1), lx = idx - ly * (TX + 1);
      const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
      ok[u] = idx < NP && gx >= 0 && gy >= 0 && gx < nx && gy < ny;
      own[u] = ok[u] && lx > 0 && ly > 0;
      j[u] = gx + (int64_t)nx * gy;
    }
    if (cluster) grid_codes_cluster<U>(j, ok, csum, ccnt, f, st, q, x1v, own);
    else grid_codes<2, U>(j, ok, pv, Q, f, st, q, x1v, own);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int idx = threadIdx.x + 256 * u;
      if (idx >= NP) continue;
      const int ly = idx / (TX + 1), lx = idx - ly * (TX + 1);
      if (own[u]) q1[j[u]] = q[u];
      s[ly][lx] = q[u];
    }
  }
  __syncthreads();
  unsigned int nesc = 0;
  for (int idx = threadIdx.x; idx < TY * TX; idx += blockDim.x) {
    const int ly = idx / TX, lx = idx - ly * TX;
    const int gx = x0 + lx, gy = y0 + ly;
    const bool valid = gx < nx && gy < ny;
    int sym = 0;
    if (valid) {
      const int d = wadd(wsub(wsub(s[ly + 1][lx + 1], s[ly + 1][lx]), s[ly][lx + 1]), s[ly][lx]);
      const int64_t j = gx + (int64_t)nx * gy;
      if (d >= -(R1 - 1) && d <= R1 - 2) {
        sym = d + R1;
      } else {
        sym = 0;
        val1[j] = d;
        nesc++;
      }
      sym1[j] = (unsigned short)sym;
    }
    hist_add(shist, sym, valid);
  }
  if (nesc) atomicAdd(&st->nout1, nesc);
  __syncthreads();
  for (int i = threadIdx.x; i < nsym; i += blockDim.x)
    if (shist[i]) atomicAdd(hist1 + i, shist[i]);
}

// 3D grid codes: f and the rescale once per grid point (U points per thread,
// their plan records and vertex-code gathers issued together); k_grid3d then
// takes the Lorenzo differences from q1, halo included, with no point
// computed twice. Four resident blocks per SM (64 registers, no spills)
// keep more gathers in flight.
__global__ void __launch_bounds__(256, 4) k_grid_codes3d(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.x);
  const PlanView &pv = A.pv;
  Status *st = c.st;
  int *__restrict__ q1 = c.q1;
  double *__restrict__ x1v =
      A.open[blockIdx.x] ? (double *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.x1v) : nullptr;
  const bool cluster = A.fop[blockIdx.x] == MCC_F_CLUSTER;
  const unsigned long long *csum =
      (const unsigned long long *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.csum);
  const unsigned int *ccnt = (const unsigned int *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.ccnt);
  if (block_failed(st)) return;
  const FieldParams f = st->f;
  constexpr int U = 4;
  const int64_t n_g = pv.n_g;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  for (int64_t j0 = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; j0 < n_g; j0 += U * stride) {
    int64_t j[U];
    bool ok[U];
    int q[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      j[u] = j0 + u * stride;
      ok[u] = j[u] < n_g;
    }
    if (cluster) grid_codes_cluster<U>(j, ok, csum, ccnt, f, st, q, x1v, ok);
    else grid_codes<3, U>(j, ok, pv, c.Q, f, st, q, x1v, ok);
#pragma unroll
    for (int u = 0; u < U; u++)
      if (ok[u]) q1[j[u]] = q[u];
  }
}

// 3D: tiles of TX x TY points walking a segment of SZ planes in z; the tile
// and its halo (the plane below, the row and column before) are read from q1.
template <int TX, int TY, int SZ>
__global__ void __launch_bounds__(TX *TY) k_grid3d(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.x);
  const PlanView &pv = A.pv;
  Status *st = c.st;
  const int R1 = A.R1;
  int *__restrict__ q1 = c.q1;
  unsigned short *__restrict__ sym1 = c.sym1;
  int *__restrict__ val1 = c.val1;
  unsigned int *hist1 = c.hist1;
  const int txs = (A.pv.nx + TX - 1) / TX;
  extern __shared__ unsigned int shist[];
  // the tile with its halo plane, row and column
  __shared__ int s[SZ + 1][TY + 1][TX + 1];
  if (block_failed(st)) return;
  const int nsym = 2 * R1;
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) shist[i] = 0;
  const int nx = pv.nx, ny = pv.ny, nz = pv.nz;
  const int x0 = (blockIdx.y % txs) * TX, y0 = (blockIdx.y / txs) * TY, z0 = blockIdx.z * SZ;
  const int64_t sxy = (int64_t)nx * ny;
  constexpr int NP = (SZ + 1) * (TY + 1) * (TX + 1), U = 4;
  constexpr int NT = TX * TY;
  for (int base = 0; base < NP; base += U * NT) {  // U points per thread at once
    int q[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int idx = base + threadIdx.x + NT * u;
      const int lz = idx / ((TY + 1) * (TX + 1)), rem = idx - lz * ((TY + 1) * (TX + 1));
      const int ly = rem / (TX + 1), lx = rem - ly * (TX + 1);
      const int gx = x0 - 1 + lx, gy = y0 - 1 + ly, gz = z0 - 1 + lz;
      const bool ok = idx < NP && gx >= 0 && gy >= 0 && gz >= 0 && gx < nx && gy < ny && gz < nz;
      q[u] = ok ? __ldcg(q1 + gx + (int64_t)nx * gy + sxy * gz) : 0;  // 0 outside the grid
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int idx = base + threadIdx.x + NT * u;
      if (idx >= NP) continue;
      const int lz = idx / ((TY + 1) * (TX + 1)), rem = idx - lz * ((TY + 1) * (TX + 1));
      const int ly = rem / (TX + 1), lx = rem - ly * (TX + 1);
      s[lz][ly][lx] = q[u];
    }
  }
  __syncthreads();
  unsigned int nesc = 0;
  // each thread walks one (x, y) column of the tile along z: the 3D Lorenzo
  // difference is the plane's 2D difference e(z) minus e(z - 1), the latter
  // kept from the previous step (the same sum as the 7-neighbour form,
  // wrapping int32 arithmetic)
  const int ly = threadIdx.x / TX, lx = threadIdx.x - ly * TX;
  auto plane_diff = [&](int zz) {  // 2D Lorenzo difference in tile plane zz
    int e = s[zz][ly + 1][lx + 1];
    e = wsub(e, s[zz][ly + 1][lx]);
    e = wsub(e, s[zz][ly][lx + 1]);
    return wadd(e, s[zz][ly][lx]);
  };
  int e_prev = plane_diff(0);
  for (int lz = 0; lz < SZ; lz++) {
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    const bool valid = gx < nx && gy < ny && gz < nz;
    int sym = 0;
    const int e_cur = plane_diff(lz + 1);
    const int d = wsub(e_cur, e_prev);
    e_prev = e_cur;
    if (valid) {
      const int64_t j = gx + (int64_t)nx * gy + sxy * gz;
      if (d >= -(R1 - 1) && d <= R1 - 2) {
        sym = d + R1;
      } else {
        sym = 0;
        val1[j] = d;
        nesc++;
      }
      sym1[j] = (unsigned short)sym;
    }
    hist_add(shist, sym, valid);
  }
  if (nesc) atomicAdd(&st->nout1, nesc);
  __syncthreads();
  for (int i = threadIdx.x; i < nsym; i += blockDim.x)
    if (shist[i]) atomicAdd(hist1 + i, shist[i]);
}

// ---------------------------------------------------------------------------
// k_node: residual codes at the vertices
// ---------------------------------------------------------------------------
// Residual symbol of one vertex: raw (guard failed or the code leaves int32),
// a code within the alphabet, or an escape whose value goes to val2.
__device__ __forceinline__ int residual_symbol(long long q2, bool guard_fail, int R2, int64_t i,
                                               int *__restrict__ val2) {
  if (guard_fail || q2 <= -2147483648ll || q2 > 2147483647ll) return 2 * R2 - 1;  // INT32_MIN reserved
  if (q2 >= -(R2 - 1) && q2 <= R2 - 2) return (int)q2 + R2;
  val2[i] = (int)q2;
  return 0;
}

// Open loop (Algorithm 3 as printed): q2 = round(x / s2 - K - g(x1)) with
// x1 the grid values before quantisation, evaluated as (Q - g) + (u - rint(u))
// (u = x / s2) so that both terms stay small; every vertex is reconstructed
// as the decompressor will, s2 (K + q2 + g(x1')), and checked against
// tau1 + tau2 after the cast to T (Sec. III); violators are stored raw.
template <int DIM, typename T>
__device__ __forceinline__ void node_open(const CompArgs &A, const Ctx &c, const FieldParams &f,
                                          unsigned int *shist) {
  const PlanView &pv = A.pv;
  const T *__restrict__ x = (const T *)c.x;
  const int *__restrict__ Q = c.Q;
  const int *__restrict__ q1 = c.q1;
  const double *__restrict__ x1v =
      (const double *)(A.ws0 + (int64_t)blockIdx.x * A.wss + A.W.x1v);
  unsigned short *__restrict__ sym2 = c.sym2;
  const int R2 = A.R2;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const double tau = __dadd_rn(f.tau1, f.tau2);
  const bool near = A.gop[blockIdx.x] == MCC_G_NEAREST;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  const int64_t nloop = (n + stride - 1) / stride * stride;  // uniform trip count per warp
  for (int64_t i0 = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i0 < nloop; i0 += stride) {
    const bool valid = i0 < n;
    int sym = 0;
    if (valid) {
      const int64_t i = i0;
      const uint32_t cl = __ldg(pv.cell + i);
      const float fx = __fmul_rn(__uint2float_rn(__ldg(pv.frac + i)), 0x1p-15f);
      const float fy = __fmul_rn(__uint2float_rn(__ldg(pv.frac + n + i)), 0x1p-15f);
      const float fz =
          DIM == 3 ? __fmul_rn(__uint2float_rn(__ldg(pv.frac + 2 * n + i)), 0x1p-15f) : 0.0f;
      double gv, gq;
      if (near) {  // nearest-node g: the node's values themselves
        const uint32_t m = nearest_node<DIM>(cl, __ldg(pv.frac + i), __ldg(pv.frac + n + i),
                                             DIM == 3 ? __ldg(pv.frac + 2 * n + i) : 0u, nx, sxy);
        gv = __ldg(x1v + m);
        gq = __dmul_rn((double)__ldg(q1 + m), __dmul_rn((double)f.rho12_q, 0x1p-40));
      } else {
        double cv[8];
        cv[0] = __ldg(x1v + cl);
        cv[1] = __ldg(x1v + cl + 1);
        cv[2] = __ldg(x1v + cl + nx);
        cv[3] = __ldg(x1v + cl + nx + 1);
        if (DIM == 3) {
          cv[4] = __ldg(x1v + cl + sxy);
          cv[5] = __ldg(x1v + cl + sxy + 1);
          cv[6] = __ldg(x1v + cl + sxy + nx);
          cv[7] = __ldg(x1v + cl + sxy + nx + 1);
        }
        int cor[8];
        corner_codes<DIM>(q1, cl, nx, sxy, cor);
        gv = interp64<DIM>(cv, fx, fy, fz);
        gq = interp64_codes<DIM>(cor, f.rho12_q, fx, fy, fz);
      }
      const double v = (double)__ldg(x + i);
      const int Qi = __ldg(Q + i);
      const double u = __dmul_rn(v, f.inv2);
      const double r = __dadd_rn(__dsub_rn((double)Qi, gv), __dsub_rn(u, rint(u)));
      const double q2d = rint(r);
      bool raw = !(fabs(q2d) < 2147483647.0);
      const long long q2 = raw ? 0 : (long long)q2d;
      if (!raw) {
        const double xr = __dmul_rn(f.s2, __dadd_rn((double)(f.K + q2), gq));
        const double xo = sizeof(T) == 8 ? xr : (double)__double2float_rn(xr);
        raw = !(fabs(__dsub_rn(v, xo)) <= tau);
      }
      sym = residual_symbol(q2, raw, R2, i, c.val2);
      sym2[i] = (unsigned short)sym;
    }
    hist_add(shist, sym, valid);
  }
}

// Closed loop with the nearest-node g (Sec. III-B): P = round((s1/s2) q1[m])
// with m the vertex's nearest node, one gather per vertex (four vertices per
// thread and iteration); the guard as in the interpolating path.
template <int DIM, typename T>
__device__ __forceinline__ void node_nearest(const CompArgs &A, const Ctx &c, const FieldParams &f,
                                             unsigned int *shist) {
  const PlanView &pv = A.pv;
  const T *__restrict__ x = (const T *)c.x;
  const int *__restrict__ Q = c.Q;
  const int *__restrict__ q1 = c.q1;
  unsigned short *__restrict__ sym2 = c.sym2;
  const int R2 = A.R2;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  constexpr int U = 4;
  const int64_t nloop = (n + U * stride - 1) / (U * stride) * (U * stride);
  for (int64_t i0 = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i0 < nloop; i0 += U * stride) {
    int64_t iv[U];
    iv[0] = i0;
#pragma unroll
    for (int u = 1; u < U; u++) iv[u] = iv[u - 1] + stride;
    uint32_t m[U];
    int Qv[U], qm[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = iv[u] < n ? iv[u] : 0;
      m[u] = nearest_node<DIM>(__ldg(pv.cell + i), __ldg(pv.frac + i), __ldg(pv.frac + n + i),
                               DIM == 3 ? __ldg(pv.frac + 2 * n + i) : 0u, nx, sxy);
      Qv[u] = __ldg(Q + i);
    }
#pragma unroll
    for (int u = 0; u < U; u++) qm[u] = __ldg(q1 + m[u]);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = iv[u];
      const bool valid = i < n;
      int sym = 0;
      if (valid) {
        bool gfail = false;
        if (f.guard) {
          const double v = (double)__ldg(x + i);
          const double xr = __dmul_rn(f.s2, (double)((long long)Qv[u] + f.K));
          const double xo = sizeof(T) == 8 ? xr : (double)__double2float_rn(xr);
          gfail = fabs(__dsub_rn(v, xo)) > f.tau2;
        }
        const long long P = rescale(qm[u], 0.0f, f.rho12_q, f.rho12_f);
        sym = residual_symbol((long long)Qv[u] - P, gfail, R2, i, c.val2);
        sym2[i] = (unsigned short)sym;
      }
      hist_add(shist, sym, valid);
    }
  }
}

// HAS_P: some field of the launch uses the learned predictor (mode 1) or
// chooses between both (mode 2: the plain side goes to sym2 / hist2, the
// learned side to sym2b / hist2b; the histograms share the dynamic shared
// memory, the learned one at offset 2 R2). OPEN: some field of the launch
// takes the open loop (node_open; such a field has no model).
template <int DIM, typename T, bool HAS_P, bool OPEN>
__global__ void __launch_bounds__(256) k_node(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const int fi = blockIdx.x;
  const Ctx c = ctx_of(A, fi);
  const PlanView &pv = A.pv;
  const T *__restrict__ x = (const T *)c.x;
  const int *__restrict__ Q = c.Q;
  const int *__restrict__ q1 = c.q1;
  Status *st = c.st;
  const int R2 = A.R2;
  unsigned short *__restrict__ sym2 = c.sym2;
  int *__restrict__ val2 = c.val2;
  unsigned char *ws = A.ws0 + (int64_t)fi * A.wss;
  unsigned short *__restrict__ sym2b = (unsigned short *)(ws + A.W.sym2b);
  int *__restrict__ val2b = (int *)(ws + A.W.val2b);
  extern __shared__ unsigned int shist[];
  if (block_failed(st)) return;
  const int mode = HAS_P ? A.mode[fi] : MCC_PRED_ZERO;
  const bool both = mode == MCC_PRED_AUTO;
  const int nsym = 2 * R2;
  for (int i = threadIdx.x; i < (both ? 2 : 1) * nsym; i += blockDim.x) shist[i] = 0;
  __syncthreads();
  const FieldParams f = st->f;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const float *__restrict__ pcor = c.p;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  // U vertices per thread and iteration (2 in 2D, 1 in 3D), their gathers
  // issued together; uniform trip count per warp
  constexpr int U = DIM == 2 ? 2 : 1;
  const int64_t nloop = (n + U * stride - 1) / (U * stride) * (U * stride);
  if (OPEN && A.open[fi]) node_open<DIM, T>(A, c, f, shist);
  else if (OPEN && A.gop[fi] == MCC_G_NEAREST) node_nearest<DIM, T>(A, c, f, shist);
  else
  for (int64_t i0 = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; i0 < nloop; i0 += U * stride) {
    int64_t iv[U];
    iv[0] = i0;
#pragma unroll
    for (int u = 1; u < U; u++) iv[u] = iv[u - 1] + stride;
    bool valid[U];
    uint32_t cl[U];
    float fr[U][3];
    int Qv[U];
    int cor[U][8];
#pragma unroll
    for (int u = 0; u < U; u++) {
      valid[u] = iv[u] < n;
      const int64_t i = valid[u] ? iv[u] : 0;
      vertex_record<DIM>(pv.vrec, i, cl[u], fr[u]);
      Qv[u] = __ldcs(Q + i);
    }
#pragma unroll
    for (int u = 0; u < U; u++) corner_codes<DIM>(q1, cl[u], nx, sxy, cor[u]);
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t i = iv[u];
      int sym = 0, symb = 0;
      if (valid[u]) {
        const int Qi = Qv[u];
        const float acc = interp_acc<DIM>(cor[u], fr[u][0], fr[u][1], fr[u][2]);
        const int c000 = cor[u][0];
        bool gfail = false;
        if (f.guard) {  // reconstruct as the decompressor will and check |x - x'|
          const double v = (double)__ldg(x + i);
          const double xr = __dmul_rn(f.s2, (double)((long long)Qi + f.K));
          const double xo = sizeof(T) == 8 ? xr : (double)__double2float_rn(xr);
          gfail = fabs(__dsub_rn(v, xo)) > f.tau2;
        }
        const float pc = mode != MCC_PRED_ZERO ? __ldg(pcor + i) : 0.0f;
        if (both) {
          const long long P0 = rescale<false>(c000, acc, f.rho12_q, f.rho12_f);
          const long long P1 = rescale<true>(c000, acc, f.rho12_q, f.rho12_f, pc);
          sym = residual_symbol((long long)Qi - P0, gfail, R2, i, val2);
          symb = residual_symbol((long long)Qi - P1, gfail, R2, i, val2b);
          sym2b[i] = (unsigned short)symb;
        } else {
          const long long P = rescale<HAS_P>(c000, acc, f.rho12_q, f.rho12_f, pc);
          sym = residual_symbol((long long)Qi - P, gfail, R2, i, val2);
        }
        sym2[i] = (unsigned short)sym;
      }
      hist_add(shist, sym, valid[u]);
      if (both) hist_add(shist + nsym, symb, valid[u]);
    }
  }
  __syncthreads();
  unsigned int *hist2b = (unsigned int *)(ws + A.W.hist2b);
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) {
    if (shist[i]) atomicAdd(c.hist2 + i, shist[i]);
    if (both && shist[nsym + i]) atomicAdd(hist2b + i, shist[nsym + i]);
  }
}

// ---------------------------------------------------------------------------
// k_codebook: canonical Huffman code book of one component per CTA.
//
// The used symbols' (count, symbol) keys are gathered by a shared counter and
// bitonic-sorted at the next power of two of their number (with the
// zero-run stage the symbol R takes no count: its zeros are coded as run
// tokens 2R, 2R + 1). Code lengths follow the two-queue construction over
// the leaves sorted by (count, symbol): each step takes the two lightest nodes, a leaf before an
// internal node of equal weight, internal nodes in creation order. The pick
// sequence is the sorted merge of the leaves and the internal nodes, and
// internal node k is the sum of picks 2k and 2k+1; nodes created from picks
// of weight >= t weigh >= 2t, so every queued node of weight <= 2t (t the
// next pick) is picked before any node created from them. Rounds therefore
// merge that whole batch in parallel (ranks by binary search), pair it into
// new nodes, and fall back to single-thread steps when the batch is small.
// Depths by pointer jumping; counts halved (c -> max(1, c >> 1)) while a code
// exceeds lmax.
// ---------------------------------------------------------------------------
struct CodebookArgs {
  const unsigned int *hist;
  int nsym;
  unsigned int *code;
  unsigned char *len;
  unsigned char *stream_lens;  // the 2R symbols' lengths in the stream (or NULL)
  int zsym;                    // the zero-run stage's zero symbol R (no token), or -1
};

constexpr int kBatchMin = 24;

__device__ __forceinline__ unsigned long long node_w(int e, int m, const unsigned long long *sk,
                                                     const unsigned long long *Iw) {
  return e < m ? (sk[e] >> 32) : Iw[e - m];
}

__global__ void __launch_bounds__(1024) k_codebook(const __grid_constant__ CompArgs AA) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  const Ctx c = ctx_of(AA, blockIdx.y);
  Status *st = c.st;
  const int lmax = AA.lmax;
  if (block_failed(st)) return;
  const int bx = (int)blockIdx.x + AA.bx0;
  const bool c1 = bx == 0;
  // block 2: the learned side of an auto field; with auto, k_choose writes
  // the residual code lengths into the stream
  const bool side_b = bx == 2;
  const bool autof = AA.mode[blockIdx.y] == MCC_PRED_AUTO;
  if (side_b && !autof) return;
  unsigned char *ws = AA.ws0 + (int64_t)blockIdx.y * AA.wss;
  const CodebookArgs A{c1 ? c.hist1 : (side_b ? (const unsigned int *)(ws + AA.W.hist2b) : c.hist2),
                       c1 ? AA.nsym1 : AA.nsym2,
                       c1 ? c.code1 : (side_b ? (unsigned int *)(ws + AA.W.code2b) : c.code2),
                       c1 ? c.len1 : (side_b ? ws + AA.W.len2b : c.len2),
                       c1 ? c.out + AA.F.lens1 : (autof ? nullptr : c.out + AA.F.lens2),
                       AA.zr[blockIdx.y] ? (c1 ? AA.R1 : AA.R2) : -1};
  const int nsym = A.nsym;
  const int nstream = c1 ? 2 * AA.R1 : 2 * AA.R2;  // lengths stored in the lens section
  int npn = 1;  // power of two >= nsym: the shared-memory size of the sort
  while (npn < nsym) npn <<= 1;
  unsigned int *cnt = (unsigned int *)smem;                                // [nsym]
  unsigned long long *keyA = (unsigned long long *)(cnt + nsym);           // [nsym] (nsym even)
  unsigned long long *sk = keyA + nsym;                                    // [npn]
  unsigned long long *Iw = sk + npn;                                       // [nsym]
  unsigned short *parent = (unsigned short *)(Iw + nsym);                  // [2 nsym]
  unsigned short *anc1 = parent + 2 * nsym;                                // [2 nsym]
  unsigned short *mid = anc1 + 2 * nsym;                                   // [2 nsym]
  unsigned short *rank = mid + 2 * nsym;                                   // [nsym]
  unsigned char *lens = (unsigned char *)(rank + nsym);                    // [nsym]
  unsigned short *dep0 = (unsigned short *)keyA;                           // reuse [2 nsym]
  unsigned short *dep1 = dep0 + 2 * nsym;                                  // reuse [2 nsym]
  __shared__ unsigned int wcount[32][kMaxLen + 1];
  __shared__ CanonTables ct;
  __shared__ int m_sh, kpos, maxlen, sa, sb, sc, snl, sni, snleaf;

  const int tid = threadIdx.x;
  if (tid == 0) m_sh = 0;
  __syncthreads();
  {
    int mloc = 0;
    for (int s = tid; s < nsym; s += blockDim.x) {
      // with the zero-run stage the zero symbol is coded as run digits only
      cnt[s] = s == A.zsym ? 0u : A.hist[s];
      lens[s] = 0;
      mloc += cnt[s] != 0;
    }
    for (int o = 16; o; o >>= 1) mloc += __shfl_xor_sync(0xffffffffu, mloc, o);
    if ((tid & 31) == 0 && mloc) atomicAdd(&m_sh, mloc);
  }
  __syncthreads();
  const int m = m_sh;
  if (m == 1) {
    for (int s = tid; s < nsym; s += blockDim.x)
      if (cnt[s]) lens[s] = 1;
  }
  for (int round = 0; m >= 2; round++) {
    if (round > 64) {  // cannot happen with 2R <= 2^lmax (checked on the host)
      if (tid == 0) set_error(st, MCC_ERR_INVALID_ARG);
      return;
    }
    if (tid == 0) { kpos = 0; maxlen = 0; sa = 0; sb = 0; sc = 0; }
    __syncthreads();
    // the m used symbols' (count, symbol) keys, compacted into keyA in any
    // order (the sort fixes it)
    for (int s = tid; s < nsym; s += blockDim.x)
      if (cnt[s]) keyA[atomicAdd(&kpos, 1)] = ((unsigned long long)cnt[s] << 32) | (unsigned)s;
    __syncthreads();
    int mp = 1;  // power of two >= m: the sort's width (padding carries ~0)
    while (mp < m) mp <<= 1;
    // bitonic sort of the keys into sk: sk[0 .. m) are the used symbols in
    // (count, symbol) order
    if ((int)blockDim.x >= mp) {
      // one key per thread; partners closer than 32 by warp shuffles
      unsigned long long x = tid < m ? keyA[tid] : ~0ull;
      for (int kk = 2; kk <= mp; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
          unsigned long long y;
          if (j >= 32) {
            if (tid < mp) sk[tid] = x;
            __syncthreads();
            y = tid < mp ? sk[tid ^ j] : x;
            __syncthreads();
          } else {
            y = __shfl_xor_sync(0xffffffffu, x, j);
          }
          const bool up = (tid & kk) == 0, lower = (tid & j) == 0;
          x = (lower == up) ? (x < y ? x : y) : (x < y ? y : x);
        }
      if (tid < mp) sk[tid] = x;
      __syncthreads();
    } else {
      for (int i = tid; i < mp; i += blockDim.x) sk[i] = i < m ? keyA[i] : ~0ull;
      __syncthreads();
      for (int kk = 2; kk <= mp; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
          for (int i = tid; i < mp; i += blockDim.x) {
            const int q = i ^ j;
            if (q > i) {
              const unsigned long long x0 = sk[i], x1 = sk[q];
              if ((x0 > x1) == ((i & kk) == 0)) { sk[i] = x1; sk[q] = x0; }
            }
          }
          __syncthreads();
        }
    }
    for (;;) {
      if (tid == 0) {
        const int a = sa, b = sb, c = sc;
        int nl = 0, ni = 0;
        if (c < m - 1) {
          const bool leaf = a < m && (b >= c || (sk[a] >> 32) <= Iw[b]);
          const unsigned long long T = 2 * (leaf ? (sk[a] >> 32) : Iw[b]);
          int lo = a, hi = m;  // first leaf with weight > T
          while (lo < hi) { const int md = (lo + hi) >> 1; if ((sk[md] >> 32) <= T) lo = md + 1; else hi = md; }
          nl = lo - a;
          lo = b; hi = c;      // first queued internal node with weight > T
          while (lo < hi) { const int md = (lo + hi) >> 1; if (Iw[md] <= T) lo = md + 1; else hi = md; }
          ni = lo - b;
          if (nl + ni < kBatchMin) {
            // small batches: single-thread two-queue steps until a large
            // batch of leaves becomes available (a heuristic: any stopping
            // point gives the same tree)
            int aa = a, bb = b, cc = c;
            // queue heads kept in registers: the next leaf's weight and the
            // next internal node's (internal nodes are appended at cc)
            unsigned long long wl = aa < m ? sk[aa] >> 32 : ~0ull;
            unsigned long long wi = bb < cc ? Iw[bb] : ~0ull;
            for (int s = 0; s < 512 && cc < m - 1; s++) {
              int id[2];
              unsigned long long w[2];
#pragma unroll
              for (int r = 0; r < 2; r++) {
                const bool lf = aa < m && (bb >= cc || wl <= wi);
                if (lf) {
                  id[r] = aa; w[r] = wl; aa++;
                  wl = aa < m ? sk[aa] >> 32 : ~0ull;
                } else {
                  id[r] = m + bb; w[r] = wi; bb++;
                  wi = bb < cc ? Iw[bb] : ~0ull;
                }
              }
              const unsigned long long wn = w[0] + w[1];
              Iw[cc] = wn;
              parent[id[0]] = (unsigned short)(m + cc);
              parent[id[1]] = (unsigned short)(m + cc);
              if (bb == cc) wi = wn;  // the new node heads an empty queue
              cc++;
              if (cc >= m - 1 || aa + kBatchMin >= m) continue;
              const unsigned long long tn = (bb >= cc || wl <= wi) ? wl : wi;
              if ((sk[aa + kBatchMin] >> 32) <= 2 * tn) break;
            }
            sa = aa; sb = bb; sc = cc;
            nl = 0; ni = 0;
          }
        }
        snl = nl; sni = ni; snleaf = 0;
      }
      __syncthreads();
      const int a = sa, b = sb, c = sc, nl = snl, ni = sni;
      __syncthreads();  // every thread holds the round state before it changes
      if (c >= m - 1) break;
      if (nl + ni == 0) continue;  // a sequential round ran
      // parallel batch: merge ranks (leaf first on equal weight)
      for (int i = tid; i < nl + ni; i += blockDim.x) {
        int pos;
        if (i < nl) {
          const unsigned long long w = sk[a + i] >> 32;
          int lo = 0, hi = ni;  // internal nodes with weight < w
          while (lo < hi) { const int md = (lo + hi) >> 1; if (Iw[b + md] < w) lo = md + 1; else hi = md; }
          pos = i + lo;
          mid[pos] = (unsigned short)(a + i);
        } else {
          const int j = i - nl;
          const unsigned long long w = Iw[b + j];
          int lo = 0, hi = nl;  // leaves with weight <= w
          while (lo < hi) { const int md = (lo + hi) >> 1; if ((sk[a + md] >> 32) <= w) lo = md + 1; else hi = md; }
          pos = j + lo;
          mid[pos] = (unsigned short)(m + b + j);
        }
      }
      __syncthreads();
      const int be = (nl + ni) & ~1;
      for (int i = tid; i < be / 2; i += blockDim.x) {
        const int e0 = mid[2 * i], e1 = mid[2 * i + 1];
        Iw[c + i] = node_w(e0, m, sk, Iw) + node_w(e1, m, sk, Iw);
        parent[e0] = (unsigned short)(m + c + i);
        parent[e1] = (unsigned short)(m + c + i);
      }
      __syncthreads();
      if (tid == 0) {
        // picks 0 .. be-1 hold every leaf of the batch except an odd last one
        const int nleaf = nl - ((nl + ni) > be && mid[be] < m ? 1 : 0);
        sa = a + nleaf;
        sb = b + (be - nleaf);
        sc = c + be / 2;
      }
      __syncthreads();
    }
    // depths by pointer jumping from the root (node 2m-2)
    const int N = 2 * m - 1, root = 2 * m - 2;
    if (tid == 0) parent[root] = (unsigned short)root;
    __syncthreads();
    for (int v = tid; v < N; v += blockDim.x) dep0[v] = v == root ? 0 : 1;
    __syncthreads();
    unsigned short *ac = parent, *an = anc1, *dc = dep0, *dn = dep1;
    for (int span = 1; span < N; span <<= 1) {
      for (int v = tid; v < N; v += blockDim.x) {
        const unsigned short p = ac[v];
        dn[v] = (unsigned short)(dc[v] + dc[p]);
        an[v] = ac[p];
      }
      __syncthreads();
      unsigned short *t = ac; ac = an; an = t;
      t = dc; dc = dn; dn = t;
    }
    for (int v = tid; v < m; v += blockDim.x) atomicMax(&maxlen, (int)dc[v]);
    __syncthreads();
    if (maxlen <= lmax) {
      for (int v = tid; v < m; v += blockDim.x) lens[sk[v] & 0xFFFF] = (unsigned char)dc[v];
      __syncthreads();
      break;
    }
    for (int s = tid; s < nsym; s += blockDim.x)
      if (cnt[s]) cnt[s] = max(1u, cnt[s] >> 1);
    __syncthreads();
  }
  __syncthreads();
  canonical_tables(lens, nsym, &ct);
  canonical_ranks(lens, nsym, rank, wcount);
  for (int s = tid; s < nsym; s += blockDim.x) {
    const int L = lens[s];
    A.len[s] = (unsigned char)L;
    if (A.stream_lens && s < nstream) A.stream_lens[s] = (unsigned char)L;
    A.code[s] = L ? ct.first[L] + rank[s] : 0u;
  }
}

// ---------------------------------------------------------------------------
// k_choose: the auto predictor's choice per field, from the exact encoded
// size of both sides: code bits (count x length), 32 bits per escape, the raw
// values and, for the learned side, the model; a tie keeps the plain side.
// Writes the chosen code lengths into the stream.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_choose(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const int fi = blockIdx.x;
  if (A.mode[fi] != MCC_PRED_AUTO) return;
  const Ctx c = ctx_of(A, fi);
  Status *st = c.st;
  __shared__ unsigned long long part[2][8];
  __shared__ unsigned int pick;
  if (block_failed(st)) return;
  unsigned char *ws = A.ws0 + (int64_t)fi * A.wss;
  const unsigned int *h0 = c.hist2, *h1 = (const unsigned int *)(ws + A.W.hist2b);
  const unsigned char *l0 = c.len2, *l1 = ws + A.W.len2b;
  const int nsym = A.nsym2;
  unsigned long long b0 = 0, b1 = 0;
  for (int s = threadIdx.x; s < nsym; s += blockDim.x) {
    b0 += (unsigned long long)h0[s] * l0[s];
    b1 += (unsigned long long)h1[s] * l1[s];
  }
  for (int o = 16; o; o >>= 1) {
    b0 += __shfl_xor_sync(0xffffffffu, b0, o);
    b1 += __shfl_xor_sync(0xffffffffu, b1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    part[0][threadIdx.x >> 5] = b0;
    part[1][threadIdx.x >> 5] = b1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long z = 0, l = 0;
    for (int w = 0; w < 8; w++) { z += part[0][w]; l += part[1][w]; }
    const unsigned long long vbits = A.dtype == MCC_F64 ? 64 : 32;
    const int raw = 2 * A.R2 - 1;  // the raw-value symbol
    z += 32ull * h0[0] + vbits * h0[raw];
    l += 32ull * h1[0] + vbits * h1[raw] + 8ull * kModelBytes;
    pick = l < z ? 1u : 0u;
    st->pick = pick;
  }
  __syncthreads();
  const unsigned char *ls = pick ? l1 : l0;
  for (int s = threadIdx.x; s < 2 * A.R2; s += blockDim.x) c.out[A.F.lens2 + s] = ls[s];
}

size_t codebook_smem(int nsym) {
  size_t npn = 1;
  while (npn < (size_t)nsym) npn <<= 1;
  return 4 * (size_t)nsym + 8 * (size_t)nsym + 8 * npn + 8 * (size_t)nsym +
         3 * 4 * (size_t)nsym + 2 * (size_t)nsym + (size_t)nsym + 16;
}

// ---------------------------------------------------------------------------
// k_group_len: one CTA per group of 32 lane chunks. Warp w covers steps
// [w C / 8, (w+1) C / 8) of every lane; per (part, lane) bit sums and per part
// escape / raw counts go to the workspace (k_pack uses them as offsets), lane
// totals to the stream's lane table, group totals to gw / ge / gr.
// ---------------------------------------------------------------------------
constexpr int kParts = 8;

// ---------------------------------------------------------------------------
// Zero-run stage. A run of r zero symbols is coded as the digits d_i in
// {1, 2} of r = sum d_i 2^i (bijective base 2), least significant first.
// These digits are the bits of r + 1 below its leading one, each plus one
// (r + 1 = 2^n + sum (d_i - 1) 2^i), so a run has n = floor(log2(r + 1))
// digits, popc(r + 1) - 1 of them 2s.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int run_bits(unsigned int r, unsigned int l1, unsigned int l2) {
  if (!r) return 0;
  const unsigned int v = r + 1, nd = 31 - __clz(v), n2 = __popc(v) - 1;
  return (nd - n2) * l1 + n2 * l2;
}

// ---------------------------------------------------------------------------
// k_runs (zero-run stage): one CTA per group of 32 lane chunks, warp w over
// steps [w C / 8, (w+1) C / 8) of every lane as in k_group_len. Each (part,
// lane) finds the zero symbols before its first other symbol and after its
// last one, and counts the digits of the runs between; warp 0 then chains the
// parts of each lane: the run that ends at the first other symbol of part w
// began in an earlier part when the parts between hold zeros only. These runs
// go to rs[group][kParts + 1][32] (entry w: the run ending in part w, entry
// kParts: the run ending the lane), and every digit to the component's
// histogram (tokens 2R, 2R + 1). Blocks past the groups of both components
// take the learned side of an auto field.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_runs(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const int fi = blockIdx.y;
  const int64_t ng = A.ng1 + A.ng2;
  const int64_t bx = (int64_t)blockIdx.x + A.bx0;
  const bool side_b = bx >= ng;
  if (!A.zr[fi] || (side_b && A.mode[fi] != MCC_PRED_AUTO)) return;  // uniform per block
  const Ctx c = ctx_of(A, fi);
  if (block_failed(c.st)) return;
  unsigned char *ws = A.ws0 + (int64_t)fi * A.wss;
  const int64_t gi = side_b ? bx - A.ng2 : bx;  // side b: ng1 + g
  const bool c1 = gi < A.ng1;
  const int64_t g = c1 ? gi : gi - A.ng1;
  const int C = c1 ? A.C1 : A.C2, R = c1 ? A.R1 : A.R2;
  const int64_t n = c1 ? A.pv.n_g : A.pv.n_v;
  const unsigned short *sym =
      c1 ? c.sym1 : (side_b ? (const unsigned short *)(ws + A.W.sym2b) : c.sym2);
  unsigned int *hist = c1 ? c.hist1 : (side_b ? (unsigned int *)(ws + A.W.hist2b) : c.hist2);
  unsigned short *rs = (unsigned short *)(ws + (side_b ? A.W.rsb : A.W.rs)) +
                       gi * (kParts + 1) * 32;
  __shared__ unsigned short lead[kParts][32], trail[kParts][32];
  __shared__ unsigned char seen_s[kParts][32];
  __shared__ unsigned int dig[2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x < 2) dig[threadIdx.x] = 0;
  const int k0 = (w * C) / kParts, k1 = ((w + 1) * C) / kParts;
  const int64_t base = g * 32 * (int64_t)C + lane;
  unsigned int run = 0, first = 0, n1 = 0, n2 = 0;
  bool seen = false;
#pragma unroll 4
  for (int k = k0; k < k1; k++) {
    const int64_t p = base + 32 * (int64_t)k;
    if (p < n) {
      if (__ldg(sym + p) == R) {
        run++;
      } else {
        if (!seen) {
          first = run;
          seen = true;
        } else if (run) {
          const unsigned int v = run + 1, nd = 31 - __clz(v), b2 = __popc(v) - 1;
          n1 += nd - b2;
          n2 += b2;
        }
        run = 0;
      }
    }
  }
  lead[w][lane] = (unsigned short)(seen ? first : run);  // a part of zeros only: all of them
  trail[w][lane] = (unsigned short)(seen ? run : 0);
  seen_s[w][lane] = seen ? 1 : 0;
  __syncthreads();
  if (w == 0) {
    unsigned int carry = 0;
#pragma unroll
    for (int q = 0; q < kParts; q++) {
      unsigned int r = 0;
      if (seen_s[q][lane]) {
        r = carry + lead[q][lane];
        carry = trail[q][lane];
      } else {
        carry += lead[q][lane];
      }
      rs[q * 32 + lane] = (unsigned short)r;
      if (r) {
        const unsigned int v = r + 1, nd = 31 - __clz(v), b2 = __popc(v) - 1;
        n1 += nd - b2;
        n2 += b2;
      }
    }
    rs[kParts * 32 + lane] = (unsigned short)carry;
    if (carry) {
      const unsigned int v = carry + 1, nd = 31 - __clz(v), b2 = __popc(v) - 1;
      n1 += nd - b2;
      n2 += b2;
    }
  }
  for (int o = 16; o; o >>= 1) {
    n1 += __shfl_xor_sync(0xffffffffu, n1, o);
    n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  }
  if (lane == 0 && (n1 | n2)) {
    atomicAdd(&dig[0], n1);
    atomicAdd(&dig[1], n2);
  }
  __syncthreads();
  if (threadIdx.x < 2 && dig[threadIdx.x]) atomicAdd(hist + 2 * R + threadIdx.x, dig[threadIdx.x]);
}

struct GroupArgs {
  const unsigned short *sym1, *sym2;
  const unsigned char *len1, *len2;
  int64_t n1, n2, ng1, ng2;
  int C1, C2, nsym1, nsym2;
  unsigned char *ltab1, *ltab2;   // in the output stream
  unsigned int *gw, *ge, *gr;     // workspace [ng1 + ng2]
  unsigned short *pb;             // workspace [ng1 + ng2][kParts][32]
  unsigned int *pe, *pr;          // workspace [ng1 + ng2][kParts]
};

__device__ void scan_field(const CompArgs &A, int fi);

__global__ void __launch_bounds__(256) k_group_len(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.y, true);
  const Status *st = c.st;
  const GroupArgs a{c.sym1, c.sym2, c.len1, c.len2, A.pv.n_g, A.pv.n_v, A.ng1, A.ng2, A.C1, A.C2,
                    A.nsym1, A.nsym2, c.out + A.F.ltab1, c.out + A.F.ltab2, c.gw, c.ge, c.gr,
                    c.pb, c.pe, c.pr};
  __shared__ unsigned char L[2 * kMaxR];
  __shared__ unsigned int sbits[kParts][32];
  __shared__ unsigned int sesc[kParts], sraw[kParts];
  if (block_failed(st)) return;
  const int64_t gi = (int64_t)blockIdx.x + A.bx0;
  const bool c1 = gi < a.ng1;
  const int64_t g = c1 ? gi : gi - a.ng1;
  const int C = c1 ? a.C1 : a.C2;
  const int64_t n = c1 ? a.n1 : a.n2;
  const unsigned short *sym = c1 ? a.sym1 : a.sym2;
  const int nsym = c1 ? a.nsym1 : a.nsym2;
  const unsigned char *lsrc = c1 ? a.len1 : a.len2;
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) L[i] = lsrc[i];
  __syncthreads();
  const int R = c1 ? A.R1 : A.R2;
  const int rawsym = c1 ? kRawNone : 2 * A.R2 - 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k0 = (w * C) / kParts, k1 = ((w + 1) * C) / kParts;
  const int64_t base = g * 32 * (int64_t)C + lane;
  unsigned int bits = 0, esc = 0, raw = 0;
  if (!A.zr[blockIdx.y]) {
#pragma unroll 4
    for (int k = k0; k < k1; k++) {
      const int64_t p = base + 32 * (int64_t)k;
      if (p < n) {
        const int sy = __ldg(sym + p);
        bits += L[sy];
        esc += sy == 0;
        raw += sy == rawsym;
      }
    }
  } else {
    // zero-run stage: a run is costed where it ends, the runs that reach
    // back into earlier parts (and the lane's last run) from k_runs
    const unsigned int l1 = L[2 * R], l2 = L[2 * R + 1];
    unsigned int run = 0;
    bool seen = false;
#pragma unroll 4
    for (int k = k0; k < k1; k++) {
      const int64_t p = base + 32 * (int64_t)k;
      if (p < n) {
        const int sy = __ldg(sym + p);
        if (sy == R) {
          run++;
        } else {
          if (seen) bits += run_bits(run, l1, l2);
          seen = true;
          run = 0;
          bits += L[sy];
          esc += sy == 0;
          raw += sy == rawsym;
        }
      }
    }
    const unsigned short *rs = c.rs + gi * (kParts + 1) * 32;
    bits += run_bits(rs[w * 32 + lane], l1, l2);
    if (w == kParts - 1) bits += run_bits(rs[kParts * 32 + lane], l1, l2);
  }
  a.pb[(gi * kParts + w) * 32 + lane] = (unsigned short)bits;
  sbits[w][lane] = bits;
  for (int o = 16; o; o >>= 1) {
    esc += __shfl_xor_sync(0xffffffffu, esc, o);
    raw += __shfl_xor_sync(0xffffffffu, raw, o);
  }
  if (lane == 0) {
    sesc[w] = esc;
    sraw[w] = raw;
    a.pe[gi * kParts + w] = esc;
    a.pr[gi * kParts + w] = raw;
  }
  __syncthreads();
  if (w == 0) {
    unsigned int tot = 0;
#pragma unroll
    for (int q = 0; q < kParts; q++) tot += sbits[q][lane];
    // lane table: base and one-byte deltas; lanes shorter than base are
    // padded (their padding closes their last part)
    unsigned int mn = tot, mx = tot;
    for (int o = 16; o; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const unsigned int base = mx > 255u && mx - 255u > mn ? mx - 255u : mn;
    const unsigned int padded = tot < base ? base : tot;
    unsigned char *lt = (c1 ? a.ltab1 : a.ltab2) + (int64_t)g * kLtabBytes;
    if (lane == 0) { lt[0] = (unsigned char)(base & 0xFF); lt[1] = (unsigned char)(base >> 8); }
    lt[2 + lane] = (unsigned char)(padded - base);
    if (padded != tot)
      a.pb[(gi * kParts + kParts - 1) * 32 + lane] = (unsigned short)(sbits[kParts - 1][lane] + padded - tot);
    tot = padded;
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) {
      unsigned int e = 0, r = 0;
      for (int q = 0; q < kParts; q++) { e += sesc[q]; r += sraw[q]; }
      a.gw[gi] = (tot + 31) / 32;
      a.ge[gi] = e;
      a.gr[gi] = r;
    }
  }
  // the last block of the field to finish scans the group totals and writes
  // the layout and header (the former k_scan)
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0)
    last = atomicAdd(&c.st->groups_done, 1u) == (unsigned int)(a.ng1 + a.ng2) - 1u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  scan_field(A, blockIdx.y);
}

// ---------------------------------------------------------------------------
// k_scan: exclusive prefixes over groups, layout and header (one CTA)
// ---------------------------------------------------------------------------
// Exclusive prefix of n u32 values by one warp (out[0..n], out[n] = total);
// every lane owns 8 consecutive values of each 256-value chunk.
__device__ unsigned long long warp_exclusive_scan(const unsigned int *in, int64_t n,
                                                  unsigned int *out) {
  const int lane = threadIdx.x & 31;
  unsigned long long carry = 0;
  for (int64_t base = 0; base < n; base += 256) {
    unsigned int v[8];
    const int64_t i0 = base + 8 * lane;
#pragma unroll
    for (int j = 0; j < 8; j++) v[j] = i0 + j < n ? __ldcg(in + i0 + j) : 0u;  // other blocks' writes
    unsigned int tot = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) tot += v[j];
    unsigned int incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    unsigned int run = (unsigned int)carry + incl - tot;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (i0 + j < n) out[i0 + j] = run;
      run += v[j];
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) out[n] = (unsigned int)carry;
  return carry;
}

struct ScanArgs {
  const unsigned int *gw, *ge, *gr;
  int64_t ng1, ng2;
  unsigned char *out;
  uint64_t capacity;
  Layout fixed;  // fixed-size part (lens .. ltab2)
  int dtype, dim, R1, R2, C1, C2, lmax;
  int nx, ny, nz;
  int64_t n_v, n_g;
};

__device__ __forceinline__ void put32(unsigned char *p, uint32_t v) { *(uint32_t *)p = v; }
__device__ __forceinline__ void put64(unsigned char *p, uint64_t v) { *(uint64_t *)p = v; }

// Layout and header of field fi from the group totals; run by the last
// k_group_len block of the field (every thread of the block calls it).
__device__ void scan_field(const CompArgs &A, int fi) {
  const Ctx c = ctx_of(A, fi);
  Status *st = c.st;
  const ScanArgs a{c.gw, c.ge, c.gr, A.ng1, A.ng2, c.out, A.capacity, A.F, A.dtype, A.pv.dim,
                   A.R1, A.R2, A.C1, A.C2, A.lmax, A.pv.nx, A.pv.ny, A.pv.nz, A.pv.n_v, A.pv.n_g};
  __shared__ unsigned long long tot[5];
  if (block_failed(st)) return;
  const Layout F = a.fixed;
  unsigned char *o = a.out;
  // five independent prefixes, one warp each
  const int w = threadIdx.x >> 5;  // warps 0..4 scan, the others wait
  const unsigned int *src[5] = {a.gw, a.gw + a.ng1, a.ge, a.ge + a.ng1, a.gr + a.ng1};
  const uint64_t dst[5] = {F.gtab1, F.gtab2, F.etab1, F.etab2, F.rtab2};
  const int64_t cnt[5] = {a.ng1, a.ng2, a.ng1, a.ng2, a.ng2};
  if (w < 5) {
    const unsigned long long t = warp_exclusive_scan(src[w], cnt[w], (unsigned int *)(o + dst[w]));
    if ((threadIdx.x & 31) == 0) tot[w] = t;
  }
  __syncthreads();
  const int mode = A.mode[fi];
  const unsigned char *model =
      mode == MCC_PRED_LEARNED || (mode == MCC_PRED_AUTO && st->pick) ? A.model[fi] : nullptr;
  __shared__ unsigned long long model_at;  // stream offset of the model section, 0 = none
  if (threadIdx.x == 0) {
    model_at = 0;
    const unsigned long long w1 = tot[0], w2 = tot[1], e1 = tot[2], e2 = tot[3], r2 = tot[4];
    const uint64_t vsz = a.dtype == MCC_F64 ? 8 : 4;
    const Layout L = make_layout(a.R1, a.R2, a.ng1, a.ng2, e1, e2, r2, vsz, w1, w2,
                                 model ? kModelBytes : 0);
    st->L = L;
    st->w1 = w1;
    st->w2 = w2;
    st->out_size = L.total;
    if (L.total > a.capacity) {
      set_error(st, MCC_ERR_CAPACITY);
    } else {
      const FieldParams &f = st->f;
      for (int i = 0; i < (int)kHeaderBytes; i += 8) put64(o + i, 0);
      // the alignment gaps between sections are zero (no stale bytes of the
      // caller's buffer in the stream, which is then a function of the input)
      const uint64_t gap[5][2] = {{L.lens2 + 2 * (uint64_t)a.R2, L.gtab1},
                                  {L.ltab2 + kLtabBytes * (uint64_t)a.ng2, L.out1},
                                  {L.out2 + 4 * e2, L.raw},
                                  {L.raw + vsz * r2, L.bits1},
                                  {L.bits2 + 4 * w2, L.model}};
#pragma unroll
      for (int k = 0; k < 5; k++)
        for (uint64_t b = gap[k][0]; b < gap[k][1]; b++) o[b] = 0;
      put32(o + H_MAGIC, kMagic);
      put32(o + H_VERSION, kVersion);
      put32(o + H_HBYTES, kHeaderBytes);
      put32(o + H_DTYPE, (uint32_t)a.dtype);
      put32(o + H_DIM, (uint32_t)a.dim);
      const bool open = A.open[fi] != 0;
      const uint32_t zflag = A.zr[fi] ? F_ZRUN : 0u;
      if (A.one_d) put32(o + H_FLAGS, F_ONED | zflag);
      else put32(o + H_FLAGS, (f.guard || open ? F_GUARD : 0u) | (model ? F_MODEL : 0u) |
                             (open ? F_OPEN : 0u) |
                             (A.gop[fi] == MCC_G_NEAREST ? F_GNEAR : 0u) |
                             (A.fop[fi] == MCC_F_CLUSTER ? F_FCLUSTER : 0u) | zflag);
      put32(o + H_R1, (uint32_t)a.R1);
      put32(o + H_R2, (uint32_t)a.R2);
      put32(o + H_C1, (uint32_t)a.C1);
      put32(o + H_C2, (uint32_t)a.C2);
      put32(o + H_LMAX, (uint32_t)a.lmax);
      put32(o + H_NX, (uint32_t)a.nx);
      put32(o + H_NY, (uint32_t)a.ny);
      put32(o + H_NZ, (uint32_t)a.nz);
      put64(o + H_NV, (uint64_t)a.n_v);
      put64(o + H_NG, (uint64_t)a.n_g);
      put64(o + H_TAU, (uint64_t)__double_as_longlong(f.tau));
      put64(o + H_TAU1, (uint64_t)__double_as_longlong(f.tau1));
      put64(o + H_TAU2, (uint64_t)__double_as_longlong(f.tau2));
      put64(o + H_S1, (uint64_t)__double_as_longlong(f.s1));
      put64(o + H_S2, (uint64_t)__double_as_longlong(f.s2));
      put64(o + H_K, (uint64_t)f.K);
      put64(o + H_RHO21, (uint64_t)f.rho21_q);
      put64(o + H_RHO12, (uint64_t)f.rho12_q);
      put64(o + H_FILL, (uint64_t)f.fill_u);
      put64(o + H_NOUT1, e1);
      put64(o + H_NOUT2, e2);
      put64(o + H_NRAW, r2);
      put64(o + H_W1, w1);
      put64(o + H_W2, w2);
      put64(o + H_TOTAL, L.total);
      put64(o + H_MODEL, model ? kModelBytes : 0);
      put64(o + H_QHI, (uint64_t)f.Qhi);
      if (zflag) {  // the run tokens' code lengths (of the chosen residual side)
        const Ctx cc = ctx_of(A, fi, true);
        o[H_RUNLEN] = cc.len1[2 * a.R1];
        o[H_RUNLEN + 1] = cc.len1[2 * a.R1 + 1];
        if (!A.one_d) {
          o[H_RUNLEN + 2] = cc.len2[2 * a.R2];
          o[H_RUNLEN + 3] = cc.len2[2 * a.R2 + 1];
        }
      }
      // zero the alignment padding between sections
      for (uint64_t p = F.lens2 + 2 * (uint64_t)a.R2; p < F.gtab1; p++) o[p] = 0;
      for (uint64_t p = L.out2 + 4 * e2; p < L.raw; p++) o[p] = 0;
      for (uint64_t p = L.raw + vsz * r2; p < L.bits1; p++) o[p] = 0;
      for (uint64_t p = L.bits2 + 4 * w2; p < L.model; p++) o[p] = 0;
      if (model) model_at = L.model;
    }
  }
  __syncthreads();
  if (model_at) {  // the blob travels with the stream
    const unsigned int *src = (const unsigned int *)model;
    unsigned int *dst = (unsigned int *)(o + model_at);
    for (int i = threadIdx.x; i < (int)kModelBytes / 4; i += blockDim.x) dst[i] = src[i];
  }
}

// ---------------------------------------------------------------------------
// k_pack: one CTA per group; every (part, lane) writes its codes MSB-first at
// its bit offset into a shared-memory copy of the group's words, escape and
// raw values go to their index-ordered slots, then the words are copied out.
// ---------------------------------------------------------------------------
struct PackArgs {
  const unsigned short *sym1, *sym2;
  const unsigned int *code1, *code2;
  const unsigned char *len1, *len2;
  const int *val1, *val2;
  const void *x;
  int64_t n1, n2, ng1, ng2;
  int C1, C2, nsym1, nsym2, vsz;
  unsigned char *out;
  const unsigned short *pb;
  const unsigned int *pe, *pr;
};

// ZR: the batch has a field with the zero-run stage (a separate variant keeps
// the plain one's register count)
template <bool ZR>
__global__ void __launch_bounds__(256, ZR ? 5 : 6) k_pack(const __grid_constant__ CompArgs A) {
  pdl_wait();
  const Ctx c = ctx_of(A, blockIdx.y, true);
  const Status *st = c.st;
  const PackArgs a{c.sym1, c.sym2, c.code1, c.code2, c.len1, c.len2, c.val1, c.val2, c.x,
                   A.pv.n_g, A.pv.n_v, A.ng1, A.ng2, A.C1, A.C2, A.nsym1, A.nsym2,
                   A.dtype == MCC_F64 ? 8 : 4, c.out, c.pb, c.pe, c.pr};
  extern __shared__ unsigned int stage[];
  __shared__ unsigned int scl[2 * kMaxR];  // code << 5 | length (codes < 2^24, lengths <= 24)
  if (block_failed(st)) return;
  const Layout L = st->L;
  const int64_t gi = blockIdx.x;
  const bool c1 = gi < a.ng1;
  const int64_t g = c1 ? gi : gi - a.ng1;
  const int C = c1 ? a.C1 : a.C2;
  const int64_t n = c1 ? a.n1 : a.n2;
  const int nsym = c1 ? a.nsym1 : a.nsym2;
  const unsigned short *sym = c1 ? a.sym1 : a.sym2;
  const unsigned int *csrc = c1 ? a.code1 : a.code2;
  const unsigned char *lsrc = c1 ? a.len1 : a.len2;
  const int *val = c1 ? a.val1 : a.val2;
  const int R = c1 ? A.R1 : A.R2;
  const int rawsym = c1 ? kRawNone : 2 * A.R2 - 1;
  const bool zr = ZR && A.zr[blockIdx.y] != 0;
  unsigned char *o = a.out;
  const unsigned int *gtab = (const unsigned int *)(o + (c1 ? L.gtab1 : L.gtab2));
  const unsigned int *etab = (const unsigned int *)(o + (c1 ? L.etab1 : L.etab2));
  const unsigned int *rtab = (const unsigned int *)(o + L.rtab2);
  const unsigned char *ltg = o + (c1 ? L.ltab1 : L.ltab2) + (int64_t)g * kLtabBytes;
  int *outv = (int *)(o + (c1 ? L.out1 : L.out2));
  unsigned int *bits = (unsigned int *)(o + (c1 ? L.bits1 : L.bits2));

  const unsigned int w0 = gtab[g], nw = gtab[g + 1] - w0;
  for (unsigned int i = threadIdx.x; i < nw; i += blockDim.x) stage[i] = 0;
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) scl[i] = (csrc[i] << 5) | lsrc[i];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // bit offset of (part w, lane): lanes before this one, then earlier parts
  const unsigned int lb = ((unsigned int)ltg[0] | ((unsigned int)ltg[1] << 8)) + ltg[2 + lane];
  unsigned int incl = lb;
  for (int sft = 1; sft < 32; sft <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, sft);
    if (lane >= sft) incl += t;
  }
  unsigned int pos = incl - lb;
  unsigned int e_run = etab[g], r_run = c1 ? 0u : rtab[g];
  // groups without escapes / raw values (most) skip their ballots
  const bool any_esc = etab[g + 1] != e_run;
  const bool any_raw = !c1 && rtab[g + 1] != r_run;
  {  // the earlier parts' totals, their loads issued together
    unsigned int pb[kParts - 1], pe[kParts - 1], pr[kParts - 1];
#pragma unroll
    for (int q = 0; q < kParts - 1; q++) {
      const bool before = q < w;
      pb[q] = before ? a.pb[(gi * kParts + q) * 32 + lane] : 0u;
      pe[q] = before ? a.pe[gi * kParts + q] : 0u;
      pr[q] = before ? a.pr[gi * kParts + q] : 0u;
    }
#pragma unroll
    for (int q = 0; q < kParts - 1; q++) {
      pos += pb[q];
      e_run += pe[q];
      r_run += pr[q];
    }
  }
  // zero-run stage: the runs that end at this part's first other symbol and
  // at the lane's end (from k_runs)
  unsigned int rs_first = 0, rs_end = 0;
  if (zr) {
    const unsigned short *rs = c.rs + gi * (kParts + 1) * 32;
    rs_first = rs[w * 32 + lane];
    rs_end = rs[kParts * 32 + lane];
  }
  __syncthreads();
  const int k0 = (w * C) / kParts, k1 = ((w + 1) * C) / kParts;
  const int64_t base = g * 32 * (int64_t)C + lane;
  const unsigned lt = (1u << lane) - 1;
  // a code of cl >= 1 bits at the lane's bit position
  auto put = [&](unsigned int packed) {
    const unsigned int code = packed >> 5, cl = packed & 31u;
    const unsigned long long v = ((unsigned long long)code << (64 - cl)) >> (pos & 31);
    atomicOr(stage + (pos >> 5), (unsigned int)(v >> 32));
    if ((pos & 31) + cl > 32) atomicOr(stage + (pos >> 5) + 1, (unsigned int)v);
    pos += cl;
  };
  // zero-run stage: the digits of a run, least significant first (bit i of
  // r + 1 below its leading one selects token 2R + bit)
  auto put_run = [&](unsigned int r) {
    if (!r) return;
    const unsigned int v = r + 1, nd = 31 - __clz(v);
    for (unsigned int i = 0; i < nd; i++) {
      const int t = 2 * R + (int)((v >> i) & 1u);
      put(scl[t]);
    }
  };
  unsigned int run = 0;
  bool seen = false;
#pragma unroll 4
  for (int k = k0; k < k1; k++) {
    const int64_t p = base + 32 * (int64_t)k;
    const bool valid = p < n;
    const int sy = valid ? (int)__ldg(sym + p) : -1;
    if (valid) {
      if (zr && sy == R) {
        run++;
      } else {
        if (zr) {  // the run that ends here (the first one may reach back)
          put_run(seen ? run : rs_first);
          seen = true;
          run = 0;
        }
        put(scl[sy]);
      }
    }
    if (any_esc) {
      const unsigned em = __ballot_sync(0xffffffffu, sy == 0);
      if (sy == 0) outv[e_run + __popc(em & lt)] = __ldg(val + p);
      e_run += __popc(em);
    }
    if (any_raw) {
      const unsigned rm = __ballot_sync(0xffffffffu, sy == rawsym);
      if (sy == rawsym) {
        unsigned char *dst = o + L.raw + (uint64_t)a.vsz * (r_run + __popc(rm & lt));
        if (a.vsz == 8) *(unsigned long long *)dst = ((const unsigned long long *)a.x)[p];
        else *(unsigned int *)dst = ((const unsigned int *)a.x)[p];
      }
      r_run += __popc(rm);
    }
  }
  if (zr && w == kParts - 1) put_run(rs_end);  // the lane's last run
  __syncthreads();
  for (unsigned int i = threadIdx.x; i < nw; i += blockDim.x) bits[w0 + i] = stage[i];
}

inline unsigned int nblk(int64_t n, int bs) {
  const int64_t b = (n + bs - 1) / bs;
  return (unsigned int)(b < 1 ? 1 : b);
}

int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
mcc_status check_params(const mcc_params *p) {
  if (!p) return MCC_ERR_INVALID_ARG;
  if (p->dtype != MCC_F64 && p->dtype != MCC_F32) return MCC_ERR_INVALID_ARG;
  if (p->eb_mode != MCC_ABS && p->eb_mode != MCC_REL) return MCC_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !std::isfinite(p->eb)) return MCC_ERR_INVALID_ARG;
  if (!(p->grid_fraction >= 1e-3 && p->grid_fraction <= 1.0 - 1e-3)) return MCC_ERR_INVALID_ARG;
  if (p->R1 < 4 || p->R1 > kMaxR || p->R2 < 4 || p->R2 > kMaxR) return MCC_ERR_UNSUPPORTED;
  if (p->C1 < 1 || p->C1 > kMaxC || p->C2 < 1 || p->C2 > kMaxC) return MCC_ERR_UNSUPPORTED;
  if (p->lmax < 1 || p->lmax > kMaxLen) return MCC_ERR_UNSUPPORTED;
  // every symbol of an alphabet must fit in lmax bits (this also bounds the
  // code book's count halving: all counts 1 give a tree of depth log2(2R))
  if (2 * p->R1 > (1 << p->lmax) || 2 * p->R2 > (1 << p->lmax)) return MCC_ERR_INVALID_ARG;
  if (p->predictor != MCC_PRED_ZERO && p->predictor != MCC_PRED_LEARNED &&
      p->predictor != MCC_PRED_AUTO)
    return MCC_ERR_INVALID_ARG;
  if (p->predictor != MCC_PRED_ZERO && (!p->d_model || ((uintptr_t)p->d_model & 3)))
    return MCC_ERR_INVALID_ARG;
  if (p->loop != MCC_LOOP_CLOSED && p->loop != MCC_LOOP_OPEN) return MCC_ERR_INVALID_ARG;
  if (p->loop == MCC_LOOP_OPEN && p->predictor != MCC_PRED_ZERO) return MCC_ERR_INVALID_ARG;
  if (p->f_op != MCC_F_BARYCENTRIC && p->f_op != MCC_F_CLUSTER) return MCC_ERR_INVALID_ARG;
  if (p->g_op != MCC_G_MULTILINEAR && p->g_op != MCC_G_NEAREST) return MCC_ERR_INVALID_ARG;
  if (p->g_op == MCC_G_NEAREST && p->predictor != MCC_PRED_ZERO) return MCC_ERR_INVALID_ARG;
  if (p->zero_run != 0 && p->zero_run != 1) return MCC_ERR_INVALID_ARG;
  if (p->zero_run) {  // 2R + 2 tokens: the decode tables hold 2 kMaxR symbols
    if (p->R1 > kMaxR - 1 || p->R2 > kMaxR - 1) return MCC_ERR_UNSUPPORTED;
    if (2 * p->R1 + kRunTokens > (1 << p->lmax) || 2 * p->R2 + kRunTokens > (1 << p->lmax))
      return MCC_ERR_INVALID_ARG;
  }
  return MCC_OK;
}

CompressWs compress_ws_layout(const PlanView &pv, const mcc_params *p) {
  CompressWs w;
  size_t o = kStatusBytes;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  const int64_t ng1 = ngroups(pv.n_g, p->C1), ng2 = ngroups(pv.n_v, p->C2);
  // code books: 2R symbols and the zero-run stage's run tokens
  const size_t ns1 = 2 * (size_t)p->R1 + kRunTokens, ns2 = 2 * (size_t)p->R2 + kRunTokens;
  w.hist1 = take(4 * ns1);
  w.hist2 = take(4 * ns2);
  w.code1 = take(4 * ns1);
  w.code2 = take(4 * ns2);
  w.len1 = take(ns1);
  w.len2 = take(ns2);
  w.Q = take(4 * (size_t)pv.n_v);
  w.q1 = take(4 * (size_t)pv.n_g + 16);  // + 16: the corner gathers' aligned 16-byte loads
  w.sym1 = take(2 * (size_t)pv.n_g);
  w.sym2 = take(2 * (size_t)pv.n_v);
  w.val1 = take(4 * (size_t)pv.n_g);
  w.val2 = take(4 * (size_t)pv.n_v);
  w.gw = take(4 * (size_t)(ng1 + ng2));
  w.ge = take(4 * (size_t)(ng1 + ng2));
  w.gr = take(4 * (size_t)(ng1 + ng2));
  w.pb = take(2 * kParts * 32 * (size_t)(ng1 + ng2));
  w.pe = take(4 * kParts * (size_t)(ng1 + ng2));
  w.pr = take(4 * kParts * (size_t)(ng1 + ng2));
  w.p = take(4 * (size_t)pv.n_v);
  w.hist2b = take(4 * ns2);
  w.code2b = take(4 * ns2);
  w.len2b = take(ns2);
  w.sym2b = take(2 * (size_t)pv.n_v);
  w.val2b = take(4 * (size_t)pv.n_v);
  w.x1v = take(8 * (size_t)pv.n_g);
  w.rs = take(2 * (kParts + 1) * 32 * (size_t)(ng1 + ng2));
  w.rsb = take(2 * (kParts + 1) * 32 * (size_t)(ng1 + ng2));
  w.csum = take(8 * (size_t)pv.n_g);
  w.ccnt = take(4 * (size_t)pv.n_g);
  w.total = o;
  return w;
}

// Compress nf fields (nf <= kMaxBatch) of one plan: field f reads xs[f] with
// bound parameters ps[f] (dtype, R, C and lmax taken from ps[0]), uses the
// workspace region ws0 + f * wss and writes its stream to out0 + f * oss
// (at most `capacity` bytes).
mcc_status launch_compress_batch(const PlanView &pv, int nf, const void *const *xs,
                                 const mcc_params *ps, unsigned char *ws0, int64_t wss,
                                 unsigned char *out0, int64_t oss, size_t capacity,
                                 cudaStream_t stream, bool front_only) {
  if (nf < 1 || nf > kMaxBatch) return MCC_ERR_INVALID_ARG;
  const mcc_params *p = ps;
  CompArgs A;  // launch arguments (passed by value as a grid constant)
  memset(&A, 0, sizeof(A));
  A.pv = pv;
  A.W = compress_ws_layout(pv, p);
  A.ws0 = ws0;
  A.out0 = out0;
  A.wss = wss;
  A.oss = oss;
  A.capacity = capacity;
  A.nf = nf;
  A.dtype = p->dtype;
  A.R1 = p->R1;
  A.R2 = p->R2;
  A.C1 = p->C1;
  A.C2 = p->C2;
  A.lmax = p->lmax;
  for (int f = 0; f < nf; f++) {
    A.zr[f] = ps[f].zero_run ? 1 : 0;
    A.any_zr = A.any_zr || A.zr[f];
  }
  // code books over the 2R symbols, plus the run tokens when a field of the
  // batch takes the zero-run stage
  A.nsym1 = 2 * p->R1 + (A.any_zr ? kRunTokens : 0);
  A.nsym2 = 2 * p->R2 + (A.any_zr ? kRunTokens : 0);
  A.one_d = pv.dim == 1;  // the 1D coder: no residual component
  A.ng1 = ngroups(pv.n_g, p->C1);
  A.ng2 = A.one_d ? 0 : ngroups(pv.n_v, p->C2);
  A.F = make_layout(p->R1, p->R2, A.ng1, A.ng2, 0, 0, 0, 8, 0, 0);
  if (!front_only && capacity < A.F.out1) return MCC_ERR_CAPACITY;
  bool any_model = false, any_open = false, any_cluster = false;
  for (int f = 0; f < nf; f++) {
    A.open[f] = ps[f].loop == MCC_LOOP_OPEN ? 1 : 0;
    A.fop[f] = (unsigned char)ps[f].f_op;
    A.gop[f] = (unsigned char)ps[f].g_op;
    // the open-loop and nearest-node paths share the kernel variant with the
    // runtime branches
    any_open = any_open || A.open[f] || ps[f].g_op == MCC_G_NEAREST;
    any_cluster = any_cluster || ps[f].f_op == MCC_F_CLUSTER;
    A.x[f] = xs[f];
    A.rp[f] = RParams{ps[f].dtype, ps[f].eb_mode, ps[f].eb, ps[f].grid_fraction, A.one_d};
    A.mode[f] = (unsigned char)ps[f].predictor;
    A.model[f] = ps[f].predictor != MCC_PRED_ZERO ? (const unsigned char *)ps[f].d_model : nullptr;
    any_model = any_model || A.model[f];
    A.any_auto = A.any_auto || ps[f].predictor == MCC_PRED_AUTO;
  }
  const int64_t ng = A.ng1 + A.ng2;
  const int sms = num_sms();
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_pack<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_pack<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  if (cudaMemset2DAsync(ws0, (size_t)wss, 0, kStatusBytes, (size_t)nf, stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  if (any_cluster &&  // cluster sums and sizes (contiguous, one region per field)
      cudaMemset2DAsync(ws0 + A.W.csum, (size_t)wss, 0, A.W.total - A.W.csum, (size_t)nf,
                        stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  const unsigned int bpf = (unsigned int)((sms * 4 + nf - 1) / nf);  // reduce blocks per field
  // blocks per field of the grid-stride kernels: the plan's tuning, or one
  // full wave of resident blocks (0, the default)
  const int vbps = pv.vbps;
  const unsigned int ppf = (unsigned int)((sms * 8 + nf - 1) / nf);  // the 1D coder's
  {
    PROF_SCOPE("k_reduce", stream);
    if (p->dtype == MCC_F64) k_reduce<double><<<dim3(bpf, nf), 256, 0, stream>>>(A);
    else k_reduce<float><<<dim3(bpf, nf), 256, 0, stream>>>(A);
  }
  {
    PROF_SCOPE("k_prequant", stream);
    if (p->dtype == MCC_F64)
      launch_pdl(k_prequant<double>, dim3(wave_blocks(k_prequant<double>, 256, 0, vbps, sms, nf), nf),
                 dim3(256), 0, stream, A);
    else
      launch_pdl(k_prequant<float>, dim3(wave_blocks(k_prequant<float>, 256, 0, vbps, sms, nf), nf),
                 dim3(256), 0, stream, A);
  }
  const size_t hsm1 = 4 * (size_t)A.nsym1, hsm2 = 4 * (size_t)A.nsym2 * (A.any_auto ? 2 : 1);
  if (A.one_d) {
    PROF_SCOPE("k_delta1d", stream);
    launch_pdl(k_delta1d, dim3(ppf, nf), dim3(256), hsm1, stream, A);
  } else if (pv.dim == 2) {
    PROF_SCOPE("k_grid2d", stream);
    // the plan's tile (tuning): 64 x 16 by default, 32 x 32 or 128 x 8
    if (pv.tile2d == MCC_TILE_32x32)
      launch_pdl(k_grid2d<32, 32>, dim3(nf, (pv.nx + 31) / 32, (pv.ny + 31) / 32), dim3(256), hsm1,
                 stream, A);
    else if (pv.tile2d == MCC_TILE_128x8)
      launch_pdl(k_grid2d<128, 8>, dim3(nf, (pv.nx + 127) / 128, (pv.ny + 7) / 8), dim3(256), hsm1,
                 stream, A);
    else
      launch_pdl(k_grid2d<64, 16>, dim3(nf, (pv.nx + 63) / 64, (pv.ny + 15) / 16), dim3(256), hsm1,
                 stream, A);
  }
  // Two streams once q1 exists (Algorithm 3 codes x1' and x2 independently):
  // the grid component's coder (in 3D from its Lorenzo differences on: they
  // read q1 only) on the plan's second stream, beside the residual stage on
  // the caller's; they join before the bit packing (whose layout needs both
  // components). Single large fields only: with a batch, or a small field,
  // the grid coder's kernels slow the residual stage they run beside by more
  // than they hide (measured on the 2D graded and batched workloads).
  const bool fork = !front_only && pv.side != nullptr && !A.one_d && nf == 1 &&
                    pv.n_g + pv.n_v >= ((int64_t)1 << 23);
  const unsigned int txy = (unsigned int)(((pv.nx + 31) / 32) * ((pv.ny + 7) / 8));
  if (pv.dim == 3 && !A.one_d) {
    {
      PROF_SCOPE("k_grid_codes", stream);
      launch_pdl(k_grid_codes3d, dim3(nf, wave_blocks(k_grid_codes3d, 256, 0, vbps, sms, nf)),
                 dim3(256), 0, stream, A);
    }
    if (!fork) {
      PROF_SCOPE("k_grid3d", stream);
      launch_pdl(k_grid3d<32, 8, 8>, dim3(nf, txy, (pv.nz + 7) / 8), dim3(256), hsm1, stream, A);
    }
  }
  if (front_only) return cudaGetLastError() == cudaSuccess ? MCC_OK : MCC_ERR_CUDA;
  std::unique_lock<std::mutex> lock;
  const cudaStream_t side = (cudaStream_t)pv.side;
  if (fork) {
    lock = std::unique_lock<std::mutex>(*(std::mutex *)pv.mu);
    if (cudaEventRecord((cudaEvent_t)pv.ev_fork, stream) != cudaSuccess ||
        cudaStreamWaitEvent(side, (cudaEvent_t)pv.ev_fork, 0) != cudaSuccess)
      return MCC_ERR_CUDA;
    CompArgs G = A;
    G.bx0 = 0;
    if (pv.dim == 3) {
      PROF_SCOPE("k_grid3d_grid", side);
      launch_pdl(k_grid3d<32, 8, 8>, dim3(nf, txy, (pv.nz + 7) / 8), dim3(256), hsm1, side, G);
    }
    if (A.any_zr) {
      PROF_SCOPE("k_runs_grid", side);
      launch_pdl(k_runs, dim3((unsigned int)A.ng1, nf), dim3(256), 0, side, G);
    }
    {
      PROF_SCOPE("k_codebook_grid", side);
      const size_t cbsm = codebook_smem(A.nsym1);
      launch_pdl(k_codebook, dim3(1, nf), dim3(1024), cbsm, side, G);
    }
    {
      PROF_SCOPE("k_group_len_grid", side);
      launch_pdl(k_group_len, dim3((unsigned int)A.ng1, nf), dim3(256), 0, side, G);
    }
    if (cudaEventRecord((cudaEvent_t)pv.ev_join, side) != cudaSuccess) return MCC_ERR_CUDA;
  }
  if (!A.one_d && any_model) {  // learned corrections p at every vertex of the fields with a model
    PROF_SCOPE("k_predict", stream);
    PredArgs P;
    memset(&P, 0, sizeof(P));
    P.pv = pv;
    P.nf = nf;
    P.bad_model_err = MCC_ERR_INVALID_ARG;
    for (int f = 0; f < nf; f++) {
      unsigned char *ws = ws0 + (int64_t)f * wss;
      P.q1[f] = (const int *)(ws + A.W.q1);
      P.p[f] = (float *)(ws + A.W.p);
      P.model[f] = A.model[f];
      P.rho12_f[f] = &((const Status *)ws)->f.rho12_f;
      P.qhi[f] = &((const Status *)ws)->f.Qhi;
      P.st[f] = (Status *)ws;
    }
    launch_predict(P, stream, true);
  }
  if (!A.one_d) {
    PROF_SCOPE("k_node", stream);
    // variants: plain, with the learned predictor, with open-loop fields
    // (which also serves learned fields of the same batch). With the fork,
    // one wave less two SMs' worth of blocks: room for the second stream's
    // kernels beside k_node (measured on the 3D field: step 0.870 -> 0.853 ms
    // with 2 SMs' worth left, 0.856 with 4, 0.865 with 16, none: 0.870)
#define MCC_NODE_ONE(K)                                                                 \
  do {                                                                                  \
    unsigned int nb = wave_blocks(K, 256, hsm2, vbps, sms, nf);                         \
    if (fork && vbps == 0 && nb > 4u * (unsigned int)sms) nb -= 2u * (nb / (unsigned int)sms); \
    launch_pdl(K, dim3(nf, nb), dim3(256), hsm2, stream, A);                            \
  } while (0)
#define MCC_NODE(D, T)                                                                  \
  do {                                                                                  \
    if (any_open) MCC_NODE_ONE((k_node<D, T, true, true>));                            \
    else if (any_model) MCC_NODE_ONE((k_node<D, T, true, false>));                     \
    else MCC_NODE_ONE((k_node<D, T, false, false>));                                   \
  } while (0)
    if (pv.dim == 2) {
      if (p->dtype == MCC_F64) MCC_NODE(2, double);
      else MCC_NODE(2, float);
    } else {
      if (p->dtype == MCC_F64) MCC_NODE(3, double);
      else MCC_NODE(3, float);
    }
#undef MCC_NODE
#undef MCC_NODE_ONE
  }
  // the residual component's (or, on one stream, both components') blocks:
  // logical block indices from R.bx0
  CompArgs R = A;
  R.bx0 = fork ? (int)A.ng1 : 0;
  if (A.any_zr) {
    PROF_SCOPE("k_runs", stream);
    const int64_t nb = (fork ? A.ng2 : ng) + (A.any_auto ? A.ng2 : 0);
    launch_pdl(k_runs, dim3((unsigned int)nb, nf), dim3(256), 0, stream, R);
  }
  {
    PROF_SCOPE("k_codebook", stream);
    const size_t cbsm = codebook_smem(A.nsym1 > A.nsym2 ? A.nsym1 : A.nsym2);
    CompArgs Rc = A;
    Rc.bx0 = fork ? 1 : 0;
    const unsigned int nb = (fork ? 1 : 2) + (A.any_auto ? 1 : 0);
    launch_pdl(k_codebook, dim3(nb, nf), dim3(1024), cbsm, stream, Rc);
  }
  if (A.any_auto) {
    PROF_SCOPE("k_choose", stream);
    launch_pdl(k_choose, dim3(nf), dim3(256), 0, stream, A);
  }
  {
    PROF_SCOPE("k_group_len", stream);
    launch_pdl(k_group_len, dim3((unsigned int)(fork ? A.ng2 : ng), nf), dim3(256), 0, stream, R);
  }
  if (fork && cudaStreamWaitEvent(stream, (cudaEvent_t)pv.ev_join, 0) != cudaSuccess)
    return MCC_ERR_CUDA;
  {
    PROF_SCOPE("k_pack", stream);
    const int cmax = p->C1 > p->C2 ? p->C1 : p->C2;
    const size_t stage_bytes = 4 * (size_t)cmax * p->lmax;  // worst-case words of one group
    if (A.any_zr) launch_pdl(k_pack<true>, dim3((unsigned int)ng, nf), dim3(256), stage_bytes, stream, A);
    else launch_pdl(k_pack<false>, dim3((unsigned int)ng, nf), dim3(256), stage_bytes, stream, A);
  }
  if (cudaGetLastError() != cudaSuccess) return MCC_ERR_CUDA;
  return MCC_OK;
}

mcc_status launch_compress(const PlanView &pv, const void *d_values, const mcc_params *p,
                           unsigned char *ws, unsigned char *out, size_t capacity,
                           cudaStream_t stream) {
  const void *xs[1] = {d_values};
  return launch_compress_batch(pv, 1, xs, p, ws, (int64_t)compress_ws_layout(pv, p).total, out,
                               (int64_t)capacity, capacity, stream);
}
