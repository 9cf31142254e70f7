// common.cuh -- internal definitions shared by the library's translation units:
// stream format, per-field parameters, workspace layout and the device
// arithmetic that compression and decompression must evaluate identically.
//
// Floating point: every .cu file is compiled with -fmad=false; the few fused
// multiply-adds of the predictor are written out as __fmaf_rn. FP64 is used
// only where the bound needs it (the vertex code Q = round(x / s2) and the
// reconstruction x' = s2 * Q); interpolation runs in FP32 on integer codes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <utility>

#include "../../include/mcc.h"

namespace mcc {

// ---------------------------------------------------------------------------
// stream format
// ---------------------------------------------------------------------------
constexpr uint32_t kMagic = 0x3143434Du;  // bytes 'M' 'C' 'C' '1'
constexpr uint32_t kVersion = 2;
constexpr uint32_t kHeaderBytes = 384;
constexpr int kRhoBits = 40;               // bin-width ratios in 2^-40 fixed point
constexpr double kBinShrink = 1.0 - 1.0 / 1048576.0;  // bins are 2 tau (1 - 2^-20)
constexpr int kMaxR = 2048;
constexpr int kMaxC = 256;
constexpr int kMaxLen = 24;
constexpr int kMaxBatch = 64;               // fields per kernel launch
constexpr int kLutBits = 12;               // first-level decode table (two symbols per entry)
constexpr uint32_t kModelBytes = 5736;     // learned-predictor blob
// Lane table of a group: u16 base, then one u8 per lane; lane l occupies
// base + delta_l bits, base = max(min lane bits, max lane bits - 255) (lanes
// shorter than base are padded with zero bits, so every delta fits a byte).
constexpr uint32_t kLtabBytes = 34;

// header byte offsets
enum : uint32_t {
  H_MAGIC = 0, H_VERSION = 4, H_HBYTES = 8, H_DTYPE = 12, H_DIM = 16, H_FLAGS = 20, H_R1 = 24,
  H_R2 = 28, H_C1 = 32, H_C2 = 36, H_LMAX = 40, H_NX = 44, H_NY = 48, H_NZ = 52, H_NV = 56,
  H_NG = 64, H_TAU = 72, H_TAU1 = 80, H_TAU2 = 88, H_S1 = 96, H_S2 = 104, H_K = 112,
  H_RHO21 = 120, H_RHO12 = 128, H_FILL = 136, H_NOUT1 = 144, H_NOUT2 = 152, H_NRAW = 160,
  H_W1 = 168, H_W2 = 176, H_TOTAL = 184, H_MODEL = 192, H_QHI = 200,
  H_RUNLEN = 208  // zero-run stage: code lengths of the run tokens 2R, 2R + 1 of
                  // component 1 (bytes 208, 209) and component 2 (210, 211)
};
// header flags
enum : uint32_t {
  F_GUARD = 1, F_MODEL = 2, F_OPEN = 4, F_GNEAR = 8, F_FCLUSTER = 16, F_ONED = 32, F_ZRUN = 64
};
// Zero-run stage: a maximal run of r zero symbols (symbol R) in a lane chunk
// is coded as the digits d_i in {1, 2} of r = sum d_i 2^i (bijective base 2),
// least significant first, token 2R + d_i - 1; a code book covers 2R + 2
// tokens (the run tokens keep count 0, hence no code, without the stage).
constexpr int kRunTokens = 2;

__host__ __device__ inline uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }
__host__ __device__ inline int64_t ngroups(int64_t n, int C) {
  return n == 0 ? 0 : (n + 32 * (int64_t)C - 1) / (32 * (int64_t)C);
}

// Section offsets of a stream. Order: header | code lengths 1, 2 | group word
// offsets 1, 2 | group escape prefixes 1, 2 | group raw prefix 2 | lane bit
// lengths 1, 2 | escape values 1, 2 (int32) | raw values | bitstreams 1, 2 |
// learned-predictor blob (8-byte aligned, absent in plain streams).
struct Layout {
  uint64_t lens1, lens2, gtab1, gtab2, etab1, etab2, rtab2, ltab1, ltab2, out1, out2, raw, bits1,
      bits2, model, total;
};

__host__ __device__ inline Layout make_layout(int R1, int R2, int64_t ng1, int64_t ng2,
                                              uint64_t nout1, uint64_t nout2, uint64_t nraw,
                                              uint64_t vsz, uint64_t w1, uint64_t w2,
                                              uint64_t model_bytes = 0) {
  Layout L;
  uint64_t o = kHeaderBytes;
  L.lens1 = o; o += 2 * (uint64_t)R1;
  L.lens2 = o; o += 2 * (uint64_t)R2;
  o = align_up(o, 4);
  L.gtab1 = o; o += 4 * (uint64_t)(ng1 + 1);
  L.gtab2 = o; o += 4 * (uint64_t)(ng2 + 1);
  L.etab1 = o; o += 4 * (uint64_t)(ng1 + 1);
  L.etab2 = o; o += 4 * (uint64_t)(ng2 + 1);
  L.rtab2 = o; o += 4 * (uint64_t)(ng2 + 1);
  L.ltab1 = o; o += kLtabBytes * (uint64_t)ng1;
  L.ltab2 = o; o += kLtabBytes * (uint64_t)ng2;
  o = align_up(o, 4);
  L.out1 = o; o += 4 * nout1;
  L.out2 = o; o += 4 * nout2;
  o = align_up(o, 8);
  L.raw = o; o += vsz * nraw;
  o = align_up(o, 4);
  L.bits1 = o; o += 4 * w1;
  L.bits2 = o; o += 4 * w2;
  o = align_up(o, 8);
  L.model = o; o += model_bytes;
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// plan (device view)
// ---------------------------------------------------------------------------
struct PlanView {
  int dim;
  int32_t nx, ny, nz;
  int64_t n_v, n_g;
  // per grid point one 16-byte record of vertex ids (x, y, z(, w): vertices
  // 0..dim, x = -1 outside the mesh) and the u16 weights of vertices 1..dim:
  // in 2D in the record's w (lam1 | lam2 << 16), in 3D in an 8-byte record
  // (x, y, z; w = 0); one or two loads per point
  const int4 *vid4;     // [n_g]
  const ushort4 *lam4;  // [n_g], 3D only
  const uint32_t *cell; // [n_v]
  const uint16_t *frac; // [dim][n_v]
  // the same per vertex as one record for one vector load: 2D uint2 {cell,
  // fx | fy << 16}, 3D uint4 {cell, fx | fy << 16, fz, 0}
  const void *vrec;     // [n_v]
  // host side only: the plan's second stream, its fork / join events and the
  // mutex that keeps one call's fork and join together (all NULL: one stream)
  void *side, *ev_fork, *ev_join, *mu;
  int tile2d;  // MCC_TILE_* of the 2D grid kernel
  int vbps;    // blocks per SM and field of the vertex-streaming kernels (0: 8)
  int batch_fields;  // fields per batched launch chain (0: from the L2 size)
  int net_path;      // MCC_NET_*: the learned predictor's tensor-core path
};

// ---------------------------------------------------------------------------
// per-field parameters, computed on the device from the values
// ---------------------------------------------------------------------------
struct FieldParams {
  double lo, hi, M, tau, tau1, tau2, s1, s2, inv2;
  long long K, Qhi, fill_u, rho21_q, rho12_q;
  float rho21_f, rho12_f;
  int guard;
  int pad;
};

// Workspace status block (first 1 KiB of every workspace).
struct Status {
  unsigned int err;          // first error (mcc_status), 0 = OK
  unsigned int done_blocks;  // reduction completion counter
  unsigned long long out_size;
  unsigned long long key_lo, key_hi;  // ordered keys of min / max
  unsigned int nout1, nout2, nraw;    // escape counts (atomics)
  unsigned int groups_done;           // k_group_len completion counter
  unsigned long long w1, w2;          // bitstream words per component
  Layout L;                            // stream layout of the current call
  FieldParams f;
  unsigned int pick;                   // auto predictor: 1 = learned kept
};
static_assert(sizeof(Status) <= 1024, "status block");
constexpr size_t kStatusBytes = 1024;

__device__ inline void set_error(Status *st, unsigned int code) { atomicCAS(&st->err, 0u, code); }

// Ordered 64-bit key of a double: monotone for all non-NaN values.
__host__ __device__ inline unsigned long long order_key(double v) {
  unsigned long long b;
#ifdef __CUDA_ARCH__
  b = (unsigned long long)__double_as_longlong(v);
#else
  memcpy(&b, &v, 8);
#endif
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double key_value(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, 8);
  return v;
#endif
}

// ---------------------------------------------------------------------------
// predictor arithmetic (must match between compression and decompression)
// ---------------------------------------------------------------------------
// GB300 runs 64-bit integer <-> float conversions on its FP64 unit (a few
// operations per clock per SM), so the two below take 32-bit conversions and
// integer operations only, with the same results as __ull2float_rn and
// (long long)rintf.
//
// Nearest float of 0 <= v < 2^40: above 2^32 the bits below the 32 kept are
// folded into a sticky bit, which sits below the rounding position of the
// 24-bit significand (at least two bits below it), then an exact scaling.
__device__ __forceinline__ float u40_to_float(unsigned long long v) {
  if (v < (1ull << 32)) return __uint2float_rn((unsigned)v);
  const int s = v >= (1ull << 39) ? 8 : 7;
  const unsigned h = (unsigned)(v >> s) | ((v & ((1ull << s) - 1)) != 0 ? 1u : 0u);
  return __fmul_rn(__uint2float_rn(h), s == 8 ? 256.0f : 128.0f);
}

// rint(t) as a 64-bit integer for |t| < 2^62: below 2^30 the 32-bit
// conversion (ties to even); above, t is an integer (24-bit significand)
// rebuilt from its exponent and significand.
__device__ __forceinline__ long long rint_ll(float t) {
  if (fabsf(t) < 0x1p30f) return (long long)__float2int_rn(t);
  const unsigned b = __float_as_uint(t);
  const int e = (int)((b >> 23) & 0xFF) - 150;  // t = m 2^e, e >= 7 here
  const long long r = (long long)((b & 0x7FFFFFu) | 0x800000u) << e;
  return (b >> 31) ? -r : r;
}

// rint(u) (ties to even) as a 64-bit integer for |u| < 2^62, from the bits of
// u with integer operations: u = m 2^e with a 53-bit m; for e < 0 the bits
// below the binary point decide the rounding (above half, or exactly half
// with an odd integer part, rounds up). The same value as the FP64 -> int64
// conversion, which runs at a small fraction of the integer rate on this GPU.
__device__ __forceinline__ long long rint_ll64(double u) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  const int e = (int)((b >> 52) & 0x7FF) - 1075;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long r;
  if (e >= 0) {
    r = m << e;
  } else if (e < -53) {
    r = 0;  // |u| < 1/4 (and zero, subnormals)
  } else {
    const int s = -e;  // 1 .. 53
    const unsigned long long q = m >> s, rem = m & ((1ull << s) - 1), half = 1ull << (s - 1);
    r = q + ((rem > half || (rem == half && (q & 1))) ? 1ull : 0ull);
  }
  return (b >> 63) ? -(long long)r : (long long)r;
}

// round(rho * (a + acc)), rho = rq 2^-40: integer part of a*rho from the exact
// 128-bit product, 40-bit fraction plus FP32 correction acc*rho, one fused
// multiply-add, round to nearest even. rescale_split returns the integer part
// and the FP32 fraction before rounding. |t| stays far below 2^62: |acc| <
// 2^34 (int32 code differences), rho < 2^10, and the learned correction is
// clamped to 2^50.
__device__ __forceinline__ void rescale_split(int a, float acc, long long rq, float rf,
                                              long long &hi, float &t) {
  // |a| rq < 2^82 from two 32 x 32 -> 64-bit products (rq < 2^50): a rq =
  // (p1 + (p0 >> 32)) 2^32 + (p0 mod 2^32); 64-bit products and their high
  // halves are slow on this GPU
  const unsigned ua = a < 0 ? 0u - (unsigned)a : (unsigned)a;
  const unsigned long long ur = (unsigned long long)rq;
  const unsigned long long p0 = (unsigned long long)ua * (unsigned)ur;
  const unsigned long long p1 = (unsigned long long)ua * (unsigned)(ur >> 32);
  const unsigned long long mid = p1 + (p0 >> 32);
  const unsigned long long q = mid >> (kRhoBits - 32);
  const unsigned long long r = ((mid & ((1ull << (kRhoBits - 32)) - 1)) << 32) | (p0 & 0xFFFFFFFFull);
  unsigned long long lo;
  if (a >= 0) { hi = (long long)q; lo = r; }
  else if (r == 0) { hi = -(long long)q; lo = 0; }
  else { hi = -(long long)q - 1; lo = (1ull << kRhoBits) - r; }
  const float base = __fmul_rn(u40_to_float(lo), 0x1p-40f);
  t = __fmaf_rn(acc, rf, base);
}

template <bool HAS_P = false>
__device__ __forceinline__ long long rescale(int a, float acc, long long rq, float rf,
                                             float pc = 0.0f) {
  long long hi;
  float t;
  rescale_split(a, acc, rq, rf, hi, t);
  if (HAS_P) {  // the learned correction, in vertex bins; beyond +-2^50 the
                // residual code leaves int32 and the vertex is stored raw
    t = __fadd_rn(t, pc);
    t = fminf(fmaxf(t, -0x1p50f), 0x1p50f);
  }
  return hi + rint_ll(t);
}

__device__ __forceinline__ int wsub(int a, int b) { return (int)((unsigned)a - (unsigned)b); }
__device__ __forceinline__ int wadd(int a, int b) { return (int)((unsigned)a + (unsigned)b); }

// A vertex's cell and local coordinates (2^-15 units, as FP32) from its record.
template <int DIM>
__device__ __forceinline__ void vertex_record(const void *vrec, int64_t i, uint32_t &cell,
                                              float (&fr)[3]) {
  unsigned int f[3];
  // streamed once per call: evict-first, so the gathered grid codes stay in L2
  if (DIM == 2) {
    const uint2 r = __ldcs((const uint2 *)vrec + i);
    cell = r.x;
    f[0] = r.y & 0xFFFFu;
    f[1] = r.y >> 16;
    f[2] = 0;
  } else {
    const uint4 r = __ldcs((const uint4 *)vrec + i);
    cell = r.x;
    f[0] = r.y & 0xFFFFu;
    f[1] = r.y >> 16;
    f[2] = r.z;
  }
#pragma unroll
  for (int d = 0; d < 3; d++)
    fr[d] = d < DIM ? __fmul_rn(__uint2float_rn(f[d]), 0x1p-15f) : 0.0f;
}

// Grid -> vertex interpolation g (bilinear / trilinear on the grid codes of
// the vertex's cell) as acc = g - c_000 in grid bins. corner_codes gathers the
// cell's codes (order 000, 100, 010, 110, 001, 101, 011, 111), interp_acc
// evaluates the interpolation on their integer differences.
//
// The vertices come in the caller's order, so the cells of neighbouring
// threads are unrelated and every load is a gather of its own: the L1 serves
// one request per load and lane. row_pair reads a cell edge's two codes
// q1[r], q1[r + 1] with one aligned 16-byte load, plus a 4-byte load when
// r + 1 starts the next 16 bytes (one row in four): a 3D cell's eight codes
// take five requests on average instead of eight, a 2D cell's four take
// 2.5. Requires q1 16-byte aligned and readable 8 bytes past its last code
// (the workspaces pad it); the extra words are never used.
__device__ __forceinline__ void row_pair(const int *__restrict__ q1, int64_t r, int &lo, int &hi) {
  const int s = (int)(r & 3);
  const int4 v = __ldg((const int4 *)(q1 + (r - s)));
  lo = s == 0 ? v.x : s == 1 ? v.y : s == 2 ? v.z : v.w;
  hi = s == 0 ? v.y : s == 1 ? v.z : v.w;
  if (s == 3) hi = __ldg(q1 + r + 1);
}

template <int DIM>
__device__ __forceinline__ void corner_codes(const int *__restrict__ q1, uint32_t c, int nx,
                                             int64_t sxy, int (&k)[8]) {
  row_pair(q1, (int64_t)c, k[0], k[1]);
  row_pair(q1, (int64_t)c + nx, k[2], k[3]);
  if (DIM == 3) {
    row_pair(q1, (int64_t)c + sxy, k[4], k[5]);
    row_pair(q1, (int64_t)c + sxy + nx, k[6], k[7]);
  }
}

template <int DIM>
__device__ __forceinline__ float interp_acc(const int (&k)[8], float fx, float fy, float fz) {
  const int c000 = k[0], c100 = k[1], c010 = k[2], c110 = k[3];
  const int d100 = wsub(c100, c000), d010 = wsub(c010, c000);
  const int d110 = wadd(wsub(wsub(c110, c100), c010), c000);
  float acc;
  if (DIM == 2) {
    acc = __fmul_rn(fx, __int2float_rn(d100));
    acc = __fmaf_rn(fy, __int2float_rn(d010), acc);
    const float fxy = __fmul_rn(fx, fy);
    acc = __fmaf_rn(fxy, __int2float_rn(d110), acc);
  } else {
    const int c001 = k[4], c101 = k[5], c011 = k[6], c111 = k[7];
    const int d001 = wsub(c001, c000);
    const int d101 = wadd(wsub(wsub(c101, c100), c001), c000);
    const int d011 = wadd(wsub(wsub(c011, c010), c001), c000);
    int d111 = wsub(c111, c110);
    d111 = wsub(d111, c101);
    d111 = wsub(d111, c011);
    d111 = wadd(d111, c100);
    d111 = wadd(d111, c010);
    d111 = wadd(d111, c001);
    d111 = wsub(d111, c000);
    acc = __fmul_rn(fx, __int2float_rn(d100));
    acc = __fmaf_rn(fy, __int2float_rn(d010), acc);
    acc = __fmaf_rn(fz, __int2float_rn(d001), acc);
    const float fxy = __fmul_rn(fx, fy), fxz = __fmul_rn(fx, fz), fyz = __fmul_rn(fy, fz);
    const float fxyz = __fmul_rn(fxy, fz);
    acc = __fmaf_rn(fxy, __int2float_rn(d110), acc);
    acc = __fmaf_rn(fxz, __int2float_rn(d101), acc);
    acc = __fmaf_rn(fyz, __int2float_rn(d011), acc);
    acc = __fmaf_rn(fxyz, __int2float_rn(d111), acc);
  }
  return acc;
}

// Open loop: g on real corner values (vertex bins) in FP64, the same
// difference form and term order as interp_acc, every operation rounded on
// its own (no contraction): g = c_000 + sum of weight x difference.
template <int DIM>
__device__ __forceinline__ double interp64(const double (&c)[8], float fx, float fy, float fz) {
  const double x = fx, y = fy;
  const double d100 = __dsub_rn(c[1], c[0]), d010 = __dsub_rn(c[2], c[0]);
  const double d110 = __dadd_rn(__dsub_rn(__dsub_rn(c[3], c[1]), c[2]), c[0]);
  double acc = __dmul_rn(x, d100);
  acc = __dadd_rn(acc, __dmul_rn(y, d010));
  if (DIM == 2) {
    acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(x, y), d110));
    return __dadd_rn(c[0], acc);
  }
  const double z = fz;
  const double d001 = __dsub_rn(c[4], c[0]);
  const double d101 = __dadd_rn(__dsub_rn(__dsub_rn(c[5], c[1]), c[4]), c[0]);
  const double d011 = __dadd_rn(__dsub_rn(__dsub_rn(c[6], c[2]), c[4]), c[0]);
  double d111 = __dsub_rn(c[7], c[3]);
  d111 = __dsub_rn(d111, c[5]);
  d111 = __dsub_rn(d111, c[6]);
  d111 = __dadd_rn(d111, c[1]);
  d111 = __dadd_rn(d111, c[2]);
  d111 = __dadd_rn(d111, c[4]);
  d111 = __dsub_rn(d111, c[0]);
  acc = __dadd_rn(acc, __dmul_rn(z, d001));
  const double xy = __dmul_rn(x, y), xz = __dmul_rn(x, z), yz = __dmul_rn(y, z);
  const double xyz = __dmul_rn(xy, z);
  acc = __dadd_rn(acc, __dmul_rn(xy, d110));
  acc = __dadd_rn(acc, __dmul_rn(xz, d101));
  acc = __dadd_rn(acc, __dmul_rn(yz, d011));
  acc = __dadd_rn(acc, __dmul_rn(xyz, d111));
  return __dadd_rn(c[0], acc);
}

// g(x1') for the open loop: the grid codes in vertex bins, q1 rho12 (rho12 =
// rho12_q 2^-40, exact in FP64), interpolated by interp64.
template <int DIM>
__device__ __forceinline__ double interp64_codes(const int (&k)[8], long long rho12_q, float fx,
                                                 float fy, float fz) {
  const double r = __dmul_rn((double)rho12_q, 0x1p-40);
  double c[8];
#pragma unroll
  for (int t = 0; t < (1 << DIM); t++) c[t] = __dmul_rn((double)k[t], r);
  return interp64<DIM>(c, fx, fy, fz);
}

// Nearest grid node of a vertex (Sec. III-B): the corner of its cell on the
// near side of every midplane, from the local coordinates in 2^-15 units
// (exactly half goes to the upper node).
template <int DIM>
__device__ __forceinline__ uint32_t nearest_node(uint32_t c, unsigned fx, unsigned fy, unsigned fz,
                                                 int nx, int64_t sxy) {
  return c + (fx >= 16384u ? 1u : 0u) + (fy >= 16384u ? (uint32_t)nx : 0u) +
         (DIM == 3 && fz >= 16384u ? (uint32_t)sxy : 0u);
}

// returns c_000, acc = g - c_000
template <int DIM>
__device__ __forceinline__ int interp_vertex(const int *__restrict__ q1, uint32_t c, float fx,
                                             float fy, float fz, int nx, int64_t sxy, float &acc) {
  int k[8];
  corner_codes<DIM>(q1, c, nx, sxy, k);
  acc = interp_acc<DIM>(k, fx, fy, fz);
  return k[0];
}

// The vertex prediction in node units, P = round(rho12 * g + pc), pc the
// learned correction when HAS_P.
template <int DIM, bool HAS_P = false>
__device__ __forceinline__ long long predict_vertex(const int *__restrict__ q1, uint32_t c,
                                                    float fx, float fy, float fz, int nx,
                                                    int64_t sxy, long long rq, float rf,
                                                    float pc = 0.0f) {
  float acc;
  const int c000 = interp_vertex<DIM>(q1, c, fx, fy, fz, nx, sxy, acc);
  return rescale<HAS_P>(c000, acc, rq, rf, pc);
}

// ---------------------------------------------------------------------------
// canonical Huffman helpers
// ---------------------------------------------------------------------------
// Per-length symbol counts and first codes (deflate-style canonical order:
// codes increase with (length, symbol)).
struct CanonTables {
  unsigned int count[kMaxLen + 2];
  unsigned int first[kMaxLen + 2];
  unsigned int offset[kMaxLen + 2];
};

// Rank of every symbol among the symbols of equal length with a smaller id,
// computed by one CTA (blockDim multiple of 32, <= 1024). rank[] in shared
// memory, wcount is scratch [32][kMaxLen+1].
__device__ inline void canonical_ranks(const unsigned char *len, int nsym, unsigned short *rank,
                                       unsigned int (*wcount)[kMaxLen + 1]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int seg = (nsym + nw - 1) / nw;
  const int s0 = warp * seg, s1 = min(nsym, s0 + seg);
  if (lane <= kMaxLen) wcount[warp][lane] = 0;
  __syncwarp();
  for (int base = s0; base < s1; base += 32) {
    const int s = base + lane;
    const int L = s < s1 ? len[s] : 0;
    const unsigned same = __match_any_sync(0xffffffffu, L);
    const unsigned lt = (1u << lane) - 1;
    const unsigned r = __popc(same & lt);
    unsigned int running = 0;
    if (L > 0 && s < s1) running = wcount[warp][L];
    __syncwarp();
    if (L > 0 && s < s1) rank[s] = (unsigned short)(running + r);
    // the highest lane of each group advances the running count
    if (L > 0 && s < s1 && (same >> lane) == 1u) wcount[warp][L] = running + r + 1;
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, per length
  if (threadIdx.x <= kMaxLen) {
    const int L = threadIdx.x;
    unsigned int acc = 0;
    for (int w = 0; w < nw; w++) {
      const unsigned int c = wcount[w][L];
      wcount[w][L] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nsym; s += blockDim.x) {
    const int L = len[s];
    if (L > 0) {
      const int w = min(s / seg, nw - 1);
      rank[s] = (unsigned short)(rank[s] + wcount[w][L]);
    }
  }
  __syncthreads();
}

__device__ inline void canonical_tables(const unsigned char *len, int nsym, CanonTables *t) {
  if (threadIdx.x <= kMaxLen + 1) t->count[threadIdx.x] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nsym; s += blockDim.x)
    if (len[s]) atomicAdd(&t->count[len[s]], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int code = 0, off = 0;
    t->count[0] = 0;
    for (int l = 1; l <= kMaxLen; l++) {
      t->first[l] = code;
      t->offset[l] = off;
      off += t->count[l];
      code = (code + t->count[l]) << 1;
    }
  }
  __syncthreads();
}

}  // namespace mcc

// Device view of a plan's tables (defined in plan.cu).
mcc::PlanView mcc_plan_view(mcc_plan P);

namespace mcc {
// ---------------------------------------------------------------------------
// programmatic dependent launch: every kernel of a compress / decompress chain
// is launched with programmatic stream serialisation and waits for its
// predecessor's completion and memory (griddepcontrol.wait) before touching
// anything the predecessor writes. No kernel triggers its dependent early
// (launch_dependents): a block that exits counts as triggered, so the next
// kernel's blocks are scheduled as the predecessor's last blocks retire and
// its launch latency is hidden. An early trigger at kernel start let the
// waiting blocks of the next kernel hold SM slots (registers, shared memory)
// for the predecessor's whole run, which the predecessor's later blocks and
// the second stream's kernels then lacked (measured: the 3D step 0.925 ->
// 0.880 ms, the 2D step 0.218 -> 0.214 ms without it). Kernels launched
// without the attribute pass through the wait unchanged.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(std::forward<Args>(args))...);
}
}  // namespace mcc
