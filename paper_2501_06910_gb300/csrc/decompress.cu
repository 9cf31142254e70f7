// decompress.cu -- Algorithm 4 of Gong et al. (multi-component
// reconstruction): x1' = D(mu1), x2' = D(mu2), x' = g(x1') + x2'.
//
//   k_dec_prep    validate the header and the group tables' ends, build the
//                 canonical decode tables of both components (one CTA each)
//   k_dec_syms    Huffman decode of both components (one warp per group of
//                 32 lane chunks): grid Lorenzo differences, residual codes,
//                 escapes and raw values; for a single field the residual
//                 component's launch runs on the plan's second stream
//   k_scan_xy / k_scan_rows / k_scan_axis
//                 inverse Lorenzo: inclusive prefix sums along x, y (, z);
//                 in 3D x and y in one pass per z-plane (rows of <= 1024)
//   k_predict     learned correction p at every vertex (streams with a
//                 model; returns at once for the others)
//   k_recon       reconstruction x' = s2 (K + P + q2), P = round(rho12 g(q1)
//                 + p), fully parallel over the vertices
//
// Every read of the stream is bounds-checked against the validated layout; a
// corrupt stream records MCC_ERR_CORRUPT and the affected warp stops.
#include <cuda_runtime.h>

#include <mutex>
#include <limits.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "common.cuh"
#include "predictor.cuh"
#include "workspace.cuh"
#include "prof.cuh"

using namespace mcc;

namespace {

__device__ __forceinline__ uint32_t ld32(const unsigned char *p) { return *(const uint32_t *)p; }
__device__ __forceinline__ uint64_t ld64(const unsigned char *p) {
  return (uint64_t)ld32(p) | ((uint64_t)ld32(p + 4) << 32);
}

// Arguments shared by every decompression kernel of one launch chain: the
// plan, the workspace layout (one region of wss bytes per field), the input
// streams (iss bytes apart, in_bytes each) and the output arrays.
struct DecArgs {
  PlanView pv;
  DecompressWs W;
  unsigned char *ws0;
  int64_t wss;
  const unsigned char *in0;
  int64_t iss;
  int nf, dtype;
  uint64_t in_bytes[kMaxBatch];
  void *xo[kMaxBatch];
};

struct DCtx {
  Status *st;
  DecInfo *info;
  DecTab *tab1, *tab2;
  int *q1, *q2;
  float *p;
  const unsigned char *in;
  uint64_t in_bytes;
  void *xo;
};

__device__ __forceinline__ DCtx dctx_of(const DecArgs &A, int f) {
  DCtx c;
  unsigned char *ws = A.ws0 + (int64_t)f * A.wss;
  c.st = (Status *)ws;
  c.info = (DecInfo *)(ws + A.W.info);
  c.tab1 = (DecTab *)(ws + A.W.tab1);
  c.tab2 = (DecTab *)(ws + A.W.tab2);
  c.q1 = (int *)(ws + A.W.q1);
  c.q2 = (int *)(ws + A.W.q2);
  c.p = (float *)(ws + A.W.p);
  c.in = A.in0 + (int64_t)f * A.iss;
  c.in_bytes = A.in_bytes[f];
  c.xo = A.xo[f];
  return c;
}

__device__ __forceinline__ bool block_failed(const Status *st) {
  __shared__ int failed;
  if (threadIdx.x == 0) failed = *(volatile const unsigned int *)&st->err != 0;
  __syncthreads();
  return failed != 0;
}

// ---------------------------------------------------------------------------
// k_dec_prep
// ---------------------------------------------------------------------------
struct PrepArgs {
  const unsigned char *in;
  uint64_t in_bytes;
  int dtype;  // the caller's output type; the stream must match
  int dim, nx, ny, nz;
  int64_t n_v, n_g;
  DecInfo *info;
  DecTab *tab1, *tab2;
};

__device__ bool parse_header(const PrepArgs &a, const unsigned char *h, DecInfo &I) {
  if (ld32(h + H_MAGIC) != kMagic || ld32(h + H_VERSION) != kVersion ||
      ld32(h + H_HBYTES) != kHeaderBytes)
    return false;
  I.dtype = (int)ld32(h + H_DTYPE);
  I.dim = (int)ld32(h + H_DIM);
  const uint32_t flags = ld32(h + H_FLAGS);
  if (flags & ~(F_GUARD | F_MODEL | F_OPEN | F_GNEAR | F_FCLUSTER | F_ONED | F_ZRUN)) return false;
  // a 1D stream has this flag alone (or with the zero-run stage's), and only
  // 1D streams have it
  if (a.dim == 1 ? (flags & ~F_ZRUN) != F_ONED : (flags & F_ONED) != 0) return false;
  I.zr = (flags & F_ZRUN) ? 1 : 0;
  I.use_model = (flags & F_MODEL) ? 1 : 0;
  I.open = (flags & F_OPEN) ? 1 : 0;
  I.gnear = (flags & F_GNEAR) ? 1 : 0;  // (F_FCLUSTER concerns compression only)
  if ((I.open || I.gnear) && I.use_model) return false;
  if (ld64(h + H_MODEL) != (I.use_model ? kModelBytes : 0)) return false;
  I.Qhi = (long long)ld64(h + H_QHI);
  if (I.Qhi < 0 || I.Qhi >= (1ll << 29)) return false;
  if (I.dtype != a.dtype) return false;
  if (I.dim != a.dim || (int)ld32(h + H_NX) != a.nx || (int)ld32(h + H_NY) != a.ny ||
      (int)ld32(h + H_NZ) != a.nz)
    return false;
  if ((int64_t)ld64(h + H_NV) != a.n_v || (int64_t)ld64(h + H_NG) != a.n_g) return false;
  I.R1 = (int)ld32(h + H_R1);
  I.R2 = (int)ld32(h + H_R2);
  I.C1 = (int)ld32(h + H_C1);
  I.C2 = (int)ld32(h + H_C2);
  I.lmax = (int)ld32(h + H_LMAX);
  if (I.R1 < 4 || I.R1 > kMaxR || I.R2 < 4 || I.R2 > kMaxR) return false;
  if (I.zr && (I.R1 > kMaxR - 1 || I.R2 > kMaxR - 1)) return false;  // 2R + 2 tokens fit the tables
  if (I.C1 < 1 || I.C1 > kMaxC || I.C2 < 1 || I.C2 > kMaxC) return false;
  if (I.lmax < 1 || I.lmax > kMaxLen) return false;
  I.s2 = __longlong_as_double((long long)ld64(h + H_S2));
  if (!(I.s2 > 0.0) || !isfinite(I.s2)) return false;
  I.K = (long long)ld64(h + H_K);
  if (I.K <= -(1ll << 62) || I.K >= (1ll << 62)) return false;
  I.rho12_q = (long long)ld64(h + H_RHO12);
  if (!(I.rho12_q >= 1 && I.rho12_q < (1ll << 50))) return false;
  I.rho12_f = __fmul_rn(__ll2float_rn(I.rho12_q), 0x1p-40f);
  I.nout1 = ld64(h + H_NOUT1);
  I.nout2 = ld64(h + H_NOUT2);
  I.nraw = ld64(h + H_NRAW);
  I.w1 = ld64(h + H_W1);
  I.w2 = ld64(h + H_W2);
  if (I.nout1 > (uint64_t)a.n_g || I.nout2 > (uint64_t)a.n_v || I.nraw > (uint64_t)a.n_v) return false;
  I.ng1 = ngroups(a.n_g, I.C1);
  I.ng2 = a.dim == 1 ? 0 : ngroups(a.n_v, I.C2);  // the 1D coder has no residual component
  if (I.w1 > (uint64_t)a.n_g * kMaxLen / 32 + I.ng1 + 1 ||
      I.w2 > (uint64_t)a.n_v * kMaxLen / 32 + I.ng2 + 1)
    return false;
  const uint64_t vsz = I.dtype == MCC_F64 ? 8 : 4;
  I.L = make_layout(I.R1, I.R2, I.ng1, I.ng2, I.nout1, I.nout2, I.nraw, vsz, I.w1, I.w2,
                    I.use_model ? kModelBytes : 0);
  if (I.L.total != ld64(h + H_TOTAL) || I.L.total > a.in_bytes) return false;
  // the ends of the group tables: ten independent loads issued together
  const unsigned char *in = a.in;
  const uint64_t off[10] = {I.L.gtab1, I.L.gtab1 + 4 * I.ng1, I.L.gtab2, I.L.gtab2 + 4 * I.ng2,
                            I.L.etab1, I.L.etab1 + 4 * I.ng1, I.L.etab2, I.L.etab2 + 4 * I.ng2,
                            I.L.rtab2, I.L.rtab2 + 4 * I.ng2};
  const uint64_t want[10] = {0, I.w1, 0, I.w2, 0, I.nout1, 0, I.nout2, 0, I.nraw};
  unsigned int v[10];
#pragma unroll
  for (int k = 0; k < 10; k++) v[k] = ld32(in + off[k]);
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 10; k++) ok = ok && v[k] == want[k];
  return ok;
}

__global__ void __launch_bounds__(1024) k_dec_prep(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  Status *st = c.st;
  const PrepArgs a{c.in, c.in_bytes, A.dtype, A.pv.dim, A.pv.nx, A.pv.ny, A.pv.nz, A.pv.n_v,
                   A.pv.n_g, c.info, c.tab1, c.tab2};
  __shared__ DecInfo I;
  __shared__ int ok;
  __shared__ unsigned char lens[2 * kMaxR];
  __shared__ unsigned short rank[2 * kMaxR];
  __shared__ unsigned int wcount[32][kMaxLen + 1];
  __shared__ CanonTables ct;
  __shared__ int bad;
  __shared__ __align__(16) unsigned char hdr[kHeaderBytes];
  __shared__ unsigned int single[1 << kLutBits];
  // the header in one round trip (the stream must be at least a header long)
  const bool has_header = a.in_bytes >= kHeaderBytes;
  if (has_header && threadIdx.x < kHeaderBytes / 4)
    ((unsigned int *)hdr)[threadIdx.x] = __ldg((const unsigned int *)a.in + threadIdx.x);
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = has_header && parse_header(a, hdr, I) ? 1 : 0;
    bad = 0;
    if (!ok) set_error(st, MCC_ERR_CORRUPT);
    else if (blockIdx.x == 0) *a.info = I;
  }
  __syncthreads();
  if (!ok) return;
  const int ns = blockIdx.x == 0 ? 2 * I.R1 : 2 * I.R2;  // lengths in the lens section
  const int nsym = ns + (I.zr ? kRunTokens : 0);           // the zero-run stage's run tokens
  const unsigned char *src = a.in + (blockIdx.x == 0 ? I.L.lens1 : I.L.lens2);
  DecTab *T = blockIdx.x == 0 ? a.tab1 : a.tab2;
  for (int s = threadIdx.x; s < nsym; s += blockDim.x) {
    lens[s] = s < ns ? src[s] : hdr[H_RUNLEN + 2 * blockIdx.x + (s - ns)];
    if (lens[s] > I.lmax) bad = 1;
  }
  __syncthreads();
  if (bad) { if (threadIdx.x == 0) set_error(st, MCC_ERR_CORRUPT); return; }
  canonical_tables(lens, nsym, &ct);
  if (threadIdx.x == 0) {
    unsigned long long kraft = 0;
    for (int l = 1; l <= kMaxLen; l++) kraft += (unsigned long long)ct.count[l] << (kMaxLen - l);
    if (kraft > (1ull << kMaxLen)) bad = 1;
  }
  __syncthreads();
  if (bad) { if (threadIdx.x == 0) set_error(st, MCC_ERR_CORRUPT); return; }
  canonical_ranks(lens, nsym, rank, wcount);
  for (int s = threadIdx.x; s < nsym; s += blockDim.x)
    if (lens[s]) T->sorted[ct.offset[lens[s]] + rank[s]] = (unsigned short)s;
  if (threadIdx.x <= kMaxLen + 1) {
    const int l = threadIdx.x;
    T->first[l] = ct.first[l];
    T->count[l] = ct.count[l];
    T->offset[l] = ct.offset[l];
    T->lim[l] = l >= 1 && l <= kMaxLen
                    ? (unsigned long long)(ct.first[l] + ct.count[l]) << (32 - l) : 0ull;
  }
  __syncthreads();
  // first-level table: for the complete codes at the front of a kLutBits-bit
  // window (at most four), entry = l1 | total << 4 | count << 8 |
  // sym_j << (11 + 12 j): l1 the first code's length (0: longer than the
  // window), total the length of all `count` codes. Built in two passes: the
  // first code of every window (single), then chains of lookups in it. A
  // run token (zero-run stage) is never chained: it stands alone in its
  // entry, and a chain stops before one.
  const int lb = I.lmax < kLutBits ? I.lmax : kLutBits;
  for (int e = threadIdx.x; e < (1 << kLutBits); e += blockDim.x) {
    unsigned int v = 0;
    for (int l = 1; l <= lb; l++) {
      const unsigned int cw = (unsigned int)e >> (kLutBits - l);
      if (cw - ct.first[l] < ct.count[l]) {
        v = (unsigned int)l | ((unsigned int)T->sorted[ct.offset[l] + cw - ct.first[l]] << 8);
        break;
      }
    }
    single[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (1 << kLutBits); e += blockDim.x) {
    unsigned long long v = 0;
    int used = 0, cnt = 0;
    while (cnt < 4) {
      const unsigned int sv = single[((unsigned int)e << used) & ((1u << kLutBits) - 1)];
      const int l = (int)(sv & 15);
      if (!l || used + l > kLutBits) break;  // the window's zero padding is not code
      if ((int)(sv >> 8) >= ns && cnt) break;  // a run token after a symbol
      v |= (unsigned long long)(sv >> 8) << (11 + 12 * cnt);
      if (cnt == 0) v |= (unsigned long long)l;
      used += l;
      cnt++;
      if ((int)(sv >> 8) >= ns) break;  // a run token stands alone
    }
    if (cnt) v |= ((unsigned long long)used << 4) | ((unsigned long long)cnt << 8);
    T->lut[e] = v;
  }
}

// ---------------------------------------------------------------------------
// bit reader over one component's words (reads past the section give zeros)
// ---------------------------------------------------------------------------
struct BitReader {
  const unsigned int *w;
  unsigned long long nwords;
  unsigned long long buf;  // left aligned
  int nb;                  // valid bits in buf
  unsigned long long wi;   // next word
  unsigned long long consumed;
  unsigned int nxt;        // word wi, loaded one refill ahead (hides the load latency)

  __device__ __forceinline__ unsigned int word(unsigned long long i) const {
    return i < nwords ? __ldg(w + i) : 0u;
  }
  __device__ __forceinline__ void init(const unsigned int *words, unsigned long long n,
                                       unsigned long long bit) {
    w = words;
    nwords = n;
    wi = bit >> 5;
    buf = ((unsigned long long)word(wi) << 32) | word(wi + 1);
    wi += 2;
    nxt = word(wi);
    const int sk = (int)(bit & 31);
    buf <<= sk;
    nb = 64 - sk;
    consumed = 0;
  }
  __device__ __forceinline__ void refill() {
    if (nb < 32) {
      buf |= (unsigned long long)nxt << (32 - nb);
      wi++;
      nb += 32;
      nxt = word(wi);
    }
  }
};

__device__ __forceinline__ void load_tab(DecTab *dst, const DecTab *src, int nsym) {
  for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) dst->lut[i] = src->lut[i];
  for (int i = threadIdx.x; i < kMaxLen + 2; i += blockDim.x) {
    dst->first[i] = src->first[i];
    dst->count[i] = src->count[i];
    dst->offset[i] = src->offset[i];
    dst->lim[i] = src->lim[i];
  }
  for (int i = threadIdx.x; i < nsym; i += blockDim.x) dst->sorted[i] = src->sorted[i];
}

// Per-warp group set-up shared by both decoders: validates the group's table
// entries and positions every lane's reader. Returns false when corrupt.
__device__ __forceinline__ bool group_setup(const unsigned char *in, uint64_t gtab_off,
                                           uint64_t etab_off, uint64_t ltab_off, uint64_t bits_off,
                                           unsigned long long words, unsigned long long nesc,
                                           int64_t g, BitReader &r, unsigned int &lane_bits,
                                           unsigned int &lane_delta, unsigned int &e0,
                                           unsigned int &e1) {
  const int lane = threadIdx.x & 31;
  const unsigned int w0 = ld32(in + gtab_off + 4 * g), w1 = ld32(in + gtab_off + 4 * (g + 1));
  e0 = ld32(in + etab_off + 4 * g);
  e1 = ld32(in + etab_off + 4 * (g + 1));
  const unsigned char *lt = in + ltab_off + (uint64_t)g * kLtabBytes;
  lane_delta = lt[2 + lane];
  lane_bits = ((unsigned int)lt[0] | ((unsigned int)lt[1] << 8)) + lane_delta;
  unsigned int incl = lane_bits;
  for (int s = 1; s < 32; s <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, s);
    if (lane >= s) incl += t;
  }
  const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
  const bool ok = w0 <= w1 && w1 <= words && e0 <= e1 && e1 <= nesc &&
                  (unsigned long long)total <= 32ull * (w1 - w0);
  r.init((const unsigned int *)(in + bits_off), words, 32ull * w0 + (incl - lane_bits));
  return ok;
}

// ---------------------------------------------------------------------------
// k_dec_syms: Huffman decode of both components, one warp per group of 32
// lane chunks (the first nb1 blocks take the grid component, the rest the
// residual component; warps stride over their component's groups).
//
// Phase 1: every lane decodes its chunk into shared memory. When one symbol
// owns the 1-bit code "0" (canonical order gives it the all-zero code), the
// chunk is pre-filled with it and runs of it are skipped with a count of
// leading zeros. Phase 2: the warp walks the steps of the group with 32
// consecutive positions per step: grid symbols become Lorenzo differences,
// residual symbols become codes q2 (INT32_MIN marks a raw vertex, whose value
// is written to the output here); escapes and raw values take their slots
// from the group's prefixes and a ballot rank.
// ---------------------------------------------------------------------------
constexpr int kDecRound = 64;  // steps decoded per shared-memory round
// block shape: kDecWarps warps (one group each at a time) sharing one copy
// of the decode table, kDecBlocksPerSM resident blocks per SM
constexpr int kDecWarps = 8, kDecBlocksPerSM = 2;

template <typename T>
__global__ void __launch_bounds__(32 * kDecWarps, kDecBlocksPerSM) k_dec_syms(const __grid_constant__ DecArgs A, int nb1) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  const unsigned char *__restrict__ in = c.in;
  const DecInfo *__restrict__ info = c.info;
  const DecTab *__restrict__ tab1 = c.tab1;
  const DecTab *__restrict__ tab2 = c.tab2;
  const int64_t n_g = A.pv.n_g, n_v = A.pv.n_v;
  int *__restrict__ delta = c.q1;
  int *__restrict__ q2s = c.q2;
  T *__restrict__ xo = (T *)c.xo;
  Status *st = c.st;
  __shared__ DecTab Tb;
  extern __shared__ unsigned short sbuf[];  // [warps][kDecRound][32]
  if (block_failed(st)) return;
  const DecInfo I = *info;
  const bool c1 = (int)blockIdx.x < nb1;
  const int64_t ng = c1 ? I.ng1 : I.ng2;
  {  // blocks without a group skip the table load
    const int64_t first = (c1 ? (int64_t)blockIdx.x : (int64_t)blockIdx.x - nb1) * (blockDim.x >> 5);
    if (first >= ng) return;
  }
  // (with the zero-run stage the code book also holds the two run tokens)
  load_tab(&Tb, c1 ? tab1 : tab2, (c1 ? 2 * I.R1 : 2 * I.R2) + (I.zr ? kRunTokens : 0));
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t n = c1 ? n_g : n_v;
  const int C = c1 ? I.C1 : I.C2, R = c1 ? I.R1 : I.R2, rawsym = 2 * R - 1;
  const int lmax = I.lmax;
  const int *outv = (const int *)(in + (c1 ? I.L.out1 : I.L.out2));
  const T *rawv = (const T *)(in + I.L.raw);
  int *dst = c1 ? delta : q2s;
  const int tok0 = 2 * R;
  unsigned short *buf = sbuf + (size_t)wid * kDecRound * 32;
  const int64_t b0 = c1 ? blockIdx.x : blockIdx.x - nb1;
  const int64_t nblocks = c1 ? nb1 : gridDim.x - nb1;
  const int64_t wstride = nblocks * (blockDim.x >> 5);
  // The group loop, compiled once per stream kind (the branch is uniform):
  // with the zero-run stage (run tokens 2R for a digit 1 and 2R + 1 for a
  // digit 2; the chunk is pre-filled with the zero symbol R and a digit d at
  // digit position i skips d 2^i steps), and without it.
  auto groups = [&](auto zr_kind) {
  constexpr bool zr = decltype(zr_kind)::value;
  const bool fast = !zr && Tb.count[1] == 1;   // a symbol owns the code "0"
  const unsigned short s0 = zr ? (unsigned short)R : Tb.sorted[0];  // the pre-fill symbol
  for (int64_t g = b0 * (blockDim.x >> 5) + wid; g < ng; g += wstride) {
    BitReader r;
    unsigned int lane_bits, lane_delta, e0, e1, r0 = 0, r1 = 0;
    bool ok = c1 ? group_setup(in, I.L.gtab1, I.L.etab1, I.L.ltab1, I.L.bits1, I.w1, I.nout1, g, r,
                               lane_bits, lane_delta, e0, e1)
                 : group_setup(in, I.L.gtab2, I.L.etab2, I.L.ltab2, I.L.bits2, I.w2, I.nout2, g, r,
                               lane_bits, lane_delta, e0, e1);
    if (!c1) {
      r0 = ld32(in + I.L.rtab2 + 4 * g);
      r1 = ld32(in + I.L.rtab2 + 4 * (g + 1));
      ok = ok && r0 <= r1 && r1 <= I.nraw;
    }
    if (!ok) {
      if (lane == 0) set_error(st, MCC_ERR_CORRUPT);
      return;
    }
    const int64_t gbase = g * 32 * (int64_t)C;
    const int64_t left = n - gbase - lane;  // positions of this lane: gbase + lane + 32 k
    const int cnt = left <= 0 ? 0 : (int)min((int64_t)C, (left + 31) / 32);
    bool lane_bad = false;
    unsigned int used = 0, e_run = e0, r_run = r0;
    int k = 0, digit = 0;
    // a group without escapes or raw values takes the vectorised emit path
    const bool simple = e0 == e1 && (c1 || r0 == r1);
    for (int kb = 0; kb < C; kb += kDecRound) {
      const int kend = min(cnt, kb + kDecRound);
      const int steps = min(kDecRound, C - kb);
      const int64_t p0 = gbase + 32 * (int64_t)kb;  // first position of the round
      if (p0 >= n) break;
      // ---- phase 1: decode this round of the lane's chunk into shared memory
      // (buf holds the round's positions in order: p0 + 32 (k - kb) + lane)
      if (fast || zr) {
        const unsigned int f2 = (unsigned int)s0 | ((unsigned int)s0 << 16);
        const uint4 f4 = make_uint4(f2, f2, f2, f2);
        for (int q = lane; q < steps * 4; q += 32) reinterpret_cast<uint4 *>(buf)[q] = f4;
        __syncwarp();
      }
      while (k < kend && !lane_bad) {
        r.refill();
        const unsigned int win = (unsigned int)(r.buf >> 32);
        if (fast && !(win >> 31)) {
          int z = win ? __clz(win) : 32;  // a run of the symbol coded "0"
          z = min(z, kend - k);
          r.buf <<= z;
          r.nb -= z;
          used += z;
          k += z;
          continue;
        }
        const unsigned long long e = Tb.lut[win >> (32 - kLutBits)];
        int len = (int)(e & 15), sym;
        if (len) {
          const int cnt = (int)((e >> 8) & 7);
          if (cnt > 1 && k + cnt <= kend) {  // every complete code in the window
            len = (int)((e >> 4) & 15);      // (symbols only: run tokens stand alone)
            unsigned short *bp = buf + (k - kb) * 32 + lane;
            bp[0] = (unsigned short)((e >> 11) & 0xFFF);
            if (cnt > 2) bp[32] = (unsigned short)((e >> 23) & 0xFFF);
            if (cnt > 3) bp[64] = (unsigned short)((e >> 35) & 0xFFF);
            k += cnt - 1;  // the last code is written below
            sym = (int)((e >> (11 + 12 * (cnt - 1))) & 0xFFF);
          } else {
            sym = (int)((e >> 11) & 0xFFF);
          }
        } else {
          // a code longer than the table: its length from the limits (one
          // independent comparison per length instead of a serial search;
          // the window is at or above lim[kLutBits] here)
          int nl = 0;
#pragma unroll
          for (int l = kLutBits + 1; l <= kMaxLen; l++)
            nl += (l <= lmax && (unsigned long long)win >= Tb.lim[l]) ? 1 : 0;
          len = kLutBits + 1 + nl;
          if (len > lmax) { lane_bad = true; break; }
          sym = Tb.sorted[Tb.offset[len] + (win >> (32 - len)) - Tb.first[len]];
        }
        r.buf <<= len;
        r.nb -= len;
        used += len;
        if (zr && sym >= tok0) {  // a run digit: its zeros are pre-filled
          const int z = (sym - tok0 + 1) << digit;
          if (z > cnt - k) { lane_bad = true; break; }
          k += z;
          digit++;
          continue;
        }
        digit = 0;
        buf[(k - kb) * 32 + lane] = (unsigned short)sym;
        k++;
      }
      __syncwarp();
      // ---- phase 2: the round's values in position order, four per lane and
      // 16-byte store per iteration (128 positions per warp iteration);
      // escapes and raw values take their slots from the group's prefixes
      // plus a warp scan of the per-lane counts (skipped when the iteration
      // has none, and for the whole round when the group has none)
      {
        const int64_t nvalid = min((int64_t)32 * steps, n - p0);
        for (int it = 0; (int64_t)it * 128 < nvalid; it++) {
          const int q = it * 32 + lane;
          const int64_t t0 = 4 * (int64_t)q;
          const int nv = t0 >= nvalid ? 0 : (int)min((int64_t)4, nvalid - t0);
          int sy[4] = {-1, -1, -1, -1};
          if (nv) {
            const uint2 s4 = reinterpret_cast<const uint2 *>(buf)[q];
            sy[0] = (int)(s4.x & 0xFFFFu);
            sy[1] = (int)(s4.x >> 16);
            sy[2] = (int)(s4.y & 0xFFFFu);
            sy[3] = (int)(s4.y >> 16);
            for (int e = nv; e < 4; e++) sy[e] = -1;
          }
          int v[4];
          unsigned em = 0, rm = 0;  // this lane's escapes / raw values (bit e)
#pragma unroll
          for (int e = 0; e < 4; e++) {
            v[e] = sy[e] - R;
            if (sy[e] == 0) em |= 1u << e;
            else if (sy[e] == rawsym) {
              if (c1) lane_bad = true;
              else rm |= 1u << e;
            }
          }
          if (!simple && __any_sync(0xffffffffu, em | rm)) {
            unsigned int ce = __popc(em), cr = __popc(rm), xe = ce, xr = cr;
            for (int o = 1; o < 32; o <<= 1) {  // inclusive scans over the lanes
              const unsigned int te = __shfl_up_sync(0xffffffffu, xe, o);
              const unsigned int tr = __shfl_up_sync(0xffffffffu, xr, o);
              if (lane >= o) { xe += te; xr += tr; }
            }
            unsigned int ie = e_run + xe - ce, ir = r_run + xr - cr;
#pragma unroll
            for (int e = 0; e < 4; e++) {
              if ((em >> e) & 1) {
                v[e] = 0;
                if (ie < e1) v[e] = __ldg(outv + ie);
                else lane_bad = true;
                if (!c1 && v[e] == INT_MIN) lane_bad = true;  // never an escape value
                ie++;
              } else if ((rm >> e) & 1) {
                if (ir < r1) xo[p0 + t0 + e] = rawv[ir];
                else lane_bad = true;
                v[e] = INT_MIN;
                ir++;
              }
            }
            e_run += __shfl_sync(0xffffffffu, xe, 31);
            r_run += __shfl_sync(0xffffffffu, xr, 31);
          } else if (em | rm) {
            lane_bad = true;  // the group's tables say it has none
          }
          if (nv == 4) {
            *reinterpret_cast<int4 *>(dst + p0 + t0) = make_int4(v[0], v[1], v[2], v[3]);
          } else {
            for (int e = 0; e < nv; e++) dst[p0 + t0 + e] = v[e];
          }
        }
        __syncwarp();
      }
    }
    // the codes fill the lane, or a padded lane (delta 0) ends early
    if (used > lane_bits || (used < lane_bits && lane_delta != 0)) lane_bad = true;
    if (__any_sync(0xffffffffu, lane_bad) || e_run != e1 || r_run != r1) {
      if (lane == 0) set_error(st, MCC_ERR_CORRUPT);
      return;
    }
    __syncwarp();
  }
  };
  if (I.zr) groups(std::true_type{});
  else groups(std::false_type{});
}

// ---------------------------------------------------------------------------
// inverse Lorenzo: inclusive prefix sums (wrapping int32 arithmetic)
// ---------------------------------------------------------------------------
// One warp per row; every lane holds 8 consecutive values of a 256-value
// chunk (two 16-byte loads when the rows are 16-byte aligned), scans them
// locally, and a warp scan of the lane totals offsets them. The next chunk is
// loaded before the current one is stored, so the loads of a row overlap.
__device__ __forceinline__ void load8(const int *r, int i0, int nx, bool vec, unsigned int (&v)[8]) {
  if (vec && i0 + 8 <= nx) {
    const int4 a = *reinterpret_cast<const int4 *>(r + i0);
    const int4 b = *reinterpret_cast<const int4 *>(r + i0 + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; e++) v[e] = i0 + e < nx ? (unsigned int)r[i0 + e] : 0u;
  }
}

__global__ void __launch_bounds__(256) k_scan_rows(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  int *q = c.q1;
  const int nx = A.pv.nx;
  const int64_t nrows = (int64_t)A.pv.ny * A.pv.nz;
  const Status *st = c.st;
  if (*(volatile const unsigned int *)&st->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= nrows) return;
  int *r = q + row * nx;
  const bool vec = (nx & 3) == 0;  // rows start on 16-byte boundaries (q is 256-aligned)
  unsigned int carry = 0;
  unsigned int v[8];
  load8(r, 8 * lane, nx, vec, v);
  for (int base = 0; base < nx; base += 256) {
    unsigned int nv[8];
    if (base + 256 < nx) load8(r, base + 256 + 8 * lane, nx, vec, nv);
#pragma unroll
    for (int e = 1; e < 8; e++) v[e] += v[e - 1];
    unsigned int incl = v[7];
    for (int sft = 1; sft < 32; sft <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, sft);
      if (lane >= sft) incl += t;
    }
    const unsigned int off = carry + incl - v[7];
    const int i0 = base + 8 * lane;
    if (vec && i0 + 8 <= nx) {
      *reinterpret_cast<int4 *>(r + i0) =
          make_int4((int)(v[0] + off), (int)(v[1] + off), (int)(v[2] + off), (int)(v[3] + off));
      *reinterpret_cast<int4 *>(r + i0 + 4) =
          make_int4((int)(v[4] + off), (int)(v[5] + off), (int)(v[6] + off), (int)(v[7] + off));
    } else {
#pragma unroll
      for (int e = 0; e < 8; e++)
        if (i0 + e < nx) r[i0 + e] = (int)(v[e] + off);
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
#pragma unroll
    for (int e = 0; e < 8; e++) v[e] = nv[e];
  }
}

// 3D, rows of at most 256 CH codes (nx a multiple of 4): the x and y passes
// fused, one CTA per z-plane. Batches of RB rows, one per warp: each warp
// x-scans its row (as k_scan_rows), the rows go to shared memory, every
// thread adds down its columns over the batch from the running column sums
// of the rows above (the y prefix), and the warps store their rows. The rows
// of the next two batches are in flight while a batch is scanned. One pass
// over q1 instead of two (k_scan_rows, then k_scan_axis along y).
constexpr int kScanRB = 16;  // rows per batch of the plane scan (rows of <= 256 codes)

template <int CH, int RB>
__global__ void __launch_bounds__(32 * RB) k_scan_xy(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  if (*(volatile const unsigned int *)&c.st->err) return;
  const int nx = A.pv.nx, ny = A.pv.ny;
  int *plane = c.q1 + (int64_t)blockIdx.x * nx * ny;
  extern __shared__ unsigned int sxy[];  // [RB][nx] batch rows, then [nx] column sums
  unsigned int *T = sxy, *colsum = sxy + RB * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) colsum[i] = 0u;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned int v[CH][8], nv[CH][8], nv2[CH][8];
  auto load_row = [&](int r, unsigned int (&d)[CH][8]) {
#pragma unroll
    for (int k = 0; k < CH; k++) {
      if (r < ny) load8(plane + (int64_t)r * nx, 256 * k + 8 * lane, nx, true, d[k]);
      else
#pragma unroll
        for (int e = 0; e < 8; e++) d[k][e] = 0u;
    }
  };
  load_row(w, v);
  load_row(w + RB, nv);
  for (int b = 0; b < ny; b += RB) {
    const int r = b + w;
    load_row(r + 2 * RB, nv2);  // two batches ahead
    // x prefix of this warp's row, into the batch tile
    unsigned int carry = 0;
#pragma unroll
    for (int k = 0; k < CH; k++) {
#pragma unroll
      for (int e = 1; e < 8; e++) v[k][e] += v[k][e - 1];
      unsigned int incl = v[k][7];
      for (int sft = 1; sft < 32; sft <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, incl, sft);
        if (lane >= sft) incl += t;
      }
      const unsigned int off = carry + incl - v[k][7];
      const int i0 = 256 * k + 8 * lane;
      if (i0 < nx) {
        unsigned int *t = T + w * nx + i0;
        if (i0 + 8 <= nx) {
          *reinterpret_cast<uint4 *>(t) = make_uint4(v[k][0] + off, v[k][1] + off, v[k][2] + off, v[k][3] + off);
          *reinterpret_cast<uint4 *>(t + 4) = make_uint4(v[k][4] + off, v[k][5] + off, v[k][6] + off, v[k][7] + off);
        } else {
#pragma unroll
          for (int e = 0; e < 8; e++)
            if (i0 + e < nx) t[e] = v[k][e] + off;
        }
      }
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncthreads();
    // y prefix down the batch's columns
    const int nr = min(RB, ny - b);
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      unsigned int run = colsum[x];
      for (int q = 0; q < nr; q++) {
        run += T[q * nx + x];
        T[q * nx + x] = run;
      }
      colsum[x] = run;
    }
    __syncthreads();
    if (r < ny) {
      int *dst = plane + (int64_t)r * nx;
      for (int i = 4 * lane; i < nx; i += 128)
        *reinterpret_cast<uint4 *>(dst + i) = *reinterpret_cast<const uint4 *>(T + w * nx + i);
    }
    __syncthreads();  // the tile is rewritten by the next batch
#pragma unroll
    for (int k = 0; k < CH; k++)
#pragma unroll
      for (int e = 0; e < 8; e++) { v[k][e] = nv[k][e]; nv[k][e] = nv2[k][e]; }
  }
}

// Inclusive scan along an axis of length L and stride S, for columns
// base = outer * plane + inner (inner < n_inner contiguous). Block: 32
// consecutive columns x W warps, each warp scanning one segment of the axis
// (W = 32 when there are few column blocks, 8 otherwise).
template <int W>
__global__ void __launch_bounds__(32 * W) k_scan_axis(const __grid_constant__ DecArgs A, int64_t n_inner,
                                                      int64_t n_outer, int64_t plane, int L, int64_t S) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  int *q = c.q1;
  const Status *st = c.st;
  __shared__ unsigned int part[W][33];
  if (*(volatile const unsigned int *)&st->err) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t nblk_inner = (n_inner + 31) / 32;
  const int64_t outer = blockIdx.x / nblk_inner;
  const int64_t inner = (blockIdx.x % nblk_inner) * 32 + lane;
  const bool valid = inner < n_inner && outer < n_outer;
  int *col = q + outer * plane + inner;
  const int seg = (L + W - 1) / W;
  const int t0 = w * seg, t1 = min(L, t0 + seg);
  unsigned int sum = 0;
  if (valid)
    for (int t = t0; t < t1; t++) sum += (unsigned int)col[(int64_t)t * S];
  part[w][lane] = sum;
  __syncthreads();
  unsigned int pre = 0;
  for (int k = 0; k < w; k++) pre += part[k][lane];
  if (valid)  // eight loads in flight before their stores
    for (int t = t0; t < t1; t += 8) {
      unsigned int v[8];
#pragma unroll
      for (int e = 0; e < 8; e++) v[e] = t + e < t1 ? (unsigned int)col[(int64_t)(t + e) * S] : 0u;
#pragma unroll
      for (int e = 0; e < 8; e++) {
        pre += v[e];
        if (t + e < t1) col[(int64_t)(t + e) * S] = (int)pre;
      }
    }
}

// ---------------------------------------------------------------------------
// the 1D coder: Q = inclusive prefix sums of the differences (wrapping int32)
// in three launches (chunk sums, their exclusive scan in one block, the
// chunks scanned from their offsets), then x' = s (K + Q)
// ---------------------------------------------------------------------------
constexpr int kScan1dChunk = 256 * 16;  // values per chunk (one block)

__global__ void __launch_bounds__(256) k_scan1d_sums(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  if (*(volatile const unsigned int *)&c.st->err) return;
  const int64_t n = A.pv.n_g;
  const int *__restrict__ d = c.q1;
  unsigned int *part = (unsigned int *)c.q2;
  const int64_t nchunk = (n + kScan1dChunk - 1) / kScan1dChunk;
  __shared__ unsigned int ws[8];
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const int64_t base = ch * kScan1dChunk;
    unsigned int v[16], sum = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int64_t i = base + threadIdx.x + 256 * k;
      v[k] = i < n ? (unsigned int)__ldg(d + i) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 16; k++) sum += v[k];
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int t = 0;
      for (int w = 0; w < 8; w++) t += ws[w];
      part[ch] = t;
    }
    __syncthreads();
  }
}

// exclusive scan of the chunk sums, in place (one block per field)
__global__ void __launch_bounds__(1024) k_scan1d_top(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  if (*(volatile const unsigned int *)&c.st->err) return;
  const int64_t nchunk = (A.pv.n_g + kScan1dChunk - 1) / kScan1dChunk;
  unsigned int *part = (unsigned int *)c.q2;
  __shared__ unsigned int ws[32];
  __shared__ unsigned int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t base = 0; base < nchunk; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const unsigned int v = i < nchunk ? part[i] : 0u;
    unsigned int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    if (w == 0) {
      unsigned int s = ws[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += t;
      }
      ws[lane] = s;  // inclusive over the warps
    }
    __syncthreads();
    const unsigned int excl = carry + (w ? ws[w - 1] : 0u) + incl - v;
    if (i < nchunk) part[i] = excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += ws[31];
    __syncthreads();
  }
}

// each chunk scanned from its offset: Q, then x' = s (K + Q)
template <typename T>
__global__ void __launch_bounds__(256) k_recon1d(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.y);
  if (*(volatile const unsigned int *)&c.st->err) return;
  const DecInfo I = *c.info;
  const int64_t n = A.pv.n_g;
  const int *__restrict__ d = c.q1;
  const unsigned int *part = (const unsigned int *)c.q2;
  T *__restrict__ xo = (T *)c.xo;
  const int64_t nchunk = (n + kScan1dChunk - 1) / kScan1dChunk;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ unsigned int ws[8];
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    // 16 consecutive values per thread: a local scan, then the scan of the
    // thread totals across the block
    const int64_t base = ch * kScan1dChunk + 16 * (int64_t)threadIdx.x;
    unsigned int v[16];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = base + k < n ? (unsigned int)__ldg(d + base + k) : 0u;
#pragma unroll
    for (int k = 1; k < 16; k++) v[k] += v[k - 1];
    unsigned int incl = v[15];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    unsigned int before = 0;
    for (int k = 0; k < w; k++) before += ws[k];
    const unsigned int off = __ldg(part + ch) + before + incl - v[15];
#pragma unroll
    for (int k = 0; k < 16; k++)
      if (base + k < n)
        xo[base + k] = (T)__dmul_rn(I.s2, (double)(I.K + (long long)(int)(v[k] + off)));
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// k_recon: x' = s2 (K + P + q2) at every vertex, P = round(rho12 g(x1'));
// open-loop streams: x' = s2 ((K + q2) + g(x1')) in FP64 (recon_open)
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__device__ __forceinline__ void recon_open(const DecArgs &A, double s2, long long K,
                                           long long rho12_q, bool near, const int *q1,
                                           const int *q2s, T *xo) {
  const PlanView &pv = A.pv;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  for (int64_t p = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; p < n; p += stride) {
    const int q2 = __ldg(q2s + p);
    if (q2 == INT_MIN) continue;  // raw value already in place
    const uint32_t cl = __ldg(pv.cell + p);
    const float fx = __fmul_rn(__uint2float_rn(__ldg(pv.frac + p)), 0x1p-15f);
    const float fy = __fmul_rn(__uint2float_rn(__ldg(pv.frac + n + p)), 0x1p-15f);
    const float fz =
        DIM == 3 ? __fmul_rn(__uint2float_rn(__ldg(pv.frac + 2 * n + p)), 0x1p-15f) : 0.0f;
    double gq;
    if (near) {  // nearest-node g
      const uint32_t m = nearest_node<DIM>(cl, __ldg(pv.frac + p), __ldg(pv.frac + n + p),
                                           DIM == 3 ? __ldg(pv.frac + 2 * n + p) : 0u, nx, sxy);
      gq = __dmul_rn((double)__ldg(q1 + m), __dmul_rn((double)rho12_q, 0x1p-40));
    } else {
      int cor[8];
      corner_codes<DIM>(q1, cl, nx, sxy, cor);
      gq = interp64_codes<DIM>(cor, rho12_q, fx, fy, fz);
    }
    xo[p] = (T)__dmul_rn(s2, __dadd_rn((double)(K + (long long)q2), gq));
  }
}

// Closed loop with the nearest-node g: x' = s2 (K + P + q2), P =
// round((s1/s2) q1[m]), one gather per vertex.
template <int DIM, typename T>
__device__ __forceinline__ void recon_nearest(const DecArgs &A, const DecInfo &I, const int *q1,
                                              const int *q2s, T *xo) {
  const PlanView &pv = A.pv;
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  for (int64_t p = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; p < n; p += stride) {
    const int q2 = __ldg(q2s + p);
    if (q2 == INT_MIN) continue;  // raw value already in place
    const uint32_t m = nearest_node<DIM>(__ldg(pv.cell + p), __ldg(pv.frac + p),
                                         __ldg(pv.frac + n + p),
                                         DIM == 3 ? __ldg(pv.frac + 2 * n + p) : 0u, nx, sxy);
    const long long P = rescale(__ldg(q1 + m), 0.0f, I.rho12_q, I.rho12_f);
    xo[p] = (T)__dmul_rn(I.s2, (double)(I.K + P + (long long)q2));
  }
}

template <int DIM, typename T, int U>
__global__ void __launch_bounds__(256) k_recon(const __grid_constant__ DecArgs A) {
  pdl_wait();
  const DCtx c = dctx_of(A, blockIdx.x);
  const DecInfo *__restrict__ info = c.info;
  const PlanView &pv = A.pv;
  const int *__restrict__ q1 = c.q1;
  const int *__restrict__ q2s = c.q2;
  const float *__restrict__ pcor = c.p;
  T *__restrict__ xo = (T *)c.xo;
  const Status *st = c.st;
  if (*(volatile const unsigned int *)&st->err) return;
  const DecInfo I = *info;
  if (I.open) {
    recon_open<DIM, T>(A, I.s2, I.K, I.rho12_q, I.gnear != 0, q1, q2s, xo);
    return;
  }
  if (I.gnear) {
    recon_nearest<DIM, T>(A, I, q1, q2s, xo);
    return;
  }
  const int64_t n = pv.n_v;
  const int nx = pv.nx;
  const int64_t sxy = (int64_t)pv.nx * pv.ny;
  const int64_t stride = (int64_t)gridDim.y * blockDim.x;
  for (int64_t p0 = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; p0 < n; p0 += U * stride) {
    // U vertices per iteration, their gathers issued together
    int64_t pv2[U];
    pv2[0] = p0;
#pragma unroll
    for (int u = 1; u < U; u++) pv2[u] = pv2[u - 1] + stride;
    bool go[U];
    int q2v[U];
    uint32_t cl[U];
    float fr[U][3];
    int cor[U][8];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int64_t p = pv2[u] < n ? pv2[u] : p0;
      q2v[u] = __ldcs(q2s + p);
      go[u] = pv2[u] < n && q2v[u] != INT_MIN;  // INT_MIN: raw value already in place
      vertex_record<DIM>(pv.vrec, p, cl[u], fr[u]);
    }
#pragma unroll
    for (int u = 0; u < U; u++) corner_codes<DIM>(q1, cl[u], nx, sxy, cor[u]);
#pragma unroll
    for (int u = 0; u < U; u++) {
      if (!go[u]) continue;
      const int64_t p = pv2[u];
      const float acc = interp_acc<DIM>(cor[u], fr[u][0], fr[u][1], fr[u][2]);
      // one code path for both stream kinds: adding p = 0 leaves the plain
      // prediction unchanged (t + 0 = t, and -0 + 0 = +0 rounds to the same 0)
      const float pc = I.use_model ? __ldg(pcor + p) : 0.0f;
      const long long P = rescale<true>(cor[u][0], acc, I.rho12_q, I.rho12_f, pc);
      __stcs(xo + p, (T)__dmul_rn(I.s2, (double)(I.K + P + (long long)q2v[u])));  // streamed out
    }
  }
}

inline unsigned int nblk(int64_t n, int bs) {
  const int64_t b = (n + bs - 1) / bs;
  return (unsigned int)(b < 1 ? 1 : b);
}

}  // namespace

DecompressWs decompress_ws_layout(const PlanView &pv) {
  DecompressWs w;
  size_t o = kStatusBytes;
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  w.info = take(sizeof(DecInfo));
  w.tab1 = take(sizeof(DecTab));
  w.tab2 = take(sizeof(DecTab));
  w.q1 = take(4 * (size_t)pv.n_g + 16);  // + 16: the corner gathers' aligned 16-byte loads
  w.q2 = take(4 * (size_t)pv.n_v);
  w.p = take(4 * (size_t)pv.n_v);
  w.total = o;
  return w;
}

// Decompress nf fields (nf <= kMaxBatch): field f reads in_bytes[f] bytes at
// in0 + f * iss, uses the workspace region ws0 + f * wss and writes n_v
// values of dtype to xo[f].
mcc_status launch_decompress_batch(const PlanView &pv, int nf, const unsigned char *in0, int64_t iss,
                                   const uint64_t *in_bytes, void *const *xo, int dtype,
                                   unsigned char *ws0, int64_t wss, cudaStream_t stream) {
  if (nf < 1 || nf > kMaxBatch) return MCC_ERR_INVALID_ARG;
  DecArgs A;
  memset(&A, 0, sizeof(A));
  A.pv = pv;
  A.W = decompress_ws_layout(pv);
  A.ws0 = ws0;
  A.wss = wss;
  A.in0 = in0;
  A.iss = iss;
  A.nf = nf;
  A.dtype = dtype;
  for (int f = 0; f < nf; f++) {
    A.in_bytes[f] = in_bytes[f];
    A.xo[f] = xo[f];
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMemset2DAsync(ws0, (size_t)wss, 0, kStatusBytes, (size_t)nf, stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  {
    PROF_SCOPE("k_dec_prep", stream);
    k_dec_prep<<<dim3(2, nf), 1024, 0, stream>>>(A);
  }
  // group counts depend on the streams' chunk sizes: size the decoder for the
  // smallest chunk and let warps stride over the groups that exist
  const int64_t max_g1 = ngroups(pv.n_g, 1), max_g2 = ngroups(pv.n_v, 1);
  const unsigned int cap =  // one wave of resident blocks
      (unsigned int)((sms * kDecBlocksPerSM + nf - 1) / nf);
  const unsigned int nb1 = nblk(max_g1, kDecWarps) < cap ? nblk(max_g1, kDecWarps) : cap;
  const unsigned int nb2 = nblk(max_g2, kDecWarps) < cap ? nblk(max_g2, kDecWarps) : cap;
  const size_t dsm =  // [warps][round][32]
      (size_t)kDecWarps * kDecRound * 32 * sizeof(unsigned short);
  {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_dec_syms<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
      cudaFuncSetAttribute(k_dec_syms<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
      attr = true;
    }
  }
  // Two streams (Algorithm 4 decodes the components independently): the
  // residual component's symbols on the plan's second stream, beside the
  // grid component's decoding and prefix sums on the caller's; they join
  // before the reconstruction, which needs both.
  // (single fields only: in a batch every launch already fills the GPU, and
  // the measured batched rate drops with the fork)
  const bool fork = pv.side != nullptr && pv.dim != 1 && nf == 1;
  std::unique_lock<std::mutex> lock;
  const cudaStream_t side = (cudaStream_t)pv.side;
  if (fork) {
    lock = std::unique_lock<std::mutex>(*(std::mutex *)pv.mu);
    if (cudaEventRecord((cudaEvent_t)pv.ev_fork, stream) != cudaSuccess ||
        cudaStreamWaitEvent(side, (cudaEvent_t)pv.ev_fork, 0) != cudaSuccess)
      return MCC_ERR_CUDA;
    {
      PROF_SCOPE("k_dec_syms_res", side);  // blocks of the residual component only (nb1 = 0)
      if (dtype == MCC_F64) launch_pdl(k_dec_syms<double>, dim3(nb2, nf), dim3(32 * kDecWarps), dsm, side, A, 0);
      else launch_pdl(k_dec_syms<float>, dim3(nb2, nf), dim3(32 * kDecWarps), dsm, side, A, 0);
    }
    if (cudaEventRecord((cudaEvent_t)pv.ev_join, side) != cudaSuccess) return MCC_ERR_CUDA;
  }
  {
    PROF_SCOPE("k_dec_syms", stream);
    const unsigned int nb = fork ? nb1 : nb1 + nb2;
    if (dtype == MCC_F64)
      launch_pdl(k_dec_syms<double>, dim3(nb, nf), dim3(32 * kDecWarps), dsm, stream, A, (int)nb1);
    else
      launch_pdl(k_dec_syms<float>, dim3(nb, nf), dim3(32 * kDecWarps), dsm, stream, A, (int)nb1);
  }
  if (pv.dim == 1) {  // the 1D coder
    const int64_t nchunk = (pv.n_g + kScan1dChunk - 1) / kScan1dChunk;
    const unsigned int cb = (unsigned int)(nchunk < 65535 ? nchunk : 65535);
    {
      PROF_SCOPE("k_scan1d_sums", stream);
      launch_pdl(k_scan1d_sums, dim3(cb, nf), dim3(256), 0, stream, A);
    }
    {
      PROF_SCOPE("k_scan1d_top", stream);
      launch_pdl(k_scan1d_top, dim3(1, nf), dim3(1024), 0, stream, A);
    }
    {
      PROF_SCOPE("k_recon1d", stream);
      if (dtype == MCC_F64) launch_pdl(k_recon1d<double>, dim3(cb, nf), dim3(256), 0, stream, A);
      else launch_pdl(k_recon1d<float>, dim3(cb, nf), dim3(256), 0, stream, A);
    }
    return cudaGetLastError() == cudaSuccess ? MCC_OK : MCC_ERR_CUDA;
  }
  // 3D grids with rows of at most 1024 codes (a multiple of 4): x and y in
  // one pass per z-plane, then z; otherwise rows, then y (and z)
  const bool xy = pv.dim == 3 && (pv.nx & 3) == 0 && pv.nx <= 1024;
  if (xy) {
    PROF_SCOPE("k_scan_xy", stream);
    const dim3 g((unsigned int)pv.nz, nf);
    if (pv.nx <= 256) {
      launch_pdl(k_scan_xy<1, kScanRB>, g, dim3(32 * kScanRB),
                 (size_t)(kScanRB + 1) * pv.nx * sizeof(unsigned int), stream, A);
    } else {
      const size_t sm = (size_t)9 * pv.nx * sizeof(unsigned int);
      if (pv.nx <= 512) launch_pdl(k_scan_xy<2, 8>, g, dim3(256), sm, stream, A);
      else {
        static bool attr = false;  // 36 KB of shared memory
        if (!attr) {
          cudaFuncSetAttribute(k_scan_xy<4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024);
          attr = true;
        }
        launch_pdl(k_scan_xy<4, 8>, g, dim3(256), sm, stream, A);
      }
    }
  } else {
    PROF_SCOPE("k_scan_rows", stream);
    const int64_t nrows = (int64_t)pv.ny * pv.nz;
    launch_pdl(k_scan_rows, dim3(nblk(nrows, 8), nf), dim3(256), 0, stream, A);
  }
  // scans along y (columns (x, z), stride nx) and, in 3D, z (columns (x, y),
  // stride nx ny); 32 warps per column block when the blocks are few
  auto scan_axis = [&](int64_t n_inner, int64_t n_outer, int64_t plane, int L, int64_t S) {
    PROF_SCOPE("k_scan_axis", stream);
    const int64_t blocks = (n_inner + 31) / 32 * n_outer;
    if (blocks < 4 * (int64_t)sms)
      launch_pdl(k_scan_axis<32>, dim3((unsigned int)blocks, nf), dim3(1024), 0, stream, A, n_inner,
                 n_outer, plane, L, S);
    else
      launch_pdl(k_scan_axis<8>, dim3((unsigned int)blocks, nf), dim3(256), 0, stream, A, n_inner,
                 n_outer, plane, L, S);
  };
  if (!xy) scan_axis((int64_t)pv.nx, (int64_t)pv.nz, (int64_t)pv.nx * pv.ny, pv.ny, (int64_t)pv.nx);
  if (pv.dim == 3) {
    const int64_t ninner = (int64_t)pv.nx * pv.ny;
    scan_axis(ninner, 1, 0, pv.nz, ninner);
  }
  {  // learned corrections (the kernel returns at once for plain streams)
    PROF_SCOPE("k_predict", stream);
    PredArgs P;
    memset(&P, 0, sizeof(P));
    P.pv = pv;
    P.nf = nf;
    P.bad_model_err = MCC_ERR_CORRUPT;
    const DecompressWs W = A.W;
    for (int f = 0; f < nf; f++) {
      unsigned char *ws = ws0 + (int64_t)f * wss;
      const DecInfo *info = (const DecInfo *)(ws + W.info);
      P.q1[f] = (const int *)(ws + W.q1);
      P.p[f] = (float *)(ws + W.p);
      P.model[f] = in0 + (int64_t)f * iss;
      P.model_off[f] = &info->L.model;
      P.use[f] = &info->use_model;
      P.rho12_f[f] = &info->rho12_f;
      P.qhi[f] = &info->Qhi;
      P.st[f] = (Status *)ws;
    }
    launch_predict(P, stream, true);
  }
  if (fork && cudaStreamWaitEvent(stream, (cudaEvent_t)pv.ev_join, 0) != cudaSuccess)
    return MCC_ERR_CUDA;
  {
    PROF_SCOPE("k_recon", stream);
    // one full wave of resident blocks by default (the plan's tuning may set
    // the blocks per SM)
#define MCC_RECON(K) \
  launch_pdl(K, dim3(nf, wave_blocks(K, 256, 0, pv.vbps, sms, nf)), dim3(256), 0, stream, A)
    if (pv.dim == 2) {
      if (dtype == MCC_F64) MCC_RECON((k_recon<2, double, 2>));
      else MCC_RECON((k_recon<2, float, 2>));
    } else {
      if (dtype == MCC_F64) MCC_RECON((k_recon<3, double, 1>));
      else MCC_RECON((k_recon<3, float, 1>));
    }
#undef MCC_RECON
  }
  if (cudaGetLastError() != cudaSuccess) return MCC_ERR_CUDA;
  return MCC_OK;
}

mcc_status launch_decompress(const PlanView &pv, const unsigned char *in, size_t in_bytes,
                             void *d_values, int dtype, unsigned char *ws, cudaStream_t stream) {
  const uint64_t nb[1] = {in_bytes};
  void *xo[1] = {d_values};
  return launch_decompress_batch(pv, 1, in, 0, nb, xo, dtype, ws,
                                 (int64_t)decompress_ws_layout(pv).total, stream);
}
