// api.cu -- the C ABI entry points of include/mcc.h that are not the plan.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "common.cuh"
#include "workspace.cuh"

using namespace mcc;

extern "C" void mcc_params_default(mcc_params *p) {
  if (!p) return;
  p->dtype = MCC_F64;
  p->eb_mode = MCC_REL;
  p->eb = 1e-4;
  p->grid_fraction = 0.5;
  p->R1 = 512;
  p->R2 = 512;
  p->C1 = 128;
  p->C2 = 128;
  p->lmax = 24;
  p->predictor = MCC_PRED_ZERO;
  p->d_model = nullptr;
  p->loop = MCC_LOOP_CLOSED;
  p->f_op = MCC_F_BARYCENTRIC;
  p->g_op = MCC_G_MULTILINEAR;
  p->zero_run = 0;
}

extern "C" const char *mcc_status_string(mcc_status s) {
  switch (s) {
    case MCC_OK: return "ok";
    case MCC_ERR_INVALID_ARG: return "invalid argument";
    case MCC_ERR_CUDA: return "CUDA error";
    case MCC_ERR_OOM: return "out of device memory";
    case MCC_ERR_RANGE: return "error bound too small for the value range";
    case MCC_ERR_CORRUPT: return "corrupt or mismatched stream";
    case MCC_ERR_CAPACITY: return "buffer too small";
    case MCC_ERR_TIMEOUT: return "device wait timed out";
    case MCC_ERR_UNSUPPORTED: return "unsupported parameter";
  }
  return "unknown status";
}

extern "C" mcc_status mcc_workspace_size(mcc_plan plan, const mcc_params *p, size_t *cbytes,
                                         size_t *dbytes) {
  if (!plan) return MCC_ERR_INVALID_ARG;
  const PlanView pv = mcc_plan_view(plan);
  if (cbytes) {
    const mcc_status s = check_params(p);
    if (s) return s;
    *cbytes = compress_ws_layout(pv, p).total;
  }
  if (dbytes) *dbytes = decompress_ws_layout(pv).total;
  return MCC_OK;
}

extern "C" mcc_status mcc_compress_bound(mcc_plan plan, const mcc_params *p, size_t *max_bytes) {
  if (!plan || !max_bytes) return MCC_ERR_INVALID_ARG;
  const mcc_status s = check_params(p);
  if (s) return s;
  const PlanView pv = mcc_plan_view(plan);
  const int64_t ng1 = ngroups(pv.n_g, p->C1), ng2 = ngroups(pv.n_v, p->C2);
  const uint64_t vsz = p->dtype == MCC_F64 ? 8 : 4;
  const uint64_t w1 = (uint64_t)((pv.n_g * p->lmax + 31) / 32 + ng1);
  const uint64_t w2 = (uint64_t)((pv.n_v * p->lmax + 31) / 32 + ng2);
  const Layout L = make_layout(p->R1, p->R2, ng1, ng2, (uint64_t)pv.n_g, 0, (uint64_t)pv.n_v, vsz,
                               w1, w2, kModelBytes);  // room for a learned-predictor blob
  *max_bytes = L.total + 16;
  return MCC_OK;
}

static mcc_status read_status(const void *ws, cudaStream_t stream, size_t *out_size) {
  Status h;
  if (cudaMemcpyAsync(&h, ws, sizeof(Status), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  if (out_size) *out_size = (size_t)h.out_size;
  return (mcc_status)h.err;
}

extern "C" mcc_status mcc_workspace_result(const void *d_workspace, mcc_stream stream, size_t *out_size) {
  if (!d_workspace) return MCC_ERR_INVALID_ARG;
  return read_status(d_workspace, (cudaStream_t)stream, out_size);
}

extern "C" mcc_status mcc_compress(mcc_plan plan, const void *d_values, const mcc_params *p,
                                   void *d_ws, size_t ws_bytes, void *d_out, size_t capacity,
                                   size_t *out_size, mcc_stream s) {
  if (!plan || !d_values || !d_ws || !d_out) return MCC_ERR_INVALID_ARG;
  mcc_status st = check_params(p);
  if (st) return st;
  if (((uintptr_t)d_out & 7) || ((uintptr_t)d_ws & 255) ||
      ((uintptr_t)d_values & (p->dtype == MCC_F64 ? 7 : 3)))
    return MCC_ERR_INVALID_ARG;
  const PlanView pv = mcc_plan_view(plan);
  if (ws_bytes < compress_ws_layout(pv, p).total) return MCC_ERR_CAPACITY;
  cudaStream_t stream = (cudaStream_t)s;
  st = launch_compress(pv, d_values, p, (unsigned char *)d_ws, (unsigned char *)d_out, capacity, stream);
  if (st) return st;
  if (out_size) return read_status(d_ws, stream, out_size);
  return MCC_OK;
}

extern "C" mcc_status mcc_decompress(mcc_plan plan, const void *d_in, size_t in_bytes, void *d_values,
                                     int dtype, void *d_ws, size_t ws_bytes, int sync, mcc_stream s) {
  if (!plan || !d_in || !d_values || !d_ws) return MCC_ERR_INVALID_ARG;
  if (dtype != MCC_F64 && dtype != MCC_F32) return MCC_ERR_INVALID_ARG;
  if (((uintptr_t)d_in & 3) || ((uintptr_t)d_ws & 255) ||
      ((uintptr_t)d_values & (dtype == MCC_F64 ? 7 : 3)))
    return MCC_ERR_INVALID_ARG;
  const PlanView pv = mcc_plan_view(plan);
  if (ws_bytes < decompress_ws_layout(pv).total) return MCC_ERR_CAPACITY;
  cudaStream_t stream = (cudaStream_t)s;
  const mcc_status st = launch_decompress(pv, (const unsigned char *)d_in, in_bytes, d_values, dtype,
                                          (unsigned char *)d_ws, stream);
  if (st) return st;
  if (sync) return read_status(d_ws, stream, nullptr);
  return MCC_OK;
}

// ---------------------------------------------------------------------------
// batched forms
// ---------------------------------------------------------------------------
static mcc_status read_batch_status(const unsigned char *ws0, size_t wss, int n, cudaStream_t stream,
                                    size_t *sizes) {
  Status *h = new (std::nothrow) Status[n];
  if (!h) return MCC_ERR_OOM;
  mcc_status r = MCC_OK;
  if (cudaMemcpy2DAsync(h, sizeof(Status), ws0, wss, sizeof(Status), (size_t)n,
                        cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    r = MCC_ERR_CUDA;
  } else {
    for (int f = 0; f < n; f++) {
      if (sizes) sizes[f] = (size_t)h[f].out_size;
      if (r == MCC_OK && h[f].err) r = (mcc_status)h[f].err;
    }
  }
  delete[] h;
  return r;
}

// Fields per batched launch chain: the plan's tuning, or as many fields as
// keep their gathered codes (q1 and Q, 4 (n_g + n_v) bytes each) within half
// of the L2 cache -- a chain's kernels run over all its fields at once, and
// the vertex and grid kernels gather those codes at random places.
static int chain_fields(const PlanView &pv) {
  if (pv.batch_fields > 0) return pv.batch_fields;
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0)
    l2 = 64 << 20;
  const int64_t per = 4 * (pv.n_g + pv.n_v);
  const int64_t k = ((int64_t)l2 / 2) / (per > 0 ? per : 1);
  return (int)(k < 1 ? 1 : (k > kMaxBatch ? kMaxBatch : k));
}

extern "C" mcc_status mcc_compress_batch(mcc_plan plan, int n, const void *const *d_values,
                                         const mcc_params *per_field, void *d_ws, size_t ws_bytes,
                                         void *d_out, size_t slot_bytes, size_t *out_sizes,
                                         mcc_stream s) {
  if (!plan || n < 1 || !d_values || !per_field || !d_ws || !d_out) return MCC_ERR_INVALID_ARG;
  const mcc_params *p0 = per_field;
  for (int f = 0; f < n; f++) {
    const mcc_status st = check_params(per_field + f);
    if (st) return st;
    const mcc_params *p = per_field + f;
    if (p->dtype != p0->dtype || p->R1 != p0->R1 || p->R2 != p0->R2 || p->C1 != p0->C1 ||
        p->C2 != p0->C2 || p->lmax != p0->lmax)
      return MCC_ERR_INVALID_ARG;
    if (!d_values[f] || ((uintptr_t)d_values[f] & (p->dtype == MCC_F64 ? 7 : 3)))
      return MCC_ERR_INVALID_ARG;
  }
  if (((uintptr_t)d_out & 7) || (slot_bytes & 7) || ((uintptr_t)d_ws & 255)) return MCC_ERR_INVALID_ARG;
  const PlanView pv = mcc_plan_view(plan);
  const size_t wss = compress_ws_layout(pv, p0).total;
  int chain = (int)(ws_bytes / wss);
  if (chain < 1) return MCC_ERR_CAPACITY;
  if (chain > kMaxBatch) chain = kMaxBatch;
  if (chain > chain_fields(pv)) chain = chain_fields(pv);
  cudaStream_t stream = (cudaStream_t)s;
  unsigned char *out = (unsigned char *)d_out;
  for (int f0 = 0; f0 < n; f0 += chain) {
    const int nf = n - f0 < chain ? n - f0 : chain;
    const mcc_status st = launch_compress_batch(pv, nf, d_values + f0, per_field + f0,
                                                (unsigned char *)d_ws, (int64_t)wss,
                                                out + (size_t)f0 * slot_bytes, (int64_t)slot_bytes,
                                                slot_bytes, stream);
    if (st) return st;
    if (out_sizes) {
      const mcc_status r = read_batch_status((const unsigned char *)d_ws, wss, nf, stream, out_sizes + f0);
      if (r) return r;
    }
  }
  return MCC_OK;
}

extern "C" mcc_status mcc_decompress_batch(mcc_plan plan, int n, const void *d_in, size_t slot_bytes,
                                           const size_t *in_bytes, void *const *d_values, int dtype,
                                           void *d_ws, size_t ws_bytes, int sync, mcc_stream s) {
  if (!plan || n < 1 || !d_in || !in_bytes || !d_values || !d_ws) return MCC_ERR_INVALID_ARG;
  if (dtype != MCC_F64 && dtype != MCC_F32) return MCC_ERR_INVALID_ARG;
  if (((uintptr_t)d_in & 7) || (slot_bytes & 7) || ((uintptr_t)d_ws & 255)) return MCC_ERR_INVALID_ARG;
  for (int f = 0; f < n; f++)
    if (!d_values[f] || ((uintptr_t)d_values[f] & (dtype == MCC_F64 ? 7 : 3)) || in_bytes[f] > slot_bytes)
      return MCC_ERR_INVALID_ARG;
  const PlanView pv = mcc_plan_view(plan);
  const size_t wss = decompress_ws_layout(pv).total;
  int chain = (int)(ws_bytes / wss);
  if (chain < 1) return MCC_ERR_CAPACITY;
  if (chain > kMaxBatch) chain = kMaxBatch;
  if (chain > chain_fields(pv)) chain = chain_fields(pv);
  cudaStream_t stream = (cudaStream_t)s;
  for (int f0 = 0; f0 < n; f0 += chain) {
    const int nf = n - f0 < chain ? n - f0 : chain;
    uint64_t nb[kMaxBatch];
    for (int f = 0; f < nf; f++) nb[f] = in_bytes[f0 + f];
    const mcc_status st = launch_decompress_batch(
        pv, nf, (const unsigned char *)d_in + (size_t)f0 * slot_bytes, (int64_t)slot_bytes, nb,
        d_values + f0, dtype, (unsigned char *)d_ws, (int64_t)wss, stream);
    if (st) return st;
    if (sync) {
      const mcc_status r = read_batch_status((const unsigned char *)d_ws, wss, nf, stream, nullptr);
      if (r) return r;
    }
  }
  return MCC_OK;
}

// ---------------------------------------------------------------------------
// the paper's default baseline: the 1D coder on the vertex array
// ---------------------------------------------------------------------------
static PlanView plan_view_1d(int64_t n) {
  PlanView pv;
  memset(&pv, 0, sizeof(pv));
  pv.dim = 1;
  pv.nx = (int32_t)n;
  pv.ny = pv.nz = 1;
  pv.n_v = pv.n_g = n;
  return pv;
}

static mcc_status check_1d(int64_t n, const mcc_params *p) {
  if (n < 1 || n >= ((int64_t)1 << 31)) return MCC_ERR_INVALID_ARG;
  const mcc_status s = check_params(p);
  if (s) return s;
  if (p->predictor != MCC_PRED_ZERO || p->loop != MCC_LOOP_CLOSED ||
      p->f_op != MCC_F_BARYCENTRIC || p->g_op != MCC_G_MULTILINEAR)
    return MCC_ERR_INVALID_ARG;
  return MCC_OK;
}

extern "C" mcc_status mcc_workspace_size_1d(int64_t n, const mcc_params *p, size_t *cbytes,
                                            size_t *dbytes) {
  const mcc_status s = check_1d(n, p);
  if (s) return s;
  const PlanView pv = plan_view_1d(n);
  if (cbytes) *cbytes = compress_ws_layout(pv, p).total;
  if (dbytes) *dbytes = decompress_ws_layout(pv).total;
  return MCC_OK;
}

extern "C" mcc_status mcc_compress_bound_1d(int64_t n, const mcc_params *p, size_t *max_bytes) {
  if (!max_bytes) return MCC_ERR_INVALID_ARG;
  const mcc_status s = check_1d(n, p);
  if (s) return s;
  const int64_t ng1 = ngroups(n, p->C1);
  const uint64_t w1 = (uint64_t)((n * p->lmax + 31) / 32 + ng1);
  const Layout L = make_layout(p->R1, p->R2, ng1, 0, (uint64_t)n, 0, 0, 8, w1, 0, 0);
  *max_bytes = L.total + 16;
  return MCC_OK;
}

extern "C" mcc_status mcc_compress_1d(const void *d_values, int64_t n, const mcc_params *p,
                                      void *d_ws, size_t ws_bytes, void *d_out, size_t capacity,
                                      size_t *out_size, mcc_stream s) {
  if (!d_values || !d_ws || !d_out) return MCC_ERR_INVALID_ARG;
  mcc_status st = check_1d(n, p);
  if (st) return st;
  if (((uintptr_t)d_out & 7) || ((uintptr_t)d_ws & 255) ||
      ((uintptr_t)d_values & (p->dtype == MCC_F64 ? 7 : 3)))
    return MCC_ERR_INVALID_ARG;
  const PlanView pv = plan_view_1d(n);
  if (ws_bytes < compress_ws_layout(pv, p).total) return MCC_ERR_CAPACITY;
  cudaStream_t stream = (cudaStream_t)s;
  st = launch_compress(pv, d_values, p, (unsigned char *)d_ws, (unsigned char *)d_out, capacity, stream);
  if (st) return st;
  if (out_size) return read_status(d_ws, stream, out_size);
  return MCC_OK;
}

extern "C" mcc_status mcc_decompress_1d(const void *d_in, size_t in_bytes, void *d_values, int64_t n,
                                        int dtype, void *d_ws, size_t ws_bytes, int sync,
                                        mcc_stream s) {
  if (!d_in || !d_values || !d_ws) return MCC_ERR_INVALID_ARG;
  if (n < 1 || n >= ((int64_t)1 << 31)) return MCC_ERR_INVALID_ARG;
  if (dtype != MCC_F64 && dtype != MCC_F32) return MCC_ERR_INVALID_ARG;
  if (((uintptr_t)d_in & 3) || ((uintptr_t)d_ws & 255) ||
      ((uintptr_t)d_values & (dtype == MCC_F64 ? 7 : 3)))
    return MCC_ERR_INVALID_ARG;
  const PlanView pv = plan_view_1d(n);
  if (ws_bytes < decompress_ws_layout(pv).total) return MCC_ERR_CAPACITY;
  cudaStream_t stream = (cudaStream_t)s;
  const mcc_status st = launch_decompress(pv, (const unsigned char *)d_in, in_bytes, d_values, dtype,
                                          (unsigned char *)d_ws, stream);
  if (st) return st;
  if (sync) return read_status(d_ws, stream, nullptr);
  return MCC_OK;
}
