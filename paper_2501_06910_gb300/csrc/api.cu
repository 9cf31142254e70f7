// api.cu -- the C ABI entry points of include/mcc.h that are not the plan.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

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
  const Layout L = make_layout(p->R1, p->R2, ng1, ng2, (uint64_t)pv.n_g, 0, (uint64_t)pv.n_v, vsz, w1, w2);
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
