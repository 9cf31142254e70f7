// static_ws.cu -- decompression for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a memory
// budget that another allocator owns (a framework's caching allocator, an
// I/O plugin handed only the buffers it reads and writes), or code on a path
// where a device allocation would synchronise the device or fail under
// memory pressure. mcc_decompress_static gives them decompression with the
// scratch memory taken from a fixed array that is part of this library's
// device image, so the call itself allocates nothing.
//
// The array is file-scope and static, kStaticScratchBytes long: every GPU that
// loads the library holds it until the process exits. Every call on a device
// shares that device's array and leaves its contents behind; calls whose GPU
// work overlaps (two streams, or two host threads) race on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "workspace.cuh"

using namespace mcc;

namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB per device

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch in the current context. In host code g_scratch
// names a host-side stand-in, not memory the GPU can use, so the address is
// looked up with the caller's device current -- on every call, not cached: a
// context torn down and created again (cudaDeviceReset, another primary
// context) maps the array at a new address, and a cached one would be stale.
// The lookup allocates nothing; the first one on a device may load the
// library's device code.
mcc_status scratch_address(void **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MCC_ERR_CUDA;
  *out = p;
  return MCC_OK;
}

}  // namespace

extern "C" size_t mcc_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" mcc_status mcc_decompress_static(mcc_plan plan, const void *d_in, size_t in_bytes,
                                            void *d_values, int dtype, int sync,
                                            mcc_stream stream_) {
  if (!plan || !d_in || !d_values) return MCC_ERR_INVALID_ARG;
  if (dtype != MCC_F64 && dtype != MCC_F32) return MCC_ERR_INVALID_ARG;
  if (((uintptr_t)d_in & 3) || ((uintptr_t)d_values & (dtype == MCC_F64 ? 7 : 3)))
    return MCC_ERR_INVALID_ARG;
  const PlanView pv = mcc_plan_view(plan);
  if (decompress_ws_layout(pv).total > kStaticScratchBytes) return MCC_ERR_CAPACITY;
  void *ws = nullptr;
  const mcc_status s = scratch_address(&ws);
  if (s) return s;
  cudaStream_t stream = (cudaStream_t)stream_;
  // the launcher clears the status block itself; every other scratch byte is
  // written before it is read
  const mcc_status st = launch_decompress(pv, (const unsigned char *)d_in, in_bytes, d_values, dtype,
                                          (unsigned char *)ws, stream);
  if (st || !sync) return st;
  Status h;
  if (cudaMemcpyAsync(&h, ws, sizeof(Status), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return MCC_ERR_CUDA;
  return (mcc_status)h.err;
}
