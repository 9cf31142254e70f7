// graph.cu -- executable CUDA graphs of the library's asynchronous calls.
//
// A batch of many variables and timesteps on one plan is a fixed sequence of
// launches (the batched compressor and decompressor, every kernel carrying a
// field dimension); mcc_graph_begin / mcc_graph_end record the calls a caller
// makes in between on one stream (with sync = 0 and no size read-back) and
// instantiate them once, and mcc_graph_launch replays the whole batch as one
// graph launch. The plan's second stream, when a call forks onto it, joins
// the capture through its events and is joined back before the call returns.
#include <cuda_runtime.h>

#include <new>

#include "common.cuh"

struct mcc_graph_s {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};

extern "C" mcc_status mcc_graph_begin(mcc_stream s) {
  cudaStream_t stream = (cudaStream_t)s;
  if (!stream) return MCC_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return MCC_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return MCC_ERR_INVALID_ARG;  // no nested capture
  return cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess
             ? MCC_OK
             : MCC_ERR_CUDA;
}

extern "C" mcc_status mcc_graph_end(mcc_stream s, mcc_graph *out) {
  cudaStream_t stream = (cudaStream_t)s;
  if (!out) return MCC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!stream) return MCC_ERR_INVALID_ARG;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return MCC_ERR_CUDA;
  if (cs == cudaStreamCaptureStatusNone) return MCC_ERR_INVALID_ARG;  // no capture to end
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(stream, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return MCC_ERR_CUDA;  // the capture was invalidated (e.g. a synchronising call inside it)
  }
  cudaGraphExec_t e = nullptr;
  if (cudaGraphInstantiate(&e, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    cudaGetLastError();
    return MCC_ERR_CUDA;
  }
  mcc_graph_s *G = new (std::nothrow) mcc_graph_s{g, e};
  if (!G) {
    cudaGraphExecDestroy(e);
    cudaGraphDestroy(g);
    return MCC_ERR_OOM;
  }
  *out = G;
  return MCC_OK;
}

extern "C" mcc_status mcc_graph_launch(mcc_graph g, mcc_stream s) {
  if (!g) return MCC_ERR_INVALID_ARG;
  return cudaGraphLaunch(g->exec, (cudaStream_t)s) == cudaSuccess ? MCC_OK : MCC_ERR_CUDA;
}

extern "C" void mcc_graph_destroy(mcc_graph g) {
  if (!g) return;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
}
