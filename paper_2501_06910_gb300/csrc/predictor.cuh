// predictor.cuh -- the learned residual predictor (the network's definition
// shared by the inference and training kernels).
//
// Model blob (little endian, kModelBytes): magic 'MCCM', version 1, dim, n_in,
// sx, s1, s2, e3 (int32), W1 int8 [64][16], W2 int8 [64][64], W3 int8 [64],
// b1 int32 [64], b2 int32 [64], b3 int32.
//
// Inference is integer exact: features e_k = (c_k - c_000) * (s1/s2) * 2^-sx
// rounded to [-127, 127] (k = 1 .. 2^dim - 1), the local coordinates
// rounded to 0..127 and the level c_000 (s1/s2) / Qhi as a fraction of the
// value range rounded to 0..127 (Qhi the field's largest vertex code);
// h1 = act(W1 x + b1, s1), h2 = act(W2 h1 + b2, s2) with
// act(a, s) = clamp(round_half_up(a / 2^s), 0, 255); p = (W3 h2 + b3) 2^e3.
// |sums| < 2^24, so bf16 tensor-core products summed in FP32 are exact in any
// order and the decoder reproduces p bit for bit.
#pragma once

#include "common.cuh"

namespace mcc {

constexpr uint32_t kModelMagic = 0x4D43434Du;  // 'M' 'C' 'C' 'M'
constexpr int kH = 64;  // hidden units
constexpr int kK = 16;  // padded input width
enum : uint32_t {
  M_MAGIC = 0, M_VERSION = 4, M_DIM = 8, M_NIN = 12, M_SX = 16, M_S1 = 20, M_S2 = 24, M_E3 = 28,
  M_W1 = 32, M_W2 = 1056, M_W3 = 5152, M_B1 = 5216, M_B2 = 5472, M_B3 = 5728
};
static_assert(M_B3 + 8 == kModelBytes, "model layout");

// Arguments of one predictor launch, per field: the grid codes, the output
// corrections, the model blob (at model[f] + *model_off[f] when model_off[f]
// is set; NULL skips the field), an optional switch (*use[f] == 0 skips the
// field), the locations of s1/s2 in FP32 and of Qhi, and the status block.
struct PredArgs {
  PlanView pv;
  int nf;
  unsigned int bad_model_err;  // status recorded for an invalid blob
  const int *q1[kMaxBatch];
  float *p[kMaxBatch];
  const unsigned char *model[kMaxBatch];
  const uint64_t *model_off[kMaxBatch];
  const int *use[kMaxBatch];
  const float *rho12_f[kMaxBatch];
  const long long *qhi[kMaxBatch];
  Status *st[kMaxBatch];
};

}  // namespace mcc

// Launch the predictor for A.nf fields (dim 2 or 3), optionally with
// programmatic dependent launch.
cudaError_t launch_predict(const mcc::PredArgs &A, cudaStream_t stream, bool pdl);
