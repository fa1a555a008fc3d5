// Host/device interface of the tensor-core convolution kernels (internal).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace lcbp {

// epilogue flags
enum : int {
  kEpiBias = 1,      // + bias[c]
  kEpiRelu = 2,      // max(0, .)
  kEpiResid = 4,     // + resid (BF16, same padded layout as the output)
  kEpiMask = 8,      // * (mask > 0) with mask BF16 in the padded layout (ReLU backward)
  kEpiOutF32 = 16,   // write FP32 [site][C_out] (unpadded) instead of BF16
  kEpiUpdateQ = 32,  // Q[c][site] += qscale * value + rate_scale * rate[c][site], c < 5 (FP32 SoA)
};

struct ConvArgs {
  int nx, ny, nz;
  long long n;  // nx * ny * nz
  const float* bias;
  const __nv_bfloat16* resid;
  const __nv_bfloat16* mask;
  __nv_bfloat16* out_bf16;  // padded [nz+2][ny+2][nx+2][C_out]
  float* out_f32;           // [n][C_out]
  float* qstate;            // [5][n]
  float qscale;
  const float* rate;        // [5][n]: kEpiUpdateQ adds rate_scale * rate too
  float rate_scale;
  int* err;
};

// y = conv(x) on tcgen05; tmA describes the padded BF16 input (box C_in x 32 x 4 x 1,
// swizzled), tmW the BF16 weights [27][C_out][C_in] (one box of all taps)
cudaError_t conv_launch(int cin, int cout, int epi, const CUtensorMap& tmA, const CUtensorMap& tmW,
                        const ConvArgs& a, int max_ctas, cudaStream_t s);

}  // namespace lcbp
