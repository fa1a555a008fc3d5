// Host/device interface of the tensor-core convolution kernels (internal).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

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

// Padded BF16 activations are stored chunk-planar: channels in groups of 8
// (16 bytes), each group a full padded volume,
//   element (X, Y, Z, c) at (((Z * C/8 + c/8) * py + Y) * px + X) * 8 + c % 8,
// with px = nx + 2, py = ny + 2 and one ghost layer per face holding periodic
// images.  A run of consecutive sites of one group is contiguous memory.
__host__ __device__ inline long long act_off(int X, int Y, int Z, int group, int C, int px, int py) {
  return ((((long long)Z * (C / 8) + group) * py + Y) * px + X) * 8;
}
// bytes allocated after the last group of a buffer, which the window kernel's
// last copies may read past (into nothing it uses)
constexpr size_t kActTailBytes = 64 * 1024;

// geometry of the window kernel (host-computed)
struct ConvWin {
  int px, py;          // padded plane extents
  int l_first;         // linear index of the first interior site in a padded plane
  int ntiles;          // 128-row tiles covering the interior rows of a plane
  int wb;              // sites copied per channel group and plane (window, rounded up to 8)
  uint32_t lbo;        // bytes between channel groups of a staged plane (= wb * 16)
  uint32_t slot_bytes; // bytes of one staged plane
  uint32_t off_w, off_bars;
};

// one padded BF16 activation buffer: the per-tap kernel's tensor map (4-D
// view (8 px, py, C/8, pz), boxes of 32 sites x 4 rows of one group) and the
// raw pointer the window kernel copies from
struct ConvMaps {
  CUtensorMap tile;
  const void* base;
  bool use_win;
};

// window geometry for C_in, C_out on an nx x ny plane; false if it does not fit
bool conv_win_geometry(int cin, int cout, int nx, int ny, ConvWin* g, size_t* smem_bytes);

// y = conv(x) on tcgen05; m describes the padded BF16 input, tmW the BF16
// weights [27][C_out][C_in] (one box of all taps), sms the device's SM count.
// The window kernel runs where allowed, m.use_win is set and the geometry
// fits; the per-tap kernel otherwise.
cudaError_t conv_launch(int cin, int cout, int epi, const ConvMaps& m, bool allow_win, const CUtensorMap& tmW,
                        const ConvArgs& a, int sms, cudaStream_t s);

// Weight and bias gradients of one convolution on tcgen05 (dw.cu):
// dW[t][ci][co] += sum_r X(r + o_t)[ci] dY(r)[co], db[co] += sum_r dY(r)[co]
// over the interior sites, X and dY padded BF16 (C_in, C_out in {16, 32}),
// deterministic.  partial: dw_partial_floats(sms) floats of scratch.
// dw_fits: whether the staged plane windows fit shared memory (planes up to
// about 139 sites wide); otherwise the caller takes another kernel.
size_t dw_partial_floats(int sms);
bool dw_fits(int cin, int cout, int nx, int ny, int nz);
cudaError_t dw_launch(int cin, int cout, const __nv_bfloat16* X, const __nv_bfloat16* dY, int nx, int ny, int nz,
                      float* partial, float* dW, float* db, int* err, int sms, cudaStream_t s);

}  // namespace lcbp
