// Learned surrogate: a periodic 3x3x3 convolutional network that advances Q by
// k = 10 solver steps, with BF16 tensor-core forward, backward-data (conv.cu)
// and weight-gradient (dw.cu) passes, masked-MSE loss and Adam, all on device.
//
// Network (channels-last BF16 activations, FP32 accumulate):
//   x = [Q_xx Q_xy Q_xz Q_yy Q_yz, u / s_u, kappa - 1, tau, R / s_r]   (15 of 16 channels)
//   h0 = relu(conv_in x);  4 x { a = relu(conv_a h);  h = h + conv_b a };
//   y = conv_out h (5 of 16 channels);   Q(t + 10) = Q(t) + 10 R + s_dq * y
// with R = R(Q, u) the Beris-Edwards rate of the solver (Sec. 2.1 Eq.
// Qevolution, mat_der), so the network learns the correction to ten explicit
// Euler steps.
#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>

#include "../../include/lcbp.h"
#include "common.cuh"
#include "conv.h"
#include "kernels.h"
#include "runtime.h"

using namespace lcbp;

namespace lcbp {
// lattice internals needed by the surrogate step (api.cu)
int lattice_fields(lcbp_lattice* h, float** q, const float** u, int dims[3], cudaStream_t* stream);
int lattice_rate(lcbp_lattice* h, const float** rate, cudaEvent_t done);
}

namespace {

constexpr int kBlocks = 4;
constexpr int kLayers = 2 + 2 * kBlocks;
constexpr int kWidth = 32;
constexpr int kInC = 15, kOutC = 5, kPadC = 16;
constexpr int kDefaultSteps = 10;  // solver steps per call unless set otherwise

struct LayerDim {
  int cin, cout;          // true channels
  int cin_p, cout_p;      // padded to 16 / 32
};

LayerDim layer_dim(int l) {
  if (l == 0) return {kInC, kWidth, kPadC, kWidth};
  if (l == kLayers - 1) return {kWidth, kOutC, kWidth, kPadC};
  return {kWidth, kWidth, kWidth, kWidth};
}

size_t true_param_count() {
  size_t c = 0;
  for (int l = 0; l < kLayers; ++l) {
    const LayerDim d = layer_dim(l);
    c += 27 * (size_t)d.cin * d.cout + d.cout;
  }
  return c;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// network input from physical fields: Q [5][n], u [3][n], R [5][n] (FP32) -> padded BF16, 16 channels, chunk-planar
__global__ void k_sur_input(const float* __restrict__ q, const float* __restrict__ u, const float* __restrict__ r,
                            float su, float sr, float kap, float tau, int nx, int ny, int nz,
                            __nv_bfloat16* __restrict__ out) {
  const long long n = (long long)nx * ny * nz;
  const int px = nx + 2, py = ny + 2, pz = nz + 2;
  const long long np = (long long)px * py * pz;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    // padded position (X, Y, Z); 32-bit division where the padded volume allows it
    int X, Y, Z;
    if (np < (1ll << 31)) {
      const int pi = (int)p, row = pi / px;
      X = pi - row * px;
      Y = row % py;
      Z = row / py;
    } else {
      X = (int)(p % px);
      Y = (int)((p / px) % py);
      Z = (int)(p / ((long long)px * py));
    }
    const int x = X == 0 ? nx - 1 : (X > nx ? 0 : X - 1);  // periodic source
    const int y = Y == 0 ? ny - 1 : (Y > ny ? 0 : Y - 1);
    const int z = Z == 0 ? nz - 1 : (Z > nz ? 0 : Z - 1);
    const long long s = ((long long)z * ny + y) * nx + x;
    float v[16];
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c] = q[c * n + s];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[5 + c] = u ? u[c * n + s] / su : 0.f;
    v[8] = kap - 1.f;
    v[9] = tau;
#pragma unroll
    for (int c = 0; c < 5; ++c) v[10 + c] = r ? r[c * n + s] / sr : 0.f;
    v[15] = 0.f;
    uint4 pk[2];
#pragma unroll
    for (int q2 = 0; q2 < 2; ++q2) {
      __nv_bfloat16* h8 = reinterpret_cast<__nv_bfloat16*>(&pk[q2]);
#pragma unroll
      for (int j = 0; j < 8; ++j) h8[j] = __float2bfloat16_rn(v[q2 * 8 + j]);
    }
    *reinterpret_cast<uint4*>(out + act_off(X, Y, Z, 0, 16, px, py)) = pk[0];
    *reinterpret_cast<uint4*>(out + act_off(X, Y, Z, 1, 16, px, py)) = pk[1];
  }
}

// u of a lattice: rho u stored as [drho, ux, uy, uz] -> pointer to ux..uz given by caller

// masked MSE on y (FP32 [n][16], first 5 channels) against (dq - 10 R) / s_dq
// (FP32 [5][n]); writes the BF16 padded (chunk-planar) gradient d loss / d y and per-block partial sums
__global__ void k_sur_loss(const float* __restrict__ y, const float* __restrict__ target,
                           const float* __restrict__ rate, float ksteps, const float* __restrict__ mask, float inv_sdq,
                           double inv_den, int nx, int ny, int nz, __nv_bfloat16* __restrict__ grad,
                           double* __restrict__ partial) {
  const long long n = (long long)nx * ny * nz;
  const int px = nx + 2, py = ny + 2, pz = nz + 2;
  const long long np = (long long)px * py * pz;
  const float gscale = (float)(2.0 * inv_den);
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
    const int pi = (int)p, row = pi / px;  // np <= 2^31 (checked when the surrogate is made)
    const int X = pi - row * px, Y = row % py, Z = row / py;
    const int x = (X + nx - 1) % nx, yy = (Y + ny - 1) % ny, z = (Z + nz - 1) % nz;
    const long long s = ((long long)z * ny + yy) * nx + x;
    const bool interior = X >= 1 && X <= nx && Y >= 1 && Y <= ny && Z >= 1 && Z <= nz;
    const float w = mask ? mask[s] : 1.f;
    float g[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) g[c] = 0.f;
    float sq = 0.f;  // this site's w |d|^2 (FP32; the sum over sites is FP64)
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const float tc = target[c * n + s] - (rate ? ksteps * rate[c * n + s] : 0.f);
      const float d = y[s * 16 + c] - tc * inv_sdq;
      g[c] = gscale * w * d;
      sq += w * d * d;
    }
    if (interior) acc += (double)sq;
    uint4 pk[2];
#pragma unroll
    for (int q2 = 0; q2 < 2; ++q2) {
      __nv_bfloat16* h8 = reinterpret_cast<__nv_bfloat16*>(&pk[q2]);
#pragma unroll
      for (int j = 0; j < 8; ++j) h8[j] = __float2bfloat16_rn(g[q2 * 8 + j]);
    }
    *reinterpret_cast<uint4*>(grad + act_off(X, Y, Z, 0, 16, px, py)) = pk[0];
    *reinterpret_cast<uint4*>(grad + act_off(X, Y, Z, 1, 16, px, py)) = pk[1];
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// sum of nb partials times scale, by one warp in a fixed order: lane l adds
// partials l, l + 32, ... in turn, then the lanes' sums meet in a fixed tree
__global__ void k_sum(const double* __restrict__ partial, int nb, double scale, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  double s = 0;
#pragma unroll 4
  for (int i = threadIdx.x; i < nb; i += 32) s += partial[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) *out = s * scale;
}

// Weight gradient of one layer, FP32 on CUDA cores:
// dW[t][ci][co] += sum_r X(r + o_t)[ci] dY(r)[co],  db[co] += sum_r dY(r)[co]
// (padded BF16 inputs, interior sites r).  Grid: x = site chunks, y = tap.
// Each thread owns a 4 x 4 block of (ci, co).
template <int CX, int CY>
__global__ void __launch_bounds__(CX* CY / 16) k_sur_dw(const __nv_bfloat16* __restrict__ X,
                                                       const __nv_bfloat16* __restrict__ dY, int nx, int ny, int nz,
                                                       int chunk, float* __restrict__ dW, float* __restrict__ db) {
  constexpr int NT = CX * CY / 16;
  constexpr int SB = 64;  // sites staged per pass
  __shared__ float xs[SB][CX];
  __shared__ float ys[SB][CY];
  const int t = blockIdx.y;
  const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
  const long long n = (long long)nx * ny * nz;
  const int px = nx + 2, py = ny + 2;
  const int ci0 = (threadIdx.x / (CY / 4)) * 4, co0 = (threadIdx.x % (CY / 4)) * 4;
  float acc[4][4] = {};
  float bacc[4] = {};
  const long long s_begin = (long long)blockIdx.x * chunk;
  const long long s_end = s_begin + chunk < n ? s_begin + chunk : n;
  for (long long s0 = s_begin; s0 < s_end; s0 += SB) {
    __syncthreads();
    for (int e = threadIdx.x; e < SB * (CX + CY) / 8; e += NT) {
      const int row = e / ((CX + CY) / 8), part = e % ((CX + CY) / 8);
      const long long s = s0 + row;
      float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const bool inx = part < CX / 8;
      if (s < s_end) {
        const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
        const __nv_bfloat16* src;
        if (inx) src = X + act_off(x + 1 + dx, y + 1 + dy, z + 1 + dz, part, CX, px, py);
        else src = dY + act_off(x + 1, y + 1, z + 1, part - CX / 8, CY, px, py);
        const uint4 w4 = *reinterpret_cast<const uint4*>(src);
        const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&w4);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __bfloat162float(h8[j]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (inx) xs[row][part * 8 + j] = v[j];
        else ys[row][(part - CX / 8) * 8 + j] = v[j];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < SB; ++r) {
      float xv[4], yv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        xv[i] = xs[r][ci0 + i];
        yv[i] = ys[r][co0 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += xv[i] * yv[j];
      if (t == 13 && ci0 == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) bacc[j] += yv[j];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(&dW[((size_t)t * CX + ci0 + i) * CY + co0 + j], acc[i][j]);
  if (t == 13 && ci0 == 0) {
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(&db[co0 + j], bacc[j]);
  }
}

// Adam (Kingma & Ba 2015) with bias correction on FP32 master parameters
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long count, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 operand copies of one layer's FP32 master weights W[t][ci][co] (padded dims):
// forward  Wf[t][co][ci];  backward-data  Wb[26 - t][ci][co]
__global__ void k_sur_refresh(const float* __restrict__ W, int cin, int cout, __nv_bfloat16* __restrict__ Wf,
                              __nv_bfloat16* __restrict__ Wb) {
  const int total = 27 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int t = i / (cin * cout), ci = (i / cout) % cin, co = i % cout;
    const __nv_bfloat16 v = __float2bfloat16_rn(W[i]);
    Wf[((size_t)t * cout + co) * cin + ci] = v;
    if (Wb) Wb[((size_t)(26 - t) * cin + ci) * cout + co] = v;
  }
}

// master padded layout <-> true layout of the flat parameter vector
__global__ void k_sur_scatter(const float* __restrict__ src, int cin, int cout, int cin_p, int cout_p,
                              float* __restrict__ W, float* __restrict__ b, int to_padded) {
  const int nw = 27 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + cout; i += gridDim.x * blockDim.x) {
    if (i < nw) {
      const int t = i / (cin * cout), ci = (i / cout) % cin, co = i % cout;
      float* dst = &W[((size_t)t * cin_p + ci) * cout_p + co];
      if (to_padded) *dst = src[i];
      else const_cast<float*>(src)[i] = *dst;
    } else {
      const int co = i - nw;
      if (to_padded) b[co] = src[i];
      else const_cast<float*>(src)[i] = b[co];
    }
  }
}

__global__ void k_zero(float* p, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = 0.f;
}

__global__ void k_f32_soa(const float* __restrict__ y16, long long n, float* __restrict__ out5) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < 5; ++c) out5[c * n + s] = y16[s * 16 + c];
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

// padded chunk-planar activations as the 4-D tensor (8 px, py, C/8, pz): a box
// of 256 x 4 x 1 x 1 is 32 sites x 8 channels in 4 rows of one channel group
bool act_map(CUtensorMap* m, void* base, int C, int nx, int ny, int nz) {
  EncodeFn fn = encoder();
  if (!fn) return false;
  const cuuint64_t px = nx + 2, py = ny + 2, pz = nz + 2;
  const cuuint64_t dims[4] = {8 * px, py, (cuuint64_t)C / 8, pz};
  const cuuint64_t str[3] = {16 * px, 16 * px * py, 16 * px * py * (cuuint64_t)(C / 8)};
  const cuuint32_t box[4] = {256, 4, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// both views of one activation buffer; the window kernel only where its geometry fits
bool conv_maps(ConvMaps* m, void* base, int C, int nx, int ny, int nz) {
  if (!act_map(&m->tile, base, C, nx, ny, nz)) return false;
  ConvWin g;
  size_t smem = 0;
  m->base = base;
  m->use_win = conv_win_geometry(C, 32, nx, ny, &g, &smem) && conv_win_geometry(32, 16, nx, ny, &g, &smem);
  return true;
}

// weights [27][rows][K] BF16 as a 3-D tensor, one box of all taps
// Weights [27][rows][K] with tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1), viewed
// as a 4-D tensor (K, rows, dz, in-plane shift) so that the one box of all taps
// lands in shared memory shift-major: [shift][dz][rows][K].  The three z-taps of
// one in-plane shift are then adjacent, which lets one MMA with N = 2 rows
// apply two of them.
bool weight_map(CUtensorMap* m, void* base, int K, int rows) {
  EncodeFn fn = encoder();
  if (!fn) return false;
  const cuuint64_t tap = (cuuint64_t)K * 2 * rows;
  const cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, 3, 9};
  const cuuint64_t str[3] = {(cuuint64_t)K * 2, 9 * tap, tap};
  const cuuint32_t box[4] = {(cuuint32_t)K, (cuuint32_t)rows, 3, 9};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            K == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

}  // namespace

struct lcbp_surrogate {
  int nx, ny, nz;
  long long n, np;
  int training;
  int device;
  cudaStream_t stream;
  float su, sr, sdq;
  int ksteps;  // solver steps one call stands for
  int sms;
  int conv_kernel;  // LCBP_CONV_*
  bool dw_cuda_cores;  // weight gradients on the CUDA-core kernel even where the tensor-core one fits
  // parameters: FP32 master (padded) per layer, BF16 forward / backward copies
  float* master;  // all layers, padded
  size_t off_w[kLayers], off_b[kLayers];
  size_t master_count;
  __nv_bfloat16* wf[kLayers];
  __nv_bfloat16* wb[kLayers];
  CUtensorMap tmWf[kLayers], tmWb[kLayers];
  // activations (padded BF16): X (16), H[0..4], A[0..3] (32); gradients dH, dA (32), G16 (16)
  __nv_bfloat16 *X, *H[kBlocks + 1], *A[kBlocks], *dH, *dA, *G16;
  ConvMaps tmX, tmH[kBlocks + 1], tmA[kBlocks], tmdH, tmdA, tmG16;
  float* y16;     // [n][16]
  float* tgt;     // [5][n] staging of the target
  float* msk;     // [n]
  float* qin;     // [5][n] staging of input Q
  float* uin;     // [3][n] staging of input u
  float* rin;     // [5][n] staging of input R
  float *grad, *adam_m, *adam_v;
  float* dw_partial;  // per-CTA partial weight gradients of the tensor-core kernel
  double *partial, *dloss, *h_loss;
  int* d_err;
  long long adam_step;
  cudaEvent_t ev_rate, ev_update;  // cross-stream ordering with a lattice
  std::vector<void*> allocs;
};

namespace {

bool use_win(const lcbp_surrogate* s) { return s->conv_kernel != LCBP_CONV_TAPS; }

int sur_alloc(lcbp_surrogate* s, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(LCBP_ENOMEM, "surrogate allocation of %zu bytes failed", bytes);
  }
  s->allocs.push_back(*p);
  return LCBP_OK;
}

cudaError_t refresh_weights(lcbp_surrogate* s) {
  for (int l = 0; l < kLayers; ++l) {
    const LayerDim d = layer_dim(l);
    k_sur_refresh<<<64, 256, 0, s->stream>>>(s->master + s->off_w[l], d.cin_p, d.cout_p, s->wf[l],
                                             s->training ? s->wb[l] : nullptr);
  }
  return cudaGetLastError();
}

ConvArgs cargs(lcbp_surrogate* s) {
  ConvArgs a{};
  a.nx = s->nx;
  a.ny = s->ny;
  a.nz = s->nz;
  a.n = s->n;
  a.err = s->d_err;
  return a;
}

// forward pass from s->X; the final layer either writes y16 or updates q (with
// the 10 R baseline from `rate`)
cudaError_t forward(lcbp_surrogate* s, float* qupdate, const float* rate = nullptr) {
  cudaError_t e;
  ConvArgs a = cargs(s);
  // h0 = relu(conv_in x)
  a.bias = s->master + s->off_b[0];
  a.out_bf16 = s->H[0];
  e = conv_launch(16, 32, kEpiBias | kEpiRelu, s->tmX, use_win(s), s->tmWf[0], a, s->sms, s->stream);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < kBlocks; ++k) {
    const int la = 1 + 2 * k, lb = 2 + 2 * k;
    // training keeps every activation; inference ping-pongs H[0] / H[1]
    const int hin = s->training ? k : (k & 1), hout = s->training ? k + 1 : ((k + 1) & 1);
    __nv_bfloat16* abuf = s->training ? s->A[k] : s->A[0];
    const ConvMaps& tma = s->training ? s->tmA[k] : s->tmA[0];
    a = cargs(s);
    a.bias = s->master + s->off_b[la];
    a.out_bf16 = abuf;
    e = conv_launch(32, 32, kEpiBias | kEpiRelu, s->tmH[hin], use_win(s), s->tmWf[la], a, s->sms, s->stream);
    if (e != cudaSuccess) return e;
    a = cargs(s);
    a.bias = s->master + s->off_b[lb];
    a.resid = s->H[hin];
    a.out_bf16 = s->H[hout];
    e = conv_launch(32, 32, kEpiBias | kEpiResid, tma, use_win(s), s->tmWf[lb], a, s->sms, s->stream);
    if (e != cudaSuccess) return e;
  }
  const int hlast = s->training ? kBlocks : (kBlocks & 1);
  a = cargs(s);
  a.bias = s->master + s->off_b[kLayers - 1];
  if (qupdate) {
    a.qstate = qupdate;
    a.qscale = s->sdq;
    a.rate = rate;
    a.rate_scale = (float)s->ksteps;
    return conv_launch(32, 16, kEpiBias | kEpiUpdateQ, s->tmH[hlast], use_win(s), s->tmWf[kLayers - 1], a, s->sms,
                       s->stream);
  }
  a.out_f32 = s->y16;
  return conv_launch(32, 16, kEpiBias | kEpiOutF32, s->tmH[hlast], use_win(s), s->tmWf[kLayers - 1], a, s->sms, s->stream);
}

// Weight and bias gradients of layer l: on the tensor cores where the staged
// plane windows fit shared memory, else on CUDA cores (FP32 atomics)
template <int CX, int CY>
cudaError_t launch_dw(lcbp_surrogate* s, const __nv_bfloat16* X, const __nv_bfloat16* dY, int l) {
  if (!s->dw_cuda_cores && dw_fits(CX, CY, s->nx, s->ny, s->nz))
    return dw_launch(CX, CY, X, dY, s->nx, s->ny, s->nz, s->dw_partial, s->grad + s->off_w[l], s->grad + s->off_b[l],
                     s->d_err, s->sms, s->stream);
  const int chunk = 4096;
  const dim3 grid((unsigned)((s->n + chunk - 1) / chunk), 27);
  k_sur_dw<CX, CY><<<grid, CX * CY / 16, 0, s->stream>>>(X, dY, s->nx, s->ny, s->nz, chunk, s->grad + s->off_w[l],
                                                         s->grad + s->off_b[l]);
  return cudaGetLastError();
}

int check_s(lcbp_surrogate* s) {
  if (!s) return fail(LCBP_EINVAL, "null surrogate handle");
  cudaSetDevice(s->device);
  return LCBP_OK;
}

int sync_err(lcbp_surrogate* s, const char* what) {
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  int flag = 0;
  e = cudaMemcpy(&flag, s->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (flag) {
    cudaMemset(s->d_err, 0, sizeof(int));
    return fail(LCBP_ETIMEOUT, "%s: a bounded tensor-core pipeline wait timed out", what);
  }
  return LCBP_OK;
}

// stage caller fields (host or device, f32/f64) into s->qin / s->uin
// (the staging buffer holds 5 n floats = 5 n / 2 doubles)
int stage_inputs(lcbp_surrogate* s, const void* q5, const void* u3, const void* r5, int dtype) {
  const long long st = 5 * s->n / 2;
  int rc = transfer(s->qin, LCBP_F32, const_cast<void*>(q5), dtype, 5 * s->n, true, s->tgt, st, s->stream);
  if (rc) return rc;
  if (u3) rc = transfer(s->uin, LCBP_F32, const_cast<void*>(u3), dtype, 3 * s->n, true, s->tgt, st, s->stream);
  if (!rc && r5) rc = transfer(s->rin, LCBP_F32, const_cast<void*>(r5), dtype, 5 * s->n, true, s->tgt, st, s->stream);
  return rc;
}

}  // namespace

extern "C" {

size_t lcbp_surrogate_param_count(void) { return true_param_count(); }

int lcbp_surrogate_create(int nx, int ny, int nz, int training, lcbp_surrogate** out) {
  if (!out) return fail(LCBP_EINVAL, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1) return fail(LCBP_EINVAL, "sizes must be >= 1");
  if ((long long)(nx + 2) * (ny + 2) * (nz + 2) > (1ll << 31)) return fail(LCBP_EINVAL, "lattice too large");
  auto* s = new lcbp_surrogate();
  s->nx = nx;
  s->ny = ny;
  s->nz = nz;
  s->n = (long long)nx * ny * nz;
  s->np = (long long)(nx + 2) * (ny + 2) * (nz + 2);
  s->training = training ? 1 : 0;
  s->su = 1e-3f;
  s->sr = 1e-3f;
  s->sdq = 1e-3f;
  s->ksteps = kDefaultSteps;
  cudaGetDevice(&s->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  s->sms = std::max(sms, 1);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "stream");
  }
  size_t mc = 0;
  for (int l = 0; l < kLayers; ++l) {
    const LayerDim d = layer_dim(l);
    s->off_w[l] = mc;
    mc += 27 * (size_t)d.cin_p * d.cout_p;
    s->off_b[l] = mc;
    mc += d.cout_p;
  }
  s->master_count = mc;
  int rc = LCBP_OK;
  auto A = [&](void** p, size_t bytes) {
    if (!rc) rc = sur_alloc(s, p, bytes);
  };
  A((void**)&s->master, mc * 4);
  for (int l = 0; l < kLayers; ++l) {
    const LayerDim d = layer_dim(l);
    A((void**)&s->wf[l], 27 * (size_t)d.cin_p * d.cout_p * 2);
    if (s->training) A((void**)&s->wb[l], 27 * (size_t)d.cin_p * d.cout_p * 2);
  }
  // padded chunk-planar activations plus the tail the window copies may read
  const size_t b16 = (size_t)s->np * 16 * 2 + kActTailBytes, b32 = (size_t)s->np * 32 * 2 + kActTailBytes;
  A((void**)&s->X, b16);
  const int nh = s->training ? kBlocks + 1 : 2, na = s->training ? kBlocks : 1;
  for (int k = 0; k < nh; ++k) A((void**)&s->H[k], b32);
  for (int k = 0; k < na; ++k) A((void**)&s->A[k], b32);
  A((void**)&s->y16, (size_t)s->n * 16 * 4);
  A((void**)&s->tgt, (size_t)s->n * 5 * 4);
  A((void**)&s->qin, (size_t)s->n * 5 * 4);
  A((void**)&s->uin, (size_t)s->n * 3 * 4);
  A((void**)&s->rin, (size_t)s->n * 5 * 4);
  A((void**)&s->partial, 4096 * 8 + 64);
  A((void**)&s->d_err, 64);
  if (s->training) {
    A((void**)&s->dH, b32);
    A((void**)&s->dA, b32);
    A((void**)&s->G16, b16);
    A((void**)&s->msk, (size_t)s->n * 4);
    A((void**)&s->grad, mc * 4);
    A((void**)&s->adam_m, mc * 4);
    A((void**)&s->adam_v, mc * 4);
    A((void**)&s->dw_partial, dw_partial_floats(s->sms) * 4);
  }
  if (!rc) {
    e = cudaEventCreateWithFlags(&s->ev_rate, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_update, cudaEventDisableTiming);
    if (e != cudaSuccess) rc = cuda_fail(e, "events");
  }
  if (!rc) {
    s->dloss = s->partial + 4096;
    e = cudaMallocHost(&s->h_loss, 8);
    if (e != cudaSuccess) rc = cuda_fail(e, "host alloc");
  }
  if (!rc) {
    cudaMemsetAsync(s->master, 0, mc * 4, s->stream);
    cudaMemsetAsync(s->d_err, 0, 64, s->stream);
    // every activation buffer, tail included: copies of plane windows may read
    // the tail, and its bytes must be finite numbers (they meet zero gradients)
    cudaMemsetAsync(s->X, 0, b16, s->stream);
    for (int k = 0; k < nh; ++k) cudaMemsetAsync(s->H[k], 0, b32, s->stream);
    for (int k = 0; k < na; ++k) cudaMemsetAsync(s->A[k], 0, b32, s->stream);
    if (s->training) {
      cudaMemsetAsync(s->dH, 0, b32, s->stream);
      cudaMemsetAsync(s->dA, 0, b32, s->stream);
      cudaMemsetAsync(s->G16, 0, b16, s->stream);
      cudaMemsetAsync(s->adam_m, 0, mc * 4, s->stream);
      cudaMemsetAsync(s->adam_v, 0, mc * 4, s->stream);
    }
    bool ok = conv_maps(&s->tmX, s->X, 16, nx, ny, nz);
    for (int k = 0; k < nh; ++k) ok = ok && conv_maps(&s->tmH[k], s->H[k], 32, nx, ny, nz);
    for (int k = 0; k < na; ++k) ok = ok && conv_maps(&s->tmA[k], s->A[k], 32, nx, ny, nz);
    if (s->training) {
      ok = ok && conv_maps(&s->tmdH, s->dH, 32, nx, ny, nz) && conv_maps(&s->tmdA, s->dA, 32, nx, ny, nz) &&
           conv_maps(&s->tmG16, s->G16, 16, nx, ny, nz);
    }
    for (int l = 0; l < kLayers && ok; ++l) {
      const LayerDim d = layer_dim(l);
      ok = weight_map(&s->tmWf[l], s->wf[l], d.cin_p, d.cout_p);
      if (ok && s->training) ok = weight_map(&s->tmWb[l], s->wb[l], d.cout_p, d.cin_p);
    }
    if (!ok) rc = fail(LCBP_ECUDA, "tensor map encoding failed");
  }
  if (!rc) {
    e = refresh_weights(s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "surrogate set-up");
  }
  if (rc) {
    lcbp_surrogate_destroy(s);
    return rc;
  }
  *out = s;
  return LCBP_OK;
}

int lcbp_surrogate_destroy(lcbp_surrogate* s) {
  if (!s) return LCBP_OK;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_loss) cudaFreeHost(s->h_loss);
  if (s->ev_rate) cudaEventDestroy(s->ev_rate);
  if (s->ev_update) cudaEventDestroy(s->ev_update);
  cudaStreamDestroy(s->stream);
  delete s;
  return LCBP_OK;
}

int lcbp_surrogate_set_scales(lcbp_surrogate* s, double s_u, double s_r, double s_dq) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!(s_u > 0) || !(s_r > 0) || !(s_dq > 0)) return fail(LCBP_EINVAL, "scales must be > 0");
  s->su = (float)s_u;
  s->sr = (float)s_r;
  s->sdq = (float)s_dq;
  return LCBP_OK;
}

int lcbp_surrogate_set_steps(lcbp_surrogate* s, int k) {
  int rc = check_s(s);
  if (rc) return rc;
  if (k < 1 || k > 1000) return fail(LCBP_EINVAL, "steps per call must be in 1..1000, got %d", k);
  s->ksteps = k;
  return LCBP_OK;
}

int lcbp_surrogate_get_steps(lcbp_surrogate* s, int* k) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!k) return fail(LCBP_EINVAL, "k is NULL");
  *k = s->ksteps;
  return LCBP_OK;
}

int lcbp_surrogate_set_conv_kernel(lcbp_surrogate* s, int kind) {
  int rc = check_s(s);
  if (rc) return rc;
  const bool dw_cc = (kind & LCBP_CONV_DW_CUDA_CORES) != 0;
  kind &= ~LCBP_CONV_DW_CUDA_CORES;
  if (kind < LCBP_CONV_AUTO || kind > LCBP_CONV_WINDOW) return fail(LCBP_EINVAL, "unknown conv kernel %d", kind);
  if (kind == LCBP_CONV_WINDOW && !s->tmX.use_win)
    return fail(LCBP_EINVAL, "a %d x %d plane does not fit the window kernel", s->nx, s->ny);
  s->conv_kernel = kind;
  s->dw_cuda_cores = dw_cc;
  return LCBP_OK;
}

int lcbp_surrogate_set_params(lcbp_surrogate* s, const float* p, size_t count) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!p || count != true_param_count())
    return fail(LCBP_EINVAL, "expected %zu parameters, got %zu", true_param_count(), count);
  float* staging = nullptr;
  rc = sur_alloc(s, (void**)&staging, count * 4);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(staging, p, count * 4, cudaMemcpyDefault, s->stream);
  size_t off = 0;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    const LayerDim d = layer_dim(l);
    k_sur_scatter<<<64, 256, 0, s->stream>>>(staging + off, d.cin, d.cout, d.cin_p, d.cout_p, s->master + s->off_w[l],
                                             s->master + s->off_b[l], 1);
    off += 27 * (size_t)d.cin * d.cout + d.cout;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = refresh_weights(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(staging);
  s->allocs.pop_back();
  if (s->training) {
    cudaMemsetAsync(s->adam_m, 0, s->master_count * 4, s->stream);
    cudaMemsetAsync(s->adam_v, 0, s->master_count * 4, s->stream);
    s->adam_step = 0;
  }
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "set_params");
}

int lcbp_surrogate_get_params(lcbp_surrogate* s, float* p, size_t count) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!p || count != true_param_count()) return fail(LCBP_EINVAL, "expected %zu parameters", true_param_count());
  float* staging = nullptr;
  rc = sur_alloc(s, (void**)&staging, count * 4);
  if (rc) return rc;
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    const LayerDim d = layer_dim(l);
    k_sur_scatter<<<64, 256, 0, s->stream>>>(staging + off, d.cin, d.cout, d.cin_p, d.cout_p, s->master + s->off_w[l],
                                             s->master + s->off_b[l], 0);
    off += 27 * (size_t)d.cin * d.cout + d.cout;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, staging, count * 4, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(staging);
  s->allocs.pop_back();
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "get_params");
}

int lcbp_surrogate_get_grads(lcbp_surrogate* s, float* g, size_t count) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!s->training) return fail(LCBP_ESTATE, "surrogate was created without training buffers");
  if (!g || count != true_param_count()) return fail(LCBP_EINVAL, "expected %zu values", true_param_count());
  float* staging = nullptr;
  rc = sur_alloc(s, (void**)&staging, count * 4);
  if (rc) return rc;
  size_t off = 0;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    const LayerDim d = layer_dim(l);
    k_sur_scatter<<<64, 256, 0, s->stream>>>(staging + off, d.cin, d.cout, d.cin_p, d.cout_p, s->grad + s->off_w[l],
                                             s->grad + s->off_b[l], 0);
    off += 27 * (size_t)d.cin * d.cout + d.cout;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(g, staging, count * 4, cudaMemcpyDefault, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(staging);
  s->allocs.pop_back();
  return e == cudaSuccess ? LCBP_OK : cuda_fail(e, "get_grads");
}

// Weights file, version 1 (little-endian): "LCBPSURR", int32 version, int32
// blocks, width, input channels, output channels, kernel size, solver steps
// per call, int32 0, then double s_u, s_r, s_dq, uint64 count, and count FP32
// parameters in the order of lcbp_surrogate_get_params.
namespace {
struct SurHeader {
  char magic[8];
  int32_t version, blocks, width, cin, cout, ksize, steps, pad;
  double su, sr, sdq;
  uint64_t count;
};
constexpr int32_t kSurFileVersion = 1;
}  // namespace

int lcbp_surrogate_save(lcbp_surrogate* s, const char* path) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!path) return fail(LCBP_EINVAL, "path is NULL");
  const size_t count = true_param_count();
  std::vector<float> v(count);
  rc = lcbp_surrogate_get_params(s, v.data(), count);
  if (rc) return rc;
  SurHeader hd{};
  std::memcpy(hd.magic, "LCBPSURR", 8);
  hd.version = kSurFileVersion;
  hd.blocks = kBlocks;
  hd.width = kWidth;
  hd.cin = kInC;
  hd.cout = kOutC;
  hd.ksize = 3;
  hd.steps = s->ksteps;
  hd.su = s->su;
  hd.sr = s->sr;
  hd.sdq = s->sdq;
  hd.count = count;
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(LCBP_EIO, "cannot open %s for writing", path);
  const bool ok = std::fwrite(&hd, sizeof(hd), 1, fp) == 1 && std::fwrite(v.data(), 4, count, fp) == count;
  const bool closed = std::fclose(fp) == 0;
  return ok && closed ? LCBP_OK : fail(LCBP_EIO, "writing %s failed", path);
}

int lcbp_surrogate_load(lcbp_surrogate* s, const char* path) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!path) return fail(LCBP_EINVAL, "path is NULL");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return fail(LCBP_EIO, "cannot open %s", path);
  SurHeader hd{};
  const size_t count = true_param_count();
  std::vector<float> v;
  bool ok = std::fread(&hd, sizeof(hd), 1, fp) == 1;
  if (ok && (std::memcmp(hd.magic, "LCBPSURR", 8) != 0 || hd.version != kSurFileVersion)) {
    std::fclose(fp);
    return fail(LCBP_EIO, "%s is not a version-%d surrogate weights file", path, kSurFileVersion);
  }
  if (ok && (hd.blocks != kBlocks || hd.width != kWidth || hd.cin != kInC || hd.cout != kOutC || hd.ksize != 3 ||
             hd.steps < 1 || hd.count != count)) {
    std::fclose(fp);
    return fail(LCBP_EINVAL, "%s holds another network (%d blocks, width %d, %llu parameters)", path, hd.blocks,
                hd.width, (unsigned long long)hd.count);
  }
  if (ok) {
    v.resize(count);
    ok = std::fread(v.data(), 4, count, fp) == count;
  }
  std::fclose(fp);
  if (!ok) return fail(LCBP_EIO, "%s is truncated", path);
  for (float x : v)
    if (!std::isfinite(x)) return fail(LCBP_ENONFINITE, "%s holds non-finite parameters", path);
  rc = lcbp_surrogate_set_scales(s, hd.su, hd.sr, hd.sdq);
  if (!rc) rc = lcbp_surrogate_set_steps(s, hd.steps);
  return rc ? rc : lcbp_surrogate_set_params(s, v.data(), count);
}

int lcbp_surrogate_forward(lcbp_surrogate* s, const void* q5, const void* u3, const void* r5, double kappa,
                           double tau, int dtype, float* y5) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!q5 || !y5 || !valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad buffers or dtype");
  rc = stage_inputs(s, q5, u3, r5, dtype);
  if (rc) return rc;
  k_sur_input<<<grid_for(s->np), 256, 0, s->stream>>>(s->qin, u3 ? s->uin : nullptr, r5 ? s->rin : nullptr, s->su,
                                                      s->sr, (float)kappa, (float)tau, s->nx, s->ny, s->nz, s->X);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = forward(s, nullptr);
  if (e == cudaSuccess) {
    k_f32_soa<<<grid_for(s->n), 256, 0, s->stream>>>(s->y16, s->n, s->tgt);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(e, "surrogate forward");
  rc = sync_err(s, "surrogate forward");
  if (rc) return rc;
  return transfer(s->tgt, LCBP_F32, y5, LCBP_F32, 5 * s->n, false, nullptr, 0, s->stream);
}

int lcbp_surrogate_step(lcbp_surrogate* s, lcbp_lattice* h, double kappa, double tau, int ncalls) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!h || ncalls < 0) return fail(LCBP_EINVAL, "bad lattice or ncalls");
  float* q = nullptr;
  const float* u = nullptr;
  int dims[3];
  cudaStream_t hs;
  rc = lattice_fields(h, &q, &u, dims, &hs);
  if (rc) return rc;
  if (dims[0] != s->nx || dims[1] != s->ny || dims[2] != s->nz)
    return fail(LCBP_EINVAL, "surrogate built for %dx%dx%d, lattice is %dx%dx%d", s->nx, s->ny, s->nz, dims[0], dims[1],
                dims[2]);
  // The rate runs on the lattice's stream, the network on the surrogate's;
  // events order them without host round trips.
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < ncalls && e == cudaSuccess; ++c) {
    const float* r = nullptr;
    rc = lattice_rate(h, &r, s->ev_rate);
    if (rc) return rc;
    e = cudaStreamWaitEvent(s->stream, s->ev_rate, 0);
    if (e != cudaSuccess) break;
    k_sur_input<<<grid_for(s->np), 256, 0, s->stream>>>(q, u, r, s->su, s->sr, (float)kappa, (float)tau, s->nx,
                                                        s->ny, s->nz, s->X);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = forward(s, q, r);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev_update, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, s->ev_update, 0);  // next rate sees the updated Q
  }
  if (e != cudaSuccess) return cuda_fail(e, "surrogate step");
  return sync_err(s, "surrogate step");
}

int lcbp_surrogate_train_step(lcbp_surrogate* s, const void* q5, const void* u3, const void* r5, double kappa,
                              double tau, const void* dq5, const void* mask, int dtype, double lr, double* loss) {
  int rc = check_s(s);
  if (rc) return rc;
  if (!s->training) return fail(LCBP_ESTATE, "surrogate was created without training buffers");
  if (!q5 || !dq5 || !valid_dtype(dtype) || !(lr > 0)) return fail(LCBP_EINVAL, "bad arguments");
  rc = stage_inputs(s, q5, u3, r5, dtype);
  if (!rc) rc = transfer(s->tgt, LCBP_F32, const_cast<void*>(dq5), dtype, 5 * s->n, true, s->y16, 8 * s->n, s->stream);
  if (!rc && mask) rc = transfer(s->msk, LCBP_F32, const_cast<void*>(mask), dtype, s->n, true, s->y16, 8 * s->n, s->stream);
  if (rc) return rc;
  // denominator of the masked MSE: 5 channels x sum of the mask
  double den = 5.0 * (double)s->n;
  if (mask) {
    std::vector<float> hm(s->n);
    cudaError_t e0 = cudaMemcpyAsync(hm.data(), s->msk, s->n * 4, cudaMemcpyDeviceToHost, s->stream);
    if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(s->stream);
    if (e0 != cudaSuccess) return cuda_fail(e0, "mask");
    double sm = 0;
    for (float v : hm) sm += v;
    den = 5.0 * sm;
    if (!(den > 0)) return fail(LCBP_EINVAL, "mask is empty");
  }
  cudaError_t e = cudaSuccess;
  k_sur_input<<<grid_for(s->np), 256, 0, s->stream>>>(s->qin, u3 ? s->uin : nullptr, r5 ? s->rin : nullptr, s->su,
                                                      s->sr, (float)kappa, (float)tau, s->nx, s->ny, s->nz, s->X);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = forward(s, nullptr);
  const int lb = 1024;
  if (e == cudaSuccess) {
    k_sur_loss<<<lb, 256, 0, s->stream>>>(s->y16, s->tgt, r5 ? s->rin : nullptr, (float)s->ksteps,
                                           mask ? s->msk : nullptr,
                                           1.f / s->sdq, 1.0 / den, s->nx, s->ny, s->nz, s->G16, s->partial);
    k_sum<<<1, 32, 0, s->stream>>>(s->partial, lb, 1.0 / den, s->dloss);
    k_zero<<<256, 256, 0, s->stream>>>(s->grad, (long long)s->master_count);
    e = cudaGetLastError();
  }
  // ---- backward
  const int lout = kLayers - 1;
  if (e == cudaSuccess) {
    e = launch_dw<32, 16>(s, s->H[kBlocks], s->G16, lout);
    ConvArgs a = cargs(s);
    a.out_bf16 = s->dH;
    if (e == cudaSuccess) e = conv_launch(16, 32, 0, s->tmG16, use_win(s), s->tmWb[lout], a, s->sms, s->stream);
  }
  for (int k = kBlocks - 1; k >= 0 && e == cudaSuccess; --k) {
    const int la = 1 + 2 * k, lbb = 2 + 2 * k;
    // d a_k (pre-activation) = convT_b(dh) * [a_k > 0]
    ConvArgs a = cargs(s);
    a.mask = s->A[k];
    a.out_bf16 = s->dA;
    e = conv_launch(32, 32, kEpiMask, s->tmdH, use_win(s), s->tmWb[lbb], a, s->sms, s->stream);
    if (e != cudaSuccess) break;
    e = launch_dw<32, 32>(s, s->A[k], s->dH, lbb);
    if (e == cudaSuccess) e = launch_dw<32, 32>(s, s->H[k], s->dA, la);
    if (e != cudaSuccess) break;
    // dh_k = dh_{k+1} + convT_a(d pre_k)   (times [h0 > 0] for the input layer's gradient)
    a = cargs(s);
    a.resid = s->dH;
    a.out_bf16 = s->dH;
    if (k == 0) a.mask = s->H[0];
    e = conv_launch(32, 32, k == 0 ? (kEpiResid | kEpiMask) : kEpiResid, s->tmdA, use_win(s), s->tmWb[la], a, s->sms,
                    s->stream);
  }
  if (e == cudaSuccess) {
    e = launch_dw<16, 32>(s, s->X, s->dH, 0);
  }
  if (e == cudaSuccess) {
    ++s->adam_step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)s->adam_step), c2 = 1.f - powf(b2, (float)s->adam_step);
    k_adam<<<256, 256, 0, s->stream>>>(s->master, s->grad, s->adam_m, s->adam_v, (long long)s->master_count, (float)lr,
                                       b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = refresh_weights(s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_loss, s->dloss, 8, cudaMemcpyDeviceToHost, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "train step");
  rc = sync_err(s, "train step");
  if (rc) return rc;
  if (loss) *loss = *s->h_loss;
  return LCBP_OK;
}

}  // extern "C"
