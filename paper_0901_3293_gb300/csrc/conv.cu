// 3x3x3 periodic convolution as an implicit GEMM on tcgen05 tensor cores.
//
// y(r) = b + sum_t W_t^T x(r + o_t) over the 27 taps o_t, for activations
// stored BF16 channels-last with one ghost layer per face ([z+1][y+1][x+1][C],
// periodic images in the ghosts), so that every shifted tile is an in-range
// TMA box.  One CTA tile is 128 sites (32 x 4 x 1) = the M of one UMMA; the
// K loop runs over taps (C_in channels each, 16 per MMA) and N = C_out.
//
// Warp roles (192 threads):  warps 0-3 epilogue (TMEM lanes 0..127),
// warp 4 TMA producer, warp 5 MMA issuer.  A ring of A-operand stages (one
// tap each) with full/empty mbarriers feeds the MMAs; all 27 weight taps stay
// in shared memory; the FP32 accumulator is double-buffered in tensor memory
// so the epilogue of one tile overlaps the MMAs of the next.  The epilogue
// adds the bias and optionally a residual, applies ReLU or a ReLU mask, and
// writes BF16 (with ghost images), FP32, or an update of the FP32 Q field.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "conv.h"
#include "tc.cuh"

namespace lcbp {

constexpr int kConvStages = 6;
constexpr int kConvThreads = 192;
constexpr uint64_t kConvWaitNs = 2000000000ull;

template <int CIN, int COUT>
struct ConvSmem {
  static constexpr int WBYTES = ((27 * COUT * CIN * 2 + 1023) / 1024) * 1024;
  static constexpr int STAGE = 128 * CIN * 2;
  static constexpr int OFF_STAGES = WBYTES;
  static constexpr int OFF_BARS = OFF_STAGES + kConvStages * STAGE;
  // full[S], empty[S], accf[2], acce[2], wbar
  static constexpr int NBARS = 2 * kConvStages + 5;
  static constexpr size_t bytes = OFF_BARS + NBARS * 8 + 16 + 1024;  // + alignment slack
  static constexpr uint32_t SWZ = CIN == 32 ? kSwizzle64B : kSwizzle32B;
  static constexpr uint32_t SBO = 8 * CIN * 2;  // 8 rows of one swizzle span
  static constexpr uint32_t TMEM_COLS = 2 * COUT < 32 ? 32 : 2 * COUT;
};

__device__ __forceinline__ float bf2f(__nv_bfloat16 v) { return __bfloat162float(v); }


// Epilogue of one output site: v[] holds the COUT accumulator values of site (x, y, z).
template <int COUT, int EPI>
__device__ __forceinline__ void conv_epilogue(float (&v)[COUT], int x, int y, int z, const ConvArgs& a) {
  if (x >= a.nx || y >= a.ny) return;
  const int px = a.nx + 2, py = a.ny + 2;
  const long long pidx = ((long long)(z + 1) * py + (y + 1)) * px + (x + 1);
  if (EPI & kEpiBias) {
#pragma unroll
    for (int c = 0; c < COUT; ++c) v[c] += a.bias[c];
  }
  if (EPI & kEpiResid) {
    const uint4* rp = reinterpret_cast<const uint4*>(a.resid + pidx * COUT);
#pragma unroll
    for (int q = 0; q < COUT / 8; ++q) {
      const uint4 w4 = rp[q];
      const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&w4);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[q * 8 + j] += bf2f(h8[j]);
    }
  }
  if (EPI & kEpiRelu) {
#pragma unroll
    for (int c = 0; c < COUT; ++c) v[c] = fmaxf(v[c], 0.f);
  }
  if (EPI & kEpiMask) {
    const uint4* mp = reinterpret_cast<const uint4*>(a.mask + pidx * COUT);
#pragma unroll
    for (int q = 0; q < COUT / 8; ++q) {
      const uint4 w4 = mp[q];
      const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&w4);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[q * 8 + j] = bf2f(h8[j]) > 0.f ? v[q * 8 + j] : 0.f;
    }
  }
  const long long site = ((long long)z * a.ny + y) * a.nx + x;
  if (EPI & kEpiOutF32) {
    float4* op = reinterpret_cast<float4*>(a.out_f32 + site * COUT);
#pragma unroll
    for (int q = 0; q < COUT / 4; ++q) op[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if (EPI & kEpiUpdateQ) {
#pragma unroll
    for (int c = 0; c < 5; ++c)
      a.qstate[c * a.n + site] += a.qscale * v[c] + (a.rate ? a.rate_scale * a.rate[c * a.n + site] : 0.f);
  } else {
    // BF16 channels-last at the site and at every ghost image of it
    uint4 pk[COUT / 8];
#pragma unroll
    for (int q = 0; q < COUT / 8; ++q) {
      __nv_bfloat16* h8 = reinterpret_cast<__nv_bfloat16*>(&pk[q]);
#pragma unroll
      for (int j = 0; j < 8; ++j) h8[j] = __float2bfloat16_rn(v[q * 8 + j]);
    }
    // padded coordinates that hold this site: the interior one, and the
    // opposite ghost layer when the site lies on a face (both for width 1)
    const int gx[3] = {x + 1, x == a.nx - 1 ? 0 : -1, x == 0 ? a.nx + 1 : -1};
    const int gy[3] = {y + 1, y == a.ny - 1 ? 0 : -1, y == 0 ? a.ny + 1 : -1};
    const int gz[3] = {z + 1, z == a.nz - 1 ? 0 : -1, z == 0 ? a.nz + 1 : -1};
    for (int iz = 0; iz < 3; ++iz) {
      if (gz[iz] < 0) continue;
      for (int iy = 0; iy < 3; ++iy) {
        if (gy[iy] < 0) continue;
        for (int ix = 0; ix < 3; ++ix) {
          if (gx[ix] < 0) continue;
          uint4* op = reinterpret_cast<uint4*>(a.out_bf16 + (((long long)gz[iz] * py + gy[iy]) * px + gx[ix]) * COUT);
#pragma unroll
          for (int q = 0; q < COUT / 8; ++q) op[q] = pk[q];
        }
      }
    }
  }
}

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kConvThreads) k_conv_tc(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmW, ConvArgs a) {
  using L = ConvSmem<CIN, COUT>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* wsm = smem;
  unsigned char* stages = smem + L::OFF_STAGES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::OFF_BARS);
  uint64_t* full = bars;
  uint64_t* empty = bars + kConvStages;
  uint64_t* accf = bars + 2 * kConvStages;
  uint64_t* acce = accf + 2;
  uint64_t* wbar = acce + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int tiles_x = (a.nx + 31) / 32, tiles_y = (a.ny + 3) / 4;
  const int ntiles = tiles_x * tiles_y * a.nz;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kConvStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&accf[0], 1);
    mbar_init(&accf[1], 1);
    mbar_init(&acce[0], 128);
    mbar_init(&acce[1], 128);
    mbar_init(wbar, 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, L::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto bounded_wait = [&](uint64_t* bar, uint32_t parity) {
    if (*abort_flag) return false;
    if (!mbar_wait_bounded(bar, parity, kConvWaitNs)) {
      *abort_flag = 1;
      atomicExch(a.err, 1);
      return false;
    }
    return true;
  };

  if (warp == 4) {
    // ---------------- TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmW);
      mbar_arrive_expect_tx(wbar, 27 * COUT * CIN * 2);
      tma_load_3d(wsm, &tmW, 0, 0, 0, wbar);
      int k = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * 32, y0 = ((tile / tiles_x) % tiles_y) * 4, z0 = tile / (tiles_x * tiles_y);
        for (int t = 0; t < 27; ++t, ++k) {
          const int s = k % kConvStages;
          if (k >= kConvStages && !bounded_wait(&empty[s], ((k / kConvStages) - 1) & 1)) break;
          const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
          mbar_arrive_expect_tx(&full[s], L::STAGE);
          tma_load_4d(stages + s * L::STAGE, &tmA, 0, x0 + 1 + dx, y0 + 1 + dy, z0 + 1 + dz, &full[s]);
        }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_bf16(128, COUT);
      const uint32_t w_addr = smem_addr(wsm), st_addr = smem_addr(stages);
      bool ok = bounded_wait(wbar, 0);
      int k = 0, i = 0;
      for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++i) {
        const int acc = i & 1;
        if (i >= 2 && !bounded_wait(&acce[acc], ((i >> 1) - 1) & 1)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * COUT;
        for (int t = 0; t < 27; ++t, ++k) {
          const int s = k % kConvStages;
          if (!bounded_wait(&full[s], (k / kConvStages) & 1)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < CIN / 16; ++kk) {
            const uint64_t ad = umma_sdesc(st_addr + s * L::STAGE + kk * 32, L::SBO, L::SWZ);
            const uint64_t bd = umma_sdesc(w_addr + t * (COUT * CIN * 2) + kk * 32, L::SBO, L::SWZ);
            umma_bf16(d_tmem, ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
          }
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&accf[acc]);
      }
    }
  } else {
    // ---------------- epilogue: warps 0..3, one TMEM lane (= one site) per thread
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int acc = i & 1;
      // every lane waits; the warp proceeds only together (tcgen05.ld is warp-collective)
      const bool ok = __all_sync(0xffffffffu, bounded_wait(&accf[acc], (i >> 1) & 1));
      if (!ok) break;
      tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + acc * COUT;
      float v[COUT];
      if constexpr (COUT == 32) {
        uint32_t r[32];
        tmem_ld32(taddr, r);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
      } else {
        uint32_t r[16];
        tmem_ld16(taddr, r);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
      }
      tc_fence_before();
      mbar_arrive(&acce[acc]);

      const int x0 = (tile % tiles_x) * 32, y0 = ((tile / tiles_x) % tiles_y) * 4, z0 = tile / (tiles_x * tiles_y);
      const int m = warp * 32 + lane;
      conv_epilogue<COUT, EPI>(v, x0 + (m & 31), y0 + (m >> 5), z0, a);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, L::TMEM_COLS);
  }
}


// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int EPI>
cudaError_t conv_launch_t(const CUtensorMap& tmA, const CUtensorMap& tmW, const ConvArgs& a, int max_ctas,
                          cudaStream_t s) {
  using L = ConvSmem<CIN, COUT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int ntiles = ((a.nx + 31) / 32) * ((a.ny + 3) / 4) * a.nz;
  const int grid = ntiles < max_ctas ? ntiles : max_ctas;
  k_conv_tc<CIN, COUT, EPI><<<grid, kConvThreads, L::bytes, s>>>(tmA, tmW, a);
  return cudaGetLastError();
}

cudaError_t conv_launch(int cin, int cout, int epi, const CUtensorMap& tmA, const CUtensorMap& tmW,
                        const ConvArgs& a, int max_ctas, cudaStream_t s) {
#define LCBP_CONV_CASE(CI, CO, E) \
  if (cin == CI && cout == CO && epi == (E)) return conv_launch_t<CI, CO, E>(tmA, tmW, a, max_ctas, s);
  // forward: input layer, hidden layers, residual layers, output layer (FP32 out / Q update)
  LCBP_CONV_CASE(16, 32, kEpiBias | kEpiRelu)
  LCBP_CONV_CASE(32, 32, kEpiBias | kEpiRelu)
  LCBP_CONV_CASE(32, 32, kEpiBias | kEpiResid)
  LCBP_CONV_CASE(32, 16, kEpiBias | kEpiOutF32)
  LCBP_CONV_CASE(32, 16, kEpiBias | kEpiUpdateQ)
  // backward data: output layer (16 -> 32), masked, residual, residual + mask
  LCBP_CONV_CASE(16, 32, 0)
  LCBP_CONV_CASE(32, 32, kEpiMask)
  LCBP_CONV_CASE(32, 32, kEpiResid)
  LCBP_CONV_CASE(32, 32, kEpiResid | kEpiMask)
  LCBP_CONV_CASE(32, 32, 0)
#undef LCBP_CONV_CASE
  return cudaErrorInvalidValue;
}

}  // namespace lcbp
