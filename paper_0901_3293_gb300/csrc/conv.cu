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

#include <algorithm>

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

// shared-memory position of weight tap t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1):
// the weights are staged shift-major, [in-plane shift][dz][C_out][C_in]
__host__ __device__ constexpr int w_slot(int t) { return (t % 9) * 3 + t / 9; }


// Epilogue of channels c0 .. c0 + NC of one output site (x, y, z): bias from
// registers, residual / mask operands already loaded (BF16, 8 per uint4).
template <int COUT, int NC, int EPI>
__device__ __forceinline__ void conv_epilogue_part(float (&v)[NC], const float (&bias)[NC], const uint4 (&rsd)[NC / 8],
                                                   const uint4 (&msk)[NC / 8], int c0, int x, int y, int z,
                                                   const ConvArgs& a) {
  static_assert(NC % 8 == 0, "channel slices are whole 16-byte groups");
  const int px = a.nx + 2, py = a.ny + 2;
#pragma unroll
  for (int c = 0; c < NC; ++c) v[c] += bias[c];
  if (EPI & kEpiResid) {
#pragma unroll
    for (int q = 0; q < NC / 8; ++q) {
      const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&rsd[q]);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[q * 8 + j] += bf2f(h8[j]);
    }
  }
  if (EPI & kEpiRelu) {
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = fmaxf(v[c], 0.f);
  }
  if (EPI & kEpiMask) {
#pragma unroll
    for (int q = 0; q < NC / 8; ++q) {
      const __nv_bfloat16* h8 = reinterpret_cast<const __nv_bfloat16*>(&msk[q]);
#pragma unroll
      for (int j = 0; j < 8; ++j) v[q * 8 + j] = bf2f(h8[j]) > 0.f ? v[q * 8 + j] : 0.f;
    }
  }
  const long long site = ((long long)z * a.ny + y) * a.nx + x;
  if (EPI & kEpiOutF32) {
    float4* op = reinterpret_cast<float4*>(a.out_f32 + site * COUT + c0);
#pragma unroll
    for (int q = 0; q < NC / 4; ++q) op[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else if (EPI & kEpiUpdateQ) {
    // all loads first: Q and the rate may alias as far as the compiler knows, and
    // interleaved with the stores they would be five serial round trips
    constexpr int NQ = NC < 5 ? NC : 5;
    float qv[NQ], rv[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
      const bool in = c0 + c < 5;
      qv[c] = in ? a.qstate[(c0 + c) * a.n + site] : 0.f;
      rv[c] = in && a.rate ? a.rate[(c0 + c) * a.n + site] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < NQ; ++c)
      if (c0 + c < 5) a.qstate[(c0 + c) * a.n + site] = qv[c] + (a.qscale * v[c] + a.rate_scale * rv[c]);
  } else {
    uint4 pk[NC / 8];
#pragma unroll
    for (int q = 0; q < NC / 8; ++q) {
      __nv_bfloat16* h8 = reinterpret_cast<__nv_bfloat16*>(&pk[q]);
#pragma unroll
      for (int j = 0; j < 8; ++j) h8[j] = __float2bfloat16_rn(v[q * 8 + j]);
    }
    // the interior position and, for a site on a face, the opposite ghost layer
    const int gx[3] = {x + 1, x == a.nx - 1 ? 0 : -1, x == 0 ? a.nx + 1 : -1};
    const int gy[3] = {y + 1, y == a.ny - 1 ? 0 : -1, y == 0 ? a.ny + 1 : -1};
    const int gz[3] = {z + 1, z == a.nz - 1 ? 0 : -1, z == 0 ? a.nz + 1 : -1};
    for (int iz = 0; iz < 3; ++iz) {
      if (gz[iz] < 0) continue;
      for (int iy = 0; iy < 3; ++iy) {
        if (gy[iy] < 0) continue;
        for (int ix = 0; ix < 3; ++ix) {
          if (gx[ix] < 0) continue;
#pragma unroll
          for (int q = 0; q < NC / 8; ++q)
            *reinterpret_cast<uint4*>(a.out_bf16 + act_off(gx[ix], gy[iy], gz[iz], c0 / 8 + q, COUT, px, py)) = pk[q];
        }
      }
    }
  }
}

// Epilogue of one output site: v[] holds the COUT accumulator values of site
// (x, y, z); residual and mask operands are read here.
template <int COUT, int EPI>
__device__ __forceinline__ void conv_epilogue(float (&v)[COUT], int x, int y, int z, const ConvArgs& a) {
  if (x >= a.nx || y >= a.ny) return;
  const int px = a.nx + 2, py = a.ny + 2;
  float bias[COUT];
  uint4 rsd[COUT / 8], msk[COUT / 8];
#pragma unroll
  for (int c = 0; c < COUT; ++c) bias[c] = (EPI & kEpiBias) ? a.bias[c] : 0.f;
#pragma unroll
  for (int q = 0; q < COUT / 8; ++q) {
    const long long o = act_off(x + 1, y + 1, z + 1, q, COUT, px, py);
    if (EPI & kEpiResid) rsd[q] = *reinterpret_cast<const uint4*>(a.resid + o);
    if (EPI & kEpiMask) msk[q] = *reinterpret_cast<const uint4*>(a.mask + o);
  }
  conv_epilogue_part<COUT, COUT, EPI>(v, bias, rsd, msk, 0, x, y, z, a);
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
      tma_load_4d(wsm, &tmW, 0, 0, 0, 0, wbar);
      int k = 0;
      for (int tile = blockIdx.x; tile < ntiles && !*abort_flag; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * 32, y0 = ((tile / tiles_x) % tiles_y) * 4, z0 = tile / (tiles_x * tiles_y);
        for (int t = 0; t < 27; ++t, ++k) {
          const int s = k % kConvStages;
          if (k >= kConvStages && !bounded_wait(&empty[s], ((k / kConvStages) - 1) & 1)) break;
          const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
          mbar_arrive_expect_tx(&full[s], L::STAGE);
          // one box per channel group: 32 sites x 8 channels (512 B rows) x 4 rows
          for (int q = 0; q < CIN / 8; ++q)
            tma_load_4d(stages + s * L::STAGE + q * 2048, &tmA, 8 * (x0 + 1 + dx), y0 + 1 + dy, q, z0 + 1 + dz,
                        &full[s]);
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
            // A: [group][128 sites][8 channels], 16 B per site; one K step = two groups
            const uint64_t ad = umma_sdesc_noswz(st_addr + s * L::STAGE + kk * 2 * 2048, 2048u, 128u);
            const uint64_t bd = umma_sdesc(w_addr + w_slot(t) * (COUT * CIN * 2) + kk * 32, L::SBO, L::SWZ);
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
// Window kernel: one staged input window per plane serves all 27 taps.
//
// The padded plane is indexed linearly, l = Y px + X.  An M tile is 128
// consecutive l; tap (dx, dy) of it is the same 128 rows shifted by
// dy px + dx.  Each input plane is staged once per tile as the window
// [l0 - px - 1, l0 + 128 + px + 1) in the no-swizzle K-major layout
// [channel group of 8][site][8 BF16] (16 B per site, so SBO = 128 B and any
// row shift is a 16-B shift of the descriptor's start address).  In the
// chunk-planar activation layout each group's window is one contiguous run,
// brought in by one bulk copy.  A CTA
// walks a contiguous range of (tile, z) items with z fastest, so consecutive
// items reuse two of their three planes; rows of a tile that fall on ghost
// positions (X or Y on the padding) are computed and discarded.
// ---------------------------------------------------------------------------
constexpr int kWinPipes = 2;   // independent pipelines per CTA (they share the weights)
constexpr int kWinSlots = 4;   // staged planes per pipeline
constexpr int kWinAcc = 4;     // accumulator stages per pipeline in tensor memory
// warps: 4 epilogue warps per pipeline (one TMEM lane quadrant each), then one
// producer and one MMA warp per pipeline
constexpr int kWinEpiWarps = 4 * kWinPipes;
constexpr int kWinThreads = 32 * (kWinEpiWarps + 2 * kWinPipes);

template <int CIN, int COUT>
struct WinSmem {
  static constexpr int CH = CIN / 8;  // 16-byte channel groups per site
  // per pipeline: full[S], empty[S], accf[A], acce[A], done; then wbar
  static constexpr int PBARS = 2 * kWinSlots + 2 * kWinAcc + 1;
  static constexpr int NBARS = kWinPipes * PBARS + 1;
  static constexpr uint32_t SWZ = CIN == 32 ? kSwizzle64B : kSwizzle32B;
  static constexpr uint32_t WSBO = 8 * CIN * 2;
  static constexpr uint32_t PIPE_COLS = kWinAcc * 2 * COUT;  // an accumulator stage holds two output planes
  static constexpr uint32_t TMEM_COLS = kWinPipes * PIPE_COLS < 32 ? 32 : kWinPipes * PIPE_COLS;
};

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kWinThreads) k_conv_win(const void* __restrict__ base,
                                                          const __grid_constant__ CUtensorMap tmW, ConvArgs a,
                                                          ConvWin g) {
  using L = WinSmem<CIN, COUT>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* wsm = smem + g.off_w;  // 1024-aligned
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + g.off_bars);
  uint64_t* wbar = bars + kWinPipes * L::PBARS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(wbar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // role and pipeline of this warp
  const int pipe = warp < kWinEpiWarps ? warp / 4 : (warp - kWinEpiWarps) % kWinPipes;
  unsigned char* slots = smem + (size_t)pipe * kWinSlots * g.slot_bytes;  // this pipeline's planes
  uint64_t* pb = bars + pipe * L::PBARS;
  uint64_t* full = pb;
  uint64_t* empty = pb + kWinSlots;
  uint64_t* accf = pb + 2 * kWinSlots;
  uint64_t* acce = accf + kWinAcc;
  uint64_t* done = acce + kWinAcc;

  // this pipeline's items: (tile T, plane pair k) with k fastest, a contiguous
  // share of the CTA's range; pair k is output planes 2k and 2k + 1 (2k alone
  // when nz is odd and k is the last); every role walks them with incremental
  // 32-bit counters
  const int npairs = (a.nz + 1) / 2;
  const long long items = (long long)g.ntiles * npairs;
  const long long cbeg = items * blockIdx.x / gridDim.x, cend = items * (blockIdx.x + 1) / gridDim.x;
  const long long jbeg = cbeg + (cend - cbeg) * pipe / kWinPipes;
  const long long jend = cbeg + (cend - cbeg) * (pipe + 1) / kWinPipes;
  const int nitems = (int)(jend - jbeg);
  const int T0 = (int)(jbeg / npairs), k0 = (int)(jbeg % npairs);
  const long long plane = (long long)g.px * g.py;

  if (threadIdx.x == 0) {
    for (int p = 0; p < kWinPipes; ++p) {
      uint64_t* q = bars + p * L::PBARS;
      for (int i = 0; i < kWinSlots; ++i) {
        mbar_init(&q[i], 1);
        mbar_init(&q[kWinSlots + i], 1);
      }
      for (int i = 0; i < kWinAcc; ++i) {
        mbar_init(&q[2 * kWinSlots + i], 1);
        mbar_init(&q[2 * kWinSlots + kWinAcc + i], 128);
      }
      mbar_init(&q[2 * kWinSlots + 2 * kWinAcc], 1);
    }
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
  const uint32_t tmem_base = *tmem_slot + (uint32_t)pipe * L::PIPE_COLS;

  auto bounded_wait = [&](uint64_t* bar, uint32_t parity) {
    if (*abort_flag) return false;
    if (!mbar_wait_bounded(bar, parity, kConvWaitNs)) {
      *abort_flag = 1;
      atomicExch(a.err, 1);
      return false;
    }
    return true;
  };

  if (warp >= kWinEpiWarps && warp < kWinEpiWarps + kWinPipes) {
    // ---------------- TMA producer: planes in the order the items need them
    if (lane == 0) {
      if (pipe == 0) {
        tma_prefetch_desc(&tmW);
        mbar_arrive_expect_tx(wbar, 27 * COUT * CIN * 2);
        tma_load_4d(wsm, &tmW, 0, 0, 0, 0, wbar);
      }
      const uint32_t tx_bytes = (uint32_t)(L::CH * g.wb * 16);
      const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(base);
      int sl = 0;        // slot of the next plane load
      uint32_t eph = 0;  // parity of that slot's next release
      int nloads = 0;
      bool ok = true;
      int T = T0, k = k0;
      for (int it = 0; ok && it < nitems; ++it) {
        const int zA = 2 * k;
        const bool first = it == 0 || k == 0;
        // window start inside a plane: first row of the tile minus px + 1
        const long long w0 = (long long)g.l_first + (long long)T * 128 - (g.px + 1);
        // padded planes zA .. zA+3 hold input planes zA-1 .. zA+2 (zA .. zA+2 for a lone plane);
        // a pair continuing the previous one shares its first two
        const int zlast = zA + (zA + 1 < a.nz ? 3 : 2);
        for (int Z = first ? zA : zA + 2; Z <= zlast; ++Z) {
          if (nloads >= kWinSlots && !bounded_wait(&empty[sl], eph)) {
            ok = false;
            break;
          }
          unsigned char* dst = slots + (size_t)sl * g.slot_bytes;
          mbar_arrive_expect_tx(&full[sl], tx_bytes);
          for (int c = 0; c < L::CH; ++c)
            bulk_load(dst + (size_t)c * g.lbo, src + ((long long)Z * L::CH + c) * plane * 8 + w0 * 8, g.wb * 16,
                      &full[sl]);
          ++nloads;
          if (++sl == kWinSlots) {
            sl = 0;
            if (nloads > kWinSlots) eph ^= 1u;  // load n waits for release n - S: parity (n / S - 1) & 1
          }
        }
        if (++k == npairs) {
          k = 0;
          ++T;
        }
      }
      if (!ok) {
        // let copies still in flight land before the CTA's shared memory goes away
        for (int i = 0; i < kWinSlots; ++i) {
          mbar_wait_bounded(&full[i], 0, kConvWaitNs / 16);
          mbar_wait_bounded(&full[i], 1, kConvWaitNs / 16);
        }
      }
    }
  } else if (warp >= kWinEpiWarps + kWinPipes) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc1 = umma_idesc_bf16(128, COUT), idesc2 = umma_idesc_bf16(128, 2 * COUT);
      // descriptors are advanced by adding (byte offset >> 4) to the start-address field
      const uint64_t bdesc0 = umma_sdesc(smem_addr(wsm), L::WSBO, L::SWZ);
      const uint64_t adesc0 = umma_sdesc_noswz(smem_addr(slots), g.lbo, 128u);
      const uint32_t slot16 = g.slot_bytes >> 4, lbo16 = g.lbo >> 4;
      const int px = g.px;
      // weights of in-plane shift sh and z-offset dz, K chunk kc (staged [shift][dz][C_out][C_in])
      auto wdesc = [&](int sh, int dz, int kc) {
        return bdesc0 + (uint64_t)((((sh * 3 + dz + 1) * (COUT * CIN * 2)) + kc * 32) >> 4);
      };
      // row shift of in-plane shift sh in 16-byte units: px + 1 + dy px + dx
      auto row16 = [&](int sh) { return (uint32_t)(px + 1 + (sh / 3 - 1) * px + (sh % 3 - 1)); };
      bool ok = bounded_wait(wbar, 0);
      // ring state of the loads: the planes of the current item, oldest first
      int ps[4] = {0, 0, 0, 0};
      uint32_t pph[4] = {0, 0, 0, 0};
      int nsl = 0;       // slot of the next load to consume
      uint32_t nph = 0;  // its full-barrier parity
      int acc = 0;
      uint32_t aph = 0;  // accumulator-free parity
      int k = k0;
      for (int it = 0; ok && it < nitems; ++it) {
        const int zA = 2 * k;
        const bool pair = zA + 1 < a.nz, first = it == 0 || k == 0;
        const int np = pair ? 4 : 3;
        if (!first) {
          ps[0] = ps[2];
          pph[0] = pph[2];
          ps[1] = ps[3];
          pph[1] = pph[3];
        }
        for (int d = first ? 0 : 2; d < np; ++d) {
          ps[d] = nsl;
          pph[d] = nph;
          if (++nsl == kWinSlots) {
            nsl = 0;
            nph ^= 1u;
          }
        }
        if (it >= kWinAcc && !bounded_wait(&acce[acc], aph ^ 1u)) break;
        // planes already seen complete by the previous item stay loaded until released
        for (int d = first ? 0 : 2; d < np; ++d)
          if (!bounded_wait(&full[ps[d]], pph[d])) ok = false;
        if (!ok) break;
        tc_fence_after();
        // accumulator stage: block 0 (columns [0, COUT)) = output plane zA+1, block 1 = zA
        const uint32_t d0 = tmem_base + acc * 2 * COUT, d1 = d0 + COUT;
        uint64_t ab[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) ab[d] = adesc0 + (uint64_t)ps[d] * slot16;
        if (pair) {
          // input plane zA-1 feeds plane zA only (dz = -1), into block 1
#pragma unroll
          for (int sh = 0; sh < 9; ++sh)
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc)
              umma_bf16(d1, ab[0] + row16(sh) + 2u * kc * lbo16, wdesc(sh, -1, kc), idesc1,
                        (sh > 0 || kc > 0) ? 1u : 0u);
          umma_commit(&empty[ps[0]]);
          // input plane zA+2 feeds plane zA+1 only (dz = +1), into block 0
#pragma unroll
          for (int sh = 0; sh < 9; ++sh)
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc)
              umma_bf16(d0, ab[3] + row16(sh) + 2u * kc * lbo16, wdesc(sh, 1, kc), idesc1,
                        (sh > 0 || kc > 0) ? 1u : 0u);
          // input plane zA feeds both: B rows [W(dz = -1); W(dz = 0)] -> blocks 0 (zA+1) and 1 (zA)
#pragma unroll
          for (int sh = 0; sh < 9; ++sh)
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc)
              umma_bf16(d0, ab[1] + row16(sh) + 2u * kc * lbo16, wdesc(sh, -1, kc), idesc2, 1u);
          umma_commit(&empty[ps[1]]);
          // input plane zA+1 feeds both: B rows [W(dz = 0); W(dz = +1)] -> blocks 0 (zA+1) and 1 (zA)
#pragma unroll
          for (int sh = 0; sh < 9; ++sh)
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc)
              umma_bf16(d0, ab[2] + row16(sh) + 2u * kc * lbo16, wdesc(sh, 0, kc), idesc2, 1u);
        } else {
          // a lone plane zA: all 27 taps from input planes zA-1 .. zA+1, into block 1
#pragma unroll
          for (int t = 0; t < 27; ++t) {
            const int sh = t % 9, dz = t / 9 - 1;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc)
              umma_bf16(d1, ab[dz + 1] + row16(sh) + 2u * kc * lbo16, wdesc(sh, dz, kc), idesc1,
                        (t > 0 || kc > 0) ? 1u : 0u);
          }
          umma_commit(&empty[ps[0]]);
          umma_commit(&empty[ps[1]]);
        }
        umma_commit(&accf[acc]);
        if (++acc == kWinAcc) {
          acc = 0;
          aph ^= 1u;
        }
        if (++k == npairs) k = 0;
        // release the planes the next item does not share with this one
        const bool cont = it + 1 < nitems && k != 0;
        if (!cont) {
          umma_commit(&empty[ps[2]]);
          if (pair) umma_commit(&empty[ps[3]]);
        }
      }
      // every issued MMA has finished before the CTA leaves
      umma_commit(done);
      mbar_wait_bounded(done, 0, kConvWaitNs);
    }
  } else {
    // ---------------- epilogue: 4 warps per pipeline; warp w reads TMEM lanes 32 (w % 4) ..
    // (one row of the tile each), all COUT channels
    const int quad = warp % 4;
    const int m = quad * 32 + lane;
    float bias[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) bias[c] = (EPI & kEpiBias) ? a.bias[c] : 0.f;
    int T = T0, k = k0;
    // padded (X, Y) of this thread's row of tile T, advanced by 128 positions per tile
    int l = g.l_first + T * 128 + m;
    int Y = l / g.px, X = l - Y * g.px;
    int acc = 0;
    uint32_t fph = 0;
    // this thread's accumulator row of block b (COUT columns) of the current stage
    auto read_block = [&](int b, float (&v)[COUT]) {
      const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + acc * 2 * COUT + b * COUT;
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
    };
    // residual / mask operands of plane z (they do not depend on the accumulator)
    auto operands = [&](int z, uint4 (&rsd)[COUT / 8], uint4 (&msk)[COUT / 8]) {
#pragma unroll
      for (int q = 0; q < COUT / 8; ++q) {
        const long long o = act_off(X, Y, z + 1, q, COUT, g.px, g.py);
        if (EPI & kEpiResid) rsd[q] = *reinterpret_cast<const uint4*>(a.resid + o);
        if (EPI & kEpiMask) msk[q] = *reinterpret_cast<const uint4*>(a.mask + o);
      }
    };
    for (int it = 0; it < nitems; ++it) {
      const int zA = 2 * k;
      const bool pair = zA + 1 < a.nz;
      const bool real = X >= 1 && X <= g.px - 2 && Y >= 1 && Y <= g.py - 2;
      uint4 rsd[COUT / 8], msk[COUT / 8];
      if (real) operands(zA, rsd, msk);
      const bool ok = __all_sync(0xffffffffu, bounded_wait(&accf[acc], fph));
      if (!ok) break;
      tc_fence_after();
      // block 1 holds plane zA, block 0 plane zA+1 (of a pair)
      float v[COUT], v2[COUT];
      read_block(1, v);
      if (pair) read_block(0, v2);
      tc_fence_before();
      mbar_arrive(&acce[acc]);
      if (real) conv_epilogue_part<COUT, COUT, EPI>(v, bias, rsd, msk, 0, X - 1, Y - 1, zA, a);
      if (real && pair) {
        operands(zA + 1, rsd, msk);
        conv_epilogue_part<COUT, COUT, EPI>(v2, bias, rsd, msk, 0, X - 1, Y - 1, zA + 1, a);
      }
      if (++acc == kWinAcc) {
        acc = 0;
        fph ^= 1u;
      }
      if (++k == npairs) {
        k = 0;
        X += 128;
        while (X >= g.px) {
          X -= g.px;
          ++Y;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(*tmem_slot, L::TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// host launch
// ---------------------------------------------------------------------------
template <int CIN, int COUT, int EPI>
cudaError_t conv_launch_t(const CUtensorMap& tmA, const CUtensorMap& tmW, const ConvArgs& a, int sms,
                          cudaStream_t s) {
  const int max_ctas = 2 * sms;  // two CTAs fit an SM
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

bool conv_win_geometry(int cin, int cout, int nx, int ny, ConvWin* g, size_t* smem_bytes) {
  ConvWin w{};
  w.px = nx + 2;
  w.py = ny + 2;
  w.l_first = w.px + 1;
  const long long span = (long long)(w.py - 2) * w.px - 2;  // linear positions from the first to the last interior site
  w.ntiles = (int)((span + 127) / 128);
  const int W = 128 + 2 * (w.px + 1);  // window length in sites
  w.wb = (W + 7) / 8 * 8;
  // the last window of a buffer may run past its last group: stay within the tail
  const long long over = (long long)w.l_first + (long long)(w.ntiles - 1) * 128 - (w.px + 1) + w.wb -
                         (long long)w.px * w.py;
  if (over * 16 > (long long)kActTailBytes) return false;
  w.lbo = (uint32_t)w.wb * 16;
  w.slot_bytes = (uint32_t)(cin / 8) * w.lbo;
  const uint32_t slots = kWinPipes * kWinSlots * w.slot_bytes;
  w.off_w = (slots + 1023) / 1024 * 1024;
  const uint32_t wbytes = ((27 * cout * cin * 2 + 1023) / 1024) * 1024;
  w.off_bars = w.off_w + wbytes;
  const int nbars = kWinPipes * (2 * kWinSlots + 2 * kWinAcc + 1) + 1;
  const size_t need = (size_t)w.off_bars + nbars * 8 + 16 + 1024;  // + base alignment
  if (need > 227 * 1024) return false;
  *g = w;
  *smem_bytes = need;
  return true;
}

template <int CIN, int COUT, int EPI>
cudaError_t conv_launch_win_t(const void* base, const CUtensorMap& tmW, const ConvArgs& a, const ConvWin& g,
                              size_t smem, int sms, cudaStream_t s) {
  static size_t attr = 0;
  static int per_sm = 1;
  if (attr < smem) {
    cudaError_t e =
        cudaFuncSetAttribute(k_conv_win<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv_win<CIN, COUT, EPI>, kWinThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    attr = smem;
  }
  // one wave of persistent CTAs, each taking an equal share of the (tile, plane pair)
  // items; a CTA's accumulators may fill the SM's 512 tensor-memory columns
  const long long items = (long long)g.ntiles * ((a.nz + 1) / 2);
  const int tmem_per_sm = std::max(1, 512 / (int)WinSmem<CIN, COUT>::TMEM_COLS);
  const int grid = (int)std::min<long long>(items, (long long)std::min(per_sm, tmem_per_sm) * sms);
  k_conv_win<CIN, COUT, EPI><<<grid, kWinThreads, smem, s>>>(base, tmW, a, g);
  return cudaGetLastError();
}

cudaError_t conv_launch(int cin, int cout, int epi, const ConvMaps& m, bool allow_win, const CUtensorMap& tmW,
                        const ConvArgs& a, int sms, cudaStream_t s) {
  ConvWin g;
  size_t smem = 0;
  if (allow_win && m.use_win && conv_win_geometry(cin, cout, a.nx, a.ny, &g, &smem)) {
#define LCBP_CONV_WIN_CASE(CI, CO, E) \
  if (cin == CI && cout == CO && epi == (E)) return conv_launch_win_t<CI, CO, E>(m.base, tmW, a, g, smem, sms, s);
    LCBP_CONV_WIN_CASE(16, 32, kEpiBias | kEpiRelu)
    LCBP_CONV_WIN_CASE(32, 32, kEpiBias | kEpiRelu)
    LCBP_CONV_WIN_CASE(32, 32, kEpiBias | kEpiResid)
    LCBP_CONV_WIN_CASE(32, 16, kEpiBias | kEpiOutF32)
    LCBP_CONV_WIN_CASE(32, 16, kEpiBias | kEpiUpdateQ)
    LCBP_CONV_WIN_CASE(16, 32, 0)
    LCBP_CONV_WIN_CASE(32, 32, kEpiMask)
    LCBP_CONV_WIN_CASE(32, 32, kEpiResid)
    LCBP_CONV_WIN_CASE(32, 32, kEpiResid | kEpiMask)
    LCBP_CONV_WIN_CASE(32, 32, 0)
#undef LCBP_CONV_WIN_CASE
    return cudaErrorInvalidValue;
  }
  const CUtensorMap& tmA = m.tile;
#define LCBP_CONV_CASE(CI, CO, E) \
  if (cin == CI && cout == CO && epi == (E)) return conv_launch_t<CI, CO, E>(tmA, tmW, a, sms, s);
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
