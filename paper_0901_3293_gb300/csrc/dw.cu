// Weight gradient of a periodic 3x3x3 convolution on tcgen05 tensor cores.
//
//   dW[t][ci][co] = sum_r X(r + o_t)[ci] dY(r)[co],   db[co] = sum_r dY(r)[co]
//
// over the interior sites r, for BF16 activations X (C_in channels) and
// upstream gradients dY (C_out channels) in the padded chunk-planar layout of
// conv.h.  As a GEMM the reduction runs over sites: K = sites, and both
// operands hold 8 channels per 16-byte site, i.e. they are MN-major.
//
// Work item: 128 consecutive linear positions l0 .. l0+127 of one padded
// plane Z (straddling rows; ghost positions are masked).  For it the CTA
// stages, for dz = -1, 0, 1 and every channel group g, the window
// [l0 - px - 1, l0 + 128 + px + 1) of plane Z + dz, each at its own slot of a
// uniform stride W sites, slot = 3-group index (dz + 1) C_in / 8 + g.  The A
// operand of one MMA is then 128 rows = (dz, ci) (rows past 3 C_in are spare),
// and an in-plane tap (dx, dy) is the same operand at a start address
// 16 B x ((dy + 1) px + dx + 1) further: one MMA with M = 128, N = C_out,
// K = 16 applies the three taps (dx, dy, -1..1) at once.  B is the dY tile of
// the item, with dY zeroed by the CTA at ghost positions and past the last
// interior position.  Slot 12 of A holds ones, so row 96 of every
// accumulator is sum_k dY: the bias gradient.  The nine in-plane shifts
// accumulate into nine TMEM blocks of C_out columns over all of a CTA's
// items; the CTA then writes its partial sums, and a second kernel adds the
// partials of all CTAs in a fixed order (deterministic).
//
// Only slots 0..12 are staged per stage; rows 104..127 of the A operand (the
// spare slots 13..15) read whatever follows (the stage's dY tile, the next
// stage, or padding) into accumulator rows that are never read.  That keeps
// three stages in shared memory for planes up to 64 sites wide.
//
// Warp roles (256 threads): warps 0-3 mask dY and run the epilogue (TMEM
// lanes 0..127), warp 4 copies (cp.async.bulk), warps 5-7 issue the MMAs,
// each the three shifts of one dx into its own accumulator blocks: one
// issuing thread cannot keep the tensor core busy with N = C_out MMAs.
// Every barrier wait is bounded; a timeout sets the error flag.
#include <cuda_bf16.h>

#include "conv.h"
#include "tc.cuh"

namespace lcbp {

namespace {

constexpr int kDwIssuers = 3;  // MMA-issuing warps (one per dx)
constexpr int kDwThreads = 32 * (5 + kDwIssuers);
constexpr int kDwMaxStages = 3;
constexpr int kDwSlots = 16;     // A operand rows: 16 slots of W sites (rows 8 slot .. 8 slot + 7)
constexpr int kDwStaged = 13;    // slots staged per stage (the last is the ones slot)
constexpr int kDwOnesSlot = 12;  // rows 96..103: ones
constexpr uint64_t kDwWaitNs = 2000000000ull;

struct DwGeom {
  int px, py;
  int l_first, l_last;  // first / last interior linear position of a padded plane
  int tiles;            // 128-position items per plane
  int items;            // tiles * nz
  int W;                // window sites per slot (multiple of 8)
  int stages;           // pipeline stages (3 where they fit, else 2)
  uint32_t a_bytes, b_bytes, stage_bytes, off_bars;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kDwThreads, 1) k_dw_tc(const __nv_bfloat16* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ dY, DwGeom g,
                                                         float* __restrict__ partial, int* __restrict__ err) {
  constexpr int CG = CIN / 8, OG = COUT / 8;
  constexpr int NOUT = 27 * CIN * COUT + COUT;  // values of one CTA's partial
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + g.off_bars);
  const int stages = g.stages;
  uint64_t* full = bars;                      // [stages]: copies landed
  uint64_t* masked = bars + kDwMaxStages;     // [stages]: dY masked (128 arrivals)
  uint64_t* empty = bars + 2 * kDwMaxStages;  // [stages]: every issuer's MMAs done with the stage
  uint64_t* done = bars + 3 * kDwMaxStages;   // all MMAs done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int i0 = (int)((long long)g.items * blockIdx.x / gridDim.x);
  const int i1 = (int)((long long)g.items * (blockIdx.x + 1) / gridDim.x);
  const int nit = i1 - i0;
  const long long plane = (long long)g.px * g.py;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&masked[s], 128);
      mbar_init(&empty[s], kDwIssuers);
    }
    mbar_init(done, kDwIssuers);
    *abort_flag = 0;
    mbar_init_fence();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  // the ones slot of every stage (read by the MMAs through the async proxy)
  if (warp < 4) {
    const uint4 one = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);  // eight BF16 1.0
    for (int s = 0; s < stages; ++s) {
      uint4* o = reinterpret_cast<uint4*>(smem + s * g.stage_bytes + (size_t)kDwOnesSlot * g.W * 16);
      for (int k = threadIdx.x; k < g.W; k += 128) o[k] = one;
    }
    fence_proxy_async();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto bounded_wait = [&](uint64_t* bar, uint32_t parity) {
    if (*abort_flag) return false;
    if (!mbar_wait_bounded(bar, parity, kDwWaitNs)) {
      *abort_flag = 1;
      atomicExch(err, 1);
      return false;
    }
    return true;
  };
  auto item_l0 = [&](int item) { return g.l_first + (item % g.tiles) * 128; };
  auto item_Z = [&](int item) { return item / g.tiles + 1; };  // padded plane of the output sites

  if (warp == 4) {
    // ---------------- producer: the three plane windows and the dY tile of each item
    if (lane == 0) {
      const uint32_t tx = (uint32_t)(3 * CG * g.W * 16 + OG * 128 * 16);
      for (int it = 0; it < nit; ++it) {
        const int s = it % stages;
        if (it >= stages && !bounded_wait(&empty[s], ((it / stages) - 1) & 1)) break;
        const int item = i0 + it, Z = item_Z(item), l0 = item_l0(item);
        unsigned char* st = smem + s * g.stage_bytes;
        mbar_arrive_expect_tx(&full[s], tx);
        for (int dz = 0; dz < 3; ++dz)
          for (int q = 0; q < CG; ++q) {
            const __nv_bfloat16* src = X + (((long long)(Z + dz - 1) * CG + q) * plane + (l0 - g.px - 1)) * 8;
            bulk_load(st + (size_t)(dz * CG + q) * g.W * 16, src, (uint32_t)(g.W * 16), &full[s]);
          }
        for (int q = 0; q < OG; ++q) {
          const __nv_bfloat16* src = dY + (((long long)Z * OG + q) * plane + l0) * 8;
          bulk_load(st + g.a_bytes + q * 2048, src, 2048u, &full[s]);
        }
      }
    }
  } else if (warp >= 5) {
    // ---------------- MMA issuers: warp 5 + j issues the shifts sh = 3 (dy + 1) + j
    // (dx = j - 1) into accumulator blocks sh of C_out columns
    if (lane == 0) {
      const int j = warp - 5;
      constexpr uint32_t idesc = umma_idesc_bf16(128, COUT) | (1u << 15) | (1u << 16);  // A, B MN-major
      // MN-major, no swizzle: 8-site core-matrix columns 128 B apart along K,
      // 8-row groups one slot (A) / one channel group (B) apart along M / N.
      // A shifted or later operand is the same descriptor with its start
      // address (bits 0-13, in 16-byte units) advanced: shared addresses stay
      // below 256 KB, so the sum never carries out of that field.
      const uint64_t ad0 = umma_sdesc_noswz(smem_addr(smem), 128u, (uint32_t)g.W * 16u);
      const uint64_t bd0 = umma_sdesc_noswz(smem_addr(smem) + g.a_bytes, 128u, 2048u);
      for (int it = 0; it < nit; ++it) {
        const int s = it % stages;
        if (!bounded_wait(&masked[s], (it / stages) & 1)) break;
        tc_fence_after();
        const uint64_t so = (uint64_t)((s * g.stage_bytes) >> 4);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const uint64_t ad = ad0 + so + (uint64_t)(r * g.px + j);  // window offset (dy + 1) px + (dx + 1)
          const uint32_t d = tmem_base + (uint32_t)(3 * r + j) * COUT;
#pragma unroll
          for (int kk = 0; kk < 8; ++kk)
            umma_bf16(d, ad + (uint64_t)(kk * 16), bd0 + so + (uint64_t)(kk * 16), idesc, (it > 0 || kk > 0) ? 1u : 0u);
        }
        umma_commit(&empty[s]);
      }
      umma_commit(done);
    }
  } else {
    // ---------------- warps 0-3: zero dY at ghost positions and past the last
    // interior position, then (after all items) the epilogue
    const int k = threadIdx.x;  // position within the item
    for (int it = 0; it < nit; ++it) {
      const int s = it % stages;
      if (!bounded_wait(&full[s], (it / stages) & 1)) break;
      const int l = item_l0(i0 + it) + k, xg = l % g.px;
      if (l > g.l_last || xg == 0 || xg == g.px - 1) {
        unsigned char* b = smem + s * g.stage_bytes + g.a_bytes;
#pragma unroll
        for (int q = 0; q < OG; ++q) *reinterpret_cast<uint4*>(b + q * 2048 + k * 16) = make_uint4(0, 0, 0, 0);
      }
      fence_proxy_async();
      mbar_arrive(&masked[s]);
    }
    // wait for the MMAs to finish even after an abort (the tensor memory is
    // released below), then read the accumulators unless something timed out
    const bool landed = mbar_wait_bounded(done, 0, kDwWaitNs);
    if (!landed) atomicExch(err, 1);
    const bool ok = __all_sync(0xffffffffu, landed && !*abort_flag);
    if (ok) {
      tc_fence_after();
      const int m = warp * 32 + lane;  // accumulator row = TMEM lane
      float* out = partial + (size_t)blockIdx.x * NOUT;
#pragma unroll 1
      for (int sh = 0; sh < 9; ++sh) {
        float v[COUT];
        const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + sh * COUT;
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
        if (m < 3 * CIN) {
          const int t = 9 * (m / CIN) + sh, ci = m % CIN;
#pragma unroll
          for (int c = 0; c < COUT; ++c) out[((size_t)t * COUT + c) * CIN + ci] = v[c];  // lanes: consecutive ci
        } else if (m == 8 * kDwOnesSlot && sh == 0) {
#pragma unroll
          for (int c = 0; c < COUT; ++c) out[27 * CIN * COUT + c] = v[c];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
  }
}

// dW += sum over parts of the partials, db likewise, in a fixed order: a
// block takes 32 consecutive values; warp w adds parts w, w + 8, w + 16, ...
// in turn (coalesced 128-byte rows), then thread l of warp 0 adds the eight
// warps' sums in warp order.  A CTA's partial holds the weight gradients as
// [tap][C_out][C_in] (its epilogue threads are the C_in rows, so each of its
// stores is one coalesced row) and then the C_out bias gradients.
constexpr int kRedWarps = 8;
__global__ void __launch_bounds__(32 * kRedWarps) k_dw_reduce(const float* __restrict__ partial, int nparts, int cin,
                                                              int cout, float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float red[kRedWarps][32];
  const int nw = 27 * cin * cout, count = nw + cout;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int i = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (i < count) {
#pragma unroll 4
    for (int p = warp; p < nparts; p += kRedWarps) s += partial[(size_t)p * count + i];
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && i < count) {
    float t = red[0][lane];
#pragma unroll
    for (int w = 1; w < kRedWarps; ++w) t += red[w][lane];
    if (i < nw) {
      const int tap = i / (cin * cout), r = i % (cin * cout), co = r / cin, ci = r % cin;
      dW[((size_t)tap * cin + ci) * cout + co] += t;
    } else {
      db[i - nw] += t;
    }
  }
}

size_t dw_smem_bytes(const DwGeom& g) {
  return (size_t)g.off_bars + (3 * kDwMaxStages + 1) * 8 + 16 + 1024;
}

bool dw_geometry(int cin, int cout, int nx, int ny, int nz, DwGeom* g, size_t* smem) {
  g->px = nx + 2;
  g->py = ny + 2;
  g->l_first = g->px + 1;
  g->l_last = ny * g->px + nx;
  g->tiles = (g->l_last - g->l_first + 128) / 128;
  g->items = g->tiles * nz;
  g->W = ((128 + 2 * g->px + 2) + 7) / 8 * 8;
  g->a_bytes = (uint32_t)kDwStaged * g->W * 16;
  g->b_bytes = (uint32_t)(cout / 8) * 2048;
  g->stage_bytes = (g->a_bytes + g->b_bytes + 1023) / 1024 * 1024;
  for (g->stages = kDwMaxStages; g->stages >= 2; --g->stages) {
    // after the last stage: its spare A slots (13..15), which the MMAs read,
    // and 4 KB so that the last B core matrices of a stage stay inside the
    // allocation under either reading of the operand strides
    g->off_bars = g->stages * g->stage_bytes + (uint32_t)(kDwSlots - kDwStaged) * g->W * 16 + 4096;
    *smem = dw_smem_bytes(*g);
    if (*smem <= 227 * 1024) break;
  }
  (void)cin;
  return g->stages >= 2 && *smem <= 227 * 1024 && g->W < 16384;
}

}  // namespace

size_t dw_partial_floats(int sms) { return (size_t)sms * (27 * 32 * 32 + 32); }

bool dw_fits(int cin, int cout, int nx, int ny, int nz) {
  DwGeom g;
  size_t smem = 0;
  return dw_geometry(cin, cout, nx, ny, nz, &g, &smem);
}

template <int CIN, int COUT>
static cudaError_t dw_launch_t(const __nv_bfloat16* X, const __nv_bfloat16* dY, int nx, int ny, int nz, float* partial,
                               float* dW, float* db, int* err, int sms, cudaStream_t s) {
  DwGeom g;
  size_t smem = 0;
  if (!dw_geometry(CIN, COUT, nx, ny, nz, &g, &smem)) return cudaErrorInvalidValue;
  // at least 120 KB: one CTA per SM, so the CTA's 512 tensor-memory columns are never contended
  if (smem < 120 * 1024) smem = 120 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_dw_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = g.items < sms ? g.items : sms;
  k_dw_tc<CIN, COUT><<<grid, kDwThreads, smem, s>>>(X, dY, g, partial, err);
  const int nw = 27 * CIN * COUT;
  k_dw_reduce<<<(nw + COUT + 31) / 32, 32 * kRedWarps, 0, s>>>(partial, grid, CIN, COUT, dW, db);
  return cudaGetLastError();
}

cudaError_t dw_launch(int cin, int cout, const __nv_bfloat16* X, const __nv_bfloat16* dY, int nx, int ny, int nz,
                      float* partial, float* dW, float* db, int* err, int sms, cudaStream_t s) {
  if (cin == 32 && cout == 32) return dw_launch_t<32, 32>(X, dY, nx, ny, nz, partial, dW, db, err, sms, s);
  if (cin == 16 && cout == 32) return dw_launch_t<16, 32>(X, dY, nx, ny, nz, partial, dW, db, err, sms, s);
  if (cin == 32 && cout == 16) return dw_launch_t<32, 16>(X, dY, nx, ny, nz, partial, dW, db, err, sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace lcbp
