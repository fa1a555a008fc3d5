// Fast path of the coupled step: two z-marching kernels with TMA-staged planes.
//
//   k_qside  (Q^n, rho u^n)            -> sigma_LC, b, Q*            (88 B/site FP32)
//            H, sigma_LC, tau and the body force b = D0_b tau_ab - H_gn D0_a Q_gn,
//            then the Heun predictor Q* = Q + R(Q, u)   (Sec. 2.1 Eq. Qevolution,
//            mat_der, BEstress; Sec. 2.2 Eq. eq7a, spurious)
//   k_lbq    (f^n, rho u^n, sigma, b, Q*, Q^n) -> f^{n+1}, rho u^{n+1}, Q^{n+1}   (244 B/site FP32)
//            predictor-corrector D3Q15 LB (Sec. 2.2 Eq. eq2, eq4, feq, coeff) and the
//            Heun corrector Q^{n+1} = (Q + Q* + R(Q*)) / 2
//
// A CTA owns a column tile of TX x TY sites and marches through ZC planes.
// Planes of the fields it reads with a halo are brought into shared memory
// by 4-D TMA tile loads (x, y, z, component) into a ring of slots, each slot
// with its own mbarrier; the load of a plane is issued one or two planes
// before the CTA needs it, so HBM traffic overlaps compute.  A TMA box is 40
// elements wide (x0-4 .. x0+35, 16-byte aligned start); out-of-range halo
// cells of edge tiles are zero-filled by TMA and then overwritten with their
// periodic images by plain loads.  Populations are pulled straight from
// global memory (each is used once).
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace lcbp {

constexpr int ZM_TX = 32;   // tile width in x (one warp)
constexpr int ZM_BX = 40;   // TMA box width in elements
constexpr int ZM_XOFF = 4;  // box column of global x0
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on any barrier wait

__host__ __device__ constexpr int align_elems(int elems, int esize) {
  // round an element count up so that it spans a multiple of 128 bytes
  return ((elems * esize + 127) / 128) * 128 / esize;
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Overwrite out-of-range cells of a TMA-loaded plane with periodic images.
// Layout [comp][row][ZM_BX]; row r <-> global y = gy0 + r, column c <->
// global x = x0 - ZM_XOFF + c; only columns [c0, c1) are needed.
template <typename real>
__device__ void patch_plane(real* slot, int ncomp, int rows, int c0, int c1, const real* __restrict__ g, long long n,
                            int nx, int ny, int gz, int x0, int gy0) {
  const int w = c1 - c0;
  const int cells = rows * w;
  for (int t = threadIdx.x; t < cells; t += blockDim.x) {
    const int r = t / w, c = c0 + t % w;
    const int gx = x0 - ZM_XOFF + c, gy = gy0 + r;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) continue;
    const long long s = ((long long)gz * ny + wrap(gy, ny)) * nx + wrap(gx, nx);
    for (int k = 0; k < ncomp; ++k) slot[(k * rows + r) * ZM_BX + c] = g[k * n + s];
  }
}

template <typename real>
__device__ __forceinline__ Sym5<real> ld5(const real* sl, int comp_stride, int idx) {
  Sym5<real> v;
  v.xx = sl[idx];
  v.xy = sl[comp_stride + idx];
  v.xz = sl[2 * comp_stride + idx];
  v.yy = sl[3 * comp_stride + idx];
  v.yz = sl[4 * comp_stride + idx];
  return v;
}

// ---------------------------------------------------------------------------
// Kernel A: H, sigma, tau, b and the Heun predictor
// ---------------------------------------------------------------------------
template <typename real, int TY>
struct QsideSmem {
  static constexpr int QROWS = TY + 4, UROWS = TY + 2, TROWS = TY + 2, TCOLS = ZM_TX + 2;
  static constexpr int QSLOTS = 5, USLOTS = 4;
  static constexpr int QCS = QROWS * ZM_BX, UCS = UROWS * ZM_BX;  // per-component strides
  static constexpr int QSLOT = align_elems(5 * QCS, sizeof(real)), USLOT = align_elems(4 * UCS, sizeof(real));
  static constexpr int TSLOT = 3 * TROWS * TCOLS, HSLOT = 5 * TY * ZM_TX;
  static constexpr int OFF_U = QSLOTS * QSLOT, OFF_T = OFF_U + USLOTS * USLOT;
  static constexpr int OFF_H = OFF_T + 3 * TSLOT, OFF_BAR = align_elems(OFF_H + 2 * HSLOT, sizeof(real));
  static constexpr size_t bytes = sizeof(real) * (size_t)OFF_BAR + 16 * 8 + 16;
};

template <typename real, int TY>
__global__ void __launch_bounds__(ZM_TX* TY) k_qside(const __grid_constant__ CUtensorMap tmQ,
                                                     const __grid_constant__ CUtensorMap tmU, ZmGeom G,
                                                     Model<real> m, const real* __restrict__ Q,
                                                     const real* __restrict__ rhou, const real* __restrict__ bext,
                                                     real* __restrict__ sigma, real* __restrict__ bout,
                                                     real* __restrict__ Qs, int* __restrict__ err) {
  using L = QsideSmem<real, TY>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* base = reinterpret_cast<real*>(smem_raw);
  real* qring = base;
  real* uring = base + L::OFF_U;
  real* tring = base + L::OFF_T;
  real* hbuf = base + L::OFF_H;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L::OFF_BAR);  // 5 Q + 4 u
  int* abort_flag = reinterpret_cast<int*>(bars + 16);

  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const long long n = G.n;
  const int bt = blockIdx.x;
  const int x0 = (bt % G.tiles_x) * ZM_TX;
  const int y0 = ((bt / G.tiles_x) % G.tiles_y) * TY;
  const int z0 = (bt / (G.tiles_x * G.tiles_y)) * G.zc;
  const int z1 = min(z0 + G.zc, nz);
  const int tx = threadIdx.x % ZM_TX, ty = threadIdx.x / ZM_TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < nx && gy < ny;
  const bool edge_q = x0 - 2 < 0 || x0 + ZM_TX + 2 > nx || y0 - 2 < 0 || y0 + TY + 2 > ny;
  const bool edge_u = x0 - 1 < 0 || x0 + ZM_TX + 1 > nx || y0 - 1 < 0 || y0 + TY + 1 > ny;
  constexpr uint32_t qbytes = 5 * L::QCS * sizeof(real), ubytes = 4 * L::UCS * sizeof(real);

  if (threadIdx.x == 0) {
    for (int i = 0; i < L::QSLOTS + L::USLOTS; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    mbar_init_fence();
    tma_prefetch_desc(&tmQ);
    tma_prefetch_desc(&tmU);
  }
  __syncthreads();

  // plane p of Q lives in slot (p - (z0-2)) % 5, of rho u in slot (p - (z0-1)) % 4
  auto qslot = [&](int p) { return qring + ((p - (z0 - 2)) % L::QSLOTS) * L::QSLOT; };
  auto uslot = [&](int p) { return uring + ((p - (z0 - 1)) % L::USLOTS) * L::USLOT; };
  auto issue_q = [&](int p) {
    const int k = p - (z0 - 2);
    uint64_t* bar = &bars[k % L::QSLOTS];
    mbar_arrive_expect_tx(bar, qbytes);
    tma_load_4d(qslot(p), &tmQ, x0 - ZM_XOFF, y0 - 2, wrap(p, nz), 0, bar);
  };
  auto issue_u = [&](int p) {
    const int k = p - (z0 - 1);
    uint64_t* bar = &bars[L::QSLOTS + k % L::USLOTS];
    mbar_arrive_expect_tx(bar, ubytes);
    tma_load_4d(uslot(p), &tmU, x0 - ZM_XOFF, y0 - 1, wrap(p, nz), 0, bar);
  };
  // Wait for a plane, then patch its periodic halo.  Every thread reaches the
  // __syncthreads that follows a wait, so a timeout cannot strand part of the CTA.
  auto wait_q = [&](int p) {
    const int k = p - (z0 - 2);
    if (!mbar_wait_bounded(&bars[k % L::QSLOTS], (k / L::QSLOTS) & 1, kWaitLimitNs)) *abort_flag = 1;
    else if (edge_q) patch_plane(qslot(p), 5, L::QROWS, 2, ZM_TX + 6, Q, n, nx, ny, wrap(p, nz), x0, y0 - 2);
  };
  auto wait_u = [&](int p) {
    const int k = p - (z0 - 1);
    if (!mbar_wait_bounded(&bars[L::QSLOTS + k % L::USLOTS], (k / L::USLOTS) & 1, kWaitLimitNs)) *abort_flag = 1;
    else if (edge_u) patch_plane(uslot(p), 4, L::UROWS, 3, ZM_TX + 5, rhou, n, nx, ny, wrap(p, nz), x0, y0 - 1);
  };
  auto tslot = [&](int p) { return tring + wrap(p - z0, 3) * L::TSLOT; };
  auto hslot = [&](int p) { return hbuf + ((p - z0 + 2) & 1) * L::HSLOT; };

  // H and tau of plane p on the tile plus a one-site ring (Q planes p-1..p+1)
  auto field_plane = [&](int p) {
    const bool own = p >= z0 && p < z1;
    const real* qm = qslot(p - 1);
    const real* qc = qslot(p);
    const real* qp = qslot(p + 1);
    real* tp = tslot(p);
    real* hp = hslot(p);
    for (int t = threadIdx.x; t < L::TROWS * L::TCOLS; t += blockDim.x) {
      const int r = t / L::TCOLS, c = t % L::TCOLS;
      const int idx = (r + 1) * ZM_BX + (c + 3);  // position in the Q box
      Stencil7<real> st;
      st.c = ld5(qc, L::QCS, idx);
      st.xm = ld5(qc, L::QCS, idx - 1);
      st.xp = ld5(qc, L::QCS, idx + 1);
      st.ym = ld5(qc, L::QCS, idx - ZM_BX);
      st.yp = ld5(qc, L::QCS, idx + ZM_BX);
      st.zm = ld5(qm, L::QCS, idx);
      st.zp = ld5(qp, L::QCS, idx);
      Sym5<real> dq[3];
      const Sym5<real> h = molecular_field(st, m, dq);
      Sym5<real> sg;
      real tu[3];
      lc_stress(st.c, h, m.xi, sg, tu);
      // sigma of an interior site of a plane this CTA owns goes straight out
      const int sx = x0 + c - 1, sy = y0 + r - 1;
      if (own && r >= 1 && r <= TY && c >= 1 && c <= ZM_TX && sx < nx && sy < ny)
        store5(sigma, n, ((long long)p * ny + sy) * nx + sx, sg);
      const int ti = r * L::TCOLS + c;
      tp[ti] = tu[0];
      tp[L::TROWS * L::TCOLS + ti] = tu[1];
      tp[2 * L::TROWS * L::TCOLS + ti] = tu[2];
      if (r >= 1 && r <= TY && c >= 1 && c <= ZM_TX) {
        const int i = (r - 1) * ZM_TX + (c - 1);
        hp[0 * TY * ZM_TX + i] = h.xx;
        hp[1 * TY * ZM_TX + i] = h.xy;
        hp[2 * TY * ZM_TX + i] = h.xz;
        hp[3 * TY * ZM_TX + i] = h.yy;
        hp[4 * TY * ZM_TX + i] = h.yz;
      }
    }
  };

  // ---- prologue: Q planes z0-2..z0+2, u planes z0-1..z0+1; H, tau of z0-1 and z0
  bool aborted = false;
  if (threadIdx.x == 0) {
    for (int p = z0 - 2; p <= z0 + 2; ++p) issue_q(p);
    for (int p = z0 - 1; p <= z0 + 1; ++p) issue_u(p);
  }
  for (int p = z0 - 2; p <= z0 + 1; ++p) wait_q(p);
  wait_u(z0 - 1);
  wait_u(z0);
  __syncthreads();
  aborted = *abort_flag != 0;
  if (!aborted) {
    field_plane(z0 - 1);
    field_plane(z0);
  }

  for (int z = z0; z < z1 && !aborted; ++z) {
    if (threadIdx.x == 0) {
      fence_proxy_async();
      if (z + 3 <= z1 + 1) issue_q(z + 3);
      if (z + 2 <= z1) issue_u(z + 2);
    }
    wait_q(z + 2);
    wait_u(z + 1);
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      break;
    }
    field_plane(z + 1);
    __syncthreads();
    if (valid) {
      const long long s = ((long long)z * ny + gy) * nx + gx;
      const real* qm = qslot(z - 1);
      const real* qc = qslot(z);
      const real* qp = qslot(z + 1);
      const int qi = (ty + 2) * ZM_BX + (tx + ZM_XOFF);
      const Sym5<real> q = ld5(qc, L::QCS, qi);
      Sym5<real> dq[3];
      dq[0] = half_diff(ld5(qc, L::QCS, qi + 1), ld5(qc, L::QCS, qi - 1));
      dq[1] = half_diff(ld5(qc, L::QCS, qi + ZM_BX), ld5(qc, L::QCS, qi - ZM_BX));
      dq[2] = half_diff(ld5(qp, L::QCS, qi), ld5(qm, L::QCS, qi));
      const Sym5<real> h = ld5(hslot(z), TY * ZM_TX, ty * ZM_TX + tx);
      // body force; tau = [xy, xz, yz] with tau_yx = -tau_xy etc.
      const real* tm = tslot(z - 1);
      const real* tc = tslot(z);
      const real* tpz = tslot(z + 1);
      constexpr int TCS = L::TROWS * L::TCOLS;
      const int ti = (ty + 1) * L::TCOLS + (tx + 1);
      const real half = real(0.5);
      real bx = half * (tc[ti + L::TCOLS] - tc[ti - L::TCOLS]) + half * (tpz[TCS + ti] - tm[TCS + ti]);
      real by = -half * (tc[ti + 1] - tc[ti - 1]) + half * (tpz[2 * TCS + ti] - tm[2 * TCS + ti]);
      real bz = -half * (tc[TCS + ti + 1] - tc[TCS + ti - 1]) -
                half * (tc[2 * TCS + ti + L::TCOLS] - tc[2 * TCS + ti - L::TCOLS]);
      bx -= ddot(h, dq[0]);
      by -= ddot(h, dq[1]);
      bz -= ddot(h, dq[2]);
      if (bext) {
        bx += bext[s];
        by += bext[n + s];
        bz += bext[2 * n + s];
      }
      // velocity and its gradient from the rho u ring (components 1..3)
      const real* um = uslot(z - 1);
      const real* uc = uslot(z);
      const real* up = uslot(z + 1);
      const int ui = (ty + 1) * ZM_BX + (tx + ZM_XOFF);
      real u[3], w[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int o = (a + 1) * L::UCS + ui;
        u[a] = uc[o];
        w[a][0] = half * (uc[o + 1] - uc[o - 1]);
        w[a][1] = half * (uc[o + ZM_BX] - uc[o - ZM_BX]);
        w[a][2] = half * (up[o] - um[o]);
      }
      const Sym5<real> r = be_rate(q, h, dq, u, w, m, true);
      bout[s] = bx;
      bout[n + s] = by;
      bout[2 * n + s] = bz;
      const Sym5<real> qs = {q.xx + r.xx, q.xy + r.xy, q.xz + r.xz, q.yy + r.yy, q.yz + r.yz};
      store5(Qs, n, s, qs);
    }
    __syncthreads();
  }
  if (aborted && threadIdx.x == 0) {
    // a barrier wait timed out: record it and give copies in flight a
    // bounded chance to land before the CTA's shared memory is released
    atomicExch(err, 1);
    for (int i = 0; i < L::QSLOTS + L::USLOTS; ++i) {
      mbar_wait_bounded(&bars[i], 0, kWaitLimitNs / 16);
      mbar_wait_bounded(&bars[i], 1, kWaitLimitNs / 16);
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel B: LB predictor-corrector and the Heun corrector
// ---------------------------------------------------------------------------
template <typename real, int TY>
struct LbqSmem {
  static constexpr int ROWS = TY + 2, SLOTS = 4;
  static constexpr int CS = ROWS * ZM_BX;  // per-component stride
  // one slot: [drho ux uy uz] [sigma 5] [b 3] [Q* 5], each group 128-byte aligned
  static constexpr int OFF_S = align_elems(4 * CS, sizeof(real));
  static constexpr int OFF_B = OFF_S + align_elems(5 * CS, sizeof(real));
  static constexpr int OFF_Q = OFF_B + align_elems(3 * CS, sizeof(real));
  static constexpr int SLOT = OFF_Q + align_elems(5 * CS, sizeof(real));
  static constexpr size_t bytes = sizeof(real) * (size_t)SLOTS * SLOT + 8 * 8 + 16;
};

template <typename real, int TY>
__global__ void __launch_bounds__(ZM_TX* TY, TY == 8 ? 2 : 1)
    k_lbq(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmS,
          const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmQs, ZmGeom G, Model<real> m,
          const real* __restrict__ f, const real* __restrict__ rhou, const real* __restrict__ sigma,
          const real* __restrict__ bf, const real* __restrict__ Qs, const real* __restrict__ Qin,
          real* __restrict__ fnew, real* __restrict__ rhou_new, real* __restrict__ Qout, int* __restrict__ err) {
  using L = LbqSmem<real, TY>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* ring = reinterpret_cast<real*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + L::SLOTS * L::SLOT);
  int* abort_flag = reinterpret_cast<int*>(bars + 8);

  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const long long n = G.n;
  const int bt = blockIdx.x;
  const int x0 = (bt % G.tiles_x) * ZM_TX;
  const int y0 = ((bt / G.tiles_x) % G.tiles_y) * TY;
  const int z0 = (bt / (G.tiles_x * G.tiles_y)) * G.zc;
  const int z1 = min(z0 + G.zc, nz);
  const int tx = threadIdx.x % ZM_TX, ty = threadIdx.x / ZM_TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool valid = gx < nx && gy < ny;
  const bool edge = x0 - 1 < 0 || x0 + ZM_TX + 1 > nx || y0 - 1 < 0 || y0 + TY + 1 > ny;
  constexpr int CS = L::CS;
  constexpr uint32_t slot_bytes = (uint32_t)(17 * CS * sizeof(real));

  if (threadIdx.x == 0) {
    for (int i = 0; i < L::SLOTS; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    mbar_init_fence();
    tma_prefetch_desc(&tmU);
    tma_prefetch_desc(&tmS);
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmQs);
  }
  __syncthreads();

  auto slot = [&](int p) { return ring + ((p - (z0 - 1)) % L::SLOTS) * L::SLOT; };
  auto issue = [&](int p) {
    const int k = p - (z0 - 1);
    uint64_t* bar = &bars[k % L::SLOTS];
    real* sl = slot(p);
    const int zz = wrap(p, nz);
    mbar_arrive_expect_tx(bar, slot_bytes);
    tma_load_4d(sl, &tmU, x0 - ZM_XOFF, y0 - 1, zz, 0, bar);
    tma_load_4d(sl + L::OFF_S, &tmS, x0 - ZM_XOFF, y0 - 1, zz, 0, bar);
    tma_load_4d(sl + L::OFF_B, &tmB, x0 - ZM_XOFF, y0 - 1, zz, 0, bar);
    tma_load_4d(sl + L::OFF_Q, &tmQs, x0 - ZM_XOFF, y0 - 1, zz, 0, bar);
  };
  auto wait = [&](int p) {
    const int k = p - (z0 - 1);
    if (!mbar_wait_bounded(&bars[k % L::SLOTS], (k / L::SLOTS) & 1, kWaitLimitNs)) {
      *abort_flag = 1;
    } else if (edge) {
      real* sl = slot(p);
      const int zz = wrap(p, nz);
      patch_plane(sl, 4, L::ROWS, 3, ZM_TX + 5, rhou, n, nx, ny, zz, x0, y0 - 1);
      patch_plane(sl + L::OFF_S, 5, L::ROWS, 3, ZM_TX + 5, sigma, n, nx, ny, zz, x0, y0 - 1);
      patch_plane(sl + L::OFF_B, 3, L::ROWS, 3, ZM_TX + 5, bf, n, nx, ny, zz, x0, y0 - 1);
      patch_plane(sl + L::OFF_Q, 5, L::ROWS, 3, ZM_TX + 5, Qs, n, nx, ny, zz, x0, y0 - 1);
    }
  };
  // neighbour data: component k of [drho ux uy uz | sigma | b]
  auto Nv = [&](const real* sl, int k, int idx) {
    const int off = k < 4 ? k * CS : (k < 9 ? L::OFF_S + (k - 4) * CS : L::OFF_B + (k - 9) * CS);
    return sl[off + idx];
  };

  bool aborted = false;
  if (threadIdx.x == 0)
    for (int p = z0 - 1; p <= z0 + 1; ++p) issue(p);
  wait(z0 - 1);
  wait(z0);

  // periodic source coordinates of the pull
  const int xm = wrap(gx - 1, nx), xp = wrap(gx + 1, nx);
  const int ym = wrap(gy - 1, ny), yp = wrap(gy + 1, ny);

  for (int z = z0; z < z1; ++z) {
    if (threadIdx.x == 0) {
      fence_proxy_async();
      if (z + 2 <= z1) issue(z + 2);
    }
    // populations f_i(y - e_i), issued before the barrier wait so that they overlap it
    real fin[NV];
    if (valid) {
      const int zm = z == 0 ? nz - 1 : z - 1, zp = z + 1 == nz ? 0 : z + 1;
      // three row bases per plane: rows y-1, y, y+1 of planes z-1, z, z+1
      const long long rb[3][3] = {
          {((long long)zm * ny + ym) * nx, ((long long)zm * ny + gy) * nx, ((long long)zm * ny + yp) * nx},
          {((long long)z * ny + ym) * nx, ((long long)z * ny + gy) * nx, ((long long)z * ny + yp) * nx},
          {((long long)zp * ny + ym) * nx, ((long long)zp * ny + gy) * nx, ((long long)zp * ny + yp) * nx}};
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const int sx = ex(i) > 0 ? xm : ex(i) < 0 ? xp : gx;
        fin[i] = __ldg(f + i * n + rb[1 - ez(i)][1 - ey(i)] + sx);
      }
    }
    wait(z + 1);
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      break;
    }
    if (valid) {
      const long long s = ((long long)z * ny + gy) * nx + gx;
      const real* nm = slot(z - 1);
      const real* nc = slot(z);
      const real* np = slot(z + 1);
      const int ci = (ty + 1) * ZM_BX + (tx + ZM_XOFF);
      const real inv_tau = m.inv_tau;
      real ds[NV], dh[NV];
      Sym5<real> sig_y;
      real b_y[3];
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const real* sl = ez(i) > 0 ? nm : ez(i) < 0 ? np : nc;
        const int idx = ci - ey(i) * ZM_BX - ex(i);
        const real drho = Nv(sl, 0, idx);
        const real ux = Nv(sl, 1, idx), uy = Nv(sl, 2, idx), uz = Nv(sl, 3, idx);
        const Sym5<real> sv = {Nv(sl, 4, idx), Nv(sl, 5, idx), Nv(sl, 6, idx), Nv(sl, 7, idx), Nv(sl, 8, idx)};
        const real bx = Nv(sl, 9, idx), by = Nv(sl, 10, idx), bz = Nv(sl, 11, idx);
        if (i == 0) {
          sig_y = sv;
          b_y[0] = bx; b_y[1] = by; b_y[2] = bz;
        }
        const real usq = ux * ux + uy * uy + uz * uz;
        const real C = -(fin[i] - feq_delta(i, drho, real(1) + drho, ux, uy, uz, usq, sv)) * inv_tau +
                       force_dir(i, bx, by, bz);
        ds[i] = fin[i] + C;
        dh[i] = fin[i] + real(0.5) * C;
      }
      real drs = real(0), jx = real(0), jy = real(0), jz = real(0);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        drs += ds[i];
        jx += real(ex(i)) * ds[i];
        jy += real(ey(i)) * ds[i];
        jz += real(ez(i)) * ds[i];
      }
      const real rs = real(1) + drs;
      const real inv_rs = real(1) / rs;
      const real usx = jx * inv_rs, usy = jy * inv_rs, usz = jz * inv_rs;
      const real ussq = usx * usx + usy * usy + usz * usz;
      real dr1 = real(0), j1x = real(0), j1y = real(0), j1z = real(0);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const real Cs = -(ds[i] - feq_delta(i, drs, rs, usx, usy, usz, ussq, sig_y)) * inv_tau +
                        force_dir(i, b_y[0], b_y[1], b_y[2]);
        const real fo = dh[i] + real(0.5) * Cs;
        fnew[i * n + s] = fo;
        dr1 += fo;
        j1x += real(ex(i)) * fo;
        j1y += real(ey(i)) * fo;
        j1z += real(ez(i)) * fo;
      }
      const real inv_r1 = real(1) / (real(1) + dr1);
      rhou_new[s] = dr1;
      rhou_new[n + s] = j1x * inv_r1;
      rhou_new[2 * n + s] = j1y * inv_r1;
      rhou_new[3 * n + s] = j1z * inv_r1;

      // Heun corrector with u^n
      const real* sm = nm + L::OFF_Q;
      const real* sc = nc + L::OFF_Q;
      const real* sp = np + L::OFF_Q;
      Stencil7<real> st;
      st.c = ld5(sc, CS, ci);
      st.xm = ld5(sc, CS, ci - 1);
      st.xp = ld5(sc, CS, ci + 1);
      st.ym = ld5(sc, CS, ci - ZM_BX);
      st.yp = ld5(sc, CS, ci + ZM_BX);
      st.zm = ld5(sm, CS, ci);
      st.zp = ld5(sp, CS, ci);
      Sym5<real> dq[3];
      const Sym5<real> h = molecular_field(st, m, dq);
      real u[3], w[3][3];
      const real half = real(0.5);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        u[a] = Nv(nc, a + 1, ci);
        w[a][0] = half * (Nv(nc, a + 1, ci + 1) - Nv(nc, a + 1, ci - 1));
        w[a][1] = half * (Nv(nc, a + 1, ci + ZM_BX) - Nv(nc, a + 1, ci - ZM_BX));
        w[a][2] = half * (Nv(np, a + 1, ci) - Nv(nm, a + 1, ci));
      }
      const Sym5<real> r = be_rate(st.c, h, dq, u, w, m, true);
      const Sym5<real> q0 = load5(Qin, n, s);
      const Sym5<real> q1 = {half * (q0.xx + st.c.xx + r.xx), half * (q0.xy + st.c.xy + r.xy),
                             half * (q0.xz + st.c.xz + r.xz), half * (q0.yy + st.c.yy + r.yy),
                             half * (q0.yz + st.c.yz + r.yz)};
      store5(Qout, n, s, q1);
    }
    __syncthreads();
  }
  if (aborted && threadIdx.x == 0) {
    atomicExch(err, 1);
    for (int i = 0; i < L::SLOTS; ++i) {
      mbar_wait_bounded(&bars[i], 0, kWaitLimitNs / 16);
      mbar_wait_bounded(&bars[i], 1, kWaitLimitNs / 16);
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename real>
constexpr int zm_ty() {
  return sizeof(real) == 4 ? 8 : 4;
}

template <typename real>
int zm_tile_rows() {
  return zm_ty<real>();
}

template <typename real>
cudaError_t zm_prepare() {
  constexpr int TY = zm_ty<real>();
  cudaError_t e = cudaFuncSetAttribute(k_qside<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)QsideSmem<real, TY>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lbq<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)LbqSmem<real, TY>::bytes);
  return e;
}

ZmGeom zm_geom(int nx, int ny, int nz, int zc, int ty) {
  ZmGeom G;
  G.nx = nx;
  G.ny = ny;
  G.nz = nz;
  G.zc = zc;
  G.n = (long long)nx * ny * nz;
  G.tiles_x = (nx + ZM_TX - 1) / ZM_TX;
  G.tiles_y = (ny + ty - 1) / ty;
  G.tiles_z = (nz + zc - 1) / zc;
  return G;
}

template <typename real>
cudaError_t launch_step_zm(const ZmArgs& a, cudaStream_t s) {
  constexpr int TY = zm_ty<real>();
  const ZmGeom G = zm_geom(a.nx, a.ny, a.nz, a.zc, TY);
  const int grid = G.tiles_x * G.tiles_y * G.tiles_z;
  const Model<real> m = *static_cast<const Model<real>*>(a.model);
  if (a.events) cudaEventRecord(a.events[0], s);
  k_qside<real, TY><<<grid, ZM_TX * TY, QsideSmem<real, TY>::bytes, s>>>(
      *a.tm_q, *a.tm_u, G, m, static_cast<const real*>(a.q), static_cast<const real*>(a.rhou),
      static_cast<const real*>(a.bext), static_cast<real*>(a.sigma), static_cast<real*>(a.b),
      static_cast<real*>(a.qs), a.err);
  if (a.events) cudaEventRecord(a.events[1], s);
  k_lbq<real, TY><<<grid, ZM_TX * TY, LbqSmem<real, TY>::bytes, s>>>(
      *a.tm_u, *a.tm_sigma, *a.tm_b, *a.tm_qs, G, m, static_cast<const real*>(a.f),
      static_cast<const real*>(a.rhou), static_cast<const real*>(a.sigma), static_cast<const real*>(a.b),
      static_cast<const real*>(a.qs), static_cast<const real*>(a.q), static_cast<real*>(a.fnew),
      static_cast<real*>(a.rhou_new), static_cast<real*>(a.qout ? a.qout : a.q), a.err);
  if (a.events) cudaEventRecord(a.events[2], s);
  return cudaGetLastError();
}

template cudaError_t zm_prepare<float>();
template cudaError_t zm_prepare<double>();
template int zm_tile_rows<float>();
template int zm_tile_rows<double>();
template cudaError_t launch_step_zm<float>(const ZmArgs&, cudaStream_t);
template cudaError_t launch_step_zm<double>(const ZmArgs&, cudaStream_t);

}  // namespace lcbp
