// Fast path of the coupled step: two z-marching kernels with TMA-staged planes.
//
//   k_qside  (Q^n, rho u^n)            -> P, Q*, rho - 1             (100 B/site FP32)
//            H, sigma_LC, tau and the body force b = D0_b tau_ab - H_gn D0_a Q_gn,
//            then the Heun predictor Q* = Q + R(Q, u)   (Sec. 2.1 Eq. Qevolution,
//            mat_der, BEstress; Sec. 2.2 Eq. eq7a, spurious), and P: the ten
//            coefficients of the site's LB pre-collision terms f^eq_i / tau_f + p_i
//            (Sec. 2.2 Eq. feq, coeff, eq4), built from rho^n, u^n, sigma_LC and b
//   k_lbq    (f^n, rho u^n, P, Q*, Q^n) -> f^{n+1}, rho u^{n+1}, Q^{n+1}   (256 B/site FP32)
//            predictor-corrector D3Q15 LB (Sec. 2.2 Eq. eq2, eq4, feq, coeff) and the
//            Heun corrector Q^{n+1} = (Q + Q* + R(Q*)) / 2
//
// A CTA owns a column tile of TX x TY sites and marches through ZC planes.
// Planes of the fields it reads with a halo are brought into shared memory by
// TMA tile loads into a ring of slots, each slot with its own mbarrier; the
// load of a plane is issued one or two planes before the CTA needs it, so HBM
// traffic overlaps compute.  The state Q and rho u lives in padded mirrors
// whose ghost columns and rows hold the periodic images, and P, Q* go from
// k_qside to k_lbq through a scratch padded the same way (kernels.h), so no
// staged box needs patching; k_qside writes the scratch's images and k_lbq the
// mirrors'.  Mirrors and scratch hold a site's values as 16-byte vectors.
// Populations are pulled straight from global memory (each is used once).
#include <cuda.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace lcbp {

constexpr int ZM_TX = 32;   // tile width in x (one warp)
constexpr int ZM_BX = 40;   // TMA box width in elements
constexpr int ZM_XOFF = 4;  // box column of global x0
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s bound on any barrier wait

// Staged boxes of the state fields Q (halo 2) and rho u (halo 1) from their
// padded mirrors (site x at mirror column x + 32, y at row y + 2 (Q) or y + 1
// (rho u)), whose ghosts hold the periodic images, for tiles TX sites wide.
// QW, UW: box widths in sites; QX, UX: the box column of x0.  The Q box (for
// its plain yz array) is TX + 8 wide from x0 - 4, a 16-byte aligned start; the
// rho u mirror, 16 bytes per site, stages just x0 - 1 .. x0 + TX.  QPX, QPY,
// UPX, UPY: the mirror offsets of a site.
template <int TX>
struct StateBoxT {
  static constexpr int QW = TX + 2 * ZM_XOFF, QX = ZM_XOFF, QPX = kZmMirX, QPY = 2;
  static constexpr int UW = TX + 2, UX = 1, UPX = kZmMirX, UPY = 1;
};
using StateBox = StateBoxT<ZM_TX>;
static_assert(StateBox::QW == ZM_BX && StateBox::UW == kZmBoxXU && ZM_TX + 2 == kZmBoxXP, "box widths");

__host__ __device__ constexpr int align_elems(int elems, int esize) {
  // round an element count up so that it spans a multiple of 128 bytes
  return ((elems * esize + 127) / 128) * 128 / esize;
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Sites per thread (SPT): with SPT = 2 a thread computes rows y and y + TY/2 of
// the tile in the two lanes of a packed Vec2<float>, which halves the FP32
// instruction count but also the resident warps (shared memory, not threads,
// bounds the CTAs per SM).  Both builds exist for FP32; the autotuner times
// them.  FP64 uses SPT = 1.
template <typename real, int SPT>
struct LaneT {
  using V = real;
};
template <typename real>
struct LaneT<real, 2> {
  using V = Vec2<real>;
};

// value at element i0 (lane 0) and i1 (lane 1) of a shared or global array
template <int SPT, typename real>
__device__ __forceinline__ typename LaneT<real, SPT>::V vld(const real* p, int i0, int i1) {
  if constexpr (SPT == 1) return p[i0];
  else return Vec2<real>(p[i0], p[i1], 0);
}
template <int SPT, typename real, typename V>
__device__ __forceinline__ real lane(const V& v, int k) {
  if constexpr (SPT == 1) return v;
  else return k == 0 ? v.lo() : v.hi();
}
template <int SPT, typename real>
__device__ __forceinline__ Sym5<typename LaneT<real, SPT>::V> ld5v(const real* sl, int cs, int i0, int i1) {
  Sym5<typename LaneT<real, SPT>::V> v;
  v.xx = vld<SPT>(sl, i0, i1);
  v.xy = vld<SPT>(sl, cs + i0, cs + i1);
  v.xz = vld<SPT>(sl, 2 * cs + i0, 2 * cs + i1);
  v.yy = vld<SPT>(sl, 3 * cs + i0, 3 * cs + i1);
  v.yz = vld<SPT>(sl, 4 * cs + i0, 4 * cs + i1);
  return v;
}
// The four values at 16-byte aligned element i (a group of the padded
// scratch), as one vector access: float4, or two double2 for FP64.
template <typename real>
__device__ __forceinline__ void ld4(const real* p, int i, real v[4]) {
  if constexpr (sizeof(real) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p + i);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p + i), c = *reinterpret_cast<const double2*>(p + i + 2);
    v[0] = a.x, v[1] = a.y, v[2] = c.x, v[3] = c.y;
  }
}
template <typename real>
__device__ __forceinline__ void st4(real* p, real a, real b, real c, real d) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
    *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
  }
}
// st4 to global memory as a streaming store (evict-first in L2): the
// step's outputs, which no CTA of the kernel reads again, leave L2 to the
// staged halos and pulled populations that neighbouring tiles share
template <typename real>
__device__ __forceinline__ void st4g(real* p, real a, real b, real c, real d) {
  if constexpr (sizeof(real) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(a, b));
    __stcs(reinterpret_cast<double2*>(p + 2), make_double2(c, d));
  }
}
// a group at element i0 (lane 0) and i1 (lane 1)
template <int SPT, typename real>
__device__ __forceinline__ void ld4v(const real* p, int i0, int i1, typename LaneT<real, SPT>::V v[4]) {
  if constexpr (SPT == 1) {
    ld4(p, i0, v);
  } else {
    real a[4], c[4];
    ld4(p, i0, a);
    ld4(p, i1, c);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = Vec2<real>(a[j], c[j], 0);
  }
}

template <typename V, typename real>
__device__ __forceinline__ Model<V> widen(const Model<real>& m) {
  Model<V> w;
  w.a_bulk = V(m.a_bulk);
  w.b_bulk = V(m.b_bulk);
  w.K = V(m.K);
  w.kq0x2 = V(m.kq0x2);
  w.kq0sq4 = V(m.kq0sq4);
  w.Gamma = V(m.Gamma);
  w.xi = V(m.xi);
  w.inv_tau = V(m.inv_tau);
  w.c_div = V(m.c_div);
  return w;
}

// ---------------------------------------------------------------------------
// Kernel A: H, sigma, tau, b and the Heun predictor
// ---------------------------------------------------------------------------
template <typename real, int TY, int TX = ZM_TX>
struct QsideSmem {
  using B = StateBoxT<TX>;
  static constexpr int QROWS = TY + 4, UROWS = TY + 2, TROWS = TY + 2, TCOLS = TX + 2;
  static constexpr int QSLOTS = 5, USLOTS = 4;
  static constexpr int QCS = QROWS * B::QW, UCS = UROWS * B::UW;  // per-component strides
  static constexpr int QSLOT = align_elems(5 * QCS, sizeof(real)), USLOT = align_elems(4 * UCS, sizeof(real));
  // own cells of a plane: H (5 components) then sigma_LC (5)
  static constexpr int TSLOT = 3 * TROWS * TCOLS, HSLOT = 10 * TY * TX;
  static constexpr int OFF_U = QSLOTS * QSLOT, OFF_T = OFF_U + USLOTS * USLOT;
  static constexpr int OFF_H = OFF_T + 3 * TSLOT, OFF_BAR = align_elems(OFF_H + 2 * HSLOT, sizeof(real));
  // barriers, then the abort flag
  static constexpr size_t bytes = sizeof(real) * (size_t)OFF_BAR + 16 * 8 + 16;
};

// Threads of a k_qside CTA: enough to cover the H / tau ring of a plane
// ((TY + 2) x (TX + 2) cells, a pair per thread with SPT = 2) in one pass, and
// at least the TY / SPT rows of the output pass.
template <int TY, int SPT, int TX = ZM_TX>
constexpr int qside_threads() {
  constexpr int ring = (TY + 2) / SPT * (TX + 2), out = TX * TY / SPT;
  return ((ring > out ? ring : out) + 31) / 32 * 32;
}

// Tile bt (TX x TY sites) of one lattice (or of replica rc of a batch class,
// whose fields are 5-D tensors with the replica outermost: BATCH) of the
// k_qside step.
// WALLS: walls half a spacing below z = 0 and above z = nz-1.  The ghost
// planes z = -1 and z = nz hold the anchored qw in every Q stencil, carry no
// molecular field (tau = 0 there) and the velocity -u of the adjacent plane.
template <typename real, int TY, int SPT, bool BATCH, bool WALLS, int TX = ZM_TX>
__device__ __forceinline__ void qside_body(const CUtensorMap* tmQ, const CUtensorMap* tmQ1, const CUtensorMap* tmU,
                                           const ZmGeom G,
                                           const Model<real> m, int bt, int rc, const real* __restrict__ bext,
                                           real* __restrict__ pq, int* __restrict__ err, const Sym5<real> qw) {
  using L = QsideSmem<real, TY, TX>;
  using B = StateBoxT<TX>;
  using V = typename LaneT<real, SPT>::V;
  constexpr int TYH = TY / SPT;  // rows handled by one pass of the CTA
  static_assert(TY % SPT == 0 && (TY + 2) % SPT == 0, "tile rows must split evenly between the lanes");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* base = reinterpret_cast<real*>(smem_raw);
  real* qring = base;
  real* uring = base + L::OFF_U;
  real* tring = base + L::OFF_T;
  real* hbuf = base + L::OFF_H;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + L::OFF_BAR);  // 5 Q + 4 u
  int* abort_flag = reinterpret_cast<int*>(bars + 16);

  // element offsets within one lattice (or replica) fit in 32 bits: the host
  // takes this path only where 15 components of every field do
  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int n = (int)G.n;
  const int x0 = (bt % G.tiles_x) * TX;
  const int y0 = ((bt / G.tiles_x) % G.tiles_y) * TY;
  const int z0 = (bt / (G.tiles_x * G.tiles_y)) * G.zc;
  const int z1 = min(z0 + G.zc, nz);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;  // rows ty + k * TYH, k < SPT
  const int gx = x0 + tx;
  constexpr uint32_t qbytes = 5 * L::QCS * sizeof(real), ubytes = 4 * L::UCS * sizeof(real);

  if (threadIdx.x == 0) {
    for (int i = 0; i < L::QSLOTS + L::USLOTS; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    mbar_init_fence();
    tma_prefetch_desc(tmQ);
    tma_prefetch_desc(tmQ1);
    tma_prefetch_desc(tmU);
  }
  __syncthreads();

  // plane p of Q lives in slot (p - (z0-2)) % 5, of rho u in slot (p - (z0-1)) % 4
  // (the plane offsets below are never negative: unsigned arithmetic keeps the ring
  // index a plain multiply-shift or mask)
  auto qslot = [&](int p) { return qring + ((unsigned)(p - (z0 - 2)) % L::QSLOTS) * L::QSLOT; };
  auto uslot = [&](int p) { return uring + ((unsigned)(p - (z0 - 1)) % L::USLOTS) * L::USLOT; };
  auto issue_q = [&](int p) {
    const unsigned k = p - (z0 - 2);
    uint64_t* bar = &bars[k % L::QSLOTS];
    mbar_arrive_expect_tx(bar, qbytes);
    // the mirror's [xx xy xz yy] vectors, then its yz array (replica rc of a batch class)
    const int X = x0 - B::QX + B::QPX, Y = y0 - 2 + B::QPY;
    if constexpr (BATCH) {
      tma_load_4d(qslot(p), tmQ, 4 * X, Y, wrap(p, nz), rc, bar);
      tma_load_4d(qslot(p) + 4 * L::QCS, tmQ1, X, Y, wrap(p, nz), rc, bar);
    } else {
      tma_load_3d(qslot(p), tmQ, 4 * X, Y, wrap(p, nz), bar);
      tma_load_3d(qslot(p) + 4 * L::QCS, tmQ1, X, Y, wrap(p, nz), bar);
    }
  };
  auto issue_u = [&](int p) {
    const unsigned k = p - (z0 - 1);
    uint64_t* bar = &bars[L::QSLOTS + k % L::USLOTS];
    mbar_arrive_expect_tx(bar, ubytes);
    if constexpr (BATCH)
      tma_load_4d(uslot(p), tmU, 4 * (x0 - B::UX + B::UPX), y0 - 1 + B::UPY, wrap(p, nz), rc, bar);
    else
      tma_load_3d(uslot(p), tmU, 4 * (x0 - B::UX + B::UPX), y0 - 1 + B::UPY, wrap(p, nz), bar);
  };
  // Q and rho u at box index i0 (lane 0) and i1 (lane 1) of a staged slot:
  // the mirrors stage [row][col][4] vectors (Q: then its yz as [row][col])
  auto ldq = [&](const real* sl, int i0, int i1) -> Sym5<V> {
    V a[4];
    ld4v<SPT>(sl, 4 * i0, 4 * i1, a);
    return {a[0], a[1], a[2], a[3], vld<SPT>(sl, 4 * L::QCS + i0, 4 * L::QCS + i1)};
  };
  auto ldu = [&](const real* sl, int i0, int i1, V v[4]) {  // [rho - 1, u_x, u_y, u_z]
    ld4v<SPT>(sl, 4 * i0, 4 * i1, v);
  };
  // Wait for a plane.  Every thread reaches the __syncthreads that follows a
  // wait, so a timeout cannot strand part of the CTA.
  auto wait_q = [&](int p) {
    const unsigned k = p - (z0 - 2);
    const bool ok = mbar_wait_bounded(&bars[k % L::QSLOTS], (k / L::QSLOTS) & 1, kWaitLimitNs);
    if (!ok) *abort_flag = 1;
    return ok;
  };
  auto wait_u = [&](int p) {
    const unsigned k = p - (z0 - 1);
    const bool ok = mbar_wait_bounded(&bars[L::QSLOTS + k % L::USLOTS], (k / L::USLOTS) & 1, kWaitLimitNs);
    if (!ok) *abort_flag = 1;
    return ok;
  };
  // a staged Q plane beyond a wall: qw in every cell (no periodic images)
  auto ghost = [&](int p) { return WALLS && (p < 0 || p >= nz); };
  auto fill_q = [&](int p) {
    real* sl = qslot(p);
    for (int t = threadIdx.x; t < L::QCS; t += blockDim.x) {
      st4(sl + 4 * t, qw.xx, qw.xy, qw.xz, qw.yy);
      sl[4 * L::QCS + t] = qw.yz;
    }
  };
  auto tslot = [&](int p) { return tring + ((unsigned)(p - z0 + 3) % 3u) * L::TSLOT; };
  auto hslot = [&](int p) { return hbuf + ((unsigned)(p - z0 + 2) & 1u) * L::HSLOT; };

  // H and tau of plane p on the tile plus a one-site ring (Q planes p-1..p+1);
  // a thread takes cells (r, c) and (r + TROWS / SPT, c) together
  const Model<V> mv = widen<V>(m);
  // With one site per thread, threads 0 .. TY*32-1 take the tile's own cells
  // in the order of the output pass and keep the gradients of their cell in
  // registers for it (dq_next); H goes through hslot; the ring cells go to
  // the threads after them.  With two sites per thread the output pass
  // recomputes the gradients from the staged Q.
  // With one site per thread the own cell's tau_xz, tau_yz of the plane just
  // computed stay in registers too (tz_next): the output pass of plane z reads
  // tau of plane z+1 only in its own column, so it needs no barrier after the
  // pass over plane z+1.
  Sym5<V> dq_next[3];
  V tz_next[2];
  auto field_plane = [&](int p) {
    if (ghost(p)) {  // tau = 0 beyond a wall; H there is never read
      for (int t = threadIdx.x; t < L::TSLOT; t += blockDim.x) tslot(p)[t] = real(0);
      tz_next[0] = tz_next[1] = V(0);
      return;
    }
    const real* qm = qslot(p - 1);
    const real* qc = qslot(p);
    const real* qp = qslot(p + 1);
    real* tp = tslot(p);
    real* hp = hslot(p);
    if constexpr (SPT == 1) {
      constexpr int NIN = TY * TX, TC = L::TCOLS;
      const int t = threadIdx.x;
      int r = -1, c = 0;
      if (t < NIN) {
        r = t / TX + 1;
        c = t % TX + 1;
      } else {
        const int u = t - NIN;
        if (u < TC) {
          r = 0;
          c = u;
        } else if (u < 2 * TC) {
          r = L::TROWS - 1;
          c = u - TC;
        } else if (u < 2 * TC + TY) {
          r = u - 2 * TC + 1;
          c = 0;
        } else if (u < 2 * TC + 2 * TY) {
          r = u - 2 * TC - TY + 1;
          c = TC - 1;
        }
      }
      if (r >= 0) {
        const int i0 = (r + 1) * B::QW + (c + B::QX - 1);  // position in the Q box
        Stencil7<V> st;
        st.c = ldq(qc, i0, i0);
        st.xm = ldq(qc, i0 - 1, i0 - 1);
        st.xp = ldq(qc, i0 + 1, i0 + 1);
        st.ym = ldq(qc, i0 - B::QW, i0 - B::QW);
        st.yp = ldq(qc, i0 + B::QW, i0 + B::QW);
        st.zm = ldq(qm, i0, i0);
        st.zp = ldq(qp, i0, i0);
        Sym5<V> dq[3];
        const Sym5<V> h = molecular_field<true>(st, mv, dq);
        Sym5<V> sg;
        V tu[3];
        // the ring warps (t >= NIN, a warp-uniform split) need tau only
        if (t < NIN) lc_stress(st.c, h, mv.xi, sg, tu);
        else lc_tau(st.c, h, tu);
        const int ti = r * TC + c;
        tp[ti] = tu[0];
        tp[L::TROWS * TC + ti] = tu[1];
        tp[2 * L::TROWS * TC + ti] = tu[2];
        if (t < NIN) {
          hp[0 * NIN + t] = h.xx;
          hp[1 * NIN + t] = h.xy;
          hp[2 * NIN + t] = h.xz;
          hp[3 * NIN + t] = h.yy;
          hp[4 * NIN + t] = h.yz;
          hp[5 * NIN + t] = sg.xx;
          hp[6 * NIN + t] = sg.xy;
          hp[7 * NIN + t] = sg.xz;
          hp[8 * NIN + t] = sg.yy;
          hp[9 * NIN + t] = sg.yz;
          dq_next[0] = dq[0];
          dq_next[1] = dq[1];
          dq_next[2] = dq[2];
          tz_next[0] = tu[1];
          tz_next[1] = tu[2];
        }
      }
      return;
    }
    constexpr int RH = L::TROWS / SPT;
    for (int t = threadIdx.x; t < RH * L::TCOLS; t += blockDim.x) {
      const int r0 = t / L::TCOLS, c = t % L::TCOLS;
      const int i0 = (r0 + 1) * B::QW + (c + B::QX - 1);  // position in the Q box
      const int i1 = i0 + RH * B::QW;
      Stencil7<V> st;
      st.c = ldq(qc, i0, i1);
      st.xm = ldq(qc, i0 - 1, i1 - 1);
      st.xp = ldq(qc, i0 + 1, i1 + 1);
      st.ym = ldq(qc, i0 - B::QW, i1 - B::QW);
      st.yp = ldq(qc, i0 + B::QW, i1 + B::QW);
      st.zm = ldq(qm, i0, i1);
      st.zp = ldq(qp, i0, i1);
      Sym5<V> dq[3];
      const Sym5<V> h = molecular_field<true>(st, mv, dq);
      Sym5<V> sg;
      V tu[3];
      lc_stress(st.c, h, mv.xi, sg, tu);
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        const int r = r0 + k * RH;
        const int ti = r * L::TCOLS + c;
        tp[ti] = lane<SPT, real>(tu[0], k);
        tp[L::TROWS * L::TCOLS + ti] = lane<SPT, real>(tu[1], k);
        tp[2 * L::TROWS * L::TCOLS + ti] = lane<SPT, real>(tu[2], k);
        if (r >= 1 && r <= TY && c >= 1 && c <= TX) {
          const int i = (r - 1) * TX + (c - 1);
          hp[0 * TY * TX + i] = lane<SPT, real>(h.xx, k);
          hp[1 * TY * TX + i] = lane<SPT, real>(h.xy, k);
          hp[2 * TY * TX + i] = lane<SPT, real>(h.xz, k);
          hp[3 * TY * TX + i] = lane<SPT, real>(h.yy, k);
          hp[4 * TY * TX + i] = lane<SPT, real>(h.yz, k);
          hp[5 * TY * TX + i] = lane<SPT, real>(sg.xx, k);
          hp[6 * TY * TX + i] = lane<SPT, real>(sg.xy, k);
          hp[7 * TY * TX + i] = lane<SPT, real>(sg.xz, k);
          hp[8 * TY * TX + i] = lane<SPT, real>(sg.yy, k);
          hp[9 * TY * TX + i] = lane<SPT, real>(sg.yz, k);
        }
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
  if (WALLS && !aborted && (z0 < 2 || z0 + 1 >= nz)) {
    for (int p = z0 - 2; p <= z0 + 1; ++p)
      if (ghost(p)) fill_q(p);
    __syncthreads();
  }
  if (!aborted) {
    field_plane(z0 - 1);
    field_plane(z0);
  }

  // Per plane one CTA barrier, after the waits (a uniform abort decision),
  // and with two sites per thread a second one after the H / tau
  // pass.  A thread past the first barrier of plane z knows every thread has
  // finished plane z-1, the last reader of the Q and u slots the next loads
  // overwrite (planes z-2) and of the tau / H slots this plane's pass
  // overwrites (planes z-2 and z-1), so no barrier closes the plane.  The
  // output pass of plane z reads tau of planes z-1 and z and H of plane z,
  // written in earlier planes' passes, and tau of plane z+1 in its own column
  // (one site per thread: from registers; two: from the slot, after the
  // second barrier).
  for (int z = z0; z < z1 && !aborted; ++z) {
    wait_q(z + 2);
    wait_u(z + 1);
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      break;
    }
    if (ghost(z + 2)) {  // a wall's ghost plane
      fill_q(z + 2);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      fence_proxy_async();
      if (z + 3 <= z1 + 1) issue_q(z + 3);
      if (z + 2 <= z1) issue_u(z + 2);
    }
    // H and the gradients of plane z, kept from the previous pass (one site per thread)
    const Sym5<V> dq_cur[3] = {dq_next[0], dq_next[1], dq_next[2]};
    field_plane(z + 1);
    if constexpr (SPT != 1) __syncthreads();
    if (ty < TYH && gx < nx && y0 + ty < ny) {
      const real* qm = qslot(z - 1);
      const real* qc = qslot(z);
      const real* qp = qslot(z + 1);
      const int qi0 = (ty + 2) * B::QW + (tx + B::QX), qi1 = qi0 + TYH * B::QW;
      const Sym5<V> q = ldq(qc, qi0, qi1);
      Sym5<V> dq[3], h;
      if constexpr (SPT == 1) {
        dq[0] = dq_cur[0];
        dq[1] = dq_cur[1];
        dq[2] = dq_cur[2];
        const int hi0 = ty * TX + tx;
        h = ld5v<SPT>(hslot(z), TY * TX, hi0, hi0);
      } else {
        dq[0] = diff5(ldq(qc, qi0 + 1, qi1 + 1), ldq(qc, qi0 - 1, qi1 - 1));
        dq[1] = diff5(ldq(qc, qi0 + B::QW, qi1 + B::QW), ldq(qc, qi0 - B::QW, qi1 - B::QW));
        dq[2] = diff5(ldq(qp, qi0, qi1), ldq(qm, qi0, qi1));
        const int hi0 = ty * TX + tx;
        h = ld5v<SPT>(hslot(z), TY * TX, hi0, hi0 + TYH * TX);
      }
      // body force; tau = [xy, xz, yz] with tau_yx = -tau_xy etc.
      const real* tm = tslot(z - 1);
      const real* tc = tslot(z);
      const real* tpz = tslot(z + 1);
      constexpr int TCS = L::TROWS * L::TCOLS;
      const int t0 = (ty + 1) * L::TCOLS + (tx + 1), t1 = t0 + TYH * L::TCOLS;
      auto T = [&](const real* sl, int off) { return vld<SPT>(sl, t0 + off, t1 + off); };
      const V half = V(0.5);
      V tz_p[2];  // tau_xz, tau_yz of plane z+1 at the site
      if constexpr (SPT == 1) {
        tz_p[0] = tz_next[0];
        tz_p[1] = tz_next[1];
      } else {
        tz_p[0] = T(tpz, TCS);
        tz_p[1] = T(tpz, 2 * TCS);
      }
      V bx = half * (T(tc, L::TCOLS) - T(tc, -L::TCOLS)) + half * (tz_p[0] - T(tm, TCS));
      V by = -(half * (T(tc, 1) - T(tc, -1))) + half * (tz_p[1] - T(tm, 2 * TCS));
      V bz = -(half * (T(tc, TCS + 1) - T(tc, TCS - 1))) -
             half * (T(tc, 2 * TCS + L::TCOLS) - T(tc, 2 * TCS - L::TCOLS));
      bx -= half * ddot(h, dq[0]);  // (dq: twice the central derivatives)
      by -= half * ddot(h, dq[1]);
      bz -= half * ddot(h, dq[2]);
      // velocity and its gradient from the rho u ring (components 1..3)
      const real* um = uslot(z - 1);
      const real* uc = uslot(z);
      const real* up = uslot(z + 1);
      const int u0 = (ty + 1) * B::UW + (tx + B::UX), u1 = u0 + TYH * B::UW;
      V u[3], w[3][3], drho;
      {
        V c[4], xp[4], xm[4], yp[4], ym[4], zp[4], zm[4];  // [rho - 1, u_x, u_y, u_z]
        ldu(uc, u0, u1, c);
        ldu(uc, u0 + 1, u1 + 1, xp);
        ldu(uc, u0 - 1, u1 - 1, xm);
        ldu(uc, u0 + B::UW, u1 + B::UW, yp);
        ldu(uc, u0 - B::UW, u1 - B::UW, ym);
        ldu(up, u0, u1, zp);
        ldu(um, u0, u1, zm);
        drho = c[0];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          u[a] = c[1 + a];
          w[a][0] = xp[1 + a] - xm[1 + a];  // twice the central derivatives
          w[a][1] = yp[1 + a] - ym[1 + a];
          V upz = zp[1 + a], umz = zm[1 + a];
          if (WALLS && z == 0) umz = -u[a];  // no slip half a spacing beyond the wall
          if (WALLS && z == nz - 1) upz = -u[a];
          w[a][2] = upz - umz;
        }
      }
      const Sym5<V> r = be_rate<true>(q, h, dq, u, w, mv, true);
      // The site's 16 values (four groups; rho - 1 in the last place) of the
      // padded scratch for lane k:
      // at the site's padded position, and at its periodic images in the ghost
      // columns and rows where the site lies on a lattice face.
      const int nxp = G.nxp, nyp = G.nyp, gs = 4 * G.nxp * G.nyp;  // gs: group stride
      auto put = [&](const V* P, const V* qs, const V& dr) {
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
          const int gy = y0 + ty + k * TYH;
          if (gy >= ny) continue;
          auto L = [&](const V& v) { return lane<SPT, real>(v, k); };
          const real g0[4] = {L(P[6]), L(P[3]), L(P[4]), L(P[5])};
          const real g1[4] = {L(P[7]), L(P[8]), L(P[9]), L(P[0])};
          const real g2[4] = {L(P[1]), L(P[2]), L(qs[4]), L(dr)};
          const real g3[4] = {L(qs[0]), L(qs[1]), L(qs[2]), L(qs[3])};
          auto put1 = [&](int xx, int yy) {
            real* d = pq + ((z * kZmPQG * nyp + yy) * nxp + xx) * 4;
            st4g(d, g0[0], g0[1], g0[2], g0[3]);
            st4g(d + gs, g1[0], g1[1], g1[2], g1[3]);
            st4g(d + 2 * gs, g2[0], g2[1], g2[2], g2[3]);
            st4g(d + 3 * gs, g3[0], g3[1], g3[2], g3[3]);
          };
          put1(gx + 1, gy + 1);
          if (gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1) {
            const int xg = gx == 0 ? nx + 1 : (gx == nx - 1 ? 0 : -1);  // nx >= 4: not both
            const int yg[2] = {gy == 0 ? ny + 1 : -1, gy == ny - 1 ? 0 : -1};
            if (xg >= 0) put1(xg, gy + 1);
            for (int j = 0; j < 2; ++j)
              if (yg[j] >= 0) {
                put1(gx + 1, yg[j]);
                if (xg >= 0) put1(xg, yg[j]);
              }
          }
        }
      };
      const V qv[5] = {q.xx + r.xx, q.xy + r.xy, q.xz + r.xz, q.yy + r.yy, q.yz + r.yz};
      // The site's LB pre-collision coefficients from rho^n, u^n, sigma_LC and
      // b (the external force included): with j = rho u,
      //   F_a = [drho/30 - rho u^2/12 + (j_a u_a - sigma_aa)/2] / tau_f,
      //   V_a = (j_a / tau_f + b_a) / 3,   C = [drho/30 + rho u^2/48] / tau_f,
      //   W_ab = (j_a u_b - sigma_ab) / (8 tau_f),
      // so that f^eq_i / tau_f + p_i (Sec. 2.2 Eq. feq, coeff, eq4; T = 1/3,
      // sigma traceless, deviations from the rest weights) is F_a + s V_a for the
      // face direction s e_a and C + (s . V) / 8 + sum_{a<b} s_a s_b W_ab for the
      // corner direction s.
      V bt[3] = {bx, by, bz};
      if (bext) {
        int sb[SPT];
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
          const int gyk = y0 + ty + k * TYH;
          sb[k] = (z * ny + (gyk < ny ? gyk : y0 + ty)) * nx + gx;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) bt[a] += vld<SPT>(bext, a * n + sb[0], a * n + sb[SPT - 1]);
      }
      const int hs0 = ty * TX + tx;
      const Sym5<V> sg = ld5v<SPT>(hslot(z) + 5 * TY * TX, TY * TX, hs0, hs0 + TYH * TX);
      const V it = mv.inv_tau;
      const V rho = V(1) + drho;
      const V jx = rho * u[0], jy = rho * u[1], jz = rho * u[2];
      const V rusq = jx * u[0] + jy * u[1] + jz * u[2];
      const V d30 = drho * LCBP_Q(1, 30);
      const V fb = d30 - rusq * LCBP_Q(1, 12);
      const V it8 = it * LCBP_Q(1, 8);
      V P[10];
      P[0] = (fb + half * (jx * u[0] - sg.xx)) * it;
      P[1] = (fb + half * (jy * u[1] - sg.yy)) * it;
      P[2] = (fb + half * (jz * u[2] + (sg.xx + sg.yy))) * it;
      P[3] = (jx * it + bt[0]) * LCBP_Q(1, 3);
      P[4] = (jy * it + bt[1]) * LCBP_Q(1, 3);
      P[5] = (jz * it + bt[2]) * LCBP_Q(1, 3);
      P[6] = (d30 + rusq * LCBP_Q(1, 48)) * it;
      P[7] = (jx * u[1] - sg.xy) * it8;
      P[8] = (jx * u[2] - sg.xz) * it8;
      P[9] = (jy * u[2] - sg.yz) * it8;
      put(P, qv, drho);
    }
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

// FP32: two CTAs per SM (shared memory allows two; the bound keeps the registers within it)
template <typename real, int TY, int SPT, bool WALLS>
__global__ void __launch_bounds__(qside_threads<TY, SPT>(), sizeof(real) == 4 ? 2 : 1)
    k_qside(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmQ1,
            const __grid_constant__ CUtensorMap tmU, ZmGeom G, Model<real> m, const real* __restrict__ bext,
            real* __restrict__ pq, int* __restrict__ err, Sym5<real> qw) {
  qside_body<real, TY, SPT, false, WALLS>(&tmQ, &tmQ1, &tmU, G, m, blockIdx.x, 0, bext, pq, err, qw);
}

// The CTA's batch class, its replica and tile: classes own consecutive CTA ranges.
struct ZmItem {
  int k;   // class
  int j;   // replica position within the class (the 5-D tensor coordinate)
  int bt;  // tile within the replica
};
__device__ __forceinline__ ZmItem zm_item(const ZmBatch& B) {
  ZmItem it{0, 0, 0};
  int cta0 = B.c[0].cta0, per = B.c[0].ctas_per_rep;
#pragma unroll
  for (int i = 1; i < kZmMaxClasses; ++i)
    if (i < B.nclass && (int)blockIdx.x >= B.c[i].cta0) {
      it.k = i;
      cta0 = B.c[i].cta0;
      per = B.c[i].ctas_per_rep;
    }
  const int local = (int)blockIdx.x - cta0;
  it.j = local / per;
  it.bt = local % per;
  return it;
}

// geometry of class k, selected at compile-time indices of the parameter array
__device__ __forceinline__ ZmGeom zm_class_geom(const ZmBatch& B, int k) {
  ZmGeom G = B.c[0].G;
#pragma unroll
  for (int i = 1; i < kZmMaxClasses; ++i)
    if (i == k) G = B.c[i].G;
  return G;
}

template <typename real, int TY>
__global__ void __launch_bounds__(qside_threads<TY, 1>(), sizeof(real) == 4 ? 2 : 1)
    k_qside_batch(const __grid_constant__ ZmBatchMaps maps, ZmBatch B, const Replica<real>* __restrict__ reps,
                  const int* __restrict__ order, real* __restrict__ pq, int* __restrict__ err) {
  const ZmItem it = zm_item(B);
  const ZmGeom G = zm_class_geom(B, it.k);
  int rep0 = B.c[0].rep0;
  long long pq0 = B.c[0].pq0;
#pragma unroll
  for (int i = 1; i < kZmMaxClasses; ++i)
    if (i == it.k) {
      rep0 = B.c[i].rep0;
      pq0 = B.c[i].pq0;
    }
  const int r = order[rep0 + it.j];
  const Model<real> m = reps[r].m;
  // the class's maps (replica it.j is their outermost coordinate), selected at
  // compile-time offsets (a runtime index into the parameter arrays would copy
  // them to local memory)
  const CUtensorMap *mq = &maps.q[0], *mq1 = &maps.q1[0], *mu = &maps.u[0];
#pragma unroll
  for (int i = 1; i < kZmMaxClasses; ++i)
    if (i == it.k) {
      mq = &maps.q[i];
      mq1 = &maps.q1[i];
      mu = &maps.u[i];
    }
  real* const pqr = pq + pq0 + (long long)it.j * kZmPQ * G.cp;
  // a class of narrow tiles (kZmNarrowX wide, twice the rows: FP32 only)
  if constexpr (sizeof(real) == 4) {
    if (G.tx == kZmNarrowX) {
      qside_body<real, 2 * TY, 1, true, false, kZmNarrowX>(mq, mq1, mu, G, m, it.bt, it.j, nullptr, pqr, err,
                                                           Sym5<real>{});
      return;
    }
  }
  qside_body<real, TY, 1, true, false>(mq, mq1, mu, G, m, it.bt, it.j, nullptr, pqr, err, Sym5<real>{});
}

// The positions of a padded mirror (site x at column x + px, y at row y + h)
// that hold the value of site (gx, gy): its own, and each ghost position in
// the h columns and rows next to the lattice whose periodic image it is
// (lattice faces only; nx >= 2h gives a site at most one x image).  put1(X, Y)
// is called for each.
template <typename F>
__device__ __forceinline__ void mirror_positions(int px, int h, int nx, int ny, int gx, int gy, F&& put1) {
  const int X = gx + px, Y = gy + h;
  put1(X, Y);
  if (gx >= h && gx < nx - h && gy >= h && gy < ny - h) return;
  // x = nx + gx (site gx < h) or x = gx - nx (site gx >= nx - h)
  const int xg = gx < h ? nx + px + gx : (gx >= nx - h ? gx - nx + px : -1);
  if (xg >= 0) put1(xg, Y);
  for (int g = 0; g < h; ++g) {  // ghost rows y = g - h and y = ny + g (several when ny < 2h)
    const int ya = wrap(g - h, ny) == gy ? g : -1, yb = wrap(ny + g, ny) == gy ? ny + h + g : -1;
    if (ya >= 0) {
      put1(X, ya);
      if (xg >= 0) put1(xg, ya);
    }
    if (yb >= 0) {
      put1(X, yb);
      if (xg >= 0) put1(xg, yb);
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel B: LB predictor-corrector and the Heun corrector
// ---------------------------------------------------------------------------
template <typename real, int TY, int TX = ZM_TX>
struct LbqSmem {
  static constexpr int ROWS = TY + 2, SLOTS = 4;
  static constexpr int GS = ROWS * (TX + 2) * 4;          // one group of the P / Q* box: [row][TX + 2][4]
  static constexpr int CSU = ROWS * StateBoxT<TX>::UW;  // sites of the u box
  // one slot: the four groups of the padded scratch, then the u box of the
  // rho u mirror's [rho-1 u_x u_y u_z] vectors
  static constexpr int OFF_U = align_elems(kZmPQG * GS, sizeof(real));
  static constexpr int SLOT = OFF_U + align_elems(4 * CSU, sizeof(real));
  static constexpr uint32_t TX_BYTES = (uint32_t)((kZmPQG * GS + 4 * CSU) * sizeof(real));
  // barriers, then the abort flag
  static constexpr size_t bytes = sizeof(real) * (size_t)SLOTS * SLOT + 8 * 8 + 16;
};

// WALLS: walls half a spacing below z = 0 and above z = nz-1.  A population
// that would arrive from beyond a wall is the reflected one of the same site
// (half-way bounce-back); the staged Q* of a ghost plane is the anchored qw and
// its velocity is -u of the adjacent plane.
// tmF, tmF1, tmF2, tmQ, tmQ1: maps of f^n (boxes of the tile's rows with
// every population, and of one halo row with one or two populations) and of
// the Q^n mirror in tile-sized boxes (for a batch the class's, with the
// replica outermost), whose planes are prefetched into L2 one plane before
// the loads read them
template <typename real, int TY, int SPT, bool BATCH, bool WALLS, int TX = ZM_TX>
__device__ __forceinline__ void lbq_body(const CUtensorMap* tmPQ, const CUtensorMap* tmU3, const CUtensorMap* tmF,
                                         const CUtensorMap* tmF1, const CUtensorMap* tmF2,
                                         const CUtensorMap* tmQ, const CUtensorMap* tmQ1, const ZmGeom& G,
                                         const Model<real>& m, int bt, int rc, const real* __restrict__ f,
                                         const real* __restrict__ Qin, real* __restrict__ fnew,
                                         real* __restrict__ rhou_new, real* __restrict__ Qout,
                                         int* __restrict__ err, const Sym5<real> qw) {
  using L = LbqSmem<real, TY, TX>;
  using B = StateBoxT<TX>;
  using V = typename LaneT<real, SPT>::V;
  constexpr int TYH = TY / SPT;  // a thread takes rows ty + k * TYH, k < SPT
  constexpr int AW = TX + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* ring = reinterpret_cast<real*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + L::SLOTS * L::SLOT);
  int* abort_flag = reinterpret_cast<int*>(bars + 8);

  const int nx = G.nx, ny = G.ny, nz = G.nz;
  const int n = (int)G.n;  // (32-bit element offsets, as in k_qside)
  const int x0 = (bt % G.tiles_x) * TX;
  const int y0 = ((bt / G.tiles_x) % G.tiles_y) * TY;
  const int z0 = (bt / (G.tiles_x * G.tiles_y)) * G.zc;
  const int z1 = min(z0 + G.zc, nz);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gx = x0 + tx;
  int gy[SPT];
  bool lane_ok[SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    lane_ok[k] = gx < nx && y0 + ty + k * TYH < ny;
    // a lane past the ragged y edge reads lane 0's site and stores nothing
    gy[k] = lane_ok[k] ? y0 + ty + k * TYH : y0 + ty;
  }
  const bool valid = lane_ok[0];

  if (threadIdx.x == 0) {
    for (int i = 0; i < L::SLOTS; ++i) mbar_init(&bars[i], 1);
    *abort_flag = 0;
    mbar_init_fence();
    tma_prefetch_desc(tmPQ);
    tma_prefetch_desc(tmU3);
    tma_prefetch_desc(tmF);
    tma_prefetch_desc(tmF1);
    tma_prefetch_desc(tmF2);
    tma_prefetch_desc(tmQ);
    tma_prefetch_desc(tmQ1);
  }
  __syncthreads();

  auto slot = [&](int p) { return ring + ((unsigned)(p - (z0 - 1)) % L::SLOTS) * L::SLOT; };
  // plane p: the padded P / Q* box (site (x, y) at padded (x + 1, y + 1), so the
  // box starting at padded (x0, y0) covers x0-1 .. x0+TX) and the u box of rho u
  auto issue = [&](int p) {
    const unsigned k = p - (z0 - 1);
    uint64_t* bar = &bars[k % L::SLOTS];
    real* sl = slot(p);
    const int zz = wrap(p, nz);
    mbar_arrive_expect_tx(bar, L::TX_BYTES);
    // the scratch as (4 X, Y, group, z): x coordinate in elements of 4 per site
    if constexpr (BATCH) tma_load_5d(sl, tmPQ, 4 * x0, y0, 0, zz, rc, bar);
    else tma_load_4d(sl, tmPQ, 4 * x0, y0, 0, zz, bar);
    // the populations of plane p (pulled from plane p-1 on) and Q^n of plane
    // p-1, into L2 a plane ahead of their plain loads.  Q^n in tile-sized
    // boxes (the tile's own sites); f for the tile's rows with all 15
    // populations and, of the halo rows, only the populations that move into
    // the tile: +y (3; 7, 8; 11, 12) from row y0 - 1, -y (4; 9, 10; 13, 14)
    // from the row after the tile
    const int X = x0 + B::QPX, Y = y0 + B::QPY;
    const int ya = wrap(y0 - 1, ny), yb = wrap(min(y0 + TY, ny), ny), xf = x0 - ZM_XOFF;
    if constexpr (BATCH) {
      tma_load_4d(sl + L::OFF_U, tmU3, 4 * (x0 - B::UX + B::UPX), y0 - 1 + B::UPY, zz, rc, bar);
      tma_prefetch_l2_5d(tmF, xf, y0, zz, 0, rc);
      tma_prefetch_l2_5d(tmF1, xf, ya, zz, 3, rc);
      tma_prefetch_l2_5d(tmF2, xf, ya, zz, 7, rc);
      tma_prefetch_l2_5d(tmF2, xf, ya, zz, 11, rc);
      tma_prefetch_l2_5d(tmF1, xf, yb, zz, 4, rc);
      tma_prefetch_l2_5d(tmF2, xf, yb, zz, 9, rc);
      tma_prefetch_l2_5d(tmF2, xf, yb, zz, 13, rc);
      tma_prefetch_l2_4d(tmQ, 4 * X, Y, wrap(p - 1, nz), rc);
      tma_prefetch_l2_4d(tmQ1, X, Y, wrap(p - 1, nz), rc);
    } else {
      tma_load_3d(sl + L::OFF_U, tmU3, 4 * (x0 - B::UX + B::UPX), y0 - 1 + B::UPY, zz, bar);
      tma_prefetch_l2_4d(tmF, xf, y0, zz, 0);
      tma_prefetch_l2_4d(tmF1, xf, ya, zz, 3);
      tma_prefetch_l2_4d(tmF2, xf, ya, zz, 7);
      tma_prefetch_l2_4d(tmF2, xf, ya, zz, 11);
      tma_prefetch_l2_4d(tmF1, xf, yb, zz, 4);
      tma_prefetch_l2_4d(tmF2, xf, yb, zz, 9);
      tma_prefetch_l2_4d(tmF2, xf, yb, zz, 13);
      tma_prefetch_l2_3d(tmQ, 4 * X, Y, wrap(p - 1, nz));
      tma_prefetch_l2_3d(tmQ1, X, Y, wrap(p - 1, nz));
    }
  };
  auto wait = [&](int p) {
    const unsigned k = p - (z0 - 1);
    const bool ok = mbar_wait_bounded(&bars[k % L::SLOTS], (k / L::SLOTS) & 1, kWaitLimitNs);
    if (!ok) *abort_flag = 1;
    return ok;
  };
  // a staged plane beyond a wall: only its Q* is read (the anchored qw)
  auto ghost = [&](int p) { return WALLS && (p < 0 || p >= nz); };
  auto fill = [&](int p) {
    real* sl = slot(p);
    for (int t = threadIdx.x; t < L::GS / 4; t += blockDim.x) {  // Q*_yz in G2, the rest in G3
      sl[2 * L::GS + 4 * t + 2] = qw.yz;
      st4(sl + 3 * L::GS + 4 * t, qw.xx, qw.xy, qw.xz, qw.yy);
    }
  };
  // group g of the P / Q* box at box index idx (lane 0) and idx + TYH rows
  // (lane 1), and value l of it; the same for the u box
  auto PG = [&](const real* sl, int g, int idx, V v[4]) {
    ld4v<SPT>(sl, g * L::GS + 4 * idx, g * L::GS + 4 * (idx + TYH * AW), v);
  };
  auto PS = [&](const real* sl, int g, int l, int idx) {
    return vld<SPT>(sl, g * L::GS + 4 * idx + l, g * L::GS + 4 * (idx + TYH * AW) + l);
  };
  // u = (u_x, u_y, u_z) at u-box index idx (lane 0) and idx + TYH rows (lane 1)
  auto U3 = [&](const real* sl, int idx, V u[3]) {
    V v[4];
    ld4v<SPT>(sl + L::OFF_U, 4 * idx, 4 * (idx + TYH * B::UW), v);
    u[0] = v[1], u[1] = v[2], u[2] = v[3];
  };
  // acc +/- v by the sign of e (compile-time after unrolling)
  auto acc = [](V& a, int e, V v) {
    if (e > 0) a += v;
    else if (e < 0) a -= v;
  };

  bool aborted = false;
  if (threadIdx.x == 0)
    for (int p = z0 - 1; p <= z0 + 1; ++p) issue(p);
  wait(z0 - 1);
  wait(z0);

  // periodic source coordinates of the pull
  const int xm = wrap(gx - 1, nx), xp = wrap(gx + 1, nx);
  int ym[SPT], yp[SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    ym[k] = wrap(gy[k] - 1, ny);
    yp[k] = wrap(gy[k] + 1, ny);
  }
  const V inv_tau = V(m.inv_tau);
  const V it3 = V(m.inv_tau) * LCBP_Q(1, 3), it8 = V(m.inv_tau) * LCBP_Q(1, 8);
  const Model<V> mv = widen<V>(m);

  // One CTA barrier per plane, after the wait: past it every thread has
  // finished plane z-1, the last reader of the slot that the load of plane
  // z+2 overwrites (plane z-2), so that load is issued right after it.
  for (int z = z0; z < z1; ++z) {
    // populations f_i(y - e_i) and the site's rho - 1, issued before the
    // barrier wait so that they overlap it
    real fin_l[SPT][NV];
    const bool wlo = WALLS && z == 0, whi = WALLS && z == nz - 1;
    // beside a wall, the bounce-back directions read the reflected population
    // of the site itself (a build of its own; every other plane pulls)
    auto pull = [&](auto wall_plane) {
      constexpr bool WP = decltype(wall_plane)::value;
      const bool wl = WP && wlo, wh = WP && whi;
      const int zm = z == 0 ? nz - 1 : z - 1, zp = z + 1 == nz ? 0 : z + 1;
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        // three row bases per plane: rows y-1, y, y+1 of planes z-1, z, z+1
        const int rb[3][3] = {{(zm * ny + ym[k]) * nx, (zm * ny + gy[k]) * nx, (zm * ny + yp[k]) * nx},
                              {(z * ny + ym[k]) * nx, (z * ny + gy[k]) * nx, (z * ny + yp[k]) * nx},
                              {(zp * ny + ym[k]) * nx, (zp * ny + gy[k]) * nx, (zp * ny + yp[k]) * nx}};
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const int sx = ex(i) > 0 ? xm : ex(i) < 0 ? xp : gx;
          if ((ez(i) > 0 && wl) || (ez(i) < 0 && wh)) fin_l[k][i] = __ldg(f + (opp(i) * n + rb[1][1] + gx));
          else fin_l[k][i] = __ldg(f + (i * n + rb[1 - ez(i)][1 - ey(i)] + sx));
        }
      }
    };
    if (valid) {
      if (WALLS && (wlo || whi)) pull(std::true_type{});
      else pull(std::false_type{});
    }
    wait(z + 1);
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      break;
    }
    if (threadIdx.x == 0) {
      fence_proxy_async();
      if (z + 2 <= z1) issue(z + 2);
    }
    // a wall's ghost plane: the anchored Q*
    if (WALLS && (ghost(z + 1) || (z == z0 && ghost(z0 - 1)))) {
      if (ghost(z + 1)) fill(z + 1);
      if (z == z0 && ghost(z0 - 1)) fill(z0 - 1);
      __syncthreads();
    }
    // a plane beside a wall runs a build of the plane's work with the
    // bounce-back; every other plane runs the periodic build
    auto plane_work = [&](auto wall_plane) {
      constexpr bool WP = decltype(wall_plane)::value;
      const bool wl = WP && wlo, wh = WP && whi;
      int s[SPT];
#pragma unroll
      for (int k = 0; k < SPT; ++k) s[k] = (z * ny + gy[k]) * nx + gx;
      const real* nm = slot(z - 1);
      const real* nc = slot(z);
      const real* np = slot(z + 1);
      const int ca = (ty + 1) * AW + (tx + 1);          // the site in the P / Q* box
      const int cu = (ty + 1) * B::UW + (tx + B::UX);   // the site in the u box
      V fin[NV], ds[NV], dh[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if constexpr (SPT == 1) fin[i] = fin_l[0][i];
        else fin[i] = V(fin_l[0][i], fin_l[SPT - 1][i], 0);
      }
      // the site's G0 .. G2 of the scratch: [C V], [W F_x], [F_y F_z Q*_yz rho-1]
      V c0[4], c1[4], c2[4];
      PG(nc, 0, ca, c0);
      PG(nc, 1, ca, c1);
      PG(nc, 2, ca, c2);
      const V drho_y = c2[3];
      V u_y[3];
      U3(nc, cu, u_y);
      const V rho_y = V(1) + drho_y;
      const V jn[3] = {rho_y * u_y[0], rho_y * u_y[1], rho_y * u_y[2]};
      const V rusq_n = jn[0] * u_y[0] + jn[1] * u_y[1] + jn[2] * u_y[2];
      // f^eq_i / tau_f + p_i at the source site y - e_i from its staged
      // coefficients; at a wall the bounce-back directions take the site's own
      // term of the opposite direction (all signs flipped)
      V pre[NV];
      pre[0] = (drho_y * LCBP_Q(8, 15) - rusq_n * LCBP_Q(2, 3)) * inv_tau;
#pragma unroll
      for (int i = 1; i < NV; ++i) {
        const bool bb = (ez(i) > 0 && wl) || (ez(i) < 0 && wh);
        const real* sl = bb ? nc : (ez(i) > 0 ? nm : ez(i) < 0 ? np : nc);
        const int idx = bb ? ca : ca - ey(i) * AW - ex(i);
        if (i <= 6) {
          const int a = (i - 1) / 2;
          // F_a: G1.3 (x), G2.0 (y), G2.1 (z); V_a: G0.(1 + a)
          const V Fa = a == 0 ? PS(sl, 1, 3, idx) : PS(sl, 2, a - 1, idx), Va = PS(sl, 0, 1 + a, idx);
          pre[i] = ((i & 1) != 0) != bb ? Fa + Va : Fa - Va;  // odd i: the + direction
        } else {
          V g0[4], g1[4];  // [C, V_x, V_y, V_z], [W_xy, W_xz, W_yz, F_x]
          PG(sl, 0, idx, g0);
          PG(sl, 1, idx, g1);
          const V vs = signed_sum(ex(i), g0[1], ey(i), g0[2], ez(i), g0[3]);
          const V ws = signed_sum(ex(i) * ey(i), g1[0], ex(i) * ez(i), g1[1], ey(i) * ez(i), g1[2]);
          pre[i] = bb ? (g0[0] + ws) - LCBP_Q(1, 8) * vs : (g0[0] + ws) + LCBP_Q(1, 8) * vs;
        }
      }
      // C_i = (f^eq - f_i) / tau_f + p_i; predictor f* = f + C, and f + C / 2
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const V C = pre[i] - fin[i] * inv_tau;
        ds[i] = fin[i] + C;
        dh[i] = fin[i] + V(0.5) * C;
      }
      V drs = ds[0], jx = V(0), jy = V(0), jz = V(0);
#pragma unroll
      for (int i = 1; i < NV; ++i) {
        drs += ds[i];
        acc(jx, ex(i), ds[i]);
        acc(jy, ey(i), ds[i]);
        acc(jz, ez(i), ds[i]);
      }
      const V rs = V(1) + drs;
      const V inv_rs = recip(rs);
      const V us[3] = {jx * inv_rs, jy * inv_rs, jz * inv_rs};
      const V js[3] = {jx, jy, jz};
      const V rusq_s = jx * us[0] + jy * us[1] + jz * us[2];
      // Corrector: the same coefficients for (rho*, u*) with sigma and b held
      // at the site's step-n values.  P(y) holds them for (rho^n, u^n), so
      // each takes the change of its moment part.
      const V dd = (drs - drho_y) * LCBP_Q(1, 30) - (rusq_s - rusq_n) * LCBP_Q(1, 12);
      const V Fn[3] = {c1[3], c2[0], c2[1]};
      V Fs[3], Vs[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Fs[a] = Fn[a] + (dd + V(0.5) * (js[a] * us[a] - jn[a] * u_y[a])) * inv_tau;
        Vs[a] = c0[1 + a] + (js[a] - jn[a]) * it3;
      }
      const V Ws[3] = {c1[0] + (js[0] * us[1] - jn[0] * u_y[1]) * it8,
                       c1[1] + (js[0] * us[2] - jn[0] * u_y[2]) * it8,
                       c1[2] + (js[1] * us[2] - jn[1] * u_y[2]) * it8};
      const V Cs0 = (drs * LCBP_Q(1, 30) + rusq_s * LCBP_Q(1, 48)) * inv_tau;
      V dr1 = V(0), j1x = V(0), j1y = V(0), j1z = V(0);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        V prs;
        if (i == 0) {
          prs = (drs * LCBP_Q(8, 15) - rusq_s * LCBP_Q(2, 3)) * inv_tau;
        } else if (i <= 6) {
          const int a = (i - 1) / 2;
          prs = (i & 1) ? Fs[a] + Vs[a] : Fs[a] - Vs[a];
        } else {
          prs = (Cs0 + signed_sum(ex(i) * ey(i), Ws[0], ex(i) * ez(i), Ws[1], ey(i) * ez(i), Ws[2])) +
                LCBP_Q(1, 8) * signed_sum(ex(i), Vs[0], ey(i), Vs[1], ez(i), Vs[2]);
        }
        const V Cs = prs - ds[i] * inv_tau;
        const V fo = dh[i] + V(0.5) * Cs;
#pragma unroll
        for (int k = 0; k < SPT; ++k)
          if (lane_ok[k]) __stcs(&fnew[i * n + s[k]], lane<SPT, real>(fo, k));  // (streaming: not re-read here)
        dr1 = i == 0 ? fo : dr1 + fo;
        acc(j1x, ex(i), fo);
        acc(j1y, ey(i), fo);
        acc(j1z, ez(i), fo);
      }
      const V inv_r1 = recip(V(1) + dr1);
      const V u1x = j1x * inv_r1, u1y = j1y * inv_r1, u1z = j1z * inv_r1;
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        if (!lane_ok[k]) continue;
        const real a = lane<SPT, real>(dr1, k), b = lane<SPT, real>(u1x, k), c = lane<SPT, real>(u1y, k),
                   d = lane<SPT, real>(u1z, k);
        const int nxm = G.nxm, nyu = G.nyu;
        mirror_positions(B::UPX, 1, nx, ny, gx, gy[k],
                         [&](int X, int Y) { st4g(rhou_new + 4 * ((z * nyu + Y) * nxm + X), a, b, c, d); });
      }

      // Heun corrector with u^n
      // Q* at a box index: G3 = [xx xy xz yy] and G2.2 = yz
      auto QS = [&](const real* sl, int idx) {
        V g3[4];
        PG(sl, 3, idx, g3);
        return Sym5<V>{g3[0], g3[1], g3[2], g3[3], PS(sl, 2, 2, idx)};
      };
      Stencil7<V> st;
      V g3c[4];
      PG(nc, 3, ca, g3c);
      st.c = Sym5<V>{g3c[0], g3c[1], g3c[2], g3c[3], c2[2]};
      st.xm = QS(nc, ca - 1);
      st.xp = QS(nc, ca + 1);
      st.ym = QS(nc, ca - AW);
      st.yp = QS(nc, ca + AW);
      st.zm = QS(nm, ca);
      st.zp = QS(np, ca);
      Sym5<V> dq[3];
      const Sym5<V> h = molecular_field<true>(st, mv, dq);
      V w[3][3];
      const V half = V(0.5);
      V uxp[3], uxm[3], uyp[3], uym[3], uzp[3], uzm[3];
      U3(nc, cu + 1, uxp);
      U3(nc, cu - 1, uxm);
      U3(nc, cu + B::UW, uyp);
      U3(nc, cu - B::UW, uym);
      U3(np, cu, uzp);
      U3(nm, cu, uzm);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        w[a][0] = uxp[a] - uxm[a];  // twice the central derivatives
        w[a][1] = uyp[a] - uym[a];
        V upz = uzp[a], umz = uzm[a];
        if (wl) umz = -u_y[a];  // no slip half a spacing beyond the wall
        if (wh) upz = -u_y[a];
        w[a][2] = upz - umz;
      }
      const Sym5<V> r = be_rate<true>(st.c, h, dq, u_y, w, mv, true);
      // Q^n of the site: the flat field, or the Q mirror ([xx xy xz yy]
      // vectors, then the yz array)
      int sq[SPT];
#pragma unroll
      for (int k = 0; k < SPT; ++k) sq[k] = (z * G.nyq + gy[k] + B::QPY) * G.nxm + gx + B::QPX;
      const int cq = (int)G.cq;
      V qa[4];
      ld4v<SPT>(Qin, 4 * sq[0], 4 * sq[SPT - 1], qa);
      const Sym5<V> q0 = {qa[0], qa[1], qa[2], qa[3], vld<SPT>(Qin, 4 * cq + sq[0], 4 * cq + sq[SPT - 1])};
      const Sym5<V> q1 = {half * (q0.xx + st.c.xx + r.xx), half * (q0.xy + st.c.xy + r.xy),
                          half * (q0.xz + st.c.xz + r.xz), half * (q0.yy + st.c.yy + r.yy),
                          half * (q0.yz + st.c.yz + r.yz)};
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        if (!lane_ok[k]) continue;
        const real a = lane<SPT, real>(q1.xx, k), b = lane<SPT, real>(q1.xy, k), c = lane<SPT, real>(q1.xz, k),
                   d = lane<SPT, real>(q1.yy, k), e = lane<SPT, real>(q1.yz, k);
        const int nxm = G.nxm, nyq = G.nyq, cq4 = 4 * (int)G.cq;
        mirror_positions(B::QPX, 2, nx, ny, gx, gy[k], [&](int X, int Y) {
          const int o = (z * nyq + Y) * nxm + X;
          st4g(Qout + 4 * o, a, b, c, d);
          __stcs(&Qout[cq4 + o], e);
        });
      }
    };
    if (valid) {
      if (WALLS && (wlo || whi)) plane_work(std::true_type{});
      else plane_work(std::false_type{});
    }
  }
  if (aborted && threadIdx.x == 0) {
    atomicExch(err, 1);
    for (int i = 0; i < L::SLOTS; ++i) {
      mbar_wait_bounded(&bars[i], 0, kWaitLimitNs / 16);
      mbar_wait_bounded(&bars[i], 1, kWaitLimitNs / 16);
    }
  }
}

template <typename real, int TY, int SPT, bool WALLS>
__global__ void __launch_bounds__(ZM_TX* TY / SPT, 2)
    k_lbq(const __grid_constant__ CUtensorMap tmPQ, const __grid_constant__ CUtensorMap tmU3,
          const __grid_constant__ CUtensorMap tmF, const __grid_constant__ CUtensorMap tmF1,
          const __grid_constant__ CUtensorMap tmF2, const __grid_constant__ CUtensorMap tmQ,
          const __grid_constant__ CUtensorMap tmQ1, ZmGeom G, Model<real> m, const real* __restrict__ f,
          const real* __restrict__ Qin, real* __restrict__ fnew, real* __restrict__ rhou_new, real* __restrict__ Qout,
          int* __restrict__ err, Sym5<real> qw) {
  lbq_body<real, TY, SPT, false, WALLS>(&tmPQ, &tmU3, &tmF, &tmF1, &tmF2, &tmQ, &tmQ1, G, m, blockIdx.x, 0, f, Qin,
                                        fnew, rhou_new, Qout, err, qw);
}

template <typename real, int TY>
__global__ void __launch_bounds__(ZM_TX* TY, 2)
    k_lbq_batch(const __grid_constant__ ZmBatchMaps maps, ZmBatch B, const Replica<real>* __restrict__ reps,
                const int* __restrict__ order, const real* __restrict__ f, const real* __restrict__ Qin,
                real* __restrict__ fnew, real* __restrict__ rhou_new, real* __restrict__ Qout,
                int* __restrict__ err) {
  const ZmItem it = zm_item(B);
  const ZmGeom G = zm_class_geom(B, it.k);
  int rep0 = B.c[0].rep0;
  long long qm0 = B.c[0].qm0, um0 = B.c[0].um0;
#pragma unroll
  for (int i = 1; i < kZmMaxClasses; ++i)
    if (i == it.k) {
      rep0 = B.c[i].rep0;
      qm0 = B.c[i].qm0;
      um0 = B.c[i].um0;
    }
  const int r = order[rep0 + it.j];
  const long long o = reps[r].base;  // the flat populations of the replica
  const long long qo = qm0 + (long long)it.j * 5 * G.cq, uo = um0 + (long long)it.j * 4 * G.cu;  // its mirrors
  const Model<real> m = reps[r].m;
  const CUtensorMap *mpq = &maps.pq[0], *mu3 = &maps.u3[0], *mf = &maps.f[0], *mf1 = &maps.f1[0],
                    *mf2 = &maps.f2[0], *mq = &maps.qpf[0], *mq1 = &maps.q1pf[0];
#pragma unroll
  for (int i = 1; i < kZmMaxClasses; ++i)
    if (i == it.k) {
      mpq = &maps.pq[i];
      mu3 = &maps.u3[i];
      mf = &maps.f[i];
      mf1 = &maps.f1[i];
      mf2 = &maps.f2[i];
      mq = &maps.qpf[i];
      mq1 = &maps.q1pf[i];
    }
  if constexpr (sizeof(real) == 4) {
    if (G.tx == kZmNarrowX) {
      lbq_body<real, 2 * TY, 1, true, false, kZmNarrowX>(mpq, mu3, mf, mf1, mf2, mq, mq1, G, m, it.bt, it.j,
                                                         f + NV * o, Qin + qo, fnew + NV * o, rhou_new + uo,
                                                         Qout + qo, err, Sym5<real>{});
      return;
    }
  }
  lbq_body<real, TY, 1, true, false>(mpq, mu3, mf, mf1, mf2, mq, mq1, G, m, it.bt, it.j, f + NV * o, Qin + qo,
                                     fnew + NV * o, rhou_new + uo, Qout + qo, err, Sym5<real>{});
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

// A narrow batch tile has the sites, threads and at most the shared memory of a full one
static_assert(kZmNarrowX * 2 * zm_ty<float>() == ZM_TX * zm_ty<float>(), "narrow tile sites");
static_assert(qside_threads<2 * zm_ty<float>(), 1, kZmNarrowX>() == qside_threads<zm_ty<float>(), 1>(),
              "narrow k_qside threads");
static_assert(QsideSmem<float, 2 * zm_ty<float>(), kZmNarrowX>::bytes <= QsideSmem<float, zm_ty<float>()>::bytes &&
                  LbqSmem<float, 2 * zm_ty<float>(), kZmNarrowX>::bytes <= LbqSmem<float, zm_ty<float>()>::bytes,
              "narrow tiles fit the full tiles' shared memory");

// sites per thread the kernels are built for: FP32 one or two, FP64 one
template <typename real>
constexpr int zm_max_spt() {
  return sizeof(real) == 4 ? 2 : 1;
}

template <typename real, int SPT, bool WALLS>
cudaError_t zm_prepare_spt() {
  constexpr int TY = zm_ty<real>();
  cudaError_t e = cudaFuncSetAttribute(k_qside<real, TY, SPT, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)QsideSmem<real, TY>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lbq<real, TY, SPT, WALLS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)LbqSmem<real, TY>::bytes);
  return e;
}

// lattices with walls run one site per thread
template <typename real>
cudaError_t zm_prepare() {
  cudaError_t e = zm_prepare_spt<real, 1, false>();
  if (e == cudaSuccess) e = zm_prepare_spt<real, 1, true>();
  if constexpr (zm_max_spt<real>() == 2)
    if (e == cudaSuccess) e = zm_prepare_spt<real, 2, false>();
  return e;
}

template <typename real>
int zm_spt_max() {
  return zm_max_spt<real>();
}

// CTAs of k_lbq (the longer kernel) resident per SM at `spt` sites per thread
template <typename real, int SPT>
int zm_resident_spt() {
  constexpr int TY = zm_ty<real>();
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lbq<real, TY, SPT, false>, ZM_TX * TY / SPT,
                                                    LbqSmem<real, TY>::bytes) != cudaSuccess)
    n = 1;
  return n > 0 ? n : 1;
}

template <typename real>
int zm_resident(int spt) {
  if constexpr (zm_max_spt<real>() == 2)
    if (spt == 2) return zm_resident_spt<real, 2>();
  return zm_resident_spt<real, 1>();
}

ZmGeom zm_geom(int nx, int ny, int nz, int zc, int ty) {
  ZmGeom G;
  G.nx = nx;
  G.ny = ny;
  G.nz = nz;
  G.zc = zc;
  G.n = (long long)nx * ny * nz;
  G.tx = ZM_TX;
  G.ty = ty;
  G.tiles_x = (nx + ZM_TX - 1) / ZM_TX;
  G.tiles_y = (ny + ty - 1) / ty;
  G.tiles_z = (nz + zc - 1) / zc;
  G.nxp = nx + kZmPadX;
  G.nyp = ny + 2;
  G.cp = (long long)G.nxp * G.nyp * nz;
  G.nxm = zm_mirror_nx(nx);
  G.nyq = ny + 4;
  G.nyu = ny + 2;
  G.cq = (long long)G.nxm * G.nyq * nz;
  G.cu = (long long)G.nxm * G.nyu * nz;
  return G;
}

template <typename real, int SQ, int SPT, bool WALLS>
cudaError_t launch_step_zm_spt(const ZmArgs& a, cudaStream_t s) {
  constexpr int TY = zm_ty<real>();
  // each kernel marches its own planes per CTA
  const ZmGeom G = zm_geom(a.nx, a.ny, a.nz, a.zc, TY), Gq = zm_geom(a.nx, a.ny, a.nz, a.zc_q > 0 ? a.zc_q : a.zc, TY);
  const int grid = G.tiles_x * G.tiles_y * G.tiles_z, grid_q = Gq.tiles_x * Gq.tiles_y * Gq.tiles_z;
  const Model<real> m = *static_cast<const Model<real>*>(a.model);
  Sym5<real> qw{};
  if (WALLS) qw = {(real)a.q_wall[0], (real)a.q_wall[1], (real)a.q_wall[2], (real)a.q_wall[3], (real)a.q_wall[4]};
  if (a.events) cudaEventRecord(a.events[0], s);
  k_qside<real, TY, SQ, WALLS><<<grid_q, qside_threads<TY, SQ>(), QsideSmem<real, TY>::bytes, s>>>(
      *a.tm_q, *a.tm_q1, *a.tm_u, Gq, m, static_cast<const real*>(a.bext), static_cast<real*>(a.pq), a.err, qw);
  if (a.events) cudaEventRecord(a.events[1], s);
  k_lbq<real, TY, SPT, WALLS><<<grid, ZM_TX * TY / SPT, LbqSmem<real, TY>::bytes, s>>>(
      *a.tm_pq, *a.tm_u3, *a.tm_f, *a.tm_f1, *a.tm_f2, *a.tm_qpf, *a.tm_q1pf, G, m, static_cast<const real*>(a.f),
      static_cast<const real*>(a.q), static_cast<real*>(a.fnew), static_cast<real*>(a.rhou_new),
      static_cast<real*>(a.qout ? a.qout : a.q), a.err, qw);
  if (a.events) cudaEventRecord(a.events[2], s);
  return cudaGetLastError();
}

// sites per thread chosen for each kernel separately (FP32: 1 or 2 each; walls and FP64: 1)
template <typename real>
cudaError_t launch_step_zm(const ZmArgs& a, cudaStream_t s) {
  if (a.q_wall) return launch_step_zm_spt<real, 1, 1, true>(a, s);
  if constexpr (zm_max_spt<real>() == 2) {
    const int sq = a.spt_q > 0 ? a.spt_q : a.spt;
    if (sq == 2 && a.spt == 2) return launch_step_zm_spt<real, 2, 2, false>(a, s);
    if (sq == 2) return launch_step_zm_spt<real, 2, 1, false>(a, s);
    if (a.spt == 2) return launch_step_zm_spt<real, 1, 2, false>(a, s);
  }
  return launch_step_zm_spt<real, 1, 1, false>(a, s);
}

template <typename real>
cudaError_t zm_batch_prepare() {
  constexpr int TY = zm_ty<real>();
  cudaError_t e = cudaFuncSetAttribute(k_qside_batch<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)QsideSmem<real, TY>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lbq_batch<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)LbqSmem<real, TY>::bytes);
  return e;
}

template <typename real>
cudaError_t launch_step_zm_batch(const ZmBatchArgs& a, cudaStream_t s) {
  constexpr int TY = zm_ty<real>();
  const auto* reps = static_cast<const Replica<real>*>(a.reps);
  if (a.events) cudaEventRecord(a.events[0], s);
  k_qside_batch<real, TY><<<a.Bq.total_ctas, qside_threads<TY, 1>(), QsideSmem<real, TY>::bytes, s>>>(
      *a.maps, a.Bq, reps, a.order, static_cast<real*>(a.pq), a.err);
  if (a.events) cudaEventRecord(a.events[1], s);
  k_lbq_batch<real, TY><<<a.B.total_ctas, ZM_TX * TY, LbqSmem<real, TY>::bytes, s>>>(
      *a.maps, a.B, reps, a.order, static_cast<const real*>(a.f), static_cast<const real*>(a.q),
      static_cast<real*>(a.fnew), static_cast<real*>(a.rhou_new), static_cast<real*>(a.qout ? a.qout : a.q), a.err);
  if (a.events) cudaEventRecord(a.events[2], s);
  return cudaGetLastError();
}

template cudaError_t zm_prepare<float>();
template cudaError_t zm_prepare<double>();
template cudaError_t zm_batch_prepare<float>();
template cudaError_t zm_batch_prepare<double>();
template cudaError_t launch_step_zm_batch<float>(const ZmBatchArgs&, cudaStream_t);
template cudaError_t launch_step_zm_batch<double>(const ZmBatchArgs&, cudaStream_t);
template int zm_tile_rows<float>();
template int zm_tile_rows<double>();
template int zm_spt_max<float>();
template int zm_spt_max<double>();
template int zm_resident<float>(int);
template int zm_resident<double>(int);
template cudaError_t launch_step_zm<float>(const ZmArgs&, cudaStream_t);
template cudaError_t launch_step_zm<double>(const ZmArgs&, cudaStream_t);

}  // namespace lcbp
