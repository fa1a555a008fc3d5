// The three kernels of one coupled step (Sec. 2.2, hybrid scheme).
//
//   k_field          Q^n            -> H(Q^n), sigma_LC, tau          (Eq. Qevolution, BEstress)
//   k_force_predict  Q^n, H, tau, u -> b (Eq. eq7a + spurious), Q* = Q^n + R(Q^n)   (Heun predictor)
//   k_lb_correct     f^n, rho u, sigma, b, Q*, Q^n
//                    -> f^{n+1}, rho u^{n+1} (Eq. eq2, eq4, feq, coeff),
//                       Q^{n+1} = (Q^n + Q* + R(Q*)) / 2                       (Heun corrector)
//
// One thread per site; each CTA walks a list of tiles (replica, origin) so
// that a single launch covers every replica of a batch.  Neighbour values
// come through the read-only data path (L1/L2); the halo of a tile is
// re-read from L2, not from HBM.
#include "common.cuh"
#include "kernels.h"

namespace lcbp {

template <typename real>
__device__ __forceinline__ bool tile_site(const Replica<real>* reps, const Tile* tiles, int t, TileShape ts,
                                          Replica<real>& R, int& x, int& y, int& z) {
  const Tile tl = tiles[t];
  R = reps[tl.rep];
  const int tid = threadIdx.x;
  const int lx = tid % ts.tx;
  const int ly = (tid / ts.tx) % ts.ty;
  const int lz = tid / (ts.tx * ts.ty);
  x = tl.x0 + lx;
  y = tl.y0 + ly;
  z = tl.z0 + lz;
  return lz < ts.tz && x < R.nx && y < R.ny && z < R.nz;
}

// velocity at a site from the stored moments [rho, ux, uy, uz]
template <typename real>
__device__ __forceinline__ void load_u(const real* __restrict__ ru, long long n, long long s, real u[3]) {
  u[0] = __ldg(ru + n + s);
  u[1] = __ldg(ru + 2 * n + s);
  u[2] = __ldg(ru + 3 * n + s);
}

// W_ab = D0_b u_a from the 6 face neighbours; beyond a wall the ghost velocity
// is -u of the site itself (no slip half a spacing away), u_own = u at b.s
template <typename real>
__device__ __forceinline__ void velocity_gradient(const real* __restrict__ ru, long long n, const Nbr& b,
                                                  int nx, int ny, real w[3][3], const real* u_own = nullptr) {
  real up[3], um[3];
  load_u(ru, n, b.at(b.xp, b.y, b.z, nx, ny), up);
  load_u(ru, n, b.at(b.xm, b.y, b.z, nx, ny), um);
#pragma unroll
  for (int a = 0; a < 3; ++a) w[a][0] = real(0.5) * (up[a] - um[a]);
  load_u(ru, n, b.at(b.x, b.yp, b.z, nx, ny), up);
  load_u(ru, n, b.at(b.x, b.ym, b.z, nx, ny), um);
#pragma unroll
  for (int a = 0; a < 3; ++a) w[a][1] = real(0.5) * (up[a] - um[a]);
  load_u(ru, n, b.at(b.x, b.y, b.zp, nx, ny), up);
  load_u(ru, n, b.at(b.x, b.y, b.zm, nx, ny), um);
  if (u_own && b.whi) {
#pragma unroll
    for (int a = 0; a < 3; ++a) up[a] = -u_own[a];
  }
  if (u_own && b.wlo) {
#pragma unroll
    for (int a = 0; a < 3; ++a) um[a] = -u_own[a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) w[a][2] = real(0.5) * (up[a] - um[a]);
}

// ---------------------------------------------------------------------------
// DIV: the lattice has L2 != K (the divergence term of H is compiled in only here)
template <typename real, bool FLOW, bool DIV = false>
__global__ void __launch_bounds__(256) k_field(const Replica<real>* __restrict__ reps,
                                               const Tile* __restrict__ tiles, int ntiles, TileShape ts,
                                               const real* __restrict__ Q, real* __restrict__ H,
                                               real* __restrict__ sigma, real* __restrict__ tau) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int x, y, z;
    if (!tile_site(reps, tiles, t, ts, R, x, y, z)) continue;
    const long long n = R.n;
    const Nbr nb = make_nbr(x, y, z, R.nx, R.ny, R.nz, R.walls);
    const Stencil7<real> st = load_stencil(Q + 5 * R.base, n, nb, R);
    Sym5<real> dq[3];
    Sym5<real> h = molecular_field(st, R.m, dq);
    if (DIV) add_div_field(h, Q + 5 * R.base, n, x, y, z, R.nx, R.ny, R.nz, R.m.c_div);
    store5(H + 5 * R.base, n, nb.s, h);
    if (FLOW) {
      Sym5<real> sg;
      real tu[3];
      lc_stress(st.c, h, R.m.xi, sg, tu);
      store5(sigma + 5 * R.base, n, nb.s, sg);
      real* tp = tau + 3 * R.base;
      tp[nb.s] = tu[0];
      tp[n + nb.s] = tu[1];
      tp[2 * n + nb.s] = tu[2];
    }
  }
}

// ---------------------------------------------------------------------------
// DO_B: body force b = D0_b tau_ab - H_gn D0_a Q_gn (+ external force)
// DO_QS: Heun predictor Q* = Q + R(Q, u); FLOW: u from the stored moments,
//        else u = 0.
template <typename real, bool FLOW, bool DO_B, bool DO_QS, bool BEXT>
__global__ void __launch_bounds__(256) k_force_predict(const Replica<real>* __restrict__ reps,
                                                       const Tile* __restrict__ tiles, int ntiles, TileShape ts,
                                                       const real* __restrict__ Q, const real* __restrict__ H,
                                                       const real* __restrict__ tau, const real* __restrict__ rhou,
                                                       const real* __restrict__ bext, real* __restrict__ bout,
                                                       real* __restrict__ Qs) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int x, y, z;
    if (!tile_site(reps, tiles, t, ts, R, x, y, z)) continue;
    const long long n = R.n;
    const Nbr nb = make_nbr(x, y, z, R.nx, R.ny, R.nz, R.walls);
    const Stencil7<real> st = load_stencil(Q + 5 * R.base, n, nb, R);
    Sym5<real> dq[3];
    dq[0] = half_diff(st.xp, st.xm);
    dq[1] = half_diff(st.yp, st.ym);
    dq[2] = half_diff(st.zp, st.zm);
    const Sym5<real> h = load5(H + 5 * R.base, n, nb.s);
    if (DO_B) {
      const real* tp = tau + 3 * R.base;
      auto tv = [&](int c, long long s) { return __ldg(tp + c * n + s); };
      // tau on a ghost plane beyond a wall is 0 (the wall carries no molecular field)
      auto tvzp = [&](int c, long long s) { return nb.whi ? real(0) : tv(c, s); };
      auto tvzm = [&](int c, long long s) { return nb.wlo ? real(0) : tv(c, s); };
      const long long sxp = nb.at(nb.xp, y, z, R.nx, R.ny), sxm = nb.at(nb.xm, y, z, R.nx, R.ny);
      const long long syp = nb.at(x, nb.yp, z, R.nx, R.ny), sym = nb.at(x, nb.ym, z, R.nx, R.ny);
      const long long szp = nb.at(x, y, nb.zp, R.nx, R.ny), szm = nb.at(x, y, nb.zm, R.nx, R.ny);
      // tau = [xy, xz, yz], tau_yx = -tau_xy etc.
      const real half = real(0.5);
      real bx = half * (tv(0, syp) - tv(0, sym)) + half * (tvzp(1, szp) - tvzm(1, szm));
      real by = -half * (tv(0, sxp) - tv(0, sxm)) + half * (tvzp(2, szp) - tvzm(2, szm));
      real bz = -half * (tv(1, sxp) - tv(1, sxm)) - half * (tv(2, syp) - tv(2, sym));
      bx -= ddot(h, dq[0]);
      by -= ddot(h, dq[1]);
      bz -= ddot(h, dq[2]);
      if (BEXT) {
        const real* be = bext + 3 * R.base;
        bx += __ldg(be + nb.s);
        by += __ldg(be + n + nb.s);
        bz += __ldg(be + 2 * n + nb.s);
      }
      real* bo = bout + 3 * R.base;
      bo[nb.s] = bx;
      bo[n + nb.s] = by;
      bo[2 * n + nb.s] = bz;
    }
    if (DO_QS) {
      real u[3] = {real(0), real(0), real(0)};
      real w[3][3] = {};
      if (FLOW) {
        const real* ru = rhou + 4 * R.base;
        load_u(ru, n, nb.s, u);
        velocity_gradient(ru, n, nb, R.nx, R.ny, w, u);
      }
      const Sym5<real> r = be_rate(st.c, h, dq, u, w, R.m, FLOW);
      const Sym5<real> qs = {st.c.xx + r.xx, st.c.xy + r.xy, st.c.xz + r.xz, st.c.yy + r.yy, st.c.yz + r.yz};
      store5(Qs + 5 * R.base, n, nb.s, qs);
    }
  }
}

// ---------------------------------------------------------------------------
// DO_LB: predictor-corrector LB (pull form) writing f^{n+1} and its moments.
// DO_Q2: Heun corrector for Q with u from `rhou_q` (u^n for Jacobi coupling,
//        u^{n+1} for Gauss-Seidel), in place on Q.
template <typename real, bool FLOW, bool DO_LB, bool DO_Q2, bool WALLS = false, bool DIV = false>
__global__ void __launch_bounds__(256) k_lb_correct(const Replica<real>* __restrict__ reps,
                                                    const Tile* __restrict__ tiles, int ntiles, TileShape ts,
                                                    const real* __restrict__ f, const real* __restrict__ rhou,
                                                    const real* __restrict__ sigma, const real* __restrict__ bf,
                                                    real* __restrict__ fnew, real* __restrict__ rhou_new,
                                                    const real* __restrict__ Qs, const real* __restrict__ rhou_q,
                                                    const real* Qin, real* Qout) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int x, y, z;
    if (!tile_site(reps, tiles, t, ts, R, x, y, z)) continue;
    const long long n = R.n;
    const int nx = R.nx, ny = R.ny;
    // walls: Q and u ghosts are handled at run time; the LB bounce-back is
    // compiled in only for WALLS (a lattice with walls launches that build)
    const Nbr nb = make_nbr(x, y, z, nx, ny, R.nz, R.walls);
    if (DO_LB) {
      // populations and density are stored as deviations df = f - w, drho = rho - 1
      const real* fr = f + 15 * R.base;
      const real* ru = rhou + 4 * R.base;
      const real* sg = sigma + 5 * R.base;
      const real* bb = bf + 3 * R.base;
      const real inv_tau = R.m.inv_tau;
      real ds[NV], dh[NV];  // predictor f* and f + C/2, pulled from y - e_i (deviation form)
      Sym5<real> sig_y;
      real b_y[3];
      real drho_y = real(0), u_y[3] = {real(0), real(0), real(0)};
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if (WALLS && ((ez(i) > 0 && nb.wlo) || (ez(i) < 0 && nb.whi))) {
          // half-way bounce-back: the population arriving from beyond the wall
          // is the reflected one of this site, [f + C]_opp(i)(y)
          const int o = opp(i);
          const real di = __ldg(fr + o * n + nb.s);
          const real usq = u_y[0] * u_y[0] + u_y[1] * u_y[1] + u_y[2] * u_y[2];
          const real C = -(di - feq_delta(o, drho_y, real(1) + drho_y, u_y[0], u_y[1], u_y[2], usq, sig_y)) * inv_tau +
                         force_dir(o, b_y[0], b_y[1], b_y[2]);
          ds[i] = di + C;
          dh[i] = di + real(0.5) * C;
          continue;
        }
        // source site y - e_i
        const int sx = ex(i) > 0 ? nb.xm : ex(i) < 0 ? nb.xp : x;
        const int sy = ey(i) > 0 ? nb.ym : ey(i) < 0 ? nb.yp : y;
        const int sz = ez(i) > 0 ? nb.zm : ez(i) < 0 ? nb.zp : z;
        const long long src = ((long long)sz * ny + sy) * nx + sx;
        const real di = __ldg(fr + i * n + src);
        const real drho = __ldg(ru + src);
        const real ux = __ldg(ru + n + src), uy = __ldg(ru + 2 * n + src), uz = __ldg(ru + 3 * n + src);
        const Sym5<real> s = load5(sg, n, src);
        const real bx = __ldg(bb + src), by = __ldg(bb + n + src), bz = __ldg(bb + 2 * n + src);
        if (i == 0) {
          sig_y = s;
          b_y[0] = bx; b_y[1] = by; b_y[2] = bz;
          drho_y = drho;
          u_y[0] = ux; u_y[1] = uy; u_y[2] = uz;
        }
        const real usq = ux * ux + uy * uy + uz * uz;
        const real C = -(di - feq_delta(i, drho, real(1) + drho, ux, uy, uz, usq, s)) * inv_tau +
                       force_dir(i, bx, by, bz);
        ds[i] = di + C;
        dh[i] = di + real(0.5) * C;
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
      real* fo = fnew + 15 * R.base;
      real dr1 = real(0), j1x = real(0), j1y = real(0), j1z = real(0);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const real Cs = -(ds[i] - feq_delta(i, drs, rs, usx, usy, usz, ussq, sig_y)) * inv_tau +
                        force_dir(i, b_y[0], b_y[1], b_y[2]);
        const real fo_i = dh[i] + real(0.5) * Cs;
        fo[i * n + nb.s] = fo_i;
        dr1 += fo_i;
        j1x += real(ex(i)) * fo_i;
        j1y += real(ey(i)) * fo_i;
        j1z += real(ez(i)) * fo_i;
      }
      real* rn = rhou_new + 4 * R.base;
      const real inv_r1 = real(1) / (real(1) + dr1);
      rn[nb.s] = dr1;
      rn[n + nb.s] = j1x * inv_r1;
      rn[2 * n + nb.s] = j1y * inv_r1;
      rn[3 * n + nb.s] = j1z * inv_r1;
    }
    if (DO_Q2) {
      const Stencil7<real> st = load_stencil(Qs + 5 * R.base, n, nb, R);
      Sym5<real> dq[3];
      Sym5<real> h = molecular_field(st, R.m, dq);
      if (DIV) add_div_field(h, Qs + 5 * R.base, n, x, y, z, nx, ny, R.nz, R.m.c_div);
      real u[3] = {real(0), real(0), real(0)};
      real w[3][3] = {};
      if (FLOW) {
        const real* ru = rhou_q + 4 * R.base;
        load_u(ru, n, nb.s, u);
        velocity_gradient(ru, n, nb, nx, ny, w, u);
      }
      const Sym5<real> r = be_rate(st.c, h, dq, u, w, R.m, FLOW);
      const Sym5<real> q0 = load5(Qin + 5 * R.base, n, nb.s);
      const real half = real(0.5);
      const Sym5<real> q1 = {half * (q0.xx + st.c.xx + r.xx), half * (q0.xy + st.c.xy + r.xy),
                             half * (q0.xz + st.c.xz + r.xz), half * (q0.yy + st.c.yy + r.yy),
                             half * (q0.yz + st.c.yz + r.yz)};
      store5(Qout + 5 * R.base, n, nb.s, q1);
    }
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// the field and corrector kernels in the build with or without the divergence
// term of H (L2 != K); walls and L2 never come together
template <typename real, bool FLOW, typename... Args>
void launch_fld(bool div, int grid, int threads, cudaStream_t s, Args... args) {
  if (div) k_field<real, FLOW, true><<<grid, threads, 0, s>>>(args...);
  else k_field<real, FLOW, false><<<grid, threads, 0, s>>>(args...);
}
template <typename real, bool FLOW, bool DO_LB, bool DO_Q2, bool WALLS, typename... Args>
void launch_lbc(bool div, int grid, int threads, cudaStream_t s, Args... args) {
  if constexpr (!WALLS && DO_Q2) {
    if (div) {
      k_lb_correct<real, FLOW, DO_LB, DO_Q2, false, true><<<grid, threads, 0, s>>>(args...);
      return;
    }
  }
  k_lb_correct<real, FLOW, DO_LB, DO_Q2, WALLS, false><<<grid, threads, 0, s>>>(args...);
}

template <typename real>
cudaError_t launch_step(const StepArgs& a, cudaStream_t s) {
  const auto* reps = static_cast<const Replica<real>*>(a.reps);
  const int threads = a.ts.tx * a.ts.ty * a.ts.tz;
  // persistent CTAs walk the tile list when a cap is given
  const int grid = a.max_grid > 0 && a.max_grid < a.ntiles ? a.max_grid : a.ntiles;
  void* qout = a.qout ? a.qout : a.q;
  auto Rp = [](void* p) { return static_cast<real*>(p); };
  auto Cp = [](const void* p) { return static_cast<const real*>(p); };
  int k = 0;
  auto mark = [&]() {
    if (a.events) cudaEventRecord(a.events[k], s);
    ++k;
  };
  mark();
  if (a.flow_on) {
    launch_fld<real, true>(a.div, grid, threads, s, reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Rp(a.h), Rp(a.sigma),
                           Rp(a.tau));
    mark();
    if (a.coupling == 0) {
      if (a.bext)
        k_force_predict<real, true, true, true, true><<<grid, threads, 0, s>>>(
            reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Cp(a.h), Cp(a.tau), Cp(a.rhou), Cp(a.bext), Rp(a.b), Rp(a.qs));
      else
        k_force_predict<real, true, true, true, false><<<grid, threads, 0, s>>>(
            reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Cp(a.h), Cp(a.tau), Cp(a.rhou), nullptr, Rp(a.b), Rp(a.qs));
      mark();
      if (a.walls)
        launch_lbc<real, true, true, true, true>(a.div, grid, threads, s, reps, a.tiles, a.ntiles, a.ts, Cp(a.f),
                                                 Cp(a.rhou), Cp(a.sigma), Cp(a.b), Rp(a.fnew), Rp(a.rhou_new),
                                                 Cp(a.qs), Cp(a.rhou), Cp(a.q), Rp(qout));
      else
        launch_lbc<real, true, true, true, false>(a.div, grid, threads, s, reps, a.tiles, a.ntiles, a.ts, Cp(a.f),
                                                  Cp(a.rhou), Cp(a.sigma), Cp(a.b), Rp(a.fnew), Rp(a.rhou_new),
                                                  Cp(a.qs), Cp(a.rhou), Cp(a.q), Rp(qout));
      mark();
    } else {
      // Gauss-Seidel: b, LB, then the Heun stages with u^{n+1}
      if (a.bext)
        k_force_predict<real, true, true, false, true><<<grid, threads, 0, s>>>(
            reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Cp(a.h), Cp(a.tau), Cp(a.rhou), Cp(a.bext), Rp(a.b), nullptr);
      else
        k_force_predict<real, true, true, false, false><<<grid, threads, 0, s>>>(
            reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Cp(a.h), Cp(a.tau), Cp(a.rhou), nullptr, Rp(a.b), nullptr);
      mark();
      if (a.walls)
        k_lb_correct<real, true, true, false, true><<<grid, threads, 0, s>>>(
            reps, a.tiles, a.ntiles, a.ts, Cp(a.f), Cp(a.rhou), Cp(a.sigma), Cp(a.b), Rp(a.fnew), Rp(a.rhou_new),
            nullptr, nullptr, nullptr, nullptr);
      else
        k_lb_correct<real, true, true, false><<<grid, threads, 0, s>>>(
            reps, a.tiles, a.ntiles, a.ts, Cp(a.f), Cp(a.rhou), Cp(a.sigma), Cp(a.b), Rp(a.fnew), Rp(a.rhou_new),
            nullptr, nullptr, nullptr, nullptr);
      mark();
      k_force_predict<real, true, false, true, false><<<grid, threads, 0, s>>>(
          reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Cp(a.h), nullptr, Cp(a.rhou_new), nullptr, nullptr, Rp(a.qs));
      mark();
      launch_lbc<real, true, false, true, false>(a.div, grid, threads, s, reps, a.tiles, a.ntiles, a.ts,
                                                 (const real*)nullptr, (const real*)nullptr, (const real*)nullptr,
                                                 (const real*)nullptr, (real*)nullptr, (real*)nullptr, Cp(a.qs),
                                                 Cp(a.rhou_new), Cp(a.q), Rp(qout));
      mark();
    }
  } else {
    launch_fld<real, false>(a.div, grid, threads, s, reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Rp(a.h), (real*)nullptr,
                            (real*)nullptr);
    mark();
    k_force_predict<real, false, false, true, false><<<grid, threads, 0, s>>>(
        reps, a.tiles, a.ntiles, a.ts, Cp(a.q), Cp(a.h), nullptr, nullptr, nullptr, nullptr, Rp(a.qs));
    mark();
    launch_lbc<real, false, false, true, false>(a.div, grid, threads, s, reps, a.tiles, a.ntiles, a.ts,
                                                (const real*)nullptr, (const real*)nullptr, (const real*)nullptr,
                                                (const real*)nullptr, (real*)nullptr, (real*)nullptr, Cp(a.qs),
                                                (const real*)nullptr, Cp(a.q), Rp(qout));
    mark();
  }
  return cudaGetLastError();
}

template cudaError_t launch_step<float>(const StepArgs&, cudaStream_t);
template cudaError_t launch_step<double>(const StepArgs&, cudaStream_t);

// sigma_LC(Q) only (used to build the initial equilibrium distributions)
template <typename real>
cudaError_t launch_field(const StepArgs& a, cudaStream_t s) {
  const auto* reps = static_cast<const Replica<real>*>(a.reps);
  const int threads = a.ts.tx * a.ts.ty * a.ts.tz;
  launch_fld<real, true>(a.div, a.ntiles, threads, s, reps, a.tiles, a.ntiles, a.ts, static_cast<const real*>(a.q),
                         static_cast<real*>(a.h), static_cast<real*>(a.sigma), static_cast<real*>(a.tau));
  return cudaGetLastError();
}
template cudaError_t launch_field<float>(const StepArgs&, cudaStream_t);
template cudaError_t launch_field<double>(const StepArgs&, cudaStream_t);

// Beris-Edwards rate R(Q, u) = Gamma H + S(W, Q) - u.grad Q at every site of
// every replica (Sec. 2.1 Eq. Qevolution, mat_der) in one pass: the stencil of
// Q gives H and the gradients, the stencil of u gives W (u = 0 without flow).
// The same per-site functions as the Heun predictor, so R is what the step
// adds to Q there.
template <typename real, bool FLOW, bool DIV = false>
__global__ void __launch_bounds__(256) k_rate(const Replica<real>* __restrict__ reps, const Tile* __restrict__ tiles,
                                              int ntiles, TileShape ts, const real* __restrict__ Q,
                                              const real* __restrict__ rhou, real* __restrict__ Rout) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int x, y, z;
    if (!tile_site(reps, tiles, t, ts, R, x, y, z)) continue;
    const long long n = R.n;
    const Nbr nb = make_nbr(x, y, z, R.nx, R.ny, R.nz, R.walls);
    const Stencil7<real> st = load_stencil(Q + 5 * R.base, n, nb, R);
    Sym5<real> dq[3];
    Sym5<real> h = molecular_field(st, R.m, dq);
    if (DIV) add_div_field(h, Q + 5 * R.base, n, x, y, z, R.nx, R.ny, R.nz, R.m.c_div);
    real u[3] = {real(0), real(0), real(0)};
    real w[3][3] = {};
    if (FLOW) {
      const real* ru = rhou + 4 * R.base;
      load_u(ru, n, nb.s, u);
      velocity_gradient(ru, n, nb, R.nx, R.ny, w, u);
    }
    const Sym5<real> r = be_rate(st.c, h, dq, u, w, R.m, FLOW);
    store5(Rout + 5 * R.base, n, nb.s, r);
  }
}

// R(Q^n, u^n) into a.qs
template <typename real>
cudaError_t launch_rate(const StepArgs& a, cudaStream_t s) {
  const auto* reps = static_cast<const Replica<real>*>(a.reps);
  const int threads = a.ts.tx * a.ts.ty * a.ts.tz;
  const real* q = static_cast<const real*>(a.q);
  const real* ru = static_cast<const real*>(a.rhou);
  real* out = static_cast<real*>(a.qs);
  if (a.flow_on) {
    if (a.div) k_rate<real, true, true><<<a.ntiles, threads, 0, s>>>(reps, a.tiles, a.ntiles, a.ts, q, ru, out);
    else k_rate<real, true, false><<<a.ntiles, threads, 0, s>>>(reps, a.tiles, a.ntiles, a.ts, q, ru, out);
  } else {
    if (a.div) k_rate<real, false, true><<<a.ntiles, threads, 0, s>>>(reps, a.tiles, a.ntiles, a.ts, q, ru, out);
    else k_rate<real, false, false><<<a.ntiles, threads, 0, s>>>(reps, a.tiles, a.ntiles, a.ts, q, ru, out);
  }
  return cudaGetLastError();
}
template cudaError_t launch_rate<float>(const StepArgs&, cudaStream_t);
template cudaError_t launch_rate<double>(const StepArgs&, cudaStream_t);

}  // namespace lcbp
