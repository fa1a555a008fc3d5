// Initial states, moments, dtype conversion and FP64 diagnostics.
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace lcbp {

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): k-th output of the generator
// seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t k) {
  return (double)(splitmix64(seed, k) >> 11) * 0x1.0p-53;
}

template <typename real>
__device__ __forceinline__ bool tile_coords(const Replica<real>* reps, const Tile* tiles, int t, TileShape ts,
                                            Replica<real>& R, int& rep, int& x, int& y, int& z) {
  const Tile tl = tiles[t];
  rep = tl.rep;
  R = reps[rep];
  const int tid = threadIdx.x;
  x = tl.x0 + tid % ts.tx;
  y = tl.y0 + (tid / ts.tx) % ts.ty;
  z = tl.z0 + tid / (ts.tx * ts.ty);
  return x < R.nx && y < R.ny && z < R.nz;
}

// uniaxial Q = S (n n - I/3) in 5 components
__device__ __forceinline__ void uniaxial(double S, double nx, double ny, double nz, double q[5]) {
  q[0] = S * (nx * nx - 1.0 / 3.0);
  q[1] = S * nx * ny;
  q[2] = S * nx * nz;
  q[3] = S * (ny * ny - 1.0 / 3.0);
  q[4] = S * ny * nz;
}

__device__ __forceinline__ void bpii(double A, double k, int x, int y, int z, double q[5]) {
  const double cx = cos(k * x), cy = cos(k * y), cz = cos(k * z);
  q[0] = A * (cz - cy);
  q[1] = A * sin(k * z);
  q[2] = A * sin(k * y);
  q[3] = A * (cx - cz);
  q[4] = A * sin(k * x);
}

template <typename real>
__global__ void k_init_q(const Replica<real>* __restrict__ reps, const Tile* __restrict__ tiles, int ntiles,
                         TileShape ts, const double* __restrict__ q0s, const double* __restrict__ s_helix,
                         const uint64_t* __restrict__ seeds, InitQArgs a, real* __restrict__ Q) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int rep, x, y, z;
    if (!tile_coords(reps, tiles, t, ts, R, rep, x, y, z)) continue;
    const double q0 = q0s[rep];
    double q[5] = {0, 0, 0, 0, 0};
    switch (a.kind) {
      case 0: bpii(a.amplitude, 2.0 * q0, x, y, z, q); break;
      case 1: uniaxial(a.amplitude, 0.0, cos(q0 * x), sin(q0 * x), q); break;
      case 2: uniaxial(a.amplitude, sin(q0 * y), 0.0, cos(q0 * y), q); break;
      case 3: uniaxial(a.amplitude, cos(q0 * z), sin(q0 * z), 0.0, q); break;
      case 4: break;
      case 5:
        if (z < a.z0) bpii(a.amplitude, 2.0 * q0, x, y, z, q);
        else uniaxial(s_helix[rep], 0.0, cos(q0 * x), sin(q0 * x), q);
        break;
      case 6:
        if (z < a.z0) bpii(a.amplitude, 2.0 * q0, x, y, z, q);
        break;
      case 7:
        if (z < a.z0) bpii(a.amplitude, 2.0 * q0, x, y, z, q);
        else uniaxial(s_helix[rep], cos(q0 * z), sin(q0 * z), 0.0, q);
        break;
      default: break;
    }
    const long long s = ((long long)z * R.ny + y) * R.nx + x;
    if (a.noise != 0.0) {
      const uint64_t seed = seeds[rep];
#pragma unroll
      for (int c = 0; c < 5; ++c)
        q[c] += a.noise * (2.0 * uniform01(seed, 5ull * (uint64_t)s + (uint64_t)c) - 1.0);
    }
    real* qp = Q + 5 * R.base;
#pragma unroll
    for (int c = 0; c < 5; ++c) qp[c * R.n + s] = (real)q[c];
  }
}

template <typename real>
cudaError_t launch_init_q(const void* reps, const Tile* tiles, int ntiles, TileShape ts, const double* q0s,
                          const double* s_helix, const uint64_t* seeds, InitQArgs a, void* q, cudaStream_t s) {
  k_init_q<real><<<ntiles, ts.tx * ts.ty * ts.tz, 0, s>>>(static_cast<const Replica<real>*>(reps), tiles, ntiles, ts,
                                                           q0s, s_helix, seeds, a, static_cast<real*>(q));
  return cudaGetLastError();
}
template cudaError_t launch_init_q<float>(const void*, const Tile*, int, TileShape, const double*, const double*,
                                          const uint64_t*, InitQArgs, void*, cudaStream_t);
template cudaError_t launch_init_q<double>(const void*, const Tile*, int, TileShape, const double*, const double*,
                                           const uint64_t*, InitQArgs, void*, cudaStream_t);

// ---------------------------------------------------------------------------
template <typename real>
__global__ void k_init_feq(const Replica<real>* __restrict__ reps, const Tile* __restrict__ tiles, int ntiles,
                           TileShape ts, real rho0, const real* __restrict__ u3, const real* __restrict__ sigma,
                           real* __restrict__ f) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int rep, x, y, z;
    if (!tile_coords(reps, tiles, t, ts, R, rep, x, y, z)) continue;
    const long long n = R.n;
    const long long s = ((long long)z * R.ny + y) * R.nx + x;
    real ux = 0, uy = 0, uz = 0;
    if (u3) {
      const real* up = u3 + 3 * R.base;
      ux = up[s];
      uy = up[n + s];
      uz = up[2 * n + s];
    }
    const Sym5<real> sg = load5(sigma + 5 * R.base, n, s);
    const real usq = ux * ux + uy * uy + uz * uz;
    real* fp = f + 15 * R.base;
    // stored as deviations from the rest weights
#pragma unroll
    for (int i = 0; i < NV; ++i) fp[i * n + s] = feq_delta(i, rho0 - real(1), rho0, ux, uy, uz, usq, sg);
  }
}

template <typename real>
cudaError_t launch_init_feq(const void* reps, const Tile* tiles, int ntiles, TileShape ts, double rho0,
                            const void* u3, const void* sigma, void* f, cudaStream_t s) {
  k_init_feq<real><<<ntiles, ts.tx * ts.ty * ts.tz, 0, s>>>(static_cast<const Replica<real>*>(reps), tiles, ntiles,
                                                             ts, (real)rho0, static_cast<const real*>(u3),
                                                             static_cast<const real*>(sigma), static_cast<real*>(f));
  return cudaGetLastError();
}
template cudaError_t launch_init_feq<float>(const void*, const Tile*, int, TileShape, double, const void*,
                                            const void*, void*, cudaStream_t);
template cudaError_t launch_init_feq<double>(const void*, const Tile*, int, TileShape, double, const void*,
                                             const void*, void*, cudaStream_t);

// f = f^eq(rho, u, sigma) from the stored moments (deviation storage)
template <typename real>
__global__ void k_feq_from_moments(const Replica<real>* __restrict__ reps, const Tile* __restrict__ tiles, int ntiles,
                                   TileShape ts, const real* __restrict__ rhou, const real* __restrict__ sigma,
                                   real* __restrict__ f) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int rep, x, y, z;
    if (!tile_coords(reps, tiles, t, ts, R, rep, x, y, z)) continue;
    const long long n = R.n;
    const long long s = ((long long)z * R.ny + y) * R.nx + x;
    const real* rp = rhou + 4 * R.base;
    const real drho = rp[s], ux = rp[n + s], uy = rp[2 * n + s], uz = rp[3 * n + s];
    const Sym5<real> sg = load5(sigma + 5 * R.base, n, s);
    const real usq = ux * ux + uy * uy + uz * uz;
    real* fp = f + 15 * R.base;
#pragma unroll
    for (int i = 0; i < NV; ++i) fp[i * n + s] = feq_delta(i, drho, real(1) + drho, ux, uy, uz, usq, sg);
  }
}

template <typename real>
cudaError_t launch_feq_from_moments(const void* reps, const Tile* tiles, int ntiles, TileShape ts, const void* rhou,
                                    const void* sigma, void* f, cudaStream_t s) {
  k_feq_from_moments<real><<<ntiles, ts.tx * ts.ty * ts.tz, 0, s>>>(static_cast<const Replica<real>*>(reps), tiles,
                                                                     ntiles, ts, static_cast<const real*>(rhou),
                                                                     static_cast<const real*>(sigma),
                                                                     static_cast<real*>(f));
  return cudaGetLastError();
}
template cudaError_t launch_feq_from_moments<float>(const void*, const Tile*, int, TileShape, const void*, const void*,
                                                    void*, cudaStream_t);
template cudaError_t launch_feq_from_moments<double>(const void*, const Tile*, int, TileShape, const void*,
                                                     const void*, void*, cudaStream_t);

template <typename real>
__global__ void k_moments(const Replica<real>* __restrict__ reps, const Tile* __restrict__ tiles, int ntiles,
                          TileShape ts, const real* __restrict__ f, real* __restrict__ rhou) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    Replica<real> R;
    int rep, x, y, z;
    if (!tile_coords(reps, tiles, t, ts, R, rep, x, y, z)) continue;
    const long long n = R.n;
    const long long s = ((long long)z * R.ny + y) * R.nx + x;
    const real* fp = f + 15 * R.base;
    // deviation storage: drho = sum df_i, rho u = sum df_i e_i (sum w_i e_i = 0)
    real dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const real fi = fp[i * n + s];
      dr += fi;
      jx += real(ex(i)) * fi;
      jy += real(ey(i)) * fi;
      jz += real(ez(i)) * fi;
    }
    real* rp = rhou + 4 * R.base;
    const real r = real(1) + dr;
    rp[s] = dr;
    rp[n + s] = jx / r;
    rp[2 * n + s] = jy / r;
    rp[3 * n + s] = jz / r;
  }
}

template <typename real>
cudaError_t launch_moments(const void* reps, const Tile* tiles, int ntiles, TileShape ts, const void* f, void* rhou,
                           cudaStream_t s) {
  k_moments<real><<<ntiles, ts.tx * ts.ty * ts.tz, 0, s>>>(static_cast<const Replica<real>*>(reps), tiles, ntiles,
                                                            ts, static_cast<const real*>(f), static_cast<real*>(rhou));
  return cudaGetLastError();
}
template cudaError_t launch_moments<float>(const void*, const Tile*, int, TileShape, const void*, void*, cudaStream_t);
template cudaError_t launch_moments<double>(const void*, const Tile*, int, TileShape, const void*, void*,
                                            cudaStream_t);

// ---------------------------------------------------------------------------
template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

cudaError_t launch_convert(const void* src, int sd, void* dst, int dd, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const long long want = (n + threads - 1) / threads;
  const int grid = (int)(want < 65536 ? want : 65536);
  if (sd == 0 && dd == 1)
    k_convert<float, double><<<grid, threads, 0, s>>>(static_cast<const float*>(src), static_cast<double*>(dst), n);
  else if (sd == 1 && dd == 0)
    k_convert<double, float><<<grid, threads, 0, s>>>(static_cast<const double*>(src), static_cast<float*>(dst), n);
  else if (sd == 0 && dd == 0)
    k_convert<float, float><<<grid, threads, 0, s>>>(static_cast<const float*>(src), static_cast<float*>(dst), n);
  else
    k_convert<double, double><<<grid, threads, 0, s>>>(static_cast<const double*>(src), static_cast<double*>(dst), n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deviation storage <-> boundary layout.  For a field of `comps` components
// of n sites: dst[c n + s] = src[c n + s] + sign * shift(c), with shift(c) the
// rest weight w_c (populations) or 1 (density).  In place is allowed.
// ---------------------------------------------------------------------------
template <typename real>
__global__ void k_shift(const real* src, real* dst, long long n, int kind, real sign) {
  // component c = blockIdx.y: no thread divides a 64-bit index
  const int c = blockIdx.y;
  const real w = sign * (kind == 0 ? (real)rest_weight(c) : real(1));
  const real* s = src + (long long)c * n;
  real* d = dst + (long long)c * n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    d[k] = s[k] + w;
}

template <typename real>
cudaError_t launch_shift(const void* src, void* dst, long long n, int comps, int kind, int sign, cudaStream_t s) {
  if (n <= 0 || comps <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const int grid = (int)(want < 4096 ? want : 4096);
  k_shift<real><<<dim3(grid, comps), 256, 0, s>>>(static_cast<const real*>(src), static_cast<real*>(dst), n, kind,
                                                   (real)sign);
  return cudaGetLastError();
}
template cudaError_t launch_shift<float>(const void*, void*, long long, int, int, int, cudaStream_t);
template cudaError_t launch_shift<double>(const void*, void*, long long, int, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Diagnostics: F_h (Sec. 2.1, the lattice energy whose gradient is H), mass,
// momentum, the defect fraction #(lambda_max(Q) < threshold) / N (Sec. 2.1)
// and a count of non-finite sites, in one pass.  The per-site arithmetic runs
// in the state's precision (C = real); every sum over sites is FP64.
// ---------------------------------------------------------------------------
// lambda_max(a) < t  <=>  t I - a is positive definite  <=>  the leading
// principal minors of t I - a are all positive (Sylvester's criterion)
__device__ __forceinline__ bool top_eigenvalue_below(double xx, double xy, double xz, double yy, double yz,
                                                     double t) {
  const double zz = -xx - yy;
  const double b00 = t - xx, b11 = t - yy, b22 = t - zz;
  const double m2 = b00 * b11 - xy * xy;
  const double m3 = b00 * (b11 * b22 - yz * yz) - xy * (xy * b22 + yz * xz) - xz * (xy * yz + b11 * xz);
  return b00 > 0.0 && m2 > 0.0 && m3 > 0.0;
}

// The same decision for a site of the state's precision.  FP32: the minors in
// FP32 decide unless one lies within 1e-4 m^k of zero (m: the largest entry of
// t I - Q in size, k: the minor's order), far above their rounding error (a
// few ulp of m^k); such sites are decided in FP64 as above.
// tf: t rounded to FP32 (by the caller, once)
template <typename C>
__device__ __forceinline__ bool top_eigenvalue_below(const Sym5<C>& q, double t, float tf) {
  if constexpr (sizeof(C) == 8) {
    return top_eigenvalue_below(q.xx, q.xy, q.xz, q.yy, q.yz, t);
  } else {
    const float zz = -q.xx - q.yy;
    const float b00 = tf - q.xx, b11 = tf - q.yy, b22 = tf - zz;
    const float m = fmaxf(fmaxf(fmaxf(fabsf(b00), fabsf(b11)), fmaxf(fabsf(b22), fabsf(q.xy))),
                          fmaxf(fabsf(q.xz), fabsf(q.yz)));
    const float m2 = b00 * b11 - q.xy * q.xy;
    const float m3 =
        b00 * (b11 * b22 - q.yz * q.yz) - q.xy * (q.xy * b22 + q.yz * q.xz) - q.xz * (q.xy * q.yz + b11 * q.xz);
    const float e1 = 1e-4f * m, e2 = e1 * m, e3 = e2 * m;
    if (b00 < -e1 || m2 < -e2 || m3 < -e3) return false;
    if (b00 > e1 && m2 > e2 && m3 > e3) return true;
    return top_eigenvalue_below((double)q.xx, (double)q.xy, (double)q.xz, (double)q.yy, (double)q.yz, t);
  }
}

template <typename C>
__device__ __forceinline__ void full3(const Sym5<C>& q, C m[3][3]) {
  m[0][0] = q.xx; m[0][1] = q.xy; m[0][2] = q.xz;
  m[1][0] = q.xy; m[1][1] = q.yy; m[1][2] = q.yz;
  m[2][0] = q.xz; m[2][1] = q.yz; m[2][2] = -q.xx - q.yy;
}

// |b - a|^2 over all nine components of two traceless symmetric tensors
template <typename C>
__device__ __forceinline__ C dist2(const Sym5<C>& a, const Sym5<C>& b) {
  const C dxx = b.xx - a.xx, dyy = b.yy - a.yy, dzz = -dxx - dyy;
  const C dxy = b.xy - a.xy, dxz = b.xz - a.xz, dyz = b.yz - a.yz;
  return dxx * dxx + dyy * dyy + dzz * dzz + C(2) * (dxy * dxy + dxz * dxz + dyz * dyz);
}

// A_ab eps_agd B_db for one direction g
template <typename C>
__device__ __forceinline__ C eps_contract(const C A[3][3], const C B[3][3], int g) {
  C v = C(0);
  for (int b = 0; b < 3; ++b) {
    if (g == 0) v += A[2][b] * B[1][b] - A[1][b] * B[2][b];
    else if (g == 1) v += A[0][b] * B[2][b] - A[2][b] * B[0][b];
    else v += A[1][b] * B[0][b] - A[0][b] * B[1][b];
  }
  return v;
}

// energy of the bond from A (at r) to B (at r + e_g): (K/2)|B - A|^2 + K q0 (A:eps_g B - B:eps_g A)
template <typename C>
__device__ __forceinline__ C bond_energy(const Sym5<C>& a, const Sym5<C>& b, int g, C K, C q0) {
  C A[3][3], B[3][3];
  full3(a, A);
  full3(b, B);
  return C(0.5) * K * dist2(a, b) + K * q0 * (eps_contract(A, B, g) - eps_contract(B, A, g));
}

// Q:C with C_ab = eps_agd d_g Q_db for the raw differences d_g = Q(r + e_g) -
// Q(r - e_g) (twice the central derivatives), contracted in closed form on the
// five stored components:
//   C_xb = d_y Q_zb - d_z Q_yb,  C_yb = d_z Q_xb - d_x Q_zb,  C_zb = d_x Q_yb - d_y Q_xb
template <typename C>
__device__ __forceinline__ C chiral_contraction(const Sym5<C>& q, const Sym5<C>& dx, const Sym5<C>& dy,
                                                const Sym5<C>& dz) {
  const C qzz = q.zz();
  const C c_xx = dy.xz - dz.xy, c_xy = dy.yz - dz.yy, c_xz = dy.zz() - dz.yz;
  const C c_yx = dz.xx - dx.xz, c_yy = dz.xy - dx.yz, c_yz = dz.xz - dx.zz();
  const C c_zx = dx.xy - dy.xx, c_zy = dx.yy - dy.xy, c_zz = dx.yz - dy.xz;
  return q.xx * c_xx + q.xy * (c_xy + c_yx) + q.xz * (c_xz + c_zx) + q.yy * c_yy + q.yz * (c_yz + c_zy) +
         qzz * c_zz;
}

// sums per block: [F_h, mass, Px, Py, Pz, defects, nonfinite, 0].  WALLS: F_h
// in bond form with the anchored ghost planes (a build of its own, so that the
// periodic build keeps few registers and many warps per SM).
template <typename real, bool WALLS>
// (FP32: four CTAs per SM, 64 registers)
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 4 : 2)
    k_diag(DiagGeom g, const real* __restrict__ Q, const real* __restrict__ f, int with_f, double threshold,
           double* __restrict__ partials) {
  using C = real;
  // F_h, then sum(rho - 1), P: FP64; the sites, defects and non-finite sites counted
  double aF = 0.0, aR = 0.0, aJx = 0.0, aJy = 0.0, aJz = 0.0;
  int sites = 0, defects = 0, bad = 0;
  const real* qp = Q + 5 * g.base;
  const real* fp = f ? f + 15 * g.base : nullptr;
  const long long n = g.n;
  const C A0 = (C)g.A0, gam = (C)g.gamma, K = (C)g.K, q0 = (C)g.q0;
  const C a2 = C(0.5) * A0 * (C(1) - gam / C(3)), a3 = A0 * gam, a4 = C(0.25) * A0 * gam;
  // the chiral and divergence terms take raw differences: factors 1/2 and 1/4 folded in
  const C kq0h = K * q0, kq0sq = C(2) * K * q0 * q0, cdiv4 = C(0.25) * (C)g.c_div;
  // decided once: FP64 arithmetic is scarce, so the loop keeps only its FP64 sums
  const bool has_div = g.c_div != 0.0, small = g.n < (1ll << 31);
  const float tf = (float)threshold;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (small) {  // 32-bit index arithmetic
      const int si = (int)s, row = si / g.nx;
      x = si - row * g.nx;
      z = row / g.ny;
      y = row - z * g.ny;
    } else {
      const long long row = s / g.nx;
      x = (int)(s - row * g.nx);
      z = (int)(row / g.ny);
      y = (int)(row - (long long)z * g.ny);
    }
    const int xp = x + 1 == g.nx ? 0 : x + 1, xm = x == 0 ? g.nx - 1 : x - 1;
    const int yp = y + 1 == g.ny ? 0 : y + 1, ym = y == 0 ? g.ny - 1 : y - 1;
    const int zp = z + 1 == g.nz ? 0 : z + 1, zm = z == 0 ? g.nz - 1 : z - 1;
    auto at = [&](int xx, int yy, int zz) { return ((long long)zz * g.ny + yy) * g.nx + xx; };
    const Sym5<C> qc = load5(qp, n, s);
    const Sym5<C> qxp = load5(qp, n, at(xp, y, z)), qyp = load5(qp, n, at(x, yp, z)), qzp = load5(qp, n, at(x, y, zp));
    const bool finite = isfinite(qc.xx) && isfinite(qc.xy) && isfinite(qc.xz) && isfinite(qc.yy) && isfinite(qc.yz);
    const C qzz = -qc.xx - qc.yy;
    const C tr2 = qc.xx * qc.xx + qc.yy * qc.yy + qzz * qzz + C(2) * (qc.xy * qc.xy + qc.xz * qc.xz + qc.yz * qc.yz);
    // Tr Q^3 = 3 det Q for a traceless Q
    const C det = qc.xx * (qc.yy * qzz - qc.yz * qc.yz) - qc.xy * (qc.xy * qzz - qc.yz * qc.xz) +
                  qc.xz * (qc.xy * qc.yz - qc.yy * qc.xz);
    const C bulk = a2 * tr2 - a3 * det + a4 * tr2 * tr2;
    C Fs;
    if constexpr (!WALLS) {
      const C grad2 = dist2(qc, qxp) + dist2(qc, qyp) + dist2(qc, qzp);
      const Sym5<C> dx = diff5(qxp, load5(qp, n, at(xm, y, z)));
      const Sym5<C> dy = diff5(qyp, load5(qp, n, at(x, ym, z)));
      const Sym5<C> dz = diff5(qzp, load5(qp, n, at(x, y, zm)));
      // 2 K q0 Q:C with C from central derivatives = K q0 (Q:C of the raw differences)
      Fs = bulk + C(0.5) * K * grad2 + kq0h * chiral_contraction(qc, dx, dy, dz) + kq0sq * tr2;
      if (has_div) {
        // div_a = sum_b D0_b Q_ab; raw differences carry twice it
        const C vx = dx.xx + dy.xy + dz.xz, vy = dx.xy + dy.yy + dz.yz, vz = dx.xz + dy.yz + dz.zz();
        Fs -= cdiv4 * (vx * vx + vy * vy + vz * vz);
      }
    } else {
      // bond form: this site's three forward bonds (the z bond of the top plane
      // ends on the anchored ghost) and, on the bottom plane, the bond from the
      // ghost below; every bond touching the lattice is counted once
      const Sym5<C> qw = {(C)g.qw[0], (C)g.qw[1], (C)g.qw[2], (C)g.qw[3], (C)g.qw[4]};
      C Fb = bond_energy(qc, qxp, 0, K, q0) + bond_energy(qc, qyp, 1, K, q0);
      Fb += bond_energy(qc, z == g.nz - 1 ? qw : qzp, 2, K, q0);
      if (z == 0) Fb += bond_energy(qw, qc, 2, K, q0);
      Fs = bulk + Fb + kq0sq * tr2;
    }
    aF += (double)Fs;
    defects += finite && top_eigenvalue_below(qc, threshold, tf) ? 1 : 0;
    ++sites;
    bool ffin = true;
    if (with_f) {
      // deviation storage: rho = 1 + sum df_i; the per-site sums of the small
      // deviations in the state's precision, the sum over sites in FP64
      C r = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const C fi = fp[i * n + s];
        ffin = ffin && isfinite(fi);
        r += fi;
        if (ex(i) > 0) jx += fi; else if (ex(i) < 0) jx -= fi;
        if (ey(i) > 0) jy += fi; else if (ey(i) < 0) jy -= fi;
        if (ez(i) > 0) jz += fi; else if (ez(i) < 0) jz -= fi;
      }
      aR += (double)r;
      aJx += (double)jx;
      aJy += (double)jy;
      aJz += (double)jz;
    }
    bad += finite && ffin ? 0 : 1;
  }
  // mass = sites + sum(rho - 1).  Block reduction in a fixed order: a shuffle
  // tree within each warp, then warp 0 adds the eight warps' sums in order.
  double acc[7] = {aF, with_f ? aR + (double)sites : 0.0, aJx, aJy, aJz, (double)defects, (double)bad};
#pragma unroll
  for (int k = 0; k < 7; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
  __shared__ double red[8][8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 7; ++k) red[warp][k] = acc[k];
  __syncthreads();
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    double t = 0.0;
    if (k < 7)
      for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[w][k];
    partials[blockIdx.x * 8 + k] = t;
  }
}

// the block partials summed per quantity: warp k sums quantity k, lanes
// striding over the blocks, then a shuffle tree (a fixed order)
__global__ void k_diag_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x / 32, lane = threadIdx.x % 32;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partials[b * 8 + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[k] = s;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded barrier wait: a barrier that expects one arrival
// which never comes, so the wait runs into its limit and reports it.
// ---------------------------------------------------------------------------
__global__ void k_wait_probe(uint64_t limit_ns, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0) *flag = ok ? 0 : 1;
}

cudaError_t launch_wait_probe(uint64_t limit_ns, int* flag, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(limit_ns, flag);
  return cudaGetLastError();
}

constexpr int kDiagBlocks = 512;

template <typename real>
cudaError_t launch_diag_one(const DiagGeom& g, const void* q, const void* f, int with_f, double threshold,
                            double* partials, double* out, cudaStream_t s) {
  static_assert(kDiagBlocks * 8 == kDiagPartials, "the partials buffer holds 8 values per block");
  if (g.walls)
    k_diag<real, true><<<kDiagBlocks, 256, 0, s>>>(g, static_cast<const real*>(q), static_cast<const real*>(f),
                                                    with_f, threshold, partials);
  else
    k_diag<real, false><<<kDiagBlocks, 256, 0, s>>>(g, static_cast<const real*>(q), static_cast<const real*>(f),
                                                     with_f, threshold, partials);
  k_diag_final<<<1, 256, 0, s>>>(partials, kDiagBlocks, out);
  return cudaGetLastError();
}
template cudaError_t launch_diag_one<float>(const DiagGeom&, const void*, const void*, int, double, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_diag_one<double>(const DiagGeom&, const void*, const void*, int, double, double*, double*,
                                             cudaStream_t);

}  // namespace lcbp
