// Initial states, moments, dtype conversion and FP64 diagnostics.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

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
__global__ void k_shift(const real* src, real* dst, long long n, int comps, int kind, real sign) {
  const long long total = n * comps;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(k / n);
    const real w = kind == 0 ? (real)rest_weight(c) : real(1);
    dst[k] = src[k] + sign * w;
  }
}

template <typename real>
cudaError_t launch_shift(const void* src, void* dst, long long n, int comps, int kind, int sign, cudaStream_t s) {
  const long long total = n * comps;
  if (total <= 0) return cudaSuccess;
  const long long want = (total + 255) / 256;
  const int grid = (int)(want < 65536 ? want : 65536);
  k_shift<real><<<grid, 256, 0, s>>>(static_cast<const real*>(src), static_cast<real*>(dst), n, comps, kind,
                                      (real)sign);
  return cudaGetLastError();
}
template cudaError_t launch_shift<float>(const void*, void*, long long, int, int, int, cudaStream_t);
template cudaError_t launch_shift<double>(const void*, void*, long long, int, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Diagnostics in FP64.  Largest eigenvalue of a symmetric 3x3 matrix by the
// trigonometric closed form (O. K. Smith, CACM 4(4):168, 1961).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lambda_max(const double a[3][3]) {
  const double p1 = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
  const double qm = (a[0][0] + a[1][1] + a[2][2]) / 3.0;
  const double d0 = a[0][0] - qm, d1 = a[1][1] - qm, d2 = a[2][2] - qm;
  const double p2 = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * p1;
  if (p2 <= 0.0) return qm;
  const double p = sqrt(p2 / 6.0);
  const double b00 = d0 / p, b11 = d1 / p, b22 = d2 / p;
  const double b01 = a[0][1] / p, b02 = a[0][2] / p, b12 = a[1][2] / p;
  const double det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
  double r = 0.5 * det;
  r = r < -1.0 ? -1.0 : (r > 1.0 ? 1.0 : r);
  const double phi = acos(r) / 3.0;
  return qm + 2.0 * p * cos(phi);
}

template <typename real>
__device__ __forceinline__ void q9(const real* __restrict__ qp, long long n, long long s, double m[3][3]) {
  const double xx = qp[s], xy = qp[n + s], xz = qp[2 * n + s], yy = qp[3 * n + s], yz = qp[4 * n + s];
  m[0][0] = xx; m[0][1] = xy; m[0][2] = xz;
  m[1][0] = xy; m[1][1] = yy; m[1][2] = yz;
  m[2][0] = xz; m[2][1] = yz; m[2][2] = -xx - yy;
}

// A_ab eps_agd B_db for one direction g
__device__ __forceinline__ double eps_contract(const double A[3][3], const double B[3][3], int g) {
  double v = 0;
  for (int b = 0; b < 3; ++b) {
    if (g == 0) v += A[2][b] * B[1][b] - A[1][b] * B[2][b];
    else if (g == 1) v += A[0][b] * B[2][b] - A[2][b] * B[0][b];
    else v += A[1][b] * B[0][b] - A[0][b] * B[1][b];
  }
  return v;
}

// energy of the bond from A (at r) to B (at r + e_g): (K/2)|B - A|^2 + K q0 (A:eps_g B - B:eps_g A)
__device__ __forceinline__ double bond_energy(const double A[3][3], const double B[3][3], int g, double K,
                                              double q0) {
  double d2 = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) d2 += (B[a][b] - A[a][b]) * (B[a][b] - A[a][b]);
  return 0.5 * K * d2 + K * q0 * (eps_contract(A, B, g) - eps_contract(B, A, g));
}

// sums per block: [F_h, mass, Px, Py, Pz, defects, nonfinite, 0]
template <typename real>
__global__ void __launch_bounds__(256) k_diag(DiagGeom g, const real* __restrict__ Q, const real* __restrict__ f,
                                              int with_f, double threshold, double* __restrict__ partials) {
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  const real* qp = Q + 5 * g.base;
  const real* fp = f ? f + 15 * g.base : nullptr;
  const long long n = g.n;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % g.nx);
    const int y = (int)((s / g.nx) % g.ny);
    const int z = (int)(s / ((long long)g.nx * g.ny));
    const int xp = x + 1 == g.nx ? 0 : x + 1, xm = x == 0 ? g.nx - 1 : x - 1;
    const int yp = y + 1 == g.ny ? 0 : y + 1, ym = y == 0 ? g.ny - 1 : y - 1;
    const int zp = z + 1 == g.nz ? 0 : z + 1, zm = z == 0 ? g.nz - 1 : z - 1;
    auto at = [&](int xx, int yy, int zz) { return ((long long)zz * g.ny + yy) * g.nx + xx; };
    double Qc[3][3], Qp[3][3][3], Qm[3][3][3];
    q9(qp, n, s, Qc);
    q9(qp, n, at(xp, y, z), Qp[0]);
    q9(qp, n, at(x, yp, z), Qp[1]);
    q9(qp, n, at(x, y, zp), Qp[2]);
    q9(qp, n, at(xm, y, z), Qm[0]);
    q9(qp, n, at(x, ym, z), Qm[1]);
    q9(qp, n, at(x, y, zm), Qm[2]);
    double tr2 = 0, tr3 = 0, grad2 = 0, chiral = 0;
    bool finite = true;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        finite = finite && isfinite(Qc[a][b]);
        tr2 += Qc[a][b] * Qc[a][b];
        for (int c = 0; c < 3; ++c) tr3 += Qc[a][b] * Qc[b][c] * Qc[c][a];
        for (int d = 0; d < 3; ++d) {
          const double fd = Qp[d][a][b] - Qc[a][b];
          grad2 += fd * fd;
        }
      }
    // C_ab = eps_agd D0_g Q_db
    for (int b = 0; b < 3; ++b) {
      const double Cx = 0.5 * (Qp[1][2][b] - Qm[1][2][b]) - 0.5 * (Qp[2][1][b] - Qm[2][1][b]);
      const double Cy = 0.5 * (Qp[2][0][b] - Qm[2][0][b]) - 0.5 * (Qp[0][2][b] - Qm[0][2][b]);
      const double Cz = 0.5 * (Qp[0][1][b] - Qm[0][1][b]) - 0.5 * (Qp[1][0][b] - Qm[1][0][b]);
      chiral += Qc[0][b] * Cx + Qc[1][b] * Cy + Qc[2][b] * Cz;
    }
    const double bulk = 0.5 * g.A0 * (1.0 - g.gamma / 3.0) * tr2 - g.A0 * g.gamma / 3.0 * tr3 +
                        0.25 * g.A0 * g.gamma * tr2 * tr2;
    if (!g.walls) {
      acc[0] += bulk + 0.5 * g.K * grad2 + 2.0 * g.K * g.q0 * chiral + 2.0 * g.K * g.q0 * g.q0 * tr2;
      if (g.c_div != 0.0) {
        // div_a = sum_b D0_b Q_ab from the face neighbours
        double d2 = 0;
        for (int a = 0; a < 3; ++a) {
          double dv = 0;
          for (int b = 0; b < 3; ++b) dv += 0.5 * (Qp[b][a][b] - Qm[b][a][b]);
          d2 += dv * dv;
        }
        acc[0] -= g.c_div * d2;
      }
    } else {
      // bond form: this site's three forward bonds (the z bond of the top plane
      // ends on the anchored ghost) and, on the bottom plane, the bond from the
      // ghost below; every bond touching the lattice is counted once
      double Qw[3][3];
      Qw[0][0] = g.qw[0]; Qw[0][1] = g.qw[1]; Qw[0][2] = g.qw[2];
      Qw[1][0] = g.qw[1]; Qw[1][1] = g.qw[3]; Qw[1][2] = g.qw[4];
      Qw[2][0] = g.qw[2]; Qw[2][1] = g.qw[4]; Qw[2][2] = -g.qw[0] - g.qw[3];
      double Fb = bond_energy(Qc, Qp[0], 0, g.K, g.q0) + bond_energy(Qc, Qp[1], 1, g.K, g.q0);
      Fb += bond_energy(Qc, z == g.nz - 1 ? Qw : Qp[2], 2, g.K, g.q0);
      if (z == 0) Fb += bond_energy(Qw, Qc, 2, g.K, g.q0);
      acc[0] += bulk + Fb + 2.0 * g.K * g.q0 * g.q0 * tr2;
    }
    acc[5] += finite && lambda_max(Qc) < threshold ? 1.0 : 0.0;
    if (with_f) {
      double r = 1.0, jx = 0, jy = 0, jz = 0;  // deviation storage: rho = 1 + sum df_i
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const double fi = fp[i * n + s];
        finite = finite && isfinite(fi);
        r += fi;
        jx += ex(i) * fi;
        jy += ey(i) * fi;
        jz += ez(i) * fi;
      }
      acc[1] += r;
      acc[2] += jx;
      acc[3] += jy;
      acc[4] += jz;
    }
    acc[6] += finite ? 0.0 : 1.0;
  }
  // block reduction in a fixed order
  __shared__ double red[8][256];
  for (int k = 0; k < 7; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int k = 0; k < 7; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < 7; ++k) partials[blockIdx.x * 8 + k] = red[k][0];
    partials[blockIdx.x * 8 + 7] = 0.0;
  }
}

__global__ void k_diag_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  if (threadIdx.x < 8) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * 8 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

constexpr int kDiagBlocks = 512;

template <typename real>
cudaError_t launch_diag_one(const DiagGeom& g, const void* q, const void* f, int with_f, double threshold,
                            double* partials, double* out, cudaStream_t s) {
  k_diag<real><<<kDiagBlocks, 256, 0, s>>>(g, static_cast<const real*>(q), static_cast<const real*>(f), with_f,
                                           threshold, partials);
  k_diag_final<<<1, 32, 0, s>>>(partials, kDiagBlocks, out);
  return cudaGetLastError();
}
template cudaError_t launch_diag_one<float>(const DiagGeom&, const void*, const void*, int, double, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_diag_one<double>(const DiagGeom&, const void*, const void*, int, double, double*, double*,
                                             cudaStream_t);

}  // namespace lcbp
