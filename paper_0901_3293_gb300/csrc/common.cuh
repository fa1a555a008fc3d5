// Internal definitions shared by the CUDA translation units of liblcbp.
//
// Layout in HBM: every field is structure-of-arrays.  A batch holds R >= 1
// replicas (a single lattice is R = 1); replica r owns sites
// [base_r, base_r + n_r) of the concatenated site range, and a field with C
// components stores replica r at  field + C * base_r  as  [c][z][y][x].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lcbp {

// ---------------------------------------------------------------------------
// Model parameters of one replica (Sec. 2.1 Eq. free_energy, Qevolution,
// mat_der; Sec. 2.2 Eq. eq4).  Derived coefficients are precomputed on the
// host in double and rounded once to the state type.
// ---------------------------------------------------------------------------
template <typename real>
struct Model {
  real a_bulk;   // A0 (1 - gamma/3)
  real b_bulk;   // A0 gamma
  real K;        // one-constant elastic constant
  real kq0x2;    // 2 K q0
  real kq0sq4;   // 4 K q0^2
  real Gamma;    // rotational diffusion constant
  real xi;       // flow-aligning parameter
  real inv_tau;  // 1 / tau_f
  real c_div;    // (K - L2) / 2: weight of -(div Q)^2 (0 = one-constant energy)
};

// geometry + parameters of one replica, read by every CTA of its tiles
template <typename real>
struct Replica {
  int nx, ny, nz;
  int walls;       // 1: solid walls half a spacing below z = 0 and above z = nz-1
  long long n;     // nx * ny * nz
  long long base;  // first site of this replica in the concatenated range
  Model<real> m;
  real qw[5];      // anchored Q on the ghost planes beyond the walls (q5 order)
};

// One unit of kernel work: a tile of TX x TY x TZ sites of replica `rep`
// whose first site is (x0, y0, z0).  Tiles may hang over the lattice edge.
struct Tile {
  int rep;
  int x0, y0, z0;
};

// tile shape chosen per lattice (autotuned); blockDim.x == tx * ty * tz
struct TileShape {
  int tx, ty, tz;
};

// ---------------------------------------------------------------------------
// D3Q15 velocity set (Sec. 2.2 Eq. latvects), boundary ordering: rest,
// +x -x +y -y +z -z, then (+-1,+-1,+-1) lexicographic with + before -.
// ---------------------------------------------------------------------------
constexpr int NV = 15;
__host__ __device__ constexpr int ex(int i) {
  return i == 1 ? 1 : i == 2 ? -1 : (i >= 7 ? (i < 11 ? 1 : -1) : 0);
}
__host__ __device__ constexpr int ey(int i) {
  return i == 3 ? 1 : i == 4 ? -1 : (i >= 7 ? (((i - 7) & 2) ? -1 : 1) : 0);
}
__host__ __device__ constexpr int ez(int i) {
  return i == 5 ? 1 : i == 6 ? -1 : (i >= 7 ? (((i - 7) & 1) ? -1 : 1) : 0);
}

// opposite direction: 1..6 pair up (+x,-x), (+y,-y), (+z,-z); the corners are
// ordered lexicographically with + first, so i and 21 - i are opposite
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : 21 - i); }

// ---------------------------------------------------------------------------
// Symmetric traceless tensors in 5 components [xx, xy, xz, yy, yz].
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Two-site vectors.  The fast kernels compute two lattice sites per thread in
// the two lanes of a Vec2; for FP32 the lanes are packed into one 64-bit
// register and added / multiplied with the paired FP32 instructions of the
// sm_100 family (add / sub / mul .f32x2), which halves the floating-point
// instruction count.  Vec2<double> is a plain pair.
// ---------------------------------------------------------------------------
template <typename T>
struct Vec2 {
  T x, y;
  __device__ __forceinline__ Vec2() : x(T(0)), y(T(0)) {}
  __device__ __forceinline__ Vec2(double v) : x(T(v)), y(T(v)) {}
  __device__ __forceinline__ Vec2(float v) : x(T(v)), y(T(v)) {}
  __device__ __forceinline__ Vec2(int v) : x(T(v)), y(T(v)) {}
  __device__ __forceinline__ Vec2(T a, T b, int) : x(a), y(b) {}
  __device__ __forceinline__ T lo() const { return x; }
  __device__ __forceinline__ T hi() const { return y; }
};
template <typename T>
__device__ __forceinline__ Vec2<T> operator+(Vec2<T> a, Vec2<T> b) { return Vec2<T>(a.x + b.x, a.y + b.y, 0); }
template <typename T>
__device__ __forceinline__ Vec2<T> operator-(Vec2<T> a, Vec2<T> b) { return Vec2<T>(a.x - b.x, a.y - b.y, 0); }
template <typename T>
__device__ __forceinline__ Vec2<T> operator*(Vec2<T> a, Vec2<T> b) { return Vec2<T>(a.x * b.x, a.y * b.y, 0); }
template <typename T>
__device__ __forceinline__ Vec2<T> operator-(Vec2<T> a) { return Vec2<T>(-a.x, -a.y, 0); }

template <>
struct Vec2<float> {
  unsigned long long b;  // lane 0 in the low word, lane 1 in the high word
  __device__ __forceinline__ Vec2() : b(0ull) {}
  __device__ __forceinline__ Vec2(float v) { asm("mov.b64 %0, {%1, %1};" : "=l"(b) : "f"(v)); }
  __device__ __forceinline__ Vec2(double v) : Vec2((float)v) {}
  __device__ __forceinline__ Vec2(int v) : Vec2((float)v) {}
  __device__ __forceinline__ Vec2(float a, float c, int) { asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(a), "f"(c)); }
  __device__ __forceinline__ float lo() const {
    float a;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(a) : "l"(b));
    return a;
  }
  __device__ __forceinline__ float hi() const {
    float c;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(c) : "l"(b));
    return c;
  }
};
using F2 = Vec2<float>;
// no rounding modifier: the code generator may fuse a multiply and an add
__device__ __forceinline__ F2 operator+(F2 a, F2 c) {
  F2 r;
  asm("add.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(c.b));
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 c) {
  F2 r;
  asm("sub.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(c.b));
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 c) {
  F2 r;
  asm("mul.f32x2 %0, %1, %2;" : "=l"(r.b) : "l"(a.b), "l"(c.b));
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a) { return F2(0.f) - a; }

template <typename T>
__device__ __forceinline__ Vec2<T>& operator+=(Vec2<T>& a, Vec2<T> c) { return a = a + c; }
template <typename T>
__device__ __forceinline__ Vec2<T>& operator-=(Vec2<T>& a, Vec2<T> c) { return a = a - c; }
template <typename T>
__device__ __forceinline__ Vec2<T>& operator*=(Vec2<T>& a, Vec2<T> c) { return a = a * c; }
// lane-wise reciprocal
template <typename T>
__device__ __forceinline__ Vec2<T> recip(Vec2<T> a) { return Vec2<T>(T(1) / a.lo(), T(1) / a.hi(), 0); }
__device__ __forceinline__ float recip(float a) { return 1.f / a; }
__device__ __forceinline__ double recip(double a) { return 1.0 / a; }

template <typename T>
struct ScalarOf { using type = T; };
template <typename T>
struct ScalarOf<Vec2<T>> { using type = T; };
// the rational constant a / b in the scalar type of `real`, folded at compile time
#define LCBP_Q(a, b) real(typename ScalarOf<real>::type(a) / typename ScalarOf<real>::type(b))

template <typename real>
struct Sym5 {
  real xx, xy, xz, yy, yz;
  __device__ __forceinline__ real zz() const { return -xx - yy; }
};

template <typename real>
struct Mat3 {
  real a[3][3];
};

template <typename real>
__device__ __forceinline__ Mat3<real> full(const Sym5<real>& s) {
  Mat3<real> m;
  m.a[0][0] = s.xx; m.a[0][1] = s.xy; m.a[0][2] = s.xz;
  m.a[1][0] = s.xy; m.a[1][1] = s.yy; m.a[1][2] = s.yz;
  m.a[2][0] = s.xz; m.a[2][1] = s.yz; m.a[2][2] = -s.xx - s.yy;
  return m;
}

// A_ab B_ab of two symmetric traceless tensors
template <typename real>
__device__ __forceinline__ real ddot(const Sym5<real>& a, const Sym5<real>& b) {
  return a.xx * b.xx + a.yy * b.yy + a.zz() * b.zz() +
         real(2) * (a.xy * b.xy + a.xz * b.xz + a.yz * b.yz);
}

template <typename real>
__device__ __forceinline__ Sym5<real> load5(const real* __restrict__ p, long long n, long long s) {
  Sym5<real> q;
  q.xx = __ldg(p + s);
  q.xy = __ldg(p + n + s);
  q.xz = __ldg(p + 2 * n + s);
  q.yy = __ldg(p + 3 * n + s);
  q.yz = __ldg(p + 4 * n + s);
  return q;
}

template <typename real>
__device__ __forceinline__ void store5(real* __restrict__ p, long long n, long long s, const Sym5<real>& q) {
  p[s] = q.xx;
  p[n + s] = q.xy;
  p[2 * n + s] = q.xz;
  p[3 * n + s] = q.yy;
  p[4 * n + s] = q.yz;
}

// Periodic neighbourhood of one site: linear indices of the 6 face
// neighbours and the wrapped coordinates.
struct Nbr {
  int x, y, z, xm, xp, ym, yp, zm, zp;
  bool wlo, whi;  // the z-1 / z+1 neighbour is a ghost plane beyond a wall
  long long s;
  __device__ __forceinline__ long long at(int xx, int yy, int zz, int nx, int ny) const {
    return ((long long)zz * ny + yy) * nx + xx;
  }
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, int nx, int ny, int nz, int walls = 0) {
  Nbr b;
  b.x = x; b.y = y; b.z = z;
  b.wlo = walls && z == 0;
  b.whi = walls && z == nz - 1;
  b.xm = x == 0 ? nx - 1 : x - 1;
  b.xp = x == nx - 1 ? 0 : x + 1;
  b.ym = y == 0 ? ny - 1 : y - 1;
  b.yp = y == ny - 1 ? 0 : y + 1;
  b.zm = z == 0 ? nz - 1 : z - 1;
  b.zp = z == nz - 1 ? 0 : z + 1;
  b.s = ((long long)z * ny + y) * nx + x;
  return b;
}

// Q and its 6 face neighbours, as needed by every stencil of the step.
template <typename real>
struct Stencil7 {
  Sym5<real> c, xm, xp, ym, yp, zm, zp;
};

template <typename real>
__device__ __forceinline__ Stencil7<real> load_stencil(const real* __restrict__ q, long long n,
                                                       const Nbr& b, int nx, int ny) {
  Stencil7<real> st;
  st.c = load5(q, n, b.s);
  st.xm = load5(q, n, b.at(b.xm, b.y, b.z, nx, ny));
  st.xp = load5(q, n, b.at(b.xp, b.y, b.z, nx, ny));
  st.ym = load5(q, n, b.at(b.x, b.ym, b.z, nx, ny));
  st.yp = load5(q, n, b.at(b.x, b.yp, b.z, nx, ny));
  st.zm = load5(q, n, b.at(b.x, b.y, b.zm, nx, ny));
  st.zp = load5(q, n, b.at(b.x, b.y, b.zp, nx, ny));
  return st;
}

// the same with the anchored ghost planes of walled replicas (strong anchoring:
// Q = qw on the planes z = -1 and z = nz)
template <typename real>
__device__ __forceinline__ Stencil7<real> load_stencil(const real* __restrict__ q, long long n, const Nbr& b,
                                                       const Replica<real>& R) {
  Stencil7<real> st = load_stencil(q, n, b, R.nx, R.ny);
  if (b.wlo || b.whi) {
    const Sym5<real> w = {R.qw[0], R.qw[1], R.qw[2], R.qw[3], R.qw[4]};
    if (b.wlo) st.zm = w;
    if (b.whi) st.zp = w;
  }
  return st;
}

template <typename real>
__device__ __forceinline__ Sym5<real> half_diff(const Sym5<real>& p, const Sym5<real>& m) {
  const real h = real(0.5);
  return {h * (p.xx - m.xx), h * (p.xy - m.xy), h * (p.xz - m.xz), h * (p.yy - m.yy), h * (p.yz - m.yz)};
}

// p - m: twice the central difference
template <typename real>
__device__ __forceinline__ Sym5<real> diff5(const Sym5<real>& p, const Sym5<real>& m) {
  return {p.xx - m.xx, p.xy - m.xy, p.xz - m.xz, p.yy - m.yy, p.yz - m.yz};
}

// ---------------------------------------------------------------------------
// Molecular field, Sec. 2.1 Eq. (Qevolution) with the one-constant energy:
// H = -A0(1-g/3) Q + A0 g (QQ - Tr(Q^2)/3 I) - A0 g Tr(Q^2) Q
//     + K Lap7 Q - 2 K q0 (C + C^T) - 4 K q0^2 Q,   C_ab = eps_agd D0_g Q_db.
// Also returns the three central derivatives D0_g Q for reuse (RAW: twice
// them, the plain differences Q(+) - Q(-), which saves the halving; the
// chiral coefficient takes the factor instead).
// ---------------------------------------------------------------------------
template <bool RAW = false, typename real>
__device__ __forceinline__ Sym5<real> molecular_field(const Stencil7<real>& st, const Model<real>& m,
                                                      Sym5<real> dq[3]) {
  const Sym5<real>& q = st.c;
  if constexpr (RAW) {
    dq[0] = diff5(st.xp, st.xm);
    dq[1] = diff5(st.yp, st.ym);
    dq[2] = diff5(st.zp, st.zm);
  } else {
    dq[0] = half_diff(st.xp, st.xm);
    dq[1] = half_diff(st.yp, st.ym);
    dq[2] = half_diff(st.zp, st.zm);
  }
  const real qzz = q.zz();
  // Q.Q (symmetric)
  const real qq_xx = q.xx * q.xx + q.xy * q.xy + q.xz * q.xz;
  const real qq_xy = q.xx * q.xy + q.xy * q.yy + q.xz * q.yz;
  const real qq_xz = q.xx * q.xz + q.xy * q.yz + q.xz * qzz;
  const real qq_yy = q.xy * q.xy + q.yy * q.yy + q.yz * q.yz;
  const real qq_yz = q.xy * q.xz + q.yy * q.yz + q.yz * qzz;
  const real qq_zz = q.xz * q.xz + q.yz * q.yz + qzz * qzz;
  const real trq2 = qq_xx + qq_yy + qq_zz;
  const real third = LCBP_Q(1, 3);
  // 7-point Laplacian
  auto lap = [&](real c, real a, real b, real cc, real d, real e, real f) {
    return (a + b) + (cc + d) + (e + f) - real(6) * c;
  };
  const real l_xx = lap(q.xx, st.xm.xx, st.xp.xx, st.ym.xx, st.yp.xx, st.zm.xx, st.zp.xx);
  const real l_xy = lap(q.xy, st.xm.xy, st.xp.xy, st.ym.xy, st.yp.xy, st.zm.xy, st.zp.xy);
  const real l_xz = lap(q.xz, st.xm.xz, st.xp.xz, st.ym.xz, st.yp.xz, st.zm.xz, st.zp.xz);
  const real l_yy = lap(q.yy, st.xm.yy, st.xp.yy, st.ym.yy, st.yp.yy, st.zm.yy, st.zp.yy);
  const real l_yz = lap(q.yz, st.xm.yz, st.xp.yz, st.ym.yz, st.yp.yz, st.zm.yz, st.zp.yz);
  // C_ab = eps_agd D0_g Q_db :  C_xb = D0y Q_zb - D0z Q_yb,  C_yb = D0z Q_xb - D0x Q_zb,
  //                             C_zb = D0x Q_yb - D0y Q_xb
  const Sym5<real>& dx = dq[0];
  const Sym5<real>& dy = dq[1];
  const Sym5<real>& dz = dq[2];
  const real c_xx = dy.xz - dz.xy;
  const real c_xy = dy.yz - dz.yy;
  const real c_xz = dy.zz() - dz.yz;
  const real c_yx = dz.xx - dx.xz;
  const real c_yy = dz.xy - dx.yz;
  const real c_yz = dz.xz - dx.zz();
  const real c_zx = dx.xy - dy.xx;
  const real c_zy = dx.yy - dy.xy;
  const real c_zz = dx.yz - dy.xz;
  (void)c_zz;
  const real bulk_iso = m.a_bulk + m.b_bulk * trq2 + m.kq0sq4;  // coefficient of -Q
  const real kc = RAW ? real(0.5) * m.kq0x2 : m.kq0x2;           // of C + C^T
  Sym5<real> H;
  H.xx = -bulk_iso * q.xx + m.b_bulk * (qq_xx - third * trq2) + m.K * l_xx - kc * (c_xx + c_xx);
  H.xy = -bulk_iso * q.xy + m.b_bulk * qq_xy + m.K * l_xy - kc * (c_xy + c_yx);
  H.xz = -bulk_iso * q.xz + m.b_bulk * qq_xz + m.K * l_xz - kc * (c_xz + c_zx);
  H.yy = -bulk_iso * q.yy + m.b_bulk * (qq_yy - third * trq2) + m.K * l_yy - kc * (c_yy + c_yy);
  H.yz = -bulk_iso * q.yz + m.b_bulk * qq_yz + m.K * l_yz - kc * (c_yz + c_zy);
  return H;
}

// ---------------------------------------------------------------------------
// Stress, Sec. 2.1 Eq. (BEstress):
// sigma_LC = 2 xi (Q + I/3) Tr(QH) - xi (H (Q+I/3) + (Q+I/3) H)   (symmetric, traceless)
// tau = Q H - H Q  (antisymmetric; returned as [xy, xz, yz])
// ---------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ void lc_stress(const Sym5<real>& q, const Sym5<real>& h, real xi,
                                          Sym5<real>& sigma, real tau[3]) {
  const Mat3<real> Q = full(q);
  const Mat3<real> H = full(h);
  real QH[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) QH[a][b] = Q.a[a][0] * H.a[0][b] + Q.a[a][1] * H.a[1][b] + Q.a[a][2] * H.a[2][b];
  // (HQ)_ab = (QH)_ba since both are symmetric
  const real trqh = QH[0][0] + QH[1][1] + QH[2][2];
  const real two_xi_tr = real(2) * xi * trqh;
  const real two_third_xi = LCBP_Q(2, 3) * xi;
  // With P = Q + I/3:  H P + P H = H Q + Q H + 2H/3, and 2 xi P Tr(QH) carries
  // the isotropic part (2 xi / 3) Tr(QH) I on the diagonal.  The total is
  // traceless, so sigma_zz = -sigma_xx - sigma_yy holds and 5 components suffice.
  const real iso = LCBP_Q(1, 3) * two_xi_tr;
  sigma.xx = two_xi_tr * q.xx + iso - xi * (QH[0][0] + QH[0][0]) - two_third_xi * h.xx;
  sigma.xy = two_xi_tr * q.xy - xi * (QH[0][1] + QH[1][0]) - two_third_xi * h.xy;
  sigma.xz = two_xi_tr * q.xz - xi * (QH[0][2] + QH[2][0]) - two_third_xi * h.xz;
  sigma.yy = two_xi_tr * q.yy + iso - xi * (QH[1][1] + QH[1][1]) - two_third_xi * h.yy;
  sigma.yz = two_xi_tr * q.yz - xi * (QH[1][2] + QH[2][1]) - two_third_xi * h.yz;
  tau[0] = QH[0][1] - QH[1][0];
  tau[1] = QH[0][2] - QH[2][0];
  tau[2] = QH[1][2] - QH[2][1];
}

// tau = Q H - H Q alone, as [xy, xz, yz]: (QH)_ab - (QH)_ba from the six
// off-diagonal entries of Q H
template <typename real>
__device__ __forceinline__ void lc_tau(const Sym5<real>& q, const Sym5<real>& h, real tau[3]) {
  const Mat3<real> Q = full(q);
  const Mat3<real> H = full(h);
  auto QH = [&](int a, int b) { return Q.a[a][0] * H.a[0][b] + Q.a[a][1] * H.a[1][b] + Q.a[a][2] * H.a[2][b]; };
  tau[0] = QH(0, 1) - QH(1, 0);
  tau[1] = QH(0, 2) - QH(2, 0);
  tau[2] = QH(1, 2) - QH(2, 1);
}

// ---------------------------------------------------------------------------
// dQ/dt of Eq. (Qevolution) + (mat_der):  Gamma H + S_traceless(W, Q) - u . D0 Q
// with W_ab = D0_b u_a given as w[a][b] (RAW: dq and w are twice the central
// derivatives, the plain differences; the factor 1/2 goes into the constants).
// ---------------------------------------------------------------------------
template <bool RAW = false, typename real>
__device__ __forceinline__ Sym5<real> be_rate(const Sym5<real>& q, const Sym5<real>& h, const Sym5<real> dq[3],
                                              const real u[3], const real w[3][3], const Model<real>& m,
                                              bool flow) {
  Sym5<real> r;
  r.xx = m.Gamma * h.xx;
  r.xy = m.Gamma * h.xy;
  r.xz = m.Gamma * h.xz;
  r.yy = m.Gamma * h.yy;
  r.yz = m.Gamma * h.yz;
  if (!flow) return r;
  const real xi = m.xi;
  const Mat3<real> Q = full(q);
  // S = xi (D P + P D) + (O P - P O) - 2 xi P Tr(QW), with D and O the
  // symmetric and antisymmetric parts of W and P = Q + I/3.  With
  // A = xi D + O, i.e. A_ab = ((xi + 1) W_ab + (xi - 1) W_ba) / 2, the first two
  // terms are A P + (A P)^T, and A P = A Q + A / 3, so only A Q is a product.
  // Tr S = (2 xi / 3) Tr D exactly (Tr P = 1, Tr(A Q) = Q:D = Tr(QW)), which the
  // traceless projection removes from the diagonal.
  const real hw = RAW ? real(0.5) : real(1);  // w holds hw^-1 W
  const real xw = hw * xi, cpl = real(0.5) * hw * (xi + real(1)), cmi = real(0.5) * hw * (xi - real(1));
  real A[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) A[a][b] = a == b ? xw * w[a][a] : cpl * w[a][b] + cmi * w[b][a];
  const real trQW = Q.a[0][0] * w[0][0] + Q.a[1][1] * w[1][1] + Q.a[2][2] * w[2][2] +
                    Q.a[0][1] * (w[0][1] + w[1][0]) + Q.a[0][2] * (w[0][2] + w[2][0]) +
                    Q.a[1][2] * (w[1][2] + w[2][1]);  // (times hw^-1)
  auto AQ = [&](int a, int b) { return A[a][0] * Q.a[0][b] + A[a][1] * Q.a[1][b] + A[a][2] * Q.a[2][b]; };
  const real two_xi_tr = real(2) * xw * trQW;
  const real xi3 = LCBP_Q(1, 3) * xw;
  // diagonal: 2 (AQ)_aa + (2 xi / 3) W_aa - 2 xi (Q_aa + 1/3) Tr(QW) - (2 xi / 9) Tr W
  const real diag0 = LCBP_Q(2, 9) * xw * (w[0][0] + w[1][1] + w[2][2]) + LCBP_Q(1, 3) * two_xi_tr;
  real S[3][3];
  S[0][0] = real(2) * (AQ(0, 0) + xi3 * w[0][0]) - two_xi_tr * Q.a[0][0] - diag0;
  S[1][1] = real(2) * (AQ(1, 1) + xi3 * w[1][1]) - two_xi_tr * Q.a[1][1] - diag0;
  S[0][1] = (AQ(0, 1) + AQ(1, 0)) + xi3 * (w[0][1] + w[1][0]) - two_xi_tr * Q.a[0][1];
  S[0][2] = (AQ(0, 2) + AQ(2, 0)) + xi3 * (w[0][2] + w[2][0]) - two_xi_tr * Q.a[0][2];
  S[1][2] = (AQ(1, 2) + AQ(2, 1)) + xi3 * (w[1][2] + w[2][1]) - two_xi_tr * Q.a[1][2];
  const real ux = u[0], uy = u[1], uz = u[2];
  auto adv = [&](real gx, real gy, real gz) { return ux * gx + uy * gy + uz * gz; };  // (times hw^-1)
  r.xx += S[0][0] - hw * adv(dq[0].xx, dq[1].xx, dq[2].xx);
  r.xy += S[0][1] - hw * adv(dq[0].xy, dq[1].xy, dq[2].xy);
  r.xz += S[0][2] - hw * adv(dq[0].xz, dq[1].xz, dq[2].xz);
  r.yy += S[1][1] - hw * adv(dq[0].yy, dq[1].yy, dq[2].yy);
  r.yz += S[1][2] - hw * adv(dq[0].yz, dq[1].yz, dq[2].yz);
  return r;
}

// ---------------------------------------------------------------------------
// LB equilibrium and forcing for one direction, Sec. 2.2 Eq. (feq), (coeff),
// T = 1/3:  f_i^eq = A_s + B_s u.e + C_s u^2 + D_s (u.e)^2 + e.E_s.e ,  p_i = P_s b.e
//
// Storage precision: populations are kept as deviations from the rest-state
// weights, df_i = f_i - w_i with w = (8/15, 1/30 x 14) = f^eq(rho=1, u=0,
// sigma=0), and the density as drho = rho - 1.  The deviations are O(1e-3),
// so FP32 state keeps ~3 more decimal digits than storing f itself, and mass
// is conserved to that finer rounding.  feq_delta returns f_i^eq - w_i.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr double rest_weight(int i) { return i == 0 ? 8.0 / 15.0 : 1.0 / 30.0; }

// s_a x + s_b y + s_c z for signs s in {-1, 0, 1}.  With the signs known at
// compile time (unrolled direction loops) only the additions and subtractions
// of the nonzero terms remain, for the scalar and the packed types alike.
template <typename real>
__device__ __forceinline__ real signed_sum(int sa, real x, int sb, real y, int sc, real z) {
  real pos = real(0), neg = real(0);
  int np = 0, nn = 0;
  auto put = [&](int sgn, real v) {
    if (sgn > 0) {
      pos = np ? pos + v : v;
      ++np;
    } else if (sgn < 0) {
      neg = nn ? neg + v : v;
      ++nn;
    }
  };
  put(sa, x);
  put(sb, y);
  put(sc, z);
  if (np && nn) return pos - neg;
  if (np) return pos;
  if (nn) return -neg;
  return real(0);
}

template <typename real>
__device__ __forceinline__ real feq_delta(int i, real drho, real rho, real ux, real uy, real uz, real usq,
                                          const Sym5<real>& s) {
  // A_0 = rho - 14 rho/30 = w_0 rho; A_1 = A_2 = w_s rho  ->  A_s - w_s = w_s drho
  if (i == 0) return drho * LCBP_Q(8, 15) - rho * (LCBP_Q(2, 3) * usq);
  const real eu = signed_sum(ex(i), ux, ey(i), uy, ez(i), uz);
  if (i <= 6) {
    // faces: A1 = rho/30, B1 = rho/3, C1 = -rho/12, D1 = rho/2, E1 = -sigma/2
    const real base = drho * LCBP_Q(1, 30) + rho * (eu * LCBP_Q(1, 3) - usq * LCBP_Q(1, 12) + eu * eu * real(0.5));
    if (i <= 2) return base - real(0.5) * s.xx;
    if (i <= 4) return base - real(0.5) * s.yy;
    return base + real(0.5) * (s.xx + s.yy);  // sigma_zz = -sigma_xx - sigma_yy
  }
  // corners: A2 = rho/30, B2 = rho/24, C2 = -rho/24, D2 = rho/16, E2 = -sigma/16 with
  // e.sigma.e = 2 (ex ey sxy + ex ez sxz + ey ez syz) for a traceless sigma
  const real off = signed_sum(ex(i) * ey(i), s.xy, ex(i) * ez(i), s.xz, ey(i) * ez(i), s.yz);
  return drho * LCBP_Q(1, 30) + rho * (eu * LCBP_Q(1, 24) - usq * LCBP_Q(1, 24) + eu * eu * LCBP_Q(1, 16)) -
         LCBP_Q(1, 8) * off;
}

template <typename real>
__device__ __forceinline__ real force_dir(int i, real bx, real by, real bz) {
  if (i == 0) return real(0);
  const real eb = signed_sum(ex(i), bx, ey(i), by, ez(i), bz);
  return (i <= 6 ? LCBP_Q(1, 3) : LCBP_Q(1, 24)) * eb;
}

// ---------------------------------------------------------------------------
// The (div Q)^2 part of the energy for L2 != K: F gains -c sum_x |div Q|^2 with
// div_a = sum_b D0_b Q_ab, so dF/dQ gains c (D0_b div_a + D0_a div_b) and H the
// negative of that, made traceless.  div is taken at the 6 face neighbours
// from their own face neighbours (Q at distance 2 on the axes and on the 12
// in-plane diagonals).  Periodic lattice.
// ---------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ void add_div_field(Sym5<real>& h, const real* __restrict__ q, long long n, int x, int y,
                                              int z, int nx, int ny, int nz, real c) {
  auto wr = [](int v, int m) { return v < 0 ? v + m : (v >= m ? v - m : v); };
  auto at = [&](int xx, int yy, int zz) {
    return ((long long)wr(zz, nz) * ny + wr(yy, ny)) * nx + wr(xx, nx);
  };
  // column b of Q at site s: (Q_xb, Q_yb, Q_zb)
  auto col = [&](long long s, int b, real out[3]) {
    const Sym5<real> v = load5(q, n, s);
    if (b == 0) { out[0] = v.xx; out[1] = v.xy; out[2] = v.xz; }
    else if (b == 1) { out[0] = v.xy; out[1] = v.yy; out[2] = v.yz; }
    else { out[0] = v.xz; out[1] = v.yz; out[2] = -v.xx - v.yy; }
  };
  real dv[3][2][3];  // div_a at x + s e_g: [g][s = +, -][a]
  for (int g = 0; g < 3; ++g)
    for (int sg = 0; sg < 2; ++sg) {
      const int o = sg == 0 ? 1 : -1;
      const int yx = x + (g == 0 ? o : 0), yy = y + (g == 1 ? o : 0), yz = z + (g == 2 ? o : 0);
      real d[3] = {real(0), real(0), real(0)};
      for (int b = 0; b < 3; ++b) {
        real cp[3], cm[3];
        col(at(yx + (b == 0), yy + (b == 1), yz + (b == 2)), b, cp);
        col(at(yx - (b == 0), yy - (b == 1), yz - (b == 2)), b, cm);
        for (int a = 0; a < 3; ++a) d[a] += real(0.5) * (cp[a] - cm[a]);
      }
      for (int a = 0; a < 3; ++a) dv[g][sg][a] = d[a];
    }
  // M_ab = D0_b div_a;  G = c (M + M^T)
  real M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) M[a][b] = real(0.5) * (dv[b][0][a] - dv[b][1][a]);
  const real Gxx = c * (M[0][0] + M[0][0]), Gyy = c * (M[1][1] + M[1][1]), Gzz = c * (M[2][2] + M[2][2]);
  const real tr3 = (Gxx + Gyy + Gzz) * LCBP_Q(1, 3);
  h.xx += tr3 - Gxx;
  h.yy += tr3 - Gyy;
  h.xy -= c * (M[0][1] + M[1][0]);
  h.xz -= c * (M[0][2] + M[2][0]);
  h.yz -= c * (M[1][2] + M[2][1]);
}

}  // namespace lcbp
