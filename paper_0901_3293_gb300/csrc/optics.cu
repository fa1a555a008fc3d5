// Polarised-light texture of the order-parameter field (Sec. 2.3): the
// transmitted intensity S_0 between crossed linear polarisers of light that
// crosses the lattice along +z, every plane a uniaxial retarder.
//
// Per site: director d = unit eigenvector of the largest eigenvalue q of Q;
// beta = atan2(d_x, d_y); delta = 2 pi q h / lambda (n_o n_e / sqrt(n_o^2
// sin^2 alpha + n_e^2 cos^2 alpha) - n_o) with cos alpha = d_z.  The Mueller
// matrix of a plane leaves S_0 unchanged and acts on (S_1, S_2, S_3) by the
// 3x3 block B(beta, delta), so a column is the ordered product
// T = B(Nz-1) ... B(0), taken per wavelength.
//
// Layout of the work: a CTA covers 32 consecutive x of one row y (lanes, so
// the Q loads coalesce) and splits its planes into kTexChunks chunks, one warp
// each; every thread multiplies the blocks of its chunk, and the chunk
// products are combined in order through shared memory.  Where the image has
// too few 32-column rows to fill the GPU, the planes of a column are first
// split into S ranges taken by different CTAs, and a second kernel multiplies
// the S range products in order.  cos 2 beta and sin 2 beta come
// from d_x, d_y directly: (d_y^2 - d_x^2, 2 d_x d_y) / (d_x^2 + d_y^2).
#include "../../include/lcbp.h"
#include "common.cuh"
#include "kernels.h"
#include "runtime.h"

namespace lcbp {

constexpr int kTexChunks = 8;
constexpr int kTexMaxLambda = 4;

struct OpticsArgs {
  int nx, ny, nz;
  long long n;
  int nl;
  float two_pi_h_over_lambda[kTexMaxLambda];
  float weight[kTexMaxLambda];
  float n_o, n_e;
  float c_in, s_in, c_out, s_out;  // cos / sin of twice the polariser and analyser angles
};

// largest eigenvalue and its unit eigenvector of a symmetric 3x3 matrix
// (eigenvalue: trigonometric closed form, Smith 1961; eigenvector: the largest
// cross product of two rows of A - q I)
template <typename T>
__device__ __forceinline__ void eig_top(const T a[3][3], T& q, T d[3]) {
  const T p1 = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
  const T qm = (a[0][0] + a[1][1] + a[2][2]) / T(3);
  const T d0 = a[0][0] - qm, d1 = a[1][1] - qm, d2 = a[2][2] - qm;
  const T p2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * p1;
  d[0] = T(0);
  d[1] = T(0);
  d[2] = T(1);
  if (!(p2 > T(0))) {
    q = qm;
    return;
  }
  const T p = sqrt(p2 / T(6));
  const T b00 = d0 / p, b11 = d1 / p, b22 = d2 / p;
  const T b01 = a[0][1] / p, b02 = a[0][2] / p, b12 = a[1][2] / p;
  const T det = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
  T r = det / T(2);
  r = r < T(-1) ? T(-1) : (r > T(1) ? T(1) : r);
  q = qm + T(2) * p * cos(acos(r) / T(3));
  const T r0[3] = {a[0][0] - q, a[0][1], a[0][2]};
  const T r1[3] = {a[1][0], a[1][1] - q, a[1][2]};
  const T r2[3] = {a[2][0], a[2][1], a[2][2] - q};
  auto cross = [](const T u[3], const T v[3], T w[3]) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
  };
  T c0[3], c1[3], c2[3];
  cross(r0, r1, c0);
  cross(r0, r2, c1);
  cross(r1, r2, c2);
  const T n0 = c0[0] * c0[0] + c0[1] * c0[1] + c0[2] * c0[2];
  const T n1 = c1[0] * c1[0] + c1[1] * c1[1] + c1[2] * c1[2];
  const T n2 = c2[0] * c2[0] + c2[1] * c2[1] + c2[2] * c2[2];
  // the best-conditioned of the three (selected without indexing, so it stays in registers)
  const bool s0 = n0 >= n1 && n0 >= n2, s1 = !s0 && n1 >= n2;
  const T bn = s0 ? n0 : (s1 ? n1 : n2);
  if (bn > T(0)) {
    const T inv = T(1) / sqrt(bn);
    d[0] = (s0 ? c0[0] : (s1 ? c1[0] : c2[0])) * inv;
    d[1] = (s0 ? c0[1] : (s1 ? c1[1] : c2[1])) * inv;
    d[2] = (s0 ? c0[2] : (s1 ? c1[2] : c2[2])) * inv;
  }
}

// P <- B P for the 3x3 block of one plane
__device__ __forceinline__ void apply_plane(float P[9], float cb, float sb, float cd, float sd) {
  const float B[9] = {cb * cb + sb * sb * cd, cb * sb * (1.f - cd), -sb * sd,
                      cb * sb * (1.f - cd),   sb * sb + cb * cb * cd, cb * sd,
                      sb * sd,                -cb * sd,               cd};
  float R[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[3 * i + j] = B[3 * i] * P[j] + B[3 * i + 1] * P[3 + j] + B[3 * i + 2] * P[6 + j];
#pragma unroll
  for (int k = 0; k < 9; ++k) P[k] = R[k];
}

// S_out[0] of one column from the product T of its planes' blocks, summed over
// the wavelengths with their weights: T acts on the polarised input
// (S_1, S_2, S_3) = (c_in, s_in, 0) / 2 and the analyser reads the result.
__device__ __forceinline__ float analyse(const OpticsArgs& a, int l, const float T[9]) {
  const float v0 = 0.5f * a.c_in, v1 = 0.5f * a.s_in;
  const float r0 = T[0] * v0 + T[1] * v1, r1 = T[3] * v0 + T[4] * v1;
  return a.weight[l] * 0.5f * (0.5f + a.c_out * r0 + a.s_out * r1);
}

// One work unit: 32 columns x of row y, planes [z_begin, z_end) of split sp of
// S; the 8 warps take consecutive sub-chunks and their products are combined
// in order by a tree in shared memory.  With S = 1 the unit writes the image;
// otherwise it writes its 3x3 products to part[((sp * nl + l) * 9 + k) * nx * ny + pixel].
template <typename real>
__global__ void __launch_bounds__(32 * kTexChunks) k_texture(const real* __restrict__ Q, OpticsArgs a, int S,
                                                             float* __restrict__ img, float* __restrict__ part) {
  __shared__ float sp_part[kTexChunks][kTexMaxLambda][9][32];
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
  const int tiles_x = (a.nx + 31) / 32;
  const int items = tiles_x * a.ny;
  const long long pix = (long long)a.nx * a.ny;
  for (int u = blockIdx.x; u < items * S; u += gridDim.x) {
    const int t = u % items, sp = u / items;
    const int x = (t % tiles_x) * 32 + lane, y = t / tiles_x;
    const bool valid = x < a.nx;
    const int zb = (int)((long long)sp * a.nz / S), ze = (int)((long long)(sp + 1) * a.nz / S);
    const int chunk = (ze - zb + kTexChunks - 1) / kTexChunks;
    float P[kTexMaxLambda][9];
#pragma unroll
    for (int l = 0; l < kTexMaxLambda; ++l)
#pragma unroll
      for (int k = 0; k < 9; ++k) P[l][k] = (k % 4 == 0) ? 1.f : 0.f;
    const int z_lo = zb + w * chunk, z_hi = min(ze, z_lo + chunk);
    for (int z = z_lo; valid && z < z_hi; ++z) {
      const long long s = ((long long)z * a.ny + y) * a.nx + x;
      const float xx = (float)Q[s], xy = (float)Q[a.n + s], xz = (float)Q[2 * a.n + s];
      const float yy = (float)Q[3 * a.n + s], yz = (float)Q[4 * a.n + s];
      const float m[3][3] = {{xx, xy, xz}, {xy, yy, yz}, {xz, yz, -xx - yy}};
      float q, d[3];
      eig_top(m, q, d);
      const float rxy = d[0] * d[0] + d[1] * d[1];
      float cb = 1.f, sb = 0.f;
      if (rxy > 0.f) {
        const float inv = 1.f / rxy;
        cb = (d[1] * d[1] - d[0] * d[0]) * inv;
        sb = 2.f * d[0] * d[1] * inv;
      }
      const float cos2 = d[2] * d[2];
      const float n_eff = a.n_o * a.n_e * rsqrtf(a.n_o * a.n_o * (1.f - cos2) + a.n_e * a.n_e * cos2);
#pragma unroll
      for (int l = 0; l < kTexMaxLambda; ++l) {
        if (l < a.nl) {
          const float delta = a.two_pi_h_over_lambda[l] * q * (n_eff - a.n_o);
          float sd, cd;
          sincosf(delta, &sd, &cd);
          apply_plane(P[l], cb, sb, cd, sd);
        }
      }
    }
#pragma unroll
    for (int l = 0; l < kTexMaxLambda; ++l)
#pragma unroll
      for (int k = 0; k < 9; ++k) sp_part[w][l][k][lane] = P[l][k];
    __syncthreads();
    // tree: warp w takes the product of chunks w + st (later) and w (earlier)
    for (int st = 1; st < kTexChunks; st *= 2) {
      if (w % (2 * st) == 0) {
        for (int l = 0; l < a.nl; ++l) {
          float R[9];
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
              R[3 * i + j] = sp_part[w + st][l][3 * i][lane] * sp_part[w][l][j][lane] +
                             sp_part[w + st][l][3 * i + 1][lane] * sp_part[w][l][3 + j][lane] +
                             sp_part[w + st][l][3 * i + 2][lane] * sp_part[w][l][6 + j][lane];
#pragma unroll
          for (int k = 0; k < 9; ++k) sp_part[w][l][k][lane] = R[k];
        }
      }
      __syncthreads();
    }
    if (w == 0 && valid) {
      const long long px = (long long)y * a.nx + x;
      if (S == 1) {
        float out = 0.f;
        for (int l = 0; l < a.nl; ++l) {
          float T[9];
#pragma unroll
          for (int k = 0; k < 9; ++k) T[k] = sp_part[0][l][k][lane];
          out += analyse(a, l, T);
        }
        img[px] = out;
      } else {
        for (int l = 0; l < a.nl; ++l)
#pragma unroll
          for (int k = 0; k < 9; ++k) part[((long long)(sp * a.nl + l) * 9 + k) * pix + px] = sp_part[0][l][k][lane];
      }
    }
    __syncthreads();
  }
}

// image from S split products per column: T = T_{S-1} ... T_0 per wavelength
__global__ void k_texture_combine(OpticsArgs a, int S, const float* __restrict__ part, float* __restrict__ img) {
  const long long pix = (long long)a.nx * a.ny;
  for (long long px = blockIdx.x * (long long)blockDim.x + threadIdx.x; px < pix; px += (long long)gridDim.x * blockDim.x) {
    float out = 0.f;
    for (int l = 0; l < a.nl; ++l) {
      float T[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
      for (int sp = 0; sp < S; ++sp) {
        const float* M = part + (long long)(sp * a.nl + l) * 9 * pix + px;
        float R[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            R[3 * i + j] = M[(3 * i) * pix] * T[j] + M[(3 * i + 1) * pix] * T[3 + j] + M[(3 * i + 2) * pix] * T[6 + j];
#pragma unroll
        for (int k = 0; k < 9; ++k) T[k] = R[k];
      }
      out += analyse(a, l, T);
    }
    img[px] = out;
  }
}

// Splits of z per column: enough work units for about two per SM, each warp
// keeping at least 4 planes, and the split products fitting in `scratch_floats`
// after the image.
int texture_splits(int nx, int ny, int nz, int nl, long long scratch_floats, int sms) {
  const long long items = (long long)((nx + 31) / 32) * ny;
  const long long pix = (long long)nx * ny, pix_r = (pix + 63) / 64 * 64;
  long long S = (2LL * sms + items - 1) / items;
  S = std::min<long long>(S, std::max(1, nz / (4 * kTexChunks)));
  S = std::min<long long>(S, std::max<long long>(1, (scratch_floats - pix_r) / (9LL * nl * pix)));
  return (int)std::max<long long>(1, S);
}

template <typename real>
cudaError_t launch_texture(const void* q, int nx, int ny, int nz, const lcbp_optics& o, float* d_img,
                           long long scratch_floats, cudaStream_t s) {
  OpticsArgs a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.n = (long long)nx * ny * nz;
  a.nl = o.nlambda;
  for (int l = 0; l < o.nlambda; ++l) {
    a.two_pi_h_over_lambda[l] = (float)(2.0 * 3.14159265358979323846 * o.h / o.lambda[l]);
    a.weight[l] = (float)o.weight[l];
  }
  a.n_o = (float)o.n_o;
  a.n_e = (float)o.n_e;
  a.c_in = (float)std::cos(2.0 * o.phi_in);
  a.s_in = (float)std::sin(2.0 * o.phi_in);
  a.c_out = (float)std::cos(2.0 * o.phi_out);
  a.s_out = (float)std::sin(2.0 * o.phi_out);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long pix = (long long)nx * ny;
  const int S = texture_splits(nx, ny, nz, a.nl, scratch_floats, sms);
  float* part = d_img + ((pix + 63) / 64) * 64;  // split products after the image (256-byte aligned)
  const long long units = (long long)((nx + 31) / 32) * ny * S;
  const int grid = (int)std::min<long long>(units, 65535);
  k_texture<real><<<grid, 32 * kTexChunks, 0, s>>>(static_cast<const real*>(q), a, S, d_img, part);
  if (S > 1) {
    const int g2 = (int)std::min<long long>((pix + 255) / 256, 65535);
    k_texture_combine<<<g2, 256, 0, s>>>(a, S, part, d_img);
  }
  return cudaGetLastError();
}

template cudaError_t launch_texture<float>(const void*, int, int, int, const lcbp_optics&, float*, long long,
                                           cudaStream_t);
template cudaError_t launch_texture<double>(const void*, int, int, int, const lcbp_optics&, float*, long long,
                                            cudaStream_t);

}  // namespace lcbp

extern "C" int lcbp_optics_default(lcbp_optics* o) {
  if (!o) return lcbp::fail(LCBP_EINVAL, "o is NULL");
  *o = lcbp_optics{};
  o->nlambda = 3;
  o->lambda[0] = 16.0;
  o->lambda[1] = 18.0;
  o->lambda[2] = 20.0;
  o->weight[0] = 0.2;
  o->weight[1] = 0.6;
  o->weight[2] = 0.2;
  o->n_o = 1.5;
  o->n_e = 2.0;
  o->h = 1.0;
  o->phi_in = 0.0;
  o->phi_out = 1.5707963267948966;
  return LCBP_OK;
}
