// Whole-field operations on device arrays: the count of non-finite values
// (used to refuse uploads), the largest absolute difference of two fields
// (used by the surrogate judge to compare a surrogate call with plain steps),
// both reduced in a fixed order, and the copies between a field and its
// padded mirror with periodic ghosts (the fast step's state layout).
#include <cmath>

#include "kernels.h"

namespace lcbp {

namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 512;

template <typename real>
__global__ void k_count_nonfinite(const real* __restrict__ v, long long n, unsigned long long* __restrict__ partial) {
  unsigned long long c = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    c += isfinite(v[i]) ? 0ull : 1ull;
  __shared__ unsigned long long red[kRedThreads];
  red[threadIdx.x] = c;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// max |a - b| over n values, as a double; a NaN anywhere gives NaN
template <typename real>
__global__ void k_max_abs_diff(const real* __restrict__ a, const real* __restrict__ b, long long n,
                               double* __restrict__ partial) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = fabs((double)a[i] - (double)b[i]);
    m = (d > m || d != d) ? d : m;
  }
  __shared__ double red[kRedThreads];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      const double o = red[threadIdx.x + s];
      if (o > red[threadIdx.x] || o != o) red[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <typename T>
__global__ void k_final_sum(const T* __restrict__ partial, int nb, T* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    T s = 0;
    for (int i = 0; i < nb; ++i) s += partial[i];
    *out = s;
  }
}

__global__ void k_final_max(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < nb; ++i) {
      const double v = partial[i];
      if (v > m || v != v) m = v;
    }
    *out = m;
  }
}

int blocks_for(long long n) {
  const long long b = (n + kRedThreads - 1) / kRedThreads;
  return (int)(b < kRedBlocks ? (b > 0 ? b : 1) : kRedBlocks);
}

}  // namespace

size_t state_check_scratch_bytes() { return (size_t)(kRedBlocks + 1) * 8; }

template <typename real>
cudaError_t launch_count_nonfinite(const void* v, long long n, void* scratch, unsigned long long* out,
                                   cudaStream_t s) {
  auto* partial = static_cast<unsigned long long*>(scratch);
  const int nb = blocks_for(n);
  k_count_nonfinite<real><<<nb, kRedThreads, 0, s>>>(static_cast<const real*>(v), n, partial);
  k_final_sum<unsigned long long><<<1, 32, 0, s>>>(partial, nb, out);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_max_abs_diff(const void* a, const void* b, long long n, void* scratch, double* out,
                                cudaStream_t s) {
  auto* partial = static_cast<double*>(scratch);
  const int nb = blocks_for(n);
  k_max_abs_diff<real><<<nb, kRedThreads, 0, s>>>(static_cast<const real*>(a), static_cast<const real*>(b), n,
                                                   partial);
  k_final_max<<<1, 32, 0, s>>>(partial, nb, out);
  return cudaGetLastError();
}

// A padded mirror holds its first 4G components interleaved by fours
// ([group][z][Y][X][4]) and the others as plain arrays ([z][Y][X]) after
// them.  The copies below walk it by units (a group of four components, or
// one plain component) and rows: one CTA per (unit, plane, row), threads
// along the row, so no thread divides a 64-bit index and a group moves as one
// 16-byte vector (FP32) per site.
__device__ __forceinline__ int wrap_mod(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

template <typename real>
__device__ __forceinline__ void put4(real* p, real a, real b, real c, real d) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
    *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
  }
}
template <typename real>
__device__ __forceinline__ void get4(const real* p, real v[4]) {
  if constexpr (sizeof(real) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
}

// every padded position of every component: flat[c][z][wrap(Y - hy)][wrap(X - hx)]
template <typename real>
__global__ void k_pack(const real* __restrict__ flat, real* __restrict__ padded, int C, int G, int nx, int ny, int nz,
                       int hx, int hy, int nxp, int nyp) {
  const long long rows = (long long)(G + C - 4 * G) * nz * nyp;
  const long long plane = (long long)ny * nx, cstride = plane * nz;    // flat component stride
  const long long pplane = (long long)nyp * nxp, pstride = pplane * nz;  // padded plain-component stride
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int Y = (int)(r % nyp);
    const long long uz = r / nyp;
    const int z = (int)(uz % nz), u = (int)(uz / nz);
    const int y = wrap_mod(Y - hy, ny);
    const real* src = flat + (long long)z * plane + (long long)y * nx;
    if (u < G) {
      src += (long long)(4 * u) * cstride;
      real* dst = padded + (((long long)u * nz + z) * nyp + Y) * nxp * 4;
      for (int X = threadIdx.x; X < nxp; X += blockDim.x) {
        const int x = wrap_mod(X - hx, nx);
        put4(dst + (long long)X * 4, src[x], src[cstride + x], src[2 * cstride + x], src[3 * cstride + x]);
      }
    } else {
      src += (long long)(4 * G + (u - G)) * cstride;
      real* dst = padded + 4 * (long long)G * pstride + (long long)(u - G) * pstride + (long long)z * pplane +
                  (long long)Y * nxp;
      for (int X = threadIdx.x; X < nxp; X += blockDim.x) dst[X] = src[wrap_mod(X - hx, nx)];
    }
  }
}

// flat[c][z][y][x] = the padded value at (x + hx, y + hy)
template <typename real>
__global__ void k_unpack(const real* __restrict__ padded, real* __restrict__ flat, int C, int G, int nx, int ny,
                         int nz, int hx, int hy, int nxp, int nyp) {
  const long long rows = (long long)(G + C - 4 * G) * nz * ny;
  const long long plane = (long long)ny * nx, cstride = plane * nz;
  const long long pplane = (long long)nyp * nxp, pstride = pplane * nz;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const int y = (int)(r % ny);
    const long long uz = r / ny;
    const int z = (int)(uz % nz), u = (int)(uz / nz);
    real* dst = flat + (long long)z * plane + (long long)y * nx;
    if (u < G) {
      dst += (long long)(4 * u) * cstride;
      const real* src = padded + (((long long)u * nz + z) * nyp + (y + hy)) * nxp * 4;
      for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        real v[4];
        get4(src + (long long)(x + hx) * 4, v);
        dst[x] = v[0];
        dst[cstride + x] = v[1];
        dst[2 * cstride + x] = v[2];
        dst[3 * cstride + x] = v[3];
      }
    } else {
      dst += (long long)(4 * G + (u - G)) * cstride;
      const real* src = padded + 4 * (long long)G * pstride + (long long)(u - G) * pstride + (long long)z * pplane +
                        (long long)(y + hy) * nxp;
      for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = src[x + hx];
    }
  }
}

int copy_grid(long long rows) { return (int)(rows < (1ll << 30) ? (rows > 0 ? rows : 1) : (1ll << 30)); }

template <typename real>
cudaError_t launch_pack(const void* flat, void* padded, int C, int G, int nx, int ny, int nz, int hx, int hy,
                        int nxp, int nyp, cudaStream_t s) {
  const long long rows = (long long)(C - 3 * G) * nz * nyp;
  k_pack<real><<<copy_grid(rows), 128, 0, s>>>(static_cast<const real*>(flat), static_cast<real*>(padded), C, G, nx,
                                               ny, nz, hx, hy, nxp, nyp);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack(const void* padded, void* flat, int C, int G, int nx, int ny, int nz, int hx, int hy,
                          int nxp, int nyp, cudaStream_t s) {
  const long long rows = (long long)(C - 3 * G) * nz * ny;
  k_unpack<real><<<copy_grid(rows), 128, 0, s>>>(static_cast<const real*>(padded), static_cast<real*>(flat), C, G,
                                                 nx, ny, nz, hx, hy, nxp, nyp);
  return cudaGetLastError();
}

template cudaError_t launch_pack<float>(const void*, void*, int, int, int, int, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_pack<double>(const void*, void*, int, int, int, int, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_unpack<float>(const void*, void*, int, int, int, int, int, int, int, int, int,
                                          cudaStream_t);
template cudaError_t launch_unpack<double>(const void*, void*, int, int, int, int, int, int, int, int, int,
                                           cudaStream_t);

template cudaError_t launch_count_nonfinite<float>(const void*, long long, void*, unsigned long long*, cudaStream_t);
template cudaError_t launch_count_nonfinite<double>(const void*, long long, void*, unsigned long long*, cudaStream_t);
template cudaError_t launch_max_abs_diff<float>(const void*, const void*, long long, void*, double*, cudaStream_t);
template cudaError_t launch_max_abs_diff<double>(const void*, const void*, long long, void*, double*, cudaStream_t);

}  // namespace lcbp
