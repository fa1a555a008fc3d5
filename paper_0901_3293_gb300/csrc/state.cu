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

// Element of component c at padded position (X, Y) of plane z in a padded
// mirror whose first 4G components are interleaved by fours
// ([group][z][Y][X][4]) and whose others follow as plain arrays ([z][Y][X]).
__device__ __forceinline__ long long mirror_at(int c, int z, int Y, int X, int G, int nz, int nxp, int nyp) {
  if (c < 4 * G) return ((((long long)(c >> 2) * nz + z) * nyp + Y) * nxp + X) * 4 + (c & 3);
  return 4LL * G * nz * nyp * nxp + (((long long)(c - 4 * G) * nz + z) * nyp + Y) * nxp + X;
}

// every padded position of component c: flat[c][z][wrap(Y - hy)][wrap(X - hx)]
template <typename real>
__global__ void k_pack(const real* __restrict__ flat, real* __restrict__ padded, int C, int G, int nx, int ny, int nz,
                       int hx, int hy, int nxp, int nyp) {
  const long long total = (long long)C * nz * nyp * nxp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(i % nxp);
    const long long r = i / nxp;
    const int Y = (int)(r % nyp);
    const long long cz = r / nyp;  // c * nz + z
    const int z = (int)(cz % nz), c = (int)(cz / nz);
    int x = (X - hx) % nx, y = (Y - hy) % ny;
    x += x < 0 ? nx : 0;
    y += y < 0 ? ny : 0;
    padded[mirror_at(c, z, Y, X, G, nz, nxp, nyp)] = flat[(cz * ny + y) * nx + x];
  }
}

// flat[c][z][y][x] = the padded value at (x + hx, y + hy)
template <typename real>
__global__ void k_unpack(const real* __restrict__ padded, real* __restrict__ flat, int C, int G, int nx, int ny,
                         int nz, int hx, int hy, int nxp, int nyp) {
  const long long total = (long long)C * nz * ny * nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const long long r = i / nx;
    const int y = (int)(r % ny);
    const long long cz = r / ny;
    const int z = (int)(cz % nz), c = (int)(cz / nz);
    flat[i] = padded[mirror_at(c, z, y + hy, x + hx, G, nz, nxp, nyp)];
  }
}

template <typename real>
cudaError_t launch_pack(const void* flat, void* padded, int C, int G, int nx, int ny, int nz, int hx, int hy,
                        int nxp, int nyp, cudaStream_t s) {
  k_pack<real><<<4096, 256, 0, s>>>(static_cast<const real*>(flat), static_cast<real*>(padded), C, G, nx, ny, nz, hx,
                                    hy, nxp, nyp);
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_unpack(const void* padded, void* flat, int C, int G, int nx, int ny, int nz, int hx, int hy,
                          int nxp, int nyp, cudaStream_t s) {
  k_unpack<real><<<4096, 256, 0, s>>>(static_cast<const real*>(padded), static_cast<real*>(flat), C, G, nx, ny, nz,
                                      hx, hy, nxp, nyp);
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
