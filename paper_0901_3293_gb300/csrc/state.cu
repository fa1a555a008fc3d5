// Whole-field checks on device arrays: the count of non-finite values (used
// to refuse uploads) and the largest absolute difference of two fields (used
// by the surrogate judge to compare a surrogate call with plain steps).
// Both reduce in a fixed order, so a result never depends on scheduling.
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

template cudaError_t launch_count_nonfinite<float>(const void*, long long, void*, unsigned long long*, cudaStream_t);
template cudaError_t launch_count_nonfinite<double>(const void*, long long, void*, unsigned long long*, cudaStream_t);
template cudaError_t launch_max_abs_diff<float>(const void*, const void*, long long, void*, double*, cudaStream_t);
template cudaError_t launch_max_abs_diff<double>(const void*, const void*, long long, void*, double*, cudaStream_t);

}  // namespace lcbp
