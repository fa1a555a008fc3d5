// Allocation-free free-energy reduction.
//
// Some callers cannot allocate device memory at the moment they need the
// free energy: code running while a stream is being captured into a CUDA
// graph (cudaMalloc is not capturable), code inside a framework whose caching
// allocator owns the whole device heap, or a real-time loop that must never
// touch the allocator.  This entry point serves them: it reduces a
// caller-owned device Q field with the same FP64 diagnostics kernel as
// lcbp_free_energy, but its scratch (the per-block partial sums) lives in a
// fixed file-scope device array instead of memory obtained with cudaMalloc.
#include <cstdint>
#include <mutex>

#include "../../include/lcbp.h"
#include "kernels.h"
#include "runtime.h"

namespace {

// Partial sums of the reduction (kDiagPartials doubles) plus its 8-value
// result: 32.8 KB held by every GPU that loads the library, until exit.
constexpr int kScratchDoubles = lcbp::kDiagPartials + 8;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the symbol name in host code is only a stand-in, not an address).
int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lcbp::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return lcbp::fail(LCBP_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return lcbp::cuda_fail(e, "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LCBP_OK;
}

}  // namespace

extern "C" int lcbp_free_energy_noalloc(const void* q5, int dtype, int nx, int ny, int nz, double A0, double gamma,
                                        double K, double q0, void* stream, double* F) {
  using namespace lcbp;
  if (!q5 || !F) return fail(LCBP_EINVAL, "q5 and F must not be NULL");
  if (!valid_dtype(dtype)) return fail(LCBP_EINVAL, "bad dtype %d", dtype);
  if (nx < 1 || ny < 1 || nz < 1) return fail(LCBP_EINVAL, "lattice sizes must be >= 1");
  const long long n = (long long)nx * ny * nz;
  if (n > LCBP_NOALLOC_MAX_SITES)
    return fail(LCBP_EINVAL, "%lld sites exceed the allocation-free maximum of %lld", n,
                (long long)LCBP_NOALLOC_MAX_SITES);
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DiagGeom g{nx, ny, nz, n, 0, A0, gamma, K, q0};
  double* partials = scratch;
  double* out = scratch + kDiagPartials;
  cudaError_t e = dtype == LCBP_F64 ? launch_diag_one<double>(g, q5, nullptr, 0, 0.0, partials, out, st)
                                    : launch_diag_one<float>(g, q5, nullptr, 0, 0.0, partials, out, st);
  double res[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, out, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "free_energy_noalloc");
  if (res[6] != 0.0) return fail(LCBP_ENONFINITE, "%.0f sites hold NaN or Inf", res[6]);
  *F = res[0];
  return LCBP_OK;
}
