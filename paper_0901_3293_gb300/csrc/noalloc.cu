// Allocation-free free-energy reduction.
//
// Some callers cannot allocate device memory at the moment they need the
// free energy: code inside a framework whose caching allocator owns the whole
// device heap, or a real-time loop that must never touch the allocator.  This
// entry point serves them: it reduces a caller-owned device Q field with the
// same FP64 diagnostics kernel as lcbp_free_energy, but its scratch (the
// per-block partial sums) lives in a fixed file-scope device array instead of
// memory obtained with cudaMalloc.  It covers a periodic lattice with the
// one-constant energy (L2 = K, no walls).
#include <cstdint>
#include <mutex>

#include <cuda.h>

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
// per device: the unique ID of the context the address was looked up in
// (a context handle can be reused after a reset; the ID is not), and the address
struct ScratchAddr {
  unsigned long long ctx_id;
  double* ptr;
};
ScratchAddr g_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// driver entry points, found once through the runtime
template <typename Fn>
Fn driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    return reinterpret_cast<Fn>(p);
  return nullptr;
}

// ID of the current context; 0 if none is current
int current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    get = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  });
  if (!get || !get_id) return lcbp::fail(LCBP_ECUDA, "cuCtxGetCurrent / cuCtxGetId unavailable");
  CUcontext ctx = nullptr;
  if (get(&ctx) != CUDA_SUCCESS) return lcbp::fail(LCBP_ECUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return lcbp::fail(LCBP_ECUDA, "cuCtxGetId failed");
  return LCBP_OK;
}

// Device address of the scratch on the current device (the symbol name in
// host code is only a stand-in, not an address).  It is looked up on the
// first call in each context of a device: a call after cudaDeviceReset, which
// ends the context and unloads the module, looks it up again.
int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lcbp::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return lcbp::fail(LCBP_EINVAL, "device ordinal %d out of range", dev);
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (id == 0 || !g_scratch[dev].ptr || g_scratch[dev].ctx_id != id) {
    // the lookup also brings up the device's primary context if none is current
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return lcbp::cuda_fail(e, "cudaGetSymbolAddress");
    rc = current_context_id(&id);
    if (rc) return rc;
    if (id == 0) return lcbp::fail(LCBP_ECUDA, "no current CUDA context");
    g_scratch[dev] = {id, static_cast<double*>(p)};
  }
  *out = g_scratch[dev].ptr;
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
