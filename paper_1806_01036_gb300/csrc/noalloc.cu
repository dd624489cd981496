// noalloc.cu — eo_gram_dd_noalloc: the compensated Gram product without any
// device allocation and without a context.
//
// Some callers cannot allocate device memory at the moment they need a Gram
// matrix: a component whose device memory is entirely owned by another pool
// (for example a framework's caching allocator that has reserved the GPU), or
// a latency-critical loop that must not pay for cudaMalloc/cudaFree, which
// can synchronize the whole device.  This entry point serves them: its only
// scratch is the file-scope array below, which every GPU that loads the
// library holds until the process exits.
//
// The array's name in host code is a host-side stand-in, not a device
// address, so the device address is looked up with cudaGetSymbolAddress
// (with the device current) and passed to the kernels.  The lookup is done
// once per device context: the address is cached with the unique id of the
// context it belongs to, and looked up again when the device's context has
// been re-created (after cudaDeviceReset the module is loaded anew and the
// array may move).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace {

// Largest block width served here, and the scratch that covers it: at most
// 152 row chunks (one per SM) of kx*ky partial sums of 32 bytes each.
constexpr int kNoallocKmax = EO_NOALLOC_KMAX;
constexpr size_t kNoallocBytes = EO_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// The driver's id of the current context (unique over the process's
// lifetime, unlike the handle, whose value a re-created context may reuse).
bool current_context_id(unsigned long long* id) {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
  });
  CUcontext c = nullptr;
  return get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch on the current device: looked up on
// the first call in each context of the device, cached for later calls.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // (no current context yet: the id is unknown, and the lookup below creates
  // and binds the device's context, so the next call finds it cached)
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev] || !have_id || g_ctx_id[dev] != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = p;
    g_ctx_id[dev] = have_id ? id : 0;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" eo_status eo_gram_dd_noalloc(int64_t n, int kx, const double* X, int64_t ldx, int ky, const double* Y,
                                        int64_t ldy, double* G_hi, double* G_lo, int ldg, void* cuda_stream) {
  const bool sym = Y == nullptr;
  if (sym) {
    ky = kx;
    ldy = ldx;
  }
  const int64_t mn = n > 1 ? n : 1;
  if (n < 0 || n > EO_NOALLOC_NMAX || kx < 1 || ky < 1 || kx > kNoallocKmax || ky > kNoallocKmax) return EO_EINVAL;
  if ((!X && n > 0) || !G_hi || ldx < mn || ldy < mn || ldg < kx) return EO_EINVAL;
  // Every partial sum the kernels read is written by the same call first, so
  // nothing in the array has to start at zero.
  if (eo::fx_gram_scratch_bytes(n, kx, ky, sym) > kNoallocBytes) return EO_EINVAL;
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return EO_ECUDA;
  }
  cudaError_t e = eo::launch_fx_gram(n, kx, X, ldx, ky, sym ? X : Y, ldy, sym, scratch, G_hi, G_lo, ldg, nullptr,
                                     static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EO_ECUDA;
  }
  return EO_OK;
}
