// Allocation-free equal-time entry point.
//
// Some callers cannot allocate device memory: code running inside a memory
// pool or arena that owns the whole device budget, plugins loaded into a host
// application whose allocator must not be bypassed, or a process that has to
// stay within a fixed footprint decided up front.  dqmc_greens_noalloc serves
// them: it computes the same G / log det / sign as dqmc_greens, but every
// intermediate lives in one file-scope device array of fixed size, so the call
// itself issues no cudaMalloc, cudaFree or allocating library routine.
#include "common.cuh"

namespace {

// Fixed scratch: 32 MiB per device, reserved when the library's device code
// is loaded on that device and held until the process exits.
constexpr size_t kScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

}  // namespace

extern "C" dqmc_status dqmc_greens_noalloc(void* stream, int batch, int N, int M, const double* K,
                                           double dtau, const double* V, int k, double* G,
                                           double* logdet, int* sign, int* status) {
  // In host code g_scratch names a host-side stand-in, not device memory, so
  // the array's device address is looked up in the current context on every
  // call.  Once the module is loaded this is a table lookup; no address is
  // cached, so a context created later on the same device (an application
  // that binds its own context, or one re-created after cudaDeviceReset)
  // never receives a stale address.  The first call in a context may load the
  // module, which is why it has to come before any stream capture.
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return DQMC_ERR_CUDA;
  }
  return dqmc::greens_on_workspace(stream, p, kScratchBytes, batch, N, M, K, dtau, V, k, G,
                                   logdet, sign, status);
}
