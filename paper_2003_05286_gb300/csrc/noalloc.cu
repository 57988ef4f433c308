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

// Device address of g_scratch per device (host code only ever holds the
// symbol's host-side stand-in otherwise, which must not reach a kernel).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" dqmc_status dqmc_greens_noalloc(void* stream, int batch, int N, int M, const double* K,
                                           double dtau, const double* V, int k, double* G,
                                           double* logdet, int* sign, int* status) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return DQMC_ERR_UNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    // one-time set-up on this device (the current one): resolve the array's
    // device address.  Racing first calls from two host threads store the
    // same value.
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return DQMC_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  return dqmc::greens_on_workspace(stream, g_scratch_addr[dev], kScratchBytes, batch, N, M, K,
                                   dtau, V, k, G, logdet, sign, status);
}
