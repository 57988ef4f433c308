// FP64 arithmetic rate of the device: the roofline denominator of every FP64
// kernel of the library.  The paper has no counterpart; this measures the
// machine, not the method.
//
// Three loop kernels, each a grid of several CTAs per SM whose warps issue
// only independent FP64 operations (no memory traffic inside the loop):
//   DFMA       fma.rn.f64 on 8 independent chains per thread (2 flop each);
//   DMMA m8n8k4   mma.sync.aligned.m8n8k4.row.col.f64 (512 flop per warp
//              instruction), 4 independent accumulators per warp;
//   DMMA m16n8k8  mma.sync.aligned.m16n8k8.row.col.f64 (2048 flop per warp
//              instruction), 2 independent accumulators per warp.
// Each thread writes one sum at the end so the loops cannot be removed.  The
// host times one launch with CUDA events after one warm-up launch.
#include <cstdio>

#include "common.cuh"

namespace {

constexpr int RATE_THREADS = 256;

__global__ void __launch_bounds__(RATE_THREADS) dfma_loop_kernel(double* sink, int iters,
                                                                 double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (double)(threadIdx.x + i) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  sink[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void dmma_m8n8k4(double& d0, double& d1, double a, double b) {
  asm volatile(
      "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
      : "+d"(d0), "+d"(d1)
      : "d"(a), "d"(b));
}

__device__ __forceinline__ void dmma_m16n8k8(double* d, const double* a, const double* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}

__global__ void __launch_bounds__(RATE_THREADS) dmma884_loop_kernel(double* sink, int iters,
                                                                    double a, double b) {
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = 0.0;
  const double av = a * (double)(threadIdx.x & 7), bv = b;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
      for (int i = 0; i < 4; ++i) dmma_m8n8k4(c[i][0], c[i][1], av, bv);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  sink[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(RATE_THREADS) dmma1688_loop_kernel(double* sink, int iters,
                                                                     double a, double b) {
  double c[2][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) c[i][j] = 0.0;
  double av[4], bv[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) av[j] = a * (double)((threadIdx.x + j) & 7);
  bv[0] = b;
  bv[1] = -b;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int i = 0; i < 2; ++i) dmma_m16n8k8(c[i], av, bv);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) s += c[i][j];
  sink[blockIdx.x * (long long)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" dqmc_status dqmc_selftest_fp64_rate(void* stream, int kind, int iters, double* tflops,
                                               double* ms_out) {
  if (!tflops || kind < 0 || kind > 2 || iters < 1 || iters > (1 << 24)) return DQMC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = dqmc::device_sms();
  const int blocks = 4 * sms;                 // 32 warps per SM
  const long long threads = (long long)blocks * RATE_THREADS;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dqmc_status rc = DQMC_OK;
  if (cudaMalloc(&sink, sizeof(double) * threads) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_NOMEM;
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = DQMC_ERR_CUDA;
  // flops of one launch: per thread (DFMA) or per warp (DMMA) instruction count x flops
  double flops = 0.0;
  const long long warps = threads / 32;
  if (kind == 0) flops = (double)threads * iters * 16 * 8 * 2.0;
  else if (kind == 1) flops = (double)warps * iters * 4 * 4 * (2.0 * 8 * 8 * 4);
  else flops = (double)warps * iters * 8 * 2 * (2.0 * 16 * 8 * 8);
  auto launch = [&](int n) {
    if (kind == 0) dfma_loop_kernel<<<blocks, RATE_THREADS, 0, st>>>(sink, n, 0.999999, 1e-7);
    else if (kind == 1) dmma884_loop_kernel<<<blocks, RATE_THREADS, 0, st>>>(sink, n, 1e-3, 1e-3);
    else dmma1688_loop_kernel<<<blocks, RATE_THREADS, 0, st>>>(sink, n, 1e-3, 1e-3);
    return cudaGetLastError();
  };
  float ms = 0.f;
  if (rc == DQMC_OK && launch(iters / 8 > 0 ? iters / 8 : 1) != cudaSuccess) rc = DQMC_ERR_CUDA;
  if (rc == DQMC_OK) {
    cudaEventRecord(e0, st);
    if (launch(iters) != cudaSuccess) rc = DQMC_ERR_CUDA;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = DQMC_ERR_CUDA;
  }
  if (rc == DQMC_OK && ms > 0.f) {
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaGetLastError();
  return rc;
}
