// The k slice products of one chunk in one launch, for N <= 128 (Sec. 2,
// Eq. (Ztr); the naive products between two re-factorisations, Sec. 4.1).
//
// Forward chain:  C <- E diag(e^{V_l}) C   for l = lo .. hi
// Backward chain: C <- diag(e^{V_l}) E^T C for l = hi .. lo   (B_l^T, App. A)
//
// A column block of C evolves on its own through the whole chunk (every slice
// multiplies from the left), so one CTA owns 16 columns of one instance and
// applies all slices with E, the block and its scaled copy in shared memory.
// For small N a separate launch per slice spends most of its time outside
// the FMAs (short K loop, tile loads, stores, tail waves); here the FP64 pipe
// is the only limit.  Every output is one FMA chain over m in increasing
// order with the row scale staged once per element (forward) or applied once
// to the sum (backward), as the batched GEMM does, so results are bitwise
// those of k separate products.
#include "common.cuh"

namespace dqmc {

namespace {

constexpr int CS_CB = 16;      // columns per CTA
constexpr int CS_NT = 256;     // threads per CTA: 16 columns x 16 row groups

template <int RPT>
__global__ void __launch_bounds__(CS_NT, 1) chain_small_kernel(const ChainSmallArgs a) {
  extern __shared__ __align__(16) double cs_smem[];
  const int N = a.N;
  double* Es = cs_smem;                       // Es[m * N + i] = E(i, m) of the product
  double* Ps = Es + (long long)N * N;         // current block, N x CB
  double* Qs = Ps + (long long)N * CS_CB;     // scaled copy / next block, N x CB
  const int b = blockIdx.y;
  const int c0 = blockIdx.x * CS_CB;
  const int tid = threadIdx.x;
  const int c = tid % CS_CB, r0 = tid / CS_CB;   // this thread: column c0 + c, rows r0 + 16 q
  const double* X = a.X + (long long)b * a.sX;
  double* C = a.C + (long long)b * a.sC;
  const double* ev = a.expV + (long long)(b / a.divS) * a.sV + (long long)(b % a.divS) * a.sV_inner;
  // launch contract (debug build): CS_NT threads, RPT rows per thread that
  // cover N, column blocks that cover N, shared memory for E and two blocks
  if (!DQMC_CHECK(blockDim.x == CS_NT && N <= 16 * RPT && (int)gridDim.x * CS_CB >= N, N) ||
      !DQMC_CHECK(dyn_smem_bytes() >= (unsigned)(((long long)N * N + 2LL * N * CS_CB) * 8),
                  dyn_smem_bytes()))
    return;
  int nsl = a.nslices;
  if (a.lim) {                                 // slices past the instance's own chain end
    const int last = a.lim[b] - a.lim_base + 1;
    nsl = last < nsl ? (last > 0 ? last : 0) : nsl;
  }

  for (long long e = tid; e < (long long)N * N; e += CS_NT) {
    const int m = (int)(e / N), i = (int)(e % N);
    Es[e] = a.transE ? a.E[(long long)m * N + i] : a.E[(long long)i * N + m];
  }
  for (int e = tid; e < N * CS_CB; e += CS_NT) {
    const int m = e / CS_CB, j = e % CS_CB;
    Ps[e] = c0 + j < N ? X[(long long)m * N + c0 + j] : 0.0;
  }
  __syncthreads();

  for (int s = 0; s < nsl; ++s) {
    const int l = a.dir > 0 ? a.lo + s : a.hi - s;
    const double* sc = ev + (long long)(l - 1) * N;
    double acc[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) acc[q] = 0.0;
    if (a.dir > 0) {
      // C_new = E (diag(e^{V_l}) C): the scaled block first, then the product
      for (int e = tid; e < N * CS_CB; e += CS_NT) Qs[e] = Ps[e] * sc[e / CS_CB];
      __syncthreads();
      for (int m = 0; m < N; ++m) {
        const double x = Qs[m * CS_CB + c];
        const double* er = Es + (long long)m * N;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int i = r0 + 16 * q;
          if (i < N) acc[q] = fma(er[i], x, acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int i = r0 + 16 * q;
        if (i < N) Ps[i * CS_CB + c] = acc[q];     // Qs is no longer read
      }
    } else {
      // C_new = diag(e^{V_l}) (E^T C)
      for (int m = 0; m < N; ++m) {
        const double x = Ps[m * CS_CB + c];
        const double* er = Es + (long long)m * N;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int i = r0 + 16 * q;
          if (i < N) acc[q] = fma(er[i], x, acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int i = r0 + 16 * q;
        if (i < N) Qs[i * CS_CB + c] = acc[q] * sc[i];
      }
      __syncthreads();
      double* t = Ps; Ps = Qs; Qs = t;
    }
    __syncthreads();
  }

  for (int e = tid; e < N * CS_CB; e += CS_NT) {
    const int m = e / CS_CB, j = e % CS_CB;
    if (c0 + j < N) C[(long long)m * N + c0 + j] = Ps[e];
  }
}

template <int RPT>
cudaError_t launch_chain_small(const ChainSmallArgs& a, cudaStream_t st) {
  const size_t sm = ((size_t)a.N * a.N + 2 * (size_t)a.N * CS_CB) * sizeof(double);
  cudaError_t e = allow_dyn_smem(chain_small_kernel<RPT>);
  if (e != cudaSuccess) return e;
  const dim3 grid((a.N + CS_CB - 1) / CS_CB, a.batch);
  chain_small_kernel<RPT><<<grid, CS_NT, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t chain_small(const ChainSmallArgs& a, cudaStream_t st) {
  if (a.batch <= 0 || a.nslices <= 0) return cudaSuccess;
  if (a.N < 1 || a.N > CHAIN_SMALL_MAX_N || a.batch > 65535) return cudaErrorInvalidValue;
  if (a.N <= 16) return launch_chain_small<1>(a, st);
  if (a.N <= 32) return launch_chain_small<2>(a, st);
  if (a.N <= 64) return launch_chain_small<4>(a, st);
  return launch_chain_small<8>(a, st);
}

}  // namespace dqmc

DQMC_CHECK_UNIT(chain_small)
