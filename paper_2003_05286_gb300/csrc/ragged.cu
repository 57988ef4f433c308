// Gather/scatter kernels of the ragged batch: instances of different N, M, k,
// dtau and K share one call; the host groups them by (N, k, dtau, K) and each
// group runs the uniform path with a per-instance chain length M_b.
#include "common.cuh"

namespace dqmc {

namespace {
constexpr int TPB = 256;
inline int nblocks(long long n) { return grid_stride_blocks(n, TPB); }
}  // namespace

// out[(b*Mp + l)*N + i] = exp(V_pool[offV[b] + l*N + i]) for l < Mb[b], 1 beyond.
__global__ void exp_gather_kernel(const double* V, const long long* offV, const int* Mb, int batch,
                                  int Mp, int N, double* out, int* status) {
  const long long per = (long long)Mp * N, total = per * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / per);
    long long r = e % per;
    int l = (int)(r / N);
    double v = 1.0;
    if (l < Mb[b]) {
      double x = V[offV[b] + r];
      if (!isfinite(x) && status) atomicOr(&status[b], DQMC_STATUS_NONFINITE_INPUT);
      v = exp(x);
    }
    out[e] = v;
  }
}

cudaError_t exp_gather(const double* V, const long long* offV, const int* Mb, int batch, int Mp,
                       int N, double* out, int* status, cudaStream_t st) {
  long long total = (long long)Mp * N * batch;
  if (total <= 0) return cudaSuccess;
  exp_gather_kernel<<<nblocks(total), TPB, 0, st>>>(V, offV, Mb, batch, Mp, N, out, status);
  return cudaGetLastError();
}

// G_pool[offG[b] + ij] = G_local[b*N*N + ij]
__global__ void scatter_mats_kernel(const double* src, const long long* offG, int N, int batch,
                                    double* dst) {
  const long long NN = (long long)N * N, total = NN * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    dst[offG[e / NN] + e % NN] = src[e];
}

cudaError_t scatter_mats(const double* src, const long long* offG, int N, int batch, double* dst,
                         cudaStream_t st) {
  long long total = (long long)N * N * batch;
  if (total <= 0) return cudaSuccess;
  scatter_mats_kernel<<<nblocks(total), TPB, 0, st>>>(src, offG, N, batch, dst);
  return cudaGetLastError();
}

// out_x[gidx[b]] = x[b] for the per-instance scalars (each output nullable).
__global__ void scatter_scalars_kernel(const int* gidx, int batch, const double* ld, const int* sg,
                                       const int* stt, double* ld_out, int* sg_out, int* st_out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x) {
    int g = gidx[b];
    if (ld_out) ld_out[g] = ld[b];
    if (sg_out) sg_out[g] = sg[b];
    if (st_out) st_out[g] = stt[b];
  }
}

cudaError_t scatter_scalars(const int* gidx, int batch, const double* ld, const int* sg,
                            const int* stt, double* ld_out, int* sg_out, int* st_out,
                            cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  scatter_scalars_kernel<<<nblocks(batch), TPB, 0, st>>>(gidx, batch, ld, sg, stt, ld_out, sg_out,
                                                         st_out);
  return cudaGetLastError();
}

// Contiguous blocks of len doubles: gather dst[b*len + i] = src[offs[b] + i],
// scatter dst[offs[b] + i] = src[b*len + i].
__global__ void move_blocks_kernel(const double* src, double* dst, const long long* offs,
                                   long long len, int batch, int scatter) {
  const long long total = len * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / len, i = e % len;
    if (scatter) dst[offs[b] + i] = src[e];
    else dst[e] = src[offs[b] + i];
  }
}

cudaError_t move_blocks(const double* src, double* dst, const long long* offs, long long len,
                        int batch, int scatter, cudaStream_t st) {
  const long long total = len * batch;
  if (total <= 0) return cudaSuccess;
  move_blocks_kernel<<<nblocks(total), TPB, 0, st>>>(src, dst, offs, len, batch, scatter);
  return cudaGetLastError();
}

}  // namespace dqmc
