// Small element-wise kernels of the method: exp(+-V_l) of the slice matrices
// (Sec. 2), the D+ = max(D,1) / D- = min(D,1) splits of Loh's inversions
// (Eqs. (inversion_loh), (inversion_tdgf_loh)), the log-det accumulation,
// the gradient read-out 1 - G_l(i,i), and the scaling step of the matrix
// exponential exp(-dtau K).  They are O(N^2) per instance against O(N^3) for
// the products and QR, so they are written for clarity: grid-stride loops.
#include "common.cuh"

namespace dqmc {

int device_sms() {
  constexpr int kMaxDev = 64;
  static int cache[kMaxDev] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  if (dev >= 0 && dev < kMaxDev && __atomic_load_n(&cache[dev], __ATOMIC_RELAXED) > 0)
    return __atomic_load_n(&cache[dev], __ATOMIC_RELAXED);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    cudaGetLastError();
    return 152;
  }
  if (dev >= 0 && dev < kMaxDev) __atomic_store_n(&cache[dev], sms, __ATOMIC_RELAXED);
  return sms;
}

int device_smem_optin() {
  constexpr int kMaxDev = 64;
  static int cache[kMaxDev] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 227 * 1024;
  }
  if (dev >= 0 && dev < kMaxDev && __atomic_load_n(&cache[dev], __ATOMIC_RELAXED) > 0)
    return __atomic_load_n(&cache[dev], __ATOMIC_RELAXED);
  int b = 0;
  if (cudaDeviceGetAttribute(&b, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      b <= 0) {
    cudaGetLastError();
    return 227 * 1024;
  }
  if (dev >= 0 && dev < kMaxDev) __atomic_store_n(&cache[dev], b, __ATOMIC_RELAXED);
  return b;
}

namespace {
constexpr int TPB = 256;
inline int nblocks(long long n) { return grid_stride_blocks(n, TPB); }

__device__ __forceinline__ double dmode(double d, int mode) {
  switch (mode) {
    case 1: return 1.0 / fmax(d, 1.0);   // D_p^{-1}
    case 2: return fmin(d, 1.0);         // D_m
    case 3: return fmax(d, 1.0);         // D_p
    case 4: return 1.0 / d;              // D^{-1}
    case 5: return d;                    // D
    default: return 1.0;
  }
}
}  // namespace

__global__ void exp_vec_kernel(const double* v, double* out, long long n, double sgn,
                               long long per, int* status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double x = v[i];
    if (!isfinite(x) && status) atomicOr(&status[i / per], DQMC_STATUS_NONFINITE_INPUT);
    out[i] = exp(sgn * x);
  }
}

cudaError_t exp_vec(const double* v, double* out, long long n, double sgn,
                    long long per_instance, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  exp_vec_kernel<<<nblocks(n), TPB, 0, st>>>(v, out, n, sgn, per_instance, status);
  return cudaGetLastError();
}

__global__ void axpby2_kernel(const Axpby2Args a) {
  const long long NN = (long long)a.N * a.N;
  const long long total = NN * a.batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / NN);
    long long ij = e % NN;
    int i = (int)(ij / a.N), j = (int)(ij % a.N);
    double v = 0.0;
    if (a.A) {
      double x = a.A[(long long)(b / a.divA) * a.sA + ij];
      if (a.ra) x *= dmode(a.ra[(long long)(b / a.divRA) * a.sra + i], a.ra_mode);
      if (a.ca) x *= dmode(a.ca[(long long)(b / a.divCA) * a.sca + j], a.ca_mode);
      v = x;
    }
    if (a.B) {
      double y = a.B[(long long)(b / a.divB) * a.sB + ij];
      if (a.rb) y *= dmode(a.rb[(long long)(b / a.divRB) * a.srb + i], a.rb_mode);
      if (a.cb) y *= dmode(a.cb[(long long)(b / a.divCB) * a.scb + j], a.cb_mode);
      v += y;
    }
    a.C[(long long)(b / a.divC) * a.sC + ij] = v;
  }
}

cudaError_t axpby2(const Axpby2Args& a, cudaStream_t st) {
  long long total = (long long)a.N * a.N * a.batch;
  if (total <= 0) return cudaSuccess;
  axpby2_kernel<<<nblocks(total), TPB, 0, st>>>(a);
  return cudaGetLastError();
}

__global__ void dsplit_kernel(const double* D, long long sD, int n, int batch, double* out,
                              int mode) {
  const long long total = (long long)n * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long b = e / n, i = e % n;
    out[e] = dmode(D[b * sD + i], mode);
  }
}

// len[b*P0 + c] = number of slices in chunk c of a chain of M slices cut
// every k (0 for the padding chunks c >= ceil(M/k))
__global__ void chunk_len_kernel(int* len, long long total, int P0, int nc, int k, int M) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % P0);
    len[e] = c < nc - 1 ? k : (c == nc - 1 ? M - (nc - 1) * k : 0);
  }
}

cudaError_t chunk_len(int* len, int batch, int P0, int nc, int k, int M, cudaStream_t st) {
  const long long total = (long long)batch * P0;
  if (total <= 0) return cudaSuccess;
  chunk_len_kernel<<<nblocks(total), TPB, 0, st>>>(len, total, P0, nc, k, M);
  return cudaGetLastError();
}

// Slot j of instance b (q = b*nt + j) after s one-slice steps from the grid
// point tau_j = jk holds the value at l = jk + s: copied to out[b][l] while
// l stays below the next grid point and l < M; slot nt-1 (tau = M dtau) is
// copied at s = 0 only.
__global__ void scatter_tau_kernel(const double* cur, long long Q, int nt, int N, int k, int M,
                                   int s, double* out) {
  const long long NN = (long long)N * N, total = Q * NN;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long q = e / NN, ij = e % NN;
    const int j = (int)(q % nt);
    const long long b = q / nt;
    int l;
    if (j == nt - 1) {
      if (s != 0) continue;
      l = M;
    } else {
      l = j * k + s;
      const int end = (j + 1) * k < M ? (j + 1) * k : M;
      if (l >= end) continue;
    }
    out[(b * (M + 1) + l) * NN + ij] = cur[e];
  }
}

cudaError_t scatter_tau(const double* cur, long long Q, int nt, int N, int k, int M, int s,
                        double* out, cudaStream_t st) {
  const long long total = Q * N * (long long)N;
  if (total <= 0) return cudaSuccess;
  scatter_tau_kernel<<<nblocks(total), TPB, 0, st>>>(cur, Q, nt, N, k, M, s, out);
  return cudaGetLastError();
}

cudaError_t dsplit_vec(const double* D, long long sD, int n, int batch, double* out, int mode,
                       cudaStream_t st) {
  long long total = (long long)n * batch;
  if (total <= 0) return cudaSuccess;
  dsplit_kernel<<<nblocks(total), TPB, 0, st>>>(D, sD, n, batch, out, mode);
  return cudaGetLastError();
}

// out[(b*Mp + l)*N + i] = exp(sgn * V[(b*M + l)*N + i]) for l < M, 1 for M <= l < Mp
__global__ void exp_pad_kernel(const double* V, double* out, int batch, int M, int Mp, int N,
                               double sgn, int* status, const int* shift) {
  const long long total = (long long)batch * Mp * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long b = e / ((long long)Mp * N);
    long long r = e % ((long long)Mp * N);
    int l = (int)(r / N), i = (int)(r % N);
    double v = 1.0;
    if (l < M) {
      // shift[b]: slice l of the staged chain is slice l + shift[b] (mod M) of V
      const int ls = shift ? (int)(((long long)l + shift[b]) % M + M) % M : l;
      double x = V[(b * M + ls) * N + i];
      if (!isfinite(x) && status) atomicOr(&status[b], DQMC_STATUS_NONFINITE_INPUT);
      v = exp(sgn * x);
    }
    out[e] = v;
  }
}

cudaError_t exp_pad(const double* V, double* out, int batch, int M, int Mp, int N, double sgn,
                    int* status, cudaStream_t st, const int* shift) {
  long long total = (long long)batch * Mp * N;
  if (total <= 0) return cudaSuccess;
  exp_pad_kernel<<<nblocks(total), TPB, 0, st>>>(V, out, batch, M, Mp, N, sgn, status, shift);
  return cudaGetLastError();
}

// y[(b / ydiv) * sy_outer + (b % ydiv) * sy + i] = 1 - G_b(i, i)
__global__ void one_minus_diag_kernel(const double* G, long long sG, int N, int batch,
                                      double* y, long long sy, int ydiv, long long sy_outer) {
  const long long total = (long long)N * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / N), i = (int)(e % N);
    double g = G[(long long)b * sG + (long long)i * N + i];
    y[(long long)(b / ydiv) * sy_outer + (long long)(b % ydiv) * sy + i] = 1.0 - g;
  }
}

cudaError_t one_minus_diag(const double* G, long long sG, int N, int batch, double* y,
                           long long sy, int ydiv, long long sy_outer, cudaStream_t st) {
  long long total = (long long)N * batch;
  if (total <= 0) return cudaSuccess;
  one_minus_diag_kernel<<<nblocks(total), TPB, 0, st>>>(G, sG, N, batch, y, sy, ydiv, sy_outer);
  return cudaGetLastError();
}

// one warp per instance: logdet = sum_i log max(D_i, 1) + lad
__global__ void finish_logdet_kernel(const double* D, long long sD, int N, int batch, const double* lad,
                                     const int* s1, const int* s2, double* logdet, int* sign,
                                     int* status, int plain) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int b = w; b < batch; b += nw) {
    double s = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double d = D[(long long)b * sD + i];
      s += log(plain ? d : fmax(d, 1.0));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) {
      double ld = s + (lad ? lad[b] : 0.0);
      if (logdet) logdet[b] = ld;
      int sg = (s1 ? s1[b] : 1) * (s2 ? s2[b] : 1);
      if (sign) sign[b] = sg;
      if (!isfinite(ld) && status) atomicOr(&status[b], DQMC_STATUS_NONFINITE_OUTPUT);
    }
  }
}

cudaError_t finish_logdet(const double* D, long long sD, int N, int batch, const double* lad, const int* s1,
                          const int* s2, double* logdet, int* sign, int* status,
                          cudaStream_t st, int plain) {
  if (batch <= 0) return cudaSuccess;
  int blocks = (batch * 32 + TPB - 1) / TPB;
  if (blocks > 4096) blocks = 4096;
  finish_logdet_kernel<<<blocks, TPB, 0, st>>>(D, sD, N, batch, lad, s1, s2, logdet, sign, status,
                                               plain);
  return cudaGetLastError();
}

__global__ void copy_mats_kernel(const double* in, long long sin, double* out, long long sout,
                                 int N, int batch, int transpose, int divin, int divout) {
  const long long NN = (long long)N * N, total = NN * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / NN);
    long long ij = e % NN;
    int i = (int)(ij / N), j = (int)(ij % N);
    long long src = transpose ? (long long)j * N + i : ij;
    out[(long long)(b / divout) * sout + ij] = in[(long long)(b / divin) * sin + src];
  }
}

cudaError_t copy_mats(const double* in, long long sin, double* out, long long sout, int N,
                      int batch, int transpose, int divin, int divout, cudaStream_t st) {
  long long total = (long long)N * N * batch;
  if (total <= 0) return cudaSuccess;
  copy_mats_kernel<<<nblocks(total), TPB, 0, st>>>(in, sin, out, sout, N, batch, transpose,
                                                   divin, divout);
  return cudaGetLastError();
}

// A_b <- diag(v_b) A_b (row i of instance b scaled by v[b*sv + i]).
__global__ void scale_rows_kernel(double* A, long long sA, const double* v, long long sv, int N,
                                  int batch) {
  const long long NN = (long long)N * N, total = NN * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / NN);
    long long ij = e % NN;
    A[(long long)b * sA + ij] *= v[(long long)b * sv + ij / N];
  }
}

cudaError_t scale_rows(double* A, long long sA, const double* v, long long sv, int N, int batch,
                       cudaStream_t st) {
  long long total = (long long)N * N * batch;
  if (total <= 0) return cudaSuccess;
  scale_rows_kernel<<<nblocks(total), TPB, 0, st>>>(A, sA, v, sv, N, batch);
  return cudaGetLastError();
}

__global__ void set_identity_kernel(double* A, long long sA, int N, int batch) {
  const long long NN = (long long)N * N, total = NN * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int b = (int)(e / NN);
    long long ij = e % NN;
    A[(long long)b * sA + ij] = ((ij / N) == (ij % N)) ? 1.0 : 0.0;
  }
}

cudaError_t set_identity(double* A, long long sA, int N, int batch, cudaStream_t st) {
  long long total = (long long)N * N * batch;
  if (total <= 0) return cudaSuccess;
  set_identity_kernel<<<nblocks(total), TPB, 0, st>>>(A, sA, N, batch);
  return cudaGetLastError();
}

__global__ void set_const_kernel(double* x, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

cudaError_t set_const(double* x, long long n, double v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  set_const_kernel<<<nblocks(n), TPB, 0, st>>>(x, n, v);
  return cudaGetLastError();
}

// One block: ||K||_1 (max column sum), symmetry check, and the scaling
// exponent s with ||dtau K||_1 / 2^s <= 1/2.
__global__ void expm_prepare_kernel(const double* K, int N, double dtau, double sgn, int* s_out,
                                    double* scale_out, int* asym) {
  __shared__ double red[TPB];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  double mx = 0.0;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < N; ++r) {
      double x = K[(long long)r * N + c];
      s += fabs(x);
      if (x != K[(long long)c * N + r] || !isfinite(x)) bad = 1;
    }
    mx = fmax(mx, s);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double nrm = fabs(dtau) * red[0];
    int s = 0;
    while (nrm > 0.5 && s < 60) { nrm *= 0.5; ++s; }
    *s_out = s;
    *scale_out = sgn * dtau * ldexp(1.0, -s);
    *asym = bad || (s > 12);
  }
}

cudaError_t expm_prepare(const double* K, int N, double dtau, double sgn, int* s_out,
                         double* scale_out, int* asym, cudaStream_t st) {
  expm_prepare_kernel<<<1, TPB, 0, st>>>(K, N, dtau, sgn, s_out, scale_out, asym);
  return cudaGetLastError();
}

// Taylor coefficients 1/m! of the degree-16 polynomial, m = 0..16, each the
// correctly rounded reciprocal of m! (exact in FP64 up to 18!).
struct TaylorCoef {
  double c[17];
};

// The whole matrix exponential of a small K (N <= 16) in one CTA, in shared
// memory: the same scaling as expm_prepare, then the degree-16 Taylor
// polynomial p(X) = sum_m X^m / m! of X = scale K by the method of Paterson
// and Stockmeyer (1973) with blocks of four: X^2, then X^3 and X^4 together,
// then p = B_0 + X^4 (B_1 + X^4 (B_2 + X^4 (B_3 + c_16 X^4))) with
// B_q = c_4q I + c_4q+1 X + c_4q+2 X^2 + c_4q+3 X^3 formed entrywise: five
// dependent product steps where a Horner evaluation takes sixteen (the step
// count is what bounds a single small instance).  Then s squarings.  Each
// product entry is one FMA chain over k = 0..N-1.  Replaces ~30 dependent
// launches of tiny products for a single small lattice.
__global__ void expm_small_kernel(const double* K, int N, double dtau, double sgn,
                                  const TaylorCoef cf, int max_sq, double* E, int* asym,
                                  int* status, int batch, int bad_bit) {
  __shared__ double Ks[256], T0[256], T1[256], red[256], P2[256], P3[256], P4[256];
  __shared__ int bad, s_sq;
  __shared__ double s_scale;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  double mx = 0.0;
  for (int c = tid; c < N; c += blockDim.x) {
    double sm = 0.0;
    for (int r = 0; r < N; ++r) {
      const double x = K[(long long)r * N + c];
      sm += fabs(x);
      if (x != K[(long long)c * N + r] || !isfinite(x)) bad = 1;
    }
    mx = fmax(mx, sm);
  }
  red[tid] = mx;
  for (int e = tid; e < N * N; e += blockDim.x) {
    Ks[e] = K[e];
    T0[e] = (e / N == e % N) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (tid < off) red[tid] = fmax(red[tid], red[tid + off]);
    __syncthreads();
  }
  if (tid == 0) {
    double nrm = fabs(dtau) * red[0];
    int sc = 0;
    while (nrm > 0.5 && sc < 60) { nrm *= 0.5; ++sc; }
    s_sq = sc < max_sq ? sc : max_sq;
    s_scale = sgn * dtau * ldexp(1.0, -sc);
    const int flag = bad || (sc > max_sq);
    *asym = flag;
    if (flag && status)
      for (int b = 0; b < batch; ++b) status[b] |= bad_bit;
  }
  __syncthreads();
  const int i = tid / N, j = tid % N;
  const bool own = tid < N * N;
  auto prod = [&](const double* A, const double* B) {
    double acc = 0.0;
    for (int k = 0; k < N; ++k) acc = fma(A[i * N + k], B[k * N + j], acc);
    return acc;
  };
  // B_q at this entry
  auto block = [&](int q) {
    double v = fma(cf.c[4 * q + 3], P3[tid], fma(cf.c[4 * q + 2], P2[tid], cf.c[4 * q + 1] * Ks[tid]));
    if (i == j) v += cf.c[4 * q];
    return v;
  };
  if (own) Ks[tid] *= s_scale;                    // X = scale K, in place
  __syncthreads();
  if (own) P2[tid] = prod(Ks, Ks);
  __syncthreads();
  if (own) {
    P3[tid] = prod(P2, Ks);
    P4[tid] = prod(P2, P2);
  }
  __syncthreads();
  double* cur = T0;
  double* nxt = T1;
  if (own) cur[tid] = fma(cf.c[16], P4[tid], block(3));
  __syncthreads();
  for (int q = 2; q >= 0; --q) {
    if (own) nxt[tid] = prod(P4, cur) + block(q);
    __syncthreads();
    double* t = cur; cur = nxt; nxt = t;
  }
  for (int q = 0; q < s_sq; ++q) {
    if (own) {
      double acc = 0.0;
      for (int k = 0; k < N; ++k) acc = fma(cur[i * N + k], cur[k * N + j], acc);
      nxt[tid] = acc;
    }
    __syncthreads();
    double* t = cur; cur = nxt; nxt = t;
  }
  if (own) E[tid] = cur[tid];
}

cudaError_t expm_small(const double* K, int N, double dtau, double sgn, int terms, int max_sq,
                       double* E, int* asym, int* status, int batch, int bad_bit,
                       cudaStream_t st) {
  if (N > 16 || terms != 16) return cudaErrorInvalidValue;
  TaylorCoef cf;
  double fact = 1.0;   // m!, exact in FP64 for m <= 18
  for (int m = 0; m <= 16; ++m) {
    if (m > 0) fact *= m;
    cf.c[m] = 1.0 / fact;
  }
  expm_small_kernel<<<1, 256, 0, st>>>(K, N, dtau, sgn, cf, max_sq, E, asym, status, batch,
                                       bad_bit);
  return cudaGetLastError();
}

__global__ void or_status_kernel(int* status, int batch, const int* flag, int bit) {
  if (*flag == 0) return;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += gridDim.x * blockDim.x)
    status[b] |= bit;
}

cudaError_t or_status(int* status, int batch, const int* flag, int bit, cudaStream_t st) {
  if (batch <= 0 || !status) return cudaSuccess;
  or_status_kernel<<<nblocks(batch), TPB, 0, st>>>(status, batch, flag, bit);
  return cudaGetLastError();
}

}  // namespace dqmc

namespace dqmc {

// R_q (N x ncols, row-major) = [ diag(1/max(a,1)) U_F^T | diag(min(a,1)) X_F ] (either part optional)
__global__ void build_rhs_kernel(int N, int Q, const double* UF, const double* XF, const double* DF,
                                 double* R, int ncols, int want_tt, int want_t0) {
  const long long NN = (long long)N * N;
  const long long per = (long long)N * ncols;
  const long long total = per * Q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long q = e / per, rc = e % per;
    int r = (int)(rc / ncols), c = (int)(rc % ncols);
    double a = DF[q * N + r];
    double v;
    if (want_tt && c < N) {
      v = UF[q * NN + (long long)c * N + r] / fmax(a, 1.0);
    } else {
      int cc = want_tt ? c - N : c;
      v = XF[q * NN + (long long)r * N + cc] * fmin(a, 1.0);
    }
    R[e] = v;
  }
}

cudaError_t build_rhs(int N, int Q, const double* UF, const double* XF, const double* DF, double* R,
                      int ncols, int want_tt, int want_t0, cudaStream_t st) {
  long long total = (long long)N * ncols * Q;
  if (total <= 0) return cudaSuccess;
  build_rhs_kernel<<<nblocks(total), TPB, 0, st>>>(N, Q, UF, XF, DF, R, ncols, want_tt, want_t0);
  return cudaGetLastError();
}

// dV[(b*M + l-1)*N + i] = 1 - G_q(i,i), q = b*nt + j, l = j*k + s + 1, for j < nt-1, l <= M
__global__ void grad_readout_kernel(const double* G, int N, int Q, int nt, int k, int M, int s,
                                    double* dV) {
  const long long total = (long long)N * Q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int q = (int)(e / N), i = (int)(e % N);
    int b = q / nt, j = q % nt;
    int l = j * k + s + 1;
    if (j >= nt - 1 || l > M) continue;
    dV[((long long)b * M + (l - 1)) * N + i] = 1.0 - G[(long long)q * N * N + (long long)i * N + i];
  }
}

cudaError_t grad_readout(const double* G, int N, int Q, int nt, int k, int M, int s, double* dV,
                         cudaStream_t st) {
  long long total = (long long)N * Q;
  if (total <= 0) return cudaSuccess;
  grad_readout_kernel<<<nblocks(total), TPB, 0, st>>>(G, N, Q, nt, k, M, s, dV);
  return cudaGetLastError();
}

// x[b*sx + i] = v for i < n
__global__ void set_const_strided_kernel(double* x, long long sx, int n, int batch, double v) {
  const long long total = (long long)n * batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    x[(e / n) * sx + e % n] = v;
}

cudaError_t set_const_strided(double* x, long long sx, int n, int batch, double v, cudaStream_t st) {
  long long total = (long long)n * batch;
  if (total <= 0) return cudaSuccess;
  set_const_strided_kernel<<<nblocks(total), TPB, 0, st>>>(x, sx, n, batch, v);
  return cudaGetLastError();
}

}  // namespace dqmc
