// Column-pivoted Householder QR written as U D T (Sec. 4.2.2, "QR (UDT)"),
// one CTA per instance.
//
// The input is Y = A diag(Din): the chunk product A = B_chunk U_1 and the
// scales D_1 of the running decomposition (Eq. (stabmult): (X_2 U_1) D_1 with
// X_2 the chunk).  Left Householder reflections commute with the column
// scaling, so the factorisation runs on A itself and Din enters only through
// the pivot choice (largest D_c * ||a_c||) and the output scales.  This keeps
// every squared quantity free of the e^{+-700} range that D can reach.
//
// Per step j (N steps, sequential -- the latency-bound part of the method):
//   pivot    argmax_c  log2 Din_c + 0.5 log2 ||a_c^{(j)}||^2 over c >= j,
//            evaluated in FP32 from the exponent bits (no FP64 pipe time);
//            ties go to the lowest index, as in LAPACK.
//   reflect  Householder vector of column j (fresh FP64 norm of the column).
//   update   trailing columns c > j, one thread per column, rows streamed
//            from the L2-resident row-major workspace (coalesced across c).
//   downdate ||a_c||^2 -= r_jc^2; recomputed from the column when it has lost
//            more than half of its digits (||.||^2 <= sqrt(eps) * reference),
//            the safeguard of LAPACK's xLAQP2 (Drmac & Bujanovic 2008).
// Q is then formed explicitly by backward accumulation of the reflectors.
// Outputs: U = Q, D_i = |r_ii| Din_{p_i}, T = D^{-1} R (pivoted column order,
// zeros below the diagonal), perm_i = p_i.
#include "common.cuh"

namespace dqmc {

namespace {

// log2 of a positive double as a float, from its exponent bits (exact to
// float rounding of the mantissa part).  0 maps to -inf.
__device__ __forceinline__ float log2_wide(double x) {
  if (!(x > 0.0)) return -INFINITY;
  unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ff);
  if (e == 0) return -1074.0f;   // denormal: below every normal scale
  float m = __int_as_float(0x3f800000 | (int)((bits >> 29) & 0x7fffff));   // [1, 2)
  return (float)(e - 1023) + __log2f(m);
}

template <int NT>
__device__ __forceinline__ void block_argmax(float& key, int& idx, float* sk, int* si) {
  // ties -> lowest index
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float k2 = __shfl_down_sync(0xffffffffu, key, off);
    int i2 = __shfl_down_sync(0xffffffffu, idx, off);
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sk[wid] = key; si[wid] = idx; }
  __syncthreads();
  if (wid == 0) {
    key = lane < NT / 32 ? sk[lane] : -INFINITY;
    idx = lane < NT / 32 ? si[lane] : 0x7fffffff;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      float k2 = __shfl_down_sync(0xffffffffu, key, off);
      int i2 = __shfl_down_sync(0xffffffffu, idx, off);
      if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
    }
    if (lane == 0) { sk[0] = key; si[0] = idx; }
  }
  __syncthreads();
  key = sk[0];
  idx = si[0];
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sd) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sd[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < NT / 32 ? sd[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sd[0] = v;
  }
  __syncthreads();
  v = sd[0];
  return v;
}

}  // namespace

template <int NT>
__global__ void __launch_bounds__(NT) qrp_kernel(const QrpArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N;
  double* nrm2 = reinterpret_cast<double*>(smem_raw);   // ||a_c^{(j)}||^2 (unscaled)
  double* ref2 = nrm2 + N;                              // value at the last recompute
  double* vbuf = ref2 + N;                              // Householder vector
  double* taus = vbuf + N;                              // tau_j
  double* dsc = taus + N;                               // Din, permuted with the columns
  float* logd = reinterpret_cast<float*>(dsc + N);      // log2 Din
  int* perm = reinterpret_cast<int*>(logd + N);
  __shared__ float sk[32];
  __shared__ int si[32];
  __shared__ double sd[32];
  __shared__ double s_tau, s_scal;
  __shared__ int s_flag;

  const int tid = threadIdx.x;

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    if (a.active && !a.active[b]) continue;
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    double* __restrict__ W = a.W + (long long)b * a.sW;
    double* __restrict__ U = a.U + (long long)b * a.sU;
    double* __restrict__ Dout = a.D + (long long)b * a.sD;
    double* __restrict__ T = a.T + (long long)b * a.sT;
    int* __restrict__ pout = a.perm + (long long)b * a.sperm;
    const double* Din = a.Din ? a.Din + (long long)b * a.sDin : nullptr;

    if (tid == 0) s_flag = 0;
    __syncthreads();
    int bad = 0;
    for (long long e = tid; e < (long long)N * N; e += NT) {
      double v = A[e];
      bad |= !isfinite(v);
      W[e] = v;
    }
    for (int c = tid; c < N; c += NT) {
      double d = Din ? Din[c] : 1.0;
      bad |= !(isfinite(d) && d >= 0.0);
      dsc[c] = d;
      logd[c] = log2_wide(d);
      perm[c] = c;
    }
    if (bad) atomicOr(&s_flag, DQMC_STATUS_NONFINITE_SCALE);
    __syncthreads();
    for (int c = tid; c < N; c += NT) {
      double s0 = 0.0, s1 = 0.0;
      int r = 0;
      for (; r + 1 < N; r += 2) {
        double x0 = W[(long long)r * N + c], x1 = W[(long long)(r + 1) * N + c];
        s0 = fma(x0, x0, s0);
        s1 = fma(x1, x1, s1);
      }
      if (r < N) { double x0 = W[(long long)r * N + c]; s0 = fma(x0, x0, s0); }
      nrm2[c] = s0 + s1;
      ref2[c] = s0 + s1;
    }
    __syncthreads();

    for (int j = 0; j < N; ++j) {
      // ---- pivot -------------------------------------------------------
      float key = -INFINITY;
      int idx = 0x7fffffff;
      for (int c = j + tid; c < N; c += NT) {
        float kc = logd[c] + 0.5f * log2_wide(nrm2[c]);
        if (kc > key || (kc == key && c < idx)) { key = kc; idx = c; }
      }
      block_argmax<NT>(key, idx, sk, si);
      int p = (idx >= j && idx < N) ? idx : j;
      if (p != j) {
        for (int r = tid; r < N; r += NT) {
          double t0 = W[(long long)r * N + j];
          W[(long long)r * N + j] = W[(long long)r * N + p];
          W[(long long)r * N + p] = t0;
        }
        if (tid == 0) {
          double t;
          t = nrm2[j]; nrm2[j] = nrm2[p]; nrm2[p] = t;
          t = ref2[j]; ref2[j] = ref2[p]; ref2[p] = t;
          t = dsc[j]; dsc[j] = dsc[p]; dsc[p] = t;
          float f = logd[j]; logd[j] = logd[p]; logd[p] = f;
          int q = perm[j]; perm[j] = perm[p]; perm[p] = q;
        }
      }
      __syncthreads();

      // ---- Householder reflector of column j ---------------------------
      double part = 0.0;
      for (int r = j + 1 + tid; r < N; r += NT) {
        double x = W[(long long)r * N + j];
        part = fma(x, x, part);
      }
      double sigma = block_sum<NT>(part, sd);
      if (tid == 0) {
        double alpha = W[(long long)j * N + j];
        double tau = 0.0, scal = 0.0, beta = alpha;
        if (sigma > 0.0) {
          double nrm = sqrt(fma(alpha, alpha, sigma));
          beta = alpha >= 0.0 ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        W[(long long)j * N + j] = beta;
        taus[j] = tau;
        s_tau = tau;
        s_scal = scal;
      }
      __syncthreads();
      const double tau = s_tau, scal = s_scal;
      for (int r = j + 1 + tid; r < N; r += NT) {
        double v = W[(long long)r * N + j] * scal;
        vbuf[r] = v;
        W[(long long)r * N + j] = v;
      }
      __syncthreads();

      // ---- apply to the trailing columns and downdate their norms --------
      if (tau != 0.0) {
        for (int c = j + 1 + tid; c < N; c += NT) {
          double* col = W + c;
          double w0 = col[(long long)j * N], w1 = 0.0;
          int r = j + 1;
          for (; r + 3 < N; r += 4) {
            w0 = fma(vbuf[r], col[(long long)r * N], w0);
            w1 = fma(vbuf[r + 1], col[(long long)(r + 1) * N], w1);
            w0 = fma(vbuf[r + 2], col[(long long)(r + 2) * N], w0);
            w1 = fma(vbuf[r + 3], col[(long long)(r + 3) * N], w1);
          }
          for (; r < N; ++r) w0 = fma(vbuf[r], col[(long long)r * N], w0);
          const double w = (w0 + w1) * tau;
          const double rjc = col[(long long)j * N] - w;
          col[(long long)j * N] = rjc;
          for (r = j + 1; r < N; ++r) col[(long long)r * N] = fma(-vbuf[r], w, col[(long long)r * N]);
          double n2 = fma(-rjc, rjc, nrm2[c]);
          if (n2 <= 1.4901161193847656e-8 * ref2[c]) {
            double s0 = 0.0;
            for (r = j + 1; r < N; ++r) { double x = col[(long long)r * N]; s0 = fma(x, x, s0); }
            n2 = s0;
            ref2[c] = s0;
          }
          nrm2[c] = n2;
        }
      } else {
        for (int c = j + 1 + tid; c < N; c += NT) {
          double rjc = W[(long long)j * N + c];
          double n2 = fma(-rjc, rjc, nrm2[c]);
          if (n2 <= 1.4901161193847656e-8 * ref2[c]) {
            double s0 = 0.0;
            for (int r = j + 1; r < N; ++r) { double x = W[(long long)r * N + c]; s0 = fma(x, x, s0); }
            n2 = s0;
            ref2[c] = s0;
          }
          nrm2[c] = n2;
        }
      }
      __syncthreads();
    }

    // ---- outputs D, T, perm ----------------------------------------------
    // reuse nrm2 as 1/|r_ii| and ref2 as 1/Din_i
    for (int i = tid; i < N; i += NT) {
      double rii = fabs(W[(long long)i * N + i]);
      double d = rii * dsc[i];
      if (!(d > 0.0)) atomicOr(&s_flag, DQMC_STATUS_SINGULAR);
      if (!isfinite(d)) atomicOr(&s_flag, DQMC_STATUS_NONFINITE_SCALE);
      Dout[i] = d;
      nrm2[i] = rii > 0.0 ? 1.0 / rii : 0.0;
      ref2[i] = dsc[i] > 0.0 ? 1.0 / dsc[i] : 0.0;
      pout[i] = perm[i];
    }
    __syncthreads();
    for (long long e = tid; e < (long long)N * N; e += NT) {
      int i = (int)(e / N), c = (int)(e % N);
      double v = 0.0;
      if (c >= i) v = W[e] * nrm2[i] * (dsc[c] * ref2[i]);
      T[e] = v;
    }

    // ---- U = Q = H_0 H_1 ... H_{N-1}, backward accumulation --------------
    for (long long e = tid; e < (long long)N * N; e += NT) {
      int i = (int)(e / N), c = (int)(e % N);
      U[e] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = N - 1; j >= 0; --j) {
      const double tau = taus[j];
      if (tau == 0.0) continue;   // uniform across the block
      for (int r = j + tid; r < N; r += NT) vbuf[r] = (r == j) ? 1.0 : W[(long long)r * N + j];
      __syncthreads();
      for (int c = j + tid; c < N; c += NT) {
        double* col = U + c;
        double w0 = 0.0, w1 = 0.0;
        int r = j;
        for (; r + 1 < N; r += 2) {
          w0 = fma(vbuf[r], col[(long long)r * N], w0);
          w1 = fma(vbuf[r + 1], col[(long long)(r + 1) * N], w1);
        }
        if (r < N) w0 = fma(vbuf[r], col[(long long)r * N], w0);
        const double w = (w0 + w1) * tau;
        for (r = j; r < N; ++r) col[(long long)r * N] = fma(-vbuf[r], w, col[(long long)r * N]);
      }
      __syncthreads();
    }
    if (tid == 0 && s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
    __syncthreads();
  }
}

static size_t qrp_smem(int N) { return (size_t)N * (5 * sizeof(double) + sizeof(float) + sizeof(int)) + 16; }

cudaError_t qrp_f64(const QrpArgs& a, cudaStream_t st) {
  if (a.batch <= 0 || a.N <= 0) return cudaSuccess;
  size_t sm = qrp_smem(a.N);
  int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  if (a.N <= 32) {
    cudaFuncSetAttribute(qrp_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    qrp_kernel<32><<<grid, 32, sm, st>>>(a);
  } else if (a.N <= 128) {
    cudaFuncSetAttribute(qrp_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    qrp_kernel<128><<<grid, 128, sm, st>>>(a);
  } else {
    cudaFuncSetAttribute(qrp_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    qrp_kernel<256><<<grid, 256, sm, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dqmc
