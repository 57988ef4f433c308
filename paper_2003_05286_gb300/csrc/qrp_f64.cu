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

// ties -> lowest index
__device__ __forceinline__ void warp_argmax(float& key, int& idx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float k2 = __shfl_down_sync(0xffffffffu, key, off);
    int i2 = __shfl_down_sync(0xffffffffu, idx, off);
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
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

// Strided column kernels shared by the QR steps.  One thread walks a column of
// a row-major matrix (stride ld); loads are issued 8 at a time and the next
// batch is loaded before the current one is stored, so that a thread keeps
// 8-16 L2 requests in flight instead of one (the compiler cannot reorder a
// load above a store to the same array on its own).
// dot = sum_{r=r0}^{n-1} v[r] * col[r*ld]
__device__ __forceinline__ double col_dot(const double* __restrict__ col, long long ld,
                                          const double* __restrict__ v, int r0, int n) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int r = r0;
  for (; r + 7 < n; r += 8) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = col[(long long)(r + i) * ld];
    a0 = fma(v[r + 0], x[0], a0); a1 = fma(v[r + 1], x[1], a1);
    a2 = fma(v[r + 2], x[2], a2); a3 = fma(v[r + 3], x[3], a3);
    a0 = fma(v[r + 4], x[4], a0); a1 = fma(v[r + 5], x[5], a1);
    a2 = fma(v[r + 6], x[6], a2); a3 = fma(v[r + 7], x[7], a3);
  }
  for (; r < n; ++r) a0 = fma(v[r], col[(long long)r * ld], a0);
  return (a0 + a1) + (a2 + a3);
}

// col[r*ld] -= v[r] * w  for r in [r0, n)
__device__ __forceinline__ void col_axpy(double* __restrict__ col, long long ld,
                                         const double* __restrict__ v, double w, int r0, int n) {
  int r = r0;
  if (r + 7 < n) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = col[(long long)(r + i) * ld];
    for (; r + 15 < n; r += 8) {
      double y[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) y[i] = col[(long long)(r + 8 + i) * ld];
#pragma unroll
      for (int i = 0; i < 8; ++i) col[(long long)(r + i) * ld] = fma(-v[r + i], w, x[i]);
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = y[i];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) col[(long long)(r + i) * ld] = fma(-v[r + i], w, x[i]);
    r += 8;
  }
  for (; r < n; ++r) col[(long long)r * ld] = fma(-v[r], w, col[(long long)r * ld]);
}

// sum_{r=r0}^{n-1} col[r*ld]^2
__device__ __forceinline__ double col_sumsq(const double* __restrict__ col, long long ld, int r0,
                                            int n) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int r = r0;
  for (; r + 7 < n; r += 8) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = col[(long long)(r + i) * ld];
    a0 = fma(x[0], x[0], a0); a1 = fma(x[1], x[1], a1);
    a2 = fma(x[2], x[2], a2); a3 = fma(x[3], x[3], a3);
    a0 = fma(x[4], x[4], a0); a1 = fma(x[5], x[5], a1);
    a2 = fma(x[6], x[6], a2); a3 = fma(x[7], x[7], a3);
  }
  for (; r < n; ++r) { double x = col[(long long)r * ld]; a0 = fma(x, x, a0); }
  return (a0 + a1) + (a2 + a3);
}

}  // namespace

template <int NT>
__global__ void __launch_bounds__(NT) qrp_kernel(const QrpArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N;
  // per column c (in pivoted order): squared norm, reference value of the
  // recompute test, column scale Din and its log2, original column index
  double* nrm2 = reinterpret_cast<double*>(smem_raw);
  double* ref2 = nrm2 + N;
  double* vbuf = ref2 + N;                              // reflector (factorisation) / double buffer (Q)
  double* vbuf2 = vbuf + N;
  double* taus = vbuf2 + N;
  double* dsc = taus + N;
  float* logd = reinterpret_cast<float*>(dsc + N);
  int* perm = reinterpret_cast<int*>(logd + N);
  __shared__ float sk[NT / 32];
  __shared__ int si[NT / 32];
  __shared__ double sd[NT / 32];
  __shared__ double s_alpha;
  __shared__ int s_flag;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int RPT = 4;   // rows below the diagonal per thread in the reflector pass (N <= 4 NT)

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    if (a.lim && a.lim[b] < a.lim_at) continue;   // chain of this instance already finished
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    double* __restrict__ W = a.W + (long long)b * a.sW;
    double* __restrict__ U = a.U + (long long)b * a.sU;
    double* __restrict__ Dout = a.D + (long long)b * a.sD;
    double* __restrict__ T = a.T + (long long)b * a.sT;   // holds v_j (row j) until the end
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
    {
      float key = -INFINITY;
      int idx = 0x7fffffff;
      for (int c = tid; c < N; c += NT) {
        double s0 = col_sumsq(W + c, N, 0, N);
        nrm2[c] = s0;
        ref2[c] = s0;
        float kc = logd[c] + 0.5f * log2_wide(s0);
        if (kc > key || (kc == key && c < idx)) { key = kc; idx = c; }
      }
      warp_argmax(key, idx);
      if (lane == 0) { sk[wid] = key; si[wid] = idx; }
    }
    __syncthreads();

    for (int j = 0; j < N; ++j) {
      // ---- pivot: reduce the per-warp candidates (every thread, same order)
      float key = sk[0];
      int idx = si[0];
      for (int w = 1; w < NT / 32; ++w) {
        if (sk[w] > key || (sk[w] == key && si[w] < idx)) { key = sk[w]; idx = si[w]; }
      }
      const int p = (idx >= j && idx < N) ? idx : j;
      // ---- swap columns j and p; the thread that swaps a row below j keeps
      // the pivot column's entry for the reflector -------------------------
      double x[RPT];
      double part = 0.0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = j + 1 + tid + q * NT;
        x[q] = 0.0;
        if (r < N) {
          double* row = W + (long long)r * N;
          const double xp = row[p];
          if (p != j) { row[p] = row[j]; row[j] = xp; }
          x[q] = xp;
          part = fma(xp, xp, part);
        }
      }
      for (int r = tid; r <= j; r += NT) {   // rows 0..j (R part and the diagonal row)
        double* row = W + (long long)r * N;
        const double xp = row[p];
        if (p != j) { row[p] = row[j]; row[j] = xp; }
        if (r == j) s_alpha = xp;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
      if (lane == 0) sd[wid] = part;
      __syncthreads();
      // ---- reflector ------------------------------------------------------
      double sigma = 0.0;
      for (int w = 0; w < NT / 32; ++w) sigma += sd[w];
      const double alpha = s_alpha;
      double tau = 0.0, scal = 0.0, beta = alpha;
      if (sigma > 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, sigma));
        beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      if (tid == 0) {
        if (p != j) {
          double t;
          t = nrm2[j]; nrm2[j] = nrm2[p]; nrm2[p] = t;
          t = ref2[j]; ref2[j] = ref2[p]; ref2[p] = t;
          t = dsc[j]; dsc[j] = dsc[p]; dsc[p] = t;
          float f = logd[j]; logd[j] = logd[p]; logd[p] = f;
          int q = perm[j]; perm[j] = perm[p]; perm[p] = q;
        }
        W[(long long)j * N + j] = beta;
        taus[j] = tau;
        T[(long long)j * N + j] = 1.0;
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = j + 1 + tid + q * NT;
        if (r < N) {
          const double v = x[q] * scal;
          vbuf[r] = v;
          T[(long long)j * N + r] = v;   // v_j stored contiguously for forming Q
        }
      }
      __syncthreads();

      // ---- apply to the trailing columns, downdate, next pivot candidates --
      key = -INFINITY;
      idx = 0x7fffffff;
      for (int c = j + 1 + tid; c < N; c += NT) {
        double* col = W + c;
        double rjc = col[(long long)j * N];
        if (tau != 0.0) {
          const double w = (rjc + col_dot(col, N, vbuf, j + 1, N)) * tau;
          rjc -= w;
          col[(long long)j * N] = rjc;
          col_axpy(col, N, vbuf, w, j + 1, N);
        }
        double n2 = fma(-rjc, rjc, nrm2[c]);
        if (n2 <= 1.4901161193847656e-8 * ref2[c]) {
          n2 = col_sumsq(col, N, j + 1, N);
          ref2[c] = n2;
        }
        nrm2[c] = n2;
        float kc = logd[c] + 0.5f * log2_wide(n2);
        if (kc > key || (kc == key && c < idx)) { key = kc; idx = c; }
      }
      warp_argmax(key, idx);
      if (lane == 0) { sk[wid] = key; si[wid] = idx; }
      __syncthreads();
    }

    // ---- U = Q = H_0 H_1 ... H_{N-1}, backward accumulation --------------
    // One barrier per reflector: while step j applies v_j (from one buffer),
    // the threads also stage v_{j-1} into the other.
    for (long long e = tid; e < (long long)N * N; e += NT) {
      int i = (int)(e / N), c = (int)(e % N);
      U[e] = (i == c) ? 1.0 : 0.0;
    }
    for (int r = N - 1 + tid; r < N; r += NT) vbuf[r] = T[(long long)(N - 1) * N + r];
    __syncthreads();
    for (int j = N - 1; j >= 0; --j) {
      double* cur = ((N - 1 - j) & 1) ? vbuf2 : vbuf;
      double* nxt = ((N - 1 - j) & 1) ? vbuf : vbuf2;
      if (j > 0)
        for (int r = j - 1 + tid; r < N; r += NT) nxt[r] = T[(long long)(j - 1) * N + r];
      const double tau = taus[j];
      if (tau != 0.0) {
        for (int c = j + tid; c < N; c += NT) {
          double* col = U + c;
          const double w = col_dot(col, N, cur, j, N) * tau;
          col_axpy(col, N, cur, w, j, N);
        }
      }
      __syncthreads();
    }

    // ---- outputs D, T, perm (T overwrites the stored reflectors) ---------
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
    __syncthreads();
    if (tid == 0 && s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
    __syncthreads();
  }
}

static size_t qrp_smem(int N) { return (size_t)N * (6 * sizeof(double) + sizeof(float) + sizeof(int)) + 16; }

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
