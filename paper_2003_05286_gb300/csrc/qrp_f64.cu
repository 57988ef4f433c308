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
//
// Two kernels compute this: qrp_fused_kernel (N <= 256, one pass over the
// trailing matrix per step) and qrp_kernel (any N, two passes per step).
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
  // launch contract (debug build): NT threads, rows of the reflector pass
  // covered, the six double, one float and one int arrays of N in shared memory
  if (!DQMC_CHECK(blockDim.x == NT && N <= RPT * NT, N) ||
      !DQMC_CHECK(dyn_smem_bytes() >= (unsigned)N * 56u, dyn_smem_bytes()))
    return;

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

// ---------------------------------------------------------------------------
// Fused variant for N <= 256: TPC threads per column, one pass per step.
//
// The kernel above needs two passes over the trailing matrix per step (the
// dot products v_j^T a_c, then the rank-1 update), each a chain of dependent
// L2 round trips for the thread that walks a column.  Here a step is a single
// pass: while column c is updated with the reflector of step j, the same
// loaded values are dotted with the reflector of step j+1.  That reflector is
// known before the pass because the next pivot only needs the downdated norms,
// and those only need r_jc = a_jc - w_c (v_j has a unit leading entry), not
// the updated column.  Per step:
//   (a) every column: w_c = tau_j d_c, r_jc, norm downdate, pivot key, vote;
//   (b) one warp: the pivot column's updated entries (a_P - v_j w_P), the
//       reflector v_{j+1}, the swap of columns j+1 and P, R entries of the
//       pivot column;
//   (c) every trailing column: a_c -= v_j w_c and d_c = v_{j+1}^T a_c.
// Two block barriers per step.  TPC threads of a column sit in one warp
// (lane = column + CPW * row group), so a load instruction of the warp reads
// TPC rows x CPW consecutive doubles, and the per-column scalars (w, norms,
// keys) are vector instructions over the warp's columns.  Q is accumulated
// backwards with the same fused pass (update with v_j, dot with v_{j-1}).
// ---------------------------------------------------------------------------
namespace {

// rows r0, r0 + TPC, ... < N of column c of the row-major M (leading dimension
// N): x_r -= va[r] w (stored if store), returns sum vb[r] x_r over the updated
// values and sets xpick to the updated value of row rpick if this thread has
// it.  Loads run one batch of B rows ahead of the stores.
//
// Every FP64 warp instruction holds the sub-partition's FP64 pipe for 64
// cycles on this part whether or not its lanes are predicated off, so the
// full batches carry no row guards and the last n mod B rows are processed in
// unguarded blocks of 4, 2 and 1 (register shifts keep the indices static)
// instead of B guarded slots.
template <int TPC>
__device__ __forceinline__ void fused_row(double* __restrict__ M, int N, int c, int r,
                                          const double* va, double w, const double* vb, int rpick,
                                          double& xpick, bool store, double xv, double& acc) {
  const double x = fma(-va[r], w, xv);
  if (store) M[(long long)r * N + c] = x;
  acc = fma(vb[r], x, acc);
  if (r == rpick) xpick = x;
}

template <int TPC, int B>
__device__ __forceinline__ double fused_pass(double* __restrict__ M, int N, int c, int r0,
                                             const double* va, double w, const double* vb,
                                             int rpick, double& xpick, bool store) {
  static_assert(B == 8, "the tail decomposition assumes batches of 8 rows");
  const int n = r0 < N ? (N - r0 + TPC - 1) / TPC : 0;
  const int nfull = n - n % B;
  double acc0 = 0.0, acc1 = 0.0;
  double xc[B];
#pragma unroll
  for (int k = 0; k < B; ++k) xc[k] = k < n ? M[(long long)(r0 + k * TPC) * N + c] : 0.0;
  int i = 0;
  for (; i < nfull; i += B) {
    double xn[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int t = i + B + k;
      xn[k] = t < n ? M[(long long)(r0 + t * TPC) * N + c] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < B; ++k)
      fused_row<TPC>(M, N, c, r0 + (i + k) * TPC, va, w, vb, rpick, xpick, store, xc[k],
                     (k & 1) ? acc1 : acc0);
#pragma unroll
    for (int k = 0; k < B; ++k) xc[k] = xn[k];
  }
  // tail: rows i .. n-1 (fewer than B), already loaded into xc[0 ..]
  const int rem = n - i;
  if (rem & 4) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      fused_row<TPC>(M, N, c, r0 + (i + k) * TPC, va, w, vb, rpick, xpick, store, xc[k],
                     (k & 1) ? acc1 : acc0);
#pragma unroll
    for (int k = 0; k < 4; ++k) xc[k] = xc[k + 4];
    i += 4;
  }
  if (rem & 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
      fused_row<TPC>(M, N, c, r0 + (i + k) * TPC, va, w, vb, rpick, xpick, store, xc[k],
                     (k & 1) ? acc1 : acc0);
    xc[0] = xc[2];
    i += 2;
  }
  if (rem & 1) fused_row<TPC>(M, N, c, r0 + i * TPC, va, w, vb, rpick, xpick, store, xc[0], acc0);
  return acc0 + acc1;
}

__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// ties -> lowest index; every lane ends with the same pair
__device__ __forceinline__ void warp_argmax_all(float& key, int& idx) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float k2 = __shfl_xor_sync(0xffffffffu, key, off);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
}

// sum over the TPC threads of a column (lanes l, l + CPW, ...)
template <int TPC>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int off = 16; off >= 32 / TPC; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace

// MINB = 2 holds the 512-thread instance (N <= 256) to 64 registers, so that
// one QR CTA and one 256-thread FP64 GEMM CTA fit an SM together: the
// pipelined FP64 chain runs the QR of one sub-batch beside the products of
// another, and the QR leaves part of its SM's FP64 pipe idle.  The register
// cap costs the QR a few spills, so chains whose step is bound by the QR's
// latency (the tensor-core chain) take MINB = 0: no minimum, the compiler's
// own register choice (an explicit minimum of 1 lets it take ~200 registers
// in the 128- and 256-thread instances and costs them resident CTAs).
template <int NT, int TPC, int NQ, int MINB = 0>
__global__ void __launch_bounds__(NT, MINB) qrp_fused_kernel(const QrpArgs a) {
  constexpr int NW = NT / 32, CPW = 32 / TPC, BATCH = 8;
  // warps of the reflector step and rows per lane each
  constexpr int NR = (NQ >= 4 && NW >= 4) ? 4 : 1, KQ = NQ / NR;
  static_assert(NQ % NR == 0, "rows of the reflector must split evenly");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N;
  // a.smem_mats: 0 = W and U in global memory, 1 = W in shared memory,
  // 2 = W and U in shared memory (U copied out at the end).  The kernel reads
  // both through plain pointers, so only where they point changes.
  const long long NNs = (long long)N * N;
  double* smW = reinterpret_cast<double*>(smem_raw);
  double* smU = smW + (a.smem_mats >= 1 ? NNs : 0);
  // per column in pivoted (logical) order; swapped together with the columns
  double* nrm2 = smW + a.smem_mats * NNs;
  double* ref2 = nrm2 + N;
  double* dsc = ref2 + N;
  double* wsm = dsc + N;     // w_c of the current step
  double* taus = wsm + N;
  double* vA = taus + N;     // reflector buffers: v_j and v_{j+1} (rotating)
  double* vB = vA + N;
  float* logd = reinterpret_cast<float*>(vB + N);
  int* perm = reinterpret_cast<int*>(logd + N);
  __shared__ float sk[NW];
  __shared__ int si[NW];
  __shared__ int s_flag;
  __shared__ double s_red[5];                  // partial sums of the reflector step, alpha

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // launch contract (debug build): NT threads, every column owned by one
  // thread group, every row by one lane of the reflector warps, and shared
  // memory for the resident matrices plus seven double, one float and one
  // int array of N
  if (!DQMC_CHECK(blockDim.x == NT && N <= NW * CPW && N <= 32 * NQ, N) ||
      !DQMC_CHECK(dyn_smem_bytes() >= (unsigned)(a.smem_mats * NNs * 8 + 64LL * N),
                  dyn_smem_bytes()))
    return;
  const int rg = lane / CPW;                   // row group: rows r = rg (mod TPC)
  const int c = wid * CPW + lane % CPW;        // this thread's column
  const bool own = c < N;
  const unsigned FULL = 0xffffffffu;

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    if (a.lim && a.lim[b] < a.lim_at) continue;   // chain of this instance already finished
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    double* __restrict__ W = a.smem_mats >= 1 ? smW : a.W + (long long)b * a.sW;
    double* __restrict__ Uout = a.U + (long long)b * a.sU;
    double* __restrict__ U = a.smem_mats >= 2 ? smU : Uout;
    double* __restrict__ Dout = a.D + (long long)b * a.sD;
    double* __restrict__ T = a.T + (long long)b * a.sT;   // v_j in row j until the end
    int* __restrict__ pout = a.perm + (long long)b * a.sperm;
    const double* Din = a.Din ? a.Din + (long long)b * a.sDin : nullptr;
    const long long NN = (long long)N * N;

    if (tid == 0) s_flag = 0;
    int bad = 0;
    for (long long e = tid; e < NN; e += NT) {
      const double v = A[e];
      bad |= !isfinite(v);
      W[e] = v;
    }
    for (int cc = tid; cc < N; cc += NT) {
      const double d = Din ? Din[cc] : 1.0;
      bad |= !(isfinite(d) && d >= 0.0);
      dsc[cc] = d;
      logd[cc] = log2_wide(d);
      perm[cc] = cc;
    }
    __syncthreads();
    if (bad) atomicOr(&s_flag, DQMC_STATUS_NONFINITE_SCALE);

    // ---- vote: argmax of the keys (ties -> lowest column), then warp 0 forms
    // the reflector for position jn from column P -------------------------
    double* vcur = vA;   // v_j
    double* vnxt = vB;   // v_{j+1}
    // The reflector's vector work (update of the pivot column, its sum of
    // squares, the scaling, the stores) is spread over NR warps, one per SM
    // sub-partition: each FP64 warp instruction holds its sub-partition's
    // pipe for 64 cycles, and this step is on every pivot step's critical
    // path.  Warp w owns rows lane + 32 (w + NR k).  The partial sums meet in
    // shared memory behind a named barrier of those NR warps and every one of
    // them forms the same scalars in the same order.
    auto vote_and_reflect = [&](float key, int idx, int jn) {
      warp_argmax(key, idx);
      if (lane == 0) { sk[wid] = key; si[wid] = idx; }
      __syncthreads();
      if (wid < NR) {
        key = lane < NW ? sk[lane] : -INFINITY;
        idx = lane < NW ? si[lane] : 0x7fffffff;
        warp_argmax_all(key, idx);
        const int P = (idx >= jn && idx < N) ? idx : jn;
        const int j = jn - 1;
        const bool upd = j >= 0;
        const double wP = upd ? wsm[P] : 0.0;
        double xp[KQ], xo[KQ];
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
          const int r = lane + 32 * (wid + NR * k);
          xp[k] = r < N ? W[(long long)r * N + P] : 0.0;
          xo[k] = (r < N && P != jn) ? W[(long long)r * N + jn] : 0.0;
        }
        double sig = 0.0, alpha = 0.0;
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
          const int r = lane + 32 * (wid + NR * k);
          if (upd && r >= j && r < N) xp[k] = fma(-vcur[r], wP, xp[k]);
          if (r == jn) alpha = xp[k];
          if (r > jn && r < N) sig = fma(xp[k], xp[k], sig);
        }
        sig = warp_sum_all(sig);
        if (NR == 1) {
          alpha = __shfl_sync(FULL, alpha, jn & 31);
        } else {
          if (lane == 0) s_red[wid] = sig;
          if (((jn >> 5) % NR) == wid && lane == (jn & 31)) s_red[NR] = alpha;
          asm volatile("bar.sync 1, %0;" ::"r"(NR * 32) : "memory");
          sig = (s_red[0] + s_red[1]) + (s_red[2] + s_red[3]);
          alpha = s_red[NR];
        }
        double tau = 0.0, scal = 0.0, beta = alpha;
        if (sig > 0.0) {
          const double nrm = sqrt(fma(alpha, alpha, sig));
          beta = alpha >= 0.0 ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
          const int r = lane + 32 * (wid + NR * k);
          if (r < N) {
            // column jn <- pivot column: R rows (final above j, updated at j), beta
            if (r < j) { if (P != jn) W[(long long)r * N + jn] = xp[k]; }
            else if (r == j) W[(long long)r * N + jn] = xp[k];
            else if (r == jn) W[(long long)r * N + jn] = beta;
            // column P <- old column jn, not yet updated by v_j
            if (P != jn) W[(long long)r * N + P] = xo[k];
            const double v = r > jn ? xp[k] * scal : (r == jn ? 1.0 : 0.0);
            vnxt[r] = v;
            if (r >= jn) T[(long long)jn * N + r] = v;
          }
        }
        if (wid == 0) {
          // the per-column bookkeeping follows the swap, one array per lane
          if (lane == 6) taus[jn] = tau;
          if (P != jn) {
            if (lane == 0) { const double t = nrm2[jn]; nrm2[jn] = nrm2[P]; nrm2[P] = t; }
            else if (lane == 1) { const double t = ref2[jn]; ref2[jn] = ref2[P]; ref2[P] = t; }
            else if (lane == 2) { const double t = dsc[jn]; dsc[jn] = dsc[P]; dsc[P] = t; }
            else if (lane == 3) { const double t = wsm[jn]; wsm[jn] = wsm[P]; wsm[P] = t; }
            else if (lane == 4) { const float f = logd[jn]; logd[jn] = logd[P]; logd[P] = f; }
            else if (lane == 5) { const int q = perm[jn]; perm[jn] = perm[P]; perm[P] = q; }
          }
        }
      }
      __syncthreads();
    };

    // ---- norms, first pivot and reflector, first dot products -------------
    {
      double ss = 0.0;
      if (own)
        for (int r = rg; r < N; r += TPC) {
          const double x = W[(long long)r * N + c];
          ss = fma(x, x, ss);
        }
      ss = group_sum<TPC>(ss);
      if (own && rg == 0) { nrm2[c] = ss; ref2[c] = ss; }
      const float key = own ? logd[c] + 0.5f * log2_wide(ss) : -INFINITY;
      vote_and_reflect(key, own ? c : 0x7fffffff, 0);
    }
    double dc = 0.0, xj = 0.0;   // v_j^T a_c and a_jc (column-uniform)
    if (own && c > 0) {
      double xp = 0.0;
      dc = fused_pass<TPC, BATCH>(W, N, c, rg, vnxt, 0.0, vnxt, 0, xp, false);
      xj = xp;
    }
    dc = group_sum<TPC>(dc);
    xj = __shfl_sync(FULL, xj, lane % CPW);   // row 0 is in row group 0
    { double* t = vcur; vcur = vnxt; vnxt = t; }

    // ---- steps j = 0 .. N-2 ------------------------------------------------
    for (int j = 0; j + 1 < N; ++j) {
      const bool act = own && c > j;
      float key = -INFINITY;
      int idx = 0x7fffffff;
      // warps whose columns are all at or left of j skip the column scalars
      // (each of them would still hold an FP64 pipe for 64 cycles)
      if (__any_sync(FULL, act)) {
        const double tau = taus[j];
        const double w = tau * dc;
        const double rjc = xj - w;
        const double n_old = act ? nrm2[c] : 0.0, r_old = act ? ref2[c] : 0.0;
        double n2 = fma(-rjc, rjc, n_old);
        const bool redo = act && n2 <= 1.4901161193847656e-8 * r_old;
        if (__any_sync(FULL, redo)) {
          // exact norm of the updated rows below j where the downdate lost too
          // many digits (the safeguard of LAPACK's xLAQP2)
          double ex = 0.0;
          if (redo)
            for (int r = j + 1 + ((rg - j - 1) % TPC + TPC) % TPC; r < N; r += TPC) {
              const double x = fma(-vcur[r], w, W[(long long)r * N + c]);
              ex = fma(x, x, ex);
            }
          ex = group_sum<TPC>(ex);
          if (redo) n2 = ex;
        }
        __syncwarp();
        if (act) {
          if (rg == 0) {
            wsm[c] = w;
            nrm2[c] = n2;
            if (redo) ref2[c] = n2;
          }
          key = logd[c] + 0.5f * log2_wide(n2);
          idx = c;
        }
      }
      vote_and_reflect(key, idx, j + 1);
      // ---- fused pass: update with v_j, dot with v_{j+1} --------------------
      if (__any_sync(FULL, own && c > j + 1)) {
        double dn = 0.0, xn = 0.0;
        if (own && c > j + 1) {
          const int r0 = j + ((rg - j) % TPC + TPC) % TPC;   // first row >= j in this row group
          dn = fused_pass<TPC, BATCH>(W, N, c, r0, vcur, wsm[c], vnxt, j + 1, xn, true);
        }
        dn = group_sum<TPC>(dn);
        xj = __shfl_sync(FULL, xn, (lane % CPW) + CPW * ((j + 1) % TPC));
        dc = dn;
      }
      double* t = vcur; vcur = vnxt; vnxt = t;
    }
    __syncthreads();

    // ---- Q = H_0 ... H_{N-1} into U, backwards ----------------------------
    for (long long e = tid; e < NN; e += NT) {
      const int i = (int)(e / N), cc = (int)(e % N);
      U[e] = i == cc ? 1.0 : 0.0;
    }
    // v_j, v_{j-1} staged one step ahead in three rotating buffers (wsm is
    // free after the factorisation)
    auto vq = [&](int k) { return k == 0 ? vA : (k == 1 ? vB : wsm); };
    for (int r = tid; r < N; r += NT) {
      vA[r] = r >= N - 1 ? T[(long long)(N - 1) * N + r] : 0.0;
      if (N >= 2) vB[r] = r >= N - 2 ? T[(long long)(N - 2) * N + r] : 0.0;
    }
    __syncthreads();
    double dq = 1.0;   // v_j^T u_c; column c enters at step c as e_c
    for (int j = N - 1; j >= 0; --j) {
      const double* vj = vq((N - 1 - j) % 3);
      const double* vm = vq((N - j) % 3);
      if (j >= 2) {
        double* vs = vq((N + 1 - j) % 3);
        for (int r = tid; r < N; r += NT) vs[r] = r >= j - 2 ? T[(long long)(j - 2) * N + r] : 0.0;
      }
      if (__any_sync(FULL, own && c >= j)) {
        if (own && c >= j) {
          if (c == j) dq = 1.0;
          const double w = taus[j] * dq;
          const int r0 = j + ((rg - j) % TPC + TPC) % TPC;
          double xdummy = 0.0;
          // rows >= j of column c; the dot with v_{j-1} needs no row j-1 (zero
          // in every column c >= j at this point)
          dq = fused_pass<TPC, BATCH>(U, N, c, r0, vj, w, j > 0 ? vm : vj, -1, xdummy, true);
        }
        dq = group_sum<TPC>(dq);
      }
      __syncthreads();
    }

    // ---- outputs D, T, perm (T overwrites the stored reflectors) -----------
    for (int i = tid; i < N; i += NT) {
      const double rii = fabs(W[(long long)i * N + i]);
      const double d = rii * dsc[i];
      if (!(d > 0.0)) atomicOr(&s_flag, DQMC_STATUS_SINGULAR);
      if (!isfinite(d)) atomicOr(&s_flag, DQMC_STATUS_NONFINITE_SCALE);
      Dout[i] = d;
      nrm2[i] = rii > 0.0 ? 1.0 / rii : 0.0;
      ref2[i] = dsc[i] > 0.0 ? 1.0 / dsc[i] : 0.0;
      pout[i] = perm[i];
    }
    __syncthreads();
    for (long long e = tid; e < NN; e += NT) {
      const int i = (int)(e / N), cc = (int)(e % N);
      T[e] = cc >= i ? W[e] * nrm2[i] * (dsc[cc] * ref2[i]) : 0.0;
      if (a.smem_mats >= 2) Uout[e] = U[e];
    }
    __syncthreads();
    if (tid == 0 && s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// qrp_small_kernel<TPC, NW>: the same factorisation for N <= 32 NW / TPC (16
// with 8 lanes per column, 32 with 4; the library launches four warps), one
// CTA per instance, two barriers per pivot step.
//
// A single small instance is latency-bound, and on GB300 every FP64 warp
// instruction holds its sub-partition's pipe for 64 cycles, so the design
// keeps the serial part of a step short and spreads the rest over four or
// eight warps (all four sub-partitions):
//   * TPC lanes own one column (rows rg + TPC k in registers); a warp owns
//     32 / TPC columns.
//   * Columns are never moved: the pivot order is recorded and applied when
//     T is written, so no column data crosses warps.
//   * The vote: each warp reduces the keys of its columns by shuffles and
//     posts its winner; after a barrier every thread picks the same winner
//     from the NW posts (ties -> lowest column, as in the kernels above;
//     non-finite keys count as -inf).
//   * The reflector: only the warp that owns the pivot column works; it
//     writes H_j = 1 - gamma u u^T in unnormalised form, u_j = alpha - beta,
//     u_r = a_rP below j, gamma = 1 / (beta (beta - alpha)) (one square root
//     and one division on the critical path, where v = u / u_j and
//     tau = gamma u_j^2 of the kernels above take two) to shared memory, and
//     a barrier publishes it.
//   * Every column not yet pivoted applies H_j and downdates its norm (the
//     xLAQP2 safeguard as above), then votes again.
// Q = H_0 ... H_{N-1} is accumulated backwards without barriers: each column
// group transforms its own column of Q.  Results agree with the other
// kernels to rounding; sums run in a different order.
// ---------------------------------------------------------------------------
// sum over the TPC lanes of a column group; every lane gets the same value
// (each butterfly level adds the same two partial sums on both sides)
template <int TPC>
__device__ __forceinline__ double col_group_sum(double v) {
#pragma unroll
  for (int off = 1; off < TPC; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <int TPC, int NW>
__global__ void __launch_bounds__(32 * NW, 2) qrp_small_kernel(const QrpArgs a) {
  constexpr int NT = 32 * NW, CPW = 32 / TPC, NMAX = NW * CPW, RPL = NMAX / TPC;
  static_assert(RPL >= 1 && RPL <= 16 && RPL * TPC == NMAX && NT <= 256, "thread mapping");
  __shared__ double s_u[NMAX][NMAX];    // u of step j at rows >= j
  __shared__ double s_gam[NMAX], s_beta[NMAX], s_dsc[NMAX], s_rinv[NMAX], s_dinv[NMAX];
  __shared__ int s_piv[NMAX];
  __shared__ float s_key[NW];
  __shared__ int s_idx[NW];
  __shared__ int s_flag;
  const int N = a.N;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int cw = lane / TPC, rg = lane % TPC;
  const int c = wid * CPW + cw;          // this lane's column
  const int gbase = lane & ~(TPC - 1);   // first lane of its column group
  const bool own = c < N;
  const unsigned FULL = 0xffffffffu;
  // launch contract (debug build): 128 threads, N columns covered
  if (!DQMC_CHECK(blockDim.x == NT && N >= 1 && N <= NMAX, N)) return;

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    if (a.lim && a.lim[b] < a.lim_at) continue;   // chain of this instance already finished
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    double* __restrict__ Uout = a.U + (long long)b * a.sU;
    double* __restrict__ Dout = a.D + (long long)b * a.sD;
    double* __restrict__ T = a.T + (long long)b * a.sT;
    int* __restrict__ pout = a.perm + (long long)b * a.sperm;
    const double* Din = a.Din ? a.Din + (long long)b * a.sDin : nullptr;

    if (tid == 0) s_flag = 0;
    int flag = 0;
    double x[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = rg + TPC * k;
      x[k] = (own && r < N) ? A[(long long)r * N + c] : 0.0;
      if (!isfinite(x[k])) flag |= DQMC_STATUS_NONFINITE_SCALE;
    }
    const double dsc = (own && Din) ? Din[c] : 1.0;
    if (!(isfinite(dsc) && dsc >= 0.0)) flag |= DQMC_STATUS_NONFINITE_SCALE;
    const float logd = own ? log2_wide(dsc) : -INFINITY;
    double nrm2 = 0.0;
#pragma unroll
    for (int k = 0; k < RPL; ++k) nrm2 = fma(x[k], x[k], nrm2);
    nrm2 = col_group_sum<TPC>(nrm2);
    double ref2 = nrm2;
    bool done = !own;      // column already pivoted (or not a column)
    int mystep = 0;        // position of this column in the pivot order
    __syncthreads();       // s_flag cleared; the previous instance's reads are over

    for (int j = 0; j < N; ++j) {
      const int k0 = j / TPC;   // rows with k < k0 lie above j
      // ---- vote ----------------------------------------------------------
      float key = done ? -INFINITY : logd + 0.5f * log2_wide(nrm2);
      if (!(key == key)) key = -INFINITY;
      int idx = done ? 0x7fffffff : c;
#pragma unroll
      for (int off = TPC; off < 32; off <<= 1) {
        const float k2 = __shfl_xor_sync(FULL, key, off);
        const int i2 = __shfl_xor_sync(FULL, idx, off);
        if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
      }
      if (lane == 0) { s_key[wid] = key; s_idx[wid] = idx; }
      __syncthreads();
      key = s_key[0];
      idx = s_idx[0];
#pragma unroll
      for (int w = 1; w < NW; ++w)
        if (s_key[w] > key || (s_key[w] == key && s_idx[w] < idx)) { key = s_key[w]; idx = s_idx[w]; }
      const int P = DQMC_CHECK(idx >= 0 && idx < N, idx) ? idx : 0;
      const bool mine = c == P;
      // ---- reflector of column P at rows >= j (the owning warp only) ---------
      if (wid == P / CPW) {
        double sp = 0.0, xjv = 0.0;
        ks_from<RPL>(k0, [&](auto K) {
          constexpr int k = decltype(K)::value;
          const int r = rg + TPC * k;
          const double t = r > j ? x[k] : 0.0;
          sp = fma(t, t, sp);
          xjv = r == j ? x[k] : xjv;
        });
        const double sig = col_group_sum<TPC>(sp);
        const double alpha = __shfl_sync(FULL, xjv, gbase | (j % TPC));
        double beta = alpha, gam = 0.0, uj = 0.0;
        if (sig > 0.0) {
          const double nrm = sqrt(fma(alpha, alpha, sig));
          beta = alpha >= 0.0 ? -nrm : nrm;
          uj = alpha - beta;
          gam = 1.0 / (beta * (beta - alpha));
        }
        if (mine) {
          ks_from<RPL>(k0, [&](auto K) {
            constexpr int k = decltype(K)::value;
            const int r = rg + TPC * k;
            if (r >= j && r < N) s_u[j][r] = r == j ? uj : x[k];
            if (r == j) x[k] = beta;              // r_jj of R
          });
          if (rg == 0) { s_gam[j] = gam; s_beta[j] = beta; s_dsc[j] = dsc; s_piv[j] = P; }
        }
      }
      if (mine) { done = true; mystep = j; }
      __syncthreads();
      // ---- apply H_j to the columns not yet pivoted, downdate their norms -----
      {
        const double gam = s_gam[j];
        double ur[RPL], pp = 0.0;
#pragma unroll
        for (int k = 0; k < RPL; ++k) ur[k] = 0.0;
        ks_from<RPL>(k0, [&](auto K) {
          constexpr int k = decltype(K)::value;
          const int r = rg + TPC * k;
          ur[k] = (r >= j && r < N) ? s_u[j][r] : 0.0;
          pp = fma(ur[k], x[k], pp);
        });
        // the group sum is a full-warp shuffle: every lane takes part, pivoted
        // columns included, before the result is discarded for them
        const double dsum = col_group_sum<TPC>(pp);
        const double w = done ? 0.0 : gam * dsum;
        double xjv = 0.0;
        ks_from<RPL>(k0, [&](auto K) {
          constexpr int k = decltype(K)::value;
          if (!done) x[k] = fma(-ur[k], w, x[k]);
          xjv = rg + TPC * k == j ? x[k] : xjv;
        });
        const double rjc = __shfl_sync(FULL, xjv, gbase | (j % TPC));   // updated a_jc
        double n2 = fma(-rjc, rjc, nrm2);
        const bool redo = !done && n2 <= 1.4901161193847656e-8 * ref2;
        if (__any_sync(FULL, redo)) {
          double ex = 0.0;
          ks_from<RPL>(k0, [&](auto K) {
            constexpr int k = decltype(K)::value;
            const double t = rg + TPC * k > j ? x[k] : 0.0;
            ex = fma(t, t, ex);
          });
          ex = col_group_sum<TPC>(ex);
          if (redo) n2 = ex;
        }
        if (!done) {
          nrm2 = n2;
          if (redo) ref2 = n2;
        }
      }
    }

    // ---- outputs D_i = |r_ii| Din_{p_i}, perm and T = D^{-1} R in pivot order ----
    if (tid < N) {
      const double ri = fabs(s_beta[tid]);
      const double d = ri * s_dsc[tid];
      if (!(d > 0.0)) flag |= DQMC_STATUS_SINGULAR;
      if (!isfinite(d)) flag |= DQMC_STATUS_NONFINITE_SCALE;
      Dout[tid] = d;
      pout[tid] = s_piv[tid];
      s_rinv[tid] = ri > 0.0 ? 1.0 / ri : 0.0;
      s_dinv[tid] = s_dsc[tid] > 0.0 ? 1.0 / s_dsc[tid] : 0.0;
    }
    flag = __reduce_or_sync(FULL, flag);
    if (lane == 0 && flag) atomicOr(&s_flag, flag);
    __syncthreads();
    if (own) {
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int i = rg + TPC * k;
        // this column is column mystep of R: rows above mystep hold R, row
        // mystep holds r_jj, the rows below are not part of R
        if (i < N) T[(long long)i * N + mystep] = i <= mystep ? x[k] * s_rinv[i] * (dsc * s_dinv[i]) : 0.0;
      }
    }
    // ---- Q = H_0 ... H_{N-1} on the identity, backwards, column by column ----
    double q[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) q[k] = rg + TPC * k == c ? 1.0 : 0.0;
    for (int j = N - 1; j >= 0; --j) {
      const int k0 = j / TPC;
      const double gam = s_gam[j];
      double ur[RPL], pp = 0.0;
#pragma unroll
      for (int k = 0; k < RPL; ++k) ur[k] = 0.0;
      ks_from<RPL>(k0, [&](auto K) {
        constexpr int k = decltype(K)::value;
        const int r = rg + TPC * k;
        ur[k] = (r >= j && r < N) ? s_u[j][r] : 0.0;
        pp = fma(ur[k], q[k], pp);
      });
      const double w = gam * col_group_sum<TPC>(pp);
      ks_from<RPL>(k0, [&](auto K) {
        constexpr int k = decltype(K)::value;
        q[k] = fma(-ur[k], w, q[k]);
      });
    }

#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = rg + TPC * k;
      if (own && r < N) Uout[(long long)r * N + c] = q[k];
    }
    __syncthreads();
    if (tid == 0 && s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
  }
}

template <int TPC, int NW>
static cudaError_t launch_qrp_small(const QrpArgs& a, cudaStream_t st) {
  const int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  qrp_small_kernel<TPC, NW><<<grid, 32 * NW, 0, st>>>(a);
  return cudaGetLastError();
}

static size_t qrp_fused_smem(int N) {
  return (size_t)N * (7 * sizeof(double) + sizeof(float) + sizeof(int)) + 16;
}

// Shared memory a CTA may use (opt-in limit of the SM).
constexpr size_t kSmemLimit = 227 * 1024;

// The working matrix W (and, when both fit, the accumulated Q) in shared
// memory: every step of the factorisation reads and updates the trailing
// columns, and from L2 each of those passes costs a round trip the step has
// to wait for.  N <= 160 fits W, N <= 112 fits W and Q.
template <int NT, int TPC, int NQ, int MINB = 0>
static cudaError_t launch_qrp_fused(const QrpArgs& a0, cudaStream_t st) {
  QrpArgs a = a0;
  const size_t base = qrp_fused_smem(a.N), mat = (size_t)a.N * a.N * sizeof(double);
  a.smem_mats = base + 2 * mat <= kSmemLimit ? 2 : (base + mat <= kSmemLimit ? 1 : 0);
  const size_t sm = base + a.smem_mats * mat;
  const int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  cudaError_t e = allow_dyn_smem(qrp_fused_kernel<NT, TPC, NQ, MINB>);
  if (e != cudaSuccess) return e;
  qrp_fused_kernel<NT, TPC, NQ, MINB><<<grid, NT, sm, st>>>(a);
  return cudaGetLastError();
}

static size_t qrp_smem(int N) { return (size_t)N * (6 * sizeof(double) + sizeof(float) + sizeof(int)) + 16; }

cudaError_t qrp_f64(const QrpArgs& a, cudaStream_t st) {
  if (a.batch <= 0 || a.N <= 0) return cudaSuccess;
  // N <= 32: four warps, two barriers per pivot step (qrp_small_kernel).  Its
  // eight-warp form for N <= 64 was measured and not taken: on the 8 x 8,
  // beta = 40 batch it moved more G(tau, 0) points of ill-conditioned fields
  // past 1e-10 than the full-size test admits
  if (a.N <= 16) return launch_qrp_small<8, 4>(a, st);
  if (a.N <= 32) return launch_qrp_small<4, 4>(a, st);
  if (a.N <= 64) return launch_qrp_fused<128, 2, 2>(a, st);
  if (a.N <= 128) return launch_qrp_fused<256, 2, 4>(a, st);
  if (a.N <= 256)
    return a.share_sm ? launch_qrp_fused<512, 2, 8, 2>(a, st) : launch_qrp_fused<512, 2, 8>(a, st);
  size_t sm = qrp_smem(a.N);
  int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  if (a.N <= 32) {
    allow_dyn_smem(qrp_kernel<32>);
    qrp_kernel<32><<<grid, 32, sm, st>>>(a);
  } else if (a.N <= 128) {
    allow_dyn_smem(qrp_kernel<128>);
    qrp_kernel<128><<<grid, 128, sm, st>>>(a);
  } else {
    allow_dyn_smem(qrp_kernel<256>);
    qrp_kernel<256><<<grid, 256, sm, st>>>(a);
  }
  return cudaGetLastError();
}


}  // namespace dqmc

DQMC_CHECK_UNIT(qrp)
