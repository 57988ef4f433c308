// LU with partial pivoting and multi-right-hand-side solve, one CTA per
// instance.  Every inverse the inversion schemes write (X^{-1}, the bracket
// of Eq. (inversion_loh), the middle matrix of Eq. (inversion_tdgf_loh)) is
// evaluated as a solve with this kernel, never as an explicit inverse.
//
// The augmented matrix [opA(A) | opR(R)] (N x (N + nrhs), row-major, in the
// L2-resident workspace) is eliminated column by column with row pivoting
// (largest |a_rj|, lowest row on ties); one thread owns one column, so each
// rank-1 update streams rows that are contiguous across the threads of a
// warp.  Back substitution then runs without any synchronisation: each
// right-hand-side column belongs to one thread.  log|det| and the sign of
// det(opA(A)) come out of the pivots.  Systems with N <= 32 and N + nrhs <= 64
// take lu_small_kernel below (the columns in registers, one barrier per step).
#include "common.cuh"

namespace dqmc {

// RPT * NT >= N: rows of the pivot column each thread keeps in registers.
template <int NT, int RPT>
__global__ void __launch_bounds__(NT) lu_kernel(const LuArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N, nr = a.nrhs, Wd = N + nr;
  // a.smem_w: the augmented matrix lives in shared memory (else in the
  // workspace, L2-resident); the kernel reads it through a plain pointer
  double* smW = reinterpret_cast<double*>(smem_raw);
  double* lbuf = smW + (a.smem_w ? (long long)N * Wd : 0);   // multipliers of the current column
  double* dinv = lbuf + N;                              // 1 / u_jj
  double* apiv = dinv + N;                              // |u_jj|: log det is summed at the end
  __shared__ unsigned long long sk[32];
  __shared__ int si[32];
  __shared__ double sv[32];
  __shared__ int s_flag, s_sign;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // launch contract (debug build): NT threads, the pivot column held in
  // RPT registers per thread, leading dimensions that cover their rows, and
  // shared memory for the multipliers, the reciprocal and absolute pivots
  // and, when resident, the augmented matrix
  if (!DQMC_CHECK(blockDim.x == NT && N <= RPT * NT, N) ||
      !DQMC_CHECK(a.Rdiag || a.ldr >= (a.transR ? N : nr), a.ldr) ||
      !DQMC_CHECK(a.ldz >= (a.transZ ? N : nr), a.ldz) ||
      !DQMC_CHECK(dyn_smem_bytes() >= (unsigned)(((a.smem_w ? (long long)N * Wd : 0) + 3LL * N) * 8),
                  dyn_smem_bytes()))
    return;

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    double* __restrict__ W = a.smem_w ? smW : a.W + (long long)b * a.sW;
    if (tid == 0) { s_flag = 0; s_sign = 1; }

    // ---- load [opA(A) | opR(R)] ------------------------------------------
    for (long long e = tid; e < (long long)N * N; e += NT) {
      int r = (int)(e / N), c = (int)(e % N);
      // read contiguous memory: for transA the contiguous index is the row of W
      double v = a.transA ? A[(long long)c * N + r] : A[e];
      W[(long long)r * Wd + c] = v;
    }
    if (a.Rdiag) {
      const double* Rd = a.Rdiag + (long long)b * a.sRdiag;
      for (long long e = tid; e < (long long)N * nr; e += NT) {
        int r = (int)(e / nr), c = (int)(e % nr);
        double v = 0.0;
        if (r == c) v = a.invRdiag ? 1.0 / Rd[r] : Rd[r];
        W[(long long)r * Wd + N + c] = v;
      }
    } else {
      const double* R = a.R + (long long)b * a.sR;
      for (long long e = tid; e < (long long)N * nr; e += NT) {
        int r, c;
        double v;
        if (!a.transR) { r = (int)(e / nr); c = (int)(e % nr); v = R[(long long)r * a.ldr + c]; }
        else { c = (int)(e / N); r = (int)(e % N); v = R[(long long)c * a.ldr + r]; }
        W[(long long)r * Wd + N + c] = v;
      }
    }
    __syncthreads();

    // ---- elimination with partial pivoting -------------------------------
    // Per column j, three barriers: (1) candidates of the pivot search (the
    // column is kept in registers), (2) multipliers + row swap, (3) update.
    // The pivot value travels with its candidate: between (1) and (2) thread
    // 0 swaps rows j and p (column j included), so W[p][j] is not re-read.
    for (int j = 0; j < N; ++j) {
      double x[RPT];
      unsigned long long key = 0ull;   // |a_rj| bits (sign cleared), ordered like the values
      int idx = 0x7fffffff;
      double val = 0.0;                // a_rj of the candidate
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = j + tid + q * NT;
        x[q] = r < N ? W[(long long)r * Wd + j] : 0.0;
        if (r < N) {
          unsigned long long k2 = (unsigned long long)__double_as_longlong(x[q]) & 0x7fffffffffffffffull;
          if (k2 > key || (k2 == key && r < idx)) { key = k2; idx = r; val = x[q]; }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        unsigned long long k2 = __shfl_down_sync(0xffffffffu, key, off);
        int i2 = __shfl_down_sync(0xffffffffu, idx, off);
        double v2 = __shfl_down_sync(0xffffffffu, val, off);
        if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; val = v2; }
      }
      if (lane == 0) { sk[wid] = key; si[wid] = idx; sv[wid] = val; }
      const double ajj = W[(long long)j * Wd + j];
      __syncthreads();
      key = sk[0];
      idx = si[0];
      val = sv[0];
      for (int w = 1; w < NT / 32; ++w)
        if (sk[w] > key || (sk[w] == key && si[w] < idx)) { key = sk[w]; idx = si[w]; val = sv[w]; }
      const int p = (idx >= j && idx < N) ? idx : j;
      const double piv = p == j ? ajj : val;
      const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
      // multipliers of rows r > j after the swap (row p then holds the old row j)
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = j + tid + q * NT;
        if (r > j && r < N) lbuf[r] = (r == p ? ajj : x[q]) * inv;
      }
      if (p != j) {
        for (int c = j + tid; c < Wd; c += NT) {
          double t = W[(long long)j * Wd + c];
          W[(long long)j * Wd + c] = W[(long long)p * Wd + c];
          W[(long long)p * Wd + c] = t;
        }
      }
      if (tid == 0) {
        if (piv == 0.0) s_flag |= DQMC_STATUS_SINGULAR;
        if (p != j) s_sign = -s_sign;
        if (piv < 0.0) s_sign = -s_sign;
        apiv[j] = fabs(piv);
        dinv[j] = inv;
      }
      __syncthreads();
      for (int c = j + 1 + tid; c < Wd; c += NT) {
        double* col = W + c;
        const double pj = col[(long long)j * Wd];
        if (pj == 0.0) continue;
        // col[r] -= l_r * pj, 8 rows per batch, next batch loaded before the stores
        int r = j + 1;
        if (r + 7 < N) {
          double y0[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) y0[i] = col[(long long)(r + i) * Wd];
          for (; r + 15 < N; r += 8) {
            double y[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) y[i] = col[(long long)(r + 8 + i) * Wd];
#pragma unroll
            for (int i = 0; i < 8; ++i) col[(long long)(r + i) * Wd] = fma(-lbuf[r + i], pj, y0[i]);
#pragma unroll
            for (int i = 0; i < 8; ++i) y0[i] = y[i];
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) col[(long long)(r + i) * Wd] = fma(-lbuf[r + i], pj, y0[i]);
          r += 8;
        }
        for (; r < N; ++r) col[(long long)r * Wd] = fma(-lbuf[r], pj, col[(long long)r * Wd]);
      }
      __syncthreads();
    }

    // ---- back substitution, one thread per right-hand side ---------------
    double* __restrict__ Z = a.Z + (long long)b * a.sZ;
    for (int c = tid; c < nr; c += NT) {
      double* col = W + N + c;
      for (int i = N - 1; i >= 0; --i) {
        const double* urow = W + (long long)i * Wd;
        double s0 = col[(long long)i * Wd], s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int m = i + 1;
        for (; m + 7 < N; m += 8) {
          double x[8], u[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) { x[q] = col[(long long)(m + q) * Wd]; u[q] = urow[m + q]; }
          s0 = fma(-u[0], x[0], s0); s1 = fma(-u[1], x[1], s1);
          s2 = fma(-u[2], x[2], s2); s3 = fma(-u[3], x[3], s3);
          s0 = fma(-u[4], x[4], s0); s1 = fma(-u[5], x[5], s1);
          s2 = fma(-u[6], x[6], s2); s3 = fma(-u[7], x[7], s3);
        }
        for (; m < N; ++m) s0 = fma(-urow[m], col[(long long)m * Wd], s0);
        col[(long long)i * Wd] = ((s0 + s1) + (s2 + s3)) * dinv[i];
      }
    }
    // log|det| = sum_j log|u_jj|, taken here rather than once per elimination
    // step on its critical path: strided partial sums per thread, then a
    // fixed-order reduction (lane 0 of each warp, warps in order)
    if (a.logabsdet) {
      double ls = 0.0;
      for (int jj = tid; jj < N; jj += NT) ls += log(apiv[jj]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, off);
      if (lane == 0) sv[wid] = ls;
    }
    __syncthreads();
    for (long long e = tid; e < (long long)N * nr; e += NT) {
      if (!a.transZ) {
        int r = (int)(e / nr), c = (int)(e % nr);
        Z[(long long)r * a.ldz + c] = W[(long long)r * Wd + N + c];
      } else {
        int c = (int)(e / N), r = (int)(e % N);
        Z[(long long)c * a.ldz + r] = W[(long long)r * Wd + N + c];
      }
    }
    if (tid == 0) {
      if (a.logabsdet) {
        double lad = 0.0;
        for (int w = 0; w < NT / 32; ++w) lad += sv[w];
        a.logabsdet[b] = lad;
      }
      if (a.sign) a.sign[b] = s_sign;
      if (s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// lu_small_kernel<NW, RPL>: the same solve for N <= 4 RPL and N + nrhs <= 8 NW
// (NW warps), one barrier per elimination step.
//
// For a small system the kernel above is latency-bound: three barriers per
// column, and with one thread per column at most one warp does the update.
// Here four lanes own one column of [opA(A) | opR(R)] (rows rg + 4 k in
// registers).  At step j the warp owning column j finds the pivot (largest
// |a_rj|, lowest row on ties, as above), forms the multipliers with the one
// division of the step and posts them; after the barrier every other column
// swaps rows j and p and eliminates below j in registers.  U then goes to
// shared memory and each right-hand-side column solves U z = y on its own
// (column-oriented substitution with the reciprocal pivots).  log|det| is
// summed at the end, the sign follows the swaps and the pivot signs.
// ---------------------------------------------------------------------------
template <int NW, int RPL>
__global__ void __launch_bounds__(32 * NW) lu_small_kernel(const LuArgs a) {
  constexpr int TPC = 4, CPW = 32 / TPC, WMAX = NW * CPW, NMAX = TPC * RPL;
  static_assert(WMAX >= NMAX, "the columns of A fit the warps");
  __shared__ double s_l[NMAX][NMAX];   // multipliers of step j at rows > j
  __shared__ double s_u[NMAX][NMAX];   // U, row-major, after the elimination
  __shared__ double s_inv[NMAX], s_apv[NMAX], s_ls[NW];
  __shared__ int s_p[NMAX];
  __shared__ int s_flag, s_sign;
  const int N = a.N, nr = a.nrhs, Wd = N + nr;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int cw = lane / TPC, rg = lane % TPC, gbase = lane & ~(TPC - 1);
  const int c = wid * CPW + cw;         // this lane's column of the augmented matrix
  const bool own = c < Wd;
  const unsigned FULL = 0xffffffffu;
  // launch contract (debug build): NW warps covering the columns, RPL rows
  // per lane covering N, leading dimensions that cover their rows
  if (!DQMC_CHECK(blockDim.x == 32 * NW && N >= 1 && N <= NMAX && Wd <= WMAX, Wd) ||
      !DQMC_CHECK(a.Rdiag || a.ldr >= (a.transR ? N : nr), a.ldr) ||
      !DQMC_CHECK(a.ldz >= (a.transZ ? N : nr), a.ldz))
    return;

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    double* __restrict__ Z = a.Z + (long long)b * a.sZ;
    if (tid == 0) { s_flag = 0; s_sign = 1; }
    double x[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = rg + TPC * k;
      double v = 0.0;
      if (own && r < N) {
        if (c < N) {
          v = a.transA ? A[(long long)c * N + r] : A[(long long)r * N + c];
        } else if (a.Rdiag) {
          const double* Rd = a.Rdiag + (long long)b * a.sRdiag;
          if (r == c - N) v = a.invRdiag ? 1.0 / Rd[r] : Rd[r];
        } else {
          const double* R = a.R + (long long)b * a.sR;
          const int cc = c - N;
          v = a.transR ? R[(long long)cc * a.ldr + r] : R[(long long)r * a.ldr + cc];
        }
      }
      x[k] = v;
    }
    __syncthreads();   // s_flag, s_sign set; the previous instance's reads are over

    for (int j = 0; j < N; ++j) {
      const int k0 = j / TPC;   // rows with k < k0 lie above j
      if (wid == j / CPW) {
        // ---- pivot of column j (its four lanes; the rest of the warp idles)
        const bool mine = c == j;
        unsigned long long key = 0ull;   // |a_rj| bits, ordered like the values
        int idx = 0x7fffffff;
        double val = 0.0, ajj = 0.0;
#pragma unroll
        for (int k = 0; k < RPL; ++k) {
          const int r = rg + TPC * k;
          if (mine && r >= j && r < N) {
            const unsigned long long k2 =
                (unsigned long long)__double_as_longlong(x[k]) & 0x7fffffffffffffffull;
            if (k2 > key || (k2 == key && r < idx)) { key = k2; idx = r; val = x[k]; }
          }
          ajj = r == j ? x[k] : ajj;
        }
#pragma unroll
        for (int off = 1; off < TPC; off <<= 1) {
          const unsigned long long k2 = __shfl_xor_sync(FULL, key, off);
          const int i2 = __shfl_xor_sync(FULL, idx, off);
          const double v2 = __shfl_xor_sync(FULL, val, off);
          if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; val = v2; }
        }
        ajj = __shfl_sync(FULL, ajj, gbase | (j % TPC));
        // only the lanes of column j hold a candidate
        const int p = (idx >= j && idx < N) ? idx : j;
        if (mine) (void)DQMC_CHECK(idx >= j && idx < N, idx);
        const double piv = p == j ? ajj : val;
        const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
        if (mine) {
          // multipliers of rows r > j after the swap (row p then holds the old row j)
          ks_from<RPL>(k0, [&](auto K) {
            constexpr int k = decltype(K)::value;
            const int r = rg + TPC * k;
            if (r > j && r < N) s_l[j][r] = (r == p ? ajj : x[k]) * inv;
            if (r == j) x[k] = piv;   // u_jj; the rest of column j is not needed
          });
          if (rg == 0) {
            s_p[j] = p;
            s_inv[j] = inv;
            s_apv[j] = fabs(piv);
            if (piv == 0.0) s_flag |= DQMC_STATUS_SINGULAR;
            if ((p != j) != (piv < 0.0)) s_sign = -s_sign;
          }
        }
      }
      __syncthreads();
      // ---- columns c > j: swap rows j and p, eliminate below j -----------------
      const int p = s_p[j];
      double vj = 0.0, vp = 0.0;
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int r = rg + TPC * k;
        vj = r == j ? x[k] : vj;
        vp = r == p ? x[k] : vp;
      }
      vj = __shfl_sync(FULL, vj, gbase | (j % TPC));   // old a_jc
      vp = __shfl_sync(FULL, vp, gbase | (p % TPC));   // old a_pc: row j after the swap
      if (own && c > j) {
        ks_from<RPL>(k0, [&](auto K) {
          constexpr int k = decltype(K)::value;
          const int r = rg + TPC * k;
          double y = r == p ? vj : x[k];
          if (r == j) y = vp;
          else if (r > j && r < N) y = fma(-s_l[j][r], vp, y);
          x[k] = y;
        });
      }
    }
    // ---- U to shared memory, then z_m = y_m / u_mm, y_r -= u_rm z_m (r < m) -----
    if (own && c < N) {
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int r = rg + TPC * k;
        if (r <= c) s_u[r][c] = x[k];
      }
    }
    __syncthreads();
    // every lane runs the substitution (its shuffles need the whole warp); only
    // the right-hand-side columns keep the result
    for (int m = N - 1; m >= 0; --m) {
      double ym = 0.0;
#pragma unroll
      for (int k = 0; k < RPL; ++k) ym = rg + TPC * k == m ? x[k] : ym;
      const double zm = __shfl_sync(FULL, ym, gbase | (m % TPC)) * s_inv[m];
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int r = rg + TPC * k;
        if (r == m) x[k] = zm;
        else if (r < m) x[k] = fma(-s_u[r][m], zm, x[k]);
      }
    }
    if (own && c >= N) {
      const int cc = c - N;
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int r = rg + TPC * k;
        if (r < N) {
          if (a.transZ) Z[(long long)cc * a.ldz + r] = x[k];
          else Z[(long long)r * a.ldz + cc] = x[k];
        }
      }
    }
    // log|det| = sum of log|u_jj| in a fixed order (lane 0 of each warp, warps in order)
    if (a.logabsdet) {
      double ls = 0.0;
      for (int jj = tid; jj < N; jj += 32 * NW) ls += log(s_apv[jj]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) ls += __shfl_xor_sync(FULL, ls, off);
      if (lane == 0) s_ls[wid] = ls;
    }
    __syncthreads();
    if (tid == 0) {
      if (a.logabsdet) {
        double lad = 0.0;
        for (int w = 0; w < NW; ++w) lad += s_ls[w];
        a.logabsdet[b] = lad;
      }
      if (a.sign) a.sign[b] = s_sign;
      if (s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
    }
    __syncthreads();   // shared memory is reused by the next instance
  }
}

template <int NW, int RPL>
static cudaError_t launch_lu_small(const LuArgs& a, cudaStream_t st) {
  const int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  lu_small_kernel<NW, RPL><<<grid, 32 * NW, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t lu_solve_f64(const LuArgs& a0, cudaStream_t st) {
  if (a0.batch <= 0 || a0.N <= 0) return cudaSuccess;
  // small systems: four lanes per column, one barrier per step (lu_small_kernel)
  if (a0.N <= 32 && a0.nrhs >= 0 && a0.N + a0.nrhs <= 64) {
    const int wd = a0.N + a0.nrhs;
    if (a0.N <= 16) return wd <= 32 ? launch_lu_small<4, 4>(a0, st) : launch_lu_small<8, 4>(a0, st);
    return wd <= 32 ? launch_lu_small<4, 8>(a0, st) : launch_lu_small<8, 8>(a0, st);
  }
  LuArgs a = a0;
  size_t sm = (size_t)a.N * 3 * sizeof(double) + 16;
  // the augmented matrix in shared memory when it fits (227 KB per CTA): every
  // elimination step reads and updates the trailing block
  const size_t wb = (size_t)a.N * (a.N + a.nrhs) * sizeof(double);
  a.smem_w = sm + wb <= 227 * 1024 ? 1 : 0;
  if (a.smem_w) sm += wb;
  int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  if (a.N + a.nrhs <= 64) {
    allow_dyn_smem(lu_kernel<64, 1>);
    lu_kernel<64, 1><<<grid, 64, sm, st>>>(a);
  } else if (a.N + a.nrhs <= 256) {
    allow_dyn_smem(lu_kernel<256, 1>);
    lu_kernel<256, 1><<<grid, 256, sm, st>>>(a);
  } else {
    allow_dyn_smem(lu_kernel<512, 2>);
    lu_kernel<512, 2><<<grid, 512, sm, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dqmc

DQMC_CHECK_UNIT(lu)
