// One-sided (Hestenes) Jacobi SVD as the alternative stabiliser of the chain:
// the decomposition B = U D X of Sec. 4.2 with U, X = V^T orthogonal, the
// paper's accurate SVD variant (Sec. 4.2.1).  One CTA per instance.
//
// The columns a_p of Y = A diag(Din) are orthogonalised pairwise: for a pair
// with alpha = |a_p|^2, beta = |a_q|^2, gamma = a_p . a_q the rotation
//   zeta = (beta - alpha) / (2 gamma),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2),  s = c t,
//   a_p <- c a_p - s a_q,  a_q <- s a_p + c a_q      (same on the columns of V)
// makes them orthogonal.  The N - 1 rounds of a sweep follow the circle
// method, so the N/2 pairs of a round are disjoint and run in parallel, four
// lanes per pair.  A pair is skipped when |gamma| <= N eps sqrt(alpha) sqrt(beta);
// the sweeps end when none rotates (at most max_sweeps, else the status bit
// DQMC_STATUS_NOT_CONVERGED).  Then D_p = |a_p|, U = [a_p / D_p], and the
// rotated identity holds V^T, so that X' = V^T X_prev.  Y is applied with its
// column scale: the rotations keep the relative accuracy of graded columns.
//
// The columns live transposed in the workspace (row p of W is a_p) so that a
// pair's four lanes stream contiguous memory; W and V^T stay L2-resident.
#include "common.cuh"

namespace dqmc {

namespace {

// Pair i of round r of the circle method on Np (even) indices.
__device__ __forceinline__ void round_pair(int Np, int r, int i, int& p, int& q) {
  const int m = Np - 1;
  if (i == 0) {
    p = 0;
    q = r % m + 1;
  } else {
    p = (r + i) % m + 1;
    q = ((r - i) % m + m) % m + 1;
  }
}

}  // namespace

template <int NT>
__global__ void __launch_bounds__(NT) jacobi_svd_kernel(const JacobiArgs a) {
  constexpr int TPP = 4;                 // lanes per pair
  __shared__ double sig[512];
  __shared__ int s_rot, s_flag;
  const int N = a.N, Np = N + (N & 1);
  const int tid = threadIdx.x, g = tid / TPP, l4 = tid % TPP;
  const double tol = N * 1.1102230246251565e-16;
  // launch contract (debug build): four lanes for each of the Np / 2 pairs,
  // singular values of at most 512 columns in shared memory
  if (!DQMC_CHECK(blockDim.x == NT && TPP * (Np / 2) <= NT && N <= 512, N)) return;

  for (int b = blockIdx.x; b < a.batch; b += gridDim.x) {
    if (a.lim && a.lim[b] < a.lim_at) continue;   // chain of this instance already finished
    const double* __restrict__ A = a.A + (long long)b * a.sA;
    const double* Din = a.Din ? a.Din + (long long)b * a.sDin : nullptr;
    double* __restrict__ W = a.W + (long long)b * a.sW;
    double* __restrict__ Vt = a.Vt + (long long)b * a.sVt;
    if (tid == 0) s_flag = 0;
    int bad = 0;
    for (long long e = tid; e < (long long)N * N; e += NT) {
      const int r = (int)(e / N), p = (int)(e % N);
      const double v = A[e] * (Din ? Din[p] : 1.0);
      bad |= !isfinite(v);
      W[(long long)p * N + r] = v;
      Vt[(long long)p * N + r] = p == r ? 1.0 : 0.0;
    }
    __syncthreads();
    if (bad) atomicOr(&s_flag, DQMC_STATUS_NONFINITE_SCALE);

    bool converged = false;
    for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
      if (tid == 0) s_rot = 0;
      __syncthreads();
      int rot = 0;
      for (int r = 0; r < Np - 1; ++r) {
        int p = 0, q = 0;
        const bool grp = g < Np / 2;
        if (grp) round_pair(Np, r, g, p, q);
        const bool act = grp && p < N && q < N;
        double al = 0.0, be = 0.0, ga = 0.0;
        if (act) {
          const double* x = W + (long long)p * N;
          const double* y = W + (long long)q * N;
          for (int row = l4; row < N; row += TPP) {
            const double xv = x[row], yv = y[row];
            al = fma(xv, xv, al);
            be = fma(yv, yv, be);
            ga = fma(xv, yv, ga);
          }
        }
#pragma unroll
        for (int off = 1; off < TPP; off <<= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, off);
          be += __shfl_xor_sync(0xffffffffu, be, off);
          ga += __shfl_xor_sync(0xffffffffu, ga, off);
        }
        if (act && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const double z = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, z) / (fabs(z) + hypot(1.0, z));
          const double c = 1.0 / sqrt(fma(t, t, 1.0)), s = c * t;
          double* x = W + (long long)p * N;
          double* y = W + (long long)q * N;
          double* vx = Vt + (long long)p * N;
          double* vy = Vt + (long long)q * N;
          for (int row = l4; row < N; row += TPP) {
            const double xv = x[row], yv = y[row];
            x[row] = fma(c, xv, -s * yv);
            y[row] = fma(s, xv, c * yv);
            const double ux = vx[row], uy = vy[row];
            vx[row] = fma(c, ux, -s * uy);
            vy[row] = fma(s, ux, c * uy);
          }
          if (l4 == 0) ++rot;
        }
        __syncthreads();   // the next round pairs these columns with others
      }
      if (rot) atomicAdd(&s_rot, rot);
      __syncthreads();
      const bool done = s_rot == 0;
      __syncthreads();     // everyone has read s_rot before it is reset
      if (done) {
        converged = true;
        break;
      }
    }
    if (!converged && tid == 0) s_flag |= DQMC_STATUS_NOT_CONVERGED;

    // D_p = |a_p| (scaled sum of squares), U = [a_p / D_p]
    for (int p = tid; p < N; p += NT) {
      const double* x = W + (long long)p * N;
      double mx = 0.0;
      for (int r = 0; r < N; ++r) mx = fmax(mx, fabs(x[r]));
      double ss = 0.0;
      if (mx > 0.0)
        for (int r = 0; r < N; ++r) {
          const double u = x[r] / mx;
          ss = fma(u, u, ss);
        }
      const double d = mx * sqrt(ss);
      sig[p] = d;
      a.D[(long long)b * a.sD + p] = d;
      if (!(d > 0.0)) atomicOr(&s_flag, DQMC_STATUS_SINGULAR);
      if (!isfinite(d)) atomicOr(&s_flag, DQMC_STATUS_NONFINITE_SCALE);
    }
    __syncthreads();
    double* __restrict__ U = a.U + (long long)b * a.sU;
    for (long long e = tid; e < (long long)N * N; e += NT) {
      const int r = (int)(e / N), p = (int)(e % N);
      U[e] = sig[p] > 0.0 ? W[(long long)p * N + r] / sig[p] : 0.0;
    }
    __syncthreads();
    if (tid == 0 && s_flag && a.status) atomicOr(&a.status[b / a.status_div], s_flag);
    __syncthreads();
  }
}

template <int NT>
static cudaError_t launch_jacobi(const JacobiArgs& a, cudaStream_t st) {
  const int grid = a.batch < (1 << 30) ? a.batch : (1 << 30);
  jacobi_svd_kernel<NT><<<grid, NT, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t jacobi_svd_f64(const JacobiArgs& a, cudaStream_t st) {
  if (a.batch <= 0 || a.N <= 0) return cudaSuccess;
  if (a.N > 512) return cudaErrorInvalidValue;
  // four lanes per pair: 2 * (N rounded up to even) lanes cover the N/2 pairs
  if (a.N <= 32) return launch_jacobi<64>(a, st);
  if (a.N <= 64) return launch_jacobi<128>(a, st);
  if (a.N <= 128) return launch_jacobi<256>(a, st);
  if (a.N <= 256) return launch_jacobi<512>(a, st);
  return launch_jacobi<1024>(a, st);
}

}  // namespace dqmc

DQMC_CHECK_UNIT(jacobi)
