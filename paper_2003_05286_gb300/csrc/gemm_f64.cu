// Batched FP64 GEMM with fused diagonal scalings.
//
// GB300 executes FP64 at 1/64 of the FP32 rate (measured: 1.20 TFLOP/s with
// DFMA, 1.05 TFLOP/s with the f64 mma.sync shapes), so every dense product of
// the method is bound by the FP64 pipe: shared-memory and L2 traffic are
// tiny next to it.  The kernel is therefore a plain register-tiled DFMA GEMM
// whose only job is to keep the FP64 pipe busy: 4x4 (or 3x3) outputs per thread,
// double-buffered shared-memory tiles filled from registers one K-block
// ahead, and every diagonal factor of the method (exp(V_l) of the slice
// matrix, the D+/D- splits, the column scale of Eq. (stabmult)) applied while
// a tile is staged or written, never as a separate pass.
#include "common.cuh"

namespace dqmc {

template <int BM, int BN, int BK, int TM, int TN>
// At most 168 registers (the 64 x 64 tile takes 120): a 256-thread CTA then
// fits an SM beside one 512-thread pivoted-QR CTA of 64 registers, so the
// products of one sub-batch can share SMs with the QRs of another.
__global__ void __maxnreg__(168)
gemm_f64_kernel(const GemmArgs a) {
  constexpr int NTX = BN / TN;
  constexpr int NT = (BM / TM) * NTX;
  constexpr int A_PER = (BM * BK) / NT;
  constexpr int B_PER = (BK * BN) / NT;
  static_assert((BM * BK) % NT == 0 && (BK * BN) % NT == 0, "tile/thread mismatch");

  __shared__ __align__(16) double As[2][BK][BM];
  __shared__ __align__(16) double Bs[2][BK][BN];
  // launch contract (debug build): the thread mapping needs exactly NT
  // threads, and every leading dimension must cover its row
  if (!DQMC_CHECK(blockDim.x == NT, blockDim.x) ||
      !DQMC_CHECK(a.lda >= (a.transA ? a.M : a.K) && a.ldb >= (a.transB ? a.K : a.N) &&
                      a.ldc >= a.N, a.ldc))
    return;

  for (int b = blockIdx.z; b < a.batch; b += gridDim.z) {
  if (b != (int)blockIdx.z) __syncthreads();   // shared tiles are reused across batch entries
  const int m0 = blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;

  const double* __restrict__ A = a.A + (long long)(b / a.divA) * a.sA;
  const double* __restrict__ B = a.B + (long long)(b / a.divB) * a.sB;
  double* __restrict__ C = a.C + (long long)(b / a.divC) * a.sC;
  const double* ms = a.ms ? a.ms + (long long)(b / a.divS) * a.sms + (long long)(b % a.divS) * a.sms_inner : nullptr;
  const double* rs = a.rs ? a.rs + (long long)(b / a.divS) * a.srs : nullptr;
  const double* cs = a.cs ? a.cs + (long long)(b / a.divS) * a.scs : nullptr;
  const int* perm = a.permB ? a.permB + (long long)(b / a.divB) * a.sperm : nullptr;

  if ((a.skip_if && *a.skip_if <= a.skip_at) || (a.lim && a.lim[b] < a.lim_at)) {
    // identity pass: C = opB(B) restricted to this tile (square problems only)
    for (int e = tid; e < BM * BN; e += NT) {
      int m = m0 + e / BN, n = n0 + e % BN;
      if (m < a.M && n < a.N) C[(long long)m * a.ldc + n] = B[(long long)m * a.ldb + n];
    }
    continue;
  }

  double alpha = a.alpha;
  if (a.alpha_ptr) alpha *= *a.alpha_ptr;

  const int kbeg = a.upperA ? (m0 / BK) * BK : 0;
  const int kend = a.K;

  double ra[A_PER], rb[B_PER];

  auto load_tiles = [&](int kb) {
#pragma unroll
    for (int i = 0; i < A_PER; ++i) {
      int e = tid + i * NT;
      int m, k;
      double v = 0.0;
      if (!a.transA) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      int gm = m0 + m, gk = kb + k;
      if (gm < a.M && gk < a.K && !(a.upperA && gk < gm)) {
        v = a.transA ? A[(long long)gk * a.lda + gm] : A[(long long)gm * a.lda + gk];
      }
      ra[i] = v;
    }
#pragma unroll
    for (int i = 0; i < B_PER; ++i) {
      int e = tid + i * NT;
      int k, n;
      double v = 0.0;
      if (!a.transB) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      int gk = kb + k, gn = n0 + n;
      if (gk < a.K && gn < a.N) {
        int row = perm ? perm[gk] : gk;
        if (!DQMC_CHECK(row >= 0 && row < a.K, row)) row = gk;   // a permutation of 0..K-1
        v = a.transB ? B[(long long)gn * a.ldb + row] : B[(long long)row * a.ldb + gn];
        if (ms) v *= ms[gk];
      }
      rb[i] = v;
    }
  };
  auto store_tiles = [&](int buf) {
#pragma unroll
    for (int i = 0; i < A_PER; ++i) {
      int e = tid + i * NT;
      int m, k;
      if (!a.transA) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      As[buf][k][m] = ra[i];
    }
#pragma unroll
    for (int i = 0; i < B_PER; ++i) {
      int e = tid + i * NT;
      int k, n;
      if (!a.transB) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      Bs[buf][k][n] = rb[i];
    }
  };

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  if (kbeg < kend) {
    load_tiles(kbeg);
    store_tiles(0);
    __syncthreads();
    int buf = 0;
    for (int kb = kbeg; kb < kend; kb += BK) {
      const bool more = kb + BK < kend;
      if (more) load_tiles(kb + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double af[TM], bf[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) af[i] = As[buf][kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bf[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(af[i], bf[j], acc[i][j]);
      }
      if (more) {
        store_tiles(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int m = m0 + ty * TM + i;
    if (m >= a.M) continue;
    double r = alpha * (rs ? rs[m] : 1.0);
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int n = n0 + tx * TN + j;
      if (n >= a.N) continue;
      double v = acc[i][j] * r;
      if (cs) v *= cs[n];
      if (a.addIdentity && m == n) v += 1.0;
      C[(long long)m * a.ldc + n] = v;
    }
  }
  }  // batch loop
}

// Tile edge for an M x N output: the one that pads the least (every FMA of a
// padded row or column is wasted FP64-pipe time, e.g. 64-tiles on N = 144 do
// 1.78x the work, 48-tiles exactly 1x); ties go to 64 for large problems and
// to 32 (more CTAs) for small ones.  The K order is the same for every tile,
// so the results do not depend on the choice.
static int pick_tile(int M, int N) {
  const int prefs_big[3] = {64, 48, 32}, prefs_small[3] = {32, 48, 64};
  const int* prefs = (M >= 96 && N >= 96) ? prefs_big : prefs_small;
  int best = prefs[0];
  double bw = 0.0;
  for (int i = 0; i < 3; ++i) {
    const int t = prefs[i];
    const double w = (double)((M + t - 1) / t * t) * (double)((N + t - 1) / t * t);
    if (i == 0 || w < bw) { best = t; bw = w; }
  }
  return best;
}

template <int BM, int BN, int TM, int TN>
static void launch_gemm(const GemmArgs& a, int zb, cudaStream_t st) {
  constexpr int BK = 16;
  dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, zb);
  gemm_f64_kernel<BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, st>>>(a);
}

// Small products.  One SM sub-partition issues an FP64 warp instruction every
// 64 cycles, so a CTA whose outputs sit in one or two warps is bound by that
// issue rate, not by the launch: a 16 x 16 x 16 product on the 64-thread
// 32-tile (3/4 of it padding) takes ~15 us.  Outputs of at most 16 x 16 take a
// 16-tile with one output per thread (8 warps, two per sub-partition); outputs
// of at most 32 x 32 take a 256-thread 32-tile with 2 x 2 per thread while the
// batch leaves most SMs idle.  The K order per output is unchanged.
static int small_tile_ctas() {
  static const int n = [] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    return 2 * sms;
  }();
  return n;
}

cudaError_t gemm_f64(const GemmArgs& a, cudaStream_t st) {
  if (a.batch <= 0 || a.M <= 0 || a.N <= 0) return cudaSuccess;
  const int zb = a.batch < 65535 ? a.batch : 65535;   // grid z limit; the kernel loops
  if (!a.tile && a.M <= 16 && a.N <= 16) {
    launch_gemm<16, 16, 1, 1>(a, zb, st);                      // 256 threads, 1 output each
    return cudaGetLastError();
  }
  if (!a.tile && a.M <= 32 && a.N <= 32 && a.batch < small_tile_ctas()) {
    launch_gemm<32, 32, 2, 2>(a, zb, st);                      // 256 threads, 2x2 each
    return cudaGetLastError();
  }
  const int tile = a.tile ? a.tile : pick_tile(a.M, a.N);
  if (!a.tile) {
    // a product too small to fill the GPU with this tile (a single instance,
    // e.g. the Taylor steps of the matrix exponential: 16 CTAs of 64 x 64 at
    // N = 256) takes 16 x 16 tiles, one output per thread, so that every SM
    // gets FP64 work; the K order of each output is unchanged
    const long long ctas = (long long)zb * ((a.M + tile - 1) / tile) * ((a.N + tile - 1) / tile);
    if (ctas < device_sms()) {
      launch_gemm<16, 16, 1, 1>(a, zb, st);
      return cudaGetLastError();
    }
  }
  if (tile == 64) launch_gemm<64, 64, 4, 4>(a, zb, st);        // 256 threads, 4x4 each
  else if (tile == 48) launch_gemm<48, 48, 3, 3>(a, zb, st);   // 256 threads, 3x3 each
  else launch_gemm<32, 32, 4, 4>(a, zb, st);                   // 64 threads, 4x4 each
  return cudaGetLastError();
}

}  // namespace dqmc

DQMC_CHECK_UNIT(gemm)
