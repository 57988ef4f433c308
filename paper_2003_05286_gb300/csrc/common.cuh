// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dqmc.h"

namespace dqmc {

// SM count of the current device (queried once per device index and kept:
// it is a property of the GPU, not of a context).
int device_sms();

// Largest dynamic shared memory a CTA of the current device may opt into
// (queried once per device index and kept).
int device_smem_optin();

// Opts a kernel into the device's whole dynamic shared memory rather than the
// size of the launch at hand: one function (one template instance) serves
// launches of different sizes (e.g. the QR with its matrix resident at
// N = 144 and in L2 at N = 256), and a CUDA graph recorded with several of
// them must not depend on which launch set the attribute last.  The
// attribute only caps; each launch still allocates its own size.  The cap is
// the opt-in limit less the kernel's static shared memory (their sum may not
// exceed the limit).
template <class Kernel>
inline cudaError_t allow_dyn_smem(Kernel* kernel) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              device_smem_optin() - (int)fa.sharedSizeBytes);
}

// Grid of a grid-stride element-wise kernel over n items with tpb threads per
// block: enough blocks for n, at most 64 per SM of the current device.
inline int grid_stride_blocks(long long n, int tpb) {
  long long g = (n + tpb - 1) / tpb;
  const long long cap = 64LL * device_sms();
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// Batched FP64 GEMM with fused diagonal scalings (the slice-chain product of
// Sec. 2, Eq. (Ztr) and every dense product of the inversion schemes).
//
//   C_b = alpha * diag(rs_b) * opA(A_b) * diag(ms_b) * opB(B_b) * diag(cs_b)  (+ I)
//
// opA(A) is M x K, opB(B) is K x N, all row-major with leading dimensions.
// Row k of opB(B) is taken from row permB[k] of opB's source when permB is
// set.  upperA declares opA(A) upper triangular (entries below the diagonal
// are skipped, not read).  Per-instance pointers advance by the strides
// (stride 0 = shared by the batch).  alpha_ptr (device scalar) multiplies
// alpha when set.  skip_if (device int) + skip_at: the launch is a copy
// C_b = B_b when *skip_if <= skip_at (used by the scaling-and-squaring loop
// of the matrix exponential).
// ---------------------------------------------------------------------------
struct GemmArgs {
  int M = 0, N = 0, K = 0, batch = 0;
  const double* A = nullptr; long long lda = 0, sA = 0; int transA = 0;
  const double* B = nullptr; long long ldb = 0, sB = 0; int transB = 0;
  double* C = nullptr; long long ldc = 0, sC = 0;
  const double* ms = nullptr; long long sms = 0;
  const double* rs = nullptr; long long srs = 0;
  const double* cs = nullptr; long long scs = 0;
  const int* permB = nullptr; long long sperm = 0;
  int upperA = 0;
  int addIdentity = 0;
  double alpha = 1.0;
  const double* alpha_ptr = nullptr;
  const int* skip_if = nullptr; int skip_at = 0;
  // per-instance copy-through: when lim[b] < lim_at the launch writes
  // C_b = B_b for that instance (ragged chains of different length)
  const int* lim = nullptr; int lim_at = 0;
  long long sms_inner = 0;   // ms_b = ms + (b / divS) * sms + (b % divS) * sms_inner
  // batch index b maps to instance pointers through b / bdiv (so that a
  // shared operand can be indexed per group of bdiv problems): pointer of
  // operand X is base + (b / divX) * sX.
  int divA = 1, divB = 1, divC = 1, divS = 1;
  int tile = 0;   // CTA tile edge: 0 = by size, 32 or 64
};

cudaError_t gemm_f64(const GemmArgs& a, cudaStream_t st);

// ---------------------------------------------------------------------------
// The slice products of one chunk in one launch for N <= CHAIN_SMALL_MAX_N
// (chain_small.cu): for s = 0 .. nslices-1 with l = lo + s (dir > 0) or
// l = hi - s (dir < 0)
//   dir > 0:  C_b <- E diag(ev_b(l)) C_b        dir < 0:  C_b <- diag(ev_b(l)) E^T C_b
// starting from C_b = X_b (transE selects E^T for the backward chain), with
// ev_b(l) = expV + (b / divS) sV + (b % divS) sV_inner + (l - 1) N.  With lim,
// instance b applies only the slices s with lim[b] >= lim_base + s (its
// chain has ended after that), so its result is then the last one computed.
// Bitwise the result of the corresponding gemm_f64 launches.
// ---------------------------------------------------------------------------
constexpr int CHAIN_SMALL_MAX_N = 128;
struct ChainSmallArgs {
  int N = 0, batch = 0, nslices = 0, dir = 1, lo = 1, hi = 1;
  const double* E = nullptr; int transE = 0;
  const double* X = nullptr; long long sX = 0;
  double* C = nullptr; long long sC = 0;
  const double* expV = nullptr; long long sV = 0, sV_inner = 0; int divS = 1;
  const int* lim = nullptr; int lim_base = 1;
};
cudaError_t chain_small(const ChainSmallArgs& a, cudaStream_t st);

// ---------------------------------------------------------------------------
// Column-pivoted Householder QR, one CTA per instance (Sec. 4.2.2).
//   Y = A diag(Din) ;  Y P = Q R ;  U = Q, D = |diag R|, T = D^{-1} R (upper,
//   pivoted column order, zeros below the diagonal), perm = P as an index map.
// W is an N x N workspace per instance.
// ---------------------------------------------------------------------------
struct QrpArgs {
  int N = 0, batch = 0;
  const double* A = nullptr; long long sA = 0;
  const double* Din = nullptr; long long sDin = 0;   // nullable
  double* W = nullptr; long long sW = 0;
  double* U = nullptr; long long sU = 0;
  double* D = nullptr; long long sD = 0;
  double* T = nullptr; long long sT = 0;
  int* perm = nullptr; long long sperm = 0;
  int* status = nullptr; int status_div = 1;          // nullable
  const int* lim = nullptr; int lim_at = 0;           // skip instance b when lim[b] < lim_at
  int smem_mats = 0;                                  // set by the launcher
  int share_sm = 0;   // N <= 256: the register-capped kernel that fits beside an FP64 GEMM CTA
};

cudaError_t qrp_f64(const QrpArgs& a, cudaStream_t st);

// One-sided Jacobi SVD, one CTA per instance (jacobi_f64.cu):
//   A diag(Din) = U diag(D) V^T,  V^T written to Vt (row-major); W is an N x N
// workspace per instance.  N <= 512.
struct JacobiArgs {
  int N = 0, batch = 0, max_sweeps = 60;
  const double* A = nullptr; long long sA = 0;
  const double* Din = nullptr; long long sDin = 0;   // nullable
  double* W = nullptr; long long sW = 0;
  double* U = nullptr; long long sU = 0;
  double* D = nullptr; long long sD = 0;
  double* Vt = nullptr; long long sVt = 0;
  int* status = nullptr; int status_div = 1;          // nullable
  const int* lim = nullptr; int lim_at = 0;           // skip instance b when lim[b] < lim_at
};

cudaError_t jacobi_svd_f64(const JacobiArgs& a, cudaStream_t st);

// ---------------------------------------------------------------------------
// LU with partial pivoting and solve, one CTA per instance:
//   opA(A) Z = opR(R)   (A: N x N, R: N x nrhs), Z stored as opZ.
// Optionally R is a diagonal given as a vector (Rdiag, N entries) instead of
// a dense matrix.  Returns log|det opA(A)| and its sign per instance.
// Work: N x (N + nrhs) per instance.
// ---------------------------------------------------------------------------
struct LuArgs {
  int N = 0, nrhs = 0, batch = 0;
  const double* A = nullptr; long long sA = 0; int transA = 0;
  const double* R = nullptr; long long sR = 0; long long ldr = 0; int transR = 0;
  const double* Rdiag = nullptr; long long sRdiag = 0; int invRdiag = 0;
  double* Z = nullptr; long long sZ = 0; long long ldz = 0; int transZ = 0;
  double* W = nullptr; long long sW = 0;
  double* logabsdet = nullptr; int* sign = nullptr;   // per instance, nullable
  int* status = nullptr; int status_div = 1;
  int smem_w = 0;                                     // set by the launcher
};

cudaError_t lu_solve_f64(const LuArgs& a, cudaStream_t st);

// ---------------------------------------------------------------------------
// Element-wise helpers.
// ---------------------------------------------------------------------------
// out[i] = exp(sgn * v[i]) for n entries; flags non-finite inputs per instance
// (instance = i / per_instance) in status.
cudaError_t exp_vec(const double* v, double* out, long long n, double sgn,
                    long long per_instance, int* status, cudaStream_t st);
// C = rowscale1 * A * colscale1 + rowscale2 * B * colscale2, per instance,
// scales given as (Dsplit mode, vector) pairs; see elementwise.cu.
struct Axpby2Args {
  int N = 0, batch = 0;
  const double* A = nullptr; long long sA = 0;
  const double* B = nullptr; long long sB = 0;
  double* C = nullptr; long long sC = 0;
  // each scale: pointer to a D vector + mode (0: none, 1: 1/max(D,1),
  // 2: min(D,1), 3: max(D,1), 4: 1/D, 5: D)
  const double* ra = nullptr; int ra_mode = 0; long long sra = 0;
  const double* ca = nullptr; int ca_mode = 0; long long sca = 0;
  const double* rb = nullptr; int rb_mode = 0; long long srb = 0;
  const double* cb = nullptr; int cb_mode = 0; long long scb = 0;
  int divA = 1, divB = 1, divC = 1, divRA = 1, divCA = 1, divRB = 1, divCB = 1;
};
cudaError_t axpby2(const Axpby2Args& a, cudaStream_t st);
// out[b*n + i] = f(D[b*sD + i]) with mode as in Axpby2Args (4: 1/D).
cudaError_t dsplit_vec(const double* D, long long sD, int n, int batch, double* out, int mode,
                       cudaStream_t st);
// exp(sgn*V) of a batch x M x N field into a batch x Mp x N array (padding = 1);
// with shift (device, per instance) slice l is taken from slice l + shift[b] mod M.
cudaError_t exp_pad(const double* V, double* out, int batch, int M, int Mp, int N, double sgn,
                    int* status, cudaStream_t st, const int* shift = nullptr);
// y = 1 - diag(G) for a batch of N x N matrices; y_b at y + b*sy.
cudaError_t one_minus_diag(const double* G, long long sG, int N, int batch,
                           double* y, long long sy, int ydiv, long long sy_outer,
                           cudaStream_t st);
// logdet_b = sum_i log max(D_bi, 1) + logabsdet_b (plain: sum_i log D_bi + ...);
// sign_b = s1_b * s2_b; flags non-finite results.
cudaError_t finish_logdet(const double* D, long long sD, int N, int batch, const double* lad,
                          const int* s1, const int* s2, double* logdet, int* sign,
                          int* status, cudaStream_t st, int plain = 0);
// Copy of strided N x N matrices (out_b = in_b), optional transpose.
cudaError_t copy_mats(const double* in, long long sin, double* out, long long sout,
                      int N, int batch, int transpose, int divin, int divout,
                      cudaStream_t st);
// A_b <- diag(v_b) A_b for strided N x N matrices.
cudaError_t scale_rows(double* A, long long sA, const double* v, long long sv, int N, int batch,
                       cudaStream_t st);
// Identity / ones initialisers.
cudaError_t set_identity(double* A, long long sA, int N, int batch, cudaStream_t st);
cudaError_t set_const(double* x, long long n, double v, cudaStream_t st);
cudaError_t chunk_len(int* len, int batch, int P0, int nc, int k, int M, cudaStream_t st);
cudaError_t scatter_tau(const double* cur, long long Q, int nt, int N, int k, int M, int s,
                        double* out, cudaStream_t st);
// 1-norm based scaling for the matrix exponential: s = max(0, ceil(log2(||dtau K||_1 / 0.5))),
// scale = sgn * dtau / 2^s; writes s (int) and scale (double) to device memory;
// also writes the symmetry defect flag into *asym (1 if K != K^T).
// exp(sgn dtau K) for N <= 16 in one CTA (see elementwise.cu); status |= bad_bit
// for every instance when K is not symmetric/finite or needs > max_sq squarings.
cudaError_t expm_small(const double* K, int N, double dtau, double sgn, int terms, int max_sq,
                       double* E, int* asym, int* status, int batch, int bad_bit,
                       cudaStream_t st);
cudaError_t expm_prepare(const double* K, int N, double dtau, double sgn,
                         int* s_out, double* scale_out, int* asym, cudaStream_t st);
// Right-hand sides of the two-stack inversion (see api.cu), problems q = 0..Q-1.
cudaError_t build_rhs(int N, int Q, const double* UF, const double* XF, const double* DF, double* R,
                      int ncols, int want_tt, int want_t0, cudaStream_t st);
// Gradient read-out 1 - G(i,i) of the wrap step s (see api.cu).
cudaError_t grad_readout(const double* G, int N, int Q, int nt, int k, int M, int s, double* dV,
                         cudaStream_t st);
cudaError_t set_const_strided(double* x, long long sx, int n, int batch, double v, cudaStream_t st);
// Ragged batches (ragged.cu).
cudaError_t exp_gather(const double* V, const long long* offV, const int* Mb, int batch, int Mp,
                       int N, double* out, int* status, cudaStream_t st);
cudaError_t scatter_mats(const double* src, const long long* offG, int N, int batch, double* dst,
                         cudaStream_t st);
// Blocks of len doubles between a pool (at offs[b]) and a contiguous batch:
// gather (scatter = 0) pool -> batch, scatter (1) batch -> pool.
cudaError_t move_blocks(const double* src, double* dst, const long long* offs, long long len,
                        int batch, int scatter, cudaStream_t st);
cudaError_t scatter_scalars(const int* gidx, int batch, const double* ld, const int* sg,
                            const int* stt, double* ld_out, int* sg_out, int* st_out,
                            cudaStream_t st);
// Field the status flag of the symmetry check into every instance's status.
cudaError_t or_status(int* status, int batch, const int* flag, int bit, cudaStream_t st);

}  // namespace dqmc

namespace dqmc {
// Equal-time G / log det on a caller-supplied device workspace (api.cu).
dqmc_status greens_on_workspace(void* stream, void* ws, size_t ws_bytes, int batch, int N, int M,
                                const double* K, double dtau, const double* V, int k, double* G,
                                double* logdet, int* sign, int* status);
}  // namespace dqmc

#include <cuda_bf16.h>
namespace dqmc {
// Error-free BF16 slicing and tensor-core slice products (ozaki_tc.cu).
cudaError_t ozaki_split(const double* X, long long ldm, long long ldj, long long sX,
                        const double* sc, long long ssc, int N, int PJ, int PM, int R, int s,
                        __nv_bfloat16* S, long long sS, int* e, long long se, int batch,
                        cudaStream_t st, const int* gm = nullptr, long long sgm = 0);
// lim (nullable, device, per instance) + lim_at: instances with lim[b] < lim_at
// are skipped; when csrc is set their output is the FP64 copy of
// csrc + b * scsrc (the copy-through of ragged chains that have ended).
cudaError_t ozaki_gemm(const __nv_bfloat16* As, const int* eA, long long sA, long long seA,
                       int P128, const __nv_bfloat16* Bs, const int* eB, long long seB, int PN,
                       int PK, int s, int N, int batch, double* C, long long sC, int* status,
                       cudaStream_t st, const int* lim = nullptr, int lim_at = 0,
                       const double* csrc = nullptr, long long scsrc = 0);
int oz_groups(int s, int N);
// One CTA of ozaki_gemm_kernel whose loads are never issued: its bounded
// waits run out and it ORs DQMC_STATUS_TIMEOUT into *status (device int).
cudaError_t ozaki_selftest_timeout(int* status, cudaStream_t st);
}  // namespace dqmc

// ---------------------------------------------------------------------------
// Device-side checks of the debug build (sources compiled with -DDQMC_DEBUG
// into the separate debug library).
//
// DQMC_CHECK(cond, value) evaluates cond; when it is false it records
// (source line, low 32 bits of value) in this translation unit's check word
// (the first failure since the word was last cleared is kept) and yields
// false, so the caller skips the access or leaves the kernel.  It never
// traps.  In the release build it is the constant true and cond is not
// evaluated, so the checks cost nothing there.  A device variable belongs to
// the module of its translation unit (no relocatable device code), so every
// unit has its own word; DQMC_CHECK_UNIT(name) at the end of a .cu file
// defines the host reader dqmc::check_word_<name>, which the debug read-out
// of api.cu calls for each unit.
// ---------------------------------------------------------------------------
namespace dqmc {
// Rows of a lane in the small-N kernels (qrp_small_kernel, lu_small_kernel):
// register index k as a compile-time constant.
template <int I>
struct RowIdx {
  static constexpr int value = I;
};

// f(RowIdx<k>{}) for k = k0 .. NK-1 (k0 warp-uniform): the rows below k0 are
// skipped by a jump, not predicated, because a predicated FP64 warp
// instruction still holds its sub-partition's pipe for 64 cycles
template <int NK, class F>
__device__ __forceinline__ void ks_from(int k0, F&& f) {
  static_assert(NK >= 1 && NK <= 16, "at most 16 rows per lane");
  if constexpr (NK <= 2) {
    if (k0 <= 0) f(RowIdx<0>{});
    if constexpr (NK > 1) if (k0 <= 1) f(RowIdx<1>{});
    return;
  }
  switch (k0) {
    case 0: f(RowIdx<0>{}); [[fallthrough]];
    case 1: if constexpr (NK > 1) f(RowIdx<1>{}); [[fallthrough]];
    case 2: if constexpr (NK > 2) f(RowIdx<2>{}); [[fallthrough]];
    case 3: if constexpr (NK > 3) f(RowIdx<3>{}); [[fallthrough]];
    case 4: if constexpr (NK > 4) f(RowIdx<4>{}); [[fallthrough]];
    case 5: if constexpr (NK > 5) f(RowIdx<5>{}); [[fallthrough]];
    case 6: if constexpr (NK > 6) f(RowIdx<6>{}); [[fallthrough]];
    case 7: if constexpr (NK > 7) f(RowIdx<7>{}); [[fallthrough]];
    case 8: if constexpr (NK > 8) f(RowIdx<8>{}); [[fallthrough]];
    case 9: if constexpr (NK > 9) f(RowIdx<9>{}); [[fallthrough]];
    case 10: if constexpr (NK > 10) f(RowIdx<10>{}); [[fallthrough]];
    case 11: if constexpr (NK > 11) f(RowIdx<11>{}); [[fallthrough]];
    case 12: if constexpr (NK > 12) f(RowIdx<12>{}); [[fallthrough]];
    case 13: if constexpr (NK > 13) f(RowIdx<13>{}); [[fallthrough]];
    case 14: if constexpr (NK > 14) f(RowIdx<14>{}); [[fallthrough]];
    case 15: if constexpr (NK > 15) f(RowIdx<15>{}); [[fallthrough]];
    default: break;
  }
}

}  // namespace dqmc

namespace dqmc {
// Bytes of dynamic shared memory the running kernel was launched with.
__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
}  // namespace dqmc

#ifdef DQMC_DEBUG
namespace dqmc {
static __device__ unsigned long long g_check_word;
static __device__ __noinline__ void check_failed(int line, long long value) {
  const unsigned long long w = (1ull << 63) | ((unsigned long long)(line & 0x7fffffff) << 32) |
                               (unsigned long long)(unsigned int)value;
  atomicCAS(&g_check_word, 0ull, w);
}
}  // namespace dqmc
#define DQMC_CHECK(cond, value) \
  ((cond) ? true : (::dqmc::check_failed(__LINE__, (long long)(value)), false))
#define DQMC_CHECK_UNIT(name)                                                      \
  namespace dqmc {                                                                 \
  unsigned long long check_word_##name(bool clear) {                               \
    unsigned long long w = 0;                                                      \
    if (cudaMemcpyFromSymbol(&w, g_check_word, sizeof w) != cudaSuccess) {         \
      cudaGetLastError();                                                          \
      return ~0ull;                                                                \
    }                                                                              \
    if (clear && w) {                                                              \
      const unsigned long long z = 0;                                              \
      if (cudaMemcpyToSymbol(g_check_word, &z, sizeof z) != cudaSuccess) cudaGetLastError(); \
    }                                                                              \
    return w;                                                                      \
  }                                                                                \
  }
#else
#define DQMC_CHECK(cond, value) true
#define DQMC_CHECK_UNIT(name)
#endif
