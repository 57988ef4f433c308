/*
 * dqmc.h -- C ABI of the GB300 library for stabilised DQMC Green's functions.
 *
 * What the library computes (C. Bauer, "Fast and stable determinant quantum
 * Monte Carlo", SciPost 2020):
 *
 *   slice matrices      B_l = exp(-dtau K) exp(V_l),  l = 1..M           (Sec. 2, Eq. (Ztr))
 *   equal-time G        G = [1 + B_M ... B_1]^{-1}                        (Sec. 2, Eq. (etgf))
 *   weight              log|det(1 + B_M ... B_1)| = -log|det G|, sign    (Sec. 2, Eqs. (DQMC), (metropolis))
 *   time-displaced G    G(tau_1, 0) = B_{l_1} ... B_1 G                   (Sec. 6, Eq. (tdgf_propagate))
 *   gradient            d log|det(1 + B_M...B_1)| / dV_l(i) = 1 - G_l(i,i), with
 *                       G_l = [1 + B_{l-1}...B_1 B_M...B_l]^{-1}          (Sec. 6, Eq. (etgf_tau))
 *
 * computed the stable way the paper prescribes: naive products of k slices,
 * re-factorised after every chunk by a column-pivoted Householder QR into a
 * U D T stack (Sec. 4, Eq. (stabmult)), and inverted with Loh's D+/D- split
 * (Sec. 5, Eq. (inversion_loh); Sec. 6, Eq. (inversion_tdgf_loh)).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All floating point data are IEEE binary64 (double), row-major:
 *   element (i, j) of an N x N matrix is at [i*N + j].
 * - K: N x N real symmetric hopping matrix, shared by all instances of a call.
 * - V: batch x M x N; V[(b*M + (l-1))*N + i] is the diagonal entry i of V_l of
 *   instance b (slice l contiguous).  B_l = exp(-dtau K) diag(exp(V_l)).
 * - k: stabilisation interval, 1 <= k <= M.  Chunks are slices
 *   [c*k+1, min((c+1)*k, M)], so the last chunk may be shorter.
 * - The k-grid is tau_j = min(j*k, M) * dtau, j = 0 .. n_tau-1, with
 *   n_tau = ceil(M/k) + 1.
 * - Pointer mode (dqmc_set_pointer_mode): DQMC_PTR_DEVICE (default) -- every
 *   array argument is a device pointer owned by the caller and the call is
 *   asynchronous on the handle's stream; DQMC_PTR_HOST -- every array
 *   argument is a host pointer, the library copies inputs in and outputs out
 *   through its own device workspace and the call returns after the results
 *   are in host memory.
 * - Errors: the return value reports what is known synchronously (arguments,
 *   allocation, launch).  Numerical trouble found on the device is written to
 *   the optional per-instance status array (bit mask of dqmc_status_bits);
 *   0 means the instance is fine.  No entry point aborts, traps or throws.
 * - Thread safety: a handle must not be used by two host threads at once.
 *   Different handles are independent.
 */
#ifndef DQMC_H
#define DQMC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DQMC_OK = 0,
  DQMC_ERR_ARG = 1,        /* invalid argument (size, pointer, alignment, mode) */
  DQMC_ERR_CUDA = 2,       /* a CUDA runtime call or kernel launch failed */
  DQMC_ERR_NOMEM = 3,      /* device workspace could not be allocated */
  DQMC_ERR_NONFINITE = 4,  /* (status bit) NaN/Inf in an input or a result */
  DQMC_ERR_SINGULAR = 5,   /* (status bit) exactly singular pivot */
  DQMC_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up */
  DQMC_ERR_UNSUPPORTED = 7, /* configuration not built into this library */
  DQMC_ERR_SCRATCH = 8,     /* dqmc_greens_noalloc: problem needs more than its fixed scratch */
  DQMC_ERR_CHECK = 9        /* debug build: a device-side check failed (dqmc_debug_read) */
} dqmc_status;

/* Bits of the per-instance device status word. */
enum dqmc_status_bits {
  DQMC_STATUS_NONFINITE_INPUT = 1 << 0,  /* V contained NaN/Inf */
  DQMC_STATUS_NONFINITE_SCALE = 1 << 1,  /* a D scale overflowed or became NaN */
  DQMC_STATUS_SINGULAR = 1 << 2,         /* an LU pivot or QR diagonal was exactly 0 */
  DQMC_STATUS_NONFINITE_OUTPUT = 1 << 3, /* G or log det is not finite */
  DQMC_STATUS_BAD_K = 1 << 4,            /* K not symmetric/finite, or ||dtau K||_1 > 2048 */
  DQMC_STATUS_TIMEOUT = 1 << 5,          /* a bounded wait of a tensor-core kernel gave up */
  DQMC_STATUS_NOT_CONVERGED = 1 << 6     /* the Jacobi SVD stabiliser hit its sweep limit */
};

/* Precision of the k-slice chain products (a mixed-precision option; the
 * pivoted QR, the D splits and the inversions always run in FP64).
 * DQMC_CHAIN_BF16Xs: each FP64 operand is written in s balanced base-128
 * digits held in BF16 (error-free splitting with power-of-two row/column
 * scales), the digit products accumulate exactly in FP32 on the tcgen05
 * tensor cores and are recombined in FP64; a product is accurate to about
 * N 2^{-7s-1} of (row max x column max), normwise rather than elementwise.
 * Supported for N <= 256 in dqmc_greens, dqmc_logdet, dqmc_greens_tdisplaced,
 * dqmc_logdet_grad (both stacks) and dqmc_greens_ragged (every instance N <= 256);
 * N > 256 returns DQMC_ERR_UNSUPPORTED (dqmc_greens_noalloc takes no handle
 * and is FP64). */
typedef enum {
  DQMC_CHAIN_FP64 = 0,
  DQMC_CHAIN_BF16X3 = 3,
  DQMC_CHAIN_BF16X4 = 4,
  DQMC_CHAIN_BF16X5 = 5,
  DQMC_CHAIN_BF16X6 = 6,
  DQMC_CHAIN_BF16X7 = 7,
  DQMC_CHAIN_BF16X8 = 8
} dqmc_chain_prec;

typedef enum { DQMC_PTR_DEVICE = 0, DQMC_PTR_HOST = 1 } dqmc_pointer_mode;

typedef struct dqmc_handle_s* dqmc_handle;

/* Creates a handle bound to the current CUDA device and to the legacy default
 * stream.  The handle owns a grow-only device workspace (allocated on first
 * use, freed by dqmc_destroy).  *h is set to NULL on failure. */
dqmc_status dqmc_create(dqmc_handle* h);
dqmc_status dqmc_destroy(dqmc_handle h);
/* stream: a cudaStream_t (NULL = legacy default stream). */
dqmc_status dqmc_set_stream(dqmc_handle h, void* stream);
dqmc_status dqmc_set_pointer_mode(dqmc_handle h, dqmc_pointer_mode mode);
dqmc_status dqmc_set_chain_precision(dqmc_handle h, dqmc_chain_prec prec);
/* CUDA-graph mode (default off).  When on, a call of dqmc_greens, dqmc_logdet,
 * dqmc_greens_tdisplaced or dqmc_logdet_grad is recorded by stream capture and
 * launched as one CUDA graph; the next call with identical arguments (same
 * pointers, sizes, dtau, k) and settings replays that graph without any
 * per-kernel launch, which is what makes small problems fast.  The graph
 * reads its inputs when it runs: write new fields into the same V buffer to
 * get new results.  A call with different arguments is captured again (the
 * executable graph is updated in place when its shape allows).  Results are
 * bitwise identical to graph mode off.  dqmc_greens_ragged is recorded the
 * same way (keyed by its descriptor contents and pointers; the host-side
 * grouping and the upload of its index tables happen before the recording,
 * not in the graph).  Host pointer mode and the profiler always run without a
 * graph.  The stream may be the legacy default stream. */
dqmc_status dqmc_set_graph_mode(dqmc_handle h, int enable);
/* Tile edge of the FP64 products: 0 = chosen by size (default: the edge that
 * pads N least), 32, 48 or 64.  A tuning knob for the autotuner
 * (paper_2003_05286_gb300/tune.py); results do not depend on it. */
dqmc_status dqmc_set_gemm_tile(dqmc_handle h, int tile);

/* How the equal-time chain of dqmc_greens / dqmc_logdet is folded (FP64
 * chain precision only; the other calls and the mixed precisions always run
 * the sequential chain):
 *   DQMC_FOLD_SEQUENTIAL  chunk after chunk, Eq. (stabmult) with the running
 *                         U D X (one pivoted QR per chunk, in order);
 *   DQMC_FOLD_TREE        all chunk products at once, each decomposed, then
 *                         neighbours combined pairwise by Eq. (stabmult)
 *                         (U_2 D_2 X_2)(U_1 D_1 X_1) = (U_2 u) d (x X_1),
 *                         u d x = udt(D_2 (X_2 U_1) D_1), in ceil(log2(ceil(M/k)))
 *                         levels: fewer dependent steps, more arithmetic;
 *   DQMC_FOLD_AUTO        (default) tree when batch * ceil(M/k) is at most
 *                         the device's SM count (152 on GB300) and
 *                         ceil(M/k) >= 4, else sequential.
 * Both give G and log det of the same definition; they differ by rounding.
 * Invalid mode: DQMC_ERR_ARG. */
typedef enum { DQMC_FOLD_SEQUENTIAL = 0, DQMC_FOLD_TREE = 1, DQMC_FOLD_AUTO = 2 } dqmc_fold_mode;
dqmc_status dqmc_set_chain_fold(dqmc_handle h, int mode);

/* Inversion scheme (Sec. 5.1 and Sec. 6.1):
 *   DQMC_INV_LOH    (default) the D+/D- split of Loh et al.: Eq. (inversion_loh)
 *                   for G and log det, Eq. (inversion_tdgf_loh) for G(tau,0);
 *   DQMC_INV_PLAIN  the schemes without the split: Eq. (inversion) for G and
 *                   log det of dqmc_greens, dqmc_logdet and dqmc_greens_ragged,
 *                   and Eq. (inversion_tdgf) for G(tau,0) of the time-displaced
 *                   calls, its two terms first brought to U D X form with an
 *                   orthogonal left factor (one pivoted QR each).  G(tau,tau),
 *                   G(0,tau), the gradient and dqmc_greens_noalloc keep Loh.
 * PLAIN exists to reproduce the paper's comparison: for G(tau,0) it loses
 * accuracy at tau ~ beta/2 (Sec. 6.2.1), while both equal-time schemes agree
 * (Sec. 5.2).  Invalid scheme: DQMC_ERR_ARG. */
typedef enum { DQMC_INV_LOH = 0, DQMC_INV_PLAIN = 1 } dqmc_inversion_scheme;
dqmc_status dqmc_set_inversion_scheme(dqmc_handle h, int scheme);

/* Decomposition that stabilises the chains (Sec. 4.2):
 *   DQMC_DECOMP_QR      (default) column-pivoted Householder QR, U D X with X
 *                       triangular up to the pivot permutation (Sec. 4.2.2);
 *   DQMC_DECOMP_JACOBI  one-sided Jacobi SVD, U D V^T with X = V^T orthogonal
 *                       (the accurate SVD variant of Sec. 4.2.1); about ten
 *                       sweeps of N^2/2 plane rotations each, so 10-50x the
 *                       QR's cost: an accuracy reference, not a fast path.
 * Applies to every chain (equal-time, both stacks, ragged); the tree fold
 * and the intermediate decompositions of the inversion schemes keep QR.
 * JACOBI needs the FP64 chain precision (else DQMC_ERR_UNSUPPORTED at the
 * call) and N <= 512.  A decomposition that does not converge in 60 sweeps
 * sets DQMC_STATUS_NOT_CONVERGED.  Invalid value: DQMC_ERR_ARG. */
typedef enum { DQMC_DECOMP_QR = 0, DQMC_DECOMP_JACOBI = 1 } dqmc_decomposition;
dqmc_status dqmc_set_decomposition(dqmc_handle h, int decomposition);
/* Number of kernel launches issued by the most recent compute call. */
long long dqmc_last_launch_count(dqmc_handle h);
/* Bytes of device workspace the handle currently holds. */
long long dqmc_workspace_bytes(dqmc_handle h);
/* Device bytes the handle holds in all its grow-only buffers: the workspace,
 * the staging buffer and index tables of the ragged calls, and the two pools
 * of dqmc_register_K. */
long long dqmc_device_bytes(dqmc_handle h);
/* Cap on dqmc_device_bytes; 0 (the default) means none.  A call that would
 * grow a buffer past the cap returns DQMC_ERR_NOMEM without allocating and
 * without releasing the buffer it would have replaced, so the handle stays
 * usable for problems that fit; what that call had already written to its
 * outputs is unspecified.  Lowering the cap keeps the buffers already held.
 * It bounds the library's memory inside a larger application, and it is how
 * the tests drive the allocation-failure paths without exhausting the
 * device.  bytes < 0: DQMC_ERR_ARG. */
dqmc_status dqmc_set_memory_limit(dqmc_handle h, long long bytes);
const char* dqmc_status_string(dqmc_status s);

/* Per-kernel-class timing of subsequent compute calls: every launch of the
 * class is bracketed by CUDA events recorded on the handle's stream.  Classes:
 * 0 slice-chain GEMM (Eq. (Ztr)), 1 pivoted QR (Sec. 4.2.2), 2 X <- T X update
 * (Eq. (stabmult)), 3 LU solves of the inversions, 4 everything else.
 * dqmc_profile_read synchronises the stream and returns the summed event
 * time (ms), the launch count and the algorithmic FP64 flops of the class
 * since the last reset (any output pointer may be NULL). */
dqmc_status dqmc_profile_enable(dqmc_handle h, int enable);
dqmc_status dqmc_profile_reset(dqmc_handle h);
dqmc_status dqmc_profile_read(dqmc_handle h, int cls, double* ms, long long* launches,
                              double* flops);

/* Equal-time Green's function G = [1 + B_M ... B_1]^{-1} (Eq. (etgf)) of each
 * of `batch` instances, with log|det(1 + B_M...B_1)| and its sign.
 *   K      [N*N]            input
 *   V      [batch*M*N]      input
 *   G      [batch*N*N]      output (may be NULL: then only logdet/sign)
 *   logdet [batch]          output, may be NULL
 *   sign   [batch] int32    output (+1/-1), may be NULL
 *   status [batch] int32    output bit mask, may be NULL
 * 1 <= N <= 1024, 1 <= M, 1 <= k <= M, batch >= 0 (0 is a no-op). */
dqmc_status dqmc_greens(dqmc_handle h, int batch, int N, int M, const double* K,
                        double dtau, const double* V, int k, double* G,
                        double* logdet, int* sign, int* status);

/* log|det(1 + B_M...B_1)| and sign only (Eq. (DQMC)); same arguments. */
dqmc_status dqmc_logdet(dqmc_handle h, int batch, int N, int M, const double* K,
                        double dtau, const double* V, int k, double* logdet,
                        int* sign, int* status);

/* Time-displaced Green's functions on the k-grid (Sec. 6):
 *   Gtt [batch*n_tau*N*N]  G(tau_j, tau_j) = G_{l_j + 1}   (Eq. (etgf_tau)), may be NULL
 *   Gt0 [batch*n_tau*N*N]  G(tau_j, 0) = B_{l_j}...B_1 G_1 (Eq. (tdgf_propagate)), may be NULL
 * with l_j = min(j*k, M); entry (b, j, i, m) at ((b*n_tau + j)*N + i)*N + m.
 * Both come from the forward stack B(tau_j, 0) = U D X and the backward stack
 * B(beta, tau_j)^T = U D T (App. A) through one D+/D- split inversion per
 * tau_j (Eq. (inversion_tdgf_loh)). */
dqmc_status dqmc_greens_tdisplaced(dqmc_handle h, int batch, int N, int M,
                                   const double* K, double dtau, const double* V,
                                   int k, double* Gtt, double* Gt0, int* status);

/* As dqmc_greens_tdisplaced, plus the other time order on the same k-grid
 * (second case of Eq. (tdgf_propagate), Sec. 6):
 *   G0t [batch*n_tau*N*N]  G(0, tau_j) = -(1 - G_1) (B_{l_j}...B_1)^{-1}, may be NULL,
 * same layout as Gtt.  j = 0 holds the limit tau -> 0^+, -(1 - G_1), and
 * j = n_tau - 1 holds G(0, beta) = -G_1.  With B(tau,0) = U_F a X_F and
 * B(beta,tau)^T = U_b b T_b from the two stacks,
 *   G(0,tau) = -[B(tau,0) + B(beta,tau)^{-1}]^{-1} = -T_b^T b_m mid^{-1} a_p^{-1} U_F^T,
 * where mid is the D+/D- split middle matrix that G(tau,0) inverts and the
 * solve mid^{-1} a_p^{-1} U_F^T is the one G(tau,tau) uses: G0t costs one
 * N x N product per tau_j on top of Gtt.  Arguments, errors and status as in
 * dqmc_greens_tdisplaced. */
dqmc_status dqmc_greens_tdisplaced_ex(dqmc_handle h, int batch, int N, int M,
                                      const double* K, double dtau, const double* V,
                                      int k, double* Gtt, double* Gt0, double* G0t,
                                      int* status);

/* The same three functions at every tau_l = l dtau, l = 0..M (not only on the
 * k-grid):  Gtt, Gt0, G0t [batch*(M+1)*N*N], entry (b, l, i, m) at
 * ((b*(M+1) + l)*N + i)*N + m, each may be NULL.  Between grid points the
 * values are propagated from the stable grid values by at most k-1 one-slice
 * products (the mixture of stabilised and naive products of Sec. 4.1):
 *   G(tau_l, 0) = B_l G(tau_{l-1}, 0),   G(0, tau_l) = G(0, tau_{l-1}) B_l^{-1},
 *   G_{l+1} = B_l G_l B_l^{-1}            (Eqs. (tdgf_propagate), (etgf_tau)).
 * Values on the grid equal those of dqmc_greens_tdisplaced_ex bitwise.
 * Arguments, errors and status as in dqmc_greens_tdisplaced. */
dqmc_status dqmc_greens_tdisplaced_all(dqmc_handle h, int batch, int N, int M,
                                       const double* K, double dtau, const double* V,
                                       int k, double* Gtt, double* Gt0, double* G0t,
                                       int* status);

/* Time-displaced Green's functions from another origin tau_{l0}: for instance
 * b with origin l0[b] (0 <= l0[b] < M; l0 is a device array, or host in host
 * pointer mode), on the grid d_j = min(j k, M) dtau (every_tau = 0, n_tau
 * entries) or at every d_l = l dtau (every_tau != 0, M + 1 entries):
 *   Gtt[j] = G(tau_{l0} + d_j, tau_{l0} + d_j),
 *   Gt0[j] = G(tau_{l0} + d_j, tau_{l0}),   G0t[j] = G(tau_{l0}, tau_{l0} + d_j),
 * layouts as in dqmc_greens_tdisplaced(_all).  This is the computation from
 * origin 0 on the cyclically shifted chain (slice m taken as B_{m + l0}):
 * the products of Eq. (etgf_tau) and of the two cases of Eq. (tdgf_propagate)
 * depend only on that cyclic order.  Times past beta continue anti-periodically,
 * G(tau + beta, tau') = -G(tau, tau').  Together with l0 over the grid this
 * gives G(tau_1, tau_2) for every pair of grid times. */
dqmc_status dqmc_greens_tdisplaced_from(dqmc_handle h, int batch, int N, int M,
                                        const double* K, double dtau, const double* V,
                                        int k, const int* l0, int every_tau, double* Gtt,
                                        double* Gt0, double* G0t, int* status);

/* Gradient dV[(b*M + (l-1))*N + i] = d log|det(1 + B_M...B_1)| / dV_l(i)
 * = 1 - G_l(i,i) for every slice l (derived from Eqs. (etgf), (etgf_tau)):
 * G_l at the k-grid from the two stacks, then G_{l+1} = B_l G_l B_l^{-1}
 * between grid points.  logdet/sign/status as in dqmc_greens (may be NULL). */
dqmc_status dqmc_logdet_grad(dqmc_handle h, int batch, int N, int M,
                             const double* K, double dtau, const double* V,
                             int k, double* logdet, int* sign, double* dV,
                             int* status);

/* Ragged batch: instances of different N, M, k, dtau and K in one call.
 * desc is a HOST array of `batch` descriptors; offsets are in doubles into
 * the pools (K_pool holds each instance's N*N hopping matrix at off_K,
 * V_pool its M*N field at off_V, G_pool its N*N output at off_G).
 * Instances with equal (N, k, dtau, off_K) run as one batched chain (their M
 * may differ): instances with the same hopping matrix should point at one
 * copy of it.  logdet/sign/status are indexed by instance and may be NULL.
 * The chain precision of the handle applies (a mixed precision needs every
 * N <= 256); in CUDA-graph mode an identical second call (same descriptor
 * contents, pools and outputs) is a single graph launch.  The call
 * synchronises the handle's stream when it sees a descriptor set different
 * from the previous ragged call's (to upload the per-group index tables). */
typedef struct {
  int N, M, k, pad;
  double dtau;
  long long off_K, off_V, off_G;
} dqmc_instance;

dqmc_status dqmc_greens_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                               const double* K_pool, const double* V_pool,
                               double* G_pool, double* logdet, int* sign,
                               int* status);

/* Registered hopping matrices and device-resident descriptors (the batched
 * form of the problem statement, Sec. 2: G = [1 + B_M ... B_1]^{-1} with
 * B_l = exp(-dtau K) exp(V_l) for many instances that share a few K).
 *
 * dqmc_register_K copies the N x N hopping matrix K (a device pointer, or a
 * host pointer in host pointer mode) into the handle, computes
 * E = exp(-dtau K) once (Taylor series with scaling and squaring, Sec. 2), and
 * returns its id in *K_id (0, 1, ... in registration order).  Synchronous.
 * Errors: DQMC_ERR_ARG for bad sizes/pointers, or a K that is not symmetric,
 * not finite or has ||dtau K||_1 > 2048 (then nothing is registered);
 * DQMC_ERR_NOMEM; DQMC_ERR_UNSUPPORTED inside a stream capture.  Registered
 * matrices live until dqmc_destroy. */
dqmc_status dqmc_register_K(dqmc_handle h, int N, const double* K, double dtau, int* K_id);

/* One instance of dqmc_greens_batched: its size N (that of the registered
 * K_id), M slices, stabilisation interval k, and offsets in doubles of its
 * M x N field in V_pool and of its N x N output in G_pool. */
typedef struct {
  int N, M, k, K_id;
  long long off_V, off_G;
} dqmc_desc;

/* Equal-time G, log det and sign of `batch` instances described by a DEVICE
 * array of dqmc_desc (device pointer mode only).  dtau and exp(-dtau K) come
 * from the registration of each K_id.  The call reads the descriptors back to
 * the host once (after the work already queued on the handle's stream; this
 * synchronises the stream), groups instances of equal (N, k, K_id), and runs
 * them as dqmc_greens_ragged does (same kernels, same results for the same
 * exponentials; CUDA-graph replay in graph mode; the handle's chain
 * precision).  logdet, sign, status [batch] may be NULL.  Errors: DQMC_ERR_ARG
 * (unknown K_id, N that does not match it, bad sizes), DQMC_ERR_UNSUPPORTED
 * (host pointer mode, inside a capture, mixed precision with N > 256). */
dqmc_status dqmc_greens_batched(dqmc_handle h, int batch, const dqmc_desc* desc,
                                const double* V_pool, double* G_pool, double* logdet, int* sign,
                                int* status);

/* Ragged time-displaced G: instances of different N, M, k, dtau and K in one
 * call, pools and descriptors as for dqmc_greens_ragged.  Instance b writes
 * its n_tau(M_b, k_b) x N_b x N_b values of G(tau_j, tau_j) to Gtt_pool and of
 * G(tau_j, 0) to Gt0_pool, both at desc[b].off_G (either pool may be NULL).
 * Instances with equal (N, M, k, dtau, off_K) run as one batch of the uniform
 * path (dqmc_greens_tdisplaced); the groups run one after another, staged in
 * a second handle-owned device buffer.  status (may be NULL) is indexed by
 * instance.  Host pointer mode: DQMC_ERR_UNSUPPORTED. */
dqmc_status dqmc_greens_tdisplaced_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                                          const double* K_pool, const double* V_pool,
                                          double* Gtt_pool, double* Gt0_pool, int* status);

/* As dqmc_greens_tdisplaced_ragged, plus G(0, tau_j) of each instance in
 * G0t_pool at desc[b].off_G (see dqmc_greens_tdisplaced_ex; may be NULL). */
dqmc_status dqmc_greens_tdisplaced_ragged_ex(dqmc_handle h, int batch, const dqmc_instance* desc,
                                             const double* K_pool, const double* V_pool,
                                             double* Gtt_pool, double* Gt0_pool,
                                             double* G0t_pool, int* status);

/* Ragged log-det gradient: as dqmc_logdet_grad per instance, grouped as in
 * dqmc_greens_tdisplaced_ragged.  Instance b writes its M_b x N_b gradient
 * (layout of its V) to dV_pool at desc[b].off_G; logdet, sign and status (each
 * may be NULL) are indexed by instance. */
dqmc_status dqmc_logdet_grad_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                                    const double* K_pool, const double* V_pool, double* logdet,
                                    int* sign, double* dV_pool, int* status);

/* Allocation-free variant of dqmc_greens, for callers that cannot allocate
 * device memory (an application or pool that owns the whole device budget, a
 * plugin that must not go around its host's allocator, a process with a fixed
 * footprint).  The paper has no counterpart: this is a deployment variant.
 *
 * Same computation and arguments as dqmc_greens (device pointers only; the
 * caller passes inputs and outputs), but there is no handle: the call runs on
 * `stream` (a cudaStream_t, NULL = legacy default stream) of the current
 * device, and every intermediate lives in a file-scope device array of
 * 32 MiB (32 * 2^20 bytes) that each GPU loading the library holds until the
 * process exits.  The call issues no cudaMalloc, cudaFree or other allocating
 * routine.
 *   - Size limit: with r(x) = x rounded up to a multiple of 256 and
 *     Mp = (ceil(M/k) + 1) * k, the intermediates take
 *       S = 2 r(8N^2) + 768 + r(8 Mp N b) + 9 r(8 N^2 b) + r(16 N^2 b)
 *           + 2 r(8 N b) + r(4 N b) + r(8 b) + 3 r(4 b)      bytes (b = batch),
 *     which must not exceed 32 MiB = 33554432 bytes (e.g. N=256, M=200, k=10:
 *     batch <= 5; N=64, M=400, k=10: batch <= 58).  Larger problems return
 *     DQMC_ERR_SCRATCH before anything is launched.
 *   - Pointers: K, V, G, logdet, sign and status must be device (or managed)
 *     memory; anything else (a host buffer, pinned or not) returns DQMC_ERR_ARG
 *     before any launch.
 *   - Address of the array: looked up in the current context on every call
 *     (cudaGetSymbolAddress), never cached.  The first call in a context may
 *     load the library's device code, so make that first call before any
 *     stream capture on the device.
 *   - Every call shares the one array, which keeps the previous call's
 *     contents; the call clears what must start at zero itself.  Calls that
 *     overlap on the GPU (other streams, other host threads) race on the array
 *     and must be serialised by the caller.
 * The chain runs unpipelined on the one stream, so it is slower than
 * dqmc_greens for large batches. */
dqmc_status dqmc_greens_noalloc(void* stream, int batch, int N, int M, const double* K,
                                double dtau, const double* V, int k, double* G, double* logdet,
                                int* sign, int* status);

/* Self-test of the bounded device-side waits.  The paper has no counterpart:
 * the only waits in the library are the mbarrier waits of the tensor-core
 * slice product (DQMC_CHAIN_BF16Xs), and each gives up after about 2 s.  This
 * call launches, on `stream` (a cudaStream_t, NULL = legacy default stream),
 * one CTA of that product on internal 64 x 64 operands with its operand loads
 * switched off, so the wait for the first K-block runs out.  The CTA then ORs
 * DQMC_STATUS_TIMEOUT into *status (one device int, owned by the caller, not
 * cleared here), waits (bounded) for copies in flight, frees its tensor memory
 * and exits; the context stays usable.  Asynchronous: synchronise the stream
 * before reading *status; the launch occupies the device for about 6 s.
 * Returns DQMC_ERR_ARG for a NULL status, DQMC_ERR_CUDA if the launch fails. */
dqmc_status dqmc_selftest_wait_timeout(void* stream, int* status);

/* FP64 arithmetic rate of the current device, the denominator of the FP64
 * rooflines.  The paper has no counterpart: this measures the machine.
 *   kind 0  DFMA: fma.rn.f64 on independent chains, 2 flop per lane;
 *   kind 1  DMMA: mma.sync m8n8k4 f64 (512 flop per warp instruction);
 *   kind 2  DMMA: mma.sync m16n8k8 f64 (2048 flop per warp instruction).
 * One warm-up launch and one timed launch of `iters` loop iterations (about
 * 40 MFLOP per iteration for kinds 0 and 1, 160 MFLOP for kind 2) on 4 CTAs
 * of 256 threads per SM, on `stream` (a cudaStream_t, NULL = legacy default
 * stream), timed with CUDA events.  Synchronous: returns the achieved rate in
 * *tflops (TFLOP/s) and the launch time in *ms (may be NULL).  Allocates and
 * frees a small device buffer.  Errors: DQMC_ERR_ARG (NULL tflops, kind not
 * 0..2, iters outside 1..2^24), DQMC_ERR_NOMEM, DQMC_ERR_CUDA. */
dqmc_status dqmc_selftest_fp64_rate(void* stream, int kind, int iters, double* tflops, double* ms);

/* Debug build.  The same sources compiled with -DDQMC_DEBUG give a second
 * library, lib/libdqmc_gb300_debug.so, with the same entry points and the
 * same arithmetic (results are bitwise those of the release library).  Its
 * kernels check, on the device, the invariants their index arithmetic
 * relies on: the launch geometry and the dynamic shared memory their layout
 * needs, leading dimensions that cover their rows, gathered and pivoted row
 * indices inside the matrix, the 16-byte alignment and extent of every bulk
 * copy and vector store, and the tile window of every tensor-core MMA.  A
 * failed check never traps: it records (source file, line, the offending
 * value) -- the first failure per source file is kept -- and the thread
 * skips the access or the CTA leaves the kernel.  Each launch outside a
 * stream capture is then waited for and the records read, so the call that
 * made it returns DQMC_ERR_CHECK (a graph replay is read after its launch).
 * The debug library is slower (one synchronisation per launch).  The paper
 * has no counterpart: this is a development aid. */
/* 1 in the debug library, 0 in the release library. */
int dqmc_is_debug_build(void);
/* Synchronises the device and returns the first recorded check failure in
 * *file (a static string naming the source file; NULL when none is
 * recorded), *line and *value; clear != 0 resets the records.  Release
 * library: DQMC_ERR_UNSUPPORTED.  NULL outputs: DQMC_ERR_ARG. */
dqmc_status dqmc_debug_read(int clear, const char** file, int* line, int* value);
/* Self-test of the check mechanism (debug library): one CTA of 64 threads
 * writes x[i] = i + 1 into an internal 64-element device array behind the
 * check i < 63, so the last thread's check fails.  *fired = 1 when that
 * failure was recorded with value 63, its write was skipped and every other
 * write happened; *value = the recorded value.  The skipped write would
 * have stayed inside the array.  Synchronous on `stream` (NULL = legacy
 * default stream); clears the records of api.cu.  Release library:
 * DQMC_ERR_UNSUPPORTED. */
dqmc_status dqmc_selftest_check(void* stream, int* fired, int* value);

#ifdef __cplusplus
}
#endif
#endif /* DQMC_H */
