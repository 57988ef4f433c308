// C ABI of the library: handle, workspace, and the launch sequences of the
// stabilised DQMC path.  Every arithmetic step runs in the kernels of this
// library; this file only sizes buffers and orders launches on the handle's
// stream.
//
//   a0  E = exp(-dtau K) (and exp(+dtau K) for the gradient): Taylor series of
//       degree 16 in Horner form on dtau K / 2^s, then s squarings (s from the
//       1-norm, decided on the device so the sequence is graph-capturable).
//   a1  chunk of k slices: A <- E diag(exp V_l) A, one batched GEMM per slice
//       (Sec. 2, Eq. (Ztr); mixture of naive and stabilised products, Sec. 4.1).
//   a2-a4  Eq. (stabmult): (A U) D -> pivoted QR -> U' D' T', X <- T' X.
//   a6-a7  Eq. (inversion_loh) + log det.
//   a8  backward stack on the transposed chain (App. A).
//   a9-a10  G(tau,tau) and G(tau,0) from the two stacks through one D+/D- split
//       middle matrix (Eq. (inversion_tdgf_loh)).
//   a11 gradient 1 - G_l(i,i): checkpoints from the stacks, wrapping in between.
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "common.cuh"

using namespace dqmc;

// Kernel classes of the per-class event profiler (dqmc_profile_*).
enum { PC_CHAIN = 0, PC_QRP = 1, PC_XUPD = 2, PC_LU = 3, PC_OTHER = 4, PC_N = 5 };

struct ProfRec {
  cudaEvent_t e0, e1;
  int cls;
  double flops;
};

struct dqmc_handle_s {
  int device = 0;
  int sms = 152;                           // SM count of the device (queried at creation)
  cudaStream_t stream = nullptr;
  dqmc_pointer_mode pmode = DQMC_PTR_DEVICE;
  dqmc_chain_prec prec = DQMC_CHAIN_FP64;
  int gemm_tile = 0;
  int fold = DQMC_FOLD_AUTO;               // equal-time chain: sequential or tree
  int inv = DQMC_INV_LOH;                  // inversion scheme of G and G(tau,0)
  int decomp = DQMC_DECOMP_QR;             // chain stabiliser
  char* ws = nullptr;
  size_t ws_bytes = 0;
  long long launches = 0;
  cudaStream_t cur = nullptr;              // stream the helpers launch on
  std::vector<cudaStream_t> aux;           // extra streams of the ragged path
  std::vector<cudaEvent_t> auxev;
  // profiler
  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[PC_N] = {0}, prof_flops[PC_N] = {0};
  long long prof_count[PC_N] = {0};
  // CUDA-graph mode: the last call is kept as an instantiated graph and
  // replayed when the next call has identical arguments and settings
  bool graphs = false;
  bool capturing = false;
  size_t ws_need = 0;                      // workspace a capture found missing
  cudaStream_t gstream = nullptr;          // capture stream (the caller's may be the legacy one)
  cudaGraphExec_t gexec = nullptr;
  bool gvalid = false;
  unsigned long long gkey[24] = {0};
  long long glaunches = 0;
  // staging buffer of the grouped ragged calls (kept apart from ws, which the
  // uniform path they call may grow)
  char* rws = nullptr;
  size_t rws_bytes = 0;
  // per-group index tables of dqmc_greens_ragged (chain lengths, instance
  // indices, pool offsets): uploaded before the launches (and before a graph
  // capture) and kept apart from ws; rtab_key is the hash of the descriptor
  // set whose tables the buffer holds, so a replayed graph finds them intact
  char* rtab = nullptr;
  size_t rtab_bytes = 0;
  unsigned long long rtab_key = 0;
  cudaEvent_t rfork = nullptr;
  // hopping matrices registered with dqmc_register_K: K and exp(-dtau K) at
  // equal offsets (in doubles) of two grow-only device pools
  struct KReg { int N; double dtau; long long off; };
  std::vector<KReg> kreg;
  double* kpool = nullptr;
  double* epool = nullptr;
  long long kcap = 0, kused = 0;
  // cap on the device bytes all of the above may hold together (0: none);
  // growth past it fails with DQMC_ERR_NOMEM before any buffer is released
  size_t mem_limit = 0;
};

namespace {

constexpr int EXPM_TERMS = 16;    // Taylor degree; remainder < 0.5^17/17! ~ 2e-20 for ||.||_1 <= 1/2
constexpr int EXPM_SQUARINGS = 12;

// Carves aligned sub-buffers out of the workspace.  With base == nullptr it
// only measures.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(long long n) {
    size_t bytes = ((size_t)(n > 0 ? n : 1) * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += bytes;
    return p;
  }
};

// Device bytes the handle holds in its grow-only buffers.
size_t held_bytes(dqmc_handle h) {
  return h->ws_bytes + h->rws_bytes + h->rtab_bytes + 2 * (size_t)h->kcap * sizeof(double);
}

// Whether replacing a buffer of `old` bytes by one of `bytes` stays within the
// handle's limit.
bool within_limit(dqmc_handle h, size_t old, size_t bytes) {
  return h->mem_limit == 0 || held_bytes(h) - old + bytes <= h->mem_limit;
}

dqmc_status ensure_ws(dqmc_handle h, size_t bytes) {
  if (bytes <= h->ws_bytes) return DQMC_OK;
  if (h->capturing) {   // no allocation inside a capture: the caller grows and captures again
    h->ws_need = bytes;
    return DQMC_ERR_NOMEM;
  }
  if (!within_limit(h, h->ws_bytes, bytes)) return DQMC_ERR_NOMEM;
  size_t want = bytes + bytes / 8;
  if (!within_limit(h, h->ws_bytes, want)) want = bytes;
  h->gvalid = false;    // a captured graph refers to the old workspace
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      h->ws = nullptr;
      return DQMC_ERR_NOMEM;
    }
    want = bytes;
  }
  h->ws_bytes = want;
  return DQMC_OK;
}

cudaEvent_t pool_event(dqmc_handle h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Folds finished event pairs into the per-class totals (synchronises the stream).
void prof_collect(dqmc_handle h) {
  if (h->pending.empty()) return;
  cudaDeviceSynchronize();
  for (auto& r : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      h->prof_ms[r.cls] += ms;
      h->prof_count[r.cls] += 1;
      h->prof_flops[r.cls] += r.flops;
    }
    h->pool.push_back(r.e0);
    h->pool.push_back(r.e1);
  }
  cudaGetLastError();
  h->pending.clear();
}

// ---------------------------------------------------------------------------
// Debug build (-DDQMC_DEBUG): every translation unit with kernels has its own
// check word (common.cuh); a launch outside a stream capture is waited for
// and the words are read, so a failed device-side check surfaces as
// DQMC_ERR_CHECK from the call that made it.
// ---------------------------------------------------------------------------
#ifdef DQMC_DEBUG
}  // namespace
namespace dqmc {
unsigned long long check_word_api(bool clear);
unsigned long long check_word_gemm(bool clear);
unsigned long long check_word_qrp(bool clear);
unsigned long long check_word_lu(bool clear);
unsigned long long check_word_jacobi(bool clear);
unsigned long long check_word_chain_small(bool clear);
unsigned long long check_word_ozaki(bool clear);
}  // namespace dqmc
namespace {
struct CheckUnit {
  const char* file;
  unsigned long long (*read)(bool clear);
};
const CheckUnit kCheckUnits[] = {
    {"api.cu", dqmc::check_word_api},         {"gemm_f64.cu", dqmc::check_word_gemm},
    {"qrp_f64.cu", dqmc::check_word_qrp},     {"lu_f64.cu", dqmc::check_word_lu},
    {"jacobi_f64.cu", dqmc::check_word_jacobi}, {"chain_small.cu", dqmc::check_word_chain_small},
    {"ozaki_tc.cu", dqmc::check_word_ozaki},
};
#endif

static dqmc_status debug_after_launch(dqmc_handle h) {
#ifdef DQMC_DEBUG
  if (h->capturing) return DQMC_OK;
  // a capture the caller runs on its own stream (the allocation-free call)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->cur, &cs) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_CUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) return DQMC_OK;
  if (cudaStreamSynchronize(h->cur) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_CUDA;
  }
  for (const CheckUnit& u : kCheckUnits)
    if (u.read(false)) return DQMC_ERR_CHECK;
#else
  (void)h;
#endif
  return DQMC_OK;
}

// Launch wrapper: counts the launch, and brackets it with events when the
// profiler is on.  cls/flops classify it (flops = algorithmic FP64 flops).
// The debug build then waits for it and reads the check words.
#define CKP(cls_, flops_, expr)                                   \
  do {                                                            \
    ProfRec _r{nullptr, nullptr, (cls_), (double)(flops_)};       \
    if (h->prof) {                                                \
      _r.e0 = pool_event(h);                                      \
      _r.e1 = pool_event(h);                                      \
      cudaEventRecord(_r.e0, h->cur);                             \
    }                                                             \
    cudaError_t _e = (expr);                                      \
    h->launches++;                                                \
    if (h->prof) {                                                \
      cudaEventRecord(_r.e1, h->cur);                             \
      h->pending.push_back(_r);                                   \
      if (h->pending.size() > 4096) prof_collect(h);              \
    }                                                             \
    if (_e != cudaSuccess) return DQMC_ERR_CUDA;                  \
    dqmc_status _d = debug_after_launch(h);                       \
    if (_d != DQMC_OK) return _d;                                 \
  } while (0)
#define CK(expr) CKP(PC_OTHER, 0.0, expr)
#define CKS(expr)                                  \
  do {                                             \
    dqmc_status _s = (expr);                       \
    if (_s != DQMC_OK) return _s;                  \
  } while (0)

inline int n_chunks(int M, int k) { return (M + k - 1) / k; }
// LU factorisation (2/3 N^3) + forward and backward substitution (2 N^2 per column)
inline double lu_flops(int N, int nrhs) { return 2.0 / 3.0 * N * (double)N * N + 2.0 * N * (double)N * nrhs; }

// ---------------------------------------------------------------------------
// a0: E = exp(sgn * dtau * K)
// ---------------------------------------------------------------------------
struct ExpmWs {
  double *t0, *t1, *scale;
  int *s, *asym;
};

void take_expm(Arena& ar, int N, ExpmWs& w) {
  w.t0 = ar.take<double>((long long)N * N);
  w.t1 = ar.take<double>((long long)N * N);
  w.scale = ar.take<double>(1);
  w.s = ar.take<int>(1);
  w.asym = ar.take<int>(1);
}

// Result ends in w.t0 (the step counts are even).
dqmc_status run_expm(dqmc_handle h, const double* K, int N, double dtau, double sgn,
                     const ExpmWs& w, int* status, int batch) {
  cudaStream_t st = h->cur;
  if (N <= 16) {
    CK(expm_small(K, N, dtau, sgn, EXPM_TERMS, EXPM_SQUARINGS, w.t0, w.asym, status, batch,
                  DQMC_STATUS_BAD_K, st));
    return DQMC_OK;
  }
  CK(expm_prepare(K, N, dtau, sgn, w.s, w.scale, w.asym, st));
  CK(set_identity(w.t0, 0, N, 1, st));
  double* cur = w.t0;
  double* nxt = w.t1;
  for (int m = EXPM_TERMS; m >= 1; --m) {
    GemmArgs g;
    g.M = g.N = g.K = N;
    g.batch = 1;
    g.A = K; g.lda = N;
    g.B = cur; g.ldb = N;
    g.C = nxt; g.ldc = N;
    g.alpha = 1.0 / m;
    g.alpha_ptr = w.scale;
    g.addIdentity = 1;
    CK(gemm_f64(g, st));
    double* t = cur; cur = nxt; nxt = t;
  }
  for (int s = 0; s < EXPM_SQUARINGS; ++s) {
    GemmArgs g;
    g.M = g.N = g.K = N;
    g.batch = 1;
    g.A = cur; g.lda = N;
    g.B = cur; g.ldb = N;
    g.C = nxt; g.ldc = N;
    g.skip_if = w.s;
    g.skip_at = s;
    CK(gemm_f64(g, st));
    double* t = cur; cur = nxt; nxt = t;
  }
  if (status) CK(or_status(status, batch, w.asym, DQMC_STATUS_BAD_K, st));
  return DQMC_OK;
}

// ---------------------------------------------------------------------------
// a1-a5: one direction of the stabilised chain.
//
// dir = +1: forward, B(tau_c, 0) grows by B_l = E diag(e^{V_l}) on the left;
//           chunk c moves slot c -> c+1.
// dir = -1: backward on the transposed chain, B(beta, tau)^T grows by
//           B_l^T = diag(e^{V_l}) E^T on the left, slices from M down;
//           chunk c moves slot c+1 -> c.
// Slot s of instance b: U at U + s*slotU + b*instU (same for D, X).
// ---------------------------------------------------------------------------
struct Slots {
  double* U; long long slotU, instU;
  double* D; long long slotD, instD;
  double* X; long long slotX, instX;
  // when pingpongX is set, X alternates between X (even slots) and X2 (odd)
  // and U/D are updated in place (slot strides 0).
  double* X2 = nullptr;
};

struct ChainWs {
  double *C0, *C1, *W, *T;
  int* perm;
  // mixed-precision slice products (oz_s > 0): E slices (shared) and the
  // per-instance slices of the right operand
  int oz_s = 0, oz_P128 = 0, oz_PK = 0;
  __nv_bfloat16 *ozA = nullptr, *ozB = nullptr;
  int *ozeA = nullptr, *ozeB = nullptr;
  // per-instance slices of T' for the X update on the tensor cores
  __nv_bfloat16* ozT = nullptr;
  int* ozeT = nullptr;
};

inline int pad_to(int n, int m) { return (n + m - 1) / m * m; }

// Digit slices of E (forward chain, transposeE = 0) or E^T (backward chain)
// into a chain workspace's shared A-operand buffers.
cudaError_t split_E(const double* E, int N, int transposeE, const ChainWs& w, cudaStream_t st) {
  // row i of the A operand is a "column" of the splitter: element (m, i)
  return transposeE ? ozaki_split(E, N, 1, 0, nullptr, 0, N, w.oz_P128, w.oz_PK, 128, w.oz_s,
                                  w.ozA, 0, w.ozeA, 0, 1, st)
                    : ozaki_split(E, 1, N, 0, nullptr, 0, N, w.oz_P128, w.oz_PK, 128, w.oz_s,
                                  w.ozA, 0, w.ozeA, 0, 1, st);
}

// Mixed-precision buffers of a chain over `batch` instances with s slices.
void take_ozaki(Arena& ar, int batch, int N, int s, ChainWs& w) {
  w.oz_s = s;
  w.oz_P128 = pad_to(N, 128);
  w.oz_PK = pad_to(N, 64);
  w.ozA = ar.take<__nv_bfloat16>((long long)s * w.oz_P128 * w.oz_PK);
  w.ozeA = ar.take<int>(w.oz_P128);
  w.ozB = ar.take<__nv_bfloat16>((long long)batch * s * w.oz_PK * w.oz_PK);
  w.ozeB = ar.take<int>((long long)batch * w.oz_PK);
  w.ozT = ar.take<__nv_bfloat16>((long long)batch * s * w.oz_P128 * w.oz_PK);
  w.ozeT = ar.take<int>((long long)batch * w.oz_P128);
}

void take_chain(Arena& ar, int batch, int N, ChainWs& w) {
  long long NN = (long long)N * N;
  w.C0 = ar.take<double>(NN * batch);
  w.C1 = ar.take<double>(NN * batch);
  w.W = ar.take<double>(NN * batch);
  w.T = ar.take<double>(NN * batch);
  w.perm = ar.take<int>((long long)N * batch);
}

inline double* slotU(const Slots& s, int slot) { return s.U + slot * s.slotU; }
inline double* slotD(const Slots& s, int slot) { return s.D + slot * s.slotD; }
inline double* slotX(const Slots& s, int slot) {
  if (s.X2) return (slot & 1) ? s.X2 : s.X;
  return s.X + slot * s.slotX;
}

// a1 for chunk c: k slice products into the chunk buffers; *out = last product.
dqmc_status chunk_products(dqmc_handle h, int dir, int batch, int N, int M, int k, int c,
                           const double* E, const double* expV, long long sV, const Slots& s,
                           const ChainWs& w, const int* lim, const double** out, int* status) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const int src = dir > 0 ? c : c + 1;
  const int lo = c * k + 1;
  const int hi = (c + 1) * k < M ? (c + 1) * k : M;
  const double* prev = slotU(s, src);
  long long sprev = s.instU;
  double* bufs[2] = {w.C0, w.C1};
  int nb = 0;
  if (w.oz_s == 0 && N <= CHAIN_SMALL_MAX_N && batch <= 65535 && (dir > 0 || !lim)) {
    // small N: the whole chunk in one launch, each CTA applying every slice
    // to a block of columns held in shared memory
    ChainSmallArgs cs;
    cs.N = N; cs.batch = batch; cs.nslices = hi - lo + 1; cs.dir = dir; cs.lo = lo; cs.hi = hi;
    cs.E = E; cs.transE = dir < 0 ? 1 : 0;
    cs.X = prev; cs.sX = sprev;
    cs.C = w.C0; cs.sC = NN;
    cs.expV = expV; cs.sV = sV;
    cs.lim = lim; cs.lim_base = lo;
    CKP(PC_CHAIN, 2.0 * N * N * (double)N * batch * (hi - lo + 1), chain_small(cs, st));
    *out = w.C0;
    return DQMC_OK;
  }
  for (int i = 0; i <= hi - lo; ++i) {
    const int l = dir > 0 ? lo + i : hi - i;
    if (w.oz_s > 0) {
      // a12 on the tensor cores.  Forward: B' = diag(e^{V_l}) A, C = E B'.
      // Ragged chains (lim): slices past an instance's own M_b copy the FP64
      // input through, as the FP64 product does, so that a last partial
      // chunk ends with B_{M_b} ... B_{ck+1} U.
      // Backward (B_l^T = diag(e^{V_l}) E^T): C = E^T B' with B' = A scaled by
      // the previous slice's e^{V}; the last slice's scale is applied below.
      const int PK = w.oz_PK, sl = w.oz_s;
      const double* sc = nullptr;
      if (dir > 0) sc = expV + (long long)(l - 1) * N;
      else if (i > 0) sc = expV + (long long)l * N;       // e^{V_{l+1}}
      CK(ozaki_split(prev, N, 1, sprev, sc, sV, N, PK, PK, 64, sl, w.ozB, (long long)sl * PK * PK,
                     w.ozeB, PK, batch, st));
      CKP(PC_CHAIN, 2.0 * N * N * (double)N * batch,
          ozaki_gemm(w.ozA, w.ozeA, 0, 0, w.oz_P128, w.ozB, w.ozeB, PK, PK, PK, sl, N, batch,
                     bufs[nb], NN, status, st, lim, l, prev, sprev));
      prev = bufs[nb];
      sprev = NN;
      nb ^= 1;
      if (dir < 0 && i == hi - lo)
        CK(scale_rows(bufs[nb ^ 1], NN, expV + (long long)(l - 1) * N, sV, N, batch, st));
      continue;
    }
    GemmArgs g;
    g.M = g.N = g.K = N;
    g.batch = batch;
    g.A = E; g.lda = N; g.sA = 0;
    g.B = prev; g.ldb = N; g.sB = sprev;
    g.C = bufs[nb]; g.ldc = N; g.sC = NN;
    g.lim = lim; g.lim_at = l;
    g.tile = h->gemm_tile;
    if (dir > 0) {
      g.ms = expV + (long long)(l - 1) * N; g.sms = sV;      // E diag(e^{V_l}) A
    } else {
      g.transA = 1;                                          // diag(e^{V_l}) E^T A
      g.rs = expV + (long long)(l - 1) * N; g.srs = sV;
    }
    CKP(PC_CHAIN, 2.0 * N * N * (double)N * batch, gemm_f64(g, st));
    prev = bufs[nb];
    sprev = NN;
    nb ^= 1;
  }
  *out = prev;
  return DQMC_OK;
}

// a2-a3 for chunk c: (A) diag(D_src) -> U' D' T' (pivoted QR).
dqmc_status chunk_qr(dqmc_handle h, int dir, int batch, int N, int k, int c, const double* A,
                     const Slots& s, const ChainWs& w, int* status, const int* lim) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const int src = dir > 0 ? c : c + 1;
  const int dst = dir > 0 ? c + 1 : c;
  QrpArgs q;
  q.N = N; q.batch = batch;
  q.A = A; q.sA = NN;
  q.Din = slotD(s, src); q.sDin = s.instD;
  q.W = w.W; q.sW = NN;
  q.U = slotU(s, dst); q.sU = s.instU;
  q.D = slotD(s, dst); q.sD = s.instD;
  q.T = w.T; q.sT = NN;
  q.perm = w.perm; q.sperm = N;
  q.status = status;
  q.lim = lim; q.lim_at = c * k + 1;
  // the FP64 chain's products can share SMs with this QR (see qrp_f64.cu)
  q.share_sm = h->prec == DQMC_CHAIN_FP64 ? 1 : 0;
  if (h->decomp == DQMC_DECOMP_JACOBI) {
    // U' D' V'^T by one-sided Jacobi; V'^T goes where T' would
    JacobiArgs j;
    j.N = N; j.batch = batch;
    j.A = A; j.sA = NN;
    j.Din = q.Din; j.sDin = q.sDin;
    j.W = w.W; j.sW = NN;
    j.U = q.U; j.sU = q.sU;
    j.D = q.D; j.sD = q.sD;
    j.Vt = w.T; j.sVt = NN;
    j.status = status;
    j.lim = lim; j.lim_at = q.lim_at;
    CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * batch, jacobi_svd_f64(j, st));
    return DQMC_OK;
  }
  CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * batch, qrp_f64(q, st));
  return DQMC_OK;
}

// a4 for chunk c: X_dst = T' X_src[perm].
dqmc_status chunk_xupdate(dqmc_handle h, int dir, int batch, int N, int k, int c, const Slots& s,
                          const ChainWs& w, const int* lim, int* status) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const int src = dir > 0 ? c : c + 1;
  const int dst = dir > 0 ? c + 1 : c;
  if (w.oz_s > 0) {
    // tensor cores: slices of T' (A operand, per instance; row i of T' is a
    // "column" of the splitter) and of the rows of X_src gathered by perm.
    // Ragged chains (lim): ended instances copy X_src through unchanged.
    const int P1 = w.oz_P128, PK = w.oz_PK, sl = w.oz_s;
    CK(ozaki_split(w.T, 1, N, NN, nullptr, 0, N, P1, PK, 128, sl, w.ozT, (long long)sl * P1 * PK,
                   w.ozeT, P1, batch, st));
    CK(ozaki_split(slotX(s, src), N, 1, s.instX, nullptr, 0, N, PK, PK, 64, sl, w.ozB,
                   (long long)sl * PK * PK, w.ozeB, PK, batch, st, w.perm, N));
    CKP(PC_XUPD, (double)N * N * (double)N * batch,
        ozaki_gemm(w.ozT, w.ozeT, (long long)sl * P1 * PK, P1, P1, w.ozB, w.ozeB, PK, PK, PK, sl,
                   N, batch, slotX(s, dst), s.instX, status, st, lim, c * k + 1,
                   slotX(s, src), s.instX));
    return DQMC_OK;
  }
  const bool jac = h->decomp == DQMC_DECOMP_JACOBI;   // X' = V'^T X: dense, no pivots
  GemmArgs g;
  g.M = g.N = g.K = N;
  g.batch = batch;
  g.A = w.T; g.lda = N; g.sA = NN; g.upperA = jac ? 0 : 1;
  g.B = slotX(s, src); g.ldb = N; g.sB = s.instX;
  g.permB = jac ? nullptr : w.perm; g.sperm = N;
  g.C = slotX(s, dst); g.ldc = N; g.sC = s.instX;
  g.lim = lim; g.lim_at = c * k + 1;
  CKP(PC_XUPD, (double)N * N * (double)N * batch, gemm_f64(g, st));
  return DQMC_OK;
}

dqmc_status chunk_refactor(dqmc_handle h, int dir, int batch, int N, int k, int c,
                           const double* A, const Slots& s, const ChainWs& w, int* status,
                           const int* lim) {
  CKS(chunk_qr(h, dir, batch, N, k, c, A, s, w, status, lim));
  return chunk_xupdate(h, dir, batch, N, k, c, s, w, lim, status);
}

// lim (nullable, per instance): chain length M_b of ragged batches; slices
// past M_b are copied through and finished instances skip the QR and X update.
dqmc_status run_chain(dqmc_handle h, int dir, int batch, int N, int M, int k, const double* E,
                      const double* expV, long long sV, const Slots& s, const ChainWs& w,
                      int* status, const int* lim = nullptr) {
  const int nc = n_chunks(M, k);
  for (int step = 0; step < nc; ++step) {
    const int c = dir > 0 ? step : nc - 1 - step;
    const double* A = nullptr;
    CKS(chunk_products(h, dir, batch, N, M, k, c, E, expV, sV, s, w, lim, &A, status));
    CKS(chunk_refactor(h, dir, batch, N, k, c, A, s, w, status, lim));
  }
  return DQMC_OK;
}

dqmc_status ensure_aux(dqmc_handle h, size_t n) {
  while (h->aux.size() < n) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return DQMC_ERR_CUDA;
    h->aux.push_back(s);
    h->auxev.push_back(e);
  }
  return DQMC_OK;
}

// Two halves of a batch on two streams, staggered by one product phase:
//   stream 0:  P_A(0) R_A(0)        P_A(1) R_A(1) ...
//   stream 1:         P_B(0) R_B(0)        P_B(1) ...
// The product phases P (FP64-pipe bound, all SMs) run one after another,
// and each half's pivoted QR R (latency bound, one CTA per instance) runs
// concurrently with the other half's products, filling the FP64 pipe cycles
// the QR leaves idle.  Caller provides per-half slots/workspaces; the main
// stream is forked before and joined after.
struct ChainJob {
  int dir = +1, batch = 0;
  const double* expV = nullptr;
  long long sV = 0;
  Slots s;
  ChainWs w;
  int* status = nullptr;
  const int* lim = nullptr;   // per-instance chain length (ragged groups), nullable
};

// nj contiguous sub-batches of a batch whose slots, workspace, fields (sV
// apart), status and chain lengths (lim, nullable) are laid out per instance:
// J[q] holds instances [o_q, o_q + n_q), n_q = batch / nj or one more.
void make_sub_jobs(ChainJob* J, int nj, int dir, int batch, int N, const double* expV,
                   long long sV, const Slots& s, const ChainWs& cw, int* status,
                   const int* lim) {
  const long long NN = (long long)N * N;
  long long o = 0;
  for (int q = 0; q < nj; ++q) {
    const int nb = batch / nj + (q < batch % nj ? 1 : 0);
    J[q].dir = dir;
    J[q].batch = nb;
    J[q].expV = expV + o * sV;
    J[q].sV = sV;
    J[q].s = s;
    J[q].s.U += o * NN; J[q].s.D += o * N; J[q].s.X += o * NN; J[q].s.X2 += o * NN;
    J[q].w = cw;
    J[q].w.C0 += o * NN; J[q].w.C1 += o * NN; J[q].w.W += o * NN; J[q].w.T += o * NN;
    J[q].w.perm += o * N;
    if (cw.oz_s > 0) {
      J[q].w.ozB += o * cw.oz_s * (long long)cw.oz_PK * cw.oz_PK;
      J[q].w.ozeB += o * cw.oz_PK;
      J[q].w.ozT += o * cw.oz_s * (long long)cw.oz_P128 * cw.oz_PK;
      J[q].w.ozeT += o * cw.oz_P128;
    }
    J[q].status = status + o;
    J[q].lim = lim ? lim + o : nullptr;
    o += nb;
  }
}

// Pipelining can be switched off with DQMC_PIPELINE=0 (for A/B timing).
bool pipeline_enabled() {
  const char* e = getenv("DQMC_PIPELINE");
  return !(e && e[0] == '0');
}

// Number of staggered sub-batches of an equal-time chain: DQMC_PIPELINE=n
// (2..8) overrides the default (2 for FP64 products, 4 for tensor-core ones).
constexpr int kMaxJobs = 8;
int pipeline_jobs(bool mixed) {
  const char* e = getenv("DQMC_PIPELINE");
  if (e && e[0] >= '2' && e[0] <= '8' && e[1] == 0) return e[0] - '0';
  return mixed ? 4 : 2;
}

// The jobs run on aux streams sbase .. sbase + nj - 1, forked from and joined
// back into the current stream h->cur.
dqmc_status run_chain_multi(dqmc_handle h, const ChainJob* job, int nj, int N, int M, int k,
                            const double* E, int sbase = 0) {
  if (nj < 1 || nj > kMaxJobs || sbase < 0) return DQMC_ERR_ARG;
  CKS(ensure_aux(h, (size_t)(sbase + nj)));
  cudaStream_t main = h->cur;
  cudaStream_t* aux = h->aux.data() + sbase;
  cudaEvent_t* auxev = h->auxev.data() + sbase;
  cudaEvent_t fork = auxev[0];
  cudaEventRecord(fork, main);
  for (int i = 0; i < nj; ++i) cudaStreamWaitEvent(aux[i], fork, 0);
  cudaEvent_t ev[kMaxJobs] = {};
  dqmc_status rc = DQMC_OK;
  for (int i = 0; i < nj && rc == DQMC_OK; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) rc = DQMC_ERR_CUDA;
  const int nc = n_chunks(M, k);
  for (int step = 0; step < nc && rc == DQMC_OK; ++step) {
    for (int i = 0; i < nj && rc == DQMC_OK; ++i) {
      const ChainJob& J = job[i];
      const int c = J.dir > 0 ? step : nc - 1 - step;
      h->cur = aux[i];
      // product phases run one after another: job i after job i-1 of this
      // chunk, job 0 after the last job of the previous chunk
      if (i > 0) cudaStreamWaitEvent(h->cur, ev[i - 1], 0);
      else if (step > 0) cudaStreamWaitEvent(h->cur, ev[nj - 1], 0);
      const double* A = nullptr;
      rc = chunk_products(h, J.dir, J.batch, N, M, k, c, E, J.expV, J.sV, J.s, J.w, J.lim, &A,
                          J.status);
      if (rc != DQMC_OK) break;
      cudaEventRecord(ev[i], h->cur);
      rc = chunk_refactor(h, J.dir, J.batch, N, k, c, A, J.s, J.w, J.status, J.lim);
    }
  }
  for (int i = 0; i < nj; ++i) {
    cudaEventRecord(auxev[i], aux[i]);
    cudaStreamWaitEvent(main, auxev[i], 0);
  }
  for (int i = 0; i < nj; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  h->cur = main;
  return rc;
}

dqmc_status run_chain_pair(dqmc_handle h, const ChainJob job[2], int N, int M, int k,
                           const double* E) {
  return run_chain_multi(h, job, 2, N, M, k, E);
}

// ---------------------------------------------------------------------------
// Tree-parallel fold of the forward chain.  The pairwise product of Eq.
// (stabmult),
//   (U_2 D_2 X_2)(U_1 D_1 X_1) = (U_2 u) d (x X_1),   u d x = udt(D_2 (X_2 U_1) D_1),
// is associative, so the chunk products C_c = B_{ck+k}...B_{ck+1} can all be
// formed at once, decomposed, and folded pairwise in ceil(log2(ceil(M/k)))
// levels.  For a batch that leaves most SMs idle this replaces ceil(M/k)
// dependent pivoted QRs (one CTA per instance each) by one QR per level, each
// over batch x (chunks at that level) CTAs.
//
// The chunk count is padded to a power of two P0 with identity factors
// (copied through the products, skipped by the level-0 QR), so that the pair
// (2i, 2i+1) of instance b at a level of P factors per instance sits at
// 2 (b P/2 + i): every operand of a level is a plain strided batch.  D_2
// enters as a row scale of the product X_2 U_1 and D_1 as the QR's column
// scale.  Its largest entry is that of the left half's scales, which is no
// larger than those of the whole chain's D.
// ---------------------------------------------------------------------------
struct TreeWs {
  double *Iden, *C0, *C1, *U[2], *D[2], *X[2], *W, *T;
  int *perm, *len;
  int P0 = 1;
};

int tree_width(int nc) {
  int p = 1;
  while (p < nc) p <<= 1;
  return p;
}

void take_tree(Arena& ar, int batch, int N, int nc, TreeWs& w) {
  const long long NN = (long long)N * N;
  w.P0 = tree_width(nc);
  const long long Q = (long long)batch * w.P0, H = Q / 2 > 0 ? Q / 2 : 1;
  w.Iden = ar.take<double>(NN);
  w.C0 = ar.take<double>(Q * NN);
  w.C1 = ar.take<double>(Q * NN);
  w.U[0] = ar.take<double>(Q * NN);
  w.D[0] = ar.take<double>(Q * N);
  w.X[0] = ar.take<double>(Q * NN);
  w.U[1] = ar.take<double>(H * NN);
  w.D[1] = ar.take<double>(H * N);
  w.X[1] = ar.take<double>(H * NN);
  w.W = ar.take<double>(Q * NN);
  w.T = ar.take<double>(Q * NN);
  w.perm = ar.take<int>(Q * N);
  w.len = ar.take<int>(Q);
}

// Leaves B_M...B_1 = U D X of instance b at *U + b N^2, *D + b N, *X + b N^2.
dqmc_status run_chain_tree(dqmc_handle h, int batch, int N, int M, int k, const double* E,
                           const double* expV, long long sV, const TreeWs& w, int* status,
                           const double** Uo, const double** Do, const double** Xo) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const int nc = n_chunks(M, k), P0 = w.P0;
  const int Q = batch * P0;
  const double f2 = 2.0 * N * (double)N * N;
  // the U and X updates of a level are independent: X runs on an aux stream
  CKS(ensure_aux(h, 2));
  cudaStream_t sx = h->aux[0];
  cudaEvent_t fork = h->auxev[0], join = h->auxev[1];
  CK(set_identity(w.Iden, 0, N, 1, st));
  CK(chunk_len(w.len, batch, P0, nc, k, M, st));
  // a1: C_c for every chunk of every instance (identity for the padding)
  double* bufs[2] = {w.C0, w.C1};
  const double* prev = w.Iden;
  long long sprev = 0;
  const bool small = N <= CHAIN_SMALL_MAX_N && Q <= 65535;
  if (small) {
    // small N: the k slices of every chunk in one launch (padding chunks copy
    // the identity through)
    ChainSmallArgs cs;
    cs.N = N; cs.batch = Q; cs.nslices = k; cs.dir = 1; cs.lo = 1; cs.hi = k;
    cs.E = E; cs.X = w.Iden; cs.sX = 0;
    cs.C = bufs[0]; cs.sC = NN;
    cs.expV = expV; cs.sV = sV; cs.divS = P0; cs.sV_inner = (long long)k * N;
    cs.lim = w.len; cs.lim_base = 1;
    CKP(PC_CHAIN, f2 * Q * k, chain_small(cs, st));
    prev = bufs[0];
    sprev = NN;
  }
  for (int i = 0; i < k && !small; ++i) {
    GemmArgs g;
    g.M = g.N = g.K = N;
    g.batch = Q;
    g.A = E; g.lda = N; g.sA = 0;
    g.B = prev; g.ldb = N; g.sB = sprev;
    g.C = bufs[i & 1]; g.ldc = N; g.sC = NN;
    g.ms = expV + (long long)i * N; g.sms = sV; g.divS = P0; g.sms_inner = (long long)k * N;
    g.lim = w.len; g.lim_at = i + 1;
    g.tile = h->gemm_tile;
    CKP(PC_CHAIN, f2 * Q, gemm_f64(g, st));
    prev = bufs[i & 1];
    sprev = NN;
  }
  // a3 on every chunk: C_c = U_c D_c X_c; the padding keeps U = X = 1, D = 1
  CK(set_identity(w.U[0], NN, N, Q, st));
  CK(set_const(w.D[0], (long long)Q * N, 1.0, st));
  {
    QrpArgs q;
    q.N = N; q.batch = Q;
    q.A = prev; q.sA = NN;
    q.W = w.W; q.sW = NN;
    q.U = w.U[0]; q.sU = NN;
    q.D = w.D[0]; q.sD = N;
    q.T = w.T; q.sT = NN;
    q.perm = w.perm; q.sperm = N;
    q.status = status; q.status_div = P0;
    q.lim = w.len; q.lim_at = 1;
    CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * Q, qrp_f64(q, st));
    GemmArgs g;                                       // X_c = T' P^T (identity for the padding)
    g.M = g.N = g.K = N; g.batch = Q;
    g.A = w.T; g.lda = N; g.sA = NN; g.upperA = 1;
    g.B = w.Iden; g.ldb = N; g.sB = 0;
    g.permB = w.perm; g.sperm = N;
    g.C = w.X[0]; g.ldc = N; g.sC = NN;
    g.lim = w.len; g.lim_at = 1;
    CKP(PC_XUPD, (double)N * N * (double)N * Q, gemm_f64(g, st));
  }
  // levels: pair i of instance b = (left 2i+1, right 2i) -> i
  int cur = 0;
  for (int P = P0; P > 1; P >>= 1) {
    const int np = P / 2, B2 = batch * np, nxt = cur ^ 1;
    double* Y = w.C0;       // the chunk buffers are free after level 0
    double* Uq = w.C1;
    GemmArgs gy;                                      // Y = D_2 (X_2 U_1)
    gy.M = gy.N = gy.K = N; gy.batch = B2;
    gy.A = w.X[cur] + NN; gy.lda = N; gy.sA = 2 * NN;
    gy.B = w.U[cur]; gy.ldb = N; gy.sB = 2 * NN;
    gy.rs = w.D[cur] + N; gy.srs = 2LL * N;
    gy.C = Y; gy.ldc = N; gy.sC = NN;
    gy.tile = h->gemm_tile;
    CKP(PC_OTHER, f2 * B2, gemm_f64(gy, st));
    QrpArgs q;                                        // Y D_1 = u d x
    q.N = N; q.batch = B2;
    q.A = Y; q.sA = NN;
    q.Din = w.D[cur]; q.sDin = 2LL * N;
    q.W = w.W; q.sW = NN;
    q.U = Uq; q.sU = NN;
    q.D = w.D[nxt]; q.sD = N;
    q.T = w.T; q.sT = NN;
    q.perm = w.perm; q.sperm = N;
    q.status = status; q.status_div = np;
    CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * B2, qrp_f64(q, st));
    // U = U_2 u here and X = x X_1 on the aux stream, joined before the
    // next level's product reads both
    if (cudaEventRecord(fork, st) != cudaSuccess || cudaStreamWaitEvent(sx, fork, 0) != cudaSuccess)
      return DQMC_ERR_CUDA;
    GemmArgs gu;                                      // U = U_2 u
    gu.M = gu.N = gu.K = N; gu.batch = B2;
    gu.A = w.U[cur] + NN; gu.lda = N; gu.sA = 2 * NN;
    gu.B = Uq; gu.ldb = N; gu.sB = NN;
    gu.C = w.U[nxt]; gu.ldc = N; gu.sC = NN;
    gu.tile = h->gemm_tile;
    CKP(PC_OTHER, f2 * B2, gemm_f64(gu, st));
    GemmArgs gx;                                      // X = x X_1
    gx.M = gx.N = gx.K = N; gx.batch = B2;
    gx.A = w.T; gx.lda = N; gx.sA = NN; gx.upperA = 1;
    gx.B = w.X[cur]; gx.ldb = N; gx.sB = 2 * NN;
    gx.permB = w.perm; gx.sperm = N;
    gx.C = w.X[nxt]; gx.ldc = N; gx.sC = NN;
    h->cur = sx;
    CKP(PC_XUPD, (double)N * N * (double)N * B2, gemm_f64(gx, sx));
    h->cur = st;
    if (cudaEventRecord(join, sx) != cudaSuccess || cudaStreamWaitEvent(st, join, 0) != cudaSuccess)
      return DQMC_ERR_CUDA;
    cur = nxt;
  }
  *Uo = w.U[cur];
  *Do = w.D[cur];
  *Xo = w.X[cur];
  return DQMC_OK;
}

// Tree fold for the equal-time chain: by setting, or (auto) when the level-0
// QRs of all chunks of the batch fit in one wave of CTAs (one per SM) and the
// chain has at least four chunks.
bool use_tree(dqmc_handle h, int batch, int nc) {
  if (h->prec != DQMC_CHAIN_FP64 || h->decomp != DQMC_DECOMP_QR) return false;
  if (h->fold == DQMC_FOLD_TREE) return nc > 1;
  if (h->fold == DQMC_FOLD_SEQUENTIAL) return false;
  return nc >= 4 && (long long)batch * nc <= h->sms;
}

// ---------------------------------------------------------------------------
// a6-a7: G = [1 + U D X]^{-1} by Eq. (inversion_loh) and log|det(1 + U D X)|.
//   Y = X^{-1} D_p^{-1}           (LU solve with diagonal right-hand side)
//   Mx = Y + U D_m
//   G = Y Mx^{-1}                 (LU solve of Mx^T G^T = Y^T)
//   log|det| = sum log D_p + log|det Mx|;  sign = sign det Mx * sign det X
// ---------------------------------------------------------------------------
struct LohWs {
  double *Dpinv, *Y, *Mx, *Wlu, *lad, *Gtmp;
  int *sX, *sM;
};

void take_loh(Arena& ar, int batch, int N, LohWs& w) {
  long long NN = (long long)N * N;
  w.Dpinv = ar.take<double>((long long)N * batch);
  w.Y = ar.take<double>(NN * batch);
  w.Mx = ar.take<double>(NN * batch);
  w.Wlu = ar.take<double>(2 * NN * batch);
  w.lad = ar.take<double>(batch);
  w.sX = ar.take<int>(batch);
  w.sM = ar.take<int>(batch);
}

dqmc_status run_loh(dqmc_handle h, int batch, int N, const double* U, long long sU,
                    const double* D, long long sD, const double* X, long long sX, double* G,
                    double* logdet, int* sign, int* status, const LohWs& w) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  CK(dsplit_vec(D, sD, N, batch, w.Dpinv, 1, st));   // D_p^{-1}
  LuArgs l1;
  l1.N = N; l1.nrhs = N; l1.batch = batch;
  l1.A = X; l1.sA = sX;
  l1.Rdiag = w.Dpinv; l1.sRdiag = N;
  l1.Z = w.Y; l1.sZ = NN; l1.ldz = N;
  l1.W = w.Wlu; l1.sW = 2 * NN;
  l1.sign = w.sX;
  l1.status = status;
  CKP(PC_LU, lu_flops(N, N) * batch, lu_solve_f64(l1, st));
  Axpby2Args ax;
  ax.N = N; ax.batch = batch;
  ax.A = w.Y; ax.sA = NN;
  ax.B = U; ax.sB = sU;
  ax.cb = D; ax.cb_mode = 2; ax.scb = sD;
  ax.C = w.Mx; ax.sC = NN;
  CK(axpby2(ax, st));
  LuArgs l2;
  l2.N = N; l2.batch = batch;
  l2.A = w.Mx; l2.sA = NN; l2.transA = 1;
  if (G) {
    l2.nrhs = N;
    l2.R = w.Y; l2.sR = NN; l2.ldr = N; l2.transR = 1;
    l2.Z = G; l2.sZ = NN; l2.ldz = N; l2.transZ = 1;
  } else {
    l2.nrhs = 0;
    l2.Z = w.Y; l2.sZ = NN; l2.ldz = N;
  }
  l2.W = w.Wlu; l2.sW = 2 * NN;
  l2.logabsdet = w.lad;
  l2.sign = w.sM;
  l2.status = status;
  CKP(PC_LU, lu_flops(N, l2.nrhs) * batch, lu_solve_f64(l2, st));
  CK(finish_logdet(D, sD, N, batch, w.lad, w.sX, w.sM, logdet, sign, status, st));
  return DQMC_OK;
}

// ---------------------------------------------------------------------------
// a6-a7 by Eq. (inversion) instead (DQMC_INV_PLAIN):
//   1 + U D X = U (U^T X^{-1} + D) X,   U^T X^{-1} + D = u d x   (pivoted QR),
//   G = (x X)^{-1} d^{-1} (U u)^T,
//   log|det(1 + U D X)| = sum log d (|det U| = |det u| = |det x X| = 1),
//   sign = sign det(U u) * sign det(x X).
// ---------------------------------------------------------------------------
struct PlainWs {
  double *Iden, *C, *u, *d, *dinv, *W, *T, *xX, *P, *Y, *Wlu;
  int *perm, *s1, *s2;
};

void take_plain(Arena& ar, int batch, int N, PlainWs& w) {
  const long long NN = (long long)N * N;
  w.Iden = ar.take<double>(NN);
  w.C = ar.take<double>(NN * batch);
  w.u = ar.take<double>(NN * batch);
  w.d = ar.take<double>((long long)N * batch);
  w.dinv = ar.take<double>((long long)N * batch);
  w.W = ar.take<double>(NN * batch);
  w.T = ar.take<double>(NN * batch);
  w.xX = ar.take<double>(NN * batch);
  w.P = ar.take<double>(NN * batch);
  w.Y = ar.take<double>(NN * batch);
  w.Wlu = ar.take<double>(2 * NN * batch);
  w.perm = ar.take<int>((long long)N * batch);
  w.s1 = ar.take<int>(batch);
  w.s2 = ar.take<int>(batch);
}

dqmc_status run_one_plus(dqmc_handle h, int batch, int N, const double* U, long long sU,
                         const double* D, long long sD, const double* X, long long sX, double* G,
                         double* logdet, int* sign, int* status, const PlainWs& w) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const double f2 = 2.0 * N * (double)N * N * batch;
  CK(set_identity(w.Iden, 0, N, 1, st));
  LuArgs l1;                                          // C = U^T X^{-1}  (X^T C^T = U)
  l1.N = N; l1.nrhs = N; l1.batch = batch;
  l1.A = X; l1.sA = sX; l1.transA = 1;
  l1.R = U; l1.sR = sU; l1.ldr = N;
  l1.Z = w.C; l1.sZ = NN; l1.ldz = N; l1.transZ = 1;
  l1.W = w.Wlu; l1.sW = 2 * NN;
  l1.status = status;
  CKP(PC_LU, lu_flops(N, N) * batch, lu_solve_f64(l1, st));
  Axpby2Args ax;                                      // C + D on the diagonal
  ax.N = N; ax.batch = batch;
  ax.A = w.C; ax.sA = NN;
  ax.B = w.Iden; ax.sB = 0;
  ax.cb = D; ax.cb_mode = 5; ax.scb = sD;
  ax.C = w.C; ax.sC = NN;
  CK(axpby2(ax, st));
  QrpArgs q;                                          // = u d x
  q.N = N; q.batch = batch;
  q.A = w.C; q.sA = NN;
  q.W = w.W; q.sW = NN;
  q.U = w.u; q.sU = NN;
  q.D = w.d; q.sD = N;
  q.T = w.T; q.sT = NN;
  q.perm = w.perm; q.sperm = N;
  q.status = status;
  CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * batch, qrp_f64(q, st));
  GemmArgs gx;                                        // x X
  gx.M = gx.N = gx.K = N; gx.batch = batch;
  gx.A = w.T; gx.lda = N; gx.sA = NN; gx.upperA = 1;
  gx.B = X; gx.ldb = N; gx.sB = sX;
  gx.permB = w.perm; gx.sperm = N;
  gx.C = w.xX; gx.ldc = N; gx.sC = NN;
  CKP(PC_OTHER, f2 / 2, gemm_f64(gx, st));
  GemmArgs gp;                                        // P = U u
  gp.M = gp.N = gp.K = N; gp.batch = batch;
  gp.A = U; gp.lda = N; gp.sA = sU;
  gp.B = w.u; gp.ldb = N; gp.sB = NN;
  gp.C = w.P; gp.ldc = N; gp.sC = NN;
  CKP(PC_OTHER, f2, gemm_f64(gp, st));
  CK(dsplit_vec(w.d, N, N, batch, w.dinv, 4, st));
  GemmArgs gy = gp;                                   // Y = U u d^{-1}
  gy.C = w.Y;
  gy.cs = w.dinv; gy.scs = N;
  CKP(PC_OTHER, f2, gemm_f64(gy, st));
  LuArgs l2;                                          // (x X) G = Y^T
  l2.N = N; l2.batch = batch;
  l2.A = w.xX; l2.sA = NN;
  if (G) {
    l2.nrhs = N;
    l2.R = w.Y; l2.sR = NN; l2.ldr = N; l2.transR = 1;
    l2.Z = G; l2.sZ = NN; l2.ldz = N;
  } else {
    l2.nrhs = 0;
    l2.Z = w.C; l2.sZ = NN; l2.ldz = N;
  }
  l2.W = w.Wlu; l2.sW = 2 * NN;
  l2.sign = w.s1;
  l2.status = status;
  CKP(PC_LU, lu_flops(N, l2.nrhs) * batch, lu_solve_f64(l2, st));
  LuArgs l3;                                          // sign det(U u)
  l3.N = N; l3.nrhs = 0; l3.batch = batch;
  l3.A = w.P; l3.sA = NN;
  l3.Z = w.C; l3.sZ = NN; l3.ldz = N;
  l3.W = w.Wlu; l3.sW = 2 * NN;
  l3.sign = w.s2;
  l3.status = status;
  CKP(PC_LU, lu_flops(N, 0) * batch, lu_solve_f64(l3, st));
  CK(finish_logdet(w.d, N, N, batch, nullptr, w.s1, w.s2, logdet, sign, status, st, 1));
  return DQMC_OK;
}

// The equal-time inversion the handle's scheme selects.
dqmc_status run_inversion(dqmc_handle h, int batch, int N, const double* U, long long sU,
                          const double* D, long long sD, const double* X, long long sX, double* G,
                          double* logdet, int* sign, int* status, const LohWs& lw,
                          const PlainWs& pw) {
  if (h->inv == DQMC_INV_PLAIN)
    return run_one_plus(h, batch, N, U, sU, D, sD, X, sX, G, logdet, sign, status, pw);
  return run_loh(h, batch, N, U, sU, D, sD, X, sX, G, logdet, sign, status, lw);
}

// ---------------------------------------------------------------------------
// Argument checks and pointer-mode staging
// ---------------------------------------------------------------------------
dqmc_status check_common(dqmc_handle h, int batch, int N, int M, const double* K, double dtau,
                         const double* V, int k) {
  if (!h) return DQMC_ERR_ARG;
  if (batch < 0 || N < 1 || N > 1024 || M < 1 || k < 1 || k > M) return DQMC_ERR_ARG;
  if (!(dtau == dtau) || dtau < 0.0) return DQMC_ERR_ARG;
  if (batch > 0 && (!K || !V)) return DQMC_ERR_ARG;
  if (((uintptr_t)K | (uintptr_t)V) & 7) return DQMC_ERR_ARG;
  if (h->decomp == DQMC_DECOMP_JACOBI && (h->prec != DQMC_CHAIN_FP64 || N > 512))
    return DQMC_ERR_UNSUPPORTED;
  return DQMC_OK;
}

struct Staged {
  const double* K;
  const double* V;
};

// Host pointer mode: device copies of K and V inside the workspace.
struct HostIO {
  double* K = nullptr;
  double* V = nullptr;
};

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

dqmc_status dqmc_create(dqmc_handle* h) {
  if (!h) return DQMC_ERR_ARG;
  *h = nullptr;
  dqmc_handle x = new (std::nothrow) dqmc_handle_s();
  if (!x) return DQMC_ERR_NOMEM;
  if (cudaGetDevice(&x->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, x->device) != cudaSuccess) {
    cudaGetLastError();
    delete x;
    return DQMC_ERR_CUDA;
  }
  *h = x;
  return DQMC_OK;
}

dqmc_status dqmc_destroy(dqmc_handle h) {
  if (!h) return DQMC_ERR_ARG;
  if (h->ws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->ws);
  }
  prof_collect(h);
  for (auto e : h->pool) cudaEventDestroy(e);
  for (auto s : h->aux) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
  for (auto e : h->auxev) cudaEventDestroy(e);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  if (h->rws) cudaFree(h->rws);
  if (h->rtab) cudaFree(h->rtab);
  if (h->rfork) cudaEventDestroy(h->rfork);
  if (h->kpool) cudaFree(h->kpool);
  if (h->epool) cudaFree(h->epool);
  delete h;
  return DQMC_OK;
}

dqmc_status dqmc_set_graph_mode(dqmc_handle h, int enable) {
  if (!h) return DQMC_ERR_ARG;
  h->graphs = enable != 0;
  h->gvalid = false;
  return DQMC_OK;
}

dqmc_status dqmc_profile_enable(dqmc_handle h, int enable) {
  if (!h) return DQMC_ERR_ARG;
  prof_collect(h);
  h->prof = enable != 0;
  return DQMC_OK;
}

dqmc_status dqmc_profile_reset(dqmc_handle h) {
  if (!h) return DQMC_ERR_ARG;
  prof_collect(h);
  for (int c = 0; c < PC_N; ++c) { h->prof_ms[c] = 0; h->prof_flops[c] = 0; h->prof_count[c] = 0; }
  return DQMC_OK;
}

dqmc_status dqmc_profile_read(dqmc_handle h, int cls, double* ms, long long* launches,
                              double* flops) {
  if (!h || cls < 0 || cls >= PC_N) return DQMC_ERR_ARG;
  prof_collect(h);
  if (ms) *ms = h->prof_ms[cls];
  if (launches) *launches = h->prof_count[cls];
  if (flops) *flops = h->prof_flops[cls];
  return DQMC_OK;
}

dqmc_status dqmc_set_stream(dqmc_handle h, void* stream) {
  if (!h) return DQMC_ERR_ARG;
  h->stream = (cudaStream_t)stream;
  return DQMC_OK;
}

dqmc_status dqmc_set_pointer_mode(dqmc_handle h, dqmc_pointer_mode mode) {
  if (!h || (mode != DQMC_PTR_DEVICE && mode != DQMC_PTR_HOST)) return DQMC_ERR_ARG;
  h->pmode = mode;
  return DQMC_OK;
}

dqmc_status dqmc_set_chain_precision(dqmc_handle h, dqmc_chain_prec prec) {
  if (!h) return DQMC_ERR_ARG;
  if (prec != DQMC_CHAIN_FP64 && (prec < DQMC_CHAIN_BF16X3 || prec > DQMC_CHAIN_BF16X8))
    return DQMC_ERR_ARG;
  h->prec = prec;
  return DQMC_OK;
}

dqmc_status dqmc_set_decomposition(dqmc_handle h, int decomposition) {
  if (!h || (decomposition != DQMC_DECOMP_QR && decomposition != DQMC_DECOMP_JACOBI))
    return DQMC_ERR_ARG;
  h->decomp = decomposition;
  return DQMC_OK;
}

dqmc_status dqmc_set_inversion_scheme(dqmc_handle h, int scheme) {
  if (!h || (scheme != DQMC_INV_LOH && scheme != DQMC_INV_PLAIN)) return DQMC_ERR_ARG;
  h->inv = scheme;
  return DQMC_OK;
}

dqmc_status dqmc_set_chain_fold(dqmc_handle h, int mode) {
  if (!h || (mode != DQMC_FOLD_SEQUENTIAL && mode != DQMC_FOLD_TREE && mode != DQMC_FOLD_AUTO))
    return DQMC_ERR_ARG;
  h->fold = mode;
  return DQMC_OK;
}

dqmc_status dqmc_set_gemm_tile(dqmc_handle h, int tile) {
  if (!h || (tile != 0 && tile != 32 && tile != 48 && tile != 64)) return DQMC_ERR_ARG;
  h->gemm_tile = tile;
  return DQMC_OK;
}

long long dqmc_last_launch_count(dqmc_handle h) { return h ? h->launches : -1; }
long long dqmc_workspace_bytes(dqmc_handle h) { return h ? (long long)h->ws_bytes : -1; }
long long dqmc_device_bytes(dqmc_handle h) { return h ? (long long)held_bytes(h) : -1; }

dqmc_status dqmc_set_memory_limit(dqmc_handle h, long long bytes) {
  if (!h || bytes < 0) return DQMC_ERR_ARG;
  h->mem_limit = (size_t)bytes;
  return DQMC_OK;
}

const char* dqmc_status_string(dqmc_status s) {
  switch (s) {
    case DQMC_OK: return "ok";
    case DQMC_ERR_ARG: return "invalid argument";
    case DQMC_ERR_CUDA: return "CUDA runtime or launch failure";
    case DQMC_ERR_NOMEM: return "device workspace allocation failed";
    case DQMC_ERR_NONFINITE: return "non-finite value";
    case DQMC_ERR_SINGULAR: return "singular pivot";
    case DQMC_ERR_TIMEOUT: return "bounded device wait gave up";
    case DQMC_ERR_UNSUPPORTED: return "unsupported configuration";
    case DQMC_ERR_SCRATCH: return "problem needs more device scratch than the fixed array holds";
    case DQMC_ERR_CHECK: return "a device-side check of the debug build failed";
  }
  return "unknown status";
}

// ---------------------------------------------------------------------------
// CUDA-graph mode.  The call is recorded by stream capture on an internal
// stream (forks to the pipelining streams are captured as graph branches),
// instantiated (or the cached executable updated in place when the topology
// matches) and launched on the caller's stream.  A call whose arguments and
// settings equal the previous one's is a bare graph launch: the launch cost of
// the hundreds of small kernels of a small-N problem is paid once.  Inputs
// are read when the graph runs, so callers that update V in place get fresh
// results.  Host pointer mode and the profiler run uncaptured.
// ---------------------------------------------------------------------------
extern "C++" {
struct GraphKey {
  unsigned long long v[24];
  int n = 0;
  void add(unsigned long long x) { if (n < 24) v[n++] = x; }
  void addp(const void* p) { add((unsigned long long)(uintptr_t)p); }
  void addd(double d) { unsigned long long x; memcpy(&x, &d, 8); add(x); }
};

template <class F>
static dqmc_status graph_call(dqmc_handle h, GraphKey key, F&& body) {
  if (!h->graphs || h->pmode == DQMC_PTR_HOST || h->prof) return body();
  key.add((unsigned long long)h->prec);
  key.add((unsigned long long)h->gemm_tile);
  key.add((unsigned long long)h->fold);
  key.add((unsigned long long)h->inv);
  key.add((unsigned long long)h->decomp);
  key.add((unsigned long long)pipeline_enabled() * 16 + (unsigned long long)pipeline_jobs(h->prec != DQMC_CHAIN_FP64));
  key.addp(h->ws);
  key.addp(h->stream);
  bool same = h->gvalid && h->gexec && key.n <= 24;
  for (int i = 0; same && i < key.n; ++i) same = h->gkey[i] == key.v[i];
  if (same) {
    if (cudaGraphLaunch(h->gexec, h->stream) != cudaSuccess) return DQMC_ERR_CUDA;
    h->launches = h->glaunches;
    h->cur = h->stream;
    return debug_after_launch(h);
  }
  if (!h->gstream && cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking) != cudaSuccess)
    return DQMC_ERR_CUDA;
  cudaStream_t caller = h->stream;
  for (int attempt = 0; attempt < 2; ++attempt) {
    h->stream = h->gstream;
    if (cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      h->stream = caller;
      return DQMC_ERR_CUDA;
    }
    h->capturing = true;
    h->ws_need = 0;
    dqmc_status rc = body();
    h->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(h->gstream, &g);
    h->stream = caller;
    h->cur = caller;
    if (rc == DQMC_ERR_NOMEM && h->ws_need) {   // grow outside the capture, then record again
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      CKS(ensure_ws(h, h->ws_need));
      key.v[key.n - 2] = (unsigned long long)(uintptr_t)h->ws;
      continue;
    }
    if (rc != DQMC_OK || ce != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      h->gvalid = false;
      return rc != DQMC_OK ? rc : DQMC_ERR_CUDA;
    }
    bool ok = false;
    if (h->gexec) {
      cudaGraphExecUpdateResultInfo info;
      ok = cudaGraphExecUpdate(h->gexec, g, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
      }
    }
    if (!ok && cudaGraphInstantiate(&h->gexec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      h->gexec = nullptr;
      h->gvalid = false;
      return DQMC_ERR_CUDA;
    }
    cudaGraphDestroy(g);
    for (int i = 0; i < key.n; ++i) h->gkey[i] = key.v[i];
    h->gvalid = true;
    h->glaunches = h->launches;
    if (cudaGraphLaunch(h->gexec, h->stream) != cudaSuccess) return DQMC_ERR_CUDA;
    return debug_after_launch(h);
  }
  return DQMC_ERR_NOMEM;
}
}  // extern "C++"

// ---------------------------------------------------------------------------
// Equal-time G and log det
// ---------------------------------------------------------------------------
static dqmc_status greens_impl(dqmc_handle h, int batch, int N, int M, const double* K,
                               double dtau, const double* V, int k, double* G, double* logdet,
                               int* sign, int* status) {
  CKS(check_common(h, batch, N, M, K, dtau, V, k));
  if (h->prec != DQMC_CHAIN_FP64 && N > 256) return DQMC_ERR_UNSUPPORTED;
  h->launches = 0;
  h->cur = h->stream;
  if (batch == 0) return DQMC_OK;
  const bool host = h->pmode == DQMC_PTR_HOST;
  const long long NN = (long long)N * N;
  const int nc = n_chunks(M, k);
  const bool tree = use_tree(h, batch, nc);
  // padded slice stride of exp(V): one spare chunk, and for the tree every
  // padding chunk of its power-of-two width
  const int mp_chunks = tree && tree_width(nc) > nc + 1 ? tree_width(nc) : nc + 1;
  const long long Mp = (long long)mp_chunks * k;
  TreeWs tw;
  PlainWs pw;

  auto layout = [&](Arena& ar, ExpmWs& ew, ChainWs& cw, LohWs& lw, double*& E, double*& expV,
                    double*& U, double*& D, double*& X0, double*& X1, int*& st, HostIO& io,
                    double*& Gd, double*& ldd, int*& sgd) {
    take_expm(ar, N, ew);
    E = ew.t0;
    expV = ar.take<double>(Mp * N * batch);
    if (tree) {
      take_tree(ar, batch, N, nc, tw);
      U = D = X0 = X1 = nullptr;
    } else {
      U = ar.take<double>(NN * batch);
      D = ar.take<double>((long long)N * batch);
      X0 = ar.take<double>(NN * batch);
      X1 = ar.take<double>(NN * batch);
      take_chain(ar, batch, N, cw);
    }
    if (h->prec != DQMC_CHAIN_FP64) take_ozaki(ar, batch, N, (int)h->prec, cw);
    take_loh(ar, batch, N, lw);
    if (h->inv == DQMC_INV_PLAIN) take_plain(ar, batch, N, pw);
    st = ar.take<int>(batch);
    if (host) {
      io.K = ar.take<double>(NN);
      io.V = ar.take<double>((long long)M * N * batch);
      Gd = G ? ar.take<double>(NN * batch) : nullptr;
      ldd = ar.take<double>(batch);
      sgd = ar.take<int>(batch);
    }
  };
  ExpmWs ew; ChainWs cw; LohWs lw; HostIO io;
  double *E, *expV, *U, *D, *X0, *X1, *Gd = nullptr, *ldd = nullptr;
  int *stat, *sgd = nullptr;
  Arena measure;
  layout(measure, ew, cw, lw, E, expV, U, D, X0, X1, stat, io, Gd, ldd, sgd);
  CKS(ensure_ws(h, measure.off));
  Arena ar;
  ar.base = h->ws;
  layout(ar, ew, cw, lw, E, expV, U, D, X0, X1, stat, io, Gd, ldd, sgd);
  cudaStream_t st = h->cur;

  const double* Kd = K;
  const double* Vd = V;
  double* Gout = G;
  double* ldout = logdet;
  int* sgout = sign;
  int* stout = status ? status : stat;
  if (host) {
    if (cudaMemcpyAsync(io.K, K, NN * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(io.V, V, (size_t)M * N * batch * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return DQMC_ERR_CUDA;
    Kd = io.K;
    Vd = io.V;
    Gout = G ? Gd : nullptr;
    ldout = ldd;
    sgout = sgd;
    stout = stat;
  }
  if (cudaMemsetAsync(stout, 0, sizeof(int) * batch, st) != cudaSuccess) return DQMC_ERR_CUDA;

  CKS(run_expm(h, Kd, N, dtau, -1.0, ew, stout, batch));
  // exp(V_l) for every slice, padded to Mp slices per instance
  CK(exp_pad(Vd, expV, batch, M, (int)Mp, N, 1.0, stout, st));

  if (tree) {
    const double *Ut, *Dt, *Xt;
    CKS(run_chain_tree(h, batch, N, M, k, E, expV, Mp * N, tw, stout, &Ut, &Dt, &Xt));
    CKS(run_inversion(h, batch, N, Ut, NN, Dt, N, Xt, NN, Gout, ldout, sgout, stout, lw, pw));
  } else {
    if (cw.oz_s > 0) CK(split_E(E, N, 0, cw, st));   // E slices, shared by all instances
    CK(set_identity(U, NN, N, batch, st));
    CK(set_const(D, (long long)N * batch, 1.0, st));
    CK(set_identity(X0, NN, N, batch, st));
    Slots s;
    s.U = U; s.slotU = 0; s.instU = NN;
    s.D = D; s.slotD = 0; s.instD = N;
    s.X = X0; s.slotX = 0; s.instX = NN;
    s.X2 = X1;
    const int nj = pipeline_jobs(cw.oz_s > 0);
    if (batch >= 4 * nj && pipeline_enabled()) {
      // nj sub-batches on nj streams, product phases staggered so that the QRs
      // of some sub-batches run while the others multiply
      ChainJob J[kMaxJobs];
      make_sub_jobs(J, nj, +1, batch, N, expV, Mp * N, s, cw, stout, nullptr);
      CKS(run_chain_multi(h, J, nj, N, M, k, E));
    } else {
      CKS(run_chain(h, +1, batch, N, M, k, E, expV, Mp * N, s, cw, stout));
    }
    const double* Xf = (nc & 1) ? X1 : X0;
    CKS(run_inversion(h, batch, N, U, NN, D, N, Xf, NN, Gout, ldout, sgout, stout, lw, pw));
  }

  if (host) {
    bool ok = true;
    if (G) ok &= cudaMemcpyAsync(G, Gd, NN * batch * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (logdet) ok &= cudaMemcpyAsync(logdet, ldd, batch * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (sign) ok &= cudaMemcpyAsync(sign, sgd, batch * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (status) ok &= cudaMemcpyAsync(status, stat, batch * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok &= cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) return DQMC_ERR_CUDA;
  }
  return DQMC_OK;
}

}  // extern "C"

// Equal-time path on a caller-supplied device workspace (used by the
// allocation-free entry point in noalloc.cu).  It runs the same helpers as
// dqmc_greens with a handle that lives on the host stack, the chain in one
// stream (no pipelining, so no stream or event is created), and no
// cudaMalloc: when the problem needs more than ws_bytes it returns
// DQMC_ERR_SCRATCH before launching anything.
namespace {
// True when p is NULL or memory the device can address directly (device or
// managed); a host pointer given to a kernel would fault the context, so the
// handle-free entry point rejects it with an error code instead.
bool device_addressable(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

namespace dqmc {
dqmc_status greens_on_workspace(void* stream, void* ws, size_t ws_bytes, int batch, int N, int M,
                                const double* K, double dtau, const double* V, int k, double* G,
                                double* logdet, int* sign, int* status) {
  dqmc_handle_s local;
  dqmc_handle h = &local;
  h->stream = (cudaStream_t)stream;
  CKS(check_common(h, batch, N, M, K, dtau, V, k));
  h->cur = h->stream;
  if (batch == 0) return DQMC_OK;
  if ((((uintptr_t)G | (uintptr_t)logdet) & 7) || (((uintptr_t)sign | (uintptr_t)status) & 3))
    return DQMC_ERR_ARG;
  for (const void* p : {(const void*)K, (const void*)V, (const void*)G, (const void*)logdet,
                        (const void*)sign, (const void*)status})
    if (!device_addressable(p)) return DQMC_ERR_ARG;
  const long long NN = (long long)N * N;
  const int nc = n_chunks(M, k);
  const long long Mp = (long long)(nc + 1) * k;
  ExpmWs ew; ChainWs cw; LohWs lw;
  double *expV, *U, *D, *X0, *X1;
  int* stat;
  auto layout = [&](Arena& ar) {
    take_expm(ar, N, ew);
    expV = ar.take<double>(Mp * N * batch);
    U = ar.take<double>(NN * batch);
    D = ar.take<double>((long long)N * batch);
    X0 = ar.take<double>(NN * batch);
    X1 = ar.take<double>(NN * batch);
    take_chain(ar, batch, N, cw);
    take_loh(ar, batch, N, lw);
    stat = ar.take<int>(batch);
  };
  Arena measure;
  layout(measure);
  if (measure.off > ws_bytes) return DQMC_ERR_SCRATCH;
  Arena ar;
  ar.base = static_cast<char*>(ws);
  layout(ar);
  cudaStream_t st = h->cur;
  int* stout = status ? status : stat;
  // the workspace keeps the previous call's contents: zero what accumulates
  if (cudaMemsetAsync(stout, 0, sizeof(int) * batch, st) != cudaSuccess) return DQMC_ERR_CUDA;
  CKS(run_expm(h, K, N, dtau, -1.0, ew, stout, batch));
  CK(exp_pad(V, expV, batch, M, (int)Mp, N, 1.0, stout, st));
  CK(set_identity(U, NN, N, batch, st));
  CK(set_const(D, (long long)N * batch, 1.0, st));
  CK(set_identity(X0, NN, N, batch, st));
  Slots s;
  s.U = U; s.slotU = 0; s.instU = NN;
  s.D = D; s.slotD = 0; s.instD = N;
  s.X = X0; s.slotX = 0; s.instX = NN;
  s.X2 = X1;
  CKS(run_chain(h, +1, batch, N, M, k, ew.t0, expV, Mp * N, s, cw, stout));
  const double* Xf = (nc & 1) ? X1 : X0;
  CKS(run_loh(h, batch, N, U, NN, D, N, Xf, NN, G, logdet, sign, stout, lw));
  return DQMC_OK;
}
}  // namespace dqmc

extern "C" {

extern "C++" GraphKey key_of(int fn, int batch, int N, int M, const double* K, double dtau,
                             const double* V, int k);
extern "C++" GraphKey key_of(int fn, int batch, int N, int M, const double* K, double dtau,
                             const double* V, int k) {
  GraphKey key;
  key.add((unsigned long long)fn);
  key.add((unsigned long long)batch);
  key.add((unsigned long long)N);
  key.add((unsigned long long)M);
  key.add((unsigned long long)k);
  key.addd(dtau);
  key.addp(K);
  key.addp(V);
  return key;
}

dqmc_status dqmc_greens(dqmc_handle h, int batch, int N, int M, const double* K, double dtau,
                        const double* V, int k, double* G, double* logdet, int* sign,
                        int* status) {
  if (!h) return DQMC_ERR_ARG;
  GraphKey key = key_of(1, batch, N, M, K, dtau, V, k);
  key.addp(G); key.addp(logdet); key.addp(sign); key.addp(status);
  return graph_call(h, key, [&] {
    return greens_impl(h, batch, N, M, K, dtau, V, k, G, logdet, sign, status);
  });
}

dqmc_status dqmc_logdet(dqmc_handle h, int batch, int N, int M, const double* K, double dtau,
                        const double* V, int k, double* logdet, int* sign, int* status) {
  if (!h) return DQMC_ERR_ARG;
  GraphKey key = key_of(2, batch, N, M, K, dtau, V, k);
  key.addp(logdet); key.addp(sign); key.addp(status);
  return graph_call(h, key, [&] {
    return greens_impl(h, batch, N, M, K, dtau, V, k, nullptr, logdet, sign, status);
  });
}

}  // extern "C"


// ---------------------------------------------------------------------------
// Two stacks (App. A) and the D+/D- split middle matrix of Eq. (inversion_tdgf_loh)
//
// Forward slot j:  B(tau_j, 0)       = U_F a X_F          (Eq. (stabmult) chain)
// Backward slot j: B(beta, tau_j)^T  = U_b b T_b          (same chain on B_l^T)
// With a = a_p a_m, b = b_p b_m (a_p = max(a,1), a_m = min(a,1)):
//   mid = a_p^{-1} (U_F^T U_b) b_p^{-1} + a_m (X_F T_b^T) b_m        (all factors <= 1)
//   1 + B(tau,0) B(beta,tau)       = U_F a_p mid b_p U_b^T
//   B(tau,0)^{-1} + B(beta,tau)    = X_F^{-1} a_m^{-1} mid b_p U_b^T
//   B(tau,0) + B(beta,tau)^{-1}    = U_F a_p mid b_m^{-1} T_b^{-T}
// so that
//   G(tau,tau) = U_b b_p^{-1} mid^{-1} a_p^{-1} U_F^T
//   G(tau,0)   = U_b b_p^{-1} mid^{-1} a_m X_F
//   G(0,tau)   = -T_b^T b_m mid^{-1} a_p^{-1} U_F^T
// The second line is Eq. (inversion_tdgf_loh) with the left chain
// B_1^{-1}...B_l^{-1} = X_F^{-1} a^{-1} U_F^T taken from the forward stack
// (its scales a^{-1} split as D_Lp = a_m^{-1}, D_Lm = a_p^{-1}); the first is
// the same split applied to the equal-time bracket of App. A; the third is
// the second case of Eq. (tdgf_propagate), -(1 - G_1) B(tau,0)^{-1}
// = -[B(tau,0) + B(beta,tau)^{-1}]^{-1}.  One LU of mid serves all three:
// G(tau,tau) and G(0,tau) share the solve Z = mid^{-1} a_p^{-1} U_F^T.
// ---------------------------------------------------------------------------
namespace {

struct StackWs {
  double *UF, *DF, *XF, *Ub, *Db, *Tb;
};

void take_stacks(Arena& ar, int batch, int N, int nt, StackWs& w) {
  long long NN = (long long)N * N, Q = (long long)batch * nt;
  w.UF = ar.take<double>(Q * NN);
  w.DF = ar.take<double>(Q * N);
  w.XF = ar.take<double>(Q * NN);
  w.Ub = ar.take<double>(Q * NN);
  w.Db = ar.take<double>(Q * N);
  w.Tb = ar.take<double>(Q * NN);
}

dqmc_status run_stacks(dqmc_handle h, int batch, int N, int M, int k, const double* E,
                       const double* expV, long long sV, const StackWs& w, const ChainWs& cw,
                       const ChainWs& cw2, int* status) {
  cudaStream_t st = h->cur;
  const int nc = n_chunks(M, k), nt = nc + 1;
  const long long NN = (long long)N * N;
  // forward slot 0 and backward slot nc are the identity decomposition
  if (cw.oz_s > 0) {
    CK(split_E(E, N, 0, cw, st));
    CK(split_E(E, N, 1, cw2, st));
  }
  CK(set_identity(w.UF, nt * NN, N, batch, st));
  CK(set_const_strided(w.DF, (long long)nt * N, N, batch, 1.0, st));
  CK(set_identity(w.XF, nt * NN, N, batch, st));
  CK(set_identity(w.Ub + nc * NN, nt * NN, N, batch, st));
  CK(set_const_strided(w.Db + (long long)nc * N, (long long)nt * N, N, batch, 1.0, st));
  CK(set_identity(w.Tb + nc * NN, nt * NN, N, batch, st));
  Slots f;
  f.U = w.UF; f.slotU = NN; f.instU = nt * NN;
  f.D = w.DF; f.slotD = N; f.instD = (long long)nt * N;
  f.X = w.XF; f.slotX = NN; f.instX = nt * NN;
  Slots b;
  b.U = w.Ub; b.slotU = NN; b.instU = nt * NN;
  b.D = w.Db; b.slotD = N; b.instD = (long long)nt * N;
  b.X = w.Tb; b.slotX = NN; b.instX = nt * NN;
  if (pipeline_enabled()) {
    // the forward and backward chains are independent: run them as a pair
    ChainJob J[2];
    J[0].dir = +1; J[0].batch = batch; J[0].expV = expV; J[0].sV = sV; J[0].s = f; J[0].w = cw;
    J[0].status = status;
    J[1].dir = -1; J[1].batch = batch; J[1].expV = expV; J[1].sV = sV; J[1].s = b; J[1].w = cw2;
    J[1].status = status;
    CKS(run_chain_pair(h, J, N, M, k, E));
  } else {
    CKS(run_chain(h, +1, batch, N, M, k, E, expV, sV, f, cw, status));
    CKS(run_chain(h, -1, batch, N, M, k, E, expV, sV, b, cw2, status));
  }
  return DQMC_OK;
}

struct MidWs {
  double *C1, *C2, *mid, *R, *Z, *Wlu, *bpinv;
};

void take_mid(Arena& ar, long long Q, int N, int ncols, MidWs& w) {
  long long NN = (long long)N * N;
  w.C1 = ar.take<double>(Q * NN);
  w.C2 = ar.take<double>(Q * NN);
  w.mid = ar.take<double>(Q * NN);
  w.R = ar.take<double>(Q * N * (long long)ncols);
  w.Z = ar.take<double>(Q * N * (long long)ncols);
  w.Wlu = ar.take<double>(Q * N * (long long)(N + ncols));
  w.bpinv = ar.take<double>(Q * N);
}

// Problems q = b*nt + j over all stack slots; writes G(tau,tau) to Gtt,
// G(tau,0) to Gt0 and G(0,tau) to G0t (each may be null), each Q x N x N.
dqmc_status run_two_stack_inversion(dqmc_handle h, int Q, int N, int nt, const StackWs& w,
                                    const MidWs& m, double* Gtt, double* Gt0, double* G0t,
                                    int* status) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const bool want_z = Gtt || G0t;                      // Z = mid^{-1} a_p^{-1} U_F^T
  const int ncols = (want_z ? N : 0) + (Gt0 ? N : 0);
  if (ncols == 0) return DQMC_OK;
  const double gflops = 2.0 * N * (double)N * N * Q;
  GemmArgs g1;                                         // C1 = U_F^T U_b
  g1.M = g1.N = g1.K = N; g1.batch = Q;
  g1.A = w.UF; g1.lda = N; g1.sA = NN; g1.transA = 1;
  g1.B = w.Ub; g1.ldb = N; g1.sB = NN;
  g1.C = m.C1; g1.ldc = N; g1.sC = NN;
  CKP(PC_OTHER, gflops, gemm_f64(g1, st));
  GemmArgs g2;                                         // C2 = X_F T_b^T
  g2.M = g2.N = g2.K = N; g2.batch = Q;
  g2.A = w.XF; g2.lda = N; g2.sA = NN;
  g2.B = w.Tb; g2.ldb = N; g2.sB = NN; g2.transB = 1;
  g2.C = m.C2; g2.ldc = N; g2.sC = NN;
  CKP(PC_OTHER, gflops, gemm_f64(g2, st));
  Axpby2Args ax;                                       // mid
  ax.N = N; ax.batch = Q;
  ax.A = m.C1; ax.sA = NN;
  ax.ra = w.DF; ax.ra_mode = 1; ax.sra = N;
  ax.ca = w.Db; ax.ca_mode = 1; ax.sca = N;
  ax.B = m.C2; ax.sB = NN;
  ax.rb = w.DF; ax.rb_mode = 2; ax.srb = N;
  ax.cb = w.Db; ax.cb_mode = 2; ax.scb = N;
  ax.C = m.mid; ax.sC = NN;
  CK(axpby2(ax, st));
  CK(build_rhs(N, Q, w.UF, w.XF, w.DF, m.R, ncols, want_z, Gt0 != nullptr, st));
  LuArgs lu;
  lu.N = N; lu.nrhs = ncols; lu.batch = Q;
  lu.A = m.mid; lu.sA = NN;
  lu.R = m.R; lu.sR = (long long)N * ncols; lu.ldr = ncols;
  lu.Z = m.Z; lu.sZ = (long long)N * ncols; lu.ldz = ncols;
  lu.W = m.Wlu; lu.sW = (long long)N * (N + ncols);
  lu.status = status; lu.status_div = nt;
  CKP(PC_LU, lu_flops(N, ncols) * Q, lu_solve_f64(lu, st));
  CK(dsplit_vec(w.Db, N, N, Q, m.bpinv, 1, st));
  for (int part = 0; part < 2; ++part) {
    double* out = part == 0 ? Gtt : Gt0;
    if (!out) continue;
    GemmArgs g;                                        // G = U_b b_p^{-1} Z
    g.M = g.N = g.K = N; g.batch = Q;
    g.A = w.Ub; g.lda = N; g.sA = NN;
    g.B = m.Z + ((part == 1 && want_z) ? N : 0); g.ldb = ncols; g.sB = (long long)N * ncols;
    g.ms = m.bpinv; g.sms = N;
    g.C = out; g.ldc = N; g.sC = NN;
    CKP(PC_OTHER, gflops, gemm_f64(g, st));
  }
  if (G0t) {
    // b_m overwrites b_p^{-1}: the products above are ahead of it on the stream
    CK(dsplit_vec(w.Db, N, N, Q, m.bpinv, 2, st));
    GemmArgs g;                                        // G(0,tau) = -T_b^T b_m Z
    g.M = g.N = g.K = N; g.batch = Q;
    g.A = w.Tb; g.lda = N; g.sA = NN; g.transA = 1;
    g.B = m.Z; g.ldb = ncols; g.sB = (long long)N * ncols;
    g.ms = m.bpinv; g.sms = N;
    g.alpha = -1.0;
    g.C = G0t; g.ldc = N; g.sC = NN;
    CKP(PC_OTHER, gflops, gemm_f64(g, st));
  }
  return DQMC_OK;
}

// G(tau,0) by Eq. (inversion_tdgf) (DQMC_INV_PLAIN), the scheme Sec. 6.2.1
// shows to lose accuracy at tau ~ beta/2.  Both terms of
//   G(tau,0) = [B(tau,0)^{-1} + B(beta,tau)]^{-1} = [U_L D_L X_L + U_R D_R X_R]^{-1}
// are first brought to U D X form with an orthogonal left factor from the
// stacks, by one pivoted QR each:
//   B(tau,0)^{-1} = X_F^{-1} a^{-1} U_F^T,   udt(X_F^{-1} a^{-1}) = u_L d_L x_L,
//                   U_L = u_L, D_L = d_L, X_L = x_L U_F^T;
//   B(beta,tau)   = T_b^T b U_b^T,           udt(T_b^T b) = u_R d_R x_R,
//                   U_R = u_R, D_R = d_R, X_R = x_R U_b^T;
// then, without splitting the scales,
//   D_L X_L X_R^{-1} + U_L^T U_R D_R = u d x,   G(tau,0) = (x X_R)^{-1} d^{-1} (U_L u)^T.
struct SumWs {
  double *ones, *Xi, *ainv, *uL, *dL, *XL, *TbT, *uR, *dR, *XR, *C1, *C2, *u, *d, *dinv, *xXR,
      *Y, *W, *T, *Wlu;
  int* perm;
};

void take_sum(Arena& ar, long long Q, int N, SumWs& w) {
  const long long NN = (long long)N * N;
  w.ones = ar.take<double>(N);
  for (double** m : {&w.Xi, &w.uL, &w.XL, &w.TbT, &w.uR, &w.XR, &w.C1, &w.C2, &w.u, &w.xXR,
                     &w.Y, &w.W, &w.T})
    *m = ar.take<double>(Q * NN);
  for (double** v : {&w.ainv, &w.dL, &w.dR, &w.d, &w.dinv}) *v = ar.take<double>(Q * N);
  w.Wlu = ar.take<double>(Q * 2 * NN);
  w.perm = ar.take<int>(Q * N);
}

dqmc_status run_inv_sum_t0(dqmc_handle h, int Q, int N, int nt, const StackWs& s,
                           const SumWs& w, double* Gt0, int* status) {
  cudaStream_t st = h->cur;
  const long long NN = (long long)N * N;
  const double f2 = 2.0 * N * (double)N * N * Q;
  auto qr = [&](const double* A, const double* Din, double* U, double* D) {
    QrpArgs q;
    q.N = N; q.batch = Q;
    q.A = A; q.sA = NN;
    q.Din = Din; q.sDin = N;
    q.W = w.W; q.sW = NN;
    q.U = U; q.sU = NN;
    q.D = D; q.sD = N;
    q.T = w.T; q.sT = NN;
    q.perm = w.perm; q.sperm = N;
    q.status = status; q.status_div = nt;
    return qrp_f64(q, st);
  };
  // x P^T V^T for the last QR's T' and perm: rows of V^T gathered by perm
  auto x_times_Vt = [&](const double* Vm, double* out) {
    GemmArgs g;
    g.M = g.N = g.K = N; g.batch = Q;
    g.A = w.T; g.lda = N; g.sA = NN; g.upperA = 1;
    g.B = Vm; g.ldb = N; g.sB = NN; g.transB = 1;
    g.permB = w.perm; g.sperm = N;
    g.C = out; g.ldc = N; g.sC = NN;
    return gemm_f64(g, st);
  };
  CK(set_const(w.ones, N, 1.0, st));
  LuArgs li;                                          // X_F^{-1}
  li.N = N; li.nrhs = N; li.batch = Q;
  li.A = s.XF; li.sA = NN;
  li.Rdiag = w.ones; li.sRdiag = 0;
  li.Z = w.Xi; li.sZ = NN; li.ldz = N;
  li.W = w.Wlu; li.sW = 2 * NN;
  li.status = status; li.status_div = nt;
  CKP(PC_LU, lu_flops(N, N) * Q, lu_solve_f64(li, st));
  CK(dsplit_vec(s.DF, N, N, Q, w.ainv, 4, st));
  CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * Q, qr(w.Xi, w.ainv, w.uL, w.dL));
  CKP(PC_OTHER, f2 / 2, x_times_Vt(s.UF, w.XL));      // X_L = x_L U_F^T
  CK(copy_mats(s.Tb, NN, w.TbT, NN, N, Q, 1, 1, 1, st));
  CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * Q, qr(w.TbT, s.Db, w.uR, w.dR));
  CKP(PC_OTHER, f2 / 2, x_times_Vt(s.Ub, w.XR));      // X_R = x_R U_b^T
  LuArgs lr;                                          // C2 = X_L X_R^{-1}
  lr.N = N; lr.nrhs = N; lr.batch = Q;
  lr.A = w.XR; lr.sA = NN; lr.transA = 1;
  lr.R = w.XL; lr.sR = NN; lr.ldr = N; lr.transR = 1;
  lr.Z = w.C2; lr.sZ = NN; lr.ldz = N; lr.transZ = 1;
  lr.W = w.Wlu; lr.sW = 2 * NN;
  lr.status = status; lr.status_div = nt;
  CKP(PC_LU, lu_flops(N, N) * Q, lu_solve_f64(lr, st));
  GemmArgs g1;                                        // C1 = U_L^T U_R
  g1.M = g1.N = g1.K = N; g1.batch = Q;
  g1.A = w.uL; g1.lda = N; g1.sA = NN; g1.transA = 1;
  g1.B = w.uR; g1.ldb = N; g1.sB = NN;
  g1.C = w.C1; g1.ldc = N; g1.sC = NN;
  CKP(PC_OTHER, f2, gemm_f64(g1, st));
  Axpby2Args ax;                                      // D_L C2 + C1 D_R
  ax.N = N; ax.batch = Q;
  ax.A = w.C2; ax.sA = NN; ax.ra = w.dL; ax.ra_mode = 5; ax.sra = N;
  ax.B = w.C1; ax.sB = NN; ax.cb = w.dR; ax.cb_mode = 5; ax.scb = N;
  ax.C = w.C2; ax.sC = NN;
  CK(axpby2(ax, st));
  CKP(PC_QRP, 8.0 / 3.0 * N * N * (double)N * Q, qr(w.C2, nullptr, w.u, w.d));
  GemmArgs gx;                                        // x X_R
  gx.M = gx.N = gx.K = N; gx.batch = Q;
  gx.A = w.T; gx.lda = N; gx.sA = NN; gx.upperA = 1;
  gx.B = w.XR; gx.ldb = N; gx.sB = NN;
  gx.permB = w.perm; gx.sperm = N;
  gx.C = w.xXR; gx.ldc = N; gx.sC = NN;
  CKP(PC_OTHER, f2 / 2, gemm_f64(gx, st));
  CK(dsplit_vec(w.d, N, N, Q, w.dinv, 4, st));
  GemmArgs gy;                                        // Y = U_L u d^{-1}
  gy.M = gy.N = gy.K = N; gy.batch = Q;
  gy.A = w.uL; gy.lda = N; gy.sA = NN;
  gy.B = w.u; gy.ldb = N; gy.sB = NN;
  gy.cs = w.dinv; gy.scs = N;
  gy.C = w.Y; gy.ldc = N; gy.sC = NN;
  CKP(PC_OTHER, f2, gemm_f64(gy, st));
  LuArgs lg;                                          // (x X_R) G = Y^T
  lg.N = N; lg.nrhs = N; lg.batch = Q;
  lg.A = w.xXR; lg.sA = NN;
  lg.R = w.Y; lg.sR = NN; lg.ldr = N; lg.transR = 1;
  lg.Z = Gt0; lg.sZ = NN; lg.ldz = N;
  lg.W = w.Wlu; lg.sW = 2 * NN;
  lg.status = status; lg.status_div = nt;
  CKP(PC_LU, lu_flops(N, N) * Q, lu_solve_f64(lg, st));
  return DQMC_OK;
}

}  // namespace

extern "C" {

static dqmc_status tdisplaced_impl(dqmc_handle h, int batch, int N, int M, const double* K,
                                   double dtau, const double* V, int k, double* Gtt, double* Gt0,
                                   double* G0t, int* status, bool all_tau = false,
                                   const int* shift = nullptr);

dqmc_status dqmc_greens_tdisplaced_from(dqmc_handle h, int batch, int N, int M, const double* K,
                                        double dtau, const double* V, int k, const int* l0,
                                        int every_tau, double* Gtt, double* Gt0, double* G0t,
                                        int* status) {
  if (!h) return DQMC_ERR_ARG;
  if (batch > 0 && !l0) return DQMC_ERR_ARG;
  GraphKey key = key_of(6, batch, N, M, K, dtau, V, k);
  key.addp(l0); key.add((unsigned long long)every_tau);
  key.addp(Gtt); key.addp(Gt0); key.addp(G0t); key.addp(status);
  return graph_call(h, key, [&] {
    return tdisplaced_impl(h, batch, N, M, K, dtau, V, k, Gtt, Gt0, G0t, status, every_tau != 0,
                           l0);
  });
}

dqmc_status dqmc_greens_tdisplaced_all(dqmc_handle h, int batch, int N, int M, const double* K,
                                       double dtau, const double* V, int k, double* Gtt,
                                       double* Gt0, double* G0t, int* status) {
  if (!h) return DQMC_ERR_ARG;
  GraphKey key = key_of(5, batch, N, M, K, dtau, V, k);
  key.addp(Gtt); key.addp(Gt0); key.addp(G0t); key.addp(status);
  return graph_call(h, key, [&] {
    return tdisplaced_impl(h, batch, N, M, K, dtau, V, k, Gtt, Gt0, G0t, status, true);
  });
}

dqmc_status dqmc_greens_tdisplaced_ex(dqmc_handle h, int batch, int N, int M, const double* K,
                                      double dtau, const double* V, int k, double* Gtt,
                                      double* Gt0, double* G0t, int* status) {
  if (!h) return DQMC_ERR_ARG;
  GraphKey key = key_of(3, batch, N, M, K, dtau, V, k);
  key.addp(Gtt); key.addp(Gt0); key.addp(G0t); key.addp(status);
  return graph_call(h, key, [&] {
    return tdisplaced_impl(h, batch, N, M, K, dtau, V, k, Gtt, Gt0, G0t, status);
  });
}

dqmc_status dqmc_greens_tdisplaced(dqmc_handle h, int batch, int N, int M, const double* K,
                                   double dtau, const double* V, int k, double* Gtt, double* Gt0,
                                   int* status) {
  return dqmc_greens_tdisplaced_ex(h, batch, N, M, K, dtau, V, k, Gtt, Gt0, nullptr, status);
}

static dqmc_status tdisplaced_impl(dqmc_handle h, int batch, int N, int M, const double* K,
                                   double dtau, const double* V, int k, double* Gtt, double* Gt0,
                                   double* G0t, int* status, bool all_tau, const int* shift) {
  CKS(check_common(h, batch, N, M, K, dtau, V, k));
  if (h->prec != DQMC_CHAIN_FP64 && N > 256) return DQMC_ERR_UNSUPPORTED;
  h->launches = 0;
  h->cur = h->stream;
  if (batch == 0) return DQMC_OK;
  const bool host = h->pmode == DQMC_PTR_HOST;
  const long long NN = (long long)N * N;
  const int nc = n_chunks(M, k), nt = nc + 1;
  const long long Mp = (long long)(nc + 1) * k;
  const long long Q = (long long)batch * nt;
  if (Q > (1LL << 30)) return DQMC_ERR_ARG;
  const bool plain_t0 = h->inv == DQMC_INV_PLAIN && Gt0 != nullptr;
  const int ncols = (Gtt || G0t ? N : 0) + (Gt0 && !plain_t0 ? N : 0);
  // outputs per instance: the k-grid, or (all_tau) every tau_l = l dtau, l = 0..M
  const long long outlen = all_tau ? (long long)(M + 1) * NN : (long long)nt * NN;

  ExpmWs ew, ewi; ChainWs cw, cw2; StackWs sw; MidWs mw; HostIO io; SumWs sumw;
  double *expV, *expmV = nullptr, *Gttd = nullptr, *Gt0d = nullptr, *G0td = nullptr;
  double *gq[3] = {nullptr, nullptr, nullptr}, *gtmp = nullptr;   // grid values (all_tau)
  int* stat;
  int* shiftd = nullptr;
  auto layout = [&](Arena& ar) {
    take_expm(ar, N, ew);
    expV = ar.take<double>(Mp * N * batch);
    if (all_tau) {
      take_expm(ar, N, ewi);
      if (Gtt || G0t) expmV = ar.take<double>(Mp * N * batch);
      if (Gtt) gq[0] = ar.take<double>(Q * NN);
      if (Gt0) gq[1] = ar.take<double>(Q * NN);
      if (G0t) gq[2] = ar.take<double>(Q * NN);
      gtmp = ar.take<double>(Q * NN);
    }
    take_chain(ar, batch, N, cw);
    take_chain(ar, batch, N, cw2);
    if (h->prec != DQMC_CHAIN_FP64) {
      take_ozaki(ar, batch, N, (int)h->prec, cw);
      take_ozaki(ar, batch, N, (int)h->prec, cw2);
    }
    take_stacks(ar, batch, N, nt, sw);
    take_mid(ar, Q, N, ncols > 0 ? ncols : N, mw);
    if (plain_t0) take_sum(ar, Q, N, sumw);
    stat = ar.take<int>(batch);
    if (host) {
      io.K = ar.take<double>(NN);
      io.V = ar.take<double>((long long)M * N * batch);
      if (shift) shiftd = ar.take<int>(batch);
      Gttd = Gtt ? ar.take<double>(batch * outlen) : nullptr;
      Gt0d = Gt0 ? ar.take<double>(batch * outlen) : nullptr;
      G0td = G0t ? ar.take<double>(batch * outlen) : nullptr;
    }
  };
  Arena measure;
  layout(measure);
  CKS(ensure_ws(h, measure.off));
  Arena ar;
  ar.base = h->ws;
  layout(ar);
  cudaStream_t st = h->cur;
  const double* Kd = K;
  const double* Vd = V;
  double* Gtto = Gtt;
  double* Gt0o = Gt0;
  double* G0to = G0t;
  int* stout = status ? status : stat;
  if (host) {
    if (cudaMemcpyAsync(io.K, K, NN * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(io.V, V, (size_t)M * N * batch * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return DQMC_ERR_CUDA;
    if (shift && cudaMemcpyAsync(shiftd, shift, batch * sizeof(int), cudaMemcpyHostToDevice,
                                 st) != cudaSuccess)
      return DQMC_ERR_CUDA;
    Kd = io.K; Vd = io.V; Gtto = Gttd; Gt0o = Gt0d; G0to = G0td; stout = stat;
  }
  if (cudaMemsetAsync(stout, 0, sizeof(int) * batch, st) != cudaSuccess) return DQMC_ERR_CUDA;
  CKS(run_expm(h, Kd, N, dtau, -1.0, ew, stout, batch));
  const int* sh = host ? shiftd : shift;   // time translation of the chain (nullable)
  CK(exp_pad(Vd, expV, batch, M, (int)Mp, N, 1.0, stout, st, sh));
  CKS(run_stacks(h, batch, N, M, k, ew.t0, expV, Mp * N, sw, cw, cw2, stout));
  double* out[3] = {Gtto, Gt0o, G0to};
  if (all_tau)
    for (int i = 0; i < 3; ++i) out[i] = gq[i];
  CKS(run_two_stack_inversion(h, (int)Q, N, nt, sw, mw, out[0], plain_t0 ? nullptr : out[1],
                              out[2], stout));
  if (plain_t0) CKS(run_inv_sum_t0(h, (int)Q, N, nt, sw, sumw, out[1], stout));
  if (all_tau) {
    // tau between grid points: k - 1 one-slice steps from every grid value,
    //   G(tau_l, 0) = B_l G(tau_{l-1}, 0),  G(0, tau_l) = G(0, tau_{l-1}) B_l^{-1},
    //   G_{l+1} = B_l G_l B_l^{-1}   (Eqs. (tdgf_propagate), (etgf_tau)),
    // with B_l = E e^{V_l} and B_l^{-1} = e^{-V_l} E^{-1}.
    CKS(run_expm(h, Kd, N, dtau, +1.0, ewi, nullptr, batch));
    if (expmV) CK(exp_pad(Vd, expmV, batch, M, (int)Mp, N, -1.0, nullptr, st, sh));
    double* dst[3] = {Gtto, Gt0o, G0to};
    const double f2 = 2.0 * N * (double)N * N * Q;
    for (int s = 0; s < k; ++s) {
      for (int i = 0; i < 3; ++i)
        if (out[i]) CK(scatter_tau(out[i], Q, nt, N, k, M, s, dst[i], st));
      if (s == k - 1) break;
      GemmArgs left;                                   // E diag(e^{V_l}) G
      left.M = left.N = left.K = N; left.batch = (int)Q;
      left.A = ew.t0; left.lda = N; left.sA = 0;
      left.ldb = N; left.sB = NN;
      left.ms = expV + (long long)s * N; left.sms = Mp * N;
      left.sms_inner = (long long)k * N; left.divS = nt;
      left.ldc = N; left.sC = NN;
      GemmArgs right;                                  // G diag(e^{-V_l}) E^{-1}
      right.M = right.N = right.K = N; right.batch = (int)Q;
      right.lda = N; right.sA = NN;
      right.B = ewi.t0; right.ldb = N; right.sB = 0;
      right.ms = expmV + (long long)s * N; right.sms = Mp * N;
      right.sms_inner = (long long)k * N; right.divS = nt;
      right.ldc = N; right.sC = NN;
      if (out[1]) {
        left.B = out[1]; left.C = gtmp;
        CKP(PC_OTHER, f2, gemm_f64(left, st));
        std::swap(out[1], gtmp);
      }
      if (out[2]) {
        right.A = out[2]; right.C = gtmp;
        CKP(PC_OTHER, f2, gemm_f64(right, st));
        std::swap(out[2], gtmp);
      }
      if (out[0]) {
        left.B = out[0]; left.C = gtmp;
        CKP(PC_OTHER, f2, gemm_f64(left, st));
        right.A = gtmp; right.C = out[0];
        CKP(PC_OTHER, f2, gemm_f64(right, st));
      }
    }
  }
  if (host) {
    bool ok = true;
    const size_t ob = (size_t)batch * outlen * sizeof(double);
    if (Gtt) ok &= cudaMemcpyAsync(Gtt, Gttd, ob, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (Gt0) ok &= cudaMemcpyAsync(Gt0, Gt0d, ob, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (G0t) ok &= cudaMemcpyAsync(G0t, G0td, ob, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (status) ok &= cudaMemcpyAsync(status, stat, batch * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok &= cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) return DQMC_ERR_CUDA;
  }
  return DQMC_OK;
}

// Gradient: checkpoints G(tau_j, tau_j) = G_{jk+1} from the stacks, then
// G_{l+1} = B_l G_l B_l^{-1} = E (e^{V_l} G_l e^{-V_l}) E^{-1} for the other
// slices of each chunk; dV_l(i) = 1 - G_l(i,i).  All chunks wrap in parallel.
static dqmc_status grad_impl(dqmc_handle h, int batch, int N, int M, const double* K,
                             double dtau, const double* V, int k, double* logdet, int* sign,
                             double* dV, int* status);

dqmc_status dqmc_logdet_grad(dqmc_handle h, int batch, int N, int M, const double* K, double dtau,
                             const double* V, int k, double* logdet, int* sign, double* dV,
                             int* status) {
  if (!h) return DQMC_ERR_ARG;
  GraphKey key = key_of(4, batch, N, M, K, dtau, V, k);
  key.addp(logdet); key.addp(sign); key.addp(dV); key.addp(status);
  return graph_call(h, key, [&] {
    return grad_impl(h, batch, N, M, K, dtau, V, k, logdet, sign, dV, status);
  });
}

static dqmc_status grad_impl(dqmc_handle h, int batch, int N, int M, const double* K,
                             double dtau, const double* V, int k, double* logdet, int* sign,
                             double* dV, int* status) {
  CKS(check_common(h, batch, N, M, K, dtau, V, k));
  if (h->prec != DQMC_CHAIN_FP64 && N > 256) return DQMC_ERR_UNSUPPORTED;
  h->launches = 0;
  h->cur = h->stream;
  if (batch == 0) return DQMC_OK;
  if (!dV) return DQMC_ERR_ARG;
  const bool host = h->pmode == DQMC_PTR_HOST;
  const long long NN = (long long)N * N;
  const int nc = n_chunks(M, k), nt = nc + 1;
  const long long Mp = (long long)(nc + 1) * k;
  const long long Q = (long long)batch * nt;
  if (Q > (1LL << 30)) return DQMC_ERR_ARG;

  ExpmWs ew, ewi; ChainWs cw, cw2; StackWs sw; MidWs mw; LohWs lw; HostIO io;
  double *expV, *expmV, *Gw, *W1, *dVd = nullptr, *ldd = nullptr;
  int *stat, *sgd = nullptr;
  auto layout = [&](Arena& ar) {
    take_expm(ar, N, ew);
    take_expm(ar, N, ewi);
    expV = ar.take<double>(Mp * N * batch);
    expmV = ar.take<double>(Mp * N * batch);
    take_chain(ar, batch, N, cw);
    take_chain(ar, batch, N, cw2);
    if (h->prec != DQMC_CHAIN_FP64) {
      take_ozaki(ar, batch, N, (int)h->prec, cw);
      take_ozaki(ar, batch, N, (int)h->prec, cw2);
    }
    take_stacks(ar, batch, N, nt, sw);
    take_mid(ar, Q, N, N, mw);
    take_loh(ar, batch, N, lw);
    Gw = ar.take<double>(Q * NN);
    W1 = ar.take<double>(Q * NN);
    stat = ar.take<int>(batch);
    if (host) {
      io.K = ar.take<double>(NN);
      io.V = ar.take<double>((long long)M * N * batch);
      dVd = ar.take<double>((long long)M * N * batch);
      ldd = ar.take<double>(batch);
      sgd = ar.take<int>(batch);
    }
  };
  Arena measure;
  layout(measure);
  CKS(ensure_ws(h, measure.off));
  Arena ar;
  ar.base = h->ws;
  layout(ar);
  cudaStream_t st = h->cur;
  const double* Kd = K;
  const double* Vd = V;
  double* dVo = dV;
  double* ldo = logdet;
  int* sgo = sign;
  int* stout = status ? status : stat;
  if (host) {
    if (cudaMemcpyAsync(io.K, K, NN * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(io.V, V, (size_t)M * N * batch * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
      return DQMC_ERR_CUDA;
    Kd = io.K; Vd = io.V; dVo = dVd; ldo = ldd; sgo = sgd; stout = stat;
  }
  if (cudaMemsetAsync(stout, 0, sizeof(int) * batch, st) != cudaSuccess) return DQMC_ERR_CUDA;
  CKS(run_expm(h, Kd, N, dtau, -1.0, ew, stout, batch));
  CKS(run_expm(h, Kd, N, dtau, +1.0, ewi, nullptr, batch));
  CK(exp_pad(Vd, expV, batch, M, (int)Mp, N, 1.0, stout, st));
  CK(exp_pad(Vd, expmV, batch, M, (int)Mp, N, -1.0, nullptr, st));
  CKS(run_stacks(h, batch, N, M, k, ew.t0, expV, Mp * N, sw, cw, cw2, stout));
  // log det from the full forward product B(beta, 0) = U_F a X_F (slot nc)
  CKS(run_loh(h, batch, N, sw.UF + nc * NN, nt * NN, sw.DF + (long long)nc * N, (long long)nt * N,
              sw.XF + nc * NN, nt * NN, nullptr, ldo, sgo, stout, lw));
  // checkpoints G_{jk+1}
  CKS(run_two_stack_inversion(h, (int)Q, N, nt, sw, mw, Gw, nullptr, nullptr, stout));
  const double wflops = 2.0 * N * (double)N * N * Q;
  for (int s = 0; s < k; ++s) {
    CK(grad_readout(Gw, N, (int)Q, nt, k, M, s, dVo, st));
    if (s == k - 1) break;
    GemmArgs a;                                        // W1 = E diag(e^{V_l}) G_l
    a.M = a.N = a.K = N; a.batch = (int)Q;
    a.A = ew.t0; a.lda = N; a.sA = 0;
    a.B = Gw; a.ldb = N; a.sB = NN;
    a.ms = expV + (long long)s * N; a.sms = Mp * N; a.sms_inner = (long long)k * N; a.divS = nt;
    a.C = W1; a.ldc = N; a.sC = NN;
    CKP(PC_OTHER, wflops, gemm_f64(a, st));
    GemmArgs b;                                        // G_{l+1} = W1 diag(e^{-V_l}) E^{-1}
    b.M = b.N = b.K = N; b.batch = (int)Q;
    b.A = W1; b.lda = N; b.sA = NN;
    b.B = ewi.t0; b.ldb = N; b.sB = 0;
    b.ms = expmV + (long long)s * N; b.sms = Mp * N; b.sms_inner = (long long)k * N; b.divS = nt;
    b.C = Gw; b.ldc = N; b.sC = NN;
    CKP(PC_OTHER, wflops, gemm_f64(b, st));
  }
  if (host) {
    bool ok = true;
    ok &= cudaMemcpyAsync(dV, dVd, (size_t)M * N * batch * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (logdet) ok &= cudaMemcpyAsync(logdet, ldd, batch * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (sign) ok &= cudaMemcpyAsync(sign, sgd, batch * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (status) ok &= cudaMemcpyAsync(status, stat, batch * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok &= cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) return DQMC_ERR_CUDA;
  }
  return DQMC_OK;
}

}  // extern "C"

// Ragged batch: instances are grouped by (N, k, dtau, K); each group runs the
// uniform equal-time path with per-instance chain lengths M_b on its own
// stream, so that small-N groups (latency-bound QR) overlap with large-N
// groups (FP64-bound products).  Results are scattered to the pools.
//
// The host work (grouping, workspace sizing, the per-group index tables in
// the handle's rtab buffer) happens before any launch, so the launches alone
// can be recorded as one CUDA graph in graph mode; the graph is keyed by a
// hash of the descriptors together with every pointer, and replayed for an
// identical call.
namespace {

// FNV-1a over the bytes of the descriptor array
unsigned long long hash_desc(const dqmc_instance* d, int batch) {
  unsigned long long x = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(d);
  const size_t n = (size_t)batch * sizeof(dqmc_instance);
  for (size_t i = 0; i < n; ++i) {
    x ^= p[i];
    x *= 1099511628211ull;
  }
  return x ^ (unsigned long long)batch;
}

struct RaggedGroup {
  int N, k;
  double dtau;
  long long offK;
  std::vector<int> idx;
  int Mmax = 0;
};

struct RaggedGroupWs {
  ExpmWs ew; ChainWs cw; LohWs lw; PlainWs pw;
  double *expV, *U, *D, *X0, *X1, *G, *ld;
  int *sg, *st;
  // index tables (in rtab)
  int *Mb, *gidx;
  long long *offV, *offG;
};

}  // namespace

extern "C" {

// E_pool (nullable): exp(-dtau K) of every K of K_pool at the same offsets
// (the registered hopping matrices of dqmc_greens_batched); without it each
// group computes its exponential.
static dqmc_status ragged_impl(dqmc_handle h, int batch, const dqmc_instance* desc,
                               const double* K_pool, const double* E_pool, const double* V_pool,
                               double* G_pool, double* logdet, int* sign, int* status) {
  if (!h || batch < 0) return DQMC_ERR_ARG;
  h->launches = 0;
  h->cur = h->stream;
  if (batch == 0) return DQMC_OK;
  if (!desc || !K_pool || !V_pool) return DQMC_ERR_ARG;
  if (h->pmode == DQMC_PTR_HOST) return DQMC_ERR_UNSUPPORTED;
  const bool mixed = h->prec != DQMC_CHAIN_FP64;
  if (mixed && h->decomp == DQMC_DECOMP_JACOBI) return DQMC_ERR_UNSUPPORTED;
  for (int b = 0; b < batch; ++b) {
    const dqmc_instance& d = desc[b];
    if (d.N < 1 || d.N > 1024 || d.M < 1 || d.k < 1 || d.k > d.M || !(d.dtau >= 0.0) ||
        d.off_K < 0 || d.off_V < 0 || d.off_G < 0)
      return DQMC_ERR_ARG;
    if (mixed && d.N > 256) return DQMC_ERR_UNSUPPORTED;   // tensor-core chain: N <= 256
    if (h->decomp == DQMC_DECOMP_JACOBI && d.N > 512) return DQMC_ERR_UNSUPPORTED;
  }
  // ---- groups ---------------------------------------------------------------
  std::vector<RaggedGroup> groups;
  for (int b = 0; b < batch; ++b) {
    const dqmc_instance& d = desc[b];
    RaggedGroup* g = nullptr;
    for (auto& x : groups)
      if (x.N == d.N && x.k == d.k && x.dtau == d.dtau && x.offK == d.off_K) { g = &x; break; }
    if (!g) {
      groups.push_back(RaggedGroup{d.N, d.k, d.dtau, d.off_K, {}, 0});
      g = &groups.back();
    }
    g->idx.push_back(b);
    if (d.M > g->Mmax) g->Mmax = d.M;
  }
  const int s_digits = mixed ? (int)h->prec : 0;
  // ---- workspace (h->ws) and index tables (h->rtab): one region per group ----
  std::vector<RaggedGroupWs> gw(groups.size());
  auto layout = [&](Arena& ar) {
    for (size_t i = 0; i < groups.size(); ++i) {
      const RaggedGroup& g = groups[i];
      RaggedGroupWs& w = gw[i];
      const int nb = (int)g.idx.size(), N = g.N;
      const long long NN = (long long)N * N;
      const long long Mp = (long long)(n_chunks(g.Mmax, g.k) + 1) * g.k;
      take_expm(ar, N, w.ew);
      w.expV = ar.take<double>(Mp * N * nb);
      w.U = ar.take<double>(NN * nb);
      w.D = ar.take<double>((long long)N * nb);
      w.X0 = ar.take<double>(NN * nb);
      w.X1 = ar.take<double>(NN * nb);
      take_chain(ar, nb, N, w.cw);
      if (mixed) take_ozaki(ar, nb, N, s_digits, w.cw);
      take_loh(ar, nb, N, w.lw);
      if (h->inv == DQMC_INV_PLAIN) take_plain(ar, nb, N, w.pw);
      w.G = ar.take<double>(NN * nb);
      w.ld = ar.take<double>(nb);
      w.sg = ar.take<int>(nb);
      w.st = ar.take<int>(nb);
    }
  };
  auto layout_tables = [&](Arena& ar) {
    for (size_t i = 0; i < groups.size(); ++i) {
      const int nb = (int)groups[i].idx.size();
      gw[i].Mb = ar.take<int>(nb);
      gw[i].gidx = ar.take<int>(nb);
      gw[i].offV = ar.take<long long>(nb);
      gw[i].offG = ar.take<long long>(nb);
    }
  };
  Arena measure, measure_t;
  layout(measure);
  layout_tables(measure_t);
  CKS(ensure_ws(h, measure.off));
  Arena ar;
  ar.base = h->ws;
  layout(ar);
  if (measure_t.off > h->rtab_bytes) {
    if (h->capturing) return DQMC_ERR_UNSUPPORTED;
    if (!within_limit(h, h->rtab_bytes, measure_t.off)) return DQMC_ERR_NOMEM;
    if (h->rtab) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->rtab);
      h->rtab = nullptr;
      h->rtab_bytes = 0;
    }
    h->rtab_key = 0;
    if (cudaMalloc(&h->rtab, measure_t.off) != cudaSuccess) {
      cudaGetLastError();
      h->rtab = nullptr;
      return DQMC_ERR_NOMEM;
    }
    h->rtab_bytes = measure_t.off;
  }
  Arena art;
  art.base = h->rtab;
  layout_tables(art);
  const unsigned long long dkey = hash_desc(desc, batch);
  if (h->rtab_key != dkey) {
    // the tables of this descriptor set; the copies finish before the host
    // vectors go out of scope, and before any launch that reads them
    h->rtab_key = 0;
    cudaStreamSynchronize(h->stream);
    for (size_t i = 0; i < groups.size(); ++i) {
      const RaggedGroup& g = groups[i];
      const int nb = (int)g.idx.size();
      std::vector<int> Mb(nb), gidx(nb);
      std::vector<long long> offV(nb), offG(nb);
      for (int j = 0; j < nb; ++j) {
        const dqmc_instance& d = desc[g.idx[j]];
        Mb[j] = d.M; gidx[j] = g.idx[j]; offV[j] = d.off_V; offG[j] = d.off_G;
      }
      const bool ok =
          cudaMemcpy(gw[i].Mb, Mb.data(), nb * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
          cudaMemcpy(gw[i].gidx, gidx.data(), nb * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
          cudaMemcpy(gw[i].offV, offV.data(), nb * sizeof(long long), cudaMemcpyHostToDevice) == cudaSuccess &&
          cudaMemcpy(gw[i].offG, offG.data(), nb * sizeof(long long), cudaMemcpyHostToDevice) == cudaSuccess;
      if (!ok) return DQMC_ERR_CUDA;
    }
    h->rtab_key = dkey;
  }
  // ---- streams and the fork event (created outside any capture) --------------
  // up to 8 group slots; a slot has its group's stream and nj more for the
  // staggered sub-batches of a group large enough to pipeline
  const int nj = pipeline_jobs(mixed);
  const size_t nslots = groups.size() < 8 ? groups.size() : 8;
  const size_t per_slot = (size_t)nj + 1;
  const size_t nstreams = nslots * per_slot;
  CKS(ensure_aux(h, nstreams));
  if (!h->rfork && cudaEventCreateWithFlags(&h->rfork, cudaEventDisableTiming) != cudaSuccess) {
    h->rfork = nullptr;
    return DQMC_ERR_CUDA;
  }
  GraphKey key;
  key.add(9);
  key.add((unsigned long long)batch);
  key.add(dkey);
  key.addp(K_pool); key.addp(V_pool); key.addp(G_pool);
  key.addp(logdet); key.addp(sign); key.addp(status);
  key.addp(h->rtab); key.addp(E_pool);
  return graph_call(h, key, [&]() -> dqmc_status {
    h->launches = 0;
    h->cur = h->stream;
    // the handle's stream may be a capture stream here: every launch below
    // forks from it through rfork and joins back through auxev
    if (cudaEventRecord(h->rfork, h->stream) != cudaSuccess) return DQMC_ERR_CUDA;
    for (size_t q = 0; q < nstreams; ++q) cudaStreamWaitEvent(h->aux[q], h->rfork, 0);
    dqmc_status rc = DQMC_OK;
    for (size_t i = 0; i < groups.size() && rc == DQMC_OK; ++i) {
      const RaggedGroup& g = groups[i];
      RaggedGroupWs& w = gw[i];
      const int nb = (int)g.idx.size(), N = g.N, k = g.k;
      const long long NN = (long long)N * N;
      const int ncmax = n_chunks(g.Mmax, k);
      const long long Mp = (long long)(ncmax + 1) * k;
      const size_t slot = (i % nslots) * per_slot;
      h->cur = h->aux[slot];
      cudaStream_t st = h->cur;
      rc = [&]() -> dqmc_status {
        if (cudaMemsetAsync(w.st, 0, nb * sizeof(int), st) != cudaSuccess) return DQMC_ERR_CUDA;
        const double* E = E_pool ? E_pool + g.offK : w.ew.t0;
        if (!E_pool) CKS(run_expm(h, K_pool + g.offK, N, g.dtau, -1.0, w.ew, w.st, nb));
        CK(exp_gather(V_pool, w.offV, w.Mb, nb, (int)Mp, N, w.expV, w.st, st));
        if (mixed) CK(split_E(E, N, 0, w.cw, st));   // E slices, shared by the group
        CK(set_identity(w.U, NN, N, nb, st));
        CK(set_const(w.D, (long long)N * nb, 1.0, st));
        CK(set_identity(w.X0, NN, N, nb, st));
        Slots sl;
        sl.U = w.U; sl.slotU = 0; sl.instU = NN;
        sl.D = w.D; sl.slotD = 0; sl.instD = N;
        sl.X = w.X0; sl.slotX = 0; sl.instX = NN;
        sl.X2 = w.X1;
        if (nb >= 4 * nj && pipeline_enabled()) {
          // as a uniform call: sub-batches on their own streams, staggered so
          // that the QRs of some run while the others multiply
          ChainJob J[kMaxJobs];
          make_sub_jobs(J, nj, +1, nb, N, w.expV, Mp * N, sl, w.cw, w.st, w.Mb);
          CKS(run_chain_multi(h, J, nj, N, g.Mmax, k, E, (int)slot + 1));
        } else {
          CKS(run_chain(h, +1, nb, N, g.Mmax, k, E, w.expV, Mp * N, sl, w.cw, w.st, w.Mb));
        }
        const double* Xf = (ncmax & 1) ? w.X1 : w.X0;
        CKS(run_inversion(h, nb, N, w.U, NN, w.D, N, Xf, NN, G_pool ? w.G : nullptr, w.ld, w.sg,
                          w.st, w.lw, w.pw));
        if (G_pool) CK(scatter_mats(w.G, w.offG, N, nb, G_pool, st));
        CK(scatter_scalars(w.gidx, nb, w.ld, w.sg, w.st, logdet, sign, status, st));
        return DQMC_OK;
      }();
    }
    for (size_t q = 0; q < nstreams; ++q) {
      cudaEventRecord(h->auxev[q], h->aux[q]);
      cudaStreamWaitEvent(h->stream, h->auxev[q], 0);
    }
    h->cur = h->stream;
    return rc;
  });
}

dqmc_status dqmc_greens_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                               const double* K_pool, const double* V_pool, double* G_pool,
                               double* logdet, int* sign, int* status) {
  return ragged_impl(h, batch, desc, K_pool, nullptr, V_pool, G_pool, logdet, sign, status);
}

dqmc_status dqmc_register_K(dqmc_handle h, int N, const double* K, double dtau, int* K_id) {
  if (!h || !K || !K_id || N < 1 || N > 1024 || !(dtau >= 0.0) || !(dtau < 1e300))
    return DQMC_ERR_ARG;
  if (((uintptr_t)K) & 7) return DQMC_ERR_ARG;
  if (h->capturing) return DQMC_ERR_UNSUPPORTED;
  *K_id = -1;
  const long long NN = (long long)N * N;
  h->cur = h->stream;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DQMC_ERR_CUDA;
  if (h->kused + NN > h->kcap) {
    // grow both pools; a recorded graph may refer to the old ones
    long long cap = h->kcap * 2 > h->kused + NN ? h->kcap * 2 : h->kused + NN;
    const size_t oldb = 2 * (size_t)h->kcap * sizeof(double);
    if (!within_limit(h, oldb, 2 * (size_t)cap * sizeof(double))) cap = h->kused + NN;
    if (!within_limit(h, oldb, 2 * (size_t)cap * sizeof(double))) return DQMC_ERR_NOMEM;
    double *kp = nullptr, *ep = nullptr;
    if (cudaMalloc(&kp, cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ep, cap * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      if (kp) cudaFree(kp);
      return DQMC_ERR_NOMEM;
    }
    if (h->kused > 0 &&
        (cudaMemcpy(kp, h->kpool, h->kused * sizeof(double), cudaMemcpyDeviceToDevice) != cudaSuccess ||
         cudaMemcpy(ep, h->epool, h->kused * sizeof(double), cudaMemcpyDeviceToDevice) != cudaSuccess)) {
      cudaFree(kp);
      cudaFree(ep);
      return DQMC_ERR_CUDA;
    }
    if (h->kpool) cudaFree(h->kpool);
    if (h->epool) cudaFree(h->epool);
    h->kpool = kp;
    h->epool = ep;
    h->kcap = cap;
    h->gvalid = false;
  }
  const long long off = h->kused;
  const cudaMemcpyKind kind =
      h->pmode == DQMC_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpy(h->kpool + off, K, NN * sizeof(double), kind) != cudaSuccess) return DQMC_ERR_CUDA;
  // exp(-dtau K) once, through the handle's workspace
  ExpmWs ew;
  Arena measure;
  take_expm(measure, N, ew);
  CKS(ensure_ws(h, measure.off));
  Arena ar;
  ar.base = h->ws;
  take_expm(ar, N, ew);
  CKS(run_expm(h, h->kpool + off, N, dtau, -1.0, ew, nullptr, 0));
  int bad = 0;
  if (cudaMemcpyAsync(h->epool + off, ew.t0, NN * sizeof(double), cudaMemcpyDeviceToDevice,
                      h->stream) != cudaSuccess ||
      cudaMemcpyAsync(&bad, ew.asym, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return DQMC_ERR_CUDA;
  if (bad) return DQMC_ERR_ARG;   // not symmetric / not finite / norm beyond the squarings
  h->kreg.push_back({N, dtau, off});
  h->kused += NN;
  *K_id = (int)h->kreg.size() - 1;
  return DQMC_OK;
}

dqmc_status dqmc_greens_batched(dqmc_handle h, int batch, const dqmc_desc* desc,
                                const double* V_pool, double* G_pool, double* logdet, int* sign,
                                int* status) {
  if (!h || batch < 0) return DQMC_ERR_ARG;
  h->launches = 0;
  if (batch == 0) return DQMC_OK;
  if (!desc || !V_pool) return DQMC_ERR_ARG;
  if (h->pmode == DQMC_PTR_HOST) return DQMC_ERR_UNSUPPORTED;
  if (h->capturing) return DQMC_ERR_UNSUPPORTED;
  // the descriptors live on the device: read them back once, after whatever
  // the caller queued on the stream before this call
  std::vector<dqmc_desc> d(batch);
  if (cudaMemcpyAsync(d.data(), desc, (size_t)batch * sizeof(dqmc_desc), cudaMemcpyDeviceToHost,
                      h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_ARG;
  }
  std::vector<dqmc_instance> inst(batch);
  for (int b = 0; b < batch; ++b) {
    const dqmc_desc& x = d[b];
    if (x.K_id < 0 || x.K_id >= (int)h->kreg.size() || x.N != h->kreg[x.K_id].N)
      return DQMC_ERR_ARG;
    const auto& r = h->kreg[x.K_id];
    inst[b] = dqmc_instance{x.N, x.M, x.k, 0, r.dtau, r.off, x.off_V, x.off_G};
  }
  return ragged_impl(h, batch, inst.data(), h->kpool, h->epool, V_pool, G_pool, logdet, sign,
                     status);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Ragged time-displaced G and log-det gradient: instances grouped by
// (N, M, k, dtau, K); each group is gathered into a contiguous batch, run
// through the uniform path and scattered back, one group after another on
// the handle's stream.
// ---------------------------------------------------------------------------
namespace {

struct UGroup {
  int N, M, k;
  double dtau;
  long long offK;
  std::vector<int> idx;
};

dqmc_status group_uniform(int batch, const dqmc_instance* desc, std::vector<UGroup>& groups) {
  for (int b = 0; b < batch; ++b) {
    const dqmc_instance& d = desc[b];
    if (d.N < 1 || d.N > 1024 || d.M < 1 || d.k < 1 || d.k > d.M || !(d.dtau >= 0.0) ||
        d.off_K < 0 || d.off_V < 0 || d.off_G < 0)
      return DQMC_ERR_ARG;
    UGroup* g = nullptr;
    for (auto& x : groups)
      if (x.N == d.N && x.M == d.M && x.k == d.k && x.dtau == d.dtau && x.offK == d.off_K) {
        g = &x;
        break;
      }
    if (!g) {
      groups.push_back(UGroup{d.N, d.M, d.k, d.dtau, d.off_K, {}});
      g = &groups.back();
    }
    g->idx.push_back(b);
  }
  return DQMC_OK;
}

dqmc_status ensure_rws(dqmc_handle h, size_t bytes) {
  if (bytes <= h->rws_bytes) return DQMC_OK;
  if (!within_limit(h, h->rws_bytes, bytes)) return DQMC_ERR_NOMEM;
  if (h->rws) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->rws);
    h->rws = nullptr;
    h->rws_bytes = 0;
  }
  if (cudaMalloc(&h->rws, bytes) != cudaSuccess) {
    cudaGetLastError();
    h->rws = nullptr;
    return DQMC_ERR_NOMEM;
  }
  h->rws_bytes = bytes;
  return DQMC_OK;
}

// Staging of one group: V in, `nout` output blocks of `outlen` doubles per
// instance, per-instance scalars, index tables.
struct Stage {
  double *V, *out[3], *ld;
  int *sg, *st, *gidx;
  long long *offV, *offO;
};

dqmc_status stage_group(dqmc_handle h, const UGroup& g, const dqmc_instance* desc,
                        const double* V_pool, long long outlen, int nout, Stage& S) {
  const int nb = (int)g.idx.size();
  const long long vlen = (long long)g.M * g.N;
  auto lay = [&](Arena& ar) {
    S.V = ar.take<double>(vlen * nb);
    for (int o = 0; o < 3; ++o) S.out[o] = o < nout ? ar.take<double>(outlen * nb) : nullptr;
    S.ld = ar.take<double>(nb);
    S.sg = ar.take<int>(nb);
    S.st = ar.take<int>(nb);
    S.gidx = ar.take<int>(nb);
    S.offV = ar.take<long long>(nb);
    S.offO = ar.take<long long>(nb);
  };
  Arena m;
  lay(m);
  CKS(ensure_rws(h, m.off));
  Arena ar;
  ar.base = h->rws;
  lay(ar);
  std::vector<int> gidx(nb);
  std::vector<long long> offV(nb), offO(nb);
  for (int j = 0; j < nb; ++j) {
    gidx[j] = g.idx[j];
    offV[j] = desc[g.idx[j]].off_V;
    offO[j] = desc[g.idx[j]].off_G;
  }
  cudaStream_t st = h->stream;
  if (cudaMemcpyAsync(S.gidx, gidx.data(), nb * sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(S.offV, offV.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(S.offO, offO.data(), nb * sizeof(long long), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)   // the host tables go out of scope
    return DQMC_ERR_CUDA;
  CK(move_blocks(V_pool, S.V, S.offV, vlen, nb, 0, st));
  return DQMC_OK;
}

dqmc_status check_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                         const double* K_pool, const double* V_pool) {
  if (!h || batch < 0) return DQMC_ERR_ARG;
  if (batch == 0) return DQMC_OK;
  if (!desc || !K_pool || !V_pool) return DQMC_ERR_ARG;
  if (h->pmode == DQMC_PTR_HOST) return DQMC_ERR_UNSUPPORTED;
  return DQMC_OK;
}

}  // namespace

extern "C" {

dqmc_status dqmc_greens_tdisplaced_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                                          const double* K_pool, const double* V_pool,
                                          double* Gtt_pool, double* Gt0_pool, int* status) {
  return dqmc_greens_tdisplaced_ragged_ex(h, batch, desc, K_pool, V_pool, Gtt_pool, Gt0_pool,
                                          nullptr, status);
}

dqmc_status dqmc_greens_tdisplaced_ragged_ex(dqmc_handle h, int batch, const dqmc_instance* desc,
                                             const double* K_pool, const double* V_pool,
                                             double* Gtt_pool, double* Gt0_pool,
                                             double* G0t_pool, int* status) {
  CKS(check_ragged(h, batch, desc, K_pool, V_pool));
  if (batch == 0) return DQMC_OK;
  std::vector<UGroup> groups;
  CKS(group_uniform(batch, desc, groups));
  long long launches = 0;
  for (const UGroup& g : groups) {
    const int nb = (int)g.idx.size();
    const long long outlen = (long long)(n_chunks(g.M, g.k) + 1) * g.N * g.N;
    Stage S;
    CKS(stage_group(h, g, desc, V_pool, outlen, G0t_pool ? 3 : 2, S));
    CKS(tdisplaced_impl(h, nb, g.N, g.M, K_pool + g.offK, g.dtau, S.V, g.k,
                        Gtt_pool ? S.out[0] : nullptr, Gt0_pool ? S.out[1] : nullptr,
                        G0t_pool ? S.out[2] : nullptr, S.st));
    launches += h->launches;
    cudaStream_t st = h->stream;
    if (Gtt_pool) CK(move_blocks(S.out[0], Gtt_pool, S.offO, outlen, nb, 1, st));
    if (Gt0_pool) CK(move_blocks(S.out[1], Gt0_pool, S.offO, outlen, nb, 1, st));
    if (G0t_pool) CK(move_blocks(S.out[2], G0t_pool, S.offO, outlen, nb, 1, st));
    if (status) CK(scatter_scalars(S.gidx, nb, nullptr, nullptr, S.st, nullptr, nullptr, status, st));
  }
  h->launches = launches;
  return DQMC_OK;
}

dqmc_status dqmc_logdet_grad_ragged(dqmc_handle h, int batch, const dqmc_instance* desc,
                                    const double* K_pool, const double* V_pool, double* logdet,
                                    int* sign, double* dV_pool, int* status) {
  CKS(check_ragged(h, batch, desc, K_pool, V_pool));
  if (batch == 0) return DQMC_OK;
  if (!dV_pool) return DQMC_ERR_ARG;
  std::vector<UGroup> groups;
  CKS(group_uniform(batch, desc, groups));
  long long launches = 0;
  for (const UGroup& g : groups) {
    const int nb = (int)g.idx.size();
    const long long outlen = (long long)g.M * g.N;
    Stage S;
    CKS(stage_group(h, g, desc, V_pool, outlen, 1, S));
    CKS(grad_impl(h, nb, g.N, g.M, K_pool + g.offK, g.dtau, S.V, g.k, S.ld, S.sg, S.out[0], S.st));
    launches += h->launches;
    cudaStream_t st = h->stream;
    CK(move_blocks(S.out[0], dV_pool, S.offO, outlen, nb, 1, st));
    CK(scatter_scalars(S.gidx, nb, S.ld, S.sg, S.st, logdet, sign, status, st));
  }
  h->launches = launches;
  return DQMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Read-out of the debug build's device-side checks
// ---------------------------------------------------------------------------
namespace {
// n threads write x[i] = i + 1 behind a check of i < n_checked; with
// n_checked = n - 1 the last thread's check fails, so it records its index
// and skips its write, which would have stayed inside x (n elements) anyway.
__global__ void check_selftest_kernel(double* x, int n, int n_checked) {
  const int i = threadIdx.x;
  if (i < n && DQMC_CHECK(i < n_checked, i)) x[i] = i + 1;
}
}  // namespace

extern "C" {

int dqmc_is_debug_build(void) {
#ifdef DQMC_DEBUG
  return 1;
#else
  return 0;
#endif
}

dqmc_status dqmc_debug_read(int clear, const char** file, int* line, int* value) {
  if (!file || !line || !value) return DQMC_ERR_ARG;
  *file = nullptr;
  *line = 0;
  *value = 0;
#ifdef DQMC_DEBUG
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_CUDA;
  }
  for (const CheckUnit& u : kCheckUnits) {
    const unsigned long long w = u.read(clear != 0);
    if (w == ~0ull) return DQMC_ERR_CUDA;
    if (w && !*file) {
      *file = u.file;
      *line = (int)((w >> 32) & 0x7fffffff);
      *value = (int)(unsigned int)(w & 0xffffffffull);
    }
  }
  return DQMC_OK;
#else
  (void)clear;
  return DQMC_ERR_UNSUPPORTED;
#endif
}

dqmc_status dqmc_selftest_check(void* stream, int* fired, int* value) {
  if (!fired || !value) return DQMC_ERR_ARG;
  *fired = 0;
  *value = -1;
#ifdef DQMC_DEBUG
  cudaStream_t st = (cudaStream_t)stream;
  constexpr int n = 64;
  double* x = nullptr;
  if (cudaMalloc(&x, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_NOMEM;
  }
  dqmc_status rc = DQMC_OK;
  double hx[n];
  unsigned long long w = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) rc = DQMC_ERR_CUDA;
  if (rc == DQMC_OK && dqmc::check_word_api(true) == ~0ull) rc = DQMC_ERR_CUDA;
  if (rc == DQMC_OK && cudaMemsetAsync(x, 0, n * sizeof(double), st) != cudaSuccess) rc = DQMC_ERR_CUDA;
  if (rc == DQMC_OK) {
    check_selftest_kernel<<<1, n, 0, st>>>(x, n, n - 1);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hx, x, sizeof hx, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = DQMC_ERR_CUDA;
  }
  if (rc == DQMC_OK && (w = dqmc::check_word_api(true)) == ~0ull) rc = DQMC_ERR_CUDA;
  if (rc == DQMC_OK) {
    bool writes_ok = hx[n - 1] == 0.0;
    for (int i = 0; i < n - 1; ++i) writes_ok = writes_ok && hx[i] == i + 1;
    *fired = (w >> 63) && writes_ok ? 1 : 0;
    *value = (int)(unsigned int)(w & 0xffffffffull);
  }
  cudaFree(x);
  cudaGetLastError();
  return rc;
#else
  (void)stream;
  return DQMC_ERR_UNSUPPORTED;
#endif
}

}  // extern "C"

DQMC_CHECK_UNIT(api)
