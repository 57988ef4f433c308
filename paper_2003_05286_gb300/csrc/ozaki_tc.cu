// Mixed-precision slice products on the tcgen05 tensor cores.
//
// The k-slice chain products (Sec. 2, Eq. (Ztr); a naive chunk between two
// re-factorisations, Sec. 4.1) may run in reduced precision; the pivoted QR,
// the D splits and the inversions stay FP64.  Here a product C = E * B' (E =
// exp(-dtau K), B' = diag(exp V_l) A) is evaluated from BF16 operands by the
// error-free splitting of Ozaki et al. (Numer. Algorithms 59, 2012):
//
//   * every row i of E is scaled by 2^{-eA_i} and every column j of B' by
//     2^{-eB_j} so that all entries lie in (-1/2, 1/2); each scaled entry is
//     written in s balanced base-128 digits (x = sum_p a_p 2^{-7p} + r,
//     |r| <= 2^{-7s-1}, a_p integer in [-64, 64], each digit rounded to
//     nearest and its remainder carried to the next) -- integers of at most 7
//     significant bits, exact in BF16;
//   * a digit product a_p . b_q is a sum of K <= 256 integers of magnitude
//     <= 2^12, so it is an integer below 2^20 and the FP32 accumulation of the
//     tensor core is exact; products with the same weight 2^{-7(p+q)} share
//     one TMEM accumulator (up to 16 of them, sum < 2^24);
//   * only p + q <= s + 1 is formed (the rest is below the truncation error);
//   * the epilogue adds the accumulators exactly in a 128-bit integer with
//     their relative shifts and builds the correctly rounded FP64 value with
//     integer operations, so the FP64 pipe is not used.
// The product is accurate to about N 2^{-7s-1} of (row max x column max):
// normwise, not elementwise -- entries much smaller than their column's
// largest keep correspondingly fewer digits.
//
// Digit planes are stored as contiguous tiles (128 x 32 BF16 for the A
// operand, 64 x 32 for B), each already in the 64-byte-swizzled byte order the
// tensor core reads from shared memory, so that one plain bulk copy
// (cp.async.bulk) moves a tile and no tensor map is needed.
//
// Per CTA: one 128 x 64 output tile of one instance; 8 warps; warp 0 issues the
// bulk copies of the s A-slice tiles and s B-slice tiles of a K-block into one
// of two shared-memory stages, one thread of warp 1 issues the tcgen05.mma (M=128, N=64, K=16,
// kind::f16 with BF16 inputs, FP32 accumulators in TMEM), and all eight warps
// read the accumulators back (tcgen05.ld 32x32b) for the epilogue, which
// stages the FP64 tile in the idle stage buffers and stores whole rows.  Every
// mbarrier wait is bounded (~2 s by the global timer); a CTA that gives up
// records DQMC_STATUS_TIMEOUT in its instance's status word, waits (bounded)
// for its own copies, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "common.cuh"

namespace dqmc {

namespace {

constexpr int OZ_BM = 128;       // output rows per CTA (TMEM lanes)
constexpr int OZ_BN = 64;        // output columns per CTA (TMEM columns per accumulator)
constexpr int OZ_BK = 32;        // K per stage: 32 BF16 = 64 bytes per row (64-byte swizzle)
constexpr int OZ_STAGES = 2;
constexpr int OZ_THREADS = 256;   // 8 warps: two per TMEM lane quarter in the epilogue
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;   // 8 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;   // 4 KB
// B tile slots of a stage: OZ_BZERO zero tiles, then the digit tiles 0 .. s-1,
// then zero tiles up to slot OZ_BSLOTS - 1 (see the MMA issuer)
constexpr int OZ_BZERO = 3;
constexpr int OZ_BSLOTS = OZ_BZERO + 8;
// FP64 result tile staged in shared memory for coalesced row stores (padded rows)
constexpr int OZ_C_LD = OZ_BN + 1;
constexpr int OZ_C_TILE = OZ_BM * OZ_C_LD * 8;   // 66.5 KB
constexpr unsigned long long OZ_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on a phase of an mbarrier; false after OZ_WAIT_NS.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer() - t0 > OZ_WAIT_NS) return false;
  }
}

// One contiguous global -> shared copy, completion counted in bytes on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 64-byte swizzle:
// rows of 64 bytes, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused when swizzled)
  d |= (uint64_t)(512 >> 4) << 32;                 // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)4 << 61;                          // swizzle mode: 64-byte
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 64, M = 128.
// kind::f16 instruction descriptor: BF16 A and B, FP32 accumulator, K-major
// operands, M = OZ_BM, N = n columns (a multiple of 16, at most 256)
__host__ __device__ constexpr uint32_t oz_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                     uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// S * 2^e for a signed 128-bit S, rounded to nearest even, by integer
// operations only (leading-zero count, shift, exponent assembly); results
// outside the normal range take the library conversion.
// (T 2^32 + r) 2^e correctly rounded to FP64, for |T| < 2^45 and 0 <= r < 2^32
// (the exact sum of the weight groups), with 64-bit integer operations only:
// the magnitude is split into (Ta, ra) the same way, the 53-bit mantissa taken
// from Ta and the top bits of ra, and the discarded bits of ra decide the
// round-to-nearest-even step.
__device__ __forceinline__ double split_times_pow2(long long T, unsigned int r, int e) {
  if (T == 0 && r == 0) return 0.0;
  const bool neg = T < 0;
  unsigned long long Ta;
  unsigned int ra;
  if (!neg) { Ta = (unsigned long long)T; ra = r; }
  else if (r) { Ta = (unsigned long long)(-(T + 1)); ra = (unsigned int)(0x100000000ull - r); }
  else { Ta = (unsigned long long)(-T); ra = 0u; }
  unsigned long long mant;
  int ex;
  if (Ta < (1ull << 21)) {   // below 2^53: exact
    const unsigned long long A = (Ta << 32) | ra;
    const int nb = 64 - __clzll((long long)A);
    mant = A << (53 - nb);
    ex = nb - 1 + e;
  } else {                   // 54..77 bits: drop sh = 1..24 bits of ra
    const int nb = 96 - __clzll((long long)Ta);
    const int sh = nb - 53;
    mant = (Ta << (32 - sh)) | (ra >> sh);
    const unsigned int rem = ra & ((1u << sh) - 1u), half = 1u << (sh - 1);
    ex = nb - 1 + e;
    if (rem > half || (rem == half && (mant & 1ull))) {
      if (++mant == (1ull << 53)) { mant >>= 1; ++ex; }
    }
  }
  const int be = ex + 1023;
  if (be <= 0 || be >= 2047)   // result outside the normal range: scale in FP64
    return ldexp((double)Ta * 4294967296.0 + (double)ra, e) * (neg ? -1.0 : 1.0);
  return __longlong_as_double((long long)((neg ? (1ull << 63) : 0ull) |
                                          ((unsigned long long)be << 52) |
                                          (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace

// Pair table: up to 36 (p, q) digit pairs (s <= 8) with their accumulator group.
struct OzPairs {
  int n;                 // number of pairs
  int ngroups;           // accumulators (<= 8)
  int s;                 // slices per operand
  int shift[8];          // weight 2^{shift} of group g relative to the lowest kept weight
  unsigned char p[40], q[40], g[40], first[40];
  int stall;             // self-test only: the producer issues no loads
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
ozaki_gemm_kernel(const __nv_bfloat16* __restrict__ As, long long sA, int P128,
                  const __nv_bfloat16* __restrict__ Bs, int PN, const OzPairs pr, int N, int nkb,
                  const int* __restrict__ eA, long long seA, int a_batched,
                  const int* __restrict__ eB, long long seB, double* __restrict__ C,
                  long long sC, int* status, const int* __restrict__ lim, int lim_at,
                  const double* __restrict__ csrc, long long scsrc) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage buffers
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int s = pr.s;
  const int a_bytes = s * OZ_A_TILE;
  const int stage_bytes = a_bytes + OZ_BSLOTS * OZ_B_TILE;   // shared memory per stage
  const int copy_bytes = s * (OZ_A_TILE + OZ_B_TILE);        // bytes copied into a stage
  const int data_bytes = OZ_STAGES * stage_bytes > OZ_C_TILE ? OZ_STAGES * stage_bytes : OZ_C_TILE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + data_bytes);
  uint64_t* full = bars;                    // [OZ_STAGES]
  uint64_t* empty = bars + OZ_STAGES;       // [OZ_STAGES]
  uint64_t* done = bars + 2 * OZ_STAGES;    // [1]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * OZ_STAGES + 1);
  int* s_fail = reinterpret_cast<int*>(tmem_holder + 1);
  int* s_used = s_fail + 1;   // K-blocks whose operands the MMA issuer has waited for

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n0 = blockIdx.x * OZ_BN, m0 = blockIdx.y * OZ_BM, b = blockIdx.z;
  // launch contract (debug build), before any barrier or TMEM allocation:
  // OZ_THREADS threads, 1..8 digits with their weight groups inside the
  // allocated TMEM columns, shared memory up to the last flag word, and every
  // bulk copy's source on a 16-byte boundary (tile bases, digit planes,
  // instances)
  if (!DQMC_CHECK(blockDim.x == OZ_THREADS && s >= 1 && s <= 8 &&
                      pr.ngroups * OZ_BN <= (s > 4 ? 512 : 256),
                  s) ||
      !DQMC_CHECK(dyn_smem_bytes() >= (unsigned)((base - smem_raw) + data_bytes +
                                                 (2 * OZ_STAGES + 1) * 8 + 12),
                  dyn_smem_bytes()) ||
      !DQMC_CHECK((reinterpret_cast<uintptr_t>(As) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(Bs) & 15) == 0 && (sA * 2) % 16 == 0 &&
                      ((long long)P128 * nkb * OZ_BK * 2) % 16 == 0 &&
                      ((long long)PN * nkb * OZ_BK * 2) % 16 == 0,
                  sA))
    return;
  // an instance whose (shorter) chain has already ended: copy its FP64 source
  // tile through when one is given, else leave the output alone.  The test
  // is uniform over the CTA and comes before any barrier or TMEM allocation.
  if (lim && lim[b] < lim_at) {
    if (csrc) {
      const double* src = csrc + (long long)b * scsrc;
      double* dst = C + (long long)b * sC;
      for (int e = tid; e < OZ_BM * OZ_BN; e += OZ_THREADS) {
        const int r = m0 + e / OZ_BN, c = n0 + e % OZ_BN;
        if (r < N && c < N) dst[(long long)r * N + c] = src[(long long)r * N + c];
      }
    }
    return;
  }
  const int bA = a_batched ? b : 0;   // instance of the A operand (shared when not batched)
  // accumulators: weight group g in columns [g OZ_BN, (g + 1) OZ_BN); the MMAs
  // write groups in aligned blocks of four, so more than four groups take all 512
  const uint32_t tmem_cols = s > 4 ? 512u : 256u;

  if (tid == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    *s_fail = 0;
    *s_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // zero B tile slots of both stages (never written by the copies), made
  // visible to the tensor core's (async proxy) reads
  for (int st = 0; st < OZ_STAGES; ++st) {
    uint4* zb = reinterpret_cast<uint4*>(base + st * stage_bytes + a_bytes);
    for (int i = tid; i < OZ_BSLOTS * OZ_B_TILE / 16; i += OZ_THREADS) {
      const int slot = i / (OZ_B_TILE / 16);
      if (slot < OZ_BZERO || slot >= OZ_BZERO + s) zb[i] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---- producer: bulk copies of the slice tiles of each K-block ---------
    for (int kb = 0; kb < (pr.stall ? 0 : nkb); ++kb) {
      const int st = kb % OZ_STAGES;
      if (kb >= OZ_STAGES && !mbar_wait(&empty[st], ((kb / OZ_STAGES) - 1) & 1)) {
        atomicOr(s_fail, 1);
        break;
      }
      if (*(volatile int*)s_fail) break;
      unsigned char* sb = base + st * stage_bytes;
      mbar_arrive_expect_tx(&full[st], (uint32_t)copy_bytes);
      // tile (row block, K-block kb) of every digit plane: one contiguous copy each
      const long long PK = (long long)nkb * OZ_BK;
      const __nv_bfloat16* a0 = As + (long long)bA * sA +
                                ((long long)(m0 / OZ_BM) * nkb + kb) * (OZ_BM * OZ_BK);
      const __nv_bfloat16* b0 = Bs + (long long)b * s * PN * PK +
                                ((long long)(n0 / OZ_BN) * nkb + kb) * (OZ_BN * OZ_BK);
      for (int p = 0; p < s; ++p)
        bulk_load(sb + p * OZ_A_TILE, a0 + (long long)p * P128 * PK, OZ_A_TILE, &full[st]);
      for (int q = 0; q < s; ++q)
        bulk_load(sb + a_bytes + (OZ_BZERO + q) * OZ_B_TILE, b0 + (long long)q * PN * PK,
                  OZ_B_TILE, &full[st]);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ---------------------------------------------------------
    // Every MMA has N = 4 OZ_BN and writes one aligned block of four weight
    // groups: block r (groups 4r .. 4r+3) receives, for each A digit p, one
    // MMA with the B digits q = 4r - p .. 4r - p + 3, whose products have
    // weights p + q = 4r .. 4r + 3.  Digits outside 0 .. s-1 read the zero
    // tiles around the B digits, so every kept pair (p + q <= s - 1) is formed
    // exactly once.  Consecutive MMAs then either accumulate into the same
    // block with the same shape, which the tensor core chains at full rate, or
    // write a disjoint block; MMAs into partially overlapping accumulator
    // ranges of different widths waited for one another and ran at about a
    // third of the rate.  The zero padding costs a quarter of the issued work.
    const uint32_t idesc = oz_idesc(4 * OZ_BN);
    const int nblk = s > 4 ? 2 : 1;
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % OZ_STAGES;
      if (!mbar_wait(&full[st], (kb / OZ_STAGES) & 1)) {
        atomicOr(s_fail, 1);
        break;
      }
      *(volatile int*)s_used = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // descriptors: the stage's base descriptor plus tile offsets in its
      // start-address field (address >> 4; shared addresses stay below 256 KB,
      // so the field never carries)
      const uint64_t dA = smem_desc_sw64(smem_u32(base + st * stage_bytes));
      const uint64_t dB = dA + (uint64_t)(a_bytes >> 4);
      for (int kk = 0; kk < OZ_BK / 16; ++kk) {
        const uint64_t dAk = dA + (uint64_t)(kk * 2), dBk = dB + (uint64_t)(kk * 2);
        const bool first_k = kb == 0 && kk == 0;
        for (int r = 0; r < nblk; ++r) {
          for (int pd = 0; pd < s; ++pd) {
            const int q0 = 4 * r - pd;
            if (q0 + 3 < 0 || q0 > s - 1) continue;   // no digit of this block for pd
            // p = 0 reaches every block first: it starts the accumulation
            const uint32_t acc = (first_k && pd == 0) ? 0u : 1u;
            // the four B tiles of this MMA lie inside the stage's B slots
            if (!DQMC_CHECK(OZ_BZERO + q0 >= 0 && OZ_BZERO + q0 + 4 <= OZ_BSLOTS, q0)) continue;
            umma(tmem + (uint32_t)(4 * r) * OZ_BN, dAk + (uint64_t)(pd * (OZ_A_TILE >> 4)),
                 dBk + (uint64_t)((OZ_BZERO + q0) * (OZ_B_TILE >> 4)), idesc, acc);
          }
        }
      }
      umma_commit(&empty[st]);   // frees the stage once these MMAs have read it
    }
    umma_commit(done);
  }
  __syncthreads();

  // ---- epilogue: accumulators -> int64 combination -> FP64 -----------------
  bool ok = !*(volatile int*)s_fail && mbar_wait(done, 0);
  ok = __syncthreads_and(ok) != 0;   // uniform: tcgen05.ld is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // warp w reads TMEM lanes 32 (w % 4) .. +31 (rows) and columns 32 (w / 4) .. +31
  const int row = m0 + (warp & 3) * 32 + lane;
  const int cbase = (warp >> 2) * 32;
  const int ea = row < N ? eA[(long long)bA * seA + row] : 0;
  const int* eBb = eB + (long long)b * seB;
  double* Cb = C + (long long)b * sC;
  const int shift0 = 7 * (s + 1);
  double* ctile = reinterpret_cast<double*>(base);   // OZ_BM x OZ_C_LD
  if (ok) {
    const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
    for (int c0 = cbase; c0 < cbase + 32; c0 += 8) {
      // exact sum of the groups: hi carries weights >= 2^32 (in units of 2^32)
      long long hi[8], lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) { hi[j] = 0; lo[j] = 0; }
      uint32_t r[8][8];
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (g < pr.ngroups) tmem_ld8_nowait(tmem + lane_addr + g * OZ_BN + c0, r[g]);
      tmem_wait_ld();
#pragma unroll
      for (int g = 0; g < 8; ++g) {
        if (g >= pr.ngroups) break;
        const int sh = pr.shift[g];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          // |acc| < 2^24: the 32-bit conversion is exact and stays off the FP64 pipe
          const long long v = (long long)__float2int_rn(__uint_as_float(r[g][j]));
          if (sh >= 32) hi[j] += v << (sh - 32); else lo[j] += v << sh;
        }
      }
      // S = hi 2^32 + lo = T 2^32 + r with 0 <= r < 2^32; results go to the
      // padded tile in the (now idle) stage buffers
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + c0 + j;
        double v = 0.0;
        if (row < N && col < N)
          v = split_times_pow2(hi[j] + (lo[j] >> 32), (unsigned int)(lo[j] & 0xFFFFFFFFll),
                               ea + eBb[col] - shift0);
        ctile[((warp & 3) * 32 + lane) * OZ_C_LD + c0 + j] = v;
      }
    }
  }
  if (ok) {
    __syncthreads();
    for (int e = tid; e < OZ_BM * OZ_BN; e += OZ_THREADS) {   // rows of 64 doubles
      const int r = e / OZ_BN, c = e % OZ_BN;
      if (m0 + r < N && n0 + c < N) Cb[(long long)(m0 + r) * N + n0 + c] = ctile[r * OZ_C_LD + c];
    }
  } else if (tid == 0 && status) {
    atomicOr(&status[b], DQMC_STATUS_TIMEOUT);
  }
  // on failure, let copies in flight land before the CTA exits (bounded).  A
  // stage is refilled only after the MMAs consumed its previous contents, so
  // only the K-blocks s_used and s_used + 1 can still have copies on the way.
  if (!ok && warp == 0 && lane == 0) {
    const int used = *(volatile int*)s_used;
    for (int kb = used; kb < used + OZ_STAGES && kb < nkb; ++kb)
      mbar_wait(&full[kb % OZ_STAGES], (kb / OZ_STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Splitting kernel: X (FP64, element (m, j) at X[g(m)*ldm + j*ldj], g the
// optional row gather gm, identity if null) times an optional scale sc[m]
// -> S BF16 slice planes of PJ x PM (zero padded), each stored as tiles of R
// rows j by 32 consecutive m (tile (j / R, m / 32) at ((j / R)(PM / 32) +
// m / 32) R 32 elements; inside, row r's 16-byte chunk c at chunk c ^ ((r >> 1)
// & 3): the 64-byte swizzle), and column exponents e[j] with
// max_m |x_mj| < 2^{e_j}.
// One CTA per 32 columns j of one instance; 256 threads.  Phase 1 stages the
// 32 columns in shared memory (coalesced rows) and finds each column's
// exponent; phase 2 gives every thread whole 16-byte chunks (8 consecutive m
// of one column j), so each digit plane gets one 16-byte store per chunk and
// the four lanes of a column cover one 64-byte tile row (a warp writes 512
// contiguous bytes per plane).  Digits and their BF16 encodings are built with
// integer operations only.
// ---------------------------------------------------------------------------
namespace {
// BF16 bits of an integer d with |d| <= 128.  The FP32 value with bits
// 0x4B400000 + d is 1.5 * 2^23 + d exactly (|d| < 2^22), so subtracting
// 1.5 * 2^23 leaves d as an exact FP32 number; with at most 8 significant
// bits its low 16 mantissa bits are zero and the upper half is the BF16
// encoding (0 for d = 0).  One integer add, one FP32 subtract, one shift.
__device__ __forceinline__ uint32_t small_int_bf16(int d) {
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return __float_as_uint(f) >> 16;
}
}  // namespace

template <int SL>
__global__ void __launch_bounds__(256)
ozaki_split_kernel(const double* __restrict__ X, long long ldm, long long ldj, long long sX,
                   const double* __restrict__ sc, long long ssc, int N, int PJ, int PM, int R,
                   __nv_bfloat16* __restrict__ S, long long sS, int* __restrict__ e,
                   long long se, const int* __restrict__ gm, long long sgm) {
  extern __shared__ double tile[];   // [PM][33]
  __shared__ int emax[8][32];
  const int b = blockIdx.y;
  const int j0 = blockIdx.x * 32;
  const int tid = threadIdx.x;
  // launch contract (debug build): 256 threads, whole tiles, shared memory
  // for the staged PM x 33 block
  if (!DQMC_CHECK(blockDim.x == 256 && PM % 32 == 0 && R > 0 && PJ % R == 0, PM) ||
      !DQMC_CHECK(dyn_smem_bytes() >= (unsigned)PM * 33u * 8u, dyn_smem_bytes()))
    return;
  const double* Xb = X + (long long)b * sX;
  const double* scb = sc ? sc + (long long)b * ssc : nullptr;
  const int* gmb = gm ? gm + (long long)b * sgm : nullptr;
  {
    // rows rg, rg + 8, ...: eight loads (and their gather indices) in flight
    // per thread before any is used, so a thread waits for one memory round
    // trip per eight rows instead of one per row
    const int jj = tid & 31, rg = tid >> 5;
    const int j = j0 + jj;
    int mx = 0;
    for (int mb = rg; mb < PM; mb += 64) {
      int mr[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int m = mb + 8 * u;
        mr[u] = (m < N && j < N) ? (gmb ? gmb[m] : m) : -1;
        // a gathered row must be a row of X (the pivot order of a QR)
        if (gmb && m < N && j < N && !DQMC_CHECK(mr[u] >= 0 && mr[u] < N, mr[u])) mr[u] = -1;
      }
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (mr[u] >= 0 && mr[u] < N) ? Xb[(long long)mr[u] * ldm + (long long)j * ldj] : 0.0;
      if (scb) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int m = mb + 8 * u;
          if (m < N) v[u] *= scb[m];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int m = mb + 8 * u;
        if (m < PM) tile[m * 33 + jj] = v[u];
        // biased exponent from the bits (0 for zeros): no FP64 compare
        const int ex = (int)((__double_as_longlong(v[u]) >> 52) & 0x7ff);
        mx = ex > mx ? ex : mx;
      }
    }
    emax[rg][jj] = mx;
  }
  __syncthreads();
  if (tid < 32) {
    int m2 = emax[0][tid];
    for (int r = 1; r < 8; ++r) m2 = max(m2, emax[r][tid]);
    // biased exponent E of the largest entry: max < 2^{E-1022}, so the scaled
    // entries x 2^{-(E-1021)} lie in (-1/2, 1/2); an all-zero (or denormal)
    // column keeps exponent 0
    const int ecol = m2 == 0 ? 0 : m2 - 1021;
    emax[0][tid] = ecol;
    if (j0 + tid < PJ) e[(long long)b * se + j0 + tid] = ecol;
  }
  __syncthreads();
  __nv_bfloat16* Sb = S + (long long)b * sS;
  const long long plane = (long long)PJ * PM;
  // work items: (column jj, K-block kb) pairs; 4 lanes per item, lane ch = chunk
  const int ch = tid & 3;
  const int nkb = PM / 32;
  for (int it = tid >> 2; it < 32 * nkb; it += 64) {
    const int jj = it & 31, kb = it >> 5;
    const int jc = j0 + jj;
    if (jc >= PJ) continue;
    const int ecol = emax[0][jj];
    const int m0 = kb * 32 + ch * 8;
    long long Sv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double v = tile[(m0 + k) * 33 + jj];
      unsigned long long F = 0;   // |v| 2^{-ecol} * 2^63, below 2^62
      const long long bits = __double_as_longlong(v);
      const int E = (int)((bits >> 52) & 0x7ff);
      if (E != 0) {
        const unsigned long long m53 = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = E - 1012 - ecol;   // F = m53 * 2^sh, sh <= 9
        F = sh >= 0 ? (m53 << sh) : (sh > -64 ? (m53 >> (-sh)) : 0ull);
      }
      Sv[k] = bits < 0 ? -(long long)F : (long long)F;
    }
    // element (row jc, k = m) of the R x 32 tile (row block jc / R, K-block kb):
    // this thread's 8 values form 16-byte chunk ch of tile row jr, stored at
    // chunk ch ^ ((jr >> 1) & 3) (the 64-byte swizzle)
    const int jr = jc % R;
    const long long tile_off = ((long long)(jc / R) * nkb + kb) * (R * 32) + jr * 32 +
                               ((ch ^ ((jr >> 1) & 3)) << 3);
    // digits 0..4 on the 64-bit value; after digit 4 (weight 2^{-35}) the
    // remainder is below 2^27 in magnitude, so the rest runs in 32 bits
    int Sr[8];
#pragma unroll
    for (int q = 0; q < SL; ++q) {
      const int sh = 56 - 7 * q;                        // digit weight 2^{-7(q+1)}
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        int d0, d1;
        if (q <= 4) {
          const long long e0 = (Sv[k] + (1ll << (sh - 1))) >> sh;     // nearest, in [-64, 64]
          const long long e1 = (Sv[k + 1] + (1ll << (sh - 1))) >> sh;
          Sv[k] -= e0 << sh;
          Sv[k + 1] -= e1 << sh;
          d0 = (int)e0;
          d1 = (int)e1;
          if (q == 4) {
            Sr[k] = (int)Sv[k];
            Sr[k + 1] = (int)Sv[k + 1];
          }
        } else {
          d0 = (Sr[k] + (1 << (sh - 1))) >> sh;
          d1 = (Sr[k + 1] + (1 << (sh - 1))) >> sh;
          Sr[k] -= d0 << sh;
          Sr[k + 1] -= d1 << sh;
        }
        w[k >> 1] = small_int_bf16(d0) | (small_int_bf16(d1) << 16);
      }
      if (DQMC_CHECK(tile_off + 8 <= plane &&
                         (reinterpret_cast<uintptr_t>(Sb + q * plane + tile_off) & 15) == 0,
                     tile_off))
        *reinterpret_cast<uint4*>(Sb + q * plane + tile_off) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

OzPairs oz_pairs(int s, int N) {
  OzPairs pr{};
  pr.s = s;
  // digit products are below N 2^12; 2^24 / (N 2^12) of them fit one FP32 accumulator exactly
  const int per_group = N <= 256 ? 16 : (N <= 512 ? 8 : 4);
  const int tmax = s + 1;
  int n = 0, g = 0;
  for (int t = 2; t <= tmax; ++t) {
    int in_group = per_group;   // forces a new group at each t
    for (int p = 1; p <= s; ++p) {
      const int q = t - p;
      if (q < 1 || q > s) continue;
      if (in_group == per_group) {
        pr.shift[g] = 7 * (tmax - t);
        ++g;
        in_group = 0;
      }
      pr.p[n] = (unsigned char)(p - 1);
      pr.q[n] = (unsigned char)(q - 1);
      pr.g[n] = (unsigned char)(g - 1);
      pr.first[n] = in_group == 0;
      ++in_group;
      ++n;
    }
  }
  pr.n = n;
  pr.ngroups = g;
  return pr;
}

int oz_groups(int s, int N) { return oz_pairs(s, N).ngroups; }

size_t oz_gemm_smem(int s) {
  const size_t stages = (size_t)OZ_STAGES * (s * OZ_A_TILE + OZ_BSLOTS * OZ_B_TILE);
  return (stages > (size_t)OZ_C_TILE ? stages : (size_t)OZ_C_TILE) + 1024 + 256;
}

cudaError_t ozaki_split(const double* X, long long ldm, long long ldj, long long sX,
                        const double* sc, long long ssc, int N, int PJ, int PM, int R, int s,
                        __nv_bfloat16* S, long long sS, int* e, long long se, int batch,
                        cudaStream_t st, const int* gm, long long sgm) {
  if (R < 8 || PJ % R || PM % 32) return cudaErrorInvalidValue;
  if (s < 1 || s > 8) return cudaErrorInvalidValue;
  // 16-byte chunk stores: plane and instance strides must keep 16-byte alignment
  if (((long long)PJ * PM) % 8 || sS % 8 || (reinterpret_cast<uintptr_t>(S) & 15))
    return cudaErrorInvalidValue;
  const size_t sm = (size_t)PM * 33 * sizeof(double);
  const dim3 grid((PJ + 31) / 32, batch);
  auto go = [&](auto kern) {
    allow_dyn_smem(kern);
    kern<<<grid, 256, sm, st>>>(X, ldm, ldj, sX, sc, ssc, N, PJ, PM, R, S, sS, e, se, gm, sgm);
    return cudaGetLastError();
  };
  switch (s) {
    case 1: return go(ozaki_split_kernel<1>);
    case 2: return go(ozaki_split_kernel<2>);
    case 3: return go(ozaki_split_kernel<3>);
    case 4: return go(ozaki_split_kernel<4>);
    case 5: return go(ozaki_split_kernel<5>);
    case 6: return go(ozaki_split_kernel<6>);
    case 7: return go(ozaki_split_kernel<7>);
    default: return go(ozaki_split_kernel<8>);
  }
}

// C_b = 2^{eA_b} As_b * (2^{eB_b} Bs_b)  for b < batch.  As: s planes of
// P128 x PK (rows i) in 128-row tiles (ozaki_split with R = 128) per instance
// (sA elements apart, eA_b = eA + b seA) or shared by all instances (sA = 0);
// Bs: per instance s planes of PN x PK (columns j) in 64-row tiles (R = 64);
// PK, PN multiples of 64, P128 a multiple of 128.
static cudaError_t ozaki_gemm_impl(const __nv_bfloat16* As, const int* eA, long long sA,
                                   long long seA, int P128, const __nv_bfloat16* Bs, const int* eB,
                                   long long seB, int PN, int PK, int s, int N, int batch,
                                   double* C, long long sC, int* status, cudaStream_t st,
                                   int stall, const int* lim = nullptr, int lim_at = 0,
                                   const double* csrc = nullptr, long long scsrc = 0) {
  if (sA != 0 && sA < (long long)s * P128 * PK) return cudaErrorInvalidValue;
  if (P128 % OZ_BM || PN % OZ_BN || PK % OZ_BK || PK < OZ_BK) return cudaErrorInvalidValue;
  if (s < 1 || s > 8) return cudaErrorInvalidValue;
  OzPairs pr = oz_pairs(s, N);
  if (pr.ngroups > 8 || pr.n > 40) return cudaErrorNotSupported;
  // the kernel issues the pairs of one A digit as one wide MMA: it needs one
  // group per weight (g = p + q), which holds for N <= 256
  if (pr.ngroups != s) return cudaErrorNotSupported;
  for (int i = 0; i < pr.n; ++i)
    if (pr.g[i] != pr.p[i] + pr.q[i]) return cudaErrorNotSupported;
  pr.stall = stall;
  size_t sm = oz_gemm_smem(s);
  allow_dyn_smem(ozaki_gemm_kernel);
  dim3 grid((N + OZ_BN - 1) / OZ_BN, (N + OZ_BM - 1) / OZ_BM, batch);
  ozaki_gemm_kernel<<<grid, OZ_THREADS, sm, st>>>(As, sA, P128, Bs, PN, pr, N, PK / OZ_BK, eA, seA,
                                                  sA != 0, eB, seB, C, sC, status, lim, lim_at,
                                                  csrc, scsrc);
  return cudaGetLastError();
}

cudaError_t ozaki_gemm(const __nv_bfloat16* As, const int* eA, long long sA, long long seA,
                       int P128, const __nv_bfloat16* Bs, const int* eB, long long seB, int PN,
                       int PK, int s, int N, int batch, double* C, long long sC, int* status,
                       cudaStream_t st, const int* lim, int lim_at, const double* csrc,
                       long long scsrc) {
  return ozaki_gemm_impl(As, eA, sA, seA, P128, Bs, eB, seB, PN, PK, s, N, batch, C, sC, status,
                         st, 0, lim, lim_at, csrc, scsrc);
}

// Operands of the bounded-wait self-test: one 128 x 64 tile, one slice.
static __device__ __align__(1024) __nv_bfloat16 g_selftest_A[128 * 64];
static __device__ __align__(1024) __nv_bfloat16 g_selftest_B[64 * 64];
static __device__ int g_selftest_e[128];
static __device__ double g_selftest_C[64 * 64];

cudaError_t ozaki_selftest_timeout(int* status, cudaStream_t st) {
  void *A = nullptr, *B = nullptr, *e = nullptr, *C = nullptr;
  cudaError_t r;
  if ((r = cudaGetSymbolAddress(&A, g_selftest_A)) != cudaSuccess) return r;
  if ((r = cudaGetSymbolAddress(&B, g_selftest_B)) != cudaSuccess) return r;
  if ((r = cudaGetSymbolAddress(&e, g_selftest_e)) != cudaSuccess) return r;
  if ((r = cudaGetSymbolAddress(&C, g_selftest_C)) != cudaSuccess) return r;
  return ozaki_gemm_impl(static_cast<const __nv_bfloat16*>(A), static_cast<const int*>(e), 0, 0,
                         128, static_cast<const __nv_bfloat16*>(B), static_cast<const int*>(e), 0,
                         64, 64, 1, 64, 1, static_cast<double*>(C), 0, status, st, 1);
}

}  // namespace dqmc

// Self-test of the bounded device-side waits (see include/dqmc.h).
extern "C" dqmc_status dqmc_selftest_wait_timeout(void* stream, int* status) {
  if (!status) return DQMC_ERR_ARG;
  return dqmc::ozaki_selftest_timeout(status, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? DQMC_OK
             : DQMC_ERR_CUDA;
}

DQMC_CHECK_UNIT(ozaki)
