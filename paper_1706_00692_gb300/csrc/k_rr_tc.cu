// Rayleigh-Ritz update on the tensor cores (Algorithm 2, step 3: X = Q X_Q,
// with step 4's A X = (A Q) X_Q and residual partials), FP64-accurate.
//
// The contraction index i is balanced first, exactly: with c_i the exponent of
// ||q_i|| (from the diagonal of B_Q = Q^T Q), Q X_Q = (Q D)(D^-1 X_Q) for
// D = diag(2^-c_i), so that a column of Q scaled far down (and the row of X_Q
// scaled up to compensate) no longer sets the digits' scale of a whole row or
// column. Each FP64 operand is then written exactly as signed 7-bit digits
// below a power of two: a row of Q D (or A Q D) with 2^e > its largest
// magnitude, or a column of D^-1 X_Q with 2^f > its largest magnitude, holds
//     x = sign(x) sum_{t=1..8} d_t 2^{e - 7t} + rho,   d_t in [0, 127],  |rho| < 2^{e-56},
// the digits being bit fields of the 56-bit fixed-point magnitude (integer
// operations only). Every digit is an integer of at most 7 bits, exactly a
// BF16 value, so the tensor cores form the digit products exactly; a product
// of two digits is below 2^14, and the K = m0 <= 80 terms of one digit pair,
// summed over the at most 8 pairs (a, b) of one level a + b, stay below 2^24:
// the FP32 accumulator of each level is an exact integer. Levels 2..9 are
// kept (pairs with a + b > 9 weigh below 2^-63 of the scales, like the 56-bit
// truncation) and combined exactly in integers,
//     (Q X_Q)[r][j] = 2^{e_r + f_j - 63} T,   T = sum_{d=2..9} acc_d 2^{7(9-d)}  (|T| < 2^75),
// then rounded once to FP64 (to nearest) by integer operations. The result
// carries the 56-bit truncation of the operands and one rounding: FP64
// accuracy, with the FP64 pipe (1/64 of the FP32 rate on this GPU) used only
// for the residual sums.
//
// Layout (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in TMEM,
// cta_group::1, M = 128 rows of the tile, K = m0 padded to a multiple of 16):
// operands in shared memory in the no-swizzle K-major layout of 8 x 16-byte
// core matrices (leading byte offset 128 B between core matrices along K,
// stride byte offset (K/8) x 128 B between groups of 8 rows). Output columns
// go in chunks of wc = 32 (the last one 16 when K is an odd multiple of 16).
// The 8 digit planes of a chunk of D^-1 X_Q are stored back to back, so the
// planes b = 1 .. 9 - a form one B operand of N = wc (9 - a) rows: one MMA per
// 16-wide K step writes every level a + b of digit a of the A operand, into
// TMEM columns that are contiguous when level d sits at (d - 2) wc. Shared
// memory holds the 8 digit planes of one 128-row tile of Q (then of A Q) and
// the 8 planes of the chunk; TMEM holds 2 outputs x 8 levels x wc columns.
// One persistent CTA of 512 threads per SM walks (column chunk, row tile)
// items. Every wait on the mbarrier is bounded: a wait that runs out sets
// status->tc_timeout, and the CTA stops issuing work, waits (bounded) for its
// own outstanding MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace ifeast {

namespace {

constexpr int kTcThreads = 512;
constexpr int kTcRows = 128;      // M: rows of one tile (TMEM lanes)
constexpr int kTcDigits = 8;      // digits per operand value (56 bits)
constexpr int kTcLevels = 8;      // levels d = 2..9
constexpr int kTcMaxK = 80;       // m0 padded, at most (digit sums stay below 2^24)
constexpr int kTcChunk = 32;      // output columns per item (N of one level)
constexpr long kTcSpin = 1L << 26;  // try_wait polls before a wait gives up
constexpr int kNoExp = -(1 << 20);  // exponent of 0 (and of denormals)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// element offset of (row, k) in a no-swizzle K-major tile with kp columns
__device__ __forceinline__ int core_off(int row, int k, int kp) {
  return ((row >> 3) * (kp >> 3) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);       // start address
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;    // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                        // descriptor version (tcgen05)
  return d;                                      // base offset 0, no swizzle
}

// instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTcRows >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

// bounded wait for the completion of phase `parity`; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
  for (long it = 0; it < kTcSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

// exponent e with 2^(e-1) <= |x| < 2^e for normal x; kNoExp for 0 and denormals
__device__ __forceinline__ int scale_exp(double x) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  return E == 0 ? kNoExp : E - 1022;
}

// balancing exponent c_i of column i of Q: the exponent of sqrt(B_Q[i][i])
// (0 for a zero column)
__device__ __forceinline__ int balance_exp(const double *__restrict__ Bq, int m, int i) {
  const int c = scale_exp(sqrt(Bq[(size_t)i * m + i]));
  return c == kNoExp ? 0 : c;
}

// 56-bit fixed-point magnitude of x below 2^e (|x| < 2^e), truncated;
// denormals count as 0 (far below every scale used here)
__device__ __forceinline__ unsigned long long fixed56(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0ull;
  const unsigned long long m = ((unsigned long long)b & ((1ull << 52) - 1)) | (1ull << 52);
  // |x| = m 2^(E - 1075); fixed = |x| 2^(56 - e) = m 2^(E - 1075 + 56 - e)
  const int sh = E - 1075 + 56 - e;
  if (sh >= 0) return m << sh;  // sh <= 3 since |x| < 2^e
  if (sh <= -64) return 0ull;
  return m >> (-sh);
}

__device__ __forceinline__ bool sign_bit(double x) { return __double_as_longlong(x) < 0; }

// BF16 bits of the integer d in [0, 127]: 2^23 + d is exact in FP32 and
// (2^23 + d) - 2^23 = d exactly; its low 16 bits are zero, so the upper half
// is the BF16 value
__device__ __forceinline__ uint32_t digit_bits(uint32_t d) {
  const float f = __int_as_float((int)(0x4B000000u | d)) - 8388608.0f;
  return (uint32_t)__float_as_int(f) >> 16;
}

// signed digit t (1..8) of a fixed-point magnitude, as BF16 (|d| <= 127: exact)
__device__ __forceinline__ __nv_bfloat16 digit_bf16(unsigned long long f, int t, bool neg) {
  const uint32_t d = (uint32_t)((f >> (56 - 7 * t)) & 0x7F);
  return __ushort_as_bfloat16((unsigned short)(digit_bits(d) | (neg && d ? 0x8000u : 0u)));
}

// (-1)^neg |T| 2^e2 rounded to the nearest FP64 (ties to even), T given as the
// 128-bit magnitude hi 2^64 + lo; integer operations only while the result is
// a normal number (ldexp of the rounded significand otherwise)
__device__ __forceinline__ double int128_to_double(unsigned long long hi, unsigned long long lo,
                                                   bool neg, int e2) {
  if (hi == 0 && lo == 0) return 0.0;
  const int lz = hi ? __clzll(hi) : 64 + __clzll(lo);
  unsigned long long top, rest;  // the magnitude shifted left by lz: top = bits 127..64
  if (lz == 0) {
    top = hi;
    rest = lo;
  } else if (lz < 64) {
    top = (hi << lz) | (lo >> (64 - lz));
    rest = lo << lz;
  } else {
    top = lo << (lz - 64);
    rest = 0;
  }
  unsigned long long mant = top >> 11;  // 53 bits, leading bit set
  const bool rbit = (top >> 10) & 1ull;
  const bool sticky = (top & 0x3FFull) != 0 || rest != 0;
  int p = 127 - lz;  // position of the leading bit of T
  if (rbit && (sticky || (mant & 1ull))) {
    ++mant;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      ++p;
    }
  }
  const int be = p + e2 + 1023;  // biased exponent of the result
  if (be > 0 && be < 2047) {
    const unsigned long long bits = ((unsigned long long)neg << 63) |
                                    ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
  }
  const double v = ldexp((double)mant, p - 52 + e2);
  return neg ? -v : v;
}

constexpr int kTcPrepRows = 32;  // rows per row-exponent block of k_tc_prep

// Operand preparation, one launch with two kinds of blocks (blockDim =
// 32 * kp / 8 threads; every block first forms the balancing exponents c_i):
//  * blocks 0 .. kp - 1, one per output column j (padding included): the digits
//    of D^-1 X_Q for the B operand. Column j has the scale f_j (2^f_j >
//    max_i |X_Q[i][j]| 2^c_i). Chunk c holds columns 32 c .. 32 c + wc - 1
//    (wc = min(32, kp - 32 c)); its planes t = 1..8 follow each other:
//    Bd[32 c * 8 * kp + (t - 1) * wc * kp + core_off(j - 32 c, i, kp)] = digit t
//    of X_Q[i][j] 2^c_i (signed), 0 in the padding. Block 0 also writes
//    cexp[i] = c_i.
//  * the following blocks, 32 rows each: the row exponents of Q D and A Q D,
//    rexp[o * n + r] = the e with 2^e > max_k |M[r][k]| 2^-c_k (0 for a zero
//    row), one thread per 8 consecutive columns of a row, all 8 loads in
//    flight.
__global__ void k_tc_prep(int n, int m, int kp, const double *__restrict__ XQ,
                          const double *__restrict__ Bq, const double *__restrict__ Q,
                          const double *__restrict__ AQ, __nv_bfloat16 *__restrict__ Bd,
                          int *__restrict__ fexp, int *__restrict__ cexp,
                          int *__restrict__ rexp) {
  __shared__ int se;
  __shared__ int sc[kTcMaxK];
  __shared__ int srow[2][kTcPrepRows];
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    sc[i] = i < m ? balance_exp(Bq, m, i) : 0;
    if (blockIdx.x == 0 && i < m) cexp[i] = sc[i];
  }
  if (threadIdx.x < 2 * kTcPrepRows) srow[threadIdx.x / kTcPrepRows][threadIdx.x % kTcPrepRows] = kNoExp;
  __syncthreads();
  if ((int)blockIdx.x >= kp) {  // row exponents
    const int groups = kp >> 3;
    const int lr = threadIdx.x / groups, g = threadIdx.x % groups;
    const int r = (blockIdx.x - kp) * kTcPrepRows + lr;
    if (r < n) {
      for (int o = 0; o < 2; ++o) {
        const double *M = o == 0 ? Q : AQ;
        double x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = 8 * g + e;
          x[e] = k < m ? M[(size_t)r * m + k] : 0.0;
        }
        int ex = kNoExp;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int ek = scale_exp(x[e]);
          if (ek != kNoExp) ex = max(ex, ek - sc[8 * g + e]);
        }
        atomicMax(&srow[o][lr], ex);
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kTcPrepRows) {
      const int o = threadIdx.x / kTcPrepRows, l = threadIdx.x % kTcPrepRows;
      const int rr = (blockIdx.x - kp) * kTcPrepRows + l;
      if (rr < n) rexp[(size_t)o * n + rr] = srow[o][l] == kNoExp ? 0 : srow[o][l];
    }
    return;
  }
  const int j = blockIdx.x;  // B digits of output column j
  if (threadIdx.x == 0) {
    int e = kNoExp;  // max_i of the exponent of X_Q[i][j] 2^c_i
    if (j < m)
      for (int i = 0; i < m; ++i) {
        const int ei = scale_exp(XQ[(size_t)i * m + j]);
        if (ei != kNoExp) e = max(e, ei + sc[i]);
      }
    se = e == kNoExp ? 0 : e;
    if (j < m) fexp[j] = se;
  }
  __syncthreads();
  const int c = j / kTcChunk, jj = j % kTcChunk;
  const int wc = min(kTcChunk, kp - kTcChunk * c);
  __nv_bfloat16 *Bc = Bd + (size_t)kTcChunk * c * kTcDigits * kp;
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    const bool in = j < m && i < m;
    const double x = in ? XQ[(size_t)i * m + j] : 0.0;
    // |X_Q[i][j] 2^c_i| < 2^se, i.e. |X_Q[i][j]| < 2^(se - c_i)
    const unsigned long long f = in ? fixed56(x, se - sc[i]) : 0ull;
    const bool neg = sign_bit(x);
    for (int t = 1; t <= kTcDigits; ++t)
      Bc[(size_t)(t - 1) * wc * kp + core_off(jj, i, kp)] = digit_bf16(f, t, neg);
  }
}

// X = Q X_Q, AX = AQ X_Q (never stored), Rres = AX - X Lambda (optional), and
// per-block partials of ||AX_j - lam_j X_j||^2, ||AX_j||^2, ||X_j||^2 in the
// layout of the FP64 update (part[b][3][m]).
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_update(int n, int m, int kp, int nchunks, const double *__restrict__ Q,
            const double *__restrict__ AQ, const __nv_bfloat16 *__restrict__ Bd,
            const int *__restrict__ fexp, const int *__restrict__ cexp,
            const int *__restrict__ rexp_g, const double *__restrict__ lam, double *__restrict__ X,
            double *__restrict__ Rres, double *__restrict__ part, DevStatus *__restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // A digit planes [8] (128 x kp each), then the chunk's B digit planes [8] (wc x kp each)
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *sB = sA + (size_t)kTcDigits * kTcRows * kp;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int rexp[2][kTcRows];
  __shared__ int sc[kTcMaxK];  // balancing exponents c_i (0 in the padding)
  __shared__ int sf[kTcMaxK];  // column scales f_j
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (n + kTcRows - 1) / kTcRows;
  for (int i = tid; i < kp; i += kTcThreads) {
    sc[i] = i < m ? cexp[i] : 0;
    sf[i] = i < m ? fexp[i] : 0;
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tbase)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  uint32_t commits = 0, waited = 0;  // commits on mbar issued / waited for (uniform)
  bool fail = false;
  const int groups = kp >> 3;        // groups of 8 consecutive K columns per row
  // epilogue mapping: warp w -> TMEM lanes 32 (w & 3) .. + 31, columns 8 (w >> 2) .. + 7
  const int erow = 32 * (warp & 3) + lane, ecol = 8 * (warp >> 2);
  const uint32_t sbo = (uint32_t)(kp >> 3) * 128u;
  for (int c = 0; c < nchunks && !fail; ++c) {
    const int wc = min(kTcChunk, kp - c * kTcChunk);  // output columns of this chunk
    const int j0 = c * kTcChunk;
    // B digits of this chunk to shared memory (16-byte copies); every MMA of the
    // previous chunk completed (the item loop waits for every commit)
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(Bd + (size_t)j0 * kTcDigits * kp);
      uint4 *dst = reinterpret_cast<uint4 *>(sB);
      const int words = kTcDigits * wc * kp * 2 / 16;
      for (int e = tid; e < words; e += kTcThreads) dst[e] = src[e];
    }
    double pe[8], pa[8], px[8];  // residual partial sums of this thread's columns
#pragma unroll
    for (int q = 0; q < 8; ++q) pe[q] = pa[q] = px[q] = 0.0;
    for (int tile = blockIdx.x; tile < ntiles && !fail; tile += gridDim.x) {
      const int r0 = tile * kTcRows;
      for (int o = 0; o < 2 && !fail; ++o) {
        const double *Mt = o == 0 ? Q : AQ;
        if (tid < kTcRows)  // row exponents of M D (k_tc_prep)
          rexp[o][tid] = r0 + tid < n ? rexp_g[(size_t)o * n + r0 + tid] : 0;
        // the MMAs of the previous matrix read the digit planes: wait for them
        bool gave_up = false;
        if (waited < commits) {
          gave_up = !mbar_wait(&mbar, waited & 1u);
          waited = commits;
        }
        fail = __syncthreads_or(gave_up) != 0;  // rexp visible; the same decision in every thread
        if (fail) break;
        // digit planes: one unit = 8 consecutive K columns of one row, one
        // 16-byte store per plane (they form one row of a core matrix); the 8
        // rows of a core matrix are 8 consecutive threads, whose stores fill
        // 128 contiguous bytes
        for (int u = tid; u < kTcRows * groups; u += kTcThreads) {
          const int rem = u % (8 * groups);
          const int row = 8 * (u / (8 * groups)) + (rem & 7), g = rem >> 3, gr = r0 + row;
          const int er = rexp[o][row];
          uint32_t hi[8], lo[8];  // the 56-bit magnitudes as two 28-bit halves
          uint32_t sg[4];         // sign bits of the packed element pairs
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = 8 * g + e;
            const double x = (gr < n && k < m) ? Mt[(size_t)gr * m + k] : 0.0;
            const unsigned long long f = fixed56(x, er + sc[k]);  // |M[r][k] 2^-c_k| < 2^er
            hi[e] = (uint32_t)(f >> 28);
            lo[e] = (uint32_t)(f & 0xFFFFFFFull);
            if (e & 1)
              sg[e >> 1] |= sign_bit(x) ? 0x80000000u : 0u;
            else
              sg[e >> 1] = sign_bit(x) ? 0x8000u : 0u;
          }
          const int off = core_off(row, 8 * g, kp);
#pragma unroll
          for (int t = 1; t <= kTcDigits; ++t) {
            uint32_t w[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
              // digit t: bits 28 - 7t .. of hi for t <= 4, bits 56 - 7t .. of lo for t > 4
              const uint32_t d0 = t <= 4 ? (hi[2 * e2] >> (28 - 7 * t)) & 0x7Fu
                                         : (lo[2 * e2] >> (56 - 7 * t)) & 0x7Fu;
              const uint32_t d1 = t <= 4 ? (hi[2 * e2 + 1] >> (28 - 7 * t)) & 0x7Fu
                                         : (lo[2 * e2 + 1] >> (56 - 7 * t)) & 0x7Fu;
              const uint32_t s = sg[e2] & ((d0 ? 0x8000u : 0u) | (d1 ? 0x80000000u : 0u));
              w[e2] = (digit_bits(d0) | (digit_bits(d1) << 16)) | s;
            }
            *reinterpret_cast<uint4 *>(sA + (size_t)(t - 1) * kTcRows * kp + off) =
                make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t abase = smem_u32(sA), bbase = smem_u32(sB);
          // digit a of A against planes b = 1 .. 9 - a of B: one MMA of
          // N = wc (9 - a) per K step, into levels a + 1 .. 9
          for (int a = 1; a <= kTcDigits; ++a) {
            const int nb = kTcLevels + 1 - a;
            const uint32_t idesc = idesc_bf16(wc * nb);
            const uint32_t dcol = tmem + (uint32_t)((o * kTcLevels + (a - 1)) * wc);
            const uint32_t ap = abase + (uint32_t)((a - 1) * kTcRows * kp * 2);
            for (int kk = 0; kk < kp / 16; ++kk)
              mma_bf16(dcol, smem_desc(ap + kk * 256u, sbo), smem_desc(bbase + kk * 256u, sbo),
                       idesc, (a > 1 || kk > 0) ? 1u : 0u);
          }
          mma_commit(&mbar);
        }
        ++commits;
      }
      if (fail) break;
      // all MMAs of this item complete (the last commit covers the earlier ones)
      {
        bool gave_up = false;
        if (waited < commits) {
          gave_up = !mbar_wait(&mbar, waited & 1u);
          waited = commits;
        }
        fail = __syncthreads_or(gave_up) != 0;
      }
      if (fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // epilogue: this thread's row erow, columns ecol .. ecol + 7 of the chunk;
      // output 0 (X) first, then output 1 (A X) with the residual
      const int gr = r0 + erow;
      double xv[8];
      if (ecol < wc) {
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          long long S1[8], S2[8];  // levels 2..5 and 6..9, each below 2^46
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t uu[4][8];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              const int d = 2 + 4 * half + l;
              const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                                  (uint32_t)((o * kTcLevels + (d - 2)) * wc + ecol);
              tmem_ld8(ta, uu[l]);
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              long long s = 0;
#pragma unroll
              for (int l = 0; l < 4; ++l)  // weight 2^{7(3 - l)} within the half
                s += (long long)__float2int_rn(__uint_as_float(uu[l][q])) << (7 * (3 - l));
              if (half == 0)
                S1[q] = s;
              else
                S2[q] = s;
            }
          }
          const int er = rexp[o][erow];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + ecol + q;
            if (gr >= n || j >= m) continue;
            // T = S1 2^28 + S2 as a signed 128-bit value (hi, lo)
            const unsigned long long s1lo = (unsigned long long)S1[q] << 28;
            unsigned long long lo = s1lo + (unsigned long long)S2[q];
            const unsigned long long carry = lo < s1lo ? 1ull : 0ull;
            unsigned long long hi = (unsigned long long)(S1[q] >> 36) +
                                    (unsigned long long)(S2[q] >> 63) + carry;
            const bool neg = (long long)hi < 0;
            if (neg) {  // magnitude of the two's complement value
              lo = ~lo + 1ull;
              hi = ~hi + (lo == 0 ? 1ull : 0ull);
            }
            const double val = int128_to_double(hi, lo, neg, er + sf[j] - 63);
            if (o == 0) {
              xv[q] = val;
              X[(size_t)gr * m + j] = val;
            } else {
              const double x = xv[q], ax = val;
              const double dd = fma(-lam[j], x, ax);
              if (Rres) Rres[(size_t)gr * m + j] = dd;
              pe[q] = fma(dd, dd, pe[q]);
              pa[q] = fma(ax, ax, pa[q]);
              px[q] = fma(x, x, px[q]);
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // TMEM and rexp free for the next item
    }
    // block partials of this chunk's columns: the digit planes are free (every
    // MMA completed), so they hold the per-thread sums; column group cg (8
    // columns) is summed over warps 4 cg .. 4 cg + 3 and their lanes in a
    // fixed order
    if (!fail) {
      double *dred = reinterpret_cast<double *>(smem_raw);  // [16 warps][32 lanes][9]
      for (int which = 0; which < 3; ++which) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dred[(warp * 32 + lane) * 9 + q] = which == 0 ? pe[q] : (which == 1 ? pa[q] : px[q]);
        __syncthreads();
        if (tid < kTcChunk) {
          const int cg = tid / 8, q = tid % 8;
          const int j = j0 + tid;
          if (j < m && tid < wc) {
            double sum = 0.0;
            for (int w = 0; w < 4; ++w)
              for (int l = 0; l < 32; ++l) sum += dred[((cg * 4 + w) * 32 + l) * 9 + q];
            part[((size_t)blockIdx.x * 3 + which) * m + j] = sum;
          }
        }
        __syncthreads();
      }
    }
  }
  if (fail) {
    if (tid == 0) atomicExch(&status->tc_timeout, 1);
    // wait (bounded) for this CTA's outstanding MMAs before freeing TMEM
    if (waited < commits) mbar_wait(&mbar, waited & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------
// Gram matrices on the tensor cores (Algorithm 2, step 3: B_Q = Q^T Q and
// A_Q = Q^T (A Q), B = I), FP64-accurate.
//
// The contraction runs over the n rows, so FP32 accumulation of digit
// products is exact only over a bounded number of rows: the rows go in slabs
// of kGramSlab = 96, and every value of a slab is written as eight signed
// 7-bit digits (56-bit fixed point) below a per-slab, per-column power of two
// 2^e (2^e > the column's largest magnitude in the slab). Level d = a + b of
// digit pairs (2 <= d <= 9; at most 8 pairs of 96 products below 2^14 each,
// < 2^24) is an exact FP32 sum; the slab's entry is 2^{e_i + e_j - 63} T with
// T = sum_d acc_d 2^{7(9 - d)} formed in integers and rounded once to FP64,
// and the slabs are added in FP64 in a fixed order. The dropped pairs
// (a + b > 9) and the 56-bit truncation weigh below 2^-48 ||q_i|| ||q_j|| in
// all (2^-55 of the slab maxima per product, times the 96 rows of a slab,
// bounded through sum over slabs of max_i max_j <= ||q_i|| ||q_j||), against
// the ~sqrt(n) 2^-53 ||q_i|| ||q_j|| a sequential FP64 dot product reaches.
//
// MMA shapes: M = 128 rows = the columns i of Q (rows i >= m of the A operand
// are whatever follows in shared memory: they only reach TMEM lanes that are
// never read), N = a chunk of wc <= 48 output columns j, K = the 96 rows of
// the slab. TMEM holds the 8 levels of one output (8 wc <= 384 columns), so
// B_Q's MMAs (B operand = the chunk's rows of Q's own digit planes, one MMA per
// digit pair) and A_Q's (B operand = the digit planes of the chunk's columns of
// A Q, stacked along N as in the update) run one after the other per slab.
// CTA (chunk c, member g) takes the slabs g, g + G, ... and keeps 2 x wc/4
// FP64 sums per thread; per-CTA partials are then summed in CTA order.
constexpr int kGramSlab = 96;
constexpr int kGramDigits = 8;
constexpr int kGramLevels = 8;     // levels d = 2..9
constexpr int kGramChunk = 48;     // output columns per chunk (8 x 48 <= 512 TMEM columns)
constexpr int kGramColsPerThread = kGramChunk / 4;
// digit units (column, 8 rows) of a slab per thread: (80 + 48) x 96 / 8 / 512
constexpr int kGramUnits = ((kTcMaxK + kGramChunk) * (kGramSlab / 8) + kTcThreads - 1) / kTcThreads;

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}

// 8 consecutive slab rows of one column as the 16-byte core-matrix rows of the
// eight digit planes (plane stride `pstride` elements, offset `off` in a plane)
__device__ __forceinline__ void gram_digits8(const double (&x)[8], int e, __nv_bfloat16 *planes,
                                             size_t pstride, int off) {
  unsigned long long f[8];
  uint32_t sg[4];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    f[q] = fixed56(x[q], e);
    if (q & 1)
      sg[q >> 1] |= sign_bit(x[q]) ? 0x80000000u : 0u;
    else
      sg[q >> 1] = sign_bit(x[q]) ? 0x8000u : 0u;
  }
#pragma unroll
  for (int t = 1; t <= kGramDigits; ++t) {
    uint32_t w[4];
#pragma unroll
    for (int q2 = 0; q2 < 4; ++q2) {
      const uint32_t d0 = (uint32_t)(f[2 * q2] >> (56 - 7 * t)) & 0x7Fu;
      const uint32_t d1 = (uint32_t)(f[2 * q2 + 1] >> (56 - 7 * t)) & 0x7Fu;
      const uint32_t sm = sg[q2] & ((d0 ? 0x8000u : 0u) | (d1 ? 0x80000000u : 0u));
      w[q2] = (digit_bits(d0) | (digit_bits(d1) << 16)) | sm;
    }
    *reinterpret_cast<uint4 *>(planes + (size_t)(t - 1) * pstride + off) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gram(int n, int m, int mrows, int nch, int G, const double *__restrict__ Q,
          const double *__restrict__ AQ, double *__restrict__ part,
          DevStatus *__restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // A planes: 9 x (mrows x 64), then a tail so that the 128 rows an MMA reads
  // stay inside the allocation; then the 9 planes of the chunk's A Q columns
  const size_t pa = (size_t)mrows * kGramSlab;  // elements per A plane
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *sB = sA + kGramDigits * pa + (size_t)(kTcRows - mrows) * kGramSlab;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int eA[kTcMaxK], eB[kGramChunk];  // per-slab column exponents
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.x / G, g = blockIdx.x % G;  // chunk, member
  const int j0 = c * kGramChunk;
  const int kp = (m + 15) / 16 * 16;
  const int wc = min(kGramChunk, kp - j0);       // output columns of the chunk (multiple of 16)
  const size_t pb = (size_t)wc * kGramSlab;    // elements per B plane
  const int nslab = (n + kGramSlab - 1) / kGramSlab;
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tbase)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the tail rows (read by the last plane's MMAs into unused lanes): zero
  for (size_t e = tid; e < (size_t)(kTcRows - mrows) * kGramSlab; e += kTcThreads)
    sA[kGramDigits * pa + e] = __ushort_as_bfloat16((unsigned short)0);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const uint32_t sbo = (uint32_t)(kGramSlab >> 3) * 128u;
  uint32_t commits = 0, waited = 0;
  bool fail = false;
  // drain mapping: warp w -> TMEM lanes (rows i) 32 (w & 3) + lane, columns cg * wc/4 ..
  const int ei = 32 * (warp & 3) + lane, cg = warp >> 2, cpt = wc / 4;
  double acc0[kGramColsPerThread], acc1[kGramColsPerThread];  // B_Q and A_Q sums
#pragma unroll
  for (int q = 0; q < kGramColsPerThread; ++q) acc0[q] = acc1[q] = 0.0;
  for (int sl = g; sl < nslab && !fail; sl += G) {
    const int r0 = sl * kGramSlab;
    // digit planes: unit = (column, 8 consecutive slab rows); consecutive
    // threads take consecutive columns (coalesced loads, 128-byte stores). A
    // thread holds the values of its (at most kGramUnits) units in registers:
    // their largest exponents set the per-slab column scales (shared-memory
    // maxima), and the digits are cut from the same registers after a barrier.
    for (int i = tid; i < kTcMaxK + kGramChunk; i += kTcThreads) {
      if (i < kTcMaxK)
        eA[i] = kNoExp;
      else
        eB[i - kTcMaxK] = kNoExp;
    }
    __syncthreads();  // (the previous slab's MMAs completed before its drain)
    const int unitsA = mrows * (kGramSlab / 8), unitsB = wc * (kGramSlab / 8);
    double xs[kGramUnits][8];
#pragma unroll
    for (int t = 0; t < kGramUnits; ++t) {
      const int u = tid + t * kTcThreads;
      const bool isA = u < unitsA;
      const int v = isA ? u : u - unitsA;
      const int rows = isA ? mrows : wc;
      const int col = v % rows, rg = v / rows;
      const int j = isA ? col : j0 + col;
      const double *M = isA ? Q : AQ;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = r0 + 8 * rg + q;
        xs[t][q] = (u < unitsA + unitsB && r < n && j < m) ? M[(size_t)r * m + j] : 0.0;
      }
    }
#pragma unroll
    for (int t = 0; t < kGramUnits; ++t) {
      const int u = tid + t * kTcThreads;
      if (u >= unitsA + unitsB) continue;
      const bool isA = u < unitsA;
      const int v = isA ? u : u - unitsA;
      const int col = v % (isA ? mrows : wc);
      int ex = kNoExp;
#pragma unroll
      for (int q = 0; q < 8; ++q) ex = max(ex, scale_exp(xs[t][q]));
      if (ex != kNoExp) atomicMax(isA ? &eA[col] : &eB[col], ex);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kGramUnits; ++t) {
      const int u = tid + t * kTcThreads;
      if (u >= unitsA + unitsB) continue;
      const bool isA = u < unitsA;
      const int v = isA ? u : u - unitsA;
      const int rows = isA ? mrows : wc;
      const int col = v % rows, rg = v / rows;
      int e = isA ? (col < m ? eA[col] : kNoExp) : eB[col];
      if (e == kNoExp) e = 0;
      gram_digits8(xs[t], e, isA ? sA : sB, isA ? pa : pb, core_off(col, 8 * rg, kGramSlab));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    for (int o = 0; o < 2 && !fail; ++o) {
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t abase = smem_u32(sA), bbase = smem_u32(sB);
        if (o == 0) {  // B_Q: B operand = rows j0 .. j0 + wc of Q's own planes
          const uint32_t idesc = idesc_bf16(wc);
          for (int a = 1; a <= kGramDigits; ++a)
            for (int b = 1; a + b <= kGramLevels + 1; ++b) {
              const uint32_t dcol = tmem + (uint32_t)((a + b - 2) * wc);
              const uint32_t ap = abase + (uint32_t)((a - 1) * pa * 2);
              const uint32_t bp = abase + (uint32_t)((b - 1) * pa * 2) + (uint32_t)(j0 / 8) * sbo;
              for (int kk = 0; kk < kGramSlab / 16; ++kk)
                mma_bf16(dcol, smem_desc(ap + kk * 256u, sbo), smem_desc(bp + kk * 256u, sbo),
                         idesc, (a > 1 || kk > 0) ? 1u : 0u);
            }
        } else {  // A_Q: planes b of the chunk's A Q columns, stacked along N
          const int per = 256 / wc;  // planes per MMA (N <= 256)
          for (int a = 1; a <= kGramDigits; ++a)
            for (int b0 = 1; a + b0 <= kGramLevels + 1; b0 += per) {
              const int nb = min(per, kGramLevels + 1 - a - b0 + 1);
              const uint32_t idesc = idesc_bf16(wc * nb);
              const uint32_t dcol = tmem + (uint32_t)((a + b0 - 2) * wc);
              const uint32_t ap = abase + (uint32_t)((a - 1) * pa * 2);
              const uint32_t bp = bbase + (uint32_t)((b0 - 1) * pb * 2);
              for (int kk = 0; kk < kGramSlab / 16; ++kk)
                mma_bf16(dcol, smem_desc(ap + kk * 256u, sbo), smem_desc(bp + kk * 256u, sbo),
                         idesc, (a > 1 || kk > 0) ? 1u : 0u);
            }
        }
        mma_commit(&mbar);
      }
      ++commits;
      bool gave_up = false;
      if (waited < commits) {
        gave_up = !mbar_wait(&mbar, waited & 1u);
        waited = commits;
      }
      fail = __syncthreads_or(gave_up) != 0;
      if (fail) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // drain: T = S1 2^28 + S2, S1 = levels 2..5, S2 = levels 6..9; warps whose
      // 32 TMEM lanes hold no row i < m skip it (a warp-uniform condition)
      long long S1[kGramColsPerThread], S2[kGramColsPerThread];
#pragma unroll
      for (int q = 0; q < kGramColsPerThread; ++q) S1[q] = S2[q] = 0;
      const int dlevels = 32 * (warp & 3) < m ? kGramLevels + 1 : 1;
      for (int d = 2; d <= dlevels; ++d) {
        uint32_t uu[kGramColsPerThread];
        const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                            (uint32_t)((d - 2) * wc + cg * cpt);
        if (cpt == 12) {
          uint32_t v8[8], v4[4];
          tmem_ld8(ta, v8);
          tmem_ld4(ta + 8, v4);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 8; ++q) uu[q] = v8[q];
#pragma unroll
          for (int q = 0; q < 4; ++q) uu[8 + q] = v4[q];
        } else if (cpt == 8) {
          uint32_t v8[8];
          tmem_ld8(ta, v8);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 8; ++q) uu[q] = v8[q];
#pragma unroll
          for (int q = 8; q < kGramColsPerThread; ++q) uu[q] = 0u;
        } else {  // cpt == 4
          uint32_t v4[4];
          tmem_ld4(ta, v4);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 4; ++q) uu[q] = v4[q];
#pragma unroll
          for (int q = 4; q < kGramColsPerThread; ++q) uu[q] = 0u;
        }
#pragma unroll
        for (int q = 0; q < kGramColsPerThread; ++q) {
          const long long v = (long long)__float2int_rn(__uint_as_float(uu[q]));
          if (d <= 5)
            S1[q] += v << (7 * (5 - d));
          else
            S2[q] += v << (7 * (9 - d));
        }
      }
      if (ei < m) {
#pragma unroll
        for (int q = 0; q < kGramColsPerThread; ++q) {
          const int jj = cg * cpt + q, j = j0 + jj;
          if (q >= cpt || j >= m) continue;
          const unsigned long long s1lo = (unsigned long long)S1[q] << 28;
          unsigned long long lo = s1lo + (unsigned long long)S2[q];
          const unsigned long long carry = lo < s1lo ? 1ull : 0ull;
          unsigned long long hi = (unsigned long long)(S1[q] >> 36) +
                                  (unsigned long long)(S2[q] >> 63) + carry;
          const bool neg = (long long)hi < 0;
          if (neg) {
            lo = ~lo + 1ull;
            hi = ~hi + (lo == 0 ? 1ull : 0ull);
          }
          const int ej = o == 0 ? eA[j] : eB[jj];
          const int e2 = (eA[ei] == kNoExp ? 0 : eA[ei]) + (ej == kNoExp ? 0 : ej) - 63;
          const double v = int128_to_double(hi, lo, neg, e2);
          if (o == 0)
            acc0[q] += v;
          else
            acc1[q] += v;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // TMEM free for the next pass
    }
  }
  // this CTA's partial sums: part[cta][o][i][jj] (mrows x kGramChunk per output)
  if (!fail && ei < m) {
    double *P = part + (size_t)blockIdx.x * 2 * mrows * kGramChunk;
#pragma unroll
    for (int q = 0; q < kGramColsPerThread; ++q)
      if (q < cpt) {
        P[(size_t)ei * kGramChunk + cg * cpt + q] = acc0[q];
        P[((size_t)mrows + ei) * kGramChunk + cg * cpt + q] = acc1[q];
      }
  }
  if (fail) {
    if (tid == 0) atomicExch(&status->tc_timeout, 1);
    if (waited < commits) mbar_wait(&mbar, waited & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// B_Q, A_Q from the per-CTA partials: entry (i, j) of output o is the sum over
// the G CTAs of chunk j / 48 in CTA order; each output is symmetrised as the
// mean of (i, j) and (j, i).
__global__ void k_tc_gram_reduce(int m, int mrows, int G, const double *__restrict__ part,
                                 double *__restrict__ Aq, double *__restrict__ Bq) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int i = idx / m, j = idx % m;
  if (i > j) return;
  double v[2][2];
  for (int o = 0; o < 2; ++o)
    for (int t = 0; t < 2; ++t) {
      const int r = t ? j : i, cc = t ? i : j;  // entry (r, cc)
      const int ch = cc / kGramChunk, jj = cc % kGramChunk;
      double sum = 0.0;
      for (int g = 0; g < G; ++g)
        sum += part[(((size_t)(ch * G + g) * 2 + o) * mrows + r) * kGramChunk + jj];
      v[o][t] = sum;
    }
  const double b = 0.5 * (v[0][0] + v[0][1]), a = 0.5 * (v[1][0] + v[1][1]);
  Bq[(size_t)i * m + j] = b;
  Bq[(size_t)j * m + i] = b;
  Aq[(size_t)i * m + j] = a;
  Aq[(size_t)j * m + i] = a;
}

size_t tc_gram_smem_bytes(int mrows) {
  const size_t need = ((size_t)kGramDigits * mrows * kGramSlab +
                       (size_t)(kTcRows - mrows) * kGramSlab +
                       (size_t)kGramDigits * kGramChunk * kGramSlab) * 2;
  // over half of the SM's shared memory: one CTA (holding all 512 TMEM columns) per SM
  const size_t floor_bytes = 120 * 1024;
  return need > floor_bytes ? need : floor_bytes;
}

size_t tc_smem_bytes(int kp) {
  const size_t need = (size_t)kTcDigits * kTcRows * kp * 2 + (size_t)kTcDigits * kTcChunk * kp * 2;
  // at least 16 x 32 x 9 doubles for the partials, and over half of the SM's
  // shared memory so that one CTA (holding all 512 TMEM columns) runs per SM
  const size_t floor_bytes = 120 * 1024;
  return need > floor_bytes ? need : floor_bytes;
}

// B digit planes of all chunks (kp columns x 8 planes x kp), f_j, c_i, and
// the row exponents of Q D and A Q D
size_t tc_scratch_bytes(int64_t n, int m0) {
  const int kp = (m0 + 15) / 16 * 16;
  return (size_t)kp * kTcDigits * kp * 2 + (size_t)(2 * kTcMaxK + 2 * n) * sizeof(int);
}

}  // namespace

// CTAs per column chunk of the tensor-core Gram (0: not supported)
int gram_tc_group(const RRArgs &a) {
  if (a.m0 > kTcMaxK || a.rowptrB != nullptr || a.n < (int64_t)kGramSlab * 4) return 0;
  const int mrows = (a.m0 + 7) / 8 * 8;
  const int kp = (a.m0 + 15) / 16 * 16;
  const int nch = (kp + kGramChunk - 1) / kGramChunk;
  const size_t gram_bytes = (size_t)a.Pg * 2 * ((a.m0 + 3) / 4 * 4) * ((a.m0 + 3) / 4 * 4) * 8;
  const size_t per_cta = (size_t)2 * mrows * kGramChunk * sizeof(double);
  const int nslab = (int)((a.n + kGramSlab - 1) / kGramSlab);
  int G = (a.num_sms > 0 ? a.num_sms : 1) / nch;
  G = std::min<int>(G, (int)(gram_bytes / (per_cta * nch)));
  G = std::min(G, nslab);
  return G >= 1 ? G : 0;
}

cudaError_t gram_tc(const RRArgs &a, cudaStream_t st) {
  const int G = gram_tc_group(a);
  if (G < 1) return cudaErrorInvalidValue;
  const int m = a.m0;
  const int mrows = (m + 7) / 8 * 8;
  const int kp = (m + 15) / 16 * 16;
  const int nch = (kp + kGramChunk - 1) / kGramChunk;
  k_tc_gram<<<nch * G, kTcThreads, tc_gram_smem_bytes(mrows), st>>>((int)a.n, m, mrows, nch, G,
                                                                     a.Q, a.AQ, a.gram_part,
                                                                     a.status);
  k_tc_gram_reduce<<<(m * m + 255) / 256, 256, 0, st>>>(m, mrows, G, a.gram_part, a.Aq, a.Bq);
  return cudaGetLastError();
}

bool update_resid_tc_supported(const RRArgs &a) {
  const size_t gram_bytes = (size_t)a.Pg * 2 * ((a.m0 + 3) / 4 * 4) * ((a.m0 + 3) / 4 * 4) * 8;
  return a.m0 <= kTcMaxK && a.rowptrB == nullptr && tc_scratch_bytes(a.n, a.m0) <= gram_bytes &&
         a.n >= kTcRows;
}

cudaError_t update_resid_tc(const RRArgs &a, int blocks, cudaStream_t st) {
  const int m = a.m0;
  const int kp = (m + 15) / 16 * 16;
  const int nchunks = (kp + kTcChunk - 1) / kTcChunk;
  // B digits and column scales in the Gram partials buffer, which the reduced
  // eigensolver has finished with
  __nv_bfloat16 *Bd = reinterpret_cast<__nv_bfloat16 *>(a.gram_part);
  int *fexp = reinterpret_cast<int *>(Bd + (size_t)kp * kTcDigits * kp);
  int *cexp = fexp + kTcMaxK;
  int *rexp = cexp + kTcMaxK;
  const int prep_blocks = kp + (a.n + kTcPrepRows - 1) / kTcPrepRows;
  k_tc_prep<<<prep_blocks, kTcPrepRows * (kp >> 3), 0, st>>>(a.n, m, kp, a.XQ, a.Bq, a.Q, a.AQ,
                                                              Bd, fexp, cexp, rexp);
  k_tc_update<<<blocks, kTcThreads, tc_smem_bytes(kp), st>>>(a.n, m, kp, nchunks, a.Q, a.AQ, Bd,
                                                              fexp, cexp, rexp, a.lam, a.X,
                                                              a.Rres, a.res_part, a.status);
  return cudaGetLastError();
}

cudaError_t rr_tc_init() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tc_smem_bytes(kTcMaxK));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_gram_smem_bytes(kTcMaxK));
}

}  // namespace ifeast
