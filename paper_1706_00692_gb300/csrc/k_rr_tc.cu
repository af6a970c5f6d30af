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
// truncation), combined exactly as two 64-bit integers and converted to FP64
// once:
//     (Q X_Q)[r][j] = 2^{e_r + f_j} (H 2^-35 + L 2^-63),
//     H = sum_{d=2..5} acc_d 2^{7(5-d)},  L = sum_{d=6..9} acc_d 2^{7(9-d)}.
// The result carries the 56-bit truncation of the operands and one FP64
// rounding, i.e. FP64 accuracy, with no FP64 multiply on the products.
//
// Layout (tcgen05.mma kind::f16, BF16 operands, FP32 accumulators in TMEM,
// cta_group::1, M = 128 rows of the tile, N = a 32-column (or 16-column) chunk
// of the output, K = m0 padded to a multiple of 16): operands in shared memory
// in the no-swizzle K-major layout of 8 x 16-byte core matrices (leading byte
// offset 128 B between core matrices along K, stride byte offset (K/8) x 128 B
// between groups of 8 rows). Shared memory holds the 8 digit planes of one
// 128-row tile of Q (then of A Q) and the 8 digit planes of the 32 columns of
// X_Q of the chunk; TMEM holds 2 outputs x 8 levels x 32 columns (512 columns).
// One persistent CTA of 512 threads per SM walks (column chunk, row tile)
// items. Every wait on the mbarrier is bounded: a wait that runs out sets
// status->tc_timeout, and the CTA stops issuing work, waits (bounded) for its
// own outstanding MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"

namespace ifeast {

namespace {

constexpr int kTcThreads = 512;
constexpr int kTcRows = 128;      // M: rows of one tile (TMEM lanes)
constexpr int kTcDigits = 8;      // digits per operand value (56 bits)
constexpr int kTcLevels = 8;      // levels d = 2..9
constexpr int kTcMaxK = 80;       // m0 padded, at most (digit sums stay below 2^24)
constexpr int kTcChunk = 32;      // output columns per item (N)
constexpr long kTcSpin = 1L << 26;  // try_wait polls before a wait gives up

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

constexpr int kNoExp = -(1 << 20);  // exponent of 0 (and of denormals)

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

// signed digit t (1..8) of a fixed-point magnitude, as BF16 (|d| <= 127: exact)
__device__ __forceinline__ __nv_bfloat16 digit_bf16(unsigned long long f, int t, bool neg) {
  const int d = (int)((f >> (56 - 7 * t)) & 0x7F);
  return __float2bfloat16_rn((float)(neg ? -d : d));
}

// Digits of D^-1 X_Q for the B operand: column j (the output column) has the
// scale f_j (2^f_j > max_i |X_Q[i][j]| 2^c_i); Bd[(c * 8 + t - 1) * 32 * kp +
// core_off(j - 32 c, i, kp)] = digit t of X_Q[i][j] 2^c_i (signed), 0 in the
// padding. Block 0 also writes the balancing exponents cexp[i] = c_i.
__global__ void k_tc_bdigits(int m, int kp, const double *__restrict__ XQ,
                             const double *__restrict__ Bq, __nv_bfloat16 *__restrict__ Bd,
                             int *__restrict__ fexp, int *__restrict__ cexp) {
  const int j = blockIdx.x;  // one block per output column, padding columns included
  __shared__ int se;
  __shared__ int sc[kTcMaxK];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    sc[i] = balance_exp(Bq, m, i);
    if (j == 0) cexp[i] = sc[i];
  }
  __syncthreads();
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
  for (int i = threadIdx.x; i < kp; i += blockDim.x) {
    const bool in = j < m && i < m;
    const double x = in ? XQ[(size_t)i * m + j] : 0.0;
    // |X_Q[i][j] 2^c_i| < 2^se, i.e. |X_Q[i][j]| < 2^(se - c_i)
    const unsigned long long f = in ? fixed56(x, se - sc[i]) : 0ull;
    const bool neg = x < 0.0;
    for (int t = 1; t <= kTcDigits; ++t)
      Bd[((size_t)c * kTcDigits + (t - 1)) * kTcChunk * kp + core_off(jj, i, kp)] =
          digit_bf16(f, t, neg);
  }
}

// X = Q X_Q, AX = AQ X_Q (never stored), Rres = AX - X Lambda (optional), and
// per-block partials of ||AX_j - lam_j X_j||^2, ||AX_j||^2, ||X_j||^2 in the
// layout of the FP64 update (part[b][3][m]).
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_update(int n, int m, int kp, int nchunks, const double *__restrict__ Q,
            const double *__restrict__ AQ, const __nv_bfloat16 *__restrict__ Bd,
            const int *__restrict__ fexp, const int *__restrict__ cexp,
            const double *__restrict__ lam, double *__restrict__ X,
            double *__restrict__ Rres, double *__restrict__ part, DevStatus *__restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // A digit planes [8] (128 x kp each), then B digit planes [8] (32 x kp each)
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
  __nv_bfloat16 *sB = sA + (size_t)kTcDigits * kTcRows * kp;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  __shared__ int rexp[2][kTcRows];
  __shared__ int sc[kTcMaxK];  // balancing exponents c_i (0 in the padding)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (n + kTcRows - 1) / kTcRows;
  for (int i = tid; i < kp; i += kTcThreads) sc[i] = i < m ? cexp[i] : 0;
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
  const int kq = kp >> 2;            // row-scale pass: 4 threads per row, kq columns each
  // epilogue mapping: warp w -> TMEM lanes 32 (w & 3) .. + 31, columns 8 (w >> 2) .. + 7
  const int erow = 32 * (warp & 3) + lane, ecol = 8 * (warp >> 2);
  const uint32_t sbo = (uint32_t)(kp >> 3) * 128u;
  for (int c = 0; c < nchunks && !fail; ++c) {
    const int nc = (kp - c * kTcChunk) >= kTcChunk ? kTcChunk : 16;  // N of this chunk
    const int j0 = c * kTcChunk;
    const uint32_t idesc = idesc_bf16(nc);
    // B digits of this chunk to shared memory (16-byte copies); every MMA of the
    // previous chunk completed (the item loop waits for every commit)
    {
      const uint4 *src = reinterpret_cast<const uint4 *>(Bd + (size_t)c * kTcDigits * kTcChunk * kp);
      uint4 *dst = reinterpret_cast<uint4 *>(sB);
      const int words = kTcDigits * kTcChunk * kp * 2 / 16;
      for (int e = tid; e < words; e += kTcThreads) dst[e] = src[e];
    }
    double pe[8], pa[8], px[8];  // residual partial sums of this thread's columns
#pragma unroll
    for (int q = 0; q < 8; ++q) pe[q] = pa[q] = px[q] = 0.0;
    for (int tile = blockIdx.x; tile < ntiles && !fail; tile += gridDim.x) {
      const int r0 = tile * kTcRows;
      for (int o = 0; o < 2 && !fail; ++o) {
        const double *Mt = o == 0 ? Q : AQ;
        {  // row scales of M D: 4 threads per row, kq columns each
          const int row = tid >> 2, qtr = tid & 3, gr = r0 + row;
          int ex = kNoExp;  // max_k of the exponent of M[r][k] 2^-c_k
          for (int q = 0; q < kq; ++q) {
            const int k = qtr * kq + q;
            if (gr < n && k < m) {
              const int ek = scale_exp(Mt[(size_t)gr * m + k]);
              if (ek != kNoExp) ex = max(ex, ek - sc[k]);
            }
          }
          ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 1));
          ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 2));
          if (qtr == 0) rexp[o][row] = ex == kNoExp ? 0 : ex;
        }
        // the MMAs of the previous matrix read the digit planes: wait for them
        bool gave_up = false;
        if (waited < commits) {
          gave_up = !mbar_wait(&mbar, waited & 1u);
          waited = commits;
        }
        fail = __syncthreads_or(gave_up) != 0;  // rexp visible; the same decision in every thread
        if (fail) break;
        // digit planes: one unit = 8 consecutive K columns of one row, one
        // 16-byte store per plane (they form one row of a core matrix)
        for (int u = tid; u < kTcRows * groups; u += kTcThreads) {
          const int row = u / groups, g = u % groups, gr = r0 + row;
          const int er = rexp[o][row];
          unsigned long long f[8];
          unsigned neg = 0u;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = 8 * g + e;
            const double x = (gr < n && k < m) ? Mt[(size_t)gr * m + k] : 0.0;
            f[e] = fixed56(x, er + sc[k]);  // |M[r][k] 2^-c_k| < 2^er
            neg |= (x < 0.0 ? 1u : 0u) << e;
          }
          const int off = core_off(row, 8 * g, kp);
#pragma unroll
          for (int t = 1; t <= kTcDigits; ++t) {
            __align__(16) __nv_bfloat16 dg[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) dg[e] = digit_bf16(f[e], t, (neg >> e) & 1u);
            *reinterpret_cast<uint4 *>(sA + (size_t)(t - 1) * kTcRows * kp + off) =
                *reinterpret_cast<const uint4 *>(dg);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t abase = smem_u32(sA), bbase = smem_u32(sB);
          for (int a = 1; a <= kTcDigits; ++a)
            for (int b = 1; a + b <= kTcLevels + 1; ++b) {
              const int d = a + b;  // level 2..9, first written by the pair (1, d - 1)
              const uint32_t dcol = tmem + (uint32_t)((o * kTcLevels + (d - 2)) * kTcChunk);
              const uint32_t ap = abase + (uint32_t)((a - 1) * kTcRows * kp * 2);
              const uint32_t bp = bbase + (uint32_t)((b - 1) * kTcChunk * kp * 2);
              for (int kk = 0; kk < kp / 16; ++kk)
                mma_bf16(dcol, smem_desc(ap + kk * 256u, sbo), smem_desc(bp + kk * 256u, sbo),
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
      if (ecol < nc) {
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          long long H[8], L[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) H[q] = L[q] = 0;
#pragma unroll
          for (int d = 2; d <= 9; ++d) {
            uint32_t uu[8];
            const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                                (uint32_t)((o * kTcLevels + (d - 2)) * kTcChunk + ecol);
            tmem_ld8(ta, uu);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const long long w = d <= 5 ? (1LL << (7 * (5 - d))) : (1LL << (7 * (9 - d)));
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const long long iv = __float2ll_rn(__uint_as_float(uu[q]));  // an exact integer
              if (d <= 5)
                H[q] += iv * w;
              else
                L[q] += iv * w;
            }
          }
          const int er = rexp[o][erow];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = j0 + ecol + q;
            if (gr >= n || j >= m) continue;
            const double val = ldexp(fma((double)L[q], 0x1p-63, (double)H[q] * 0x1p-35),
                                     er + fexp[j]);
            if (o == 0) {
              xv[q] = val;
              X[(size_t)gr * m + j] = val;
            } else {
              const double x = xv[q], ax = val;
              const double dd = ax - lam[j] * x;
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
          if (j < m && tid < nc) {
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

size_t tc_smem_bytes(int kp) {
  const size_t need = (size_t)kTcDigits * kTcRows * kp * 2 + (size_t)kTcDigits * kTcChunk * kp * 2;
  // at least 16 x 32 x 9 doubles for the partials, and over half of the SM's
  // shared memory so that one CTA (holding all 512 TMEM columns) runs per SM
  const size_t floor_bytes = 120 * 1024;
  return need > floor_bytes ? need : floor_bytes;
}

size_t tc_bdigit_bytes(int m0) {
  const int kp = (m0 + 15) / 16 * 16;
  const int nchunks = (kp + kTcChunk - 1) / kTcChunk;
  return (size_t)nchunks * kTcDigits * kTcChunk * kp * 2 +
         (size_t)(nchunks * kTcChunk + kTcMaxK) * sizeof(int);
}

}  // namespace

bool update_resid_tc_supported(const RRArgs &a) {
  const size_t gram_bytes = (size_t)a.Pg * 2 * ((a.m0 + 3) / 4 * 4) * ((a.m0 + 3) / 4 * 4) * 8;
  return a.m0 <= kTcMaxK && a.rowptrB == nullptr && tc_bdigit_bytes(a.m0) <= gram_bytes &&
         a.n >= kTcRows;
}

cudaError_t update_resid_tc(const RRArgs &a, int blocks, cudaStream_t st) {
  const int m = a.m0;
  const int kp = (m + 15) / 16 * 16;
  const int nchunks = (kp + kTcChunk - 1) / kTcChunk;
  // B digits and column scales in the Gram partials buffer, which the reduced
  // eigensolver has finished with
  __nv_bfloat16 *Bd = reinterpret_cast<__nv_bfloat16 *>(a.gram_part);
  int *fexp = reinterpret_cast<int *>(Bd + (size_t)nchunks * kTcDigits * kTcChunk * kp);
  int *cexp = fexp + (size_t)nchunks * kTcChunk;
  k_tc_bdigits<<<nchunks * kTcChunk, 128, 0, st>>>(m, kp, a.XQ, a.Bq, Bd, fexp, cexp);
  k_tc_update<<<blocks, kTcThreads, tc_smem_bytes(kp), st>>>(a.n, m, kp, nchunks, a.Q, a.AQ, Bd,
                                                              fexp, cexp, a.lam, a.X, a.Rres,
                                                              a.res_part, a.status);
  return cudaGetLastError();
}

cudaError_t rr_tc_init() {
  return cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)tc_smem_bytes(kTcMaxK));
}

}  // namespace ifeast
