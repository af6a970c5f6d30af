// Inner solve of IFEAST (Algorithm 2, steps 1-2) on the GPU: for every contour
// node z_k and every column b_j of the right-hand side block, GMRES on
// (z_k B - A) y = b_j with zero initial guess (Section 2.2), all C = nc * m0
// systems advanced together, then the quadrature sum Q = Re sum_k w_k Y_k.
// The right-hand sides are X (B X for a generalized problem), or, in the
// residual form, r_j = A x_j - lambda_j B x_j of the current Ritz pairs: then
// (z B - A)^{-1} B x_j = (x_j + (z B - A)^{-1} r_j) / (z - lambda_j) and only
// the correction is solved by GMRES.
//
// Data layout (all row-major, complex values interleaved as double2, or
// float2 for the FP32 basis):
//   V[s]  n x C basis vector s of every system, column c = k * m0 + j
//   W     n x C work vector (A-product, then Gram-Schmidt in place)
// One Arnoldi step s runs five kernels:
//   spmm_shift, dots W = z B V_s - A V_s, then block partials of h1_l = <V_l, W>
//   reduce           h1 (fixed-order sum of the block partials)
//   orth_update_dot  W -= sum_l h1_l V_l and partials of h2_l = <V_l, W>, ||W||^2
//   reduce           h2, ||W||^2
//   givens           h = h1 + h2, h_{s+1,s} = sqrt(||W||^2 - sum |h2_l|^2),
//                    Givens update of the least-squares problem, stop test
//   orth_finish      V_{s+1} = (W - sum_l h2_l V_l) / h_{s+1,s}
// (classical Gram-Schmidt applied twice; the norm after the second pass
// follows from the first-pass norm by Pythagoras because V_0..V_s are
// orthonormal.) Every reduction sums block partials in a fixed order, so the
// result does not depend on scheduling. With the FP32 basis the products, the
// updates and each thread's dot sums are FP32; block partials, Hessenberg
// columns, rotations and least-squares solutions stay FP64.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.h"

namespace ifeast {

namespace {

// Complex storage and arithmetic of the basis: double2 (FP64) or float2 (FP32).
template <typename CT>
struct Cx;
template <>
struct Cx<double2> {
  using R = double;
  __device__ static double2 make(double a, double b) { return make_double2(a, b); }
  __device__ static double fm(double a, double b, double c) { return fma(a, b, c); }
};
template <>
struct Cx<float2> {
  using R = float;
  __device__ static float2 make(float a, float b) { return make_float2(a, b); }
  __device__ static float fm(float a, float b, float c) { return fmaf(a, b, c); }
};

template <typename CT>
__device__ __forceinline__ CT cmul(CT a, CT b) {
  return Cx<CT>::make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += conj(a) * b
template <typename CT>
__device__ __forceinline__ void cjfma(CT &acc, CT a, CT b) {
  acc.x = Cx<CT>::fm(a.x, b.x, Cx<CT>::fm(a.y, b.y, acc.x));
  acc.y = Cx<CT>::fm(a.x, b.y, Cx<CT>::fm(-a.y, b.x, acc.y));
}
// acc -= h * v
template <typename CT>
__device__ __forceinline__ void cfms(CT &acc, CT h, CT v) {
  acc.x = Cx<CT>::fm(-h.x, v.x, Cx<CT>::fm(h.y, v.y, acc.x));
  acc.y = Cx<CT>::fm(-h.x, v.y, Cx<CT>::fm(-h.y, v.x, acc.y));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = cabs2(b);
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
template <typename CT>
__device__ __forceinline__ CT to_ct(double2 a) {
  using R = typename Cx<CT>::R;
  return Cx<CT>::make((R)a.x, (R)a.y);
}

// W = z_{node(c)} B V_s - A V_s on every active column (the first-pass dots
// follow in k_dots). CT: complex type of the basis (the arithmetic is done in
// its precision). BM: B = I (0), B with a pattern of its
// own (1), or B on A's pattern (2: one gather of V serves both products, valB
// indexed like val). A row's non-zeros are taken in groups of kNG: the group's
// indices and values are loaded together, then its gathers are issued before
// they are used, so that kNG loads per warp are in flight.
constexpr int kNG = 8;

template <typename CT, int BM>
__global__ void __launch_bounds__(kThreads)
k_spmm_shift(int n, int C, int m0, const int32_t *__restrict__ rowptr,
             const int32_t *__restrict__ colidx, const typename Cx<CT>::R *__restrict__ val,
             const CT *__restrict__ Vs, const double2 *__restrict__ z,
             const int *__restrict__ done, CT *__restrict__ W, int rows,
             const int32_t *__restrict__ rowptrB, const int32_t *__restrict__ colidxB,
             const typename Cx<CT>::R *__restrict__ valB) {
  using R = typename Cx<CT>::R;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const bool active = c < C && (done == nullptr || done[c] == 0);
  const CT zc = (c < C) ? to_ct<CT>(z[c / m0]) : Cx<CT>::make(0, 0);
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  const CT zero = Cx<CT>::make(0, 0);
  if (active) {
    for (int r = r0 + warp; r < r1; r += kWarps) {
      const size_t rc = (size_t)r * C + c;
      CT bv = BM == 0 ? Vs[rc] : zero;  // (B V_s)[r]
      CT av = zero;                      // (A V_s)[r]
      if (BM == 1) {
        const int qb = rowptrB[r], qe = rowptrB[r + 1];
        for (int q0 = qb; q0 < qe; q0 += kNG) {
          int cb[kNG];
          R b[kNG];
#pragma unroll
          for (int u = 0; u < kNG; ++u) {
            const bool in = q0 + u < qe;
            cb[u] = in ? colidxB[q0 + u] : r;
            b[u] = in ? valB[q0 + u] : R(0);
          }
          CT v[kNG];
#pragma unroll
          for (int u = 0; u < kNG; ++u) v[u] = q0 + u < qe ? Vs[(size_t)cb[u] * C + c] : zero;
#pragma unroll
          for (int u = 0; u < kNG; ++u) {
            bv.x = Cx<CT>::fm(b[u], v[u].x, bv.x);
            bv.y = Cx<CT>::fm(b[u], v[u].y, bv.y);
          }
        }
      }
      const int jb = rowptr[r], je = rowptr[r + 1];
      for (int j0 = jb; j0 < je; j0 += kNG) {
        int cj[kNG];
        R a[kNG], b[kNG];
#pragma unroll
        for (int u = 0; u < kNG; ++u) {
          const bool in = j0 + u < je;
          cj[u] = in ? colidx[j0 + u] : r;
          a[u] = in ? val[j0 + u] : R(0);
          if (BM == 2) b[u] = in ? valB[j0 + u] : R(0);
        }
        CT v[kNG];
#pragma unroll
        for (int u = 0; u < kNG; ++u) v[u] = j0 + u < je ? Vs[(size_t)cj[u] * C + c] : zero;
#pragma unroll
        for (int u = 0; u < kNG; ++u) {
          av.x = Cx<CT>::fm(a[u], v[u].x, av.x);
          av.y = Cx<CT>::fm(a[u], v[u].y, av.y);
          if (BM == 2) {
            bv.x = Cx<CT>::fm(b[u], v[u].x, bv.x);
            bv.y = Cx<CT>::fm(b[u], v[u].y, bv.y);
          }
        }
      }
      CT w = cmul(zc, bv);
      w.x -= av.x;
      w.y -= av.y;
      W[rc] = w;
    }
  }
}

// Block partials of h1_l = <V_l, W> for l in chunk blockIdx.z (l = 8 z ..
// 8 z + 7, l <= s), for the columns still running: the first Gram-Schmidt
// pass's coefficients. They run in their own kernel, in chunks of 8 basis
// vectors, so that each thread holds 8 accumulators instead of s + 1 and many
// blocks stay resident (the kernel streams the basis: its speed is the number
// of loads in flight), and so that the SpMM's gathers run at full occupancy.
constexpr int kDotChunk = 8;

template <typename CT>
__global__ void __launch_bounds__(kThreads)
k_dots(int n, int C, const CT *__restrict__ V, size_t vstride, int s,
       const int *__restrict__ done, const CT *__restrict__ W, double2 *__restrict__ part,
       int rows, int K2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const int l0 = blockIdx.z * kDotChunk;
  const bool active = c < C && done[c] == 0;
  CT acc[kDotChunk];
#pragma unroll
  for (int l = 0; l < kDotChunk; ++l) acc[l] = Cx<CT>::make(0, 0);
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  const CT *__restrict__ Vc = V + (size_t)l0 * vstride;
  if (active) {
    for (int r = r0 + warp; r < r1; r += kWarps) {
      const size_t rc = (size_t)r * C + c;
      const CT w = W[rc];
#pragma unroll
      for (int l = 0; l < kDotChunk; ++l)
        if (l0 + l <= s) cjfma(acc[l], Vc[(size_t)l * vstride + rc], w);
    }
  }
  // fixed-order block sums (warp order) in FP64, one slot at a time
  __shared__ double2 red[kWarps][32];
#pragma unroll
  for (int l = 0; l < kDotChunk; ++l) {
    if (l0 + l <= s) {  // uniform over the block
      red[warp][lane] = make_double2((double)acc[l].x, (double)acc[l].y);
      __syncthreads();
      if (warp == 0) {
        double2 t = red[0][lane];
#pragma unroll
        for (int q = 1; q < kWarps; ++q) t = cadd(t, red[q][lane]);
        if (c < C) part[((size_t)blockIdx.x * K2 + l0 + l) * C + c] = t;
      }
      __syncthreads();
    }
  }
}

// out[l * C + c] = sum over blocks b (in order) of part[(b * K2 + l) * C + c].
// Grid (nl, tiles); warp w sums blocks w, w+8, ...; the 8 warp sums are then
// added in warp order.
__global__ void __launch_bounds__(kThreads)
k_reduce_partials(int P, int C, int K2, const double2 *__restrict__ part,
                  double2 *__restrict__ out) {
  __shared__ double2 red[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int l = blockIdx.x;
  const int c = blockIdx.y * 32 + lane;
  double2 t = make_double2(0.0, 0.0);
  if (c < C)
    for (int b = warp; b < P; b += kWarps) t = cadd(t, part[((size_t)b * K2 + l) * C + c]);
  red[warp][lane] = t;
  __syncthreads();
  if (warp == 0 && c < C) {
    double2 u = red[0][lane];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) u = cadd(u, red[w][lane]);
    out[(size_t)l * C + c] = u;
  }
}

// First Gram-Schmidt pass: W -= sum_l h1_l V_l, then partials of h2_l =
// <V_l, W> (l <= s) and of ||W||^2 (stored as the real part of slot s+1).
template <int LMAX, typename CT>
__global__ void __launch_bounds__(kThreads)
k_orth_update_dot(int n, int C, const CT *__restrict__ V, size_t vstride, int s,
                  const double2 *__restrict__ H1, const int *__restrict__ done,
                  CT *__restrict__ W, double2 *__restrict__ part, int rows, int K2) {
  using R = typename Cx<CT>::R;
  __shared__ CT hs[LMAX][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const bool active = c < C && done[c] == 0;
  for (int l = warp; l <= s; l += kWarps)
    hs[l][lane] = (c < C) ? to_ct<CT>(H1[(size_t)l * C + c]) : Cx<CT>::make(0, 0);
  __syncthreads();
  CT acc[LMAX + 1];
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) acc[l] = Cx<CT>::make(0, 0);
  R nrm = 0;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  if (active) {
    for (int r = r0 + warp; r < r1; r += kWarps) {
      const size_t rc = (size_t)r * C + c;
      CT w = W[rc];
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l <= s) cfms(w, hs[l][lane], V[(size_t)l * vstride + rc]);
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l <= s) cjfma(acc[l], V[(size_t)l * vstride + rc], w);
      nrm = Cx<CT>::fm(w.x, w.x, Cx<CT>::fm(w.y, w.y, nrm));
      W[rc] = w;
    }
  }
  // store h2 partials (l <= s) and the norm partial in slot s + 1
  __shared__ double2 red[kWarps][32];
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    if (l <= s + 1) {
      red[warp][lane] = (l == s + 1) ? make_double2((double)nrm, 0.0)
                                     : make_double2((double)acc[l].x, (double)acc[l].y);
      __syncthreads();
      if (warp == 0) {
        double2 t = red[0][lane];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) t = cadd(t, red[w][lane]);
        if (c < C) part[((size_t)blockIdx.x * K2 + l) * C + c] = t;
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 basis kernels streamed through shared memory by TMA (the dots, the
// first Gram-Schmidt pass with its dots, and the finish). The arithmetic and
// its order per (row, column) are those of k_dots, k_orth_update_dot and
// k_orth_finish above; only the way the basis reaches the threads differs.
// A block owns the rows [r0, r1) of one 32-column tile; the rows go in stages
// of kTmaRows (one per warp), and for every stage one thread issues one 2D
// tile copy (kTmaRows rows x 32 complex columns, 2 kB) per basis vector and one
// for W, completing on the stage's mbarrier. Two stages are in flight, so the
// loads in flight no longer occupy registers: up to 2 x 33 x 2 kB per block.
// Every wait is bounded: a wait that runs out sets status->tc_timeout, the
// block waits (bounded) for its own copies still in flight and returns, and
// the host reports IFEAST_ERR_TIMEOUT.
constexpr int kTmaRows = kWarps;            // rows per stage: one per warp
constexpr int kTmaTileBytes = kTmaRows * 32 * 8;
constexpr long kTmaSpin = 1L << 24;

enum { kStreamDots = 0, kStreamUpdate = 1, kStreamFinish = 2 };

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity) {
  for (long it = 0; it < kTmaSpin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Issue the copies of stage st (rows r0 + st * kTmaRows ..) into buffer buf:
// vectors l0 .. l0 + nl - 1 of V, then W. Rows past n are filled with zeros.
__device__ __forceinline__ void issue_stage(const CUtensorMap *mapV, const CUtensorMap *mapW,
                                            float2 *buf, uint64_t *mbar, int tile, int row,
                                            int l0, int nl) {
  const uint32_t bytes = (uint32_t)(nl + 1) * kTmaTileBytes;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)),
               "r"(bytes)
               : "memory");
  const int x = 64 * tile;  // in floats: 32 complex columns = 256 bytes
  for (int l = 0; l < nl; ++l)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(buf + (size_t)l * kTmaRows * 32)),
        "l"(mapV), "r"(x), "r"(row), "r"(l0 + l), "r"(smem_addr(mbar))
        : "memory");
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(buf + (size_t)nl * kTmaRows * 32)),
      "l"(mapW), "r"(x), "r"(row), "r"(smem_addr(mbar))
      : "memory");
}

// MODE kStreamDots: partials of <V_l, W> for l = l0 .. l0 + 7 (<= s), like k_dots.
// MODE kStreamUpdate: W -= sum_l H[l] V_l, partials of <V_l, W> and ||W||^2,
// like k_orth_update_dot. MODE kStreamFinish: V_{s+1} = (W - sum_l H[l] V_l) *
// inv_h, like k_orth_finish.
template <int MODE, int LMAX>
__global__ void __launch_bounds__(kThreads)
k_gm_stream(const __grid_constant__ CUtensorMap mapV, const __grid_constant__ CUtensorMap mapW,
            int n, int C, int s, const double2 *__restrict__ H, const double *__restrict__ inv_h,
            const int *__restrict__ done, float2 *__restrict__ W, float2 *__restrict__ Vn,
            double2 *__restrict__ part, int rows, int K2, DevStatus *__restrict__ status) {
  constexpr int NACC = MODE == kStreamDots ? kDotChunk : LMAX + 1;
  extern __shared__ __align__(128) unsigned char gm_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ float2 hs[LMAX][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.y;
  const int c = tile * 32 + lane;
  const int l0 = MODE == kStreamDots ? blockIdx.z * kDotChunk : 0;
  const int nl = MODE == kStreamDots ? min(kDotChunk, s + 1 - l0) : s + 1;
  const size_t stage_elems = (size_t)(nl + 1) * kTmaRows * 32;
  float2 *sbuf = reinterpret_cast<float2 *>(gm_smem);
  const bool active = c < C && done[c] == 0;
  if (MODE != kStreamDots)
    for (int l = warp; l <= s; l += kWarps)
      hs[l][lane] = (c < C) ? make_float2((float)H[(size_t)l * C + c].x,
                                          (float)H[(size_t)l * C + c].y)
                            : make_float2(0.f, 0.f);
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  const int nst = r1 > r0 ? (r1 - r0 + kTmaRows - 1) / kTmaRows : 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&mbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int st = 0; st < 2 && st < nst; ++st)
      issue_stage(&mapV, &mapW, sbuf + st * stage_elems, &mbar[st], tile, r0 + st * kTmaRows, l0,
                  nl);
  }
  __syncthreads();
  float2 acc[NACC];
#pragma unroll
  for (int l = 0; l < NACC; ++l) acc[l] = make_float2(0.f, 0.f);
  float nrm = 0.f;
  bool fail = false;
  const float ih = (MODE == kStreamFinish && c < C) ? (float)inv_h[c] : 0.f;
  float2 *Vnext = MODE == kStreamFinish ? Vn : nullptr;
  int st = 0;
  for (; st < nst; ++st) {
    const int b = st & 1;
    const bool ok = mbar_wait_bounded(&mbar[b], (uint32_t)((st >> 1) & 1));
    fail = __syncthreads_or(!ok) != 0;
    if (fail) break;
    const float2 *buf = sbuf + b * stage_elems;
    const int r = r0 + st * kTmaRows + warp;
    if (active && r < r1) {
      const size_t rc = (size_t)r * C + c;
      const float2 *vrow = buf + (size_t)warp * 32 + lane;  // vector l at vrow[l * kTmaRows * 32]
      float2 w = buf[(size_t)nl * kTmaRows * 32 + warp * 32 + lane];
      if (MODE == kStreamDots) {
#pragma unroll
        for (int l = 0; l < kDotChunk; ++l)
          if (l < nl) cjfma(acc[l], vrow[(size_t)l * kTmaRows * 32], w);
      } else {
#pragma unroll
        for (int l = 0; l < LMAX; ++l)
          if (l <= s) cfms(w, hs[l][lane], vrow[(size_t)l * kTmaRows * 32]);
        if (MODE == kStreamUpdate) {
#pragma unroll
          for (int l = 0; l < LMAX; ++l)
            if (l <= s) cjfma(acc[l], vrow[(size_t)l * kTmaRows * 32], w);
          nrm = fmaf(w.x, w.x, fmaf(w.y, w.y, nrm));
          W[rc] = w;
        } else {
          Vnext[rc] = make_float2(w.x * ih, w.y * ih);
        }
      }
    }
    __syncthreads();  // every thread is done with buffer b
    if (threadIdx.x == 0 && st + 2 < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_stage(&mapV, &mapW, sbuf + b * stage_elems, &mbar[b], tile,
                  r0 + (st + 2) * kTmaRows, l0, nl);
    }
  }
  if (fail) {
    if (threadIdx.x == 0) {
      atomicExch(&status->tc_timeout, 1);
      // the copies of stages st and st + 1 may still be in flight
      for (int q = st; q < st + 2 && q < nst; ++q)
        mbar_wait_bounded(&mbar[q & 1], (uint32_t)((q >> 1) & 1));
    }
    __syncthreads();
    return;
  }
  if (MODE == kStreamFinish) return;
  // fixed-order block sums (warp order) in FP64, one slot at a time
  __shared__ double2 red[kWarps][32];
  const int nslots = MODE == kStreamDots ? nl : s + 2;
#pragma unroll
  for (int l = 0; l < NACC + (MODE == kStreamUpdate ? 1 : 0); ++l) {
    if (l < nslots) {  // uniform over the block
      if (MODE == kStreamUpdate && l == s + 1)
        red[warp][lane] = make_double2((double)nrm, 0.0);
      else
        red[warp][lane] = make_double2((double)acc[l < NACC ? l : 0].x,
                                       (double)acc[l < NACC ? l : 0].y);
      __syncthreads();
      if (warp == 0) {
        double2 t = red[0][lane];
#pragma unroll
        for (int q = 1; q < kWarps; ++q) t = cadd(t, red[q][lane]);
        if (c < C) part[((size_t)blockIdx.x * K2 + l0 + l) * C + c] = t;
      }
      __syncthreads();
    }
  }
}

// Per system c: Hessenberg column h_{l,s} = h1_l + h2_l, h_{s+1,s} from
// Pythagoras, previous Givens rotations, new rotation, rotated right-hand side
// and the stop test |g_{s+1}| <= tolc[c]. h_{s+1,s} <= brk * ||b|| is a
// breakdown (the Krylov space is invariant to the basis precision).
__global__ void k_givens(int C, int m0, int K, int s, const double2 *__restrict__ H1,
                         const double2 *__restrict__ H2, const double *__restrict__ beta,
                         const double *__restrict__ tolc, double brk,
                         double *__restrict__ inv_h, double2 *__restrict__ CS,
                         double2 *__restrict__ SN, double2 *__restrict__ R,
                         double2 *__restrict__ G, int *__restrict__ steps, int *__restrict__ done) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  if (done[c]) {
    inv_h[c] = 0.0;
    return;
  }
  double2 hcol[kMaxInner + 1];
  double sum2 = 0.0;
  for (int l = 0; l <= s; ++l) {
    const double2 h2 = H2[(size_t)l * C + c];
    hcol[l] = cadd(H1[(size_t)l * C + c], h2);
    sum2 += cabs2(h2);
  }
  const double nrm1 = H2[(size_t)(s + 1) * C + c].x;
  const double hs = sqrt(fmax(nrm1 - sum2, 0.0));
  const double b = beta[c % m0];
  const bool happy = !(hs > brk * b);
  inv_h[c] = happy ? 0.0 : 1.0 / hs;
  // apply the rotations of steps 0..s-1 (G_l = [[conj cs, conj sn], [-sn, cs]])
  for (int l = 0; l < s; ++l) {
    const double2 cs = CS[(size_t)l * C + c], sn = SN[(size_t)l * C + c];
    const double2 a = hcol[l], bb = hcol[l + 1];
    double2 t0, t1;
    t0.x = cs.x * a.x + cs.y * a.y + sn.x * bb.x + sn.y * bb.y;
    t0.y = cs.x * a.y - cs.y * a.x + sn.x * bb.y - sn.y * bb.x;
    const double2 sa = cmul(sn, a), cb = cmul(cs, bb);
    t1 = make_double2(cb.x - sa.x, cb.y - sa.y);
    hcol[l] = t0;
    hcol[l + 1] = t1;
  }
  const double rho = hypot(sqrt(cabs2(hcol[s])), hs);
  if (!(rho > 0.0)) {  // singular least-squares column: keep the s steps taken
    done[c] = 1;
    inv_h[c] = 0.0;
    return;
  }
  const double2 cs = make_double2(hcol[s].x / rho, hcol[s].y / rho);
  const double2 sn = make_double2(hs / rho, 0.0);
  for (int l = 0; l < s; ++l) R[((size_t)l * K + s) * C + c] = hcol[l];
  R[((size_t)s * K + s) * C + c] = make_double2(rho, 0.0);
  const double2 gs = G[(size_t)s * C + c];
  const double2 sg = cmul(sn, gs);
  G[(size_t)(s + 1) * C + c] = make_double2(-sg.x, -sg.y);
  G[(size_t)s * C + c] = make_double2(cs.x * gs.x + cs.y * gs.y, cs.x * gs.y - cs.y * gs.x);
  CS[(size_t)s * C + c] = cs;
  SN[(size_t)s * C + c] = sn;
  steps[c] = s + 1;
  const double res = sqrt(cabs2(G[(size_t)(s + 1) * C + c]));
  const double tol = tolc[c];
  if (happy || (tol > 0.0 && res <= tol)) done[c] = 1;
}

// V_{s+1} = (W - sum_l h2_l V_l) * inv_h on systems still running.
template <int LMAX, typename CT>
__global__ void __launch_bounds__(kThreads)
k_orth_finish(int n, int C, CT *__restrict__ V, size_t vstride, int s,
              const double2 *__restrict__ H2, const double *__restrict__ inv_h,
              const int *__restrict__ done, const CT *__restrict__ W, int rows) {
  using R = typename Cx<CT>::R;
  __shared__ CT hs[LMAX][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  for (int l = warp; l <= s; l += kWarps)
    hs[l][lane] = (c < C) ? to_ct<CT>(H2[(size_t)l * C + c]) : Cx<CT>::make(0, 0);
  __syncthreads();
  if (c >= C || done[c]) return;
  const R ih = (R)inv_h[c];
  CT *__restrict__ Vn = V + (size_t)(s + 1) * vstride;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int r = r0 + warp; r < r1; r += kWarps) {
    const size_t rc = (size_t)r * C + c;
    CT w = W[rc];
#pragma unroll
    for (int l = 0; l < LMAX; ++l)
      if (l <= s) cfms(w, hs[l][lane], V[(size_t)l * vstride + rc]);
    Vn[rc] = Cx<CT>::make(w.x * ih, w.y * ih);
  }
}

// V_0[:, k*m0 + j] = b_j / ||b_j|| for all nodes k (b = X, B X, or the
// residuals); least-squares state reset and the per-system bound on the
// least-squares residual: tol_rel ||b_j||, or in the residual form
// tol_rel ||B x_j|| |z_k - lambda_j| (the same bound on the original system,
// whose residual is the correction's divided by |z_k - lambda_j|).
template <typename CT>
__global__ void k_prep(int n, int m0, int C, int K, const double *__restrict__ X,
                       const double *__restrict__ beta, CT *__restrict__ V0,
                       double2 *__restrict__ G, int *__restrict__ steps, int *__restrict__ done,
                       double *__restrict__ tolc, const DevStatus *__restrict__ status,
                       const double2 *__restrict__ z, const double *__restrict__ lam,
                       const double *__restrict__ xnorm, int correction) {
  using R = typename Cx<CT>::R;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)n * C;
  if (idx < total) {
    const int r = (int)(idx / C), c = (int)(idx % C), j = c % m0;
    const double b = beta[j];
    V0[idx] = Cx<CT>::make((R)(b > 0.0 ? X[(size_t)r * m0 + j] / b : 0.0), 0);
  }
  if (idx < (size_t)C) {
    const int c = (int)idx, j = c % m0, k = c / m0;
    const double b = beta[j];
    G[c] = make_double2(b, 0.0);
    for (int l = 1; l <= K; ++l) G[(size_t)l * C + c] = make_double2(0.0, 0.0);
    steps[c] = 0;
    done[c] = (b > 0.0) ? 0 : 1;
    const double tol_rel = status->tol_rel;
    double t = 0.0;
    if (tol_rel > 0.0) {
      if (correction == 1) {
        const double2 d = make_double2(z[k].x - lam[j], z[k].y);
        t = tol_rel * xnorm[j] * sqrt(cabs2(d));
      } else if (correction == 2) {
        t = tol_rel;  // Alg. 2's bound tol_rel ||x_j|| with ||x_j|| = 1
      } else {
        t = tol_rel * b;
      }
    }
    tolc[c] = t;
  }
}

// y = R^{-1} g for each system (back substitution over its steps), scaled by
// the system's weight: Y[l][c] = w_k y_l, or w_k / (z_k - lambda_j) y_l in the
// residual form (Yf: the same in FP32 for the FP32 quadrature); cx[j] = Re
// sum_k w_k / (z_k - lambda_j) (residual form) or 0. Step counts are folded
// into the status record with integer atomics (order-independent).
__global__ void k_solve_y(int C, int m0, int nc, int K, const double2 *__restrict__ R,
                          const double2 *__restrict__ G, const double2 *__restrict__ wq,
                          const double2 *__restrict__ z, const double *__restrict__ lam,
                          int correction, const int *__restrict__ steps,
                          double2 *__restrict__ Y, float2 *__restrict__ Yf,
                          double *__restrict__ cx, DevStatus *__restrict__ status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int m = steps[c];
  double2 y[kMaxInner];
  for (int l = m - 1; l >= 0; --l) {
    double2 t = G[(size_t)l * C + c];
    for (int q = l + 1; q < m; ++q) {
      const double2 p = cmul(R[((size_t)l * K + q) * C + c], y[q]);
      t.x -= p.x;
      t.y -= p.y;
    }
    const double2 d = R[((size_t)l * K + l) * C + c];
    const double dd = cabs2(d);
    y[l] = make_double2((t.x * d.x + t.y * d.y) / dd, (t.y * d.x - t.x * d.y) / dd);
  }
  const int k = c / m0, j = c % m0;
  double2 wk = wq[k];
  if (correction == 1) wk = cdiv(wk, make_double2(z[k].x - lam[j], z[k].y));
  for (int l = 0; l < K; ++l) {
    const double2 v = (l < m) ? cmul(wk, y[l]) : make_double2(0.0, 0.0);
    Y[(size_t)l * C + c] = v;
    if (Yf) Yf[(size_t)l * C + c] = make_float2((float)v.x, (float)v.y);
  }
  if (cx && c < m0) {
    double t = 0.0;
    if (correction == 1)
      for (int kk = 0; kk < nc; ++kk)
        t += cdiv(wq[kk], make_double2(z[kk].x - lam[c], z[kk].y)).x;
    cx[c] = t;
  }
  atomicMax(&status->max_steps, m);
  atomicAdd((unsigned long long *)&status->total_steps, (unsigned long long)m);
}

// Q[r][j] = cx[j] X[r][j] + Re sum_k sum_{l < steps} Y[l][k*m0 + j] V_l[r][k*m0 + j]
// (cx null: no first term). FP64 basis: FP64 sums of the FP64 coefficients;
// FP32 basis: FP32 sums of the FP32 coefficients.
template <typename CT>
__global__ void k_quadrature(int n, int m0, int nc, int C, const CT *__restrict__ V,
                             size_t vstride, const double2 *__restrict__ Y,
                             const float2 *__restrict__ Yf, const int *__restrict__ steps,
                             const double *__restrict__ cx, const double *__restrict__ Xr,
                             double *__restrict__ Q, int accumulate) {
  using R = typename Cx<CT>::R;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * m0) return;
  const int r = (int)(idx / m0), j = (int)(idx % m0);
  R q = 0;
  for (int k = 0; k < nc; ++k) {
    const int c = k * m0 + j;
    const int m = steps[c];
    const size_t rc = (size_t)r * C + c;
    for (int l = 0; l < m; ++l) {
      CT yw;
      if constexpr (sizeof(R) == 8) {
        yw = Y[(size_t)l * C + c];
      } else {
        yw = Yf[(size_t)l * C + c];
      }
      const CT v = V[(size_t)l * vstride + rc];
      q = Cx<CT>::fm(yw.x, v.x, Cx<CT>::fm(-yw.y, v.y, q));
    }
  }
  const double t = cx ? cx[j] * Xr[idx] + (double)q : (double)q;
  Q[idx] = accumulate ? Q[idx] + t : t;  // later node chunks add their part
}

// Block correction for non-symmetric A (FP64 basis): E[r][c] = sum_{l <
// steps[c]} Y[l][c] V_l[r][c], the weighted solution w_k e of system c = (node
// k, column j) on row r.
__global__ void k_ns_solutions(int n, int C, const double2 *__restrict__ V, size_t vstride,
                               const double2 *__restrict__ Y, const int *__restrict__ steps,
                               double2 *__restrict__ E) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * C) return;
  const int c = (int)(idx % C);
  const int m = steps[c];
  double2 acc = make_double2(0.0, 0.0);
  for (int l = 0; l < m; ++l) {
    const double2 y = Y[(size_t)l * C + c], v = V[(size_t)l * vstride + idx];
    acc.x = fma(y.x, v.x, fma(-y.y, v.y, acc.x));
    acc.y = fma(y.x, v.y, fma(y.y, v.x, acc.y));
  }
  E[idx] = acc;
}

// Q = X Gre + Re(E M) (add_x = 0: without the first term; accumulate: Q +=),
// X n x m0 real, Gre m0 x m0, E n x C complex, M C x m0 complex (row c =
// k m0 + j holds row j of M_k). A block computes 32 rows x m0 columns: thread
// (i, ty) owns column i of rows ty, ty + 4, ...; chunks of 16 contraction
// indices of E and M are staged in shared memory.
constexpr int kNsRows = 32;
constexpr int kNsChunk = 16;
__global__ void __launch_bounds__(256)
k_ns_combine(int n, int m0, int C, const double *__restrict__ X, const double *__restrict__ Gre,
             const double2 *__restrict__ E, const double2 *__restrict__ M, int add_x,
             int accumulate, double *__restrict__ Q) {
  __shared__ double2 sE[kNsRows][kNsChunk + 1];
  __shared__ double2 sM[kNsChunk][64];
  const int i = threadIdx.x, ty = threadIdx.y;  // blockDim (64, 4)
  const int r0 = blockIdx.x * kNsRows;
  const int tid = ty * 64 + i;
  double acc[kNsRows / 4];
#pragma unroll
  for (int u = 0; u < kNsRows / 4; ++u) acc[u] = 0.0;
  // Re(E M) = E.x M.x - E.y M.y
  for (int c0 = 0; c0 < C; c0 += kNsChunk) {
    for (int e = tid; e < kNsRows * kNsChunk; e += 256) {
      const int rr = e / kNsChunk, cc = e % kNsChunk;
      const int r = r0 + rr, c = c0 + cc;
      sE[rr][cc] = (r < n && c < C) ? E[(size_t)r * C + c] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < kNsChunk * 64; e += 256) {
      const int cc = e / 64, ii = e % 64;
      const int c = c0 + cc;
      sM[cc][ii] = (c < C && ii < m0) ? M[(size_t)c * m0 + ii] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int cc = 0; cc < kNsChunk; ++cc) {
      const double2 mm = sM[cc][i];
#pragma unroll
      for (int u = 0; u < kNsRows / 4; ++u) {
        const double2 ee = sE[ty + 4 * u][cc];
        acc[u] = fma(ee.x, mm.x, fma(-ee.y, mm.y, acc[u]));
      }
    }
    __syncthreads();
  }
  if (i >= m0) return;
#pragma unroll
  for (int u = 0; u < kNsRows / 4; ++u) {
    const int r = r0 + ty + 4 * u;
    if (r >= n) continue;
    double t = acc[u];
    if (add_x)
      for (int j = 0; j < m0; ++j) t = fma(X[(size_t)r * m0 + j], Gre[(size_t)j * m0 + i], t);
    const size_t o = (size_t)r * m0 + i;
    Q[o] = accumulate ? Q[o] + t : t;
  }
}

// Tensor maps of the FP32 basis (a 3D view: 2C floats x n rows x K+1 vectors)
// and of W (2C floats x n rows), boxes of 64 floats x kTmaRows rows.
struct TmaMaps {
  CUtensorMap V, W;
};

PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// The streamed kernels need the FP32 basis, rows of 8 C bytes that are a
// multiple of 16 (C even), 16-byte aligned buffers and the encoder.
bool make_tma_maps(const GmresArgs &a, TmaMaps *m) {
  if (!a.fp32 || (a.C & 1) || a.n < 1) return false;
  if ((reinterpret_cast<uintptr_t>(a.V) | reinterpret_cast<uintptr_t>(a.W)) & 15) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
  if (!enc) return false;
  const cuuint64_t row_bytes = (cuuint64_t)a.C * 8;
  const cuuint64_t dimV[3] = {(cuuint64_t)a.C * 2, (cuuint64_t)a.n, (cuuint64_t)a.K + 1};
  const cuuint64_t strV[2] = {row_bytes, row_bytes * (cuuint64_t)a.n};
  const cuuint32_t boxV[3] = {64, (cuuint32_t)kTmaRows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  if (enc(&m->V, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.V, dimV, strV, boxV, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t dimW[2] = {(cuuint64_t)a.C * 2, (cuuint64_t)a.n};
  const cuuint64_t strW[1] = {row_bytes};
  const cuuint32_t boxW[2] = {64, (cuuint32_t)kTmaRows};
  return enc(&m->W, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, a.W, dimW, strW, boxW, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <int LMAX, typename CT>
cudaError_t launch_step(const GmresArgs &a, int s, cudaStream_t st, const TmaMaps *tma) {
  using R = typename Cx<CT>::R;
  const dim3 grid(a.tl.P, a.tl.tiles);
  const size_t vstride = (size_t)a.n * a.C;
  const int K2 = a.K + 2;
  CT *V = static_cast<CT *>(a.V);
  CT *W = static_cast<CT *>(a.W);
  const R *val, *valB;
  if constexpr (sizeof(R) == 8) {
    val = a.val;
    valB = a.valB;
  } else {
    val = a.val32;
    valB = a.valB32;
  }
  IFEAST_PROF_BEGIN(a.prof, K_GM_SPMM);
#define IFEAST_SPMM_LAUNCH(BM)                                                            \
  k_spmm_shift<CT, BM><<<grid, kThreads, 0, st>>>(a.n, a.C, a.m0, a.rowptr, a.colidx, val,   \
                                                  V + (size_t)s * vstride, a.z, a.done, W,  \
                                                  a.tl.rows, a.rowptrB, a.colidxB, valB)
  if (!a.rowptrB)
    IFEAST_SPMM_LAUNCH(0);
  else if (a.b_same_pattern)
    IFEAST_SPMM_LAUNCH(2);
  else
    IFEAST_SPMM_LAUNCH(1);
#undef IFEAST_SPMM_LAUNCH
  const dim3 gdots(a.tl.P, a.tl.tiles, (s + 1 + kDotChunk - 1) / kDotChunk);
  if constexpr (sizeof(R) == 4) {
    if (tma) {
      const size_t smem = 2 * (size_t)(kDotChunk + 1) * kTmaTileBytes;
      k_gm_stream<kStreamDots, 8><<<gdots, kThreads, smem, st>>>(
          tma->V, tma->W, a.n, a.C, s, nullptr, nullptr, a.done, nullptr, nullptr, a.part,
          a.tl.rows, K2, a.status);
    } else {
      k_dots<CT><<<gdots, kThreads, 0, st>>>(a.n, a.C, V, vstride, s, a.done, W, a.part,
                                             a.tl.rows, K2);
    }
  } else {
    k_dots<CT><<<gdots, kThreads, 0, st>>>(a.n, a.C, V, vstride, s, a.done, W, a.part,
                                           a.tl.rows, K2);
  }
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_REDUCE);
  k_reduce_partials<<<dim3(s + 1, a.tl.tiles), kThreads, 0, st>>>(a.tl.P, a.C, K2, a.part, a.H1);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_ORTH);
  bool streamed = false;
  if constexpr (sizeof(R) == 4) {
    if (tma) {
      const size_t smem = 2 * (size_t)(s + 2) * kTmaTileBytes;
      k_gm_stream<kStreamUpdate, LMAX><<<grid, kThreads, smem, st>>>(
          tma->V, tma->W, a.n, a.C, s, a.H1, nullptr, a.done, W, nullptr, a.part, a.tl.rows, K2,
          a.status);
      streamed = true;
    }
  }
  if (!streamed)
    k_orth_update_dot<LMAX, CT><<<grid, kThreads, 0, st>>>(a.n, a.C, V, vstride, s, a.H1,
                                                           a.done, W, a.part, a.tl.rows, K2);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_REDUCE);
  k_reduce_partials<<<dim3(s + 2, a.tl.tiles), kThreads, 0, st>>>(a.tl.P, a.C, K2, a.part, a.H2);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_GIVENS);
  // breakdown threshold: the basis precision's rounding level
  const double brk = sizeof(R) == 8 ? 1e-14 : 1e-6;
  k_givens<<<(a.C + 127) / 128, 128, 0, st>>>(a.C, a.m0, a.K, s, a.H1, a.H2, a.beta, a.tolc, brk,
                                              a.inv_h, a.CS, a.SN, a.R, a.G, a.steps, a.done);
  IFEAST_PROF_END(a.prof);
  if (s + 1 < a.K) {  // the last step's basis vector is never used
    IFEAST_PROF_BEGIN(a.prof, K_GM_FINISH);
    bool fstreamed = false;
    if constexpr (sizeof(R) == 4) {
      if (tma) {
        const size_t smem = 2 * (size_t)(s + 2) * kTmaTileBytes;
        k_gm_stream<kStreamFinish, LMAX><<<grid, kThreads, smem, st>>>(
            tma->V, tma->W, a.n, a.C, s, a.H2, a.inv_h, a.done, nullptr,
            V + (size_t)(s + 1) * vstride, nullptr, a.tl.rows, K2, a.status);
        fstreamed = true;
      }
    }
    if (!fstreamed)
      k_orth_finish<LMAX, CT><<<grid, kThreads, 0, st>>>(a.n, a.C, V, vstride, s, a.H2,
                                                         a.inv_h, a.done, W, a.tl.rows);
    IFEAST_PROF_END(a.prof);
  }
  return cudaGetLastError();
}

template <typename CT>
cudaError_t run_gmres(const GmresArgs &a, cudaStream_t st, const TmaMaps *tma) {
  const size_t total = (size_t)a.n * a.C;
  CT *V = static_cast<CT *>(a.V);
  IFEAST_PROF_BEGIN(a.prof, K_PREP);
  k_prep<CT><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
      a.n, a.m0, a.C, a.K, a.X, a.beta, V, a.G, a.steps, a.done, a.tolc, a.status, a.z,
      a.correction ? a.lam : nullptr, a.correction ? a.xnorm : nullptr, a.correction);
  IFEAST_PROF_END(a.prof);
  cudaError_t e = cudaGetLastError();
  for (int s = 0; s < a.K && e == cudaSuccess; ++s) {
    if (s + 1 <= 8)
      e = launch_step<8, CT>(a, s, st, tma);
    else if (s + 1 <= 16)
      e = launch_step<16, CT>(a, s, st, tma);
    else
      e = launch_step<32, CT>(a, s, st, tma);
  }
  if (e != cudaSuccess) return e;
  IFEAST_PROF_BEGIN(a.prof, K_GM_SOLVE);
  k_solve_y<<<(a.C + 127) / 128, 128, 0, st>>>(
      a.C, a.m0, a.nc, a.K, a.R, a.G, a.w, a.z, a.correction == 1 ? a.lam : nullptr,
      a.correction, a.steps, a.Y, a.fp32 ? a.Yf : nullptr, a.correction == 1 ? a.cx : nullptr,
      a.status);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_QUAD);
  if constexpr (std::is_same_v<CT, double2>) {
    if (a.correction == 2) {  // block correction: E_k, then Q from M_k (the work vector holds E)
      const size_t nc_tot = (size_t)a.n * a.C;
      double2 *E = static_cast<double2 *>(a.W);
      k_ns_solutions<<<(unsigned)((nc_tot + 255) / 256), 256, 0, st>>>(
          a.n, a.C, V, (size_t)a.n * a.C, a.Y, a.steps, E);
      k_ns_combine<<<(unsigned)((a.n + kNsRows - 1) / kNsRows), dim3(64, 4), 0, st>>>(
          a.n, a.m0, a.C, a.ns_X, a.ns_Gre, E, a.ns_M, a.accumulate ? 0 : 1, a.accumulate, a.Q);
      IFEAST_PROF_END(a.prof);
      return cudaGetLastError();
    }
  }
  const size_t nq = (size_t)a.n * a.m0;
  k_quadrature<CT><<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(
      a.n, a.m0, a.nc, a.C, V, (size_t)a.n * a.C, a.Y, a.Yf, a.steps,
      a.correction ? a.cx : nullptr, a.Xr, a.Q, a.accumulate);
  IFEAST_PROF_END(a.prof);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gmres_init() {
  const int most = 2 * (kMaxInner + 1) * kTmaTileBytes;  // s + 2 <= kMaxInner + 1 tiles per stage
  cudaError_t e = cudaFuncSetAttribute(k_gm_stream<kStreamDots, 8>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * (kDotChunk + 1) * kTmaTileBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gm_stream<kStreamUpdate, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gm_stream<kStreamUpdate, 16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gm_stream<kStreamUpdate, 32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gm_stream<kStreamFinish, 8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gm_stream<kStreamFinish, 16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gm_stream<kStreamFinish, 32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, most);
  return e;
}

RowTiling make_tiling(int64_t n, int ncols, int num_sms) {
  RowTiling t;
  t.tiles = (ncols + 31) / 32;
  const int target = 4 * num_sms;
  int P = (target + t.tiles - 1) / t.tiles;
  const int64_t maxP = (n + kWarps - 1) / kWarps;
  if (P > maxP) P = (int)maxP;
  if (P < 1) P = 1;
  t.rows = (int)((n + P - 1) / P);
  t.P = (int)((n + t.rows - 1) / t.rows);
  if (t.P < 1) t.P = 1;
  return t;
}

cudaError_t gmres_filter(const GmresArgs &a, cudaStream_t st) {
  if (a.K < 1 || a.K > kMaxInner) return cudaErrorInvalidValue;
  if (a.correction == 1 && (!a.lam || !a.xnorm || !a.Xr || !a.cx)) return cudaErrorInvalidValue;
  if (a.correction == 2 && (a.fp32 || a.m0 > 64 || !a.ns_M || !a.ns_Gre || !a.ns_X))
    return cudaErrorInvalidValue;
  if (a.fp32 && (!a.val32 || !a.Yf || (a.rowptrB && !a.valB32))) return cudaErrorInvalidValue;
  if (a.ncc < 1 || a.nc % a.ncc != 0 || a.C != a.ncc * a.m0) return cudaErrorInvalidValue;
  // passes over chunks of ncc nodes: the same kernels on the chunk's nodes and
  // weights, each pass's step counts in its slice, Q summed over the passes
  // (the first pass writes it; cx of the residual form is summed likewise)
  // the basis and W buffers are the same for every pass: one pair of maps
  TmaMaps maps;
  const bool use_tma = a.stream_tma && make_tma_maps(a, &maps);
  cudaError_t e = cudaSuccess;
  for (int k0 = 0; k0 < a.nc && e == cudaSuccess; k0 += a.ncc) {
    GmresArgs b = a;
    b.nc = a.ncc;
    b.z = a.z + k0;
    b.w = a.w + k0;
    b.steps = a.steps + (size_t)k0 * a.m0;
    b.accumulate = k0 > 0 ? 1 : 0;
    if (a.ns_M) b.ns_M = a.ns_M + (size_t)k0 * a.m0 * a.m0;
    e = a.fp32 ? run_gmres<float2>(b, st, use_tma ? &maps : nullptr)
               : run_gmres<double2>(b, st, nullptr);
  }
  return e;
}

cudaError_t spmm_shift_only(int n, const int32_t *rowptr, const int32_t *colidx,
                            const double *val, const double2 *V, double2 *W, int ncols, int m0,
                            const double2 *z, RowTiling tl, cudaStream_t st,
                            const int32_t *rowptrB, const int32_t *colidxB, const double *valB) {
  if (rowptrB)
    k_spmm_shift<double2, 1><<<dim3(tl.P, tl.tiles), kThreads, 0, st>>>(
        n, ncols, m0, rowptr, colidx, val, V, z, nullptr, W, tl.rows, rowptrB, colidxB, valB);
  else
    k_spmm_shift<double2, 0><<<dim3(tl.P, tl.tiles), kThreads, 0, st>>>(
        n, ncols, m0, rowptr, colidx, val, V, z, nullptr, W, tl.rows, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace ifeast
