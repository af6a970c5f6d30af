// Inner solve of IFEAST (Algorithm 2, steps 1-2) on the GPU: for every contour
// node z_k and every column x_j of X, GMRES on (z_k I - A) y = x_j with zero
// initial guess (Section 2.2), all C = nc * m0 systems advanced together, then
// the quadrature sum Q = Re sum_k w_k Y_k.
//
// Data layout (all row-major, complex values interleaved as double2):
//   V[s]  n x C basis vector s of every system, column c = k * m0 + j
//   W     n x C work vector (A-product, then Gram-Schmidt in place)
// One Arnoldi step s runs five kernels:
//   spmm_shift_dot   W = z V_s - A V_s and block partials of h1_l = <V_l, W>
//   reduce           h1 (fixed-order sum of the block partials)
//   orth_update_dot  W -= sum_l h1_l V_l and partials of h2_l = <V_l, W>, ||W||^2
//   reduce           h2, ||W||^2
//   givens           h = h1 + h2, h_{s+1,s} = sqrt(||W||^2 - sum |h2_l|^2),
//                    Givens update of the least-squares problem, stop test
//   orth_finish      V_{s+1} = (W - sum_l h2_l V_l) / h_{s+1,s}
// (classical Gram-Schmidt applied twice; the norm after the second pass
// follows from the first-pass norm by Pythagoras because V_0..V_s are
// orthonormal.) Every reduction sums block partials in a fixed order, so the
// result does not depend on scheduling.
#include "internal.h"

namespace ifeast {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += conj(a) * b
__device__ __forceinline__ void cjfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
// acc -= h * v
__device__ __forceinline__ void cfms(double2 &acc, double2 h, double2 v) {
  acc.x = fma(-h.x, v.x, fma(h.y, v.y, acc.x));
  acc.y = fma(-h.x, v.y, fma(-h.y, v.x, acc.y));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Sums LMAX register accumulators of the 8 warps of a block (lane = column)
// and writes them as this block's partials part[(blk * K2 + l) * C + c], l <= s.
template <int LMAX>
__device__ __forceinline__ void block_store_partials(const double2 (&acc)[LMAX], int s, int C,
                                                     int c, int K2, double2 *__restrict__ part) {
  __shared__ double2 red[kWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int l = 0; l < LMAX; ++l) {
    if (l <= s) {  // s is uniform over the block
      red[warp][lane] = acc[l];
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

// W = z_{node(c)} B V_s - A V_s on every active column (B = I when rowptrB is
// null); with DOTS also the block partials of <V_l, W>, l = 0..s.
template <int LMAX, bool DOTS>
__global__ void __launch_bounds__(kThreads)
k_spmm_shift_dot(int n, int C, int m0, const int32_t *__restrict__ rowptr,
                 const int32_t *__restrict__ colidx, const double *__restrict__ val,
                 const double2 *__restrict__ V, size_t vstride, int s,
                 const double2 *__restrict__ z, const int *__restrict__ done,
                 double2 *__restrict__ W, double2 *__restrict__ part, int rows, int K2,
                 const int32_t *__restrict__ rowptrB, const int32_t *__restrict__ colidxB,
                 const double *__restrict__ valB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const bool active = c < C && (done == nullptr || done[c] == 0);
  const double2 zc = (c < C) ? z[c / m0] : make_double2(0.0, 0.0);
  const double2 *__restrict__ Vs = V + (size_t)s * vstride;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  double2 acc[LMAX];
#pragma unroll
  for (int l = 0; l < LMAX; ++l) acc[l] = make_double2(0.0, 0.0);
  if (active) {
    for (int r = r0 + warp; r < r1; r += kWarps) {
      const size_t rc = (size_t)r * C + c;
      double2 bv;
      if (rowptrB == nullptr) {
        bv = Vs[rc];
      } else {
        bv = make_double2(0.0, 0.0);
        const int qb = rowptrB[r], qe = rowptrB[r + 1];
#pragma unroll 4
        for (int q = qb; q < qe; ++q) {
          const double b = valB[q];
          const double2 v = Vs[(size_t)colidxB[q] * C + c];
          bv.x = fma(b, v.x, bv.x);
          bv.y = fma(b, v.y, bv.y);
        }
      }
      double2 w = cmul(zc, bv);
      const int jb = rowptr[r], je = rowptr[r + 1];
#pragma unroll 4
      for (int j = jb; j < je; ++j) {
        const double a = val[j];
        const double2 v = Vs[(size_t)colidx[j] * C + c];
        w.x = fma(-a, v.x, w.x);
        w.y = fma(-a, v.y, w.y);
      }
      W[rc] = w;
      if (DOTS) {
#pragma unroll
        for (int l = 0; l < LMAX; ++l)
          if (l <= s) cjfma(acc[l], V[(size_t)l * vstride + rc], w);
      }
    }
  }
  if (DOTS) block_store_partials<LMAX>(acc, s, C, c, K2, part);
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
template <int LMAX>
__global__ void __launch_bounds__(kThreads)
k_orth_update_dot(int n, int C, const double2 *__restrict__ V, size_t vstride, int s,
                  const double2 *__restrict__ H1, const int *__restrict__ done,
                  double2 *__restrict__ W, double2 *__restrict__ part, int rows, int K2) {
  __shared__ double2 hs[LMAX][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  const bool active = c < C && done[c] == 0;
  for (int l = warp; l <= s; l += kWarps)
    hs[l][lane] = (c < C) ? H1[(size_t)l * C + c] : make_double2(0.0, 0.0);
  __syncthreads();
  double2 acc[LMAX + 1];
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) acc[l] = make_double2(0.0, 0.0);
  double nrm = 0.0;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  if (active) {
    for (int r = r0 + warp; r < r1; r += kWarps) {
      const size_t rc = (size_t)r * C + c;
      double2 w = W[rc];
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l <= s) cfms(w, hs[l][lane], V[(size_t)l * vstride + rc]);
#pragma unroll
      for (int l = 0; l < LMAX; ++l)
        if (l <= s) cjfma(acc[l], V[(size_t)l * vstride + rc], w);
      nrm = fma(w.x, w.x, fma(w.y, w.y, nrm));
      W[rc] = w;
    }
  }
  // store h2 partials (l <= s) and the norm partial in slot s + 1
  __shared__ double2 red[kWarps][32];
#pragma unroll
  for (int l = 0; l <= LMAX; ++l) {
    if (l <= s + 1) {
      red[warp][lane] = (l == s + 1) ? make_double2(nrm, 0.0) : acc[l];
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

// Per system c: Hessenberg column h_{l,s} = h1_l + h2_l, h_{s+1,s} from
// Pythagoras, previous Givens rotations, new rotation, rotated right-hand side
// and the stop test |g_{s+1}| <= tol_rel * ||x_j||.
__global__ void k_givens(int C, int m0, int K, int s, const double2 *__restrict__ H1,
                         const double2 *__restrict__ H2, const double *__restrict__ beta,
                         double *__restrict__ inv_h, double2 *__restrict__ CS,
                         double2 *__restrict__ SN, double2 *__restrict__ R,
                         double2 *__restrict__ G, int *__restrict__ steps, int *__restrict__ done,
                         const DevStatus *__restrict__ status) {
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
  const bool happy = !(hs > 1e-14 * b);
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
  const double tol = status->tol_rel;
  if (happy || (tol > 0.0 && res <= tol * b)) done[c] = 1;
}

// V_{s+1} = (W - sum_l h2_l V_l) * inv_h on systems still running.
template <int LMAX>
__global__ void __launch_bounds__(kThreads)
k_orth_finish(int n, int C, double2 *__restrict__ V, size_t vstride, int s,
              const double2 *__restrict__ H2, const double *__restrict__ inv_h,
              const int *__restrict__ done, const double2 *__restrict__ W, int rows) {
  __shared__ double2 hs[LMAX][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * 32 + lane;
  for (int l = warp; l <= s; l += kWarps)
    hs[l][lane] = (c < C) ? H2[(size_t)l * C + c] : make_double2(0.0, 0.0);
  __syncthreads();
  if (c >= C || done[c]) return;
  const double ih = inv_h[c];
  double2 *__restrict__ Vn = V + (size_t)(s + 1) * vstride;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int r = r0 + warp; r < r1; r += kWarps) {
    const size_t rc = (size_t)r * C + c;
    double2 w = W[rc];
#pragma unroll
    for (int l = 0; l < LMAX; ++l)
      if (l <= s) cfms(w, hs[l][lane], V[(size_t)l * vstride + rc]);
    Vn[rc] = make_double2(w.x * ih, w.y * ih);
  }
}

// V_0[:, k*m0 + j] = x_j / ||x_j|| for all nodes k; least-squares state reset.
__global__ void k_prep(int n, int m0, int C, int K, const double *__restrict__ X,
                       const double *__restrict__ beta, double2 *__restrict__ V0,
                       double2 *__restrict__ G, int *__restrict__ steps, int *__restrict__ done) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)n * C;
  if (idx < total) {
    const int r = (int)(idx / C), c = (int)(idx % C), j = c % m0;
    const double b = beta[j];
    V0[idx] = make_double2(b > 0.0 ? X[(size_t)r * m0 + j] / b : 0.0, 0.0);
  }
  if (idx < (size_t)C) {
    const int c = (int)idx;
    const double b = beta[c % m0];
    G[c] = make_double2(b, 0.0);
    for (int l = 1; l <= K; ++l) G[(size_t)l * C + c] = make_double2(0.0, 0.0);
    steps[c] = 0;
    done[c] = (b > 0.0) ? 0 : 1;
  }
}

// y = R^{-1} g for each system (back substitution over its steps), scaled by
// the quadrature weight of its node: Y[l][c] = w_k * y_l. Step counts are
// folded into the status record with integer atomics (order-independent).
__global__ void k_solve_y(int C, int m0, int K, const double2 *__restrict__ R,
                          const double2 *__restrict__ G, const double2 *__restrict__ wq,
                          const int *__restrict__ steps, double2 *__restrict__ Y,
                          DevStatus *__restrict__ status) {
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
  const double2 wk = wq[c / m0];
  for (int l = 0; l < K; ++l)
    Y[(size_t)l * C + c] = (l < m) ? cmul(wk, y[l]) : make_double2(0.0, 0.0);
  atomicMax(&status->max_steps, m);
  atomicAdd((unsigned long long *)&status->total_steps, (unsigned long long)m);
}

// Q[r][j] = Re sum_k sum_{l < steps} (w_k y_{k,j,l}) V_l[r][k*m0 + j].
__global__ void k_quadrature(int n, int m0, int nc, int C, const double2 *__restrict__ V,
                             size_t vstride, const double2 *__restrict__ Y,
                             const int *__restrict__ steps, double *__restrict__ Q) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * m0) return;
  const int r = (int)(idx / m0), j = (int)(idx % m0);
  double q = 0.0;
  for (int k = 0; k < nc; ++k) {
    const int c = k * m0 + j;
    const int m = steps[c];
    const size_t rc = (size_t)r * C + c;
    for (int l = 0; l < m; ++l) {
      const double2 yw = Y[(size_t)l * C + c];
      const double2 v = V[(size_t)l * vstride + rc];
      q = fma(yw.x, v.x, fma(-yw.y, v.y, q));
    }
  }
  Q[idx] = q;
}

template <int LMAX>
cudaError_t launch_step(const GmresArgs &a, int s, cudaStream_t st) {
  const dim3 grid(a.tl.P, a.tl.tiles);
  const size_t vstride = (size_t)a.n * a.C;
  const int K2 = a.K + 2;
  IFEAST_PROF_BEGIN(a.prof, K_GM_SPMM);
  k_spmm_shift_dot<LMAX, true><<<grid, kThreads, 0, st>>>(
      a.n, a.C, a.m0, a.rowptr, a.colidx, a.val, a.V, vstride, s, a.z, a.done, a.W, a.part,
      a.tl.rows, K2, a.rowptrB, a.colidxB, a.valB);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_REDUCE);
  k_reduce_partials<<<dim3(s + 1, a.tl.tiles), kThreads, 0, st>>>(a.tl.P, a.C, K2, a.part, a.H1);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_ORTH);
  k_orth_update_dot<LMAX><<<grid, kThreads, 0, st>>>(a.n, a.C, a.V, vstride, s, a.H1, a.done,
                                                     a.W, a.part, a.tl.rows, K2);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_REDUCE);
  k_reduce_partials<<<dim3(s + 2, a.tl.tiles), kThreads, 0, st>>>(a.tl.P, a.C, K2, a.part, a.H2);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_GIVENS);
  k_givens<<<(a.C + 127) / 128, 128, 0, st>>>(a.C, a.m0, a.K, s, a.H1, a.H2, a.beta, a.inv_h,
                                              a.CS, a.SN, a.R, a.G, a.steps, a.done, a.status);
  IFEAST_PROF_END(a.prof);
  if (s + 1 < a.K) {  // the last step's basis vector is never used
    IFEAST_PROF_BEGIN(a.prof, K_GM_FINISH);
    k_orth_finish<LMAX><<<grid, kThreads, 0, st>>>(a.n, a.C, a.V, vstride, s, a.H2, a.inv_h,
                                                   a.done, a.W, a.tl.rows);
    IFEAST_PROF_END(a.prof);
  }
  return cudaGetLastError();
}

}  // namespace

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
  const size_t total = (size_t)a.n * a.C;
  IFEAST_PROF_BEGIN(a.prof, K_PREP);
  k_prep<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a.n, a.m0, a.C, a.K, a.X, a.beta, a.V,
                                                           a.G, a.steps, a.done);
  IFEAST_PROF_END(a.prof);
  cudaError_t e = cudaGetLastError();
  for (int s = 0; s < a.K && e == cudaSuccess; ++s) {
    if (s + 1 <= 8)
      e = launch_step<8>(a, s, st);
    else if (s + 1 <= 16)
      e = launch_step<16>(a, s, st);
    else
      e = launch_step<32>(a, s, st);
  }
  if (e != cudaSuccess) return e;
  IFEAST_PROF_BEGIN(a.prof, K_GM_SOLVE);
  k_solve_y<<<(a.C + 127) / 128, 128, 0, st>>>(a.C, a.m0, a.K, a.R, a.G, a.w, a.steps, a.Y,
                                               a.status);
  IFEAST_PROF_END(a.prof);
  IFEAST_PROF_BEGIN(a.prof, K_GM_QUAD);
  const size_t nq = (size_t)a.n * a.m0;
  k_quadrature<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(a.n, a.m0, a.nc, a.C, a.V,
                                                             (size_t)a.n * a.C, a.Y, a.steps, a.Q);
  IFEAST_PROF_END(a.prof);
  return cudaGetLastError();
}

cudaError_t spmm_shift_only(int n, const int32_t *rowptr, const int32_t *colidx,
                            const double *val, const double2 *V, double2 *W, int ncols, int m0,
                            const double2 *z, RowTiling tl, cudaStream_t st,
                            const int32_t *rowptrB, const int32_t *colidxB, const double *valB) {
  k_spmm_shift_dot<1, false><<<dim3(tl.P, tl.tiles), kThreads, 0, st>>>(
      n, ncols, m0, rowptr, colidx, val, V, (size_t)n * ncols, 0, z, nullptr, W, nullptr, tl.rows,
      0, rowptrB, colidxB, valB);
  return cudaGetLastError();
}

}  // namespace ifeast
