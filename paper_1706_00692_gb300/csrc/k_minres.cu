// Inner solve of IFEAST on one Krylov basis per column shared by every contour
// node (Section 3: the basis of K(z I - A, x) does not depend on z).
//
// For a real symmetric A the basis is built by the Lanczos three-term
// recurrence A v_s = beta_s v_{s-1} + alpha_s v_s + beta_{s+1} v_{s+1}; every
// shifted system (z_k I - A) y = b then has the (s+1) x s tridiagonal
// least-squares problem min || ||b|| e_1 - (z_k Ibar - Tbar_s) y ||, whose
// minimiser is the MINRES/GMRES iterate (the shifted matrices are normal).
// Its QR factorisation is updated by Givens rotations (two previous rotations
// touch a new column), giving the residual norm |g_{s+1}| of every (node,
// column) pair at every step.
//
// Storage (row-major, real, T = float or double):
//   V[s]   n x m0 basis vectors (kept: the solution is sum_s V[s] y_s)
//   W0/W1  n x m0 w_s = A v_s - beta_s v_{s-1}, double-buffered by step parity
// One step s is one pass over the rows (k_lanczos_step): it materialises
// v_s = (w_{s-1} - alpha_{s-1} v_{s-1}) / beta_s for its own rows (and on the
// fly for the gathered neighbour rows of the sparse product), forms w_s and
// accumulates <v_s, v_s>, <v_s, w_s>, <w_s, w_s>. A small kernel then reduces
// them in a fixed order: alpha_s = <v,w>/<v,v>, beta_{s+1}^2 = <w,w> -
// <v,w>^2/<v,v> (the squared norm of w_s - alpha_s v_s, using the actual
// <v,v> so that rounding in earlier normalisations does not feed back), and
// advances every node's Givens QR.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "internal.h"

namespace ifeast {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Programmatic dependent launch between the kernels of the Lanczos loop: a
// kernel waits for the previous kernel of the stream (and its memory) before
// it touches anything that kernel or an earlier one wrote, and only then lets
// the next kernel launch, so the next kernel's launch and prologue overlap
// with its tail. Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// v_0 = b / ||b|| with b = X (plain right-hand side of Alg. 2 step 1) or b =
// Rres = A X - X Lambda (residual form); per-column tolerances; Givens state
// reset.
template <typename T>
__global__ void k_lz_prep(int n, int m0, int nc, int K, const double *__restrict__ rhs,
                          const double *__restrict__ rnorm, T *__restrict__ V0,
                          double *__restrict__ beta, const MinresState st) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (size_t)n * m0) {
    const int j = (int)(idx % m0);
    const double b = rnorm[j];
    const double x = b > 0.0 ? rhs[idx] / b : 0.0;
    if constexpr (std::is_same_v<T, __half>)
      V0[idx] = __float2half_rn((float)x);
    else if constexpr (std::is_same_v<T, __nv_bfloat16>)
      V0[idx] = __float2bfloat16_rn((float)x);
    else
      V0[idx] = (T)x;
  }
  if (idx < (size_t)nc * m0) {
    const int p = (int)idx;  // p = k * m0 + j
    const int j = p % m0, k = p / m0;
    const double b = rnorm[j];
    st.g[(size_t)p * (K + 1)] = make_double2(b, 0.0);
    st.steps[p] = 0;
    st.done[p] = b > 0.0 ? 0 : 1;
    // tolerance on |g_{s+1}| (the residual of this shifted solve)
    const double tol_rel = st.status->tol_rel;
    double tol = 0.0;
    if (tol_rel > 0.0) {
      tol = tol_rel * st.xnorm[j];
      if (st.correction) {  // || r - (z I - A) y' || = |z - lambda| || x - (z I - A) y ||
        const double2 d = make_double2(st.z[k].x - st.lam[j], st.z[k].y);
        tol *= sqrt(cabs2(d));
      }
    }
    st.tol[p] = tol;
  }
  if (idx < (size_t)m0) {
    st.coldone[idx] = rnorm[idx] > 0.0 ? 0 : 1;
    st.ndone[idx] = rnorm[idx] > 0.0 ? 0 : nc;  // pairs of the column already done
    beta[idx] = 0.0;  // beta_0
  }
  if (idx == 0) st.active[0] = 0;
}



// v_0 = b / ||b|| again (second pass of the two-pass mode; the same
// arithmetic as k_lz_prep, which also resets the least-squares state).
template <typename T>
__global__ void k_lz_v0(int n, int m0, const double *__restrict__ rhs,
                        const double *__restrict__ rnorm, T *__restrict__ V0) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * m0) return;
  const double b = rnorm[idx % m0];
  const double x = b > 0.0 ? rhs[idx] / b : 0.0;
  if constexpr (std::is_same_v<T, __half>)
    V0[idx] = __float2half_rn((float)x);
  else if constexpr (std::is_same_v<T, __nv_bfloat16>)
    V0[idx] = __float2bfloat16_rn((float)x);
  else
    V0[idx] = (T)x;
}

// One Lanczos step s on every column still running.
//
// A warp owns a contiguous segment of rows; lane l handles the columns
// j = l + 32 q (q < NJ) of every row. Rows are taken in packs whose non-zeros
// (at most 32) are loaded one per lane, then the gathers of 8 non-zeros are
// issued back to back before they are consumed, so that many independent
// loads are in flight per warp. The values of the row itself (w_{s-1}[r],
// v_{s-1}[r]) come from the gather of its diagonal entry when it has one.
template <typename T, int NJ, bool FIRST>
__global__ void __launch_bounds__(kThreads)
k_lanczos_step(int n, int m0, int s, const int32_t *__restrict__ rowptr,
               const int32_t *__restrict__ colidx, const T *__restrict__ val,
               T *__restrict__ V, const T *__restrict__ Wprev, T *__restrict__ Wout,
               const double *__restrict__ alpha, const double *__restrict__ beta,
               const int *__restrict__ coldone, double *__restrict__ part, int rows) {
  constexpr unsigned FULL = 0xffffffffu;
  // non-zeros gathered per batch (all issued before use), sized to the registers
  constexpr int EB = sizeof(T) == 4 ? (NJ <= 3 ? 8 : (NJ <= 5 ? 4 : 2))
                                    : (NJ <= 2 ? 8 : (NJ <= 4 ? 4 : 2));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t vs = (size_t)n * m0;
  T *__restrict__ Vs = V + (size_t)s * vs;
  // FIRST: gather v_0 = V[0] only; else gather w_{s-1} and v_{s-1}
  const T *__restrict__ G1 = FIRST ? Vs : Wprev;
  const T *__restrict__ G2 = FIRST ? Vs : V + (size_t)(s - 1) * vs;
  bool aq[NJ];
  T ap[NJ], ib[NJ], bs[NJ], vv[NJ], vw[NJ], ww[NJ];
#pragma unroll
  for (int q = 0; q < NJ; ++q) {
    const int j = lane + 32 * q;
    aq[q] = j < m0 && coldone[j] == 0;
    ap[q] = 0;
    ib[q] = 1;
    bs[q] = 0;
    if (!FIRST && aq[q]) {
      ap[q] = (T)alpha[(size_t)(s - 1) * m0 + j];
      bs[q] = (T)beta[(size_t)s * m0 + j];
      ib[q] = (T)(1.0 / beta[(size_t)s * m0 + j]);
    }
    vv[q] = vw[q] = ww[q] = 0;
  }
  const int b0 = blockIdx.x * rows, b1 = min(n, b0 + rows);
  const int seg = (rows + kWarps - 1) / kWarps;
  const int rs = min(b1, b0 + warp * seg), re = min(b1, rs + seg);

  // finishes row r: v_s[r], w_s[r] from the accumulated products and the
  // row's own w_{s-1}, v_{s-1} values (o1, o2)
  auto finish = [&](int r, const T (&acc1)[NJ], const T (&acc2)[NJ], const T (&o1)[NJ],
                    const T (&o2)[NJ]) {
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      if (!aq[q]) continue;
      const size_t rj = (size_t)r * m0 + lane + 32 * q;
      T v, w;
      if (FIRST) {
        v = o1[q];
        w = acc1[q];
      } else {
        v = (o1[q] - ap[q] * o2[q]) * ib[q];
        w = (acc1[q] - ap[q] * acc2[q]) * ib[q] - bs[q] * o2[q];
        Vs[rj] = v;
      }
      Wout[rj] = w;
      vv[q] += v * v;
      vw[q] += v * w;
      ww[q] += w * w;
    }
  };
  auto load_own = [&](int r, T (&o1)[NJ], T (&o2)[NJ]) {
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      const size_t rj = (size_t)r * m0 + lane + 32 * q;
      o1[q] = aq[q] ? G1[rj] : (T)0;
      o2[q] = (aq[q] && !FIRST) ? G2[rj] : (T)0;
    }
  };

  int r = rs;
  while (r < re) {
    const int lim = re - r;  // rows left in the segment (>= 1)
    const int rp = lane <= lim ? rowptr[r + lane] : 0x7fffffff;
    const int base = __shfl_sync(FULL, rp, 0);
    const unsigned okm = __ballot_sync(FULL, lane <= lim && rp - base <= 32);
    int R = __popc(okm) - 1;  // rows [r, r+R) hold at most 32 non-zeros
    if (R < 1) R = 1;         // a single row with more than 32: done in chunks
    const int nz_end = __shfl_sync(FULL, rp, R);
    int row = 0;
    int row_end = __shfl_sync(FULL, rp, 1);
    T acc1[NJ], acc2[NJ], o1[NJ], o2[NJ];
    bool have_own = false;
#pragma unroll
    for (int q = 0; q < NJ; ++q) acc1[q] = acc2[q] = o1[q] = o2[q] = 0;
    while (row < R && row_end == base) {  // empty rows at the start of the pack
      load_own(r + row, o1, o2);
      finish(r + row, acc1, acc2, o1, o2);
      ++row;
      row_end = row < R ? __shfl_sync(FULL, rp, row + 1) : 0x7fffffff;
    }
    for (int cb = base; cb < nz_end; cb += 32) {
      const int cnt = min(32, nz_end - cb);
      int ci = 0;
      T cv = 0;
      if (lane < cnt) {
        ci = colidx[cb + lane];
        cv = val[cb + lane];
      }
#pragma unroll
      for (int e0 = 0; e0 < 32; e0 += EB) {
        if (e0 >= cnt) break;
        T g1[EB][NJ], g2[EB][NJ];
        int cs[EB];
#pragma unroll
        for (int e = 0; e < EB; ++e) {
          const int c = __shfl_sync(FULL, ci, e0 + e);
          cs[e] = c;
#pragma unroll
          for (int q = 0; q < NJ; ++q) {
            const size_t cj = (size_t)c * m0 + lane + 32 * q;
            const bool ld = e0 + e < cnt && aq[q];
            g1[e][q] = ld ? G1[cj] : (T)0;
            g2[e][q] = (ld && !FIRST) ? G2[cj] : (T)0;
          }
        }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
          const T a = __shfl_sync(FULL, cv, e0 + e);
          if (e0 + e < cnt) {
            const int gr = r + row;
#pragma unroll
            for (int q = 0; q < NJ; ++q) {
              acc1[q] += a * g1[e][q];
              if (!FIRST) acc2[q] += a * g2[e][q];
            }
            if (cs[e] == gr) {
              have_own = true;
#pragma unroll
              for (int q = 0; q < NJ; ++q) {
                o1[q] = g1[e][q];
                o2[q] = g2[e][q];
              }
            }
            while (cb + e0 + e + 1 == row_end) {  // last non-zero of row gr (and empty rows after it)
              if (!have_own) load_own(r + row, o1, o2);
              finish(r + row, acc1, acc2, o1, o2);
#pragma unroll
              for (int q = 0; q < NJ; ++q) acc1[q] = acc2[q] = 0;
              have_own = false;
              ++row;
              row_end = row < R ? __shfl_sync(FULL, rp, row + 1) : 0x7fffffff;
            }
          }
        }
      }
    }
    r += R;
  }
  __shared__ double red[3][kWarps][32 * NJ];
#pragma unroll
  for (int q = 0; q < NJ; ++q) {
    red[0][warp][lane + 32 * q] = (double)vv[q];
    red[1][warp][lane + 32 * q] = (double)vw[q];
    red[2][warp][lane + 32 * q] = (double)ww[q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 3 * 32 * NJ; t += kThreads) {
    const int which = t / (32 * NJ), j = t % (32 * NJ);
    if (j < m0) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) acc += red[which][w][j];
      part[((size_t)blockIdx.x * 3 + which) * m0 + j] = acc;
    }
  }
}

// Fixed-order reduction of the step's block partials (P blocks) for the 32
// columns j0..j0+31, Lanczos coefficients and the Givens update of every
// node's tridiagonal least-squares problem. Called by a whole block of
// kThreads threads.
__device__ void givens_tile(int j0, int P, int m0, int nc, int K, int s,
                            const double *__restrict__ part, double *__restrict__ alpha,
                            double *__restrict__ beta, const MinresState &st, double brk2) {
  __shared__ double red[3][kWarps][32];
  __shared__ double a_s[32], b_s1[32], b_s[32];
  __shared__ int cdone[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // state of this thread's first (node, column) pair, loaded before the
  // reduction so that its latency overlaps with it
  const int t0p = threadIdx.x;
  const int k0p = t0p / 32, j0p = j0 + (t0p % 32);
  const bool pre = k0p < nc && j0p < m0;
  const int p0 = k0p * m0 + j0p;
  double2 pre_rot[4];
  double2 pre_g = make_double2(0.0, 0.0);
  int pre_done = 1;
  double pre_tol = 0.0;
  if (pre) {
    pre_done = st.done[p0];
#pragma unroll
    for (int u = 0; u < 4; ++u) pre_rot[u] = st.rot[(size_t)p0 * 4 + u];
    pre_g = st.g[(size_t)p0 * (K + 1) + s];
    pre_tol = st.tol[p0];
  }
  {
    // warp w sums blocks w, w + 8, ...: eight independent accumulator sets so
    // that eight rounds of loads are in flight, combined in a fixed order
    const int j = j0 + lane;
    double t0[8], t1[8], t2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t0[u] = t1[u] = t2[u] = 0.0;
    if (j < m0)
      for (int b = warp; b < P; b += 8 * kWarps) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int bb = b + u * kWarps;
          if (bb < P) {
            // L2 reads: the partials may have been written by other SMs in this launch
            t0[u] += __ldcg(part + ((size_t)bb * 3 + 0) * m0 + j);
            t1[u] += __ldcg(part + ((size_t)bb * 3 + 1) * m0 + j);
            t2[u] += __ldcg(part + ((size_t)bb * 3 + 2) * m0 + j);
          }
        }
      }
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s0 += t0[u];
      s1 += t1[u];
      s2 += t2[u];
    }
    red[0][warp][lane] = s0;
    red[1][warp][lane] = s1;
    red[2][warp][lane] = s2;
  }
  __syncthreads();
  if (warp == 0) {
    const int j = j0 + lane;
    double vv = 0.0, vw = 0.0, ww = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      vv += red[0][w][lane];
      vw += red[1][w][lane];
      ww += red[2][w][lane];
    }
    int cd = 1;
    if (j < m0) {
      cd = st.coldone[j];
      if (!cd) {
        const double a = vv > 0.0 ? vw / vv : 0.0;
        const double b2 = ww - (vv > 0.0 ? vw * vw / vv : 0.0);
        const double b = b2 > brk2 * ww ? sqrt(b2) : 0.0;  // 0: invariant subspace reached
        alpha[(size_t)s * m0 + j] = a;
        beta[(size_t)(s + 1) * m0 + j] = b;
        a_s[lane] = a;
        b_s1[lane] = b;
        b_s[lane] = beta[(size_t)s * m0 + j];
      }
    }
    cdone[lane] = cd;
  }
  __syncthreads();
  // Givens update for (node k, column j)
  for (int t = threadIdx.x; t < nc * 32; t += blockDim.x) {
    const int k = t / 32, jj = t % 32, j = j0 + jj;
    if (j >= m0 || cdone[jj]) continue;
    const int p = k * m0 + j;
    const bool first = t == t0p;
    if (first ? pre_done : st.done[p]) continue;
    const double a = a_s[jj], b1 = b_s1[jj], b0 = b_s[jj];
    // column s of (z I - Tbar): rows s-2 (fill), s-1, s, s+1
    double2 e2 = make_double2(0.0, 0.0);
    double2 e1 = make_double2(-b0, 0.0);
    double2 e0 = make_double2(st.z[k].x - a, st.z[k].y);
    double2 *rot = st.rot + (size_t)p * 4;  // [cs(s-2), sn(s-2), cs(s-1), sn(s-1)] by parity
    double2 rr[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) rr[u] = first ? pre_rot[u] : rot[u];
    if (s >= 2) {
      const double2 cs = rr[((s - 2) & 1) * 2], sn = rr[((s - 2) & 1) * 2 + 1];
      // rows (s-2, s-1): [conj cs, conj sn; -sn, cs] applied to (0, e1)
      const double2 t0 = make_double2(sn.x * e1.x + sn.y * e1.y, sn.x * e1.y - sn.y * e1.x);
      const double2 t1 = cmul(cs, e1);
      e2 = t0;
      e1 = t1;
    }
    if (s >= 1) {
      const double2 cs = rr[((s - 1) & 1) * 2], sn = rr[((s - 1) & 1) * 2 + 1];
      const double2 x = e1, y = e0;
      e1 = make_double2(cs.x * x.x + cs.y * x.y + sn.x * y.x + sn.y * y.y,
                        cs.x * x.y - cs.y * x.x + sn.x * y.y - sn.y * y.x);
      const double2 sx = cmul(sn, x), cy = cmul(cs, y);
      e0 = make_double2(cy.x - sx.x, cy.y - sx.y);
    }
    const double rho = hypot(sqrt(cabs2(e0)), b1);
    double2 *R = st.R + ((size_t)p * K + s) * 3;
    double2 *g = st.g + (size_t)p * (K + 1);
    if (!(rho > 0.0)) {
      st.done[p] = 1;
      continue;
    }
    // rotation annihilating the subdiagonal entry -beta_{s+1} below e0
    const double2 cs = make_double2(e0.x / rho, e0.y / rho);
    const double2 sn = make_double2(-b1 / rho, 0.0);
    R[0] = make_double2(rho, 0.0);
    R[1] = e1;
    R[2] = e2;
    rot[(s & 1) * 2] = cs;
    rot[(s & 1) * 2 + 1] = sn;
    const double2 gs = first ? pre_g : g[s];
    const double2 sg = cmul(sn, gs);
    const double2 gn = make_double2(-sg.x, -sg.y);
    g[s + 1] = gn;
    g[s] = make_double2(cs.x * gs.x + cs.y * gs.y, cs.x * gs.y - cs.y * gs.x);
    st.steps[p] = s + 1;
    const double res = sqrt(cabs2(gn));
    const double tol = first ? pre_tol : st.tol[p];
    if (b1 == 0.0 || (tol > 0.0 && res <= tol)) st.done[p] = 1;
  }
  __syncthreads();
  // column j finished when every node is done (or the basis broke down)
  if (threadIdx.x < 32) {
    const int j = j0 + threadIdx.x;
    if (j < m0 && !cdone[threadIdx.x]) {
      int all = 1;  // a broken-down basis (beta_{s+1} = 0) finishes the column
      if (b_s1[threadIdx.x] != 0.0)
        for (int k = 0; k < nc; ++k) all &= st.done[k * m0 + j];
      if (all)
        st.coldone[j] = 1;
      else
        atomicAdd(st.active, 1);
    }
  }
  __syncthreads();  // shared arrays are reused by the next tile
}

// Grid: one block per 32-column tile.
__global__ void __launch_bounds__(kThreads)
k_lanczos_givens(int P, int m0, int nc, int K, int s, const double *__restrict__ part,
                 double *__restrict__ alpha, double *__restrict__ beta, const MinresState st,
                 double brk2) {
  givens_tile(blockIdx.x * 32, P, m0, nc, K, s, part, alpha, beta, st, brk2);
}

// ---------------------------------------------------------------------------
// After an FP32 Lanczos step (k_lanczos_step_vec, k_lanczos_step_ell), only the
// reduction that gives alpha_s and beta_{s+1} stays between two consecutive
// step kernels (k_lanczos_coef_f).
// The Givens QR of every (node, column) pair does not feed the next step, so
// it runs in batches of kGivensBatch steps (k_lanczos_givens_batch): the
// columns' stop flags then lag by less than one batch, and a finished column
// runs at most that many extra Lanczos steps, whose vectors no solution uses
// (each pair keeps its own step count).
// ---------------------------------------------------------------------------
constexpr int kGivensBatch = 16;

// One block of kCoefThreads per 32-column tile, lane = column j: warp w sums
// the partial rows b = w (mod NW) with compensated (Kahan) FP32 sums, all of
// its rows' loads in flight first; warp 0 adds the warp sums and their
// compensations in warp order, again compensated, and forms in FP32
// alpha_s = <v,w>/<v,v>, beta_{s+1}^2 = <w,w> - alpha_s <v,w> (0 below the
// breakdown threshold, which finishes the column); alpha and beta are stored
// widened to FP64 for the Givens batches, and {alpha_s, beta_{s+1},
// 1/beta_{s+1}} as the float4 the next step kernel loads. Only columns
// still running (coldone[j] == 0) get coefficients. active_reset (Givens batch
// steps): cleared so that the batch that follows can raise it.
constexpr int kCoefThreads = 512;
constexpr int kCoefRows = 20;  // partial rows per warp: grids of up to 320 step blocks

__global__ void __launch_bounds__(kCoefThreads)
k_lanczos_coef_f(int P, int m0, int s, const float *__restrict__ part, double *__restrict__ alpha,
                 double *__restrict__ beta, float4 *__restrict__ cf, int *__restrict__ coldone,
                 double brk2, int *__restrict__ active_reset) {
  constexpr int NW = kCoefThreads / 32;
  __shared__ float red[3][2][NW][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 32 + lane;
  pdl_wait();  // the partials of the step kernel
  pdl_launch_next();
  if (active_reset != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *active_reset = 0;
  {
    float x[kCoefRows][3];
#pragma unroll
    for (int u = 0; u < kCoefRows; ++u) {
      const int b = warp + u * NW;
#pragma unroll
      for (int q = 0; q < 3; ++q)
        x[u][q] = (j < m0 && b < P) ? __ldcg(part + ((size_t)b * 3 + q) * m0 + j) : 0.f;
    }
    float sm[3] = {0.f, 0.f, 0.f}, cp[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kCoefRows; ++u)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float y = x[u][q] - cp[q];
        const float t = sm[q] + y;
        cp[q] = (t - sm[q]) - y;
        sm[q] = t;
      }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      red[q][0][warp][lane] = sm[q];
      red[q][1][warp][lane] = cp[q];
    }
  }
  __syncthreads();
  if (warp != 0 || j >= m0 || coldone[j]) return;
  float tot[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float S = 0.f, Cc = 0.f;
#pragma unroll
    for (int w = 0; w < 2 * NW; ++w) {
      const float x = w < NW ? red[q][0][w][lane] : -red[q][1][w - NW][lane];
      const float y = x - Cc;
      const float t = S + y;
      Cc = (t - S) - y;
      S = t;
    }
    tot[q] = S - Cc;
  }
  // FP32 arithmetic: the three sums carry the FP32 rounding of the stored
  // vectors already, and this chain gates the next step (FP64 division and
  // square root take ~1 us on this GPU's FP64 pipe)
  const float vv = tot[0], vw = tot[1], ww = tot[2];
  const float a = vv > 0.f ? vw / vv : 0.f;
  const float b2 = fmaf(-a, vw, ww);
  const float b1 = b2 > (float)brk2 * ww ? sqrtf(b2) : 0.f;  // 0: invariant subspace reached
  alpha[(size_t)s * m0 + j] = a;
  beta[(size_t)(s + 1) * m0 + j] = b1;
  cf[(size_t)(s + 1) * m0 + j] = make_float4(a, b1, b1 != 0.f ? 1.f / b1 : 0.f, 0.f);
  if (b1 == 0.f) coldone[j] = 1;
}

// Givens QR of the shifted tridiagonals (z_k I - Tbar) for steps s0 .. s1 - 1
// of every pair still running; grid (tiles, nc), one thread per (node k,
// column j). Per step: column s of (z_k I - Tbar) is (fill, -beta_s,
// z_k - alpha_s, -beta_{s+1}) in rows s-2 .. s+1; the two previous rotations
// act on it, a new rotation (formed from rsqrt of rho^2) annihilates
// -beta_{s+1}, and the rotated right-hand side gives the residual |g_{s+1}|.
// A pair stops at its tolerance (|g_{s+1}|^2 <= tol^2) or at a breakdown
// (beta_{s+1} = 0); the last pair of a column to stop finishes the column.
// Any pair still running raises *active.
// The coefficients of FP32 Lanczos vectors carry FP32 rounding, so the
// rotations and the factor R are formed in FP32 (this GPU's FP64 pipe issues
// one warp instruction per 64 cycles, and the batch is a dependent chain);
// the rotated right-hand side g, whose magnitude falls by the solve's whole
// reduction, and the stop test stay in FP64. The batch's alpha and beta are
// loaded before the chain starts.
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(32)
k_lanczos_givens_batch(int m0, int nc, int K, int s0, int s1, const double *__restrict__ alpha,
                       const double *__restrict__ beta, const MinresState st) {
  const int j = blockIdx.x * 32 + threadIdx.x, k = blockIdx.y;
  const int p = k * m0 + j;
  pdl_wait();  // alpha, beta of the batch's steps
  pdl_launch_next();
  if (j >= m0 || st.done[p]) return;
  // the last two rotations [cs, sn] by step parity, in registers
  const double2 r0 = st.rot[(size_t)p * 4 + 0], r1 = st.rot[(size_t)p * 4 + 1];
  const double2 r2 = st.rot[(size_t)p * 4 + 2], r3 = st.rot[(size_t)p * 4 + 3];
  float2 c0 = make_float2((float)r0.x, (float)r0.y), s0r = make_float2((float)r1.x, (float)r1.y);
  float2 c1 = make_float2((float)r2.x, (float)r2.y), s1r = make_float2((float)r3.x, (float)r3.y);
  double2 *g = st.g + (size_t)p * (K + 1);
  double2 gs = g[s0];
  const double tol = st.tol[p];
  const float2 zk = make_float2((float)st.z[k].x, (float)st.z[k].y);
  bool fin = false;
  for (int c = s0; c < s1 && !fin; c += kGivensBatch) {
    const int nb = min(kGivensBatch, s1 - c);
    float av[kGivensBatch], b0v[kGivensBatch], b1v[kGivensBatch];
#pragma unroll
    for (int i = 0; i < kGivensBatch; ++i) {
      const size_t o = (size_t)(c + i) * m0 + j;
      av[i] = i < nb ? (float)alpha[o] : 0.f;
      b0v[i] = i < nb ? (float)beta[o] : 0.f;
      b1v[i] = i < nb ? (float)beta[o + m0] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < kGivensBatch; ++i) {
      if (i >= nb || fin) break;
      const int s = c + i;
      const float a = av[i], b0 = b0v[i], b1 = b1v[i];
      float2 e2 = make_float2(0.f, 0.f);
      float2 e1 = make_float2(-b0, 0.f);
      float2 e0 = make_float2(zk.x - a, zk.y);
      // rotation of step s - 2 sits in the parity slot of s, that of step s - 1 in the other
      const bool odd = s & 1;
      if (s >= 2) {
        const float2 cs = odd ? c1 : c0, sn = odd ? s1r : s0r;
        e2 = make_float2(sn.x * e1.x + sn.y * e1.y, sn.x * e1.y - sn.y * e1.x);
        e1 = cmulf(cs, e1);
      }
      if (s >= 1) {
        const float2 cs = odd ? c0 : c1, sn = odd ? s0r : s1r;
        const float2 x = e1, y = e0;
        e1 = make_float2(cs.x * x.x + cs.y * x.y + sn.x * y.x + sn.y * y.y,
                         cs.x * x.y - cs.y * x.x + sn.x * y.y - sn.y * y.x);
        const float2 sx = cmulf(sn, x), cy = cmulf(cs, y);
        e0 = make_float2(cy.x - sx.x, cy.y - sx.y);
      }
      const float rho2 = e0.x * e0.x + e0.y * e0.y + b1 * b1;
      if (!(rho2 > 0.f)) {
        fin = true;
        break;
      }
      const float inv = rsqrtf(rho2);
      const float rho = rho2 * inv;
      const float2 cs = make_float2(e0.x * inv, e0.y * inv);
      const float2 sn = make_float2(-b1 * inv, 0.f);
      double2 *R = st.R + ((size_t)p * K + s) * 3;
      R[0] = make_double2(rho, 0.0);
      R[1] = make_double2(e1.x, e1.y);
      R[2] = make_double2(e2.x, e2.y);
      if (odd) {
        c1 = cs;
        s1r = sn;
      } else {
        c0 = cs;
        s0r = sn;
      }
      const double snd = sn.x, csx = cs.x, csy = cs.y;  // sn is real
      const double2 gn = make_double2(-snd * gs.x, -snd * gs.y);
      g[s + 1] = gn;
      g[s] = make_double2(csx * gs.x + csy * gs.y, csx * gs.y - csy * gs.x);
      gs = gn;
      fin = b1 == 0.f || (tol > 0.0 && cabs2(gn) <= tol * tol);
      st.steps[p] = s + 1;
    }
  }
  st.rot[(size_t)p * 4 + 0] = make_double2(c0.x, c0.y);
  st.rot[(size_t)p * 4 + 1] = make_double2(s0r.x, s0r.y);
  st.rot[(size_t)p * 4 + 2] = make_double2(c1.x, c1.y);
  st.rot[(size_t)p * 4 + 3] = make_double2(s1r.x, s1r.y);
  if (fin) {
    st.done[p] = 1;
    if (atomicAdd(&st.ndone[j], 1) == nc - 1) st.coldone[j] = 1;
  } else {
    *st.active = 1;
  }
}

// ---------------------------------------------------------------------------
// FP32 Lanczos step for m0 % 4 == 0: one thread per (row, four-column quad).
// Threads walk the rows grid-stride, so at any moment the whole grid works on
// one window of consecutive rows and the neighbour rows a stencil-like matrix
// gathers (near and far diagonals) are still in L2 from the previous window.
// Each row's non-zeros are taken in groups of kVG: the group's indices and
// values are loaded together, then all of its float4 gathers are issued before
// they are used. Same recurrence as k_lanczos_step.
// ---------------------------------------------------------------------------
constexpr int kVG = 8;        // non-zeros per gather group
constexpr int kVThreads = 512;  // one block per SM (the register file holds 512 threads)

__device__ __forceinline__ float4 f4fma(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

// Storage of the inner Krylov vectors of the FP32-arithmetic kernels: FP32, or
// FP16 (rounded to nearest; arithmetic stays FP32). Four consecutive columns
// of a row are one 16-byte (FP32) or 8-byte (FP16) access. In FP16 the work
// vectors w_s are stored divided by a scale of A (so that they stay in FP16
// range); rnd() gives the value a number has after a round trip through the
// storage type, so that the Lanczos dots are those of the stored vectors.
template <typename S>
struct Store4;
template <>
struct Store4<float> {
  static constexpr bool kHalf = false;
  static constexpr bool kScaled = false;
  using Raw = float4;  // four stored values as loaded
  __device__ static Raw load_raw(const float *p) { return *reinterpret_cast<const float4 *>(p); }
  __device__ static float4 cvt(Raw r) { return r; }
  __device__ static float4 load(const float *p) { return *reinterpret_cast<const float4 *>(p); }
  __device__ static void store(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
  __device__ static void store1(float *p, float x) { *p = x; }
  __device__ static float rnd(float x) { return x; }
};
template <>
struct Store4<__half> {
  static constexpr bool kHalf = true;
  static constexpr bool kScaled = true;  // w_s stored divided by wsc
  using Raw = uint2;
  __device__ static Raw load_raw(const __half *p) { return *reinterpret_cast<const uint2 *>(p); }
  __device__ static float4 cvt(Raw u) {
    __half2 h0, h1;
    memcpy(&h0, &u.x, 4);
    memcpy(&h1, &u.y, 4);
    const float2 a = __half22float2(h0), b = __half22float2(h1);
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ static float4 load(const __half *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    __half2 h0, h1;
    memcpy(&h0, &u.x, 4);
    memcpy(&h1, &u.y, 4);
    const float2 a = __half22float2(h0), b = __half22float2(h1);
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ static void store(__half *p, float4 v) {
    const __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
    uint2 u;
    memcpy(&u.x, &h0, 4);
    memcpy(&u.y, &h1, 4);
    *reinterpret_cast<uint2 *>(p) = u;
  }
  __device__ static void store1(__half *p, float x) { *p = __float2half_rn(x); }
  __device__ static float rnd(float x) { return __half2float(__float2half_rn(x)); }
};

// BF16: the exponent range of FP32, so the work vectors are stored unscaled
// (the kernels pass wsc = 1 and skip the scaling when kScaled is false).
template <>
struct Store4<__nv_bfloat16> {
  static constexpr bool kHalf = true;
  static constexpr bool kScaled = false;
  using Raw = uint2;
  __device__ static float4 cvt(Raw u) {
    __nv_bfloat162 h0, h1;
    memcpy(&h0, &u.x, 4);
    memcpy(&h1, &u.y, 4);
    const float2 a = __bfloat1622float2(h0), b = __bfloat1622float2(h1);
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ static Raw load_raw(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint2 *>(p);
  }
  __device__ static float4 load(const __nv_bfloat16 *p) { return cvt(load_raw(p)); }
  __device__ static void store(__nv_bfloat16 *p, float4 v) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    memcpy(&u.x, &h0, 4);
    memcpy(&u.y, &h1, 4);
    *reinterpret_cast<uint2 *>(p) = u;
  }
  __device__ static void store1(__nv_bfloat16 *p, float x) { *p = __float2bfloat16_rn(x); }
  __device__ static float rnd(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
};

// Row epilogue of the FP32-arithmetic step kernels. From the row's own
// gathered values o1 (w_{s-1}, or v_0 at s = 0) and o2 (v_{s-1}) and the row
// products acc1 = (A G1)[r], acc2 = (A v_{s-1})[r]: v_s = (w_{s-1} -
// alpha_{s-1} v_{s-1}) / beta_s, w_s = A v_s - beta_s v_{s-1} by linearity;
// both are rounded to the storage type, their dots accumulated and stored.
template <typename S, bool FIRST>
__device__ __forceinline__ void finish_row(float4 o1, float4 o2, float4 acc1, float4 acc2,
                                           const float (&ap)[4], const float (&ib)[4],
                                           const float (&bs)[4], const bool (&act)[4], bool all4,
                                           float wsc, S *__restrict__ Vs, S *__restrict__ Wout,
                                           size_t off, float (&vv)[4], float (&vw)[4],
                                           float (&ww)[4], float (&vout)[4]) {
  using St = Store4<S>;
  if (St::kScaled && !FIRST) {  // w_{s-1} is stored divided by wsc
    o1 = make_float4(o1.x * wsc, o1.y * wsc, o1.z * wsc, o1.w * wsc);
    acc1 = make_float4(acc1.x * wsc, acc1.y * wsc, acc1.z * wsc, acc1.w * wsc);
  }
  const float o1a[4] = {o1.x, o1.y, o1.z, o1.w}, o2a[4] = {o2.x, o2.y, o2.z, o2.w};
  const float a1a[4] = {acc1.x, acc1.y, acc1.z, acc1.w}, a2a[4] = {acc2.x, acc2.y, acc2.z, acc2.w};
  float v[4], w[4], wst[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (FIRST) {
      v[i] = o1a[i];
      w[i] = a1a[i];
    } else {
      v[i] = (o1a[i] - ap[i] * o2a[i]) * ib[i];
      w[i] = (a1a[i] - ap[i] * a2a[i]) * ib[i] - bs[i] * o2a[i];
    }
    wst[i] = w[i];
    if constexpr (St::kScaled) {
      v[i] = St::rnd(v[i]);
      wst[i] = St::rnd(w[i] / wsc);
      w[i] = wst[i] * wsc;
    } else if constexpr (St::kHalf) {
      v[i] = St::rnd(v[i]);
      wst[i] = St::rnd(w[i]);
      w[i] = wst[i];
    }
    if (act[i]) {
      vv[i] = fmaf(v[i], v[i], vv[i]);
      vw[i] = fmaf(v[i], w[i], vw[i]);
      ww[i] = fmaf(w[i], w[i], ww[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) vout[i] = v[i];
  if (all4) {
    if (!FIRST) St::store(Vs + off, make_float4(v[0], v[1], v[2], v[3]));
    St::store(Wout + off, make_float4(wst[0], wst[1], wst[2], wst[3]));
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (act[i]) {
        if (!FIRST) St::store1(Vs + off + i, v[i]);
        St::store1(Wout + off + i, wst[i]);
      }
  }
}

// Block partials of the FP32 step kernels: thread t holds the sums of
// columns 4 q(t) .. 4 q(t) + 3; part[block][0..2][j] = the block's <v,v>,
// <v,w>, <w,w> of column j, added in FP32 in thread order (fixed order).
__device__ __forceinline__ void store_partials_f(const float (&vv)[4], const float (&vw)[4],
                                                 const float (&ww)[4], int m0, int stride_items,
                                                 float *__restrict__ part) {
  __shared__ float red[kVThreads][13];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    red[threadIdx.x][3 * i + 0] = vv[i];
    red[threadIdx.x][3 * i + 1] = vw[i];
    red[threadIdx.x][3 * i + 2] = ww[i];
  }
  __syncthreads();
  const int MQ = m0 >> 2;
  const int base_q = (blockIdx.x * kVThreads) % MQ;
  for (int t = threadIdx.x; t < 3 * m0; t += kVThreads) {
    const int k = t / m0, j = t % m0;
    const int qj = j >> 2, ij = j & 3;
    // threads of this block with q == qj: local index l with (base_q + l) % MQ == qj
    float acc = 0.f;
    for (int l = (qj - base_q + MQ) % MQ; l < kVThreads; l += MQ)
      if (blockIdx.x * kVThreads + l < stride_items) acc += red[l][3 * ij + k];
    part[((size_t)blockIdx.x * 3 + k) * m0 + j] = acc;
  }
}

// Column mask of an FP32 step kernel: column j still runs while coldone[j] is
// 0 (set once the last Givens batch found all of its pairs done, or at a
// breakdown); in the second pass of the two-pass mode, while s < Sj[j] (the
// steps its solves took).
__device__ __forceinline__ void load_column_mask(int m0, const int *__restrict__ coldone,
                                                 int *cdone, const int *__restrict__ Sj, int s) {
  for (int j = threadIdx.x; j < m0; j += kVThreads)
    cdone[j] = Sj != nullptr ? (s < Sj[j] ? 0 : 1) : coldone[j];
  __syncthreads();
}

// Q accumulation of the second pass: Qacc[r][j] += cf[l][j] v_l[r][j] in FP32
// fused multiply-adds, in step order (the same sums as k_lz_quadrature4). The
// terms are added two steps at a time, at odd s (v_{s-1} is the row's own
// value the step already loaded), and at a column's last step when that step
// is even: one read-modify-write of Qacc per two steps.
__device__ __forceinline__ void accumulate_q(const Pass2 &p2, int m0, int s, size_t off, int q4,
                                             const float (&v)[4], const float (&vprev)[4],
                                             const bool (&act)[4]) {
  const bool odd = s & 1;
  bool cur[4], any = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    cur[i] = act[i] && (odd || s == p2.Sj[q4 + i] - 1);
    any = any || cur[i];
  }
  if (!any) return;
  const float *c = p2.cf + (size_t)s * m0 + q4;
  float4 qv = *reinterpret_cast<const float4 *>(p2.Qacc + off);
  float q[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (!cur[i]) continue;
    if (odd) q[i] = fmaf(c[i - m0], vprev[i], q[i]);  // step s - 1 (active: s - 1 < s < Sj)
    q[i] = fmaf(c[i], v[i], q[i]);
  }
  *reinterpret_cast<float4 *>(p2.Qacc + off) = make_float4(q[0], q[1], q[2], q[3]);
}

template <typename S, bool FIRST>
__global__ void __launch_bounds__(kVThreads, 1)
k_lanczos_step_vec(int n, int m0, int s, const int32_t *__restrict__ rowptr,
                   const int32_t *__restrict__ colidx, const float *__restrict__ val,
                   S *__restrict__ V, const S *__restrict__ Wprev, S *__restrict__ Wout,
                   const float4 *__restrict__ cf, const int *__restrict__ coldone,
                   float *__restrict__ part, int stride_items, float wsc, const Pass2 p2) {
  using St = Store4<S>;
  pdl_wait();
  pdl_launch_next();
  const int MQ = m0 >> 2;
  const size_t vs = (size_t)n * m0;
  // basis slot of step s: the stored basis, or a ring of three in the two-pass mode
  S *__restrict__ Vs = V + (size_t)(p2.vring ? s % p2.vring : s) * vs;
  const S *__restrict__ G1 = FIRST ? Vs : Wprev;
  const S *__restrict__ G2 =
      FIRST ? Vs : V + (size_t)(p2.vring ? (s - 1) % p2.vring : s - 1) * vs;
  const int gt = blockIdx.x * kVThreads + threadIdx.x;
  const bool thr = gt < stride_items;
  const int q = thr ? gt % MQ : 0;
  const int rstep = stride_items / MQ;
  float ap[4] = {0.f, 0.f, 0.f, 0.f}, ib[4] = {1.f, 1.f, 1.f, 1.f}, bs[4] = {0.f, 0.f, 0.f, 0.f};
  if (!FIRST && thr) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 c = cf[(size_t)s * m0 + 4 * q + i];  // alpha_{s-1}, beta_s, 1 / beta_s
      ap[i] = c.x;
      bs[i] = c.y;
      ib[i] = c.z;
    }
  }
  __shared__ int cdone[1024];
  load_column_mask(m0, coldone, cdone, p2.Sj, s);
  bool act[4];
  bool qact = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    act[i] = thr && cdone[4 * q + i] == 0;
    qact = qact || act[i];
  }
  const bool all4 = act[0] && act[1] && act[2] && act[3];
  float vv[4] = {0.f, 0.f, 0.f, 0.f}, vw[4] = {0.f, 0.f, 0.f, 0.f}, ww[4] = {0.f, 0.f, 0.f, 0.f};
  if (qact) {
    for (int r = gt / MQ; r < n; r += rstep) {
      const size_t off = (size_t)r * m0 + 4 * q;
      const int pb = rowptr[r], pe = rowptr[r + 1];
      const float4 o1 = St::load(G1 + off);
      float4 o2 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!FIRST) o2 = St::load(G2 + off);
      float4 acc1 = make_float4(0.f, 0.f, 0.f, 0.f), acc2 = acc1;
      for (int p0 = pb; p0 < pe; p0 += kVG) {
        int c[kVG];
        float a[kVG];
#pragma unroll
        for (int u = 0; u < kVG; ++u) {
          const bool in = p0 + u < pe;
          c[u] = in ? colidx[p0 + u] : r;
          a[u] = in ? val[p0 + u] : 0.f;
        }
        float4 g1[kVG], g2[kVG];
#pragma unroll
        for (int u = 0; u < kVG; ++u) {
          const bool in = p0 + u < pe;
          const size_t co = (size_t)c[u] * m0 + 4 * q;
          g1[u] = in ? St::load(G1 + co) : make_float4(0.f, 0.f, 0.f, 0.f);
          if (!FIRST) g2[u] = in ? St::load(G2 + co) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kVG; ++u) {
          acc1 = f4fma(a[u], g1[u], acc1);
          if (!FIRST) acc2 = f4fma(a[u], g2[u], acc2);
        }
      }
      float vo[4];
      finish_row<S, FIRST>(o1, o2, acc1, acc2, ap, ib, bs, act, all4, wsc, Vs, Wout, off, vv, vw,
                           ww, vo);
      if (p2.Qacc != nullptr) {
        const float vp[4] = {o2.x, o2.y, o2.z, o2.w};
        accumulate_q(p2, m0, s, off, 4 * q, vo, vp, act);
      }
    }
  }
  store_partials_f(vv, vw, ww, m0, stride_items, part);
}

// ---------------------------------------------------------------------------
// FP32 Lanczos step on a fixed-width (ELL) copy of A (k_build_ell): every row
// holds exactly W slots (W = 8 or 16), slot 0 is the diagonal entry (its value
// is 0 when A has none there), and unused slots repeat the row's own index
// with a zero value. So a row's indices are one or two 16-byte loads that do
// not wait on rowptr, the next row's indices are fetched while the current
// row's gathers are in flight, the row's own w_{s-1}[r], v_{s-1}[r] are the
// gathers of slot 0, and padding slots (index r past slot 0) are skipped.
// Element offsets are 32-bit (n * m0 < 2^31). Same recurrence as
// k_lanczos_step.
// ---------------------------------------------------------------------------
template <typename S, bool FIRST, int W>
__global__ void __launch_bounds__(kVThreads, 1)
k_lanczos_step_ell(int n, int m0, int s, const int32_t *__restrict__ colE,
                   const float *__restrict__ valE, S *__restrict__ V,
                   const S *__restrict__ Wprev, S *__restrict__ Wout,
                   const float4 *__restrict__ cf, const int *__restrict__ coldone,
                   float *__restrict__ part, int stride_items, float wsc, const Pass2 p2) {
  using St = Store4<S>;
  pdl_wait();
  pdl_launch_next();
  const int MQ = m0 >> 2;
  const size_t vs = (size_t)n * m0;
  // basis slot of step s: the stored basis, or a ring of three in the two-pass mode
  S *__restrict__ Vs = V + (size_t)(p2.vring ? s % p2.vring : s) * vs;
  const S *__restrict__ G1 = FIRST ? Vs : Wprev;
  const S *__restrict__ G2 =
      FIRST ? Vs : V + (size_t)(p2.vring ? (s - 1) % p2.vring : s - 1) * vs;
  const int gt = blockIdx.x * kVThreads + threadIdx.x;
  const bool thr = gt < stride_items;
  const int q = thr ? gt % MQ : 0;
  const int q4 = 4 * q;
  const int rstep = stride_items / MQ;
  float ap[4] = {0.f, 0.f, 0.f, 0.f}, ib[4] = {1.f, 1.f, 1.f, 1.f}, bs[4] = {0.f, 0.f, 0.f, 0.f};
  if (!FIRST && thr) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 c = cf[(size_t)s * m0 + q4 + i];  // alpha_{s-1}, beta_s, 1 / beta_s
      ap[i] = c.x;
      bs[i] = c.y;
      ib[i] = c.z;
    }
  }
  __shared__ int cdone[1024];
  load_column_mask(m0, coldone, cdone, p2.Sj, s);
  bool act[4];
  bool qact = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    act[i] = thr && cdone[q4 + i] == 0;
    qact = qact || act[i];
  }
  const bool all4 = act[0] && act[1] && act[2] && act[3];
  float vv[4] = {0.f, 0.f, 0.f, 0.f}, vw[4] = {0.f, 0.f, 0.f, 0.f}, ww[4] = {0.f, 0.f, 0.f, 0.f};
  int r = gt / MQ;
  if (qact && r < n) {
    int cn[W];
#pragma unroll
    for (int u = 0; u < W; u += 4) {
      const int4 c4 = *reinterpret_cast<const int4 *>(colE + (size_t)r * W + u);
      cn[u] = c4.x;
      cn[u + 1] = c4.y;
      cn[u + 2] = c4.z;
      cn[u + 3] = c4.w;
    }
    for (; r < n; r += rstep) {
      int c[W];
#pragma unroll
      for (int u = 0; u < W; ++u) c[u] = cn[u];
      float a[W];
#pragma unroll
      for (int u = 0; u < W; u += 4) {
        const float4 a4 = *reinterpret_cast<const float4 *>(valE + (size_t)r * W + u);
        a[u] = a4.x;
        a[u + 1] = a4.y;
        a[u + 2] = a4.z;
        a[u + 3] = a4.w;
      }
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      typename St::Raw g1[W], g2[W];  // converted where they are multiplied
      const typename St::Raw zr = {};
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int co = c[u] * m0 + q4;
        const bool ld = u == 0 || c[u] != r;
        g1[u] = ld ? St::load_raw(G1 + co) : zr;
        if (!FIRST) g2[u] = ld ? St::load_raw(G2 + co) : zr;
      }
      const int rn = r + rstep;  // next row's indices, in flight with the gathers
      if (rn < n) {
#pragma unroll
        for (int u = 0; u < W; u += 4) {
          const int4 c4 = *reinterpret_cast<const int4 *>(colE + (size_t)rn * W + u);
          cn[u] = c4.x;
          cn[u + 1] = c4.y;
          cn[u + 2] = c4.z;
          cn[u + 3] = c4.w;
        }
      }
      float4 acc1 = z4, acc2 = z4;
#pragma unroll
      for (int u = 0; u < W; ++u) {
        acc1 = f4fma(a[u], St::cvt(g1[u]), acc1);
        if (!FIRST) acc2 = f4fma(a[u], St::cvt(g2[u]), acc2);
      }
      const float4 o1 = St::cvt(g1[0]), o2 = FIRST ? z4 : St::cvt(g2[0]);
      float vo[4];
      finish_row<S, FIRST>(o1, o2, acc1, acc2, ap, ib, bs, act, all4, wsc, Vs, Wout,
                           (size_t)(r * m0 + q4), vv, vw, ww, vo);
      if (p2.Qacc != nullptr) {
        const float vp[4] = {o2.x, o2.y, o2.z, o2.w};
        accumulate_q(p2, m0, s, (size_t)(r * m0 + q4), q4, vo, vp, act);
      }
    }
  }
  store_partials_f(vv, vw, ww, m0, stride_items, part);
}

// Fixed-width copy of the CSR matrix (FP32 values) for k_lanczos_step_ell:
// slot 0 holds the diagonal entry (value 0 if the row has none), then the
// row's other entries in CSR order, then padding (index r, value 0). W must
// be at least the row length plus one when the row has no diagonal entry.
__global__ void k_build_ell(int n, int W, const int32_t *__restrict__ rowptr,
                            const int32_t *__restrict__ colidx, const float *__restrict__ val,
                            int32_t *__restrict__ colE, float *__restrict__ valE) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int pb = rowptr[r], pe = rowptr[r + 1];
  int32_t *ce = colE + (size_t)r * W;
  float *ve = valE + (size_t)r * W;
  float d = 0.f;
  int u = 1;
  for (int p = pb; p < pe; ++p) {
    if (colidx[p] == r) {
      d = val[p];
    } else if (u < W) {
      ce[u] = colidx[p];
      ve[u] = val[p];
      ++u;
    }
  }
  ce[0] = r;
  ve[0] = d;
  for (; u < W; ++u) {
    ce[u] = r;
    ve[u] = 0.f;
  }
}

// Back substitution y = R^{-1} g for each (node, column) pair, R upper
// triangular with bandwidth 3: y_l = (g_l - r_{l,l+1} y_{l+1} - r_{l,l+2}
// y_{l+2}) / r_{l,l}. The divisions do not depend on y, so they run first, in
// parallel over (pair, l), in place: g_l <- g_l / r_{l,l}, r_{l,l+1} <-
// r_{l,l+1} / r_{l,l}, r_{l,l+2} <- r_{l,l+2} / r_{l,l} (each entry is read and
// written by the thread of its row l only); the dependent recurrence is then
// two complex multiply-adds per row. Thread 0 of each pair's first block also
// forms the pair's quadrature weight wt = w_k (plain) or w_k / (z_k - lambda_j)
// (residual form).
__global__ void k_lz_solve_prep(int m0, int K, const MinresState st, double2 *__restrict__ wt) {
  const int p = blockIdx.y;
  const int k = p / m0, j = p % m0;
  const int m = st.steps[p];
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double2 w = st.w[k];
    if (st.correction) w = cdiv(w, make_double2(st.z[k].x - st.lam[j], st.z[k].y));
    wt[p] = w;
  }
  if (l >= m) return;
  double2 *R = st.R + (size_t)p * K * 3;
  double2 *g = st.g + (size_t)p * (K + 1);
  const double2 r0 = R[(size_t)l * 3];
  const double d = r0.x * r0.x + r0.y * r0.y;
  const double2 inv = make_double2(r0.x / d, -r0.y / d);  // 1 / r_{l,l}
  g[l] = cmul(g[l], inv);
  if (l + 1 < m) R[(size_t)(l + 1) * 3 + 1] = cmul(R[(size_t)(l + 1) * 3 + 1], inv);
  if (l + 2 < m) R[(size_t)(l + 2) * 3 + 2] = cmul(R[(size_t)(l + 2) * 3 + 2], inv);
}

// The recurrence of the back substitution after k_lz_solve_prep:
// Yc[k][l][j] = y_l (unweighted; k_lz_coef applies the pair's weight).
__global__ void k_lz_solve(int m0, int nc, int K, const MinresState st, double2 *__restrict__ Yc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc * m0) return;
  const int k = p / m0, j = p % m0;
  const int m = st.steps[p];
  const double2 *R = st.R + (size_t)p * K * 3;
  const double2 *g = st.g + (size_t)p * (K + 1);
  for (int l = K - 1; l >= m; --l) Yc[((size_t)k * K + l) * m0 + j] = make_double2(0.0, 0.0);
  double2 y1 = make_double2(0.0, 0.0), y2 = make_double2(0.0, 0.0);  // y_{l+1}, y_{l+2}
  // chunks of 8 rows, bottom up; the chunk's coefficients are loaded before
  // the dependent recurrence runs over them
  constexpr int CH = 8;
  for (int hi = m - 1; hi >= 0; hi -= CH) {
    double2 a[CH], b[CH], c[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int l = hi - u;
      if (l >= 0) {
        a[u] = g[l];
        b[u] = (l + 1 < m) ? R[(size_t)(l + 1) * 3 + 1] : make_double2(0.0, 0.0);
        c[u] = (l + 2 < m) ? R[(size_t)(l + 2) * 3 + 2] : make_double2(0.0, 0.0);
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int l = hi - u;
      if (l >= 0) {
        // y = a - b y1 - c y2
        double2 y;
        y.x = a[u].x - (b[u].x * y1.x - b[u].y * y1.y) - (c[u].x * y2.x - c[u].y * y2.y);
        y.y = a[u].y - (b[u].x * y1.y + b[u].y * y1.x) - (c[u].x * y2.y + c[u].y * y2.x);
        Yc[((size_t)k * K + l) * m0 + j] = y;
        y2 = y1;
        y1 = y;
      }
    }
  }
  atomicMax(&st.status->max_steps, m);
  atomicAdd((unsigned long long *)&st.status->total_steps, (unsigned long long)m);
}

// coef[l][j] = Re sum_k wt[k][j] Yc[k][l][j]; cx[j] = Re sum_k w_k/(z_k - lambda_j)
// in the residual form (the filter value of the Ritz value), else 0;
// Sj = max_k steps.
__global__ void k_lz_coef(int m0, int nc, int K, const MinresState st,
                          const double2 *__restrict__ Yc, const double2 *__restrict__ wt,
                          double *__restrict__ coef, double *__restrict__ cx,
                          int *__restrict__ Sj) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (size_t)K * m0) {
    const int l = (int)(idx / m0), j = (int)(idx % m0);
    double t = 0.0;
    for (int k = 0; k < nc; ++k) {
      const double2 w = wt[k * m0 + j], y = Yc[((size_t)k * K + l) * m0 + j];
      t += w.x * y.x - w.y * y.y;
    }
    coef[idx] = t;
    // FP32 copy (after the K x m0 doubles) for the FP32 quadrature
    reinterpret_cast<float *>(coef + (size_t)K * m0)[idx] = (float)t;
  }
  if (idx < (size_t)m0) {
    const int j = (int)idx;
    double c = 0.0;
    int mx = 0;
    for (int k = 0; k < nc; ++k) {
      if (st.correction) c += cdiv(st.w[k], make_double2(st.z[k].x - st.lam[j], st.z[k].y)).x;
      mx = max(mx, st.steps[k * m0 + j]);
    }
    cx[j] = c;
    Sj[j] = mx;
  }
}

// Q[r][j] = cx[j] X[r][j] + sum_{l < Sj} coef[l][j] V[l][r][j].
template <typename T>
__global__ void k_lz_quadrature(int n, int m0, const T *__restrict__ V, const double *__restrict__ coef,
                                const double *__restrict__ cx, const int *__restrict__ Sj,
                                const double *__restrict__ X, double *__restrict__ Q) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * m0) return;
  const int j = (int)(idx % m0);
  const int S = Sj[j];
  const size_t vs = (size_t)n * m0;
  T acc = 0;
  int l = 0;
  for (; l + 4 <= S; l += 4) {
    acc += (T)coef[(size_t)l * m0 + j] * V[(size_t)l * vs + idx];
    acc += (T)coef[(size_t)(l + 1) * m0 + j] * V[(size_t)(l + 1) * vs + idx];
    acc += (T)coef[(size_t)(l + 2) * m0 + j] * V[(size_t)(l + 2) * vs + idx];
    acc += (T)coef[(size_t)(l + 3) * m0 + j] * V[(size_t)(l + 3) * vs + idx];
  }
  for (; l < S; ++l) acc += (T)coef[(size_t)l * m0 + j] * V[(size_t)l * vs + idx];
  Q[idx] = cx[j] * X[idx] + (double)acc;
}

// FP32 or FP16 basis, m0 % 4 == 0: four columns per thread, eight basis vectors in
// flight. A column only takes the basis vectors its own solves built
// (l < Sj[j]); later ones were not written for it and are never multiplied.
template <typename ST>
__global__ void __launch_bounds__(256)
k_lz_quadrature4(int n, int m0, int K, const ST *__restrict__ V, const double *__restrict__ coef,
                 const double *__restrict__ cx, const int *__restrict__ Sj,
                 const double *__restrict__ X, double *__restrict__ Q) {
  const size_t i4 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nq = (size_t)n * m0 / 4;
  if (i4 >= nq) return;
  const int j0 = (int)((i4 * 4) % m0);
  const int s0 = Sj[j0], s1 = Sj[j0 + 1], s2 = Sj[j0 + 2], s3 = Sj[j0 + 3];
  const int S = max(max(s0, s1), max(s2, s3));
  const size_t vs = (size_t)n * m0;  // basis stride in elements
  const ST *__restrict__ V4 = V + i4 * 4;
  // FP32 coefficients (written by k_lz_coef after the FP64 ones), float4 per quad
  const float4 *__restrict__ C4 =
      reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(coef + (size_t)K * m0) + j0);
  const int cq = m0 / 4;  // float4 stride of one coefficient row
  float ax = 0.f, ay = 0.f, az = 0.f, aw = 0.f;
  int l = 0;
  for (; l + 8 <= S; l += 8) {
    float4 v[8], c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      v[u] = Store4<ST>::load(V4 + (size_t)(l + u) * vs);
      c[u] = C4[(size_t)(l + u) * cq];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int ll = l + u;
      ax = ll < s0 ? fmaf(c[u].x, v[u].x, ax) : ax;
      ay = ll < s1 ? fmaf(c[u].y, v[u].y, ay) : ay;
      az = ll < s2 ? fmaf(c[u].z, v[u].z, az) : az;
      aw = ll < s3 ? fmaf(c[u].w, v[u].w, aw) : aw;
    }
  }
  for (; l < S; ++l) {
    const float4 v = Store4<ST>::load(V4 + (size_t)l * vs);
    const float4 c = C4[(size_t)l * cq];
    ax = l < s0 ? fmaf(c.x, v.x, ax) : ax;
    ay = l < s1 ? fmaf(c.y, v.y, ay) : ay;
    az = l < s2 ? fmaf(c.z, v.z, az) : az;
    aw = l < s3 ? fmaf(c.w, v.w, aw) : aw;
  }
  const size_t e = i4 * 4;
  Q[e + 0] = cx[j0 + 0] * X[e + 0] + (double)ax;
  Q[e + 1] = cx[j0 + 1] * X[e + 1] + (double)ay;
  Q[e + 2] = cx[j0 + 2] * X[e + 2] + (double)az;
  Q[e + 3] = cx[j0 + 3] * X[e + 3] + (double)aw;
}

// Q = cx X + Qacc (second pass of the two-pass mode; the quadrature's last step)
__global__ void k_lz_combine(int n, int m0, const float *__restrict__ Qacc,
                             const double *__restrict__ cx, const double *__restrict__ X,
                             double *__restrict__ Q) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * m0) return;
  Q[e] = cx[e % m0] * X[e] + (double)Qacc[e];
}

__global__ void k_to_float(size_t n, const double *__restrict__ a, float *__restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

template <typename T, int NJ>
void launch_step_nj(const MinresArgs &a, int s, T *V, const T *Wp, T *Wo, const T *val,
                    cudaStream_t st) {
  if (s == 0)
    k_lanczos_step<T, NJ, true><<<a.tl.P, kThreads, 0, st>>>(a.n, a.m0, s, a.rowptr, a.colidx,
                                                            val, V, Wp, Wo, a.alpha, a.beta,
                                                            a.ms.coldone, a.part, a.tl.rows);
  else
    k_lanczos_step<T, NJ, false><<<a.tl.P, kThreads, 0, st>>>(a.n, a.m0, s, a.rowptr, a.colidx,
                                                             val, V, Wp, Wo, a.alpha, a.beta,
                                                             a.ms.coldone, a.part, a.tl.rows);
}

bool use_vec_step(const MinresArgs &a) { return a.fp32 && a.m0 % 4 == 0 && a.m0 <= 1024; }

bool use_ell_step(const MinresArgs &a) {
  return use_vec_step(a) && (a.ell_w == 8 || a.ell_w == 16) && (long long)a.n * a.m0 < (1LL << 31);
}

// Launch with programmatic stream serialization (see pdl_wait)
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Lanczos breakdown threshold on beta^2 / ||w||^2 for the storage precision
// ((16 u)^2 for the storage's unit roundoff u: below it the new direction is
// not resolved by the stored vectors)
template <typename T>
double brk2_of() {
  if constexpr (std::is_same_v<T, __half>) return 1e-4;
  if constexpr (std::is_same_v<T, __nv_bfloat16>) return 4e-3;
  return sizeof(T) == 4 ? 1e-6 : 1e-16;
}

// Values of A in the kernels that store the basis as T
template <typename T>
using ValOf = std::conditional_t<std::is_same_v<T, double>, double, float>;

// Blocks of k_lanczos_step_vec and the number of (row, quad) items the grid
// covers per sweep (a multiple of m0 / 4).
void vec_grid(const MinresArgs &a, int &blocks, int &stride_items) {
  const int MQ = a.m0 / 4;
  const long long need = (long long)a.n * MQ;
  long long b = std::min<long long>((need + kVThreads - 1) / kVThreads, (long long)a.P_async);
  // the coefficient kernel holds at most NW x kCoefRows partial rows
  b = std::min<long long>(b, (kCoefThreads / 32) * kCoefRows);
  if (b < 1) b = 1;
  blocks = (int)b;
  stride_items = (int)((b * kVThreads) / MQ * MQ);
  if (stride_items < MQ) {  // fewer threads than one row needs: one more block
    blocks = (MQ + kVThreads - 1) / kVThreads;
    stride_items = (blocks * kVThreads) / MQ * MQ;
  }
}

template <typename T>
cudaError_t launch_lanczos_step(const MinresArgs &a, int s, T *V, const T *Wp, T *Wo,
                                const ValOf<T> *val, const Pass2 &p2, cudaStream_t st) {
  if constexpr (sizeof(T) <= 4) {
    const int *coldone = a.ms.coldone;  // columns finished by the Givens batches
    float *part = reinterpret_cast<float *>(a.part);
    if (use_ell_step(a)) {
      int blocks, stride_items;
      vec_grid(a, blocks, stride_items);
#define IFEAST_ELL_LAUNCH(F, WW)                                                              \
  launch_pdl(k_lanczos_step_ell<T, F, WW>, dim3(blocks), dim3(kVThreads), st, a.n, a.m0, s,     \
             a.colE, a.valE, V, Wp, Wo, a.cf32, coldone, part, stride_items, a.wscale, p2)
      if (a.ell_w == 8)
        return s == 0 ? IFEAST_ELL_LAUNCH(true, 8) : IFEAST_ELL_LAUNCH(false, 8);
      return s == 0 ? IFEAST_ELL_LAUNCH(true, 16) : IFEAST_ELL_LAUNCH(false, 16);
#undef IFEAST_ELL_LAUNCH
    }
    if (use_vec_step(a)) {
      int blocks, stride_items;
      vec_grid(a, blocks, stride_items);
      if (s == 0)
        return launch_pdl(k_lanczos_step_vec<T, true>, dim3(blocks), dim3(kVThreads), st, a.n,
                          a.m0, s, a.rowptr, a.colidx, val, V, Wp, Wo, a.cf32, coldone, part,
                          stride_items, a.wscale, p2);
      return launch_pdl(k_lanczos_step_vec<T, false>, dim3(blocks), dim3(kVThreads), st, a.n, a.m0,
                        s, a.rowptr, a.colidx, val, V, Wp, Wo, a.cf32, coldone, part,
                        stride_items, a.wscale, p2);
    }
  }
  if constexpr (std::is_same_v<T, __half> || std::is_same_v<T, __nv_bfloat16>) {
    return cudaErrorInvalidValue;  // 16-bit storage needs m0 % 4 == 0 (checked at create)
  } else {
    const int nj = (a.m0 + 31) / 32;
    switch (nj) {
      case 1: launch_step_nj<T, 1>(a, s, V, Wp, Wo, val, st); break;
      case 2: launch_step_nj<T, 2>(a, s, V, Wp, Wo, val, st); break;
      case 3: launch_step_nj<T, 3>(a, s, V, Wp, Wo, val, st); break;
      case 4: launch_step_nj<T, 4>(a, s, V, Wp, Wo, val, st); break;
      case 5: launch_step_nj<T, 5>(a, s, V, Wp, Wo, val, st); break;
      case 6: launch_step_nj<T, 6>(a, s, V, Wp, Wo, val, st); break;
      case 7: launch_step_nj<T, 7>(a, s, V, Wp, Wo, val, st); break;
      case 8: launch_step_nj<T, 8>(a, s, V, Wp, Wo, val, st); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
}

// T: storage of the Krylov vectors (double, float or __half)
template <typename T>
cudaError_t run_minres(const MinresArgs &a, cudaStream_t st) {
  const size_t nm = (size_t)a.n * a.m0;
  T *V = (T *)a.V;
  T *W[2] = {(T *)a.W0, (T *)a.W1};
  const ValOf<T> *val = (const ValOf<T> *)a.val_t;
  const size_t pc = (size_t)a.nc * a.m0;
  const size_t g0 = nm > pc ? nm : pc;
  IFEAST_PROF_BEGIN(a.prof, K_PREP);
  k_lz_prep<T><<<(unsigned)((g0 + 255) / 256), 256, 0, st>>>(a.n, a.m0, a.nc, a.K, a.rhs, a.rnorm,
                                                             V, a.beta, a.ms);
  IFEAST_PROF_END(a.prof);
  const double brk2 = brk2_of<T>();
  int step_blocks = a.tl.P;
  // the FP32-arithmetic vec / ELL step kernels reduce their FP32 partials themselves
  const bool f32_partials = sizeof(T) <= 4 && use_vec_step(a);
  if (f32_partials) {
    int stride_items;
    vec_grid(a, step_blocks, stride_items);
  }
  // first pass: stored basis, or (two-pass mode) a ring of three basis slots
  const Pass2 pass1 = {nullptr, nullptr, nullptr, a.two_pass ? 3 : 0};
  cudaError_t e = cudaGetLastError();
  int s = 0, ck = 0;  // ck: checkpoints enqueued
  int s0 = 0;         // first step not yet taken by a Givens batch (FP32 kernels)
  for (; s < a.K && e == cudaSuccess; ++s) {
    const bool check = a.check_every > 0 && (s + 1) % a.check_every == 0 && s + 1 < a.K;
    IFEAST_PROF_BEGIN(a.prof, K_LZ_STEP);
    e = launch_lanczos_step<T>(a, s, V, W[(s + 1) & 1], W[s & 1], val, pass1, st);
    IFEAST_PROF_END(a.prof);
    if (check && !f32_partials && e == cudaSuccess)
      e = cudaMemsetAsync(a.ms.active, 0, sizeof(int), st);
    if (e == cudaSuccess) {
      if (f32_partials) {
        // alpha_s, beta_{s+1}; then, at batch ends and checks, the Givens QR of
        // the steps since the last batch (no memset between kernels breaks
        // their launch overlap: at a batch step the coefficient kernel clears
        // *active itself)
        const bool batch = (s + 1) % kGivensBatch == 0 || check || s + 1 == a.K;
        IFEAST_PROF_BEGIN(a.prof, K_LZ_REDUCE);
        e = launch_pdl(k_lanczos_coef_f, dim3(a.tl.tiles), dim3(kCoefThreads), st, step_blocks,
                       a.m0, s, reinterpret_cast<const float *>(a.part), a.alpha, a.beta, a.cf32,
                       a.ms.coldone, brk2, batch ? a.ms.active : nullptr);
        IFEAST_PROF_END(a.prof);
        if (batch && e == cudaSuccess) {  // the Givens QR of the steps since the last batch
          IFEAST_PROF_BEGIN(a.prof, K_LZ_GIVENS);
          e = launch_pdl(k_lanczos_givens_batch, dim3(a.tl.tiles, a.nc), dim3(32), st, a.m0, a.nc,
                         a.K, s0, s + 1, a.alpha, a.beta, a.ms);
          IFEAST_PROF_END(a.prof);
          s0 = s + 1;
        }
      } else {
        IFEAST_PROF_BEGIN(a.prof, K_LZ_GIVENS);
        k_lanczos_givens<<<a.tl.tiles, kThreads, 0, st>>>(step_blocks, a.m0, a.nc, a.K, s,
                                                          a.part, a.alpha, a.beta, a.ms, brk2);
        IFEAST_PROF_END(a.prof);
      }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (check && e == cudaSuccess) {
      // stop early once no column is still running: this checkpoint's flag is
      // copied and marked by an event; the host waits on the checkpoint
      // kCheckLag earlier, so kCheckLag * check_every steps stay queued (steps
      // after every column is done do no work and change no state)
      const int slot = ck % (kCheckLag + 1);
      e = cudaMemcpyAsync(a.active_host + slot, a.ms.active, sizeof(int), cudaMemcpyDeviceToHost,
                          st);
      if (e == cudaSuccess) e = cudaEventRecord(a.check_events[slot], st);
      ++ck;
      if (e == cudaSuccess && ck > kCheckLag) {
        const int old = (ck - 1 - kCheckLag) % (kCheckLag + 1);
        e = cudaEventSynchronize(a.check_events[old]);
        if (e == cudaSuccess && a.prof && a.prof->collect_ready()) e = cudaErrorUnknown;
        if (e == cudaSuccess && a.active_host[old] == 0) break;
        if (e == cudaSuccess && a.time_limit_ms > 0.0 &&
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a.t0)
                    .count() >= a.time_limit_ms) {
          if (a.cut) *a.cut = true;  // the steps run so far make the filter
          break;
        }
      }
    }
  }
  if (e != cudaSuccess) return e;
  IFEAST_PROF_BEGIN(a.prof, K_LZ_SOLVE);
  k_lz_solve_prep<<<dim3((unsigned)((a.K + 127) / 128), (unsigned)pc), 128, 0, st>>>(a.m0, a.K,
                                                                                   a.ms, a.wt);
  k_lz_solve<<<(unsigned)((pc + 31) / 32), 32, 0, st>>>(a.m0, a.nc, a.K, a.ms, a.Yc);
  IFEAST_PROF_END(a.prof);
  const size_t kc = (size_t)a.K * a.m0;
  IFEAST_PROF_BEGIN(a.prof, K_LZ_COEF);
  k_lz_coef<<<(unsigned)((kc + 255) / 256), 256, 0, st>>>(a.m0, a.nc, a.K, a.ms, a.Yc, a.wt, a.coef,
                                                           a.cx, a.Sj);
  IFEAST_PROF_END(a.prof);
  if constexpr (sizeof(T) <= 4) {
    if (a.two_pass) {
      // second pass: rebuild v_0 .. v_{S-1} from the stored alpha, beta (same
      // arithmetic as the first pass) and accumulate Q; the solves' steps bound
      // the pass (max over the (node, column) pairs)
      e = cudaMemcpyAsync(a.active_host, &a.ms.status->max_steps, sizeof(int),
                          cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return e;
      const int S = *a.active_host;
      if (cudaMemsetAsync(a.Qf, 0, nm * sizeof(float), st) != cudaSuccess) return cudaGetLastError();
      IFEAST_PROF_BEGIN(a.prof, K_PREP);
      k_lz_v0<T><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(a.n, a.m0, a.rhs, a.rnorm, V);
      IFEAST_PROF_END(a.prof);
      const Pass2 pass2 = {a.Qf, reinterpret_cast<const float *>(a.coef + (size_t)a.K * a.m0),
                           a.Sj, 3};
      for (int s2 = 0; s2 < S && e == cudaSuccess; ++s2) {
        IFEAST_PROF_BEGIN(a.prof, K_LZ_STEP);
        e = launch_lanczos_step<T>(a, s2, V, W[(s2 + 1) & 1], W[s2 & 1], val, pass2, st);
        IFEAST_PROF_END(a.prof);
      }
      if (e != cudaSuccess) return e;
      IFEAST_PROF_BEGIN(a.prof, K_LZ_QUAD);
      k_lz_combine<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(a.n, a.m0, a.Qf, a.cx, a.X, a.Q);
      IFEAST_PROF_END(a.prof);
      return cudaGetLastError();
    }
  }
  IFEAST_PROF_BEGIN(a.prof, K_LZ_QUAD);
  if constexpr (sizeof(T) <= 4) {
    if (a.m0 % 4 == 0)
      k_lz_quadrature4<T><<<(unsigned)((nm / 4 + 255) / 256), 256, 0, st>>>(
          a.n, a.m0, a.K, V, a.coef, a.cx, a.Sj, a.X, a.Q);
  }
  if constexpr (!std::is_same_v<T, __half> && !std::is_same_v<T, __nv_bfloat16>) {
    if (sizeof(T) == 8 || a.m0 % 4 != 0)
      k_lz_quadrature<T><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(a.n, a.m0, V, a.coef, a.cx,
                                                                       a.Sj, a.X, a.Q);
  }
  IFEAST_PROF_END(a.prof);
  return cudaGetLastError();
}

}  // namespace

cudaError_t minres_init() { return cudaSuccess; }

cudaError_t minres_filter(const MinresArgs &a, cudaStream_t st) {
  if (a.half) return run_minres<__half>(a, st);
  if (a.bf16) return run_minres<__nv_bfloat16>(a, st);
  if (a.fp32) return run_minres<float>(a, st);
  return run_minres<double>(a, st);
}

cudaError_t build_ell(int n, int W, const int32_t *rowptr, const int32_t *colidx, const float *val,
                      int32_t *colE, float *valE, cudaStream_t st) {
  k_build_ell<<<(n + 255) / 256, 256, 0, st>>>(n, W, rowptr, colidx, val, colE, valE);
  return cudaGetLastError();
}

cudaError_t convert_to_float(const double *a, float *b, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, b);
  return cudaGetLastError();
}

}  // namespace ifeast
