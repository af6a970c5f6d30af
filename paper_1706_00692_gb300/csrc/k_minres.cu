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
    V0[idx] = (T)(b > 0.0 ? rhs[idx] / b : 0.0);
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
    beta[idx] = 0.0;  // beta_0
  }
  if (idx == 0) st.active[0] = 0;
}

// One Lanczos step s on every column still running.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_lanczos_step(int n, int m0, int s, const int32_t *__restrict__ rowptr,
               const int32_t *__restrict__ colidx, const T *__restrict__ val,
               T *__restrict__ V, const T *__restrict__ Wprev, T *__restrict__ Wout,
               const double *__restrict__ alpha, const double *__restrict__ beta,
               const int *__restrict__ coldone, double *__restrict__ part, int rows) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.y * 32 + lane;
  const size_t vs = (size_t)n * m0;
  const bool act = j < m0 && coldone[j] == 0;
  T a_prev = 0, inv_b = 1, b_s = 0;
  if (act && s > 0) {
    a_prev = (T)alpha[(size_t)(s - 1) * m0 + j];
    b_s = (T)beta[(size_t)s * m0 + j];
    inv_b = (T)(1.0 / beta[(size_t)s * m0 + j]);
  }
  T *__restrict__ Vs = V + (size_t)s * vs;
  const T *__restrict__ Vp = s > 0 ? V + (size_t)(s - 1) * vs : V;
  T vv = 0, vw = 0, ww = 0;
  if (act) {
    const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
    for (int r = r0 + warp; r < r1; r += kWarps) {
      const size_t rj = (size_t)r * m0 + j;
      T v, vprev = 0;
      if (s == 0) {
        v = Vs[rj];
      } else {
        vprev = Vp[rj];
        v = (Wprev[rj] - a_prev * vprev) * inv_b;
        Vs[rj] = v;
      }
      T w = -b_s * vprev;
      const int pb = rowptr[r], pe = rowptr[r + 1];
      if (s == 0) {
#pragma unroll 4
        for (int p = pb; p < pe; ++p) w += val[p] * Vs[(size_t)colidx[p] * m0 + j];
      } else {
        T acc = 0;
#pragma unroll 4
        for (int p = pb; p < pe; ++p) {
          const size_t cj = (size_t)colidx[p] * m0 + j;
          acc += val[p] * (Wprev[cj] - a_prev * Vp[cj]);
        }
        w += acc * inv_b;
      }
      Wout[rj] = w;
      vv += v * v;
      vw += v * w;
      ww += w * w;
    }
  }
  __shared__ double red[3][kWarps][32];
  red[0][warp][lane] = (double)vv;
  red[1][warp][lane] = (double)vw;
  red[2][warp][lane] = (double)ww;
  __syncthreads();
  if (warp < 3 && j < m0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += red[warp][w][lane];
    part[((size_t)blockIdx.x * 3 + warp) * m0 + j] = t;
  }
}

// Fixed-order reduction of the step's partials, Lanczos coefficients and the
// Givens update of every node's tridiagonal least-squares problem. Grid: one
// block per 32-column tile.
__global__ void __launch_bounds__(kThreads)
k_lanczos_givens(int P, int m0, int nc, int K, int s, const double *__restrict__ part,
                 double *__restrict__ alpha, double *__restrict__ beta, const MinresState st,
                 double brk2) {
  __shared__ double red[3][kWarps][32];
  __shared__ double a_s[32], b_s1[32], b_s[32];
  __shared__ int cdone[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j0 = blockIdx.x * 32;
  {
    const int j = j0 + lane;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    if (j < m0)
      for (int b = warp; b < P; b += kWarps) {
        t0 += part[((size_t)b * 3 + 0) * m0 + j];
        t1 += part[((size_t)b * 3 + 1) * m0 + j];
        t2 += part[((size_t)b * 3 + 2) * m0 + j];
      }
    red[0][warp][lane] = t0;
    red[1][warp][lane] = t1;
    red[2][warp][lane] = t2;
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
    if (st.done[p]) continue;
    const double a = a_s[jj], b1 = b_s1[jj], b0 = b_s[jj];
    // column s of (z I - Tbar): rows s-2 (fill), s-1, s, s+1
    double2 e2 = make_double2(0.0, 0.0);
    double2 e1 = make_double2(-b0, 0.0);
    double2 e0 = make_double2(st.z[k].x - a, st.z[k].y);
    double2 *rot = st.rot + (size_t)p * 4;  // [cs(s-2), sn(s-2), cs(s-1), sn(s-1)] by parity
    if (s >= 2) {
      const double2 cs = rot[((s - 2) & 1) * 2], sn = rot[((s - 2) & 1) * 2 + 1];
      // rows (s-2, s-1): [conj cs, conj sn; -sn, cs] applied to (0, e1)
      const double2 t0 = make_double2(sn.x * e1.x + sn.y * e1.y, sn.x * e1.y - sn.y * e1.x);
      const double2 t1 = cmul(cs, e1);
      e2 = t0;
      e1 = t1;
    }
    if (s >= 1) {
      const double2 cs = rot[((s - 1) & 1) * 2], sn = rot[((s - 1) & 1) * 2 + 1];
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
    const double2 gs = g[s];
    const double2 sg = cmul(sn, gs);
    g[s + 1] = make_double2(-sg.x, -sg.y);
    g[s] = make_double2(cs.x * gs.x + cs.y * gs.y, cs.x * gs.y - cs.y * gs.x);
    st.steps[p] = s + 1;
    const double res = sqrt(cabs2(g[s + 1]));
    if (b1 == 0.0 || (st.tol[p] > 0.0 && res <= st.tol[p])) st.done[p] = 1;
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
}

// y = R^{-1} g for each (node, column) pair (banded back substitution), then
// Yc[k][l][j] = wt_{k,j} y_l with wt = w_k (plain) or w_k / (z_k - lambda_j)
// (residual form).
__global__ void k_lz_solve(int m0, int nc, int K, const MinresState st, double2 *__restrict__ Yc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nc * m0) return;
  const int k = p / m0, j = p % m0;
  const int m = st.steps[p];
  const double2 *R = st.R + (size_t)p * K * 3;
  const double2 *g = st.g + (size_t)p * (K + 1);
  double2 wt = st.w[k];
  if (st.correction) wt = cdiv(wt, make_double2(st.z[k].x - st.lam[j], st.z[k].y));
  double2 y1 = make_double2(0.0, 0.0), y2 = make_double2(0.0, 0.0);  // y_{l+1}, y_{l+2}
  for (int l = K - 1; l >= m; --l) Yc[((size_t)k * K + l) * m0 + j] = make_double2(0.0, 0.0);
  for (int l = m - 1; l >= 0; --l) {
    double2 t = g[l];
    if (l + 1 < m) {
      const double2 q = cmul(R[(size_t)(l + 1) * 3 + 1], y1);
      t.x -= q.x;
      t.y -= q.y;
    }
    if (l + 2 < m) {
      const double2 q = cmul(R[(size_t)(l + 2) * 3 + 2], y2);
      t.x -= q.x;
      t.y -= q.y;
    }
    const double2 y = cdiv(t, R[(size_t)l * 3]);
    Yc[((size_t)k * K + l) * m0 + j] = cmul(wt, y);
    y2 = y1;
    y1 = y;
  }
  atomicMax(&st.status->max_steps, m);
  atomicAdd((unsigned long long *)&st.status->total_steps, (unsigned long long)m);
}

// coef[l][j] = Re sum_k Yc[k][l][j]; cx[j] = Re sum_k w_k/(z_k - lambda_j) in the
// residual form (the filter value of the Ritz value), else 0; Sj = max_k steps.
__global__ void k_lz_coef(int m0, int nc, int K, const MinresState st,
                          const double2 *__restrict__ Yc, double *__restrict__ coef,
                          double *__restrict__ cx, int *__restrict__ Sj) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (size_t)K * m0) {
    const int l = (int)(idx / m0), j = (int)(idx % m0);
    double t = 0.0;
    for (int k = 0; k < nc; ++k) t += Yc[((size_t)k * K + l) * m0 + j].x;
    coef[idx] = t;
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

__global__ void k_to_float(size_t n, const double *__restrict__ a, float *__restrict__ b) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

template <typename T>
cudaError_t run_minres(const MinresArgs &a, cudaStream_t st) {
  const size_t nm = (size_t)a.n * a.m0;
  T *V = (T *)a.V;
  T *W[2] = {(T *)a.W0, (T *)a.W1};
  const T *val = (const T *)a.val_t;
  const size_t pc = (size_t)a.nc * a.m0;
  const size_t g0 = nm > pc ? nm : pc;
  k_lz_prep<T><<<(unsigned)((g0 + 255) / 256), 256, 0, st>>>(a.n, a.m0, a.nc, a.K, a.rhs, a.rnorm,
                                                             V, a.beta, a.ms);
  const dim3 grid(a.tl.P, a.tl.tiles);
  const double brk2 = sizeof(T) == 4 ? 1e-6 : 1e-16;
  cudaError_t e = cudaGetLastError();
  int s = 0;
  for (; s < a.K && e == cudaSuccess; ++s) {
    const bool check = a.check_every > 0 && (s + 1) % a.check_every == 0 && s + 1 < a.K;
    k_lanczos_step<T><<<grid, kThreads, 0, st>>>(a.n, a.m0, s, a.rowptr, a.colidx, val, V,
                                                  W[(s + 1) & 1], W[s & 1], a.alpha, a.beta,
                                                  a.ms.coldone, a.part, a.tl.rows);
    if (check) e = cudaMemsetAsync(a.ms.active, 0, sizeof(int), st);
    k_lanczos_givens<<<a.tl.tiles, kThreads, 0, st>>>(a.tl.P, a.m0, a.nc, a.K, s, a.part,
                                                      a.alpha, a.beta, a.ms, brk2);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (check && e == cudaSuccess) {
      // stop early once no column is still running (one small read-back)
      e = cudaMemcpyAsync(a.active_host, a.ms.active, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess && *a.active_host == 0) break;
    }
  }
  if (e != cudaSuccess) return e;
  k_lz_solve<<<(unsigned)((pc + 127) / 128), 128, 0, st>>>(a.m0, a.nc, a.K, a.ms, a.Yc);
  const size_t kc = (size_t)a.K * a.m0;
  k_lz_coef<<<(unsigned)((kc + 255) / 256), 256, 0, st>>>(a.m0, a.nc, a.K, a.ms, a.Yc, a.coef,
                                                           a.cx, a.Sj);
  k_lz_quadrature<T><<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(a.n, a.m0, V, a.coef, a.cx,
                                                                   a.Sj, a.X, a.Q);
  return cudaGetLastError();
}

}  // namespace

cudaError_t minres_filter(const MinresArgs &a, cudaStream_t st) {
  if (a.fp32) return run_minres<float>(a, st);
  return run_minres<double>(a, st);
}

cudaError_t convert_to_float(const double *a, float *b, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, b);
  return cudaGetLastError();
}

}  // namespace ifeast
