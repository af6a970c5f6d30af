// Rayleigh-Ritz and residual check of IFEAST (Algorithm 2, steps 3-4), FP64.
//   spmm_real      AQ = A Q                                   (n x m0)
//   gram           block partials of A_Q = Q^T AQ, B_Q = Q^T Q (upper triangles,
//                  4x4 register tiles over a shared-memory chunk of rows)
//   reduce_gram    fixed-order sum of the partials, mirrored to full matrices
//   reduced_eig    one CTA: B_Q = L L^T (shifted on breakdown), C = L^-1 A_Q L^-T,
//                  cyclic Jacobi C = U diag(lam) U^T, X_Q = L^-T U, ascending sort
//   update_resid   X = Q X_Q, AX = AQ X_Q (AX never stored) and block partials
//                  of ||AX_j - lam_j X_j||^2, ||AX_j||^2, ||X_j||^2
//   reduce_resid   residuals, interval count, ||R_F||, next inner tolerance
#include <algorithm>
#include <cfloat>

#include "internal.h"

namespace ifeast {

namespace {

constexpr int kGramRows = 32;  // rows of Q / AQ staged in shared memory at a time
constexpr size_t kEigSmem = 200 * 1024;  // dynamic shared memory of the reduced eigensolver

// AQ = A Q: warp per row, lane per column (32-column tiles).
__global__ void __launch_bounds__(kThreads)
k_spmm_real(int n, int m, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
            const double *__restrict__ val, const double *__restrict__ Q, double *__restrict__ AQ,
            int rows) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.y * 32 + lane;
  if (j >= m) return;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int r = r0 + warp; r < r1; r += kWarps) {
    double acc = 0.0;
    const int jb = rowptr[r], je = rowptr[r + 1];
#pragma unroll 4
    for (int p = jb; p < je; ++p) acc = fma(val[p], Q[(size_t)colidx[p] * m + j], acc);
    AQ[(size_t)r * m + j] = acc;
  }
}

// Partials of Q^T AQ and Q^T Q over this block's rows. Thread t of block
// (bx, by) owns the 4x4 output tile number by*256 + t of the upper triangle
// of tiles (m0 padded to mp = multiple of 4), or of all tiles when full != 0.
// With BQ (generalized problem) the second matrix is Q^T (B Q) instead of Q^T Q.
__global__ void __launch_bounds__(kThreads)
k_gram(int n, int m, int mp, const double *__restrict__ Q, const double *__restrict__ AQ,
       const double *__restrict__ BQ, double *__restrict__ part, int rows, int full) {
  extern __shared__ double sm[];
  double *Qs = sm;                       // kGramRows x mp
  double *As = sm + kGramRows * mp;      // kGramRows x mp
  double *Bs = BQ ? sm + 2 * kGramRows * mp : Qs;  // kGramRows x mp
  const int nt = mp / 4;
  const int ntiles = full ? nt * nt : nt * (nt + 1) / 2;
  const int tile = blockIdx.y * kThreads + threadIdx.x;
  int ti = 0, tj = 0;
  const bool own = tile < ntiles;
  if (own && full) {  // every tile (non-symmetric A_Q)
    ti = tile / nt;
    tj = tile % nt;
  } else if (own) {  // tile -> (ti, tj), ti <= tj, row-major over the upper triangle
    int t = tile, r = 0;
    while (t >= nt - r) {
      t -= nt - r;
      ++r;
    }
    ti = r;
    tj = r + t;
  }
  double a[4][4], b[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) a[p][q] = b[p][q] = 0.0;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int rb = r0; rb < r1; rb += kGramRows) {
    const int nr = min(kGramRows, r1 - rb);
    for (int e = threadIdx.x; e < kGramRows * mp; e += kThreads) {
      const int rr = e / mp, jj = e % mp;
      const bool in = rr < nr && jj < m;
      Qs[e] = in ? Q[(size_t)(rb + rr) * m + jj] : 0.0;
      As[e] = in ? AQ[(size_t)(rb + rr) * m + jj] : 0.0;
      if (BQ) Bs[e] = in ? BQ[(size_t)(rb + rr) * m + jj] : 0.0;
    }
    __syncthreads();
    if (own) {
      for (int rr = 0; rr < nr; ++rr) {
        const double *qr = Qs + rr * mp;
        const double *ar = As + rr * mp;
        const double *br = Bs + rr * mp;
        double qi[4], qj[4], aj[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          qi[p] = qr[4 * ti + p];
          qj[p] = br[4 * tj + p];
          aj[p] = ar[4 * tj + p];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            a[p][q] = fma(qi[p], aj[q], a[p][q]);
            b[p][q] = fma(qi[p], qj[q], b[p][q]);
          }
      }
    }
    __syncthreads();
  }
  if (own) {
    double *pa = part + (size_t)blockIdx.x * 2 * mp * mp;
    double *pb = pa + (size_t)mp * mp;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        pa[(size_t)(4 * ti + p) * mp + 4 * tj + q] = a[p][q];
        pb[(size_t)(4 * ti + p) * mp + 4 * tj + q] = b[p][q];
      }
  }
}

// Sum of the gram partials over blocks (fixed order), for i <= j within the
// computed tiles; mirrored into full m x m matrices. A_Q is symmetrised as
// (A_Q + A_Q^T)/2 on the diagonal tiles, where both (i, j) and (j, i) exist.
__global__ void k_reduce_gram(int Pg, int m, int mp, const double *__restrict__ part,
                              double *__restrict__ Aq, double *__restrict__ Bq) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int i = idx / m, j = idx % m;
  if (i > j) return;
  const bool same_tile = (i / 4) == (j / 4);
  double sa = 0.0, sb = 0.0, sa2 = 0.0, sb2 = 0.0;
  for (int b = 0; b < Pg; ++b) {
    const double *pa = part + (size_t)b * 2 * mp * mp;
    const double *pb = pa + (size_t)mp * mp;
    sa += pa[(size_t)i * mp + j];
    sb += pb[(size_t)i * mp + j];
    if (same_tile) {
      sa2 += pa[(size_t)j * mp + i];
      sb2 += pb[(size_t)j * mp + i];
    }
  }
  if (same_tile) {
    sa = 0.5 * (sa + sa2);
    sb = 0.5 * (sb + sb2);
  }
  Aq[(size_t)i * m + j] = sa;
  Aq[(size_t)j * m + i] = sa;
  Bq[(size_t)i * m + j] = sb;
  Bq[(size_t)j * m + i] = sb;
}

__device__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

// Right-looking Cholesky of the m x m matrix in L (lower part used). Returns
// 0 on success, 1 if a pivot was not positive.
__device__ int cholesky_inplace(double *L, int m, int *flag) {
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[(size_t)j * m + j];
      if (!(d > 0.0)) {
        *flag = 1;
      } else {
        L[(size_t)j * m + j] = sqrt(d);
      }
    }
    __syncthreads();
    if (*flag) return 1;
    const double d = L[(size_t)j * m + j];
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) L[(size_t)i * m + j] /= d;
    __syncthreads();
    const int nt = m - j - 1;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
      const int i = j + 1 + e / nt, k = j + 1 + e % nt;
      if (k <= i) L[(size_t)i * m + k] -= L[(size_t)i * m + j] * L[(size_t)k * m + j];
    }
    __syncthreads();
  }
  return 0;
}

// Cyclic Jacobi on the symmetric m x m matrix Cm (leading dimension ld) with
// rotations accumulated into U (same ld), both of type T, round-robin pairing
// so that m/2 disjoint rotations are applied at once; warp w updates the two
// rows (or columns) of pairs w, w + nwarps, ... with its lanes along them. An
// odd ld keeps the column passes free of shared-memory bank conflicts. Stops
// when the off-diagonal part's squared Frobenius norm is at most stop times
// the whole matrix's, when a sweep finds no pair worth rotating at the working
// precision, or after max_sweeps sweeps.
template <typename T>
__device__ void jacobi_rr(T *Cm, T *U, int m, int ld, int max_sweeps, double stop, double *red,
                          double *rot_c, double *rot_s, int *rot_a, int *rot_b) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int mp = m + (m & 1);
  const int npairs = mp / 2;
  __shared__ int any_rot;  // a sweep that rotates nothing ends the iteration
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = warp; i < m; i += nwarps)
      for (int k = lane; k < m; k += 32) {
        const double v = (double)Cm[(size_t)i * ld + k] * (double)Cm[(size_t)i * ld + k];
        tot += v;
        if (i != k) off += v;
      }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    if (!(off > stop * tot)) break;
    if (tid == 0) any_rot = 0;
    __syncthreads();
    for (int round = 0; round < mp - 1; ++round) {
      for (int p = tid; p < npairs; p += nth) {
        const int pa = p, pb = mp - 1 - p;
        int a = pa == 0 ? 0 : 1 + (pa - 1 + round) % (mp - 1);
        int b = pb == 0 ? 0 : 1 + (pb - 1 + round) % (mp - 1);
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        // the rotation is formed in the sweep's own precision T (FP64
        // division and square root cost ~1,100 cycles per round on this GPU)
        T c = 1, s = 0;
        if (b < m) {
          const T apq = Cm[(size_t)a * ld + b];
          const T app = Cm[(size_t)a * ld + a], aqq = Cm[(size_t)b * ld + b];
          // below this the rotation changes nothing at the working precision
          const T tiny = sizeof(T) == 4 ? (T)1e-30 : (T)1e-300;
          const T rel = sizeof(T) == 4 ? (T)FLT_EPSILON : (T)DBL_EPSILON;
          if (fabs(apq) > tiny && fabs(apq) > rel * sqrt(fabs(app * aqq))) {
            const T tau = (aqq - app) / (2 * apq);
            const T big = sizeof(T) == 4 ? (T)1e18 : (T)1e150;
            const T t = (tau >= 0 ? (T)1 : (T)-1) /
                        (fabs(tau) + (fabs(tau) < big ? sqrt(1 + tau * tau) : fabs(tau)));
            c = 1 / sqrt(1 + t * t);
            s = t * c;
            any_rot = 1;  // every writer stores the same value
          }
        }
        rot_a[p] = a;
        rot_b[p] = b < m ? b : a;
        rot_c[p] = (double)c;
        rot_s[p] = (b < m) ? (double)s : 0.0;
      }
      __syncthreads();
      // rows: C <- J^T C
      for (int p = warp; p < npairs; p += nwarps) {
        const int a = rot_a[p], b = rot_b[p];
        if (a == b || rot_s[p] == 0.0) continue;
        const T c = (T)rot_c[p], s = (T)rot_s[p];
        for (int k = lane; k < m; k += 32) {
          const T x = Cm[(size_t)a * ld + k], y = Cm[(size_t)b * ld + k];
          Cm[(size_t)a * ld + k] = c * x - s * y;
          Cm[(size_t)b * ld + k] = s * x + c * y;
        }
      }
      __syncthreads();
      // columns: C <- C J, U <- U J
      for (int p = warp; p < npairs; p += nwarps) {
        const int a = rot_a[p], b = rot_b[p];
        if (a == b || rot_s[p] == 0.0) continue;
        const T c = (T)rot_c[p], s = (T)rot_s[p];
        for (int k = lane; k < m; k += 32) {
          const T x = Cm[(size_t)k * ld + a], y = Cm[(size_t)k * ld + b];
          Cm[(size_t)k * ld + a] = c * x - s * y;
          Cm[(size_t)k * ld + b] = s * x + c * y;
          const T u = U[(size_t)k * ld + a], v = U[(size_t)k * ld + b];
          U[(size_t)k * ld + a] = c * u - s * v;
          U[(size_t)k * ld + b] = s * u + c * v;
        }
      }
      __syncthreads();
    }
    if (!any_rot) break;
  }
}

// Generalised symmetric eigenproblem A_Q X = B_Q X Lambda in one CTA.
// stage 0: the whole solve. With the cluster sweeps (k_eig_cluster.cu):
// stage 1 stops once C = L^-1 A_Q L^-T is formed and leaves C in Cg and L in
// Lg (row-major, leading dimension m); stage 2 takes the unsorted eigenvalues
// from lam and the eigenvectors V of C from Cg, sorts them and forms
// X_Q = L^-T V (launched with smem_mats = 0).
__global__ void __launch_bounds__(512)
k_reduced_eig(int m, const double *__restrict__ Aq, const double *__restrict__ Bq,
              double *__restrict__ Lg, double *__restrict__ Cg, double *__restrict__ Ug,
              double *__restrict__ XQ, double *__restrict__ lam, DevStatus *__restrict__ status,
              int smem_mats, int stage) {
  // smem_mats = how many of (C, U, L) live in shared memory (in that order)
  extern __shared__ double smem[];
  // each matrix in shared memory takes m x (m | 1) doubles (room for the odd
  // leading dimension of the mixed-precision path)
  const size_t mm_ = (size_t)m * (m | 1);
  double *Cm = smem_mats >= 1 ? smem : Cg;
  double *U = smem_mats >= 2 ? smem + mm_ : (stage == 2 ? Cg : Ug);
  double *L = smem_mats >= 3 ? smem + 2 * mm_ : Lg;
  __shared__ double red[32];
  __shared__ int flag;
  __shared__ double rot_c[kMaxM0 / 2], rot_s[kMaxM0 / 2];
  __shared__ int rot_a[kMaxM0 / 2], rot_b[kMaxM0 / 2];
  __shared__ double evals[kMaxM0];
  __shared__ int rank[kMaxM0];
  const int tid = threadIdx.x, nth = blockDim.x;
  const size_t mm = (size_t)m * m;
  if (stage == 2) {
    if (status->breakdown) return;  // stage 1 found B_Q not positive definite
    for (int i = tid; i < m; i += nth) evals[i] = lam[i];
    __syncthreads();
  } else {

  // ---- Cholesky of B_Q, with one shifted retry --------------------------
  double fro2 = 0.0;
  for (size_t e = tid; e < mm; e += nth) fro2 += Bq[e] * Bq[e];
  fro2 = block_sum(fro2, red);
  int shifted = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift =
        attempt ? 11.0 * ((double)m * m + (double)m * (m + 1)) * DBL_EPSILON * sqrt(fro2) : 0.0;
    for (size_t e = tid; e < mm; e += nth) {
      const int i = (int)(e / m), k = (int)(e % m);
      L[e] = (k <= i) ? Bq[e] + (i == k ? shift : 0.0) : 0.0;
    }
    if (tid == 0) flag = 0;
    __syncthreads();
    if (cholesky_inplace(L, m, &flag) == 0) break;
    __syncthreads();
    if (attempt == 1) {
      if (tid == 0) status->breakdown = 1;
      return;
    }
    shifted = 1;
  }
  if (tid == 0) {
    status->breakdown = 0;
    status->shifted = shifted;
  }
  __syncthreads();

  // ---- C = L^-1 A_Q L^-T ---------------------------------------------------
  // Y = L^-1 A_Q into U (thread per column), then C = L^-1 Y^T.
  for (int col = tid; col < m; col += nth) {
    for (int i = 0; i < m; ++i) {
      double t = Aq[(size_t)i * m + col];
      for (int k = 0; k < i; ++k) t -= L[(size_t)i * m + k] * U[(size_t)k * m + col];
      U[(size_t)i * m + col] = t / L[(size_t)i * m + i];
    }
  }
  __syncthreads();
  for (int col = tid; col < m; col += nth) {
    for (int i = 0; i < m; ++i) {
      double t = U[(size_t)col * m + i];
      for (int k = 0; k < i; ++k) t -= L[(size_t)i * m + k] * Cm[(size_t)k * m + col];
      Cm[(size_t)i * m + col] = t / L[(size_t)i * m + i];
    }
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nth) {
    const int i = (int)(e / m), k = (int)(e % m);
    if (i < k) {
      const double v = 0.5 * (Cm[e] + Cm[(size_t)k * m + i]);
      Cm[e] = v;
      Cm[(size_t)k * m + i] = v;
    }
  }
  for (size_t e = tid; e < mm; e += nth) U[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
  __syncthreads();
  if (stage == 1) {  // C and L to global memory for the cluster sweeps
    if (smem_mats >= 1)
      for (size_t e = tid; e < mm; e += nth) Cg[e] = Cm[e];
    if (smem_mats >= 3)
      for (size_t e = tid; e < mm; e += nth) Lg[e] = L[e];
    return;
  }

  if (smem_mats >= 3) {
    // ---- mixed precision: FP32 sweeps, FP64 re-orthonormalisation and finish
    // Dense work matrices use an odd leading dimension (bank-conflict-free
    // column access); the launch gives each of C, U, L m x ld doubles.
    const int ld = m | 1;
    const size_t ml = (size_t)m * ld;
    // C, computed above with leading dimension m, moved to ld through U's buffer
    if (ld != m) {
      for (size_t e = tid; e < mm; e += nth) U[e] = Cm[e];
      __syncthreads();
      for (int i = tid / 32; i < m; i += nth / 32)
        for (int k = tid & 31; k < m; k += 32) Cm[(size_t)i * ld + k] = U[(size_t)i * m + k];
      __syncthreads();
    }
    // FP32 Jacobi (64x the FP64 rate on this GPU) on Cf = (float) C, with its
    // rotations in Uf; both live in U's buffer.
    float *Cf = reinterpret_cast<float *>(U);
    float *Uf = Cf + ml;
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) {
        Cf[(size_t)i * ld + k] = (float)Cm[(size_t)i * ld + k];
        Uf[(size_t)i * ld + k] = i == k ? 1.f : 0.f;
      }
    __syncthreads();
    // stop near the FP32 rounding floor (off-diagonal norm ~1e-5 of the
    // matrix); the FP64 sweeps below finish the job
    jacobi_rr<float>(Cf, Uf, m, ld, 16, 1e-10, red, rot_c, rot_s, rot_a, rot_b);
    // U0 = Uf in FP64 (in L's buffer; L is kept in global memory), then
    // CholQR in FP64: G = U0^T U0 = R^T R, U0 <- U0 R^{-1}, orthonormal to
    // FP64 rounding
    double *U0 = L;
    for (size_t e = tid; e < mm; e += nth) Lg[e] = L[e];
    __syncthreads();
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) U0[(size_t)i * ld + k] = (double)Uf[(size_t)i * ld + k];
    __syncthreads();
    double *G = U;  // Cf / Uf are consumed; G is m x m compact
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) {
        double t = 0.0;
        if (k <= i)
          for (int r = 0; r < m; ++r) t += U0[(size_t)r * ld + i] * U0[(size_t)r * ld + k];
        G[(size_t)i * m + k] = t;
      }
    if (tid == 0) flag = 0;
    __syncthreads();
    cholesky_inplace(G, m, &flag);  // U0 is orthonormal to FP32 rounding: G is SPD
    __syncthreads();
    // each row x of U0 solves x_new R = x with R = G^T (upper): forward substitution
    for (int r = tid; r < m; r += nth) {
      double *x = U0 + (size_t)r * ld;
      for (int k = 0; k < m; ++k) {
        double t = x[k];
        for (int i = 0; i < k; ++i) t -= x[i] * G[(size_t)k * m + i];
        x[k] = t / G[(size_t)k * m + k];
      }
    }
    __syncthreads();
    // C' = U0^T C U0 (T = C U0 in U's buffer, C' over C)
    double *Tm = U;
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) {
        double t = 0.0;
        for (int r = 0; r < m; ++r) t += Cm[(size_t)i * ld + r] * U0[(size_t)r * ld + k];
        Tm[(size_t)i * ld + k] = t;
      }
    __syncthreads();
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) {
        if (k < i) continue;
        double t = 0.0;
        for (int r = 0; r < m; ++r) t += U0[(size_t)r * ld + i] * Tm[(size_t)r * ld + k];
        Cm[(size_t)i * ld + k] = t;
        Cm[(size_t)k * ld + i] = t;
      }
    __syncthreads();
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) U[(size_t)i * ld + k] = i == k ? 1.0 : 0.0;
    __syncthreads();
    // FP64 sweeps on the nearly diagonal C' (quadratic convergence: one or two)
    jacobi_rr<double>(Cm, U, m, ld, 60, 1e-28, red, rot_c, rot_s, rot_a, rot_b);
    for (int i = tid; i < m; i += nth) evals[i] = Cm[(size_t)i * ld + i];
    __syncthreads();
    // eigenvectors of C: U0 V (into C's buffer)
    for (int i = tid / 32; i < m; i += nth / 32)
      for (int k = tid & 31; k < m; k += 32) {
        double t = 0.0;
        for (int r = 0; r < m; ++r) t += U0[(size_t)i * ld + r] * U[(size_t)r * ld + k];
        Cm[(size_t)i * ld + k] = t;
      }
    __syncthreads();
    for (int i = tid; i < m; i += nth) {
      int r = 0;
      const double v = evals[i];
      for (int k = 0; k < m; ++k) r += (evals[k] < v) || (evals[k] == v && k < i);
      rank[i] = r;
    }
    __syncthreads();
    // X_Q = L^-T (U0 V) with L from global memory, ascending order
    for (int col = tid; col < m; col += nth) {
      const int dst = rank[col];
      for (int i = m - 1; i >= 0; --i) {
        double t = Cm[(size_t)i * ld + col];
        for (int k = i + 1; k < m; ++k) t -= Lg[(size_t)k * m + i] * XQ[(size_t)k * m + dst];
        XQ[(size_t)i * m + dst] = t / Lg[(size_t)i * m + i];
      }
      lam[dst] = evals[col];
    }
    return;
  }
  // ---- FP64 cyclic Jacobi (large m: matrices in global memory) --------------
  jacobi_rr<double>(Cm, U, m, m, 60, 1e-28, red, rot_c, rot_s, rot_a, rot_b);
  for (int i = tid; i < m; i += nth) evals[i] = Cm[(size_t)i * m + i];
  __syncthreads();
  }
  // ---- X_Q = L^-T U (back substitution per column), ascending order -------
  for (int i = tid; i < m; i += nth) {
    int r = 0;
    const double v = evals[i];
    for (int k = 0; k < m; ++k) r += (evals[k] < v) || (evals[k] == v && k < i);
    rank[i] = r;
  }
  __syncthreads();
  for (int col = tid; col < m; col += nth) {
    const int dst = rank[col];
    for (int i = m - 1; i >= 0; --i) {
      double t = U[(size_t)i * m + col];
      for (int k = i + 1; k < m; ++k) t -= L[(size_t)k * m + i] * XQ[(size_t)k * m + dst];
      XQ[(size_t)i * m + dst] = t / L[(size_t)i * m + i];
    }
    lam[dst] = evals[col];
  }
}

// X = Q X_Q, AX = AQ X_Q on this block's rows; partials per column j of
// ||AX_j - lam_j X_j||^2, ||AX_j||^2, ||X_j||^2. blockDim = (32, 8): x over
// columns j = tx + 32 q, y over rows.
template <int QMAX>
__global__ void __launch_bounds__(256)
k_update_resid(int n, int m, const double *__restrict__ Q, const double *__restrict__ AQ,
               const double *__restrict__ XQ, const double *__restrict__ lam,
               double *__restrict__ X, double *__restrict__ Rres, double *__restrict__ part,
               int rows, const double *__restrict__ BQ, double *__restrict__ BX) {
  extern __shared__ double sm[];
  const int RB = 8;
  double *Qs = sm;            // RB x m
  double *As = sm + RB * m;   // RB x m
  double *Bs = sm + 2 * RB * m;  // RB x m (generalized only)
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  double e2[QMAX], a2[QMAX], x2[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) e2[q] = a2[q] = x2[q] = 0.0;
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int rb = r0; rb < r1; rb += RB) {
    const int nr = min(RB, r1 - rb);
    for (int e = tid; e < RB * m; e += 256) {
      const int rr = e / m, jj = e % m;
      Qs[e] = rr < nr ? Q[(size_t)(rb + rr) * m + jj] : 0.0;
      As[e] = rr < nr ? AQ[(size_t)(rb + rr) * m + jj] : 0.0;
      if (BQ) Bs[e] = rr < nr ? BQ[(size_t)(rb + rr) * m + jj] : 0.0;
    }
    __syncthreads();
    if (ty < nr) {
      const double *qr = Qs + ty * m;
      const double *ar = As + ty * m;
      const double *br = Bs + ty * m;
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int j = tx + 32 * q;
        if (j < m) {
          double x = 0.0, ax = 0.0, bx = 0.0;
          for (int i = 0; i < m; ++i) {
            const double xq = XQ[(size_t)i * m + j];
            x = fma(qr[i], xq, x);
            ax = fma(ar[i], xq, ax);
            if (BQ) bx = fma(br[i], xq, bx);
          }
          X[(size_t)(rb + ty) * m + j] = x;
          if (!BQ) bx = x;
          else BX[(size_t)(rb + ty) * m + j] = bx;
          const double d = ax - lam[j] * bx;
          if (Rres) Rres[(size_t)(rb + ty) * m + j] = d;
          e2[q] = fma(d, d, e2[q]);
          a2[q] = fma(ax, ax, a2[q]);
          x2[q] = fma(bx, bx, x2[q]);  // ||B x_j||^2: norm of the next right-hand side
        }
      }
    }
    __syncthreads();
  }
  // reduce over ty (fixed order) and store this block's partials
  __shared__ double red[8][32];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    for (int which = 0; which < 3; ++which) {
      red[ty][tx] = which == 0 ? e2[q] : (which == 1 ? a2[q] : x2[q]);
      __syncthreads();
      if (ty == 0) {
        double t = 0.0;
        for (int y = 0; y < 8; ++y) t += red[y][tx];
        const int j = tx + 32 * q;
        if (j < m) part[((size_t)blockIdx.x * 3 + which) * m + j] = t;
      }
      __syncthreads();
    }
  }
}

// Column norms of X only (first iteration): partial slot 2 as in update_resid.
__global__ void k_colnorm_part(int n, int m, const double *__restrict__ X, double *__restrict__ part,
                               int rows) {
  const int j = blockIdx.y * 32 + (threadIdx.x & 31);
  const int w = threadIdx.x >> 5;
  __shared__ double red[kWarps][32];
  double t = 0.0;
  if (j < m) {
    const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
    for (int r = r0 + w; r < r1; r += kWarps) {
      const double x = X[(size_t)r * m + j];
      t = fma(x, x, t);
    }
  }
  red[w][threadIdx.x & 31] = t;
  __syncthreads();
  if (w == 0 && j < m) {
    double u = 0.0;
    for (int q = 0; q < kWarps; ++q) u += red[q][threadIdx.x];
    part[((size_t)blockIdx.x * 3 + 2) * m + j] = u;
  }
}

__global__ void k_reduce_norms(int Pr, int m, const double *__restrict__ part, double *__restrict__ beta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double t = 0.0;
  for (int b = 0; b < Pr; ++b) t += part[((size_t)b * 3 + 2) * m + j];
  beta[j] = sqrt(t);
}

// Residuals, interval count, ||R_F|| and the next inner tolerance (one block).
__global__ void k_reduce_resid(int Pr, int m, const double *__restrict__ part,
                               const double *__restrict__ lam, double emin, double emax,
                               double alpha, double *__restrict__ res, double *__restrict__ beta,
                               double *__restrict__ rnorm, DevStatus *__restrict__ status) {
  __shared__ double smax[256];
  __shared__ int scnt[256], snan[256];
  double mx = 0.0;
  int cnt = 0, bad = 0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double e = 0.0, a = 0.0, x = 0.0;
    for (int b = 0; b < Pr; ++b) {
      e += part[((size_t)b * 3 + 0) * m + j];
      a += part[((size_t)b * 3 + 1) * m + j];
      x += part[((size_t)b * 3 + 2) * m + j];
    }
    const double r = sqrt(e) / (a > 0.0 ? sqrt(a) : 1.0);
    res[j] = r;
    beta[j] = sqrt(x);
    if (rnorm) rnorm[j] = sqrt(e);
    const double l = lam[j];
    if (!isfinite(r) || !isfinite(l)) bad = 1;
    if (l > emin && l < emax) {
      ++cnt;
      mx = fmax(mx, r);
    }
  }
  smax[threadIdx.x] = mx;
  scnt[threadIdx.x] = cnt;
  snan[threadIdx.x] = bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0;
    int N = 0, B = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      M = fmax(M, smax[t]);
      N += scnt[t];
      B |= snan[t];
    }
    const double RF = N > 0 ? M : 1.0;
    status->RF = RF;
    status->count = N;
    status->nonfinite = B;
    status->tol_rel = alpha > 0.0 ? alpha * RF : 0.0;
  }
}


// ===========================================================================
// Non-Hermitian extension (real non-symmetric A): Galerkin Rayleigh-Ritz on
// span(Q). B_Q = Q^T Q = L L^T, the carried basis is X = Q L^{-T} (orthonormal
// columns), C = L^{-1} (Q^T A Q) L^{-T} is a general real matrix whose
// eigenpairs (theta_j, u_j) give the Ritz pairs (theta_j, X u_j).
// ===========================================================================

// Full sums of the gram partials: A_Q as computed (no symmetrisation), B_Q
// symmetrised.
__global__ void k_reduce_gram_full(int Pg, int m, int mp, const double *__restrict__ part,
                                   double *__restrict__ Aq, double *__restrict__ Bq) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int i = idx / m, j = idx % m;
  double sa = 0.0, sb = 0.0, sb2 = 0.0;
  for (int b = 0; b < Pg; ++b) {
    const double *pa = part + (size_t)b * 2 * mp * mp;
    const double *pb = pa + (size_t)mp * mp;
    sa += pa[(size_t)i * mp + j];
    sb += pb[(size_t)i * mp + j];
    sb2 += pb[(size_t)j * mp + i];
  }
  Aq[(size_t)i * m + j] = sa;
  Bq[(size_t)i * m + j] = 0.5 * (sb + sb2);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// principal square root
__device__ double2 zsqrt(double2 z) {
  const double r = zabs(z);
  if (r == 0.0) return make_double2(0.0, 0.0);
  const double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

constexpr int kNsMaxM0 = 64;  // largest m0 of the non-symmetric reduced solver
constexpr size_t kNsEigSmem = 6 * (size_t)kNsMaxM0 * kNsMaxM0 * sizeof(double);

// One CTA. Steps: Cholesky of B_Q (one shifted retry), L^{-1}, C = L^{-1}
// A_Q L^{-T}; Householder reduction of C to upper Hessenberg form (H = Z^T
// C Z); complex single-shift QR iteration (Wilkinson shifts, deflation on
// negligible subdiagonals, rotations applied to the whole matrix and to Z) to
// the Schur form T = W^H C W; eigenvectors of T by back substitution; u_j =
// W y_j normalised. Outputs L^{-T}, theta, U. status->breakdown = 1: B_Q not
// factorable; 2: the QR iteration did not converge in 30 m steps.
__global__ void __launch_bounds__(256)
k_reduced_eig_nonsym(int m, const double *__restrict__ Aq, const double *__restrict__ Bq,
                     double *__restrict__ LinvT, double2 *__restrict__ theta,
                     double2 *__restrict__ Uc, DevStatus *__restrict__ status) {
  extern __shared__ __align__(16) double smem[];
  const size_t mm = (size_t)m * m;
  double *L = smem;                                 // region 0: Cholesky factor, then Zr
  double *Li = smem + mm;                           // region 1: L^{-1}
  double *Y = smem + 2 * mm;                        // region 2: L^{-1} A_Q, then H
  double *Cr = smem + 4 * mm;                       // region 3: C (real), then Z
  double2 *H = reinterpret_cast<double2 *>(smem + 2 * mm);
  double2 *Z = reinterpret_cast<double2 *>(smem + 4 * mm);
  double2 *Yv = reinterpret_cast<double2 *>(smem);  // regions 0-1: eigenvectors of T
  double *Zr = L;
  __shared__ double red[32];
  __shared__ int flag, sh_l;
  __shared__ double hv[kNsMaxM0];
  __shared__ double sh_vv, sh_norm;
  __shared__ double gc[kNsMaxM0];
  __shared__ double2 gs[kNsMaxM0];
  __shared__ double2 sh_mu;
  const int tid = threadIdx.x, nth = blockDim.x;

  // ---- Cholesky of B_Q, with one shifted retry --------------------------
  double fro2 = 0.0;
  for (size_t e = tid; e < mm; e += nth) fro2 += Bq[e] * Bq[e];
  fro2 = block_sum(fro2, red);
  int shifted = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift =
        attempt ? 11.0 * ((double)m * m + (double)m * (m + 1)) * DBL_EPSILON * sqrt(fro2) : 0.0;
    for (size_t e = tid; e < mm; e += nth) {
      const int i = (int)(e / m), k = (int)(e % m);
      L[e] = (k <= i) ? Bq[e] + (i == k ? shift : 0.0) : 0.0;
    }
    if (tid == 0) flag = 0;
    __syncthreads();
    if (cholesky_inplace(L, m, &flag) == 0) break;
    __syncthreads();
    if (attempt == 1) {
      if (tid == 0) status->breakdown = 1;
      return;
    }
    shifted = 1;
  }
  if (tid == 0) {
    status->breakdown = 0;
    status->shifted = shifted;
  }
  __syncthreads();
  // ---- L^{-1} (thread per column), L^{-T} out, C = L^{-1} A_Q L^{-T} -----
  for (int j = tid; j < m; j += nth)
    for (int i = 0; i < m; ++i) {
      double t = (i == j) ? 1.0 : 0.0;
      for (int k = j; k < i; ++k) t -= L[(size_t)i * m + k] * Li[(size_t)k * m + j];
      Li[(size_t)i * m + j] = i < j ? 0.0 : t / L[(size_t)i * m + i];
    }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nth) {
    const int i = (int)(e / m), j = (int)(e % m);
    LinvT[e] = Li[(size_t)j * m + i];
    double t = 0.0;
    for (int k = 0; k <= i; ++k) t += Li[(size_t)i * m + k] * Aq[(size_t)k * m + j];
    Y[e] = t;
  }
  __syncthreads();
  for (size_t e = tid; e < mm; e += nth) {
    const int i = (int)(e / m), j = (int)(e % m);
    double t = 0.0;
    for (int k = 0; k <= j; ++k) t += Y[(size_t)i * m + k] * Li[(size_t)j * m + k];
    Cr[e] = t;
    Zr[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // ---- Householder reduction to upper Hessenberg form ---------------------
  for (int k = 0; k + 2 < m; ++k) {
    if (tid == 0) {
      double nx = 0.0;
      for (int i = k + 1; i < m; ++i) nx += Cr[(size_t)i * m + k] * Cr[(size_t)i * m + k];
      nx = sqrt(nx);
      const double x0 = Cr[(size_t)(k + 1) * m + k];
      double vv = 0.0;
      if (nx > 0.0) {
        const double al = x0 >= 0.0 ? -nx : nx;
        for (int i = k + 1; i < m; ++i) hv[i] = Cr[(size_t)i * m + k];
        hv[k + 1] = x0 - al;
        for (int i = k + 1; i < m; ++i) vv += hv[i] * hv[i];
      }
      sh_vv = vv;
    }
    __syncthreads();
    const double vv = sh_vv;
    if (vv > 0.0) {
      // C <- (I - 2 v v^T / vv) C on rows k+1.., columns k..
      for (int j = k + tid; j < m; j += nth) {
        double t = 0.0;
        for (int i = k + 1; i < m; ++i) t += hv[i] * Cr[(size_t)i * m + j];
        const double f = 2.0 * t / vv;
        for (int i = k + 1; i < m; ++i) Cr[(size_t)i * m + j] -= f * hv[i];
      }
      __syncthreads();
      // C <- C (I - 2 v v^T / vv), Z <- Z (I - 2 v v^T / vv) on columns k+1..
      for (int r = tid; r < 2 * m; r += nth) {
        double *row = r < m ? Cr + (size_t)r * m : Zr + (size_t)(r - m) * m;
        double t = 0.0;
        for (int j = k + 1; j < m; ++j) t += row[j] * hv[j];
        const double f = 2.0 * t / vv;
        for (int j = k + 1; j < m; ++j) row[j] -= f * hv[j];
      }
      __syncthreads();
      for (int i = k + 2 + tid; i < m; i += nth) Cr[(size_t)i * m + k] = 0.0;
      __syncthreads();
    }
  }
  // ---- complex copies: H = C (region 2), Z = Zr (region 3, after C is read) ----
  for (size_t e = tid; e < mm; e += nth) H[e] = make_double2(Cr[e], 0.0);
  __syncthreads();
  double hn = 0.0;
  for (size_t e = tid; e < mm; e += nth) hn += fabs(H[e].x);
  hn = block_sum(hn, red);
  for (size_t e = tid; e < mm; e += nth) Z[e] = make_double2(Zr[e], 0.0);
  if (tid == 0) sh_norm = hn > 0.0 ? hn : 1.0;
  __syncthreads();
  // ---- complex single-shift QR iteration --------------------------------
  int hi = m - 1, its = 0, total = 0;
  bool failed = false;
  while (hi > 0) {
    if (tid == 0) {
      int l = hi;
      while (l > 0) {
        double sc = zabs(H[(size_t)(l - 1) * m + l - 1]) + zabs(H[(size_t)l * m + l]);
        if (sc == 0.0) sc = sh_norm;
        if (zabs(H[(size_t)l * m + l - 1]) <= DBL_EPSILON * sc) {
          H[(size_t)l * m + l - 1] = make_double2(0.0, 0.0);
          break;
        }
        --l;
      }
      sh_l = l;
      if (l < hi) {  // shift for the active block [l, hi]
        const double2 a = H[(size_t)(hi - 1) * m + hi - 1], b = H[(size_t)(hi - 1) * m + hi];
        const double2 c = H[(size_t)hi * m + hi - 1], d = H[(size_t)hi * m + hi];
        double2 mu;
        if (its == 10 || its == 20) {  // exceptional shift
          mu = zadd(d, make_double2(zabs(c) + (hi >= 2 ? zabs(H[(size_t)(hi - 1) * m + hi - 2]) : 0.0), 0.0));
        } else {  // Wilkinson: eigenvalue of the trailing 2 x 2 closer to d
          const double2 hd = zscale(zsub(a, d), 0.5);
          const double2 disc = zsqrt(zadd(zmul(hd, hd), zmul(b, c)));
          const double2 mid = zscale(zadd(a, d), 0.5);
          const double2 e1 = zadd(mid, disc), e2 = zsub(mid, disc);
          mu = zabs(zsub(e1, d)) <= zabs(zsub(e2, d)) ? e1 : e2;
        }
        sh_mu = mu;
      }
    }
    __syncthreads();
    const int l = sh_l;
    if (l == hi) {
      --hi;
      its = 0;
      continue;
    }
    if (++total > 30 * m) {
      failed = true;
      break;
    }
    ++its;
    const double2 mu = sh_mu;
    for (int i = l + tid; i <= hi; i += nth) H[(size_t)i * m + i] = zsub(H[(size_t)i * m + i], mu);
    __syncthreads();
    // H - mu I = G^H R: rotations from the left, each on two full rows
    for (int k = l; k < hi; ++k) {
      if (tid == 0) {
        const double2 a = H[(size_t)k * m + k], b = H[(size_t)(k + 1) * m + k];
        const double na = zabs(a), nb = zabs(b);
        const double r = hypot(na, nb);
        if (r == 0.0) {
          gc[k] = 1.0;
          gs[k] = make_double2(0.0, 0.0);
        } else if (na == 0.0) {
          gc[k] = 0.0;
          gs[k] = zscale(zconj(b), 1.0 / nb);
        } else {
          gc[k] = na / r;
          gs[k] = zscale(zmul(zscale(a, 1.0 / na), zconj(b)), 1.0 / r);
        }
      }
      __syncthreads();
      const double c = gc[k];
      const double2 sn = gs[k];
      for (int j = k + tid; j < m; j += nth) {
        const double2 x = H[(size_t)k * m + j], y = H[(size_t)(k + 1) * m + j];
        H[(size_t)k * m + j] = zadd(zscale(x, c), zmul(sn, y));
        H[(size_t)(k + 1) * m + j] = zsub(zscale(y, c), zmul(zconj(sn), x));
      }
      __syncthreads();
    }
    // R G (rotations from the right) + mu I; Z <- Z G
    for (int k = l; k < hi; ++k) {
      const double c = gc[k];
      const double2 sn = gs[k];
      const int rmax = min(k + 1, hi);
      for (int i = tid; i <= rmax + m; i += nth) {
        double2 *row = i <= rmax ? H + (size_t)i * m : Z + (size_t)(i - rmax - 1) * m;
        if (i > rmax && i - rmax - 1 >= m) continue;
        const double2 x = row[k], y = row[k + 1];
        row[k] = zadd(zscale(x, c), zmul(y, zconj(sn)));
        row[k + 1] = zsub(zscale(y, c), zmul(x, sn));
      }
      __syncthreads();
    }
    for (int i = l + tid; i <= hi; i += nth) H[(size_t)i * m + i] = zadd(H[(size_t)i * m + i], mu);
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) status->breakdown = 2;
    return;
  }
  // ---- eigenvectors of the triangular T = H (thread per eigenvalue) -------
  for (int k = tid; k < m; k += nth) {
    const double2 tk = H[(size_t)k * m + k];
    const double small = DBL_EPSILON * sh_norm;
    for (int j = m - 1; j > k; --j) Yv[(size_t)j * m + k] = make_double2(0.0, 0.0);
    Yv[(size_t)k * m + k] = make_double2(1.0, 0.0);
    for (int j = k - 1; j >= 0; --j) {
      double2 sacc = make_double2(0.0, 0.0);
      for (int q = j + 1; q <= k; ++q) sacc = zadd(sacc, zmul(H[(size_t)j * m + q], Yv[(size_t)q * m + k]));
      double2 d = zsub(H[(size_t)j * m + j], tk);
      if (zabs(d) < small) d = make_double2(small, 0.0);
      Yv[(size_t)j * m + k] = zscale(zdiv(sacc, d), -1.0);
    }
    theta[k] = tk;
  }
  __syncthreads();
  // ---- u_k = W y_k (W = Z), normalised; written to Uc ----------------------
  for (size_t e = tid; e < mm; e += nth) {
    const int i = (int)(e / m), k = (int)(e % m);
    double2 t = make_double2(0.0, 0.0);
    for (int q = 0; q <= k; ++q) t = zadd(t, zmul(Z[(size_t)i * m + q], Yv[(size_t)q * m + k]));
    Uc[e] = t;
  }
  __threadfence_block();
  __syncthreads();
  for (int k = tid; k < m; k += nth) {
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) {
      const double2 u = Uc[(size_t)i * m + k];
      nrm += u.x * u.x + u.y * u.y;
    }
    nrm = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
    for (int i = 0; i < m; ++i) Uc[(size_t)i * m + k] = zscale(Uc[(size_t)i * m + k], nrm);
  }
}

// X = Q L^{-T}, AX = AQ L^{-T} on this block's rows (X written); partials per
// column j of |AX u_j - theta_j X u_j|^2, |AX u_j|^2 and the new X's column
// norm^2. blockDim = (32, 8): x over columns (j = tx, tx + 32), y over rows.
__global__ void __launch_bounds__(256)
k_update_nonsym(int n, int m, const double *__restrict__ Q, const double *__restrict__ AQ,
                const double *__restrict__ LinvT, const double2 *__restrict__ Uc,
                const double2 *__restrict__ theta, double *__restrict__ X,
                double *__restrict__ part, int rows) {
  extern __shared__ __align__(16) double sm[];
  const int RB = 8;
  // the complex tile first: 16-byte aligned for every m
  double2 *Us = reinterpret_cast<double2 *>(sm);           // m x m
  double *Ls = sm + 2 * (size_t)m * m;                     // m x m
  double *Qs = sm + 3 * (size_t)m * m;                     // RB x m
  double *As = Qs + RB * m;                                // RB x m
  double *Xs = As + RB * m;                                // RB x m (new X rows)
  double *AXs = Xs + RB * m;                               // RB x m
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  for (size_t e = tid; e < (size_t)m * m; e += 256) {
    Ls[e] = LinvT[e];
    Us[e] = Uc[e];
  }
  double e2[2] = {0.0, 0.0}, a2[2] = {0.0, 0.0}, x2[2] = {0.0, 0.0};
  const int r0 = blockIdx.x * rows;
  const int r1 = min(n, r0 + rows);
  for (int rb = r0; rb < r1; rb += RB) {
    const int nr = min(RB, r1 - rb);
    __syncthreads();
    for (int e = tid; e < RB * m; e += 256) {
      const int rr = e / m, jj = e % m;
      Qs[e] = rr < nr ? Q[(size_t)(rb + rr) * m + jj] : 0.0;
      As[e] = rr < nr ? AQ[(size_t)(rb + rr) * m + jj] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < 2; ++q) {
      const int j = tx + 32 * q;
      if (ty < nr && j < m) {
        double x = 0.0, ax = 0.0;
        for (int i = 0; i <= j; ++i) {  // L^{-T} is upper triangular
          const double l = Ls[(size_t)i * m + j];
          x = fma(Qs[ty * m + i], l, x);
          ax = fma(As[ty * m + i], l, ax);
        }
        Xs[ty * m + j] = x;
        AXs[ty * m + j] = ax;
        X[(size_t)(rb + ty) * m + j] = x;
        x2[q] = fma(x, x, x2[q]);
      }
    }
    __syncthreads();
    for (int q = 0; q < 2; ++q) {
      const int j = tx + 32 * q;
      if (ty < nr && j < m) {
        double2 xu = make_double2(0.0, 0.0), axu = make_double2(0.0, 0.0);
        for (int i = 0; i < m; ++i) {
          const double2 u = Us[(size_t)i * m + j];
          xu = zadd(xu, zscale(u, Xs[ty * m + i]));
          axu = zadd(axu, zscale(u, AXs[ty * m + i]));
        }
        const double2 d = zsub(axu, zmul(theta[j], xu));
        e2[q] += d.x * d.x + d.y * d.y;
        a2[q] += axu.x * axu.x + axu.y * axu.y;
      }
    }
  }
  __syncthreads();
  __shared__ double red[8][32];
  for (int q = 0; q < 2; ++q)
    for (int which = 0; which < 3; ++which) {
      red[ty][tx] = which == 0 ? e2[q] : (which == 1 ? a2[q] : x2[q]);
      __syncthreads();
      if (ty == 0) {
        double t = 0.0;
        for (int y = 0; y < 8; ++y) t += red[y][tx];
        const int j = tx + 32 * q;
        if (j < m) part[((size_t)blockIdx.x * 3 + which) * m + j] = t;
      }
      __syncthreads();
    }
}

// Residuals, count of Ritz values inside the circle |theta - c| < r, ||R_F||,
// the next tolerance, the new basis' column norms; lam = Re theta (one block).
__global__ void k_reduce_resid_nonsym(int Pr, int m, const double *__restrict__ part,
                                      const double2 *__restrict__ theta, double cc, double rr,
                                      double alpha, double *__restrict__ res,
                                      double *__restrict__ beta, double *__restrict__ lam,
                                      DevStatus *__restrict__ status) {
  __shared__ double smax[256];
  __shared__ int scnt[256], snan[256];
  double mx = 0.0;
  int cnt = 0, bad = 0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double e = 0.0, a = 0.0, x = 0.0;
    for (int b = 0; b < Pr; ++b) {
      e += part[((size_t)b * 3 + 0) * m + j];
      a += part[((size_t)b * 3 + 1) * m + j];
      x += part[((size_t)b * 3 + 2) * m + j];
    }
    const double r = sqrt(e) / (a > 0.0 ? sqrt(a) : 1.0);
    res[j] = r;
    beta[j] = sqrt(x);
    const double2 t = theta[j];
    lam[j] = t.x;
    if (!isfinite(r) || !isfinite(t.x) || !isfinite(t.y)) bad = 1;
    if (hypot(t.x - cc, t.y) < rr) {
      ++cnt;
      mx = fmax(mx, r);
    }
  }
  smax[threadIdx.x] = mx;
  scnt[threadIdx.x] = cnt;
  snan[threadIdx.x] = bad;
  __syncthreads();
  if (threadIdx.x == 0) {
    double M = 0.0;
    int N = 0, B = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      M = fmax(M, smax[t]);
      N += scnt[t];
      B |= snan[t];
    }
    const double RF = N > 0 ? M : 1.0;
    status->RF = RF;
    status->count = N;
    status->nonfinite = B;
    status->tol_rel = alpha > 0.0 ? alpha * RF : 0.0;
  }
}

// Ritz vectors x_q = X u_{idx[q]} (n x cap complex, row-major, cap columns)
__global__ void k_ritz_vectors_nonsym(int n, int m, const double *__restrict__ X,
                                      const double2 *__restrict__ Uc, const int *__restrict__ idx,
                                      int cnt, int cap, double2 *__restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * cnt) return;
  const int i = (int)(e / cnt), q = (int)(e % cnt);
  const int j = idx[q];
  double2 t = make_double2(0.0, 0.0);
  for (int l = 0; l < m; ++l) t = zadd(t, zscale(Uc[(size_t)l * m + j], X[(size_t)i * m + l]));
  out[(size_t)i * cap + q] = t;
}

// R = A X - X C for the carried basis X = Q L^{-T} of the non-symmetric
// iteration, from A Q of the last Rayleigh-Ritz: R = (A Q) L^{-T} - Q P with
// P = L^{-T} C (both m0 x m0, row-major). Thread (i, ty) of a (64, 4) block owns
// column i of rows blockIdx.x * 32 + ty, ty + 4, ...
__global__ void __launch_bounds__(256)
k_ns_block_residual(int n, int m0, const double *__restrict__ AQ, const double *__restrict__ Q,
                    const double *__restrict__ LinvT, const double *__restrict__ P,
                    double *__restrict__ R) {
  const int i = threadIdx.x, ty = threadIdx.y;
  if (i >= m0) return;
  for (int u = 0; u < 8; ++u) {
    const int r = blockIdx.x * 32 + ty + 4 * u;
    if (r >= n) return;
    double t = 0.0;
    for (int j = 0; j < m0; ++j)
      t = fma(AQ[(size_t)r * m0 + j], LinvT[(size_t)j * m0 + i],
              fma(-Q[(size_t)r * m0 + j], P[(size_t)j * m0 + i], t));
    R[(size_t)r * m0 + i] = t;
  }
}

}  // namespace

cudaError_t rr_init() {
  cudaError_t e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       3 * kGramRows * kMaxM0 * (int)sizeof(double));
  if (e != cudaSuccess) return e;
  e = rr_tc_init();
  if (e != cudaSuccess) return e;
  e = eig_cluster_init();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_reduced_eig_nonsym, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kNsEigSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_update_nonsym, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)((3 * kNsMaxM0 * kNsMaxM0 + 4 * 8 * kNsMaxM0) * sizeof(double)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_reduced_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kEigSmem);
}

cudaError_t rayleigh_ritz(const RRArgs &a, cudaStream_t st) {
  const int m = a.m0;
  if (m < 1 || m > kMaxM0) return cudaErrorInvalidValue;
  const int mp = (m + 3) / 4 * 4;
  // AQ = A Q
  {
    const int tiles = (m + 31) / 32;
    const int rows = (a.n + a.Pg - 1) / a.Pg;
    IFEAST_PROF_BEGIN(a.prof, K_RR_SPMM);
    k_spmm_real<<<dim3((a.n + rows - 1) / rows, tiles), kThreads, 0, st>>>(
        a.n, m, a.rowptr, a.colidx, a.val, a.Q, a.AQ, rows);
    IFEAST_PROF_END(a.prof);
    if (a.rowptrB) {
      IFEAST_PROF_BEGIN(a.prof, K_RR_SPMM);
      k_spmm_real<<<dim3((a.n + rows - 1) / rows, tiles), kThreads, 0, st>>>(
          a.n, m, a.rowptrB, a.colidxB, a.valB, a.Q, a.BQ, rows);
      IFEAST_PROF_END(a.prof);
    }
  }
  // Gram matrices: on the tensor cores (BF16 digit products, FP64-accurate,
  // k_rr_tc.cu) when the shape allows, else FP64 partials and their reduction
  if (gram_tc_group(a) > 0) {
    IFEAST_PROF_BEGIN(a.prof, K_RR_GRAM);
    cudaError_t e = gram_tc(a, st);
    IFEAST_PROF_END(a.prof);
    if (e != cudaSuccess) return e;
  } else {
    const int nt = mp / 4;
    const int ntiles = nt * (nt + 1) / 2;
    const int gy = (ntiles + kThreads - 1) / kThreads;
    const int rows = (a.n + a.Pg - 1) / a.Pg;
    const size_t smem = (a.rowptrB ? 3 : 2) * (size_t)kGramRows * mp * sizeof(double);
    IFEAST_PROF_BEGIN(a.prof, K_RR_GRAM);
    k_gram<<<dim3((a.n + rows - 1) / rows, gy), kThreads, smem, st>>>(
        a.n, m, mp, a.Q, a.AQ, a.rowptrB ? a.BQ : nullptr, a.gram_part, rows, 0);
    IFEAST_PROF_END(a.prof);
    const int pg_used = (a.n + rows - 1) / rows;
    IFEAST_PROF_BEGIN(a.prof, K_RR_GRAM_REDUCE);
    k_reduce_gram<<<(m * m + 255) / 256, 256, 0, st>>>(pg_used, m, mp, a.gram_part, a.Aq, a.Bq);
    IFEAST_PROF_END(a.prof);
  }
  // reduced eigenproblem
  {
    IFEAST_PROF_BEGIN(a.prof, K_RR_EIG);
    const cudaError_t e =
        reduced_eig_launch(m, a.Aq, a.Bq, a.L, a.Cm, a.U, a.XQ, a.lam, a.status, st);
    IFEAST_PROF_END(a.prof);
    if (e != cudaSuccess) return e;
  }
  // X = Q X_Q and residual partials: on the tensor cores (BF16 digit products,
  // FP64-accurate, k_rr_tc.cu) when the shape allows, else in FP64
  if (update_resid_tc_supported(a)) {
    const int ntiles = (a.n + 127) / 128;
    const int blocks = std::max(1, std::min(a.num_sms > 0 ? a.num_sms : 1, ntiles));
    IFEAST_PROF_BEGIN(a.prof, K_RR_UPDATE);
    cudaError_t e = update_resid_tc(a, blocks, st);
    IFEAST_PROF_END(a.prof);
    if (e != cudaSuccess) return e;
    IFEAST_PROF_BEGIN(a.prof, K_RR_RESID);
    k_reduce_resid<<<1, 256, 0, st>>>(blocks, m, a.res_part, a.lam, a.emin, a.emax, a.alpha,
                                      a.res, a.beta, a.rnorm, a.status);
    IFEAST_PROF_END(a.prof);
    return cudaGetLastError();
  }
  {
    const int rows = (a.n + a.Pr - 1) / a.Pr;
    const int pr_used = (a.n + rows - 1) / rows;
    const size_t smem = (a.rowptrB ? 3 : 2) * 8 * (size_t)m * sizeof(double);
    const double *BQ = a.rowptrB ? a.BQ : nullptr;
    const dim3 blk(32, 8);
    const int qm = (m + 31) / 32;
    IFEAST_PROF_BEGIN(a.prof, K_RR_UPDATE);
    if (qm <= 1)
      k_update_resid<1><<<pr_used, blk, smem, st>>>(a.n, m, a.Q, a.AQ, a.XQ, a.lam, a.X,
                                                     a.Rres, a.res_part, rows, BQ, a.BX);
    else if (qm <= 2)
      k_update_resid<2><<<pr_used, blk, smem, st>>>(a.n, m, a.Q, a.AQ, a.XQ, a.lam, a.X,
                                                     a.Rres, a.res_part, rows, BQ, a.BX);
    else if (qm <= 4)
      k_update_resid<4><<<pr_used, blk, smem, st>>>(a.n, m, a.Q, a.AQ, a.XQ, a.lam, a.X,
                                                     a.Rres, a.res_part, rows, BQ, a.BX);
    else
      k_update_resid<8><<<pr_used, blk, smem, st>>>(a.n, m, a.Q, a.AQ, a.XQ, a.lam, a.X,
                                                     a.Rres, a.res_part, rows, BQ, a.BX);
    IFEAST_PROF_END(a.prof);
    IFEAST_PROF_BEGIN(a.prof, K_RR_RESID);
    k_reduce_resid<<<1, 256, 0, st>>>(pr_used, m, a.res_part, a.lam, a.emin, a.emax, a.alpha,
                                      a.res, a.beta, a.rnorm, a.status);
    IFEAST_PROF_END(a.prof);
  }
  return cudaGetLastError();
}

cudaError_t reduced_eig_launch(int m, const double *Aq, const double *Bq, double *L, double *Cm,
                               double *U, double *XQ, double *lam, DevStatus *status,
                               cudaStream_t st) {
  if (m < 1 || m > kMaxM0) return cudaErrorInvalidValue;
  const size_t mat = (size_t)m * (m | 1) * sizeof(double);
  const int nmat = (int)std::min<size_t>(3, kEigSmem / mat);
  if (!eig_cluster_supported(m)) {
    k_reduced_eig<<<1, 512, nmat * mat, st>>>(m, Aq, Bq, L, Cm, U, XQ, lam, status, nmat, 0);
    return cudaGetLastError();
  }
  // C formed by one CTA, the FP64 sweeps on a cluster, the sort and X_Q by one CTA
  k_reduced_eig<<<1, 512, nmat * mat, st>>>(m, Aq, Bq, L, Cm, U, XQ, lam, status, nmat, 1);
  cudaError_t e = eig_sweeps_launch(m, Cm, lam, st);
  if (e != cudaSuccess) return e;
  k_reduced_eig<<<1, 512, 0, st>>>(m, Aq, Bq, L, Cm, U, XQ, lam, status, 0, 2);
  return cudaGetLastError();
}

cudaError_t column_norms(int n, int m, const double *X, double *part, int Pr, double *beta,
                         cudaStream_t st, Profiler *prof) {
  const int rows = (n + Pr - 1) / Pr;
  const int pr_used = (n + rows - 1) / rows;
  IFEAST_PROF_BEGIN(prof, K_NORMS);
  k_colnorm_part<<<dim3(pr_used, (m + 31) / 32), kThreads, 0, st>>>(n, m, X, part, rows);
  IFEAST_PROF_END(prof);
  IFEAST_PROF_BEGIN(prof, K_NORMS_REDUCE);
  k_reduce_norms<<<(m + 127) / 128, 128, 0, st>>>(pr_used, m, part, beta);
  IFEAST_PROF_END(prof);
  return cudaGetLastError();
}

cudaError_t spmm_block(int n, int m, const int32_t *rowptr, const int32_t *colidx,
                       const double *val, const double *X, double *Y, int P, cudaStream_t st) {
  const int rows = (n + P - 1) / P;
  k_spmm_real<<<dim3((n + rows - 1) / rows, (m + 31) / 32), kThreads, 0, st>>>(n, m, rowptr, colidx,
                                                                             val, X, Y, rows);
  return cudaGetLastError();
}

void Profiler::begin(int k) {
  ++launches[k];
  // sampling: time launch 1, 1 + N, 1 + 2N, ... of the chained Lanczos-loop kernels
  skipping = sample_every > 1 && (k == K_LZ_STEP || k == K_LZ_REDUCE || k == K_LZ_GIVENS) &&
             (launches[k] - 1) % sample_every != 0;
  if (skipping || used >= cap) return;  // pool full: the launch goes untimed
  kid[used] = k;
  cudaEventRecord(events[2 * used], stream);
}

void Profiler::end() {
  if (skipping) {
    skipping = false;
    return;
  }
  if (used >= cap) return;
  cudaEventRecord(events[2 * used + 1], stream);
  ++used;
}

int Profiler::collect_ready() {
  int done = 0;
  while (done < used && cudaEventQuery(events[2 * done + 1]) == cudaSuccess) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, events[2 * done], events[2 * done + 1]) != cudaSuccess) return 1;
    ms[kid[done]] += t;
    count[kid[done]] += 1;
    ++done;
  }
  cudaGetLastError();  // a not-ready query is not an error
  // move the pending pairs to the front (event handles are swapped, not copied)
  for (int i = done; i < used; ++i) {
    std::swap(events[2 * (i - done)], events[2 * i]);
    std::swap(events[2 * (i - done) + 1], events[2 * i + 1]);
    kid[i - done] = kid[i];
  }
  used -= done;
  return 0;
}

int Profiler::collect() {
  for (int i = 0; i < used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, events[2 * i], events[2 * i + 1]) != cudaSuccess) return 1;
    ms[kid[i]] += t;
    count[kid[i]] += 1;
  }
  used = 0;
  return 0;
}

}  // namespace ifeast

namespace ifeast {

cudaError_t rayleigh_ritz_nonsym(const RRArgs &a, const NonsymArgs &ns, cudaStream_t st) {
  const int m = a.m0;
  if (m < 1 || m > kNsMaxM0) return cudaErrorInvalidValue;
  const int mp = (m + 3) / 4 * 4;
  {
    const int tiles = (m + 31) / 32;
    const int rows = (a.n + a.Pg - 1) / a.Pg;
    IFEAST_PROF_BEGIN(a.prof, K_RR_SPMM);
    k_spmm_real<<<dim3((a.n + rows - 1) / rows, tiles), kThreads, 0, st>>>(
        a.n, m, a.rowptr, a.colidx, a.val, a.Q, a.AQ, rows);
    IFEAST_PROF_END(a.prof);
  }
  {
    const int nt = mp / 4;
    const int gy = (nt * nt + kThreads - 1) / kThreads;
    const int rows = (a.n + a.Pg - 1) / a.Pg;
    const size_t smem = 2 * (size_t)kGramRows * mp * sizeof(double);
    IFEAST_PROF_BEGIN(a.prof, K_RR_GRAM);
    k_gram<<<dim3((a.n + rows - 1) / rows, gy), kThreads, smem, st>>>(a.n, m, mp, a.Q, a.AQ,
                                                                      nullptr, a.gram_part, rows, 1);
    IFEAST_PROF_END(a.prof);
    const int pg_used = (a.n + rows - 1) / rows;
    IFEAST_PROF_BEGIN(a.prof, K_RR_GRAM_REDUCE);
    k_reduce_gram_full<<<(m * m + 255) / 256, 256, 0, st>>>(pg_used, m, mp, a.gram_part, a.Aq,
                                                            a.Bq);
    IFEAST_PROF_END(a.prof);
  }
  IFEAST_PROF_BEGIN(a.prof, K_RR_EIG);
  k_reduced_eig_nonsym<<<1, 256, 6 * (size_t)m * m * sizeof(double), st>>>(
      m, a.Aq, a.Bq, ns.LinvT, ns.theta, ns.Uc, a.status);
  IFEAST_PROF_END(a.prof);
  {
    const int rows = (a.n + a.Pr - 1) / a.Pr;
    const int pr_used = (a.n + rows - 1) / rows;
    const size_t smem = (3 * (size_t)m * m + 4 * 8 * (size_t)m) * sizeof(double);
    IFEAST_PROF_BEGIN(a.prof, K_RR_UPDATE);
    k_update_nonsym<<<pr_used, dim3(32, 8), smem, st>>>(a.n, m, a.Q, a.AQ, ns.LinvT, ns.Uc,
                                                        ns.theta, a.X, a.res_part, rows);
    IFEAST_PROF_END(a.prof);
    IFEAST_PROF_BEGIN(a.prof, K_RR_RESID);
    k_reduce_resid_nonsym<<<1, 256, 0, st>>>(pr_used, m, a.res_part, ns.theta,
                                             0.5 * (a.emin + a.emax), 0.5 * (a.emax - a.emin),
                                             a.alpha, a.res, a.beta, a.lam, a.status);
    IFEAST_PROF_END(a.prof);
  }
  return cudaGetLastError();
}

cudaError_t ns_block_residual(int n, int m0, const double *AQ, const double *Q,
                              const double *LinvT, const double *P, double *R, cudaStream_t st) {
  if (m0 < 1 || m0 > 64) return cudaErrorInvalidValue;
  k_ns_block_residual<<<(unsigned)((n + 31) / 32), dim3(64, 4), 0, st>>>(n, m0, AQ, Q, LinvT, P, R);
  return cudaGetLastError();
}

cudaError_t ritz_vectors_nonsym(int n, int m, const double *X, const double2 *Uc, const int *idx,
                                int cnt, int cap, double2 *out, cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  const size_t tot = (size_t)n * cnt;
  k_ritz_vectors_nonsym<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, m, X, Uc, idx, cnt, cap,
                                                                       out);
  return cudaGetLastError();
}

}  // namespace ifeast
