// Internal declarations shared by the CUDA translation units of libifeast.
#pragma once

#include <cuda_runtime.h>
#include <chrono>
#include <cstddef>
#include <cstdint>

#include "../../include/ifeast.h"

namespace ifeast {

constexpr int kThreads = 256;       // threads per block of the row-tiled kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxInner = 32;       // per-node GMRES basis cap (register-held dots)
constexpr int kMaxLanczos = 4096;   // shared-basis (MINRES) step cap
constexpr int kMaxNodes = 64;
constexpr int kMaxM0 = 256;         // reduced problem solved in one CTA

// Kernel classes timed by the optional profiler (CUDA events around launches).
enum KernelId {
  K_PREP = 0,      // basis start and least-squares state reset
  K_NORMS,         // column-norm partials
  K_NORMS_REDUCE,  // column-norm reduction
  K_GM_SPMM,       // per-node GMRES: shifted SpMM + first-pass dots
  K_GM_REDUCE,     // per-node GMRES: fixed-order partial reductions
  K_GM_ORTH,       // per-node GMRES: Gram-Schmidt update + second-pass dots
  K_GM_GIVENS,     // per-node GMRES: Hessenberg column, Givens, stop test
  K_GM_FINISH,     // per-node GMRES: next basis vector
  K_GM_SOLVE,      // per-node GMRES: back substitution
  K_GM_QUAD,       // per-node GMRES: quadrature sum
  K_LZ_STEP,       // shared basis: Lanczos step (SpMM + dots)
  K_LZ_GIVENS,     // shared basis: reduction + per-node Givens
  K_LZ_SOLVE,      // shared basis: back substitution
  K_LZ_COEF,       // shared basis: quadrature coefficients
  K_LZ_QUAD,       // shared basis: quadrature sum over the basis
  K_RR_SPMM,       // Rayleigh-Ritz: A Q
  K_RR_GRAM,       // Rayleigh-Ritz: Q^T A Q, Q^T Q partials
  K_RR_GRAM_REDUCE,// Rayleigh-Ritz: partial reduction
  K_RR_EIG,        // reduced generalised eigenproblem (one CTA)
  K_RR_UPDATE,     // X = Q X_Q and residual partials
  K_RR_RESID,      // residuals, interval count, ||R_F||
  K_LZ_REDUCE,     // shared basis, FP32 steps: alpha_s, beta_{s+1} from the step's partials
  K_COUNT
};

struct Profiler {
  cudaStream_t stream = nullptr;
  cudaEvent_t *events = nullptr;  // pool of 2 * cap events
  int cap = 0, used = 0;
  int *kid = nullptr;             // kernel class of each pending pair
  double ms[K_COUNT] = {0};
  long long count[K_COUNT] = {0};     // timed launches
  long long launches[K_COUNT] = {0};  // all launches
  // > 1: only every sample_every-th launch of the Lanczos step, coefficient
  // and Givens kernels is timed (events between them stop their programmatic
  // overlap)
  int sample_every = 1;
  bool skipping = false;
  void begin(int k);
  void end();
  int collect();                  // after a stream synchronisation
  int collect_ready();            // the leading pairs that have completed
};
#define IFEAST_PROF_BEGIN(p, k) \
  do {                          \
    if (p) (p)->begin(k);       \
  } while (0)
#define IFEAST_PROF_END(p) \
  do {                     \
    if (p) (p)->end();     \
  } while (0)

// Device-side record read back by the host once per outer iteration.
struct DevStatus {
  double RF;            // max relative residual over Ritz values inside the interval
  double tol_rel;       // alpha * RF for the next inner solve (0: fixed-k)
  int count;            // Ritz values inside (emin, emax)
  int breakdown;        // reduced eigensolver: 1 = B_Q not factorable
  int shifted;          // reduced eigensolver: 1 = B_Q needed the diagonal shift
  int max_steps;        // max Krylov steps over (node, column) in the last filter
  long long total_steps;// sum of Krylov steps over (node, column) in the last filter
  int nonfinite;        // a NaN/Inf was seen in the residuals
  int tc_timeout;       // tensor-core update: a bounded wait on the MMA completion ran out
};

// Row-tiled launch geometry for n x C blocks: grid (P, tiles), warp w of a
// block handles rows r0 + w, r0 + w + kWarps, ... of its chunk of rows.
struct RowTiling {
  int P;            // row chunks
  int rows;         // rows per chunk
  int tiles;        // 32-column tiles
};
RowTiling make_tiling(int64_t n, int ncols, int num_sms);

// ---- inner solve (per-node complex GMRES, FP64 or FP32) -------------------
struct GmresArgs {
  int n, m0, nc, C, K;
  int ncc;                  // nodes per inner pass: the filter runs nc / ncc passes of
                            // ncc nodes (C = ncc * m0 columns each), summing their Q
  int fp32;                 // 1: basis and work vector complex FP32, FP32 arithmetic
  const int32_t *rowptr, *colidx;
  const double *val;
  const float *val32;       // FP32 copy of val (fp32)
  const double2 *z;         // [nc]
  const double2 *w;         // [nc] quadrature weights
  const double *X;          // n x m0 right-hand sides (real): X, B X, or the residuals
  void *V;                  // (K+1) x n x C basis (double2, or float2 when fp32)
  void *W;                  // n x C work vector (same type as V)
  double2 *part;            // P x (K+2) x C block partials
  double2 *H1;              // (K+1) x C first-pass coefficients of the current step
  double2 *H2;              // (K+1) x C second-pass coefficients of the current step
  double *inv_h;            // C     1 / h_{s+1,s}
  double2 *CS, *SN;         // K x C Givens rotations
  double2 *R;               // K x K x C triangular factor, R[(l*K + s)*C + c]
  double2 *G;               // (K+1) x C rotated right-hand side
  double2 *Y;               // K x C weighted least-squares solutions
  float2 *Yf;               // K x C FP32 copy of Y (fp32 quadrature)
  double *beta;             // m0 norms of the right-hand sides
  double *tolc;             // C   bound on |g_{s+1}| (0: run all K steps)
  int *steps;               // C   Krylov steps taken
  int *done;                // C   column finished (tolerance met or breakdown)
  double *Q;                // n x m0 output
  DevStatus *status;        // tol_rel read from here, step counts written here
  RowTiling tl;
  Profiler *prof;
  const int32_t *rowptrB, *colidxB;  // B of A x = lambda B x (null: B = I)
  const double *valB;
  const float *valB32;      // FP32 copy of valB (fp32)
  int b_same_pattern;       // 1: B has A's rowptr/colidx (valB indexed like val)
  // residual form: right-hand sides r_j = A x_j - lambda_j B x_j (in X, norms in
  // beta), y = (x_j + e) / (z_k - lambda_j), Q = cx X + Re sum_k w_k e_k / (z_k - lambda_j)
  // (correction = 1). Block correction for non-symmetric A (correction = 2):
  // right-hand sides R = A X - X C (C = X^T A X, X orthonormal), E_k the
  // weighted solutions w_k (z_k I - A)^{-1} R, and
  // Q = X Re(sum_k w_k M_k) + Re sum_k E_k M_k with M_k = (z_k I - C)^{-1}
  int correction;
  const double2 *ns_M;      // correction = 2: [nc][m0][m0] M_k (row-major)
  const double *ns_Gre;     // correction = 2: m0 x m0 Re sum_k w_k M_k
  const double *ns_X;       // correction = 2: n x m0 the orthonormal basis X
  int accumulate;           // 1: Q += this pass's sum (later node chunks)
  int stream_tma;           // 1: FP32 basis kernels stream the basis by TMA (when C is even)
  const double *lam;        // [m0] Ritz values
  const double *xnorm;      // [m0] ||B x_j||
  const double *Xr;         // n x m0 the Ritz vectors x_j
  double *cx;               // [m0] Re sum_k w_k / (z_k - lambda_j)
};
cudaError_t gmres_filter(const GmresArgs &a, cudaStream_t st);
cudaError_t gmres_init();  // once per device: opt-in shared-memory sizes
cudaError_t spmm_shift_only(int n, const int32_t *rowptr, const int32_t *colidx,
                            const double *val, const double2 *V, double2 *W, int ncols,
                            int m0, const double2 *z, RowTiling tl, cudaStream_t st,
                            const int32_t *rowptrB, const int32_t *colidxB, const double *valB);

// ---- inner solve on one shared Lanczos basis per column (FP32 or FP64) ----
struct MinresState {
  const double2 *z, *w;     // [nc] nodes and weights
  const double *lam;        // [m0] Ritz values (residual form)
  const double *xnorm;      // [m0] ||x_j||
  int correction;           // 1: right-hand side is A x_j - lambda_j x_j
  double2 *g;               // [nc*m0][K+1] rotated right-hand sides
  double2 *R;               // [nc*m0][K][3] band of the triangular factor
  double2 *rot;             // [nc*m0][4] last two Givens rotations
  double *tol;              // [nc*m0] bound on |g_{s+1}|
  int *steps;               // [nc*m0]
  int *done;                // [nc*m0]
  int *coldone;             // [m0] column finished (all pairs done, or a breakdown)
  int *ndone;               // [m0] pairs of the column done (FP32 step kernels)
  int *active;              // [1] columns still running at the last checked step
  DevStatus *status;
};
// Second pass of the two-pass (memory-bounded) shared-basis mode: the basis
// is rebuilt from the stored alpha, beta and Q accumulates coef_s v_s.
struct Pass2 {
  float *Qacc;              // n x m0 FP32 accumulator (null: not the second pass)
  const float *cf;          // FP32 coefficients [K][m0]
  const int *Sj;            // second pass: column j takes the steps s < Sj[j]
  int vring;                // 0: basis slot s; 3: slot s % 3 (two-pass mode)
};

// Early exit of the Lanczos loop: the flag of checkpoint c is read after
// checkpoint c + kCheckLag has been enqueued, so the stream never drains.
constexpr int kCheckLag = 2;

struct MinresArgs {
  int n, m0, nc, K;
  int fp32;                 // FP32 arithmetic in the Krylov kernels
  int half;                 // FP16 storage of the Krylov vectors (with fp32)
  int bf16;                 // BF16 storage of the Krylov vectors (with fp32)
  float wscale;             // FP16: w_s is stored as w_s / wscale (||A||_inf); else 1
  const int32_t *rowptr, *colidx;
  const void *val_t;        // float or double values of A
  const double *rhs;        // n x m0 right-hand sides (X or A X - X Lambda)
  const double *rnorm;      // [m0] their norms
  const double *X;          // n x m0 current subspace (residual-form term)
  void *V, *W0, *W1;        // basis and double-buffered work vectors (T)
  double *part;             // P x 3 x m0
  double *alpha, *beta;     // [K][m0], [K+1][m0]
  float4 *cf32;             // [K+1][m0] FP32 {alpha_{s-1}, beta_s, 1/beta_s, 0} for step s
  double2 *Yc;              // [nc][K][m0]
  double2 *wt;              // [nc][m0] quadrature weight of each (node, column) pair
  double *coef, *cx;        // [K][m0] (+ an FP32 copy after it), [m0]
  int *Sj;                  // [m0]
  double *Q;
  RowTiling tl;
  MinresState ms;
  int check_every;          // steps between early-exit checks (0: never)
  int *active_host;         // pinned, kCheckLag + 1 slots
  cudaEvent_t *check_events;  // kCheckLag + 1 events
  Profiler *prof;
  int P_async;              // max blocks of the FP32 (row, quad) step kernel
  int ell_w;                // 8 or 16: fixed-width copy of A available (FP32), else 0
  const int32_t *colE;      // n x ell_w indices (padded with the row's own index)
  const float *valE;        // n x ell_w values (padded with zero)
  int two_pass;             // 1: three basis slots and a second pass (FP32 kernels only)
  float *Qf;                // n x m0 FP32 accumulator of the second pass
  // wall-time limit, checked at the lagged early-exit checks of the Lanczos
  // loop: past it the loop stops (the filter uses the steps run) and *cut is set
  std::chrono::steady_clock::time_point t0{};
  double time_limit_ms = 0.0;  // <= 0: none
  bool *cut = nullptr;
};
cudaError_t build_ell(int n, int W, const int32_t *rowptr, const int32_t *colidx, const float *val,
                      int32_t *colE, float *valE, cudaStream_t st);
cudaError_t minres_init();  // once per device: opt-in shared-memory sizes
cudaError_t minres_filter(const MinresArgs &a, cudaStream_t st);
cudaError_t convert_to_float(const double *a, float *b, size_t n, cudaStream_t st);

// X (n x m0 row-major) = i.i.d. N(0,1) from Philox4x32-10 blocks keyed by seed
// (element pair 2p, 2p+1 from counter p, Box-Muller; layout in ifeast.h).
cudaError_t seeded_normal(int64_t n, int m0, uint64_t seed, double *X, cudaStream_t st);
// R = A X - BX diag(lam) for n x m0 row-major blocks (BX = X for B = I), FP64.
cudaError_t residual_block(int n, int m0, const int32_t *rowptr, const int32_t *colidx,
                           const double *val, const double *X, const double *BX,
                           const double *lam, double *R, cudaStream_t st);

// ---- Rayleigh-Ritz and residual -------------------------------------------
struct RRArgs {
  int n, m0;
  const int32_t *rowptr, *colidx;
  const double *val;
  const double *Q;          // n x m0
  double *AQ;               // n x m0
  double *gram_part;        // Pg x 2 x m0p x m0p
  int Pg;
  double *Aq, *Bq;          // m0 x m0
  double *L;                // m0 x m0 scratch (Cholesky factor)
  double *Cm;               // m0 x m0 scratch (reduced standard matrix / Jacobi)
  double *U;                // m0 x m0 scratch (Jacobi eigenvectors)
  double *XQ;               // m0 x m0 B_Q-orthonormal eigenvectors
  double *lam;              // m0 ascending
  double *X;                // n x m0 new subspace
  double *res_part;         // Pr x 3 x m0
  int Pr;
  double *res;              // m0
  double *beta;             // m0 norms of the new X columns
  double *Rres;             // n x m0 A X - X Lambda of the new X (nullptr: not stored)
  double *rnorm;            // m0 ||A x_j - lambda_j x_j|| (nullptr: not stored)
  const int32_t *rowptrB, *colidxB;  // B of A x = lambda B x (null: B = I)
  const double *valB;
  double *BQ;               // n x m0 B Q (generalized only)
  double *BX;               // n x m0 B X of the new X (generalized only); beta = ||B x_j||
  double emin, emax, alpha;
  DevStatus *status;
  Profiler *prof;
  int num_sms;              // persistent grids (tensor-core update)
};
// Non-Hermitian extension (real non-symmetric A, m0 <= 64)
struct NonsymArgs {
  double *LinvT;            // m0 x m0: the carried basis is X = Q L^{-T}
  double2 *theta;           // [m0] Ritz values (unordered)
  double2 *Uc;              // m0 x m0 unit eigenvectors of C = L^{-1} Q^T A Q L^{-T}
};
cudaError_t rayleigh_ritz_nonsym(const RRArgs &a, const NonsymArgs &ns, cudaStream_t st);
// R = (A Q) L^{-T} - Q P (m0 <= 64): the block residual A X - X C of X = Q L^{-T}
// with P = L^{-T} C, right-hand sides of the non-symmetric block correction
cudaError_t ns_block_residual(int n, int m0, const double *AQ, const double *Q,
                              const double *LinvT, const double *P, double *R, cudaStream_t st);
cudaError_t ritz_vectors_nonsym(int n, int m, const double *X, const double2 *Uc, const int *idx,
                                int cnt, int cap, double2 *out, cudaStream_t st);
constexpr int kNonsymMaxM0 = 64;
cudaError_t rr_init();  // once per device: opt-in shared-memory sizes
// Tensor-core (tcgen05, BF16 digit products) form of the Rayleigh-Ritz update
// X = Q X_Q, AX = AQ X_Q with the residual partials (k_rr_tc.cu); supported for
// m0 <= 80, B = I, n >= 128. blocks: persistent CTAs (one per SM at most).
bool update_resid_tc_supported(const RRArgs &a);
cudaError_t update_resid_tc(const RRArgs &a, int blocks, cudaStream_t st);
cudaError_t rr_tc_init();
// FP64 Jacobi sweeps of the reduced eigenproblem on a thread-block cluster
// (k_eig_cluster.cu): C (m x m, row-major) in place -> its eigenvectors V,
// unsorted eigenvalues in evals
bool eig_cluster_supported(int m);
cudaError_t eig_cluster_init();
cudaError_t eig_sweeps_launch(int m, double *C, double *evals, cudaStream_t st);
// Tensor-core Gram matrices A_Q = Q^T A Q, B_Q = Q^T Q (B = I, m0 <= 80):
// gram_tc_group > 0 when supported (CTAs per 48-column chunk); gram_tc writes
// Aq and Bq (symmetric) through the Gram partials buffer.
int gram_tc_group(const RRArgs &a);
cudaError_t gram_tc(const RRArgs &a, cudaStream_t st);
cudaError_t rayleigh_ritz(const RRArgs &a, cudaStream_t st);
cudaError_t column_norms(int n, int m0, const double *X, double *part, int Pr, double *beta,
                         cudaStream_t st, Profiler *prof);
// Y = A X for an n x m0 real block (one row-tiled sparse product).
cudaError_t spmm_block(int n, int m0, const int32_t *rowptr, const int32_t *colidx,
                       const double *val, const double *X, double *Y, int P, cudaStream_t st);
// The reduced generalised eigensolver of rayleigh_ritz on caller buffers.
cudaError_t reduced_eig_launch(int m, const double *Aq, const double *Bq, double *L, double *Cm,
                               double *U, double *XQ, double *lam, DevStatus *status,
                               cudaStream_t st);

}  // namespace ifeast
