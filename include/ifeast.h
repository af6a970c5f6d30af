/*
 * ifeast.h -- C ABI of the GB300 (sm_103a) IFEAST hot path.
 *
 * IFEAST (Gavin & Polizzi, arXiv 1706.00692, Algorithm 2) finds the eigenpairs
 * (lambda, x) of a real symmetric sparse matrix A whose eigenvalues lie in an
 * interval (emin, emax). Each outer (subspace) iteration
 *   1. solves the shifted systems (z_k I - A) Y_k = X for every contour node z_k
 *      and every one of the m0 columns of X, inexactly, with a few Krylov
 *      (GMRES) steps                                         [Alg. 2 step 1]
 *   2. forms the filtered subspace Q = sum_k w_k Y_k         [Alg. 2 step 2]
 *   3. Rayleigh-Ritz: A_Q X_Q = B_Q X_Q Lambda, A_Q = Q^T A Q, B_Q = Q^T Q,
 *      X <- Q X_Q                                            [Alg. 2 step 3]
 *   4. stops once the largest relative residual ||A x_j - lambda_j x_j|| /
 *      ||A x_j|| over lambda_j in (emin, emax) is <= tol    [Alg. 2 step 4]
 * All four steps run in CUDA kernels of this library on one GPU. The host only
 * validates arguments, launches kernels and reads back one small status record
 * per outer iteration.
 *
 * Conventions
 *   - Every function returns an ifeast_status code (0 = success) unless noted.
 *   - Dense blocks are row-major: an n x m0 block stores row i at [i*m0, i*m0+m0).
 *   - CSR: rowptr int32[n+1] (rowptr[0] = 0, non-decreasing), colidx int32[nnz]
 *     in [0, n), val float64[nnz]. Pointers in ifeast_csr are HOST pointers;
 *     ifeast_create copies the matrix to device memory owned by the handle, so
 *     the caller may free its arrays when ifeast_create returns.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).
 *   - A handle is not thread-safe; distinct handles may run on distinct streams.
 */
#ifndef IFEAST_H
#define IFEAST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IFEAST_OK = 0,
  IFEAST_ERR_INVALID_ARG = 1,    /* bad CSR, m0 <= 0, emin >= emax, nc < 1, ...   */
  IFEAST_ERR_OOM = 2,            /* workspace larger than given / device memory  */
  IFEAST_ERR_CUDA = 3,           /* a CUDA runtime call failed                   */
  IFEAST_ERR_NOT_CONVERGED = 4,  /* max_outer reached; best pairs retrievable    */
  IFEAST_ERR_M0_TOO_SMALL = 5,   /* m0 Ritz values inside the interval: m0 <= m  */
  IFEAST_STATUS_NO_EIGENVALUES = 6, /* no Ritz value inside the interval         */
  IFEAST_ERR_BREAKDOWN = 7,      /* B_Q not positive definite even after a shift */
  IFEAST_ERR_TIMEOUT = 8,        /* opts.time_limit_ms ran out (last iterate kept),
                                    or a bounded device-side wait of the tensor-core
                                    Rayleigh-Ritz update ran out (iterate invalid)  */
  IFEAST_ERR_STATE = 9,          /* call out of order (e.g. eigenpairs before solve) */
  IFEAST_ERR_UNSUPPORTED = 10    /* option combination not built                 */
} ifeast_status;

/* Quadrature rules on the circle centred at c = (emin+emax)/2 with radius
 * r = (emax-emin)/2 (Eq. contour_int_quad; half-contour symmetry of Sec. 4.1):
 *   GL_HALF   nc Gauss-Legendre nodes on the upper half circle, filter taken
 *             as 2 Re of the upper-half sum
 *   TRAP_HALF nc trapezoid nodes theta_j = pi (j-1/2)/nc on the upper half
 *   TRAP_FULL nc trapezoid nodes theta_j = 2 pi (j-1/2)/nc on the full circle
 *             (nc even). A is real and X real, so the solutions at conjugate
 *             nodes are conjugate: the library runs the equal TRAP_HALF sum
 *             over the nc/2 upper nodes.                                     */
/*   USER      nc caller-given nodes and weights (ifeast_contour.user_zw). The
 *             library forms the filter as Re sum_k w_k / (z_k - lambda) like
 *             the *_HALF rules, so a rule for a real problem is given by its
 *             upper-half nodes with the factor 2 of the mirrored lower half
 *             folded into the weights (the form ifeast_contour_nodes returns).
 *             Every node needs Im z_k != 0 (a real node can hit the spectrum). */
typedef enum {
  IFEAST_GL_HALF = 0,
  IFEAST_TRAP_HALF = 1,
  IFEAST_TRAP_FULL = 2,
  IFEAST_USER = 3
} ifeast_rule;

/* Inner solver for Alg. 2 step 1.
 *   GMRES:  one complex GMRES per (node, column) pair, zero initial guess,
 *           classical Gram-Schmidt applied twice, Givens least squares
 *           (Sec. 2.2). inner_max_iters <= 32. FP64, or FP32 (FP32 basis;
 *           with the residual form below opts.correction_rf).
 *   MINRES: one real Lanczos basis per column of X, shared by all nc shifts
 *           (Sec. 3: the Krylov basis of (z I - A) does not depend on z); each
 *           (node, column) pair takes the minimal-residual solution on it
 *           (MINRES for the shifted Hermitian systems, Sec. 2) and stops on
 *           its own tolerance. From the second outer iteration on, each shifted
 *           system is solved in residual form: with r_j = A x_j - lambda_j x_j,
 *           (z I - A)^{-1} x_j = (x_j + (z I - A)^{-1} r_j) / (z - lambda_j),
 *           an identity, so the same Alg. 2 stop test applies while the Krylov
 *           solve only has to resolve r_j (this lets FP32 inner arithmetic
 *           reach FP64 eigenpair accuracy). inner_max_iters <= 4096.        */
typedef enum { IFEAST_INNER_GMRES = 0, IFEAST_INNER_MINRES = 1 } ifeast_inner;

/* Arithmetic of the inner solve (Krylov vectors, sparse products and their
 * inner products; FP32 with either inner solver, FP16 and BF16 with
 * IFEAST_INNER_MINRES only; FP32 GMRES needs a symmetric A, since its residual
 * form takes real Ritz pairs).
 *   FP64: FP64 vectors and arithmetic.
 *   FP32: FP32 vectors and arithmetic.
 *   FP16: FP16 storage of the Lanczos vectors (half the bytes of FP32),
 *         FP32 arithmetic; needs m0 % 4 == 0. The work vectors are stored
 *         scaled by 1/||A||_inf to stay in FP16 range.
 *   BF16: BF16 storage of the Lanczos vectors (8-bit exponent, so no
 *         scaling), FP32 arithmetic; needs m0 % 4 == 0.
 * The quadrature weights, least-squares updates, reduced eigenproblem,
 * Rayleigh-Ritz products and residual check are FP64 in every mode. */
typedef enum { IFEAST_FP64 = 0, IFEAST_FP32 = 1, IFEAST_FP16 = 2, IFEAST_BF16 = 3 } ifeast_precision;

typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t *rowptr;
  const int32_t *colidx;
  const double *val;
} ifeast_csr;

typedef struct {
  int rule;       /* ifeast_rule                        */
  int nc;         /* number of nodes (upper half for *_HALF rules) */
  double emin;    /* interval (emin, emax), open; the wanted eigenvalues, and
                     the circle of the built-in rules                        */
  double emax;
  const double *user_zw; /* IFEAST_USER only (else ignored): host array of nc x
                     {Re z_k, Im z_k, Re w_k, Im w_k}, copied by ifeast_create */
} ifeast_contour;

typedef struct {
  int inner_solver;     /* ifeast_inner                                         */
  int inner_max_iters;  /* k: Krylov steps per shifted system                   */
  double alpha;         /* > 0: stop a shifted solve once ||x_j - (z_k I - A) y||
                           <= alpha * ||R_F|| * ||x_j|| (Alg. 2 step 1; ||R_F||=1
                           before the first iteration); <= 0: always k steps      */
  int max_outer;        /* outer iteration cap (default 100)                     */
  double tol;           /* stop when ||R_F|| <= tol (default 1e-10)              */
  int precision;        /* ifeast_precision                                      */
  int verbose;          /* 1: one line per outer iteration on stderr             */
  int nonsymmetric;     /* 1: A is real non-symmetric (non-Hermitian extension,
                           stated without steps in the paper): Galerkin
                           Rayleigh-Ritz on span(Q) with a general reduced
                           eigensolver, complex Ritz values, a value counts when
                           it lies inside the circle |lambda - c| < r of the
                           contour, eigenpairs through ifeast_eigenpairs_complex.
                           Needs IFEAST_INNER_GMRES, B = NULL, m0 <= 64.       */
  int minres_two_pass;  /* 1 (IFEAST_INNER_MINRES with FP32 or FP16, m0 % 4 == 0):
                           keep three Lanczos vectors instead of the whole basis.
                           A first pass runs the Lanczos and Givens steps; a
                           second pass rebuilds v_0 .. v_{S-1} from the stored
                           alpha, beta with the same arithmetic and accumulates
                           the quadrature on the fly, so Q is bit-identical to
                           the stored-basis mode. Workspace O(n m0) instead of
                           O(inner_max_iters n m0); about twice the inner time. */
  double correction_rf; /* IFEAST_INNER_GMRES with IFEAST_FP32 only: once ||R_F|| of
                           the previous iteration is <= correction_rf, the shifted
                           systems are solved for the correction of the current
                           Ritz pairs, (z B - A) e = A x_j - lambda_j B x_j, and
                           y = (x_j + e) / (z - lambda_j) (an identity of the
                           shifted systems; it lets FP32 inner solves reach FP64
                           eigenpair residuals). Default 1e-3; 1 or more: from
                           the second iteration on.                            */
  double time_limit_ms; /* > 0: ifeast_solve stops once this much wall time has
                           passed: between outer iterations, and inside the
                           Lanczos loop at its lagged early-exit checks (the
                           filter then uses the steps run so far), followed by
                           that iteration's Rayleigh-Ritz. It returns
                           IFEAST_ERR_TIMEOUT with the last iterate kept (pairs
                           retrievable as after NOT_CONVERGED). <= 0: no limit. */
  int node_chunk;       /* IFEAST_INNER_GMRES: > 0 solves the shifted systems of
                           node_chunk contour nodes at a time (nc of the rule run
                           must be a multiple of it), summing their parts of Q:
                           the per-node Krylov bases then need node_chunk * m0
                           columns of workspace instead of nc * m0. The result
                           equals the all-nodes filter (same kernels, same
                           arithmetic per system). 0: all nodes at once.      */
  int plain_loads;      /* IFEAST_INNER_GMRES with IFEAST_FP32: 1 reads the
                           basis in the dot, Gram-Schmidt and finish kernels
                           with plain loads; 0 (default) streams it through
                           shared memory by TMA tile copies when the system
                           count of a pass is even (same arithmetic, same
                           results bit for bit).                              */
  int nonsym_correction; /* nonsymmetric == 1: 1 solves, from the second outer
                           iteration on, the shifted systems for the block
                           residual R = A X - X C of the orthonormal basis X
                           and its Galerkin matrix C = X^T A X, and forms
                           Q = Re sum_k w_k (X + E_k)(z_k I - C)^-1 with
                           (z_k I - A) E_k = R: the identity
                           (zI - A)^-1 X = [X + (zI - A)^-1 R](zI - C)^-1 is
                           exact, and the inner error then falls with ||R||
                           (plain form: with ||X||). Inner stop |g_{s+1}| <=
                           alpha ||R_F||. 0 (default): the plain form. Needs
                           m0 <= 64 and the FP64 basis.                       */
} ifeast_opts;

typedef struct {
  int outer_iters;            /* outer iterations run by the last solve        */
  int found;                  /* Ritz values inside (emin, emax)               */
  double RF;                  /* last ||R_F|| (max relative residual inside)   */
  int64_t total_matvecs;      /* sum over iterations of all (node, column) Krylov steps */
  int64_t seq_matvecs;        /* sum over iterations of the max steps of any (node, column) */
  int max_inner;              /* largest per-(node, column) step count seen    */
  int shifted_cholesky;       /* times B_Q needed the diagonal shift           */
  double solve_ms;            /* wall time of the last ifeast_solve (host clock) */
} ifeast_stats_t;

/* Fills *o with the defaults: GMRES, k = 10, alpha = 0 (fixed k), max_outer =
 * 100, tol = 1e-10, FP64, verbose = 0, correction_rf = 1e-3, no time limit,
 * node_chunk = 0, plain_loads = 0. */
void ifeast_default_opts(ifeast_opts *o);

/* Contour nodes and weights (Eq. contour_int_quad with the rules above) on the
 * host: zw[4*k + {0,1,2,3}] = {Re z_k, Im z_k, Re w_k, Im w_k}, k < c->nc. For
 * *_HALF rules the weights already include the factor 2 of the conjugate
 * lower half, so the filter is rho(lambda) = Re sum_k w_k / (z_k - lambda).
 * IFEAST_USER: the given nodes, validated (finite, Im z_k != 0). */
int ifeast_contour_nodes(const ifeast_contour *c, double *zw);

/* Device bytes a handle needs for (n, nnz, m0, contour, opts), B = I. */
int ifeast_workspace_bytes(int64_t n, int64_t nnz, int m0, const ifeast_contour *c,
                           const ifeast_opts *o, size_t *bytes);

/* Same for the generalized problem A x = lambda B x with nnz_b non-zeros in
 * B (nnz_b < 0: B = I). B != I needs IFEAST_INNER_GMRES (else UNSUPPORTED). */
int ifeast_workspace_bytes_generalized(int64_t n, int64_t nnz, int64_t nnz_b, int m0,
                                       const ifeast_contour *c, const ifeast_opts *o,
                                       size_t *bytes);

typedef struct ifeast_ctx *ifeast_t;

/* Validates A (square, rowptr[0] = 0, non-decreasing rowptr, rowptr[n] = nnz,
 * colidx in range), computes the contour on the host, lays out the workspace
 * and copies A into it.
 *   B          NULL: standard problem (B = I). Otherwise the symmetric positive
 *              definite B of A x = lambda B x (host CSR, same n, any pattern;
 *              definiteness is not checked): the shifted systems become
 *              (z_k B - A) Y_k = B X (Section 2.2), B_Q = Q^T B Q, the Ritz
 *              vectors are B-orthonormal and the residual is
 *              ||A x - lambda B x|| / ||A x||. Needs IFEAST_INNER_GMRES (the
 *              Krylov basis of z B - A depends on z) and the GMRES stop test
 *              is taken relative to ||B x_j||.
 *   workspace  device buffer of ws_bytes >= ifeast_workspace_bytes(...) that
 *              the caller keeps alive until ifeast_destroy; NULL makes the
 *              library cudaMalloc (and later cudaFree) its own.
 *   stream     cudaStream_t (as void*) for every later call on this handle.
 * On error *out is NULL and nothing stays allocated. */
int ifeast_create(const ifeast_csr *A, const ifeast_csr *B, const ifeast_contour *c, int m0,
                  const ifeast_opts *o, void *workspace, size_t ws_bytes, void *stream,
                  ifeast_t *out);

/* Runs Algorithm 2 from the initial subspace X0 (n x m0, row-major float64;
 * x0_on_device != 0: device pointer, else host pointer, copied in). X0 = NULL
 * starts from a random subspace (Alg. 1 input: "random" X^(0)) drawn on the
 * device from seed, as ifeast_initial_subspace below. stream: the
 * cudaStream_t (as void*) this solve runs on; NULL: the stream given to
 * ifeast_create. Returns OK on convergence, NOT_CONVERGED after max_outer
 * iterations (the last iterate is kept), TIMEOUT once opts.time_limit_ms has
 * run out (likewise), M0_TOO_SMALL if all m0 Ritz values fall inside the
 * interval, NO_EIGENVALUES if none does, BREAKDOWN if B_Q cannot be factored.
 * Blocks the calling host thread until the solve ends. */
int ifeast_solve(ifeast_t h, const double *X0, int x0_on_device, uint64_t seed, void *stream);

/* The seeded random subspace of ifeast_solve(X0 = NULL): X (n x m0 row-major
 * float64, DEVICE, caller-owned) gets i.i.d. N(0, 1) values. Element pair
 * e = 2p, 2p + 1 (row-major index) comes from one Philox4x32-10 block
 * (Salmon et al., SC'11) with counter (p mod 2^32, p div 2^32, 0, 0) and key
 * (seed mod 2^32, seed div 2^32): its words x0..x3 give the 53-bit uniforms
 * u1 = (2^26 (x0 >> 5) + (x1 >> 6) + 1) 2^-53 in (0, 1] and
 * u2 = (2^26 (x2 >> 5) + (x3 >> 6)) 2^-53 in [0, 1), and Box-Muller gives
 * X[2p] = sqrt(-2 ln u1) cos(2 pi u2), X[2p + 1] = sqrt(-2 ln u1) sin(2 pi u2).
 * Runs on stream and returns when it finished. INVALID_ARG for n < 1, m0 < 1
 * or X = NULL. */
int ifeast_initial_subspace(int64_t n, int m0, uint64_t seed, double *X, void *stream);

/* Copies the Ritz pairs with lambda inside (emin, emax), ascending:
 * evals[m], evecs (n x cap row-major: column j of the block is the j-th pair,
 * row i at evecs[i*cap + j]), resid[m] relative residuals. Any output pointer
 * may be NULL. *m_found gets the number inside (may exceed cap; then only the
 * first cap are copied). out_on_device != 0: outputs are device pointers. */
/* Non-symmetric handles (opts.nonsymmetric = 1): the Ritz pairs inside the
 * circle |lambda - c| < r, ordered by real part, the two values of a complex
 * conjugate pair adjacent with the negative imaginary part first (the pair
 * shares one real-part key, the mean of its two computed real parts). evals: 2*cap
 * doubles (re, im); evecs: n x cap complex (re, im interleaved, row-major,
 * unit 2-norm); resid: cap relative residuals ||A x - lambda x|| / ||A x||.
 * Host or device outputs as ifeast_eigenpairs; any may be NULL.
 * ifeast_eigenpairs returns UNSUPPORTED for such handles. */
int ifeast_eigenpairs_complex(ifeast_t h, int cap, int *m_found, double *evals, double *evecs,
                              double *resid, int out_on_device);

int ifeast_eigenpairs(ifeast_t h, int cap, int *m_found, double *evals, double *evecs,
                      double *resid, int out_on_device);

/* All m0 Ritz values of the last iterate (ascending) and their residuals;
 * device or host pointers as flagged. */
int ifeast_ritz_all(ifeast_t h, double *lam, double *resid, int out_on_device);

/* Counters of the last ifeast_solve. */
int ifeast_stats(ifeast_t h, ifeast_stats_t *s);

/* Human-readable name of a status code (static storage). */
const char *ifeast_strerror(int code);

/* Frees every device buffer the handle allocated; NULL is allowed. */
void ifeast_destroy(ifeast_t h);

/* ---------------------------------------------------------------------------
 * Step-level entry points. Each runs one step of the outer iteration on the
 * handle's stream with the handle's matrix and options, on caller-owned DEVICE
 * buffers, and returns after the work is enqueued and has finished (the
 * stream is synchronised). They are the same kernels ifeast_solve launches.
 * ------------------------------------------------------------------------- */

/* Alg. 2 steps 1-2: Q = Re sum_k w_k Y_k with (z_k B - A) Y_k ~= B X (B = I for
 * a standard handle) solved by the configured inner solver, using tolerance
 * alpha * RF (RF >= 0 given here).
 * X, Q: n x m0 float64 device. steps (optional, device int32[nc*m0], column
 * c = k*m0 + j) receives the Krylov steps taken by each (node, column). */
int ifeast_apply_filter(ifeast_t h, const double *X, double *Q, double RF, int32_t *steps);

/* Alg. 2 steps 1-2 in residual form (the right-hand sides ifeast_solve uses
 * from its second outer iteration on with IFEAST_INNER_MINRES, and with
 * IFEAST_INNER_GMRES + IFEAST_FP32 once ||R_F|| <= opts.correction_rf): for
 * the pairs (lam_j, x_j) given, r_j = A x_j - lam_j B x_j, the systems
 * (z_k B - A) e = r_j are solved by the inner solver (stop test
 * ||r_j - (z_k B - A) e|| <= alpha RF ||B x_j|| |z_k - lam_j|, Alg. 2's test on
 * the original system), and
 *   Q_j = Re sum_k w_k (x_j + e_kj) / (z_k - lam_j)
 *       = rho(lam_j) x_j + Re sum_k w_k e_kj / (z_k - lam_j),
 * which equals ifeast_apply_filter's Q in exact arithmetic (an identity of the
 * shifted systems). X, Q: n x m0 float64 device; lam: m0 float64 device;
 * steps as ifeast_apply_filter. UNSUPPORTED for GMRES handles in FP64 and for
 * non-symmetric handles. Overwrites the handle's last iterate: call
 * ifeast_solve again before ifeast_eigenpairs. */
int ifeast_apply_filter_residual(ifeast_t h, const double *X, const double *lam, double *Q,
                                 double RF, int32_t *steps);

/* Alg. 2 steps 3-4 on a given Q (n x m0 float64 device): Rayleigh-Ritz with
 * B_Q = Q^T B Q, A_Q = Q^T A Q, then X = Q X_Q (n x m0 device, B-orthonormal
 * Ritz vectors), lam[m0] ascending, resid[m0] relative residuals (device).
 * Returns BREAKDOWN if B_Q cannot be factored. */
int ifeast_rayleigh_ritz(ifeast_t h, const double *Q, double *X, double *lam, double *resid);

/* Non-symmetric handles: Galerkin Rayleigh-Ritz on a given Q (n x m0 device):
 * X (n x m0 device) receives the orthonormal basis Q L^{-T} of span(Q)
 * (B_Q = Q^T Q = L L^T), theta (2*m0 doubles, device) the unordered Ritz values
 * (re, im) of C = L^{-1} Q^T A Q L^{-T}, resid (m0, device) the relative
 * residuals of the unit Ritz vectors X u_j. BREAKDOWN if B_Q cannot be
 * factored or the reduced QR iteration does not converge. */
int ifeast_rayleigh_ritz_nonsym(ifeast_t h, const double *Q, double *X, double *theta,
                                double *resid);

/* One sparse product with a per-column complex shift (the operator of Alg. 2
 * step 1): W[:, c] = z[c / m0] B V[:, c] - A V[:, c] for c < ncols (B = I for
 * a standard handle), where V and W
 * are n x ncols complex float64 blocks (row-major, real and imaginary parts
 * interleaved: element (i, c) at [2*(i*ncols + c)]), z holds nc = ncols / m0
 * complex values interleaved (device). Uses the handle's A. ncols must be a
 * multiple of m0 with ncols / m0 <= 64. */
int ifeast_spmm_shift(ifeast_t h, const double *V, double *W, int ncols, int m0,
                      const double *z);

/* Rayleigh-Ritz without any device allocation, for callers that cannot call
 * cudaMalloc (code inside a fixed memory pool, a runtime that forbids device
 * allocation, or a process that reserved all device memory up front). The
 * paper has no counterpart: it is a packaging of ifeast_rayleigh_ritz.
 * Same outputs (X = Q X_Q, lam ascending, resid) for the matrix given as
 * caller-owned DEVICE CSR arrays (rowptr int32[n+1], colidx int32[nnz],
 * val float64[nnz]; not validated: the caller passes a well-formed matrix)
 * and device Q, X (n x m0 row-major), lam[m0], resid[m0]. X must not overlap
 * Q (X = Q X_Q reads every column of a row of Q while it writes that row of
 * X): overlapping ranges return INVALID_ARG before any device work.
 *   - No handle and no workspace: intermediates live in one file-scope
 *     device array of about 4.5 MiB that every GPU loading the library keeps
 *     until the process exits. m0 must be <= 64 (larger: INVALID_ARG).
 *   - The first call on a device looks up that array's device address (and
 *     sets the eigensolver's shared-memory limit); make the first call before
 *     any stream capture.
 *   - All calls share the array: calls that overlap on the GPU race, so the
 *     caller serialises them. Each call overwrites every scratch entry it
 *     reads, so results never depend on an earlier call.
 *   - Runs on stream (cudaStream_t as void*) and returns when it finished;
 *     BREAKDOWN if B_Q = Q^T Q cannot be factored. */
int ifeast_rayleigh_ritz_noalloc(int64_t n, int64_t nnz, const int32_t *rowptr,
                                 const int32_t *colidx, const double *val, int m0,
                                 const double *Q, double *X, double *lam, double *resid,
                                 void *stream);

/* ---------------------------------------------------------------------------
 * Kernel timing. on = 1: every kernel launch of the handle is bracketed by
 * CUDA events on the handle's stream (a few microseconds of overhead per
 * launch); the durations are summed per kernel class when the library next
 * synchronises its stream. on = N >= 2: the same, except that only launches
 * 1, 1 + N, 1 + 2N, ... of the chained Lanczos-loop kernels (the step
 * kernel, the kernel that reduces its partials to alpha_s, beta_{s+1}, and the
 * batched Givens QR) are timed, each class counted on its own: an
 * event between two of those kernels stops the second from launching while the
 * first runs (programmatic dependent launch), so timing all of them slows the
 * solve being timed. on = 0: off. A negative on returns IFEAST_ERR_INVALID_ARG.
 * ------------------------------------------------------------------------- */
int ifeast_set_profiling(ifeast_t h, int on);

/* Copies the summed milliseconds and the counts of timed launches of the first
 * cap kernel classes (device time between the bracketing events) into ms[] and
 * launches[] (either may be NULL); reset != 0 clears them afterwards.
 * Returns the number of kernel classes (22; each class is one kernel) on success; a NULL handle or a
 * negative cap returns IFEAST_ERR_INVALID_ARG (1). */
int ifeast_kernel_times(ifeast_t h, int cap, double *ms, int64_t *launches, int reset);

/* All launches (timed or not) of the first cap kernel classes since profiling
 * was switched on or last reset; reset != 0 clears them afterwards. Returns the
 * number of kernel classes, or IFEAST_ERR_INVALID_ARG for a NULL handle or a
 * negative cap. */
int ifeast_kernel_launches(ifeast_t h, int cap, int64_t *launches, int reset);

/* Name of kernel class k (static storage), "unknown" out of range. */
const char *ifeast_kernel_name(int k);

#ifdef __cplusplus
}
#endif
#endif
