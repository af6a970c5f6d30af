// Host side of libifeast: argument validation, contour quadrature, workspace
// layout, the outer iteration of Algorithm 2 and the C ABI of ifeast.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

using namespace ifeast;

struct ifeast_ctx {
  int64_t n = 0, nnz = 0;
  int m0 = 0, nc = 0, C = 0, K = 0;
  int ncc = 0;  // nodes per inner pass (per-node GMRES, opts.node_chunk; else nc)
  ifeast_opts opts{};
  ifeast_contour contour{};
  std::vector<double2> zh, wh;  // host copies of nodes and weights
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  RowTiling tl{};
  int Pg = 0, Pr = 0;
  // workspace
  char *ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  // device buffers (carved from ws)
  int32_t *rowptr = nullptr, *colidx = nullptr;
  double *val = nullptr;
  // B of A x = lambda B x (generalized problem; null: B = I)
  int64_t nnzB = -1;
  int32_t *rowptrB = nullptr, *colidxB = nullptr;
  double *valB = nullptr, *BQ = nullptr, *BX = nullptr;
  // non-symmetric extension
  bool nonsym = false;
  double *LinvT = nullptr;
  double2 *theta = nullptr, *Uc = nullptr;
  double2 *nsM = nullptr;             // block correction: [nc][m0][m0] (z_k I - C)^-1
  double *nsG = nullptr, *nsP = nullptr;  // Re sum_k w_k M_k; L^-T C
  int *ridx = nullptr;
  double2 *z = nullptr, *w = nullptr;
  void *V = nullptr, *W = nullptr;  // double2, or float2 for the FP32 basis
  double2 *part = nullptr, *H1 = nullptr, *H2 = nullptr;
  double *inv_h = nullptr;
  double2 *CS = nullptr, *SN = nullptr, *R = nullptr, *G = nullptr, *Y = nullptr;
  int *steps = nullptr, *done = nullptr;
  // per-node GMRES with the FP32 basis: FP32 values, FP32 weights, the
  // per-system bounds and the residual form's filter values
  float *valB32 = nullptr;
  bool b_same_pattern = false;  // B stored on A's pattern
  float2 *Yf = nullptr;
  double *tolc = nullptr, *gcx = nullptr;
  double *X = nullptr, *Q = nullptr, *AQ = nullptr, *beta = nullptr;
  double *gram_part = nullptr, *Aq = nullptr, *Bq = nullptr, *L = nullptr, *Cm = nullptr,
         *U = nullptr, *XQ = nullptr, *lam = nullptr, *res_part = nullptr, *res = nullptr;
  DevStatus *status = nullptr;
  DevStatus *status_host = nullptr;  // pinned
  // shared-basis (MINRES) mode
  // fp32: FP32 arithmetic (FP32, FP16 or BF16 storage); half / bf16: 16-bit storage
  bool minres = false, fp32 = false, half = false, bf16 = false;
  float wscale = 1.f;
  float *val32 = nullptr;
  void *LV = nullptr, *LW0 = nullptr, *LW1 = nullptr;
  bool two_pass = false;
  float *Qf = nullptr;
  double *lpart = nullptr, *lalpha = nullptr, *lbeta = nullptr, *ltol = nullptr;
  float4 *lcf32 = nullptr;

  double2 *lg = nullptr, *lR = nullptr, *lrot = nullptr, *lYc = nullptr, *lwt = nullptr;
  int *lsteps = nullptr, *ldone = nullptr, *lcoldone = nullptr, *lndone = nullptr,
      *lactive = nullptr, *lSj = nullptr;
  double *lcoef = nullptr, *lcx = nullptr, *Rres = nullptr, *rnorm = nullptr;
  int *active_host = nullptr;  // pinned, kCheckLag + 1 slots
  cudaEvent_t check_events[kCheckLag + 1] = {};
  int ell_w = 0;
  int32_t *colE = nullptr;
  float *valE = nullptr;
  Profiler prof;
  bool profiling = false;
  // results
  bool solved = false;
  ifeast_stats_t stats{};
  std::vector<double> user_zw;  // IFEAST_USER nodes (the contour points here)
};

namespace ifeast {

namespace rng_detail {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32 x 32 -> 64-bit products with the
// multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl constants
// 0x9E3779B9 and 0xBB67AE85 between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
  }
}

// One thread per element pair 2p, 2p + 1: 53-bit uniforms from the block's
// words, Box-Muller.
__global__ void k_seeded_normal(uint64_t total, uint32_t k0, uint32_t k1, double *__restrict__ X) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * p >= total) return;
  uint32_t c[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u};
  philox4x32_10(c, k0, k1);
  const double inv53 = 1.0 / 9007199254740992.0;  // 2^-53
  const double u1 = ((double)(((uint64_t)(c[0] >> 5) << 26) + (c[1] >> 6)) + 1.0) * inv53;
  const double u2 = (double)(((uint64_t)(c[2] >> 5) << 26) + (c[3] >> 6)) * inv53;
  const double rad = sqrt(-2.0 * log(u1));
  const double t = 6.283185307179586 * u2;  // the double nearest 2 pi, times u2
  X[2 * p] = rad * cos(t);
  if (2 * p + 1 < total) X[2 * p + 1] = rad * sin(t);
}

// R[r][j] = (A X)[r][j] - lam[j] BX[r][j], one thread per entry.
__global__ void k_residual_block(int n, int m, const int32_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ colidx,
                                 const double *__restrict__ val, const double *__restrict__ X,
                                 const double *__restrict__ BX, const double *__restrict__ lam,
                                 double *__restrict__ R) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * m) return;
  const int r = (int)(idx / m), j = (int)(idx % m);
  double acc = 0.0;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) acc = fma(val[p], X[(size_t)colidx[p] * m + j], acc);
  R[idx] = acc - lam[j] * BX[idx];
}

}  // namespace rng_detail

using rng_detail::k_residual_block;
using rng_detail::k_seeded_normal;

cudaError_t seeded_normal(int64_t n, int m0, uint64_t seed, double *X, cudaStream_t st) {
  const uint64_t total = (uint64_t)n * (uint64_t)m0;
  const uint64_t pairs = (total + 1) / 2;
  k_seeded_normal<<<(unsigned)((pairs + 255) / 256), 256, 0, st>>>(
      total, (uint32_t)seed, (uint32_t)(seed >> 32), X);
  return cudaGetLastError();
}

cudaError_t residual_block(int n, int m0, const int32_t *rowptr, const int32_t *colidx,
                           const double *val, const double *X, const double *BX,
                           const double *lam, double *R, cudaStream_t st) {
  const size_t total = (size_t)n * m0;
  k_residual_block<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, m0, rowptr, colidx, val, X,
                                                                    BX, lam, R);
  return cudaGetLastError();
}

}  // namespace ifeast

namespace {

// out[r * ld + q] = X[r * m0 + j0 + q], q < cnt: the in-interval Ritz vectors
__global__ void k_gather_columns(int64_t n, int m0, int j0, int cnt, int ld,
                                 const double *__restrict__ X, double *__restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)n * cnt) return;
  const size_t r = i / cnt, q = i % cnt;
  out[r * ld + q] = X[r * m0 + j0 + q];
}

struct Layout {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    off = (off + 255) / 256 * 256;
    const size_t o = off;
    off += count * sizeof(T);
    return o;
  }
};

struct Offsets {
  size_t rowptr, colidx, val, z, w, V, W, part, H1, H2, inv_h, CS, SN, R, G, Y, steps, done, X, Q,
      AQ, beta, gram_part, Aq, Bq, L, Cm, U, XQ, lam, res_part, res, status, total;
  size_t val32, LV, LW0, LW1, lpart, lalpha, lcf32, lbeta, ltol, lg, lR, lrot, lYc, lwt, lsteps, ldone,
      lcoldone, lndone, lactive, lSj, lcoef, lcx, Rres, rnorm, colE, valE;
  size_t rowptrB, colidxB, valB, BQ, BX;
  size_t LinvT, theta, Uc, ridx, nsM, nsG, nsP;
  size_t Qf;
  size_t valB32, tolc, Yf, gcx;
};

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
  return sms > 0 ? sms : 152;
}

Offsets plan(int64_t n, int64_t nnz, int m0, int nc, int ncc, int K, const RowTiling &tl, int Pg,
             int Pr,
             bool minres, int prec, int sms_for_plan, int64_t nnzB, bool nonsym,
             bool two_pass) {
  Layout L;
  Offsets o{};
  const size_t C = (size_t)ncc * m0;     // columns of one node chunk (all nodes: ncc = nc)
  const size_t Cfull = (size_t)nc * m0;
  const size_t mp = (size_t)(m0 + 3) / 4 * 4;
  o.rowptr = L.take<int32_t>(n + 1);
  o.colidx = L.take<int32_t>(nnz > 0 ? nnz : 1);
  o.val = L.take<double>(nnz > 0 ? nnz : 1);
  o.z = L.take<double2>(nc);
  o.w = L.take<double2>(nc);
  if (!minres) {  // per-node complex GMRES, FP64 or FP32 basis
    const bool fp32 = prec == IFEAST_FP32;
    const size_t es = fp32 ? sizeof(float2) : sizeof(double2);
    if (fp32) {
      o.val32 = L.take<float>(nnz > 0 ? nnz : 1);
      if (nnzB >= 0) o.valB32 = L.take<float>(nnzB > 0 ? nnzB : 1);
      o.Yf = L.take<float2>((size_t)K * C);
      // residual form: right-hand sides A X - B X Lambda, their norms, filter values
      o.Rres = L.take<double>((size_t)n * m0);
      o.rnorm = L.take<double>(m0);
      o.gcx = L.take<double>(m0);
    }
    o.tolc = L.take<double>(C);
    o.V = L.take<char>((size_t)(K + 1) * n * C * es);
    o.W = L.take<char>((size_t)n * C * es);
    o.part = L.take<double2>((size_t)tl.P * (K + 2) * C);
    o.H1 = L.take<double2>((size_t)(K + 2) * C);
    o.H2 = L.take<double2>((size_t)(K + 2) * C);
    o.inv_h = L.take<double>(C);
    o.CS = L.take<double2>((size_t)K * C);
    o.SN = L.take<double2>((size_t)K * C);
    o.R = L.take<double2>((size_t)K * K * C);
    o.G = L.take<double2>((size_t)(K + 1) * C);
    o.Y = L.take<double2>((size_t)K * C);
    o.steps = L.take<int>(Cfull);  // every node's step counts (chunks write their slice)
    o.done = L.take<int>(C);
  } else {  // shared Lanczos basis, tl tiles the n x m0 block
    const bool fp32 = prec != IFEAST_FP64;
    const size_t es = (prec == IFEAST_FP16 || prec == IFEAST_BF16)
                          ? 2 : (fp32 ? sizeof(float) : sizeof(double));
    if (fp32) {
      o.val32 = L.take<float>(nnz > 0 ? nnz : 1);
      // fixed-width copy of A for rows of at most 16 non-zeros
      o.colE = L.take<int32_t>((size_t)n * 16);
      o.valE = L.take<float>((size_t)n * 16);
    }
    // stored basis (K + 1 vectors), or three slots and an FP32 accumulator
    o.LV = L.take<char>((size_t)(two_pass ? 3 : K + 1) * n * m0 * es);
    if (two_pass) o.Qf = L.take<float>((size_t)n * m0);
    o.LW0 = L.take<char>((size_t)n * m0 * es);
    o.LW1 = L.take<char>((size_t)n * m0 * es);
    // partials of the step kernels: tl.P blocks (generic) or up to 2 per SM (FP32)
    o.lpart = L.take<double>((size_t)std::max(std::max(tl.P, 2 * sms_for_plan), 4) * 3 * m0);
    o.lalpha = L.take<double>((size_t)K * m0);
    o.lcf32 = L.take<float4>((size_t)(K + 1) * m0);

    o.lbeta = L.take<double>((size_t)(K + 1) * m0);
    o.ltol = L.take<double>(C);
    o.lg = L.take<double2>(C * (K + 1));
    o.lR = L.take<double2>(C * K * 3);
    o.lrot = L.take<double2>(C * 4);
    o.lYc = L.take<double2>(C * K);
    o.lwt = L.take<double2>(C);
    o.lsteps = L.take<int>(C);
    o.ldone = L.take<int>(C);  // pair done flags
    o.lcoldone = L.take<int>(m0);
    o.lndone = L.take<int>(m0);
    o.lactive = L.take<int>(1);
    o.lSj = L.take<int>(m0);
    o.lcoef = L.take<double>((size_t)K * m0 + ((size_t)K * m0 + 1) / 2);  // FP64 + FP32 copy
    o.lcx = L.take<double>(m0);
    o.Rres = L.take<double>((size_t)n * m0);
    o.rnorm = L.take<double>(m0);
  }
  o.X = L.take<double>((size_t)n * m0);
  o.Q = L.take<double>((size_t)n * m0);
  o.AQ = L.take<double>((size_t)n * m0);
  o.beta = L.take<double>(m0);
  o.gram_part = L.take<double>((size_t)Pg * 2 * mp * mp);
  o.Aq = L.take<double>((size_t)m0 * m0);
  o.Bq = L.take<double>((size_t)m0 * m0);
  o.L = L.take<double>((size_t)m0 * m0);
  o.Cm = L.take<double>((size_t)m0 * m0);
  o.U = L.take<double>((size_t)m0 * m0);
  o.XQ = L.take<double>((size_t)m0 * m0);
  o.lam = L.take<double>(m0);
  o.res_part = L.take<double>((size_t)Pr * 3 * m0);
  o.res = L.take<double>(m0);
  o.status = L.take<DevStatus>(1);
  if (nonsym) {  // non-symmetric extension
    o.LinvT = L.take<double>((size_t)m0 * m0);
    o.theta = L.take<double2>(m0);
    o.Uc = L.take<double2>((size_t)m0 * m0);
    o.ridx = L.take<int>(m0);
    o.nsM = L.take<double2>((size_t)nc * m0 * m0);  // block correction: M_k = (z_k I - C)^-1
    o.nsG = L.take<double>((size_t)m0 * m0);
    o.nsP = L.take<double>((size_t)m0 * m0);
    if (!o.Rres) {  // block residual R = A X - X C and its column norms (FP64 basis)
      o.Rres = L.take<double>((size_t)n * m0);
      o.rnorm = L.take<double>(m0);
    }
  }
  if (nnzB >= 0) {  // generalized problem
    o.rowptrB = L.take<int32_t>(n + 1);
    o.colidxB = L.take<int32_t>(nnzB > 0 ? nnzB : 1);
    o.valB = L.take<double>(nnzB > 0 ? nnzB : 1);
    o.BQ = L.take<double>((size_t)n * m0);
    o.BX = L.take<double>((size_t)n * m0);
  }
  o.total = (L.off + 255) / 256 * 256;
  return o;
}

int validate_contour(const ifeast_contour *c) {
  if (!c) return IFEAST_ERR_INVALID_ARG;
  if (!(c->emin < c->emax) || !std::isfinite(c->emin) || !std::isfinite(c->emax))
    return IFEAST_ERR_INVALID_ARG;
  if (c->rule == IFEAST_USER) {
    if (c->nc < 1 || c->nc > kMaxNodes || !c->user_zw) return IFEAST_ERR_INVALID_ARG;
    for (int k = 0; k < c->nc; ++k) {
      for (int q = 0; q < 4; ++q)
        if (!std::isfinite(c->user_zw[4 * k + q])) return IFEAST_ERR_INVALID_ARG;
      if (c->user_zw[4 * k + 1] == 0.0) return IFEAST_ERR_INVALID_ARG;
    }
    return IFEAST_OK;
  }
  if (c->rule == IFEAST_TRAP_FULL) {
    if (c->nc < 2 || c->nc % 2 != 0 || c->nc / 2 > kMaxNodes) return IFEAST_ERR_INVALID_ARG;
    return IFEAST_OK;
  }
  if (c->nc < 1 || c->nc > kMaxNodes) return IFEAST_ERR_INVALID_ARG;
  if (c->rule != IFEAST_GL_HALF && c->rule != IFEAST_TRAP_HALF) return IFEAST_ERR_INVALID_ARG;
  return IFEAST_OK;
}

// The rule the solver runs: a full-circle trapezoid rule on a real problem
// (real A, real X) equals the half rule on its upper nodes with the Re-sum.
ifeast_contour effective_contour(const ifeast_contour &c) {
  ifeast_contour e = c;
  if (c.rule == IFEAST_TRAP_FULL) {
    e.rule = IFEAST_TRAP_HALF;
    e.nc = c.nc / 2;
  }
  return e;
}

int validate_opts(const ifeast_opts *o) {
  if (!o) return IFEAST_ERR_INVALID_ARG;
  if (o->inner_solver == IFEAST_INNER_GMRES) {
    if (o->precision != IFEAST_FP64 && o->precision != IFEAST_FP32) return IFEAST_ERR_UNSUPPORTED;
    // the FP32 basis needs the residual form, which needs real Ritz pairs
    if (o->precision == IFEAST_FP32 && o->nonsymmetric == 1) return IFEAST_ERR_UNSUPPORTED;
    if (o->inner_max_iters < 1 || o->inner_max_iters > kMaxInner) return IFEAST_ERR_INVALID_ARG;
  } else if (o->inner_solver == IFEAST_INNER_MINRES) {
    if (o->precision != IFEAST_FP64 && o->precision != IFEAST_FP32 &&
        o->precision != IFEAST_FP16 && o->precision != IFEAST_BF16)
      return IFEAST_ERR_UNSUPPORTED;
    if (o->inner_max_iters < 1 || o->inner_max_iters > kMaxLanczos) return IFEAST_ERR_INVALID_ARG;
  } else {
    return IFEAST_ERR_UNSUPPORTED;
  }
  if (o->max_outer < 1 || !(o->tol >= 0.0) || !std::isfinite(o->alpha))
    return IFEAST_ERR_INVALID_ARG;
  if (!(o->correction_rf >= 0.0)) return IFEAST_ERR_INVALID_ARG;
  if (std::isnan(o->time_limit_ms)) return IFEAST_ERR_INVALID_ARG;
  if (o->nonsymmetric != 0 && o->nonsymmetric != 1) return IFEAST_ERR_INVALID_ARG;
  if (o->nonsymmetric && o->inner_solver != IFEAST_INNER_GMRES) return IFEAST_ERR_UNSUPPORTED;
  if (o->minres_two_pass != 0 && o->minres_two_pass != 1) return IFEAST_ERR_INVALID_ARG;
  if (o->node_chunk < 0) return IFEAST_ERR_INVALID_ARG;
  if (o->plain_loads != 0 && o->plain_loads != 1) return IFEAST_ERR_INVALID_ARG;
  if (o->nonsym_correction != 0 && o->nonsym_correction != 1) return IFEAST_ERR_INVALID_ARG;
  if (o->node_chunk > 0 && o->inner_solver != IFEAST_INNER_GMRES) return IFEAST_ERR_UNSUPPORTED;
  if (o->minres_two_pass &&
      (o->inner_solver != IFEAST_INNER_MINRES || o->precision == IFEAST_FP64))
    return IFEAST_ERR_UNSUPPORTED;
  return IFEAST_OK;
}

// Gauss-Legendre nodes/weights on (-1, 1) by Newton iteration on P_n (Golub &
// Welsch would also do; Newton from the Chebyshev-like initial guess
// cos(pi (i - 1/4)/(n + 1/2)) converges to machine precision in a few steps).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &wgt) {
  x.assign(n, 0.0);
  wgt.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = (n == 1) ? t : p1;
      const double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (t * pn - pnm1) / (t * t - 1.0);
      const double dt = pn / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    // recompute derivative at the converged point
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double pn = (n == 1) ? t : p1;
    const double pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (t * pn - pnm1) / (t * t - 1.0);
    x[i] = t;
    wgt[i] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
  // ascending nodes
  std::reverse(x.begin(), x.end());
  std::reverse(wgt.begin(), wgt.end());
}

void contour_host(const ifeast_contour *c, std::vector<double2> &z, std::vector<double2> &w) {
  const double ctr = 0.5 * (c->emin + c->emax), r = 0.5 * (c->emax - c->emin);
  z.resize(c->nc);
  w.resize(c->nc);
  if (c->rule == IFEAST_USER) {
    for (int k = 0; k < c->nc; ++k) {
      z[k] = make_double2(c->user_zw[4 * k], c->user_zw[4 * k + 1]);
      w[k] = make_double2(c->user_zw[4 * k + 2], c->user_zw[4 * k + 3]);
    }
  } else if (c->rule == IFEAST_GL_HALF) {
    std::vector<double> x, g;
    gauss_legendre(c->nc, x, g);
    for (int k = 0; k < c->nc; ++k) {
      const double th = 0.5 * M_PI * (1.0 - x[k]);
      z[k] = make_double2(ctr + r * std::cos(th), r * std::sin(th));
      w[k] = make_double2(0.5 * g[k] * r * std::cos(th), 0.5 * g[k] * r * std::sin(th));
    }
  } else {
    const double full = (c->rule == IFEAST_TRAP_FULL) ? 2.0 : 1.0;
    for (int k = 0; k < c->nc; ++k) {
      const double th = full * M_PI * (k + 0.5) / c->nc;
      z[k] = make_double2(ctr + r * std::cos(th), r * std::sin(th));
      w[k] = make_double2(r * std::cos(th) / c->nc, r * std::sin(th) / c->nc);
    }
  }
}

std::mutex g_init_mu;
bool g_init_done[64] = {false};

int ensure_device_init() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IFEAST_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev >= 0 && dev < 64 && !g_init_done[dev]) {
    if (rr_init() != cudaSuccess || minres_init() != cudaSuccess || gmres_init() != cudaSuccess)
      return IFEAST_ERR_CUDA;
    g_init_done[dev] = true;
  }
  return IFEAST_OK;
}

#define CK(call)                                  \
  do {                                            \
    if ((call) != cudaSuccess) {                  \
      return IFEAST_ERR_CUDA;                     \
    }                                             \
  } while (0)

// Per-node GMRES. correction = 0: right-hand sides X (or B X), norms in
// h->beta; correction = 1: right-hand sides h->Rres = A X - B X Lambda of the
// current Ritz pairs (norms h->rnorm, Ritz values h->lam, ||B x_j|| in h->beta).
GmresArgs gmres_args(ifeast_ctx *h, const double *X, double *Q, int correction = 0) {
  GmresArgs a{};
  a.fp32 = h->fp32 ? 1 : 0;
  a.stream_tma = h->opts.plain_loads ? 0 : 1;
  a.val32 = h->val32;
  a.valB32 = h->valB32;
  a.b_same_pattern = h->b_same_pattern ? 1 : 0;
  a.Yf = h->Yf;
  a.tolc = h->tolc;
  a.correction = correction;
  if (correction) {
    a.lam = h->lam;
    a.xnorm = h->beta;
    a.Xr = h->X;
    a.cx = h->gcx;
  }
  a.n = (int)h->n;
  a.m0 = h->m0;
  a.nc = h->nc;
  a.ncc = h->ncc;
  a.C = h->ncc * h->m0;  // columns of one inner pass
  a.K = h->K;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.val = h->val;
  a.z = h->z;
  a.w = h->w;
  a.X = X;
  a.V = h->V;
  a.W = h->W;
  a.part = h->part;
  a.H1 = h->H1;
  a.H2 = h->H2;
  a.inv_h = h->inv_h;
  a.CS = h->CS;
  a.SN = h->SN;
  a.R = h->R;
  a.G = h->G;
  a.Y = h->Y;
  a.beta = correction ? h->rnorm : h->beta;
  a.steps = h->steps;
  a.done = h->done;
  a.Q = Q;
  a.status = h->status;
  a.tl = h->tl;
  a.prof = h->profiling ? &h->prof : nullptr;
  a.rowptrB = h->rowptrB;
  a.colidxB = h->colidxB;
  a.valB = h->valB;
  return a;
}

RRArgs rr_args(ifeast_ctx *h, const double *Q, double *X) {
  RRArgs a{};
  a.n = (int)h->n;
  a.m0 = h->m0;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.val = h->val;
  a.Q = Q;
  a.AQ = h->AQ;
  a.gram_part = h->gram_part;
  a.Pg = h->Pg;
  a.Aq = h->Aq;
  a.Bq = h->Bq;
  a.L = h->L;
  a.Cm = h->Cm;
  a.U = h->U;
  a.XQ = h->XQ;
  a.lam = h->lam;
  a.X = X;
  a.res_part = h->res_part;
  a.Pr = h->Pr;
  a.res = h->res;
  a.beta = h->beta;
  a.emin = h->contour.emin;
  a.emax = h->contour.emax;
  a.alpha = h->opts.alpha;
  a.status = h->status;
  a.Rres = h->Rres;  // null unless an inner solver takes the residual form
  a.rnorm = h->rnorm;
  a.prof = h->profiling ? &h->prof : nullptr;
  a.rowptrB = h->rowptrB;
  a.colidxB = h->colidxB;
  a.valB = h->valB;
  a.BQ = h->BQ;
  a.BX = h->BX;
  a.num_sms = h->num_sms;
  return a;
}

NonsymArgs ns_args(ifeast_ctx *h) {
  NonsymArgs a;
  a.LinvT = h->LinvT;
  a.theta = h->theta;
  a.Uc = h->Uc;
  return a;
}

// Right-hand side block of the shifted systems: X (B = I) or B X written to
// h->BX, with its column norms in h->beta.
int prepare_rhs(ifeast_ctx *h, const double *X, const double **rhs) {
  Profiler *pf = h->profiling ? &h->prof : nullptr;
  if (!h->rowptrB) {
    if (column_norms((int)h->n, h->m0, X, h->res_part, h->Pr, h->beta, h->stream, pf) !=
        cudaSuccess)
      return IFEAST_ERR_CUDA;
    *rhs = X;
    return IFEAST_OK;
  }
  if (spmm_block((int)h->n, h->m0, h->rowptrB, h->colidxB, h->valB, X, h->BX, h->Pg, h->stream) !=
          cudaSuccess ||
      column_norms((int)h->n, h->m0, h->BX, h->res_part, h->Pr, h->beta, h->stream, pf) !=
          cudaSuccess)
    return IFEAST_ERR_CUDA;
  *rhs = h->BX;
  return IFEAST_OK;
}

// Block correction of the non-symmetric iteration (opts.nonsym_correction).
// From the last Rayleigh-Ritz (L^{-T} and A_Q = Q^T A Q on the device) the
// Galerkin matrix of the carried basis X = Q L^{-T} is C = L^{-1} A_Q L^{-T}. On
// the host: P = L^{-T} C, M_k = (z_k I - C)^{-1} for every node (complex
// Gauss-Jordan with partial pivoting) and Re sum_k w_k M_k; on the device the
// right-hand sides R = A X - X C = (A Q) L^{-T} - Q P and their column norms.
int ns_block_correction_setup(ifeast_ctx *h) {
  const int m = h->m0;
  const size_t mm = (size_t)m * m;
  std::vector<double> Lt(mm), Aq(mm), T(mm, 0.0), C(mm, 0.0), P(mm, 0.0), G(mm, 0.0);
  CK(cudaMemcpyAsync(Lt.data(), h->LinvT, mm * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(Aq.data(), h->Aq, mm * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < m; ++i)  // T = A_Q L^{-T}
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) T[(size_t)i * m + k] += Aq[(size_t)i * m + j] * Lt[(size_t)j * m + k];
  for (int i = 0; i < m; ++i)  // C = (L^{-T})^T T
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) C[(size_t)i * m + k] += Lt[(size_t)j * m + i] * T[(size_t)j * m + k];
  for (int i = 0; i < m; ++i)  // P = L^{-T} C
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) P[(size_t)i * m + k] += Lt[(size_t)i * m + j] * C[(size_t)j * m + k];
  std::vector<double2> M((size_t)h->nc * mm), aug((size_t)m * 2 * m);
  auto cm = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
  for (int k = 0; k < h->nc; ++k) {
    const double2 z = h->zh[k], w = h->wh[k];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < 2 * m; ++j) {
        double2 v = make_double2(0.0, 0.0);
        if (j < m) v = make_double2((i == j ? z.x : 0.0) - C[(size_t)i * m + j], i == j ? z.y : 0.0);
        else v = make_double2(j - m == i ? 1.0 : 0.0, 0.0);
        aug[(size_t)i * 2 * m + j] = v;
      }
    for (int c = 0; c < m; ++c) {  // Gauss-Jordan, pivot = largest |entry| of column c
      int p = c;
      double best = -1.0;
      for (int i = c; i < m; ++i) {
        const double2 v = aug[(size_t)i * 2 * m + c];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; p = i; }
      }
      if (!(best > 0.0)) return IFEAST_ERR_BREAKDOWN;  // a node on a Ritz value
      if (p != c)
        for (int j = 0; j < 2 * m; ++j) std::swap(aug[(size_t)p * 2 * m + j], aug[(size_t)c * 2 * m + j]);
      const double2 d = aug[(size_t)c * 2 * m + c];
      const double2 inv = make_double2(d.x / best, -d.y / best);
      for (int j = 0; j < 2 * m; ++j) aug[(size_t)c * 2 * m + j] = cm(aug[(size_t)c * 2 * m + j], inv);
      for (int i = 0; i < m; ++i) {
        if (i == c) continue;
        const double2 f = aug[(size_t)i * 2 * m + c];
        if (f.x == 0.0 && f.y == 0.0) continue;
        for (int j = 0; j < 2 * m; ++j) {
          const double2 t = cm(f, aug[(size_t)c * 2 * m + j]);
          aug[(size_t)i * 2 * m + j].x -= t.x;
          aug[(size_t)i * 2 * m + j].y -= t.y;
        }
      }
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double2 v = aug[(size_t)i * 2 * m + m + j];
        M[(size_t)k * mm + (size_t)i * m + j] = v;
        G[(size_t)i * m + j] += w.x * v.x - w.y * v.y;
      }
  }
  CK(cudaMemcpyAsync(h->nsM, M.data(), M.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->nsG, G.data(), mm * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->nsP, P.data(), mm * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  // the host arrays are read by the copies: wait before they go out of scope
  CK(cudaStreamSynchronize(h->stream));
  CK(ns_block_residual((int)h->n, m, h->AQ, h->Q, h->LinvT, h->nsP, h->Rres, h->stream));
  Profiler *pf = h->profiling ? &h->prof : nullptr;
  CK(column_norms((int)h->n, m, h->Rres, h->res_part, h->Pr, h->rnorm, h->stream, pf));
  return IFEAST_OK;
}

// Shared-basis inner solve. correction = 0: right-hand sides X (norms in
// h->beta); correction = 1: right-hand sides h->Rres = A X - X Lambda of the
// current X (norms h->rnorm, Ritz values h->lam, ||x_j|| in h->beta).
MinresArgs minres_args(ifeast_ctx *h, const double *X, double *Q, int correction) {
  MinresArgs a{};
  a.n = (int)h->n;
  a.m0 = h->m0;
  a.nc = h->nc;
  a.K = h->K;
  a.fp32 = h->fp32 ? 1 : 0;
  a.half = h->half ? 1 : 0;
  a.bf16 = h->bf16 ? 1 : 0;
  a.wscale = h->wscale;
  a.rowptr = h->rowptr;
  a.colidx = h->colidx;
  a.val_t = h->fp32 ? (const void *)h->val32 : (const void *)h->val;
  a.rhs = correction ? h->Rres : X;
  a.rnorm = correction ? h->rnorm : h->beta;
  a.X = X;
  a.V = h->LV;
  a.W0 = h->LW0;
  a.W1 = h->LW1;
  a.part = h->lpart;
  a.alpha = h->lalpha;
  a.beta = h->lbeta;
  a.cf32 = h->lcf32;

  a.Yc = h->lYc;
  a.wt = h->lwt;
  a.coef = h->lcoef;
  a.cx = h->lcx;
  a.Sj = h->lSj;
  a.Q = Q;
  a.tl = h->tl;
  a.check_every = 16;
  a.active_host = h->active_host;
  a.check_events = h->check_events;
  a.P_async = h->num_sms;  // one resident 512-thread block per SM
  a.two_pass = h->two_pass ? 1 : 0;
  a.Qf = h->Qf;
  a.ell_w = h->ell_w;
  a.colE = h->colE;
  a.valE = h->valE;
  a.prof = h->profiling ? &h->prof : nullptr;
  MinresState &m = a.ms;
  m.z = h->z;
  m.w = h->w;
  m.lam = h->lam;
  m.xnorm = h->beta;
  m.correction = correction;
  m.g = h->lg;
  m.R = h->lR;
  m.rot = h->lrot;
  m.tol = h->ltol;
  m.steps = h->lsteps;
  m.done = h->ldone;
  m.coldone = h->lcoldone;
  m.ndone = h->lndone;
  m.active = h->lactive;
  m.status = h->status;
  return a;
}

int set_tolerance(ifeast_ctx *h, double RF) {
  // status->tol_rel = alpha * RF; step counters cleared
  DevStatus s{};
  s.RF = RF;
  s.tol_rel = h->opts.alpha > 0.0 ? h->opts.alpha * RF : 0.0;
  *h->status_host = s;
  CK(cudaMemcpyAsync(h->status, h->status_host, sizeof(DevStatus), cudaMemcpyHostToDevice,
                     h->stream));
  return IFEAST_OK;
}

int clear_step_counters(ifeast_ctx *h) {
  CK(cudaMemsetAsync(&h->status->max_steps, 0, sizeof(int), h->stream));
  CK(cudaMemsetAsync(&h->status->total_steps, 0, sizeof(long long), h->stream));
  return IFEAST_OK;
}

}  // namespace

extern "C" {

void ifeast_default_opts(ifeast_opts *o) {
  if (!o) return;
  o->inner_solver = IFEAST_INNER_GMRES;
  o->inner_max_iters = 10;
  o->alpha = 0.0;
  o->max_outer = 100;
  o->tol = 1e-10;
  o->precision = IFEAST_FP64;
  o->verbose = 0;
  o->nonsymmetric = 0;
  o->minres_two_pass = 0;
  o->correction_rf = 1e-3;
  o->time_limit_ms = 0.0;
  o->node_chunk = 0;
  o->plain_loads = 0;
  o->nonsym_correction = 0;
}

const char *ifeast_strerror(int code) {
  switch (code) {
    case IFEAST_OK: return "ok";
    case IFEAST_ERR_INVALID_ARG: return "invalid argument";
    case IFEAST_ERR_OOM: return "out of memory (workspace too small or device allocation failed)";
    case IFEAST_ERR_CUDA: return "CUDA runtime error";
    case IFEAST_ERR_NOT_CONVERGED: return "not converged within max_outer iterations";
    case IFEAST_ERR_M0_TOO_SMALL: return "subspace size m0 too small for the interval";
    case IFEAST_STATUS_NO_EIGENVALUES: return "no eigenvalue found in the interval";
    case IFEAST_ERR_BREAKDOWN: return "reduced Gram matrix B_Q not positive definite";
    case IFEAST_ERR_TIMEOUT: return "bounded device wait timed out";
    case IFEAST_ERR_STATE: return "call out of order";
    case IFEAST_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int ifeast_contour_nodes(const ifeast_contour *c, double *zw) {
  if (!c || !zw) return IFEAST_ERR_INVALID_ARG;
  if (c->nc < 1 || c->nc > kMaxNodes || !(c->emin < c->emax)) return IFEAST_ERR_INVALID_ARG;
  if (c->rule != IFEAST_GL_HALF && c->rule != IFEAST_TRAP_HALF && c->rule != IFEAST_TRAP_FULL &&
      c->rule != IFEAST_USER)
    return IFEAST_ERR_INVALID_ARG;
  if (c->rule == IFEAST_USER && validate_contour(c) != IFEAST_OK) return IFEAST_ERR_INVALID_ARG;
  std::vector<double2> z, w;
  contour_host(c, z, w);
  for (int k = 0; k < c->nc; ++k) {
    zw[4 * k + 0] = z[k].x;
    zw[4 * k + 1] = z[k].y;
    zw[4 * k + 2] = w[k].x;
    zw[4 * k + 3] = w[k].y;
  }
  return IFEAST_OK;
}

int ifeast_workspace_bytes(int64_t n, int64_t nnz, int m0, const ifeast_contour *c,
                           const ifeast_opts *o, size_t *bytes) {
  return ifeast_workspace_bytes_generalized(n, nnz, -1, m0, c, o, bytes);
}

int ifeast_workspace_bytes_generalized(int64_t n, int64_t nnz, int64_t nnz_b, int m0,
                                       const ifeast_contour *c, const ifeast_opts *o,
                                       size_t *bytes) {
  if (!bytes || n < 1 || nnz < 0 || m0 < 1 || m0 > kMaxM0 || m0 > n) return IFEAST_ERR_INVALID_ARG;
  if (nnz_b > (int64_t)INT32_MAX) return IFEAST_ERR_INVALID_ARG;
  if (nnz_b >= 0 && o && o->inner_solver != IFEAST_INNER_GMRES) return IFEAST_ERR_UNSUPPORTED;
  // the non-symmetric extension: standard problem, m0 within the reduced solver's limit
  if (o && o->nonsymmetric == 1 && (nnz_b >= 0 || m0 > kNonsymMaxM0)) return IFEAST_ERR_UNSUPPORTED;
  // 16-bit storage and the two-pass mode run on the four-column kernels only
  if (o && (o->precision == IFEAST_FP16 || o->precision == IFEAST_BF16 ||
            o->minres_two_pass == 1) && m0 % 4 != 0)
    return IFEAST_ERR_UNSUPPORTED;
  if (n > (int64_t)INT32_MAX - 1 || nnz > (int64_t)INT32_MAX) return IFEAST_ERR_INVALID_ARG;
  int rc = validate_contour(c);
  if (rc) return rc;
  rc = validate_opts(o);
  if (rc) return rc;
  const int nc = effective_contour(*c).nc;
  if (o->node_chunk > 0 && nc % o->node_chunk != 0) return IFEAST_ERR_INVALID_ARG;
  const int sms = device_sms();
  const bool minres = o->inner_solver == IFEAST_INNER_MINRES;
  const int ncc = (!minres && o->node_chunk > 0) ? o->node_chunk : nc;
  RowTiling tl = make_tiling(n, minres ? 32 : ncc * m0, sms);
  if (minres) tl.tiles = (m0 + 31) / 32;  // row blocks cover every column
  const int Pg = std::max(1, (int)std::min<int64_t>(2 * sms, (n + 31) / 32));
  const int Pr = Pg;
  *bytes = plan(n, nnz, m0, nc, ncc, o->inner_max_iters, tl, Pg, Pr, minres, o->precision, sms,
                nnz_b < 0 ? -1 : nnz_b, o->nonsymmetric == 1, o->minres_two_pass == 1).total;
  return IFEAST_OK;
}

int ifeast_create(const ifeast_csr *A, const ifeast_csr *B, const ifeast_contour *c, int m0,
                  const ifeast_opts *o, void *workspace, size_t ws_bytes, void *stream,
                  ifeast_t *out) {
  if (!out) return IFEAST_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || !A->rowptr || (A->nnz > 0 && (!A->colidx || !A->val))) return IFEAST_ERR_INVALID_ARG;
  const int64_t n = A->n, nnz = A->nnz;
  if (n < 1 || nnz < 0) return IFEAST_ERR_INVALID_ARG;
  if (B && (B->n != n || !B->rowptr || B->nnz < 0 || (B->nnz > 0 && (!B->colidx || !B->val))))
    return IFEAST_ERR_INVALID_ARG;
  const int64_t nnzB = B ? B->nnz : -1;
  size_t need = 0;
  int rc = ifeast_workspace_bytes_generalized(n, nnz, nnzB, m0, c, o, &need);
  if (rc) return rc;
  // CSR structure checks on the host
  for (const ifeast_csr *M : {A, B}) {
    if (!M) continue;
    if (M->rowptr[0] != 0 || M->rowptr[n] != M->nnz) return IFEAST_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i)
      if (M->rowptr[i + 1] < M->rowptr[i]) return IFEAST_ERR_INVALID_ARG;
    for (int64_t p = 0; p < M->nnz; ++p)
      if (M->colidx[p] < 0 || M->colidx[p] >= n || !std::isfinite(M->val[p]))
        return IFEAST_ERR_INVALID_ARG;
  }
  if (workspace && ws_bytes < need) return IFEAST_ERR_OOM;
  rc = ensure_device_init();
  if (rc) return rc;

  ifeast_ctx *h = new (std::nothrow) ifeast_ctx();
  if (!h) return IFEAST_ERR_OOM;
  h->n = n;
  h->nnz = nnz;
  h->m0 = m0;
  const ifeast_contour ce = effective_contour(*c);
  h->nc = ce.nc;
  h->C = ce.nc * m0;
  h->K = o->inner_max_iters;
  h->opts = *o;
  h->contour = ce;
  if (ce.rule == IFEAST_USER) {  // the caller's array may be freed after create
    h->user_zw.assign(ce.user_zw, ce.user_zw + 4 * (size_t)ce.nc);
    h->contour.user_zw = h->user_zw.data();
  }
  h->nonsym = o->nonsymmetric == 1;
  h->stream = (cudaStream_t)stream;
  h->num_sms = device_sms();
  h->minres = o->inner_solver == IFEAST_INNER_MINRES;
  h->fp32 = o->precision == IFEAST_FP32 || o->precision == IFEAST_FP16 ||
            o->precision == IFEAST_BF16;
  h->half = o->precision == IFEAST_FP16;
  h->bf16 = o->precision == IFEAST_BF16;
  h->ncc = (!h->minres && o->node_chunk > 0) ? o->node_chunk : h->nc;
  h->tl = make_tiling(n, h->minres ? 32 : h->ncc * m0, h->num_sms);
  if (h->minres) h->tl.tiles = (m0 + 31) / 32;
  h->Pg = std::max(1, (int)std::min<int64_t>(2 * h->num_sms, (n + 31) / 32));
  h->Pr = h->Pg;
  contour_host(&ce, h->zh, h->wh);
  h->two_pass = o->minres_two_pass == 1;
  const Offsets off = plan(n, nnz, m0, h->nc, h->ncc, h->K, h->tl, h->Pg, h->Pr, h->minres,
                           o->precision,
                           h->num_sms, nnzB, h->nonsym, h->two_pass);
  if (workspace) {
    h->ws = (char *)workspace;
    h->ws_bytes = ws_bytes;
  } else {
    if (cudaMalloc(&h->ws, off.total) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return IFEAST_ERR_OOM;
    }
    h->owns_ws = true;
    h->ws_bytes = off.total;
  }
  if (cudaMallocHost(&h->status_host, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&h->active_host, (kCheckLag + 1) * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->owns_ws) cudaFree(h->ws);
    delete h;
    return IFEAST_ERR_OOM;
  }
  for (cudaEvent_t &ev : h->check_events) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ifeast_destroy(h);
      return IFEAST_ERR_CUDA;
    }
  }
  char *b = h->ws;
  h->rowptr = (int32_t *)(b + off.rowptr);
  h->colidx = (int32_t *)(b + off.colidx);
  h->val = (double *)(b + off.val);
  h->z = (double2 *)(b + off.z);
  h->w = (double2 *)(b + off.w);
  h->V = b + off.V;
  h->W = b + off.W;
  h->part = (double2 *)(b + off.part);
  h->H1 = (double2 *)(b + off.H1);
  h->H2 = (double2 *)(b + off.H2);
  h->inv_h = (double *)(b + off.inv_h);
  h->CS = (double2 *)(b + off.CS);
  h->SN = (double2 *)(b + off.SN);
  h->R = (double2 *)(b + off.R);
  h->G = (double2 *)(b + off.G);
  h->Y = (double2 *)(b + off.Y);
  h->steps = (int *)(b + off.steps);
  h->done = (int *)(b + off.done);
  if (!h->minres) {
    h->tolc = (double *)(b + off.tolc);
    if (h->fp32) {
      h->val32 = (float *)(b + off.val32);
      if (B) h->valB32 = (float *)(b + off.valB32);
      h->Yf = (float2 *)(b + off.Yf);
      h->Rres = (double *)(b + off.Rres);
      h->rnorm = (double *)(b + off.rnorm);
      h->gcx = (double *)(b + off.gcx);
    }
  }
  h->X = (double *)(b + off.X);
  h->Q = (double *)(b + off.Q);
  h->AQ = (double *)(b + off.AQ);
  h->beta = (double *)(b + off.beta);
  h->gram_part = (double *)(b + off.gram_part);
  h->Aq = (double *)(b + off.Aq);
  h->Bq = (double *)(b + off.Bq);
  h->L = (double *)(b + off.L);
  h->Cm = (double *)(b + off.Cm);
  h->U = (double *)(b + off.U);
  h->XQ = (double *)(b + off.XQ);
  h->lam = (double *)(b + off.lam);
  h->res_part = (double *)(b + off.res_part);
  h->res = (double *)(b + off.res);
  h->status = (DevStatus *)(b + off.status);
  if (h->nonsym) {
    h->LinvT = (double *)(b + off.LinvT);
    h->theta = (double2 *)(b + off.theta);
    h->Uc = (double2 *)(b + off.Uc);
    h->ridx = (int *)(b + off.ridx);
    h->nsM = (double2 *)(b + off.nsM);
    h->nsG = (double *)(b + off.nsG);
    h->nsP = (double *)(b + off.nsP);
    h->Rres = (double *)(b + off.Rres);
    h->rnorm = (double *)(b + off.rnorm);
  }
  if (B) {
    h->nnzB = nnzB;
    h->b_same_pattern =
        nnzB == nnz &&
        std::equal(A->rowptr, A->rowptr + n + 1, B->rowptr) &&
        (nnz == 0 || std::equal(A->colidx, A->colidx + nnz, B->colidx));
    h->rowptrB = (int32_t *)(b + off.rowptrB);
    h->colidxB = (int32_t *)(b + off.colidxB);
    h->valB = (double *)(b + off.valB);
    h->BQ = (double *)(b + off.BQ);
    h->BX = (double *)(b + off.BX);
  }
  if (h->minres) {
    if (h->fp32) {
      h->val32 = (float *)(b + off.val32);
      h->colE = (int32_t *)(b + off.colE);
      h->valE = (float *)(b + off.valE);
    }
    h->LV = b + off.LV;
    if (h->two_pass) h->Qf = (float *)(b + off.Qf);
    h->LW0 = b + off.LW0;
    h->LW1 = b + off.LW1;
    h->lpart = (double *)(b + off.lpart);
    h->lalpha = (double *)(b + off.lalpha);
    h->lcf32 = (float4 *)(b + off.lcf32);

    h->lbeta = (double *)(b + off.lbeta);
    h->ltol = (double *)(b + off.ltol);
    h->lg = (double2 *)(b + off.lg);
    h->lR = (double2 *)(b + off.lR);
    h->lrot = (double2 *)(b + off.lrot);
    h->lYc = (double2 *)(b + off.lYc);
    h->lwt = (double2 *)(b + off.lwt);
    h->lsteps = (int *)(b + off.lsteps);
    h->ldone = (int *)(b + off.ldone);
    h->lcoldone = (int *)(b + off.lcoldone);
    h->lndone = (int *)(b + off.lndone);
    h->lactive = (int *)(b + off.lactive);
    h->lSj = (int *)(b + off.lSj);
    h->lcoef = (double *)(b + off.lcoef);
    h->lcx = (double *)(b + off.lcx);
    h->Rres = (double *)(b + off.Rres);
    h->rnorm = (double *)(b + off.rnorm);
  }
  bool ok = cudaMemcpyAsync(h->rowptr, A->rowptr, (n + 1) * sizeof(int32_t),
                            cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
  if (nnz > 0) {
    ok = ok && cudaMemcpyAsync(h->colidx, A->colidx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice,
                               h->stream) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(h->val, A->val, nnz * sizeof(double), cudaMemcpyHostToDevice,
                               h->stream) == cudaSuccess;
  }
  if (B) {
    ok = ok && cudaMemcpyAsync(h->rowptrB, B->rowptr, (n + 1) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
    if (nnzB > 0) {
      ok = ok && cudaMemcpyAsync(h->colidxB, B->colidx, nnzB * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, h->stream) == cudaSuccess;
      ok = ok && cudaMemcpyAsync(h->valB, B->val, nnzB * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream) == cudaSuccess;
    }
  }
  ok = ok && cudaMemcpyAsync(h->z, h->zh.data(), h->nc * sizeof(double2), cudaMemcpyHostToDevice,
                             h->stream) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(h->w, h->wh.data(), h->nc * sizeof(double2), cudaMemcpyHostToDevice,
                             h->stream) == cudaSuccess;
  if (h->fp32 && nnz > 0) ok = ok && convert_to_float(h->val, h->val32, nnz, h->stream) == cudaSuccess;
  if (h->valB32 && nnzB > 0)
    ok = ok && convert_to_float(h->valB, h->valB32, nnzB, h->stream) == cudaSuccess;
  if (h->fp32 && h->minres && m0 % 4 == 0) {
    // FP16 storage keeps w_s / ||A||_inf (|w_s| <= ||A||_inf ||v_s||_inf + |beta_s| ...)
    if (h->half) {
      double mx = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        double rs = 0.0;
        for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) rs += std::fabs(A->val[p]);
        mx = std::max(mx, rs);
      }
      h->wscale = mx > 0.0 ? (float)mx : 1.f;
    }
    // ELL slots a row needs: its entries, plus slot 0 for a missing diagonal
    int64_t maxlen = 0;
    for (int64_t i = 0; i < n; ++i) {
      int64_t len = A->rowptr[i + 1] - A->rowptr[i];
      bool diag = false;
      for (int64_t p = A->rowptr[i]; p < A->rowptr[i + 1]; ++p) diag = diag || A->colidx[p] == i;
      maxlen = std::max<int64_t>(maxlen, len + (diag ? 0 : 1));
    }
    h->ell_w = maxlen <= 8 ? 8 : (maxlen <= 16 ? 16 : 0);
    if (h->ell_w)
      ok = ok && build_ell((int)n, h->ell_w, h->rowptr, h->colidx, h->val32, h->colE, h->valE,
                           h->stream) == cudaSuccess;
  }
  ok = ok && cudaStreamSynchronize(h->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ifeast_destroy(h);
    return IFEAST_ERR_CUDA;
  }
  *out = h;
  return IFEAST_OK;
}

void ifeast_destroy(ifeast_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->owns_ws && h->ws) cudaFree(h->ws);
  if (h->status_host) cudaFreeHost(h->status_host);
  if (h->active_host) cudaFreeHost(h->active_host);
  for (cudaEvent_t ev : h->check_events)
    if (ev) cudaEventDestroy(ev);
  if (h->prof.events) {
    for (int i = 0; i < 2 * h->prof.cap; ++i) cudaEventDestroy(h->prof.events[i]);
    delete[] h->prof.events;
    delete[] h->prof.kid;
  }
  delete h;
}

int ifeast_initial_subspace(int64_t n, int m0, uint64_t seed, double *X, void *stream) {
  if (n < 1 || m0 < 1 || !X) return IFEAST_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(seeded_normal(n, m0, seed, X, st));
  CK(cudaStreamSynchronize(st));
  return IFEAST_OK;
}

int ifeast_solve(ifeast_t h, const double *X0, int x0_on_device, uint64_t seed, void *stream) {
  if (!h) return IFEAST_ERR_INVALID_ARG;
  // this solve's stream (the handle's own when NULL); restored on return
  struct StreamScope {
    ifeast_ctx *h;
    cudaStream_t saved, saved_prof;
    ~StreamScope() {
      h->stream = saved;
      h->prof.stream = saved_prof;
    }
  } scope{h, h->stream, h->prof.stream};
  if (stream) {
    h->stream = (cudaStream_t)stream;
    h->prof.stream = h->stream;
  }
  const auto t0 = std::chrono::steady_clock::now();
  const double limit_ms = h->opts.time_limit_ms;
  h->solved = false;
  h->stats = ifeast_stats_t{};
  const size_t xbytes = (size_t)h->n * h->m0 * sizeof(double);
  if (X0)
    CK(cudaMemcpyAsync(h->X, X0, xbytes,
                       x0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       h->stream));
  else
    CK(seeded_normal(h->n, h->m0, seed, h->X, h->stream));
  const double *rhs = nullptr;
  int rc = prepare_rhs(h, h->X, &rhs);
  if (rc) return rc;
  rc = set_tolerance(h, 1.0);
  if (rc) return rc;
  int result = IFEAST_ERR_NOT_CONVERGED;
  for (int it = 1; it <= h->opts.max_outer; ++it) {
    rc = clear_step_counters(h);
    if (rc) return rc;
    bool cut = false;  // the Lanczos loop stopped at the time limit
    if (h->minres) {
      MinresArgs ma = minres_args(h, h->X, h->Q, it > 1 ? 1 : 0);
      ma.t0 = t0;
      ma.time_limit_ms = limit_ms;
      ma.cut = &cut;
      CK(minres_filter(ma, h->stream));
    } else if (h->fp32 && it > 1 && h->stats.RF <= h->opts.correction_rf) {  // FP32: residual form
      CK(gmres_filter(gmres_args(h, h->Rres, h->Q, 1), h->stream));
    } else if (h->nonsym && h->opts.nonsym_correction && it > 1) {  // block correction
      rc = ns_block_correction_setup(h);
      if (rc) return rc;
      GmresArgs ga = gmres_args(h, h->Rres, h->Q, 0);
      ga.correction = 2;
      ga.beta = h->rnorm;
      ga.ns_M = h->nsM;
      ga.ns_Gre = h->nsG;
      ga.ns_X = h->X;
      CK(gmres_filter(ga, h->stream));
    } else {  // right-hand sides X, or B X (norms in beta) from the previous Rayleigh-Ritz
      CK(gmres_filter(gmres_args(h, h->rowptrB ? h->BX : h->X, h->Q), h->stream));
    }
    if (h->nonsym)
      CK(rayleigh_ritz_nonsym(rr_args(h, h->Q, h->X), ns_args(h), h->stream));
    else
      CK(rayleigh_ritz(rr_args(h, h->Q, h->X), h->stream));
    CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (h->profiling && h->prof.collect()) return IFEAST_ERR_CUDA;
    const DevStatus s = *h->status_host;
    h->stats.outer_iters = it;
    h->stats.found = s.count;
    h->stats.RF = s.RF;
    h->stats.total_matvecs += s.total_steps;
    h->stats.seq_matvecs += s.max_steps;
    h->stats.max_inner = std::max(h->stats.max_inner, s.max_steps);
    h->stats.shifted_cholesky += s.shifted;
    h->solved = true;
    const double elapsed =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (h->opts.verbose)
      std::fprintf(stderr, "ifeast: iter %3d  inside %4d  RF %.3e  inner max %5d total %9lld  %.1f ms\n",
                   it, s.count, s.RF, s.max_steps, s.total_steps, elapsed);
    if (s.breakdown) {
      result = IFEAST_ERR_BREAKDOWN;
      h->solved = false;
      break;
    }
    if (s.tc_timeout) {  // a bounded device-side wait ran out: the update is incomplete
      result = IFEAST_ERR_TIMEOUT;
      h->solved = false;
      break;
    }
    if (s.count > 0 && s.RF <= h->opts.tol) {
      result = IFEAST_OK;
      break;
    }
    if (cut || (limit_ms > 0.0 && elapsed >= limit_ms)) {
      result = IFEAST_ERR_TIMEOUT;
      break;
    }
  }
  if (result == IFEAST_OK || result == IFEAST_ERR_NOT_CONVERGED) {
    if (h->stats.found >= h->m0) result = IFEAST_ERR_M0_TOO_SMALL;
    else if (h->stats.found == 0) result = IFEAST_STATUS_NO_EIGENVALUES;
  }
  h->stats.solve_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return result;
}

int ifeast_stats(ifeast_t h, ifeast_stats_t *s) {
  if (!h || !s) return IFEAST_ERR_INVALID_ARG;
  *s = h->stats;
  return IFEAST_OK;
}

int ifeast_ritz_all(ifeast_t h, double *lam, double *resid, int out_on_device) {
  if (!h) return IFEAST_ERR_INVALID_ARG;
  if (!h->solved) return IFEAST_ERR_STATE;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (lam) CK(cudaMemcpyAsync(lam, h->lam, h->m0 * sizeof(double), kind, h->stream));
  if (resid) CK(cudaMemcpyAsync(resid, h->res, h->m0 * sizeof(double), kind, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return IFEAST_OK;
}

int ifeast_eigenpairs_complex(ifeast_t h, int cap, int *m_found, double *evals, double *evecs,
                              double *resid, int out_on_device) {
  if (!h || cap < 0) return IFEAST_ERR_INVALID_ARG;
  if (!h->nonsym) return IFEAST_ERR_UNSUPPORTED;
  if (!h->solved) return IFEAST_ERR_STATE;
  const int m0 = h->m0;
  std::vector<double2> th(m0);
  std::vector<double> res(m0);
  CK(cudaMemcpyAsync(th.data(), h->theta, m0 * sizeof(double2), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(res.data(), h->res, m0 * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const double cc = 0.5 * (h->contour.emin + h->contour.emax);
  const double rr = 0.5 * (h->contour.emax - h->contour.emin);
  std::vector<int> idx;
  for (int j = 0; j < m0; ++j)
    if (std::hypot(th[j].x - cc, th[j].y) < rr) idx.push_back(j);
  // Order: ascending real part, a conjugate pair adjacent with the negative
  // imaginary part first. The reduced eigensolver works in complex arithmetic,
  // so the two values of a pair agree only to rounding: both get the mean of
  // their real parts as the sort key.
  std::vector<double> key(m0);
  for (int j = 0; j < m0; ++j) key[j] = th[j].x;
  for (int j = 0; j < m0; ++j) {
    if (th[j].y <= 0.0) continue;
    int best = -1;
    double bd = 0.0;
    for (int k = 0; k < m0; ++k) {
      if (th[k].y >= 0.0) continue;
      const double d = std::hypot(th[k].x - th[j].x, th[k].y + th[j].y);
      if (best < 0 || d < bd) best = k, bd = d;
    }
    if (best >= 0 && bd <= 1e-8 * std::hypot(th[j].x, th[j].y))
      key[j] = key[best] = 0.5 * (th[std::min(j, best)].x + th[std::max(j, best)].x);
  }
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    return key[a] < key[b] ||
           (key[a] == key[b] && (th[a].y < th[b].y || (th[a].y == th[b].y && a < b)));
  });
  const int m = (int)idx.size();
  if (m_found) *m_found = m;
  const int cnt = std::min(m, cap);
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  std::vector<double> ev(2 * (size_t)cnt), rs(cnt);
  for (int q = 0; q < cnt; ++q) {
    ev[2 * q] = th[idx[q]].x;
    ev[2 * q + 1] = th[idx[q]].y;
    rs[q] = res[idx[q]];
  }
  if (evals && cnt) CK(cudaMemcpy(evals, ev.data(), 2 * cnt * sizeof(double), kind));
  if (resid && cnt) CK(cudaMemcpy(resid, rs.data(), cnt * sizeof(double), kind));
  if (evecs && cnt) {
    CK(cudaMemcpyAsync(h->ridx, idx.data(), cnt * sizeof(int), cudaMemcpyHostToDevice,
                       h->stream));
    // the Ritz vectors go to the Q buffer (n x m0 doubles holds n x cnt complex
    // only when 2 cnt <= m0), else to a temporary allocation
    const size_t need = (size_t)h->n * cap * sizeof(double2);
    double2 *out = nullptr;
    bool own = false;
    if (out_on_device) {
      out = reinterpret_cast<double2 *>(evecs);
    } else if (need <= (size_t)h->n * m0 * sizeof(double)) {
      out = reinterpret_cast<double2 *>(h->Q);
    } else {
      if (cudaMallocAsync(reinterpret_cast<void **>(&out), need, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return IFEAST_ERR_OOM;
      }
      own = true;
    }
    CK(ritz_vectors_nonsym((int)h->n, m0, h->X, h->Uc, h->ridx, cnt, cap, out, h->stream));
    if (!out_on_device)
      CK(cudaMemcpyAsync(evecs, out, need, cudaMemcpyDeviceToHost, h->stream));
    if (own) CK(cudaFreeAsync(out, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return IFEAST_OK;
}

int ifeast_rayleigh_ritz_nonsym(ifeast_t h, const double *Q, double *X, double *theta,
                                double *resid) {
  if (!h || !Q || !X) return IFEAST_ERR_INVALID_ARG;
  if (!h->nonsym) return IFEAST_ERR_UNSUPPORTED;
  int rc = set_tolerance(h, 1.0);
  if (rc) return rc;
  CK(rayleigh_ritz_nonsym(rr_args(h, Q, X), ns_args(h), h->stream));
  CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                     h->stream));
  if (theta)
    CK(cudaMemcpyAsync(theta, h->theta, h->m0 * sizeof(double2), cudaMemcpyDeviceToDevice,
                       h->stream));
  if (resid)
    CK(cudaMemcpyAsync(resid, h->res, h->m0 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->profiling && h->prof.collect()) return IFEAST_ERR_CUDA;
  if (h->status_host->breakdown) return IFEAST_ERR_BREAKDOWN;
  return IFEAST_OK;
}

int ifeast_eigenpairs(ifeast_t h, int cap, int *m_found, double *evals, double *evecs,
                      double *resid, int out_on_device) {
  if (h && h->nonsym) return IFEAST_ERR_UNSUPPORTED;
  if (!h || cap < 0) return IFEAST_ERR_INVALID_ARG;
  if (!h->solved) return IFEAST_ERR_STATE;
  std::vector<double> lam(h->m0), res(h->m0);
  CK(cudaMemcpyAsync(lam.data(), h->lam, h->m0 * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(res.data(), h->res, h->m0 * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::vector<int> idx;
  for (int j = 0; j < h->m0; ++j)
    if (lam[j] > h->contour.emin && lam[j] < h->contour.emax) idx.push_back(j);
  const int m = (int)idx.size();
  if (m_found) *m_found = m;
  const int cnt = std::min(m, cap);
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  std::vector<double> ev(cnt), rs(cnt);
  for (int q = 0; q < cnt; ++q) {
    ev[q] = lam[idx[q]];
    rs[q] = res[idx[q]];
  }
  if (evals && cnt) CK(cudaMemcpy(evals, ev.data(), cnt * sizeof(double), kind));
  if (resid && cnt) CK(cudaMemcpy(resid, rs.data(), cnt * sizeof(double), kind));
  if (evecs && cnt) {
    // the in-interval columns are contiguous in the ascending order: idx[0]..idx[cnt-1]
    const size_t total = (size_t)h->n * cnt;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (out_on_device) {  // gathered straight into the caller's n x cap block
      k_gather_columns<<<blocks, 256, 0, h->stream>>>(h->n, h->m0, idx[0], cnt, cap, h->X, evecs);
      CK(cudaGetLastError());
    } else if (cap == cnt) {
      // gathered into the A Q scratch block (free after the solve), then one
      // contiguous copy: a strided copy of 8 cnt bytes per row is far slower
      k_gather_columns<<<blocks, 256, 0, h->stream>>>(h->n, h->m0, idx[0], cnt, cnt, h->X, h->AQ);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(evecs, h->AQ, total * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
    } else {  // wider host block: only the cnt columns may be written
      CK(cudaMemcpy2DAsync(evecs, (size_t)cap * sizeof(double), h->X + idx[0],
                           (size_t)h->m0 * sizeof(double), cnt * sizeof(double), (size_t)h->n,
                           cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
  }
  return IFEAST_OK;
}

int ifeast_apply_filter(ifeast_t h, const double *X, double *Q, double RF, int32_t *steps) {
  if (!h || !X || !Q || !(RF >= 0.0)) return IFEAST_ERR_INVALID_ARG;
  const double *rhs = nullptr;
  int rc = prepare_rhs(h, X, &rhs);
  if (rc) return rc;
  rc = set_tolerance(h, RF);
  if (rc) return rc;
  if (h->minres)
    CK(minres_filter(minres_args(h, X, Q, 0), h->stream));
  else
    CK(gmres_filter(gmres_args(h, rhs, Q), h->stream));
  if (steps)
    CK(cudaMemcpyAsync(steps, h->minres ? h->lsteps : h->steps, h->C * sizeof(int),
                       cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->profiling && h->prof.collect()) return IFEAST_ERR_CUDA;
  return IFEAST_OK;
}

int ifeast_apply_filter_residual(ifeast_t h, const double *X, const double *lam, double *Q,
                                 double RF, int32_t *steps) {
  if (!h || !X || !lam || !Q || !(RF >= 0.0)) return IFEAST_ERR_INVALID_ARG;
  if (h->nonsym || (!h->minres && !h->fp32)) return IFEAST_ERR_UNSUPPORTED;
  h->solved = false;
  Profiler *pf = h->profiling ? &h->prof : nullptr;
  const size_t nm = (size_t)h->n * h->m0;
  CK(cudaMemcpyAsync(h->X, X, nm * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->lam, lam, h->m0 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  // B x_j (x_j for B = I), its norms (the stop test's scale), r_j and ||r_j||
  const double *bx = h->X;
  if (h->rowptrB) {
    CK(spmm_block((int)h->n, h->m0, h->rowptrB, h->colidxB, h->valB, h->X, h->BX, h->Pg,
                  h->stream));
    bx = h->BX;
  }
  CK(column_norms((int)h->n, h->m0, bx, h->res_part, h->Pr, h->beta, h->stream, pf));
  CK(residual_block((int)h->n, h->m0, h->rowptr, h->colidx, h->val, h->X, bx, h->lam, h->Rres,
                    h->stream));
  CK(column_norms((int)h->n, h->m0, h->Rres, h->res_part, h->Pr, h->rnorm, h->stream, pf));
  int rc = set_tolerance(h, RF);
  if (rc) return rc;
  if (h->minres)
    CK(minres_filter(minres_args(h, h->X, Q, 1), h->stream));
  else
    CK(gmres_filter(gmres_args(h, h->Rres, Q, 1), h->stream));
  if (steps)
    CK(cudaMemcpyAsync(steps, h->minres ? h->lsteps : h->steps, h->C * sizeof(int),
                       cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->profiling && h->prof.collect()) return IFEAST_ERR_CUDA;
  return IFEAST_OK;
}

int ifeast_rayleigh_ritz(ifeast_t h, const double *Q, double *X, double *lam, double *resid) {
  if (!h || !Q || !X) return IFEAST_ERR_INVALID_ARG;
  int rc = set_tolerance(h, 1.0);
  if (rc) return rc;
  CK(rayleigh_ritz(rr_args(h, Q, X), h->stream));
  CK(cudaMemcpyAsync(h->status_host, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                     h->stream));
  if (lam) CK(cudaMemcpyAsync(lam, h->lam, h->m0 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (resid)
    CK(cudaMemcpyAsync(resid, h->res, h->m0 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (h->profiling && h->prof.collect()) return IFEAST_ERR_CUDA;
  if (h->status_host->breakdown) return IFEAST_ERR_BREAKDOWN;
  if (h->status_host->tc_timeout) return IFEAST_ERR_TIMEOUT;
  return IFEAST_OK;
}

int ifeast_spmm_shift(ifeast_t h, const double *V, double *W, int ncols, int m0, const double *z) {
  if (!h || !V || !W || !z || ncols < 1 || m0 < 1 || ncols % m0 != 0 || ncols / m0 > kMaxNodes)
    return IFEAST_ERR_INVALID_ARG;
  const RowTiling tl = make_tiling(h->n, ncols, h->num_sms);
  CK(spmm_shift_only((int)h->n, h->rowptr, h->colidx, h->val, (const double2 *)V, (double2 *)W,
                     ncols, m0, (const double2 *)z, tl, h->stream, h->rowptrB, h->colidxB,
                     h->valB));
  CK(cudaStreamSynchronize(h->stream));
  return IFEAST_OK;
}

int ifeast_set_profiling(ifeast_t h, int on) {
  if (!h || on < 0) return IFEAST_ERR_INVALID_ARG;
  if (on && !h->prof.events) {
    const int cap = 4096;
    h->prof.events = new (std::nothrow) cudaEvent_t[2 * cap];
    h->prof.kid = new (std::nothrow) int[cap];
    if (!h->prof.events || !h->prof.kid) return IFEAST_ERR_OOM;
    for (int i = 0; i < 2 * cap; ++i)
      if (cudaEventCreate(&h->prof.events[i]) != cudaSuccess) {
        for (int k = 0; k < i; ++k) cudaEventDestroy(h->prof.events[k]);
        delete[] h->prof.events;
        delete[] h->prof.kid;
        h->prof.events = nullptr;
        h->prof.kid = nullptr;
        return IFEAST_ERR_CUDA;
      }
    h->prof.cap = cap;
  }
  h->prof.stream = h->stream;
  h->prof.used = 0;
  h->prof.sample_every = on > 1 ? on : 1;
  h->prof.skipping = false;
  if (on)
    for (long long &c : h->prof.launches) c = 0;
  h->profiling = on != 0;
  return IFEAST_OK;
}

int ifeast_kernel_times(ifeast_t h, int cap, double *ms, int64_t *launches, int reset) {
  if (!h || cap < 0) return IFEAST_ERR_INVALID_ARG;
  for (int k = 0; k < K_COUNT && k < cap; ++k) {
    if (ms) ms[k] = h->prof.ms[k];
    if (launches) launches[k] = h->prof.count[k];
  }
  if (reset)
    for (int k = 0; k < K_COUNT; ++k) {
      h->prof.ms[k] = 0.0;
      h->prof.count[k] = 0;
    }
  return K_COUNT;
}

int ifeast_kernel_launches(ifeast_t h, int cap, int64_t *launches, int reset) {
  if (!h || cap < 0) return IFEAST_ERR_INVALID_ARG;
  for (int k = 0; k < K_COUNT && k < cap; ++k)
    if (launches) launches[k] = h->prof.launches[k];
  if (reset)
    for (int k = 0; k < K_COUNT; ++k) h->prof.launches[k] = 0;
  return K_COUNT;
}

const char *ifeast_kernel_name(int k) {
  static const char *names[K_COUNT] = {
      "prep",           "colnorm",          "colnorm_reduce", "gmres_spmm_dot",
      "gmres_reduce",   "gmres_orth",       "gmres_givens",   "gmres_finish",
      "gmres_solve",    "gmres_quadrature", "lanczos_step",   "lanczos_givens",
      "lanczos_solve",  "lanczos_coef",     "lanczos_quadrature", "rr_spmm",
      "rr_gram",        "rr_gram_reduce",   "rr_eig",         "rr_update_resid",
      "rr_resid_reduce", "lanczos_reduce"};
  return (k >= 0 && k < K_COUNT) ? names[k] : "unknown";
}

}  // extern "C"
