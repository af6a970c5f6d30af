// Rayleigh-Ritz step (Algorithm 2, step 3, with the step-4 residuals) for
// callers that cannot allocate device memory, e.g. code running inside a
// memory pool, a graphics or real-time runtime that forbids cudaMalloc, or a
// host that has reserved all device memory up front. It computes the same
// X, lambda and residuals as ifeast_rayleigh_ritz but takes the matrix as
// caller-owned device CSR arrays and keeps every intermediate in one
// fixed-size array in this library's device memory (no handle, no workspace).
//
// Scratch: g_scratch below, kNaScratchDoubles doubles (about 4.5 MiB), a
// file-scope __device__ array: every GPU that loads the library holds it until
// the process exits. All calls share it, so calls that overlap on the GPU
// (other streams, other host threads) race and must be serialised by the
// caller. Each call overwrites every scratch entry it reads before reading
// it, so nothing left by an earlier call leaks into the result.
//
// Differences from the handle-based kernels (same mathematics): A Q is formed
// per chunk of rows in shared memory and never stored, and A X is formed from
// the new X instead of from A Q X_Q.
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace ifeast {
namespace {

constexpr int kNaMaxM0 = 64;    // largest m0 the fixed scratch holds
constexpr int kNaBlocks = 64;   // blocks of the row-parallel kernels (partials)
constexpr int kNaRows = 16;     // rows staged per chunk in the Gram kernel
constexpr size_t kNaGram = (size_t)kNaBlocks * 2 * kNaMaxM0 * kNaMaxM0;
constexpr size_t kNaMat = (size_t)kNaMaxM0 * kNaMaxM0;
constexpr size_t kNaRes = (size_t)kNaBlocks * 2 * kNaMaxM0;
constexpr size_t kNaStatus = (sizeof(DevStatus) + sizeof(double) - 1) / sizeof(double);
constexpr size_t kNaScratchDoubles = kNaGram + 6 * kNaMat + kNaRes + kNaStatus + 8;

__device__ __align__(256) double g_scratch[kNaScratchDoubles];

// Partials of Q^T A Q and Q^T Q: each chunk of kNaRows rows stages Q and the
// rows of A Q (computed here from the CSR) in shared memory; thread t owns the
// 4x4 tile t of the upper triangle (m0 padded to mp, a multiple of 4).
__global__ void __launch_bounds__(256)
k_na_gram(int n, int m, int mp, const int32_t *__restrict__ rowptr,
          const int32_t *__restrict__ colidx, const double *__restrict__ val,
          const double *__restrict__ Q, double *__restrict__ part) {
  __shared__ double Qs[kNaRows][kNaMaxM0];
  __shared__ double As[kNaRows][kNaMaxM0];
  const int nt = mp / 4;
  const int ntiles = nt * (nt + 1) / 2;
  const int tile = threadIdx.x;
  int ti = 0, tj = 0;
  const bool own = tile < ntiles;
  if (own) {
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
  for (int r0 = blockIdx.x * kNaRows; r0 < n; r0 += gridDim.x * kNaRows) {
    for (int e = threadIdx.x; e < kNaRows * kNaMaxM0; e += blockDim.x) {
      const int rr = e / kNaMaxM0, j = e % kNaMaxM0, r = r0 + rr;
      double q = 0.0, aq = 0.0;
      if (r < n && j < m) {
        q = Q[(size_t)r * m + j];
        for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) aq = fma(val[p], Q[(size_t)colidx[p] * m + j], aq);
      }
      Qs[rr][j] = q;
      As[rr][j] = aq;
    }
    __syncthreads();
    if (own) {
      for (int rr = 0; rr < kNaRows; ++rr) {
        double qi[4], qj[4], aj[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          qi[p] = Qs[rr][4 * ti + p];
          qj[p] = Qs[rr][4 * tj + p];
          aj[p] = As[rr][4 * tj + p];
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
  // every tile of the upper triangle is written, so no stale entry is read
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

// Fixed-order sum of the partials into full symmetric A_Q, B_Q.
__global__ void k_na_reduce_gram(int nb, int m, int mp, const double *__restrict__ part,
                                 double *__restrict__ Aq, double *__restrict__ Bq) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m) return;
  const int i = idx / m, j = idx % m;
  if (i > j) return;
  const bool same_tile = (i / 4) == (j / 4);
  double sa = 0.0, sb = 0.0, sa2 = 0.0;
  for (int b = 0; b < nb; ++b) {
    const double *pa = part + (size_t)b * 2 * mp * mp;
    const double *pb = pa + (size_t)mp * mp;
    sa += pa[(size_t)i * mp + j];
    sb += pb[(size_t)i * mp + j];
    if (same_tile) sa2 += pa[(size_t)j * mp + i];
  }
  if (same_tile) sa = 0.5 * (sa + sa2);
  Aq[(size_t)i * m + j] = sa;
  Aq[(size_t)j * m + i] = sa;
  Bq[(size_t)i * m + j] = sb;
  Bq[(size_t)j * m + i] = sb;
}

// X = Q X_Q.
__global__ void k_na_update(int n, int m, const double *__restrict__ Q,
                            const double *__restrict__ XQ, double *__restrict__ X) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * m) return;
  const size_t r = idx / m;
  const int j = (int)(idx % m);
  double x = 0.0;
  for (int i = 0; i < m; ++i) x = fma(Q[r * m + i], XQ[(size_t)i * m + j], x);
  X[idx] = x;
}

// Partials of ||A x_j - lambda_j x_j||^2 and ||A x_j||^2; thread per column
// within a 32-column tile, rows strided over the grid (fixed order).
__global__ void __launch_bounds__(256)
k_na_resid(int n, int m, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx,
           const double *__restrict__ val, const double *__restrict__ X,
           const double *__restrict__ lam, double *__restrict__ part) {
  __shared__ double red[2][8][kNaMaxM0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double e2[2] = {0.0, 0.0}, a2[2] = {0.0, 0.0};
  for (int t = 0; t < 2; ++t) {
    const int j = lane + 32 * t;
    if (j >= m) continue;
    const double lj = lam[j];
    for (int r = blockIdx.x * 8 + warp; r < n; r += gridDim.x * 8) {
      double ax = 0.0;
      for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) ax = fma(val[p], X[(size_t)colidx[p] * m + j], ax);
      const double d = ax - lj * X[(size_t)r * m + j];
      e2[t] = fma(d, d, e2[t]);
      a2[t] = fma(ax, ax, a2[t]);
    }
  }
  for (int t = 0; t < 2; ++t) {
    red[0][warp][lane + 32 * t] = e2[t];
    red[1][warp][lane + 32 * t] = a2[t];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * m; e += blockDim.x) {
    const int k = e / m, j = e % m;
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[k][w][j];
    part[((size_t)blockIdx.x * 2 + k) * m + j] = s;
  }
}

__global__ void k_na_reduce_resid(int nb, int m, const double *__restrict__ part,
                                  double *__restrict__ res) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double e = 0.0, a = 0.0;
  for (int b = 0; b < nb; ++b) {
    e += part[((size_t)b * 2 + 0) * m + j];
    a += part[((size_t)b * 2 + 1) * m + j];
  }
  res[j] = sqrt(e) / (a > 0.0 ? sqrt(a) : 1.0);
}

std::mutex g_na_mu;
double *g_na_ptr[64] = {nullptr};

// Device address of g_scratch for the current device (looked up once per
// device; the host symbol itself is not a device address).
int scratch_for_current_device(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return IFEAST_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return IFEAST_ERR_CUDA;
    }
    if (rr_init() != cudaSuccess) return IFEAST_ERR_CUDA;  // shared-memory opt-in of the eigensolver
    g_na_ptr[dev] = (double *)p;
  }
  *out = g_na_ptr[dev];
  return IFEAST_OK;
}

}  // namespace
}  // namespace ifeast

using namespace ifeast;

extern "C" int ifeast_rayleigh_ritz_noalloc(int64_t n, int64_t nnz, const int32_t *rowptr,
                                            const int32_t *colidx, const double *val, int m0,
                                            const double *Q, double *X, double *lam,
                                            double *resid, void *stream) {
  if (n < 1 || nnz < 0 || n > INT32_MAX - 1 || !rowptr || (nnz > 0 && (!colidx || !val)) || !Q ||
      !X || !lam || !resid || m0 < 1 || m0 > n)
    return IFEAST_ERR_INVALID_ARG;
  if (m0 > kNaMaxM0) return IFEAST_ERR_INVALID_ARG;  // beyond the fixed scratch
  {  // X = Q X_Q reads all of a row of Q while it writes that row of X
    const uintptr_t q0 = (uintptr_t)Q, x0 = (uintptr_t)X;
    const uintptr_t len = (uintptr_t)n * (uintptr_t)m0 * sizeof(double);
    if (q0 < x0 + len && x0 < q0 + len) return IFEAST_ERR_INVALID_ARG;
  }
  double *sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int m = m0;
  const int mp = (m + 3) / 4 * 4;
  double *gram_part = sc;
  double *Aq = gram_part + kNaGram;
  double *Bq = Aq + kNaMat;
  double *L = Bq + kNaMat;
  double *Cm = L + kNaMat;
  double *U = Cm + kNaMat;
  double *XQ = U + kNaMat;
  double *res_part = XQ + kNaMat;
  DevStatus *status = reinterpret_cast<DevStatus *>(res_part + kNaRes);
  const int nb = (int)std::min<int64_t>(kNaBlocks, (n + kNaRows - 1) / kNaRows);
  if (cudaMemsetAsync(status, 0, sizeof(DevStatus), st) != cudaSuccess) return IFEAST_ERR_CUDA;
  k_na_gram<<<nb, 256, 0, st>>>((int)n, m, mp, rowptr, colidx, val, Q, gram_part);
  k_na_reduce_gram<<<(m * m + 255) / 256, 256, 0, st>>>(nb, m, mp, gram_part, Aq, Bq);
  if (cudaGetLastError() != cudaSuccess) return IFEAST_ERR_CUDA;
  if (reduced_eig_launch(m, Aq, Bq, L, Cm, U, XQ, lam, status, st) != cudaSuccess)
    return IFEAST_ERR_CUDA;
  const size_t nm = (size_t)n * m;
  k_na_update<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>((int)n, m, Q, XQ, X);
  const int nr = (int)std::min<int64_t>(kNaBlocks, (n + 7) / 8);
  k_na_resid<<<nr, 256, 0, st>>>((int)n, m, rowptr, colidx, val, X, lam, res_part);
  k_na_reduce_resid<<<(m + 127) / 128, 128, 0, st>>>(nr, m, res_part, resid);
  if (cudaGetLastError() != cudaSuccess) return IFEAST_ERR_CUDA;
  int breakdown = 0;  // pageable host copy: no allocation
  if (cudaMemcpyAsync(&breakdown, &status->breakdown, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return IFEAST_ERR_CUDA;
  return breakdown ? IFEAST_ERR_BREAKDOWN : IFEAST_OK;
}
