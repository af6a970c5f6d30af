// Reduced eigenproblem of the Rayleigh-Ritz step (Algorithm 2, step 3): the
// FP64 cyclic Jacobi sweeps on C = L^-1 A_Q L^-T, spread over a thread-block
// cluster.
//
// On one SM the FP64 sweeps of an 80 x 80 C take milliseconds (this GPU issues
// one FP64 warp instruction per 64 cycles per SM sub-partition), so here they
// run on kEigCtas CTAs of one cluster: CTA g owns rows [g R, (g + 1) R) of C
// and of the rotation product V (R = ceil(m / kEigCtas)) in its shared memory.
// One round of a sweep applies the m/2 disjoint rotations J of the round-robin
// pairing:
//   1. every CTA forms all of the round's rotations from C[a][a], C[b][b] and
//      C[a][b], read from the owners' shared memory (distributed shared
//      memory), with the rule of the single-CTA solver (while the
//      off-diagonal part is still large, tan(theta) in FP32 and c, s made
//      orthonormal in FP64 by Newton-Raphson steps for 1/sqrt(1 + t^2));
//   2. C <- J^T C: each new row combines the CTA's old row with its partner
//      row (read from the partner's owner) into the second buffer;
//   3. cluster barrier;
//   4. C <- C J and V <- V J on the CTA's own rows (columns a and b);
//   5. cluster barrier, and the buffers swap.
// A sweep starts with the squared off-diagonal and whole Frobenius norms,
// summed per CTA and then over the CTAs in rank order (the same value in
// every CTA, so every CTA takes the same branches). k_reduced_eig forms C
// before (stage 1) and sorts the pairs and solves X_Q = L^-T V after (stage 2).
#include <cooperative_groups.h>

#include <cfloat>

#include "internal.h"

namespace cg = cooperative_groups;

namespace ifeast {

namespace {

constexpr int kEigCtas = 8;       // CTAs of the cluster (portable size)
constexpr int kEigThreads = 256;  // threads per CTA
constexpr int kEigMinM = 24;     // below this one CTA is as fast
constexpr int kRowBatch = 4;     // partner-row elements a thread loads at once
// squared off-diagonal / whole norm above which a sweep forms its rotation
// angles in FP32
constexpr double kCoarseAngles = 1e-10;

// Dynamic shared memory of k_eig_sweeps for an m x m problem: two buffers of
// the CTA's rows of C (the row phase writes the other one) and its rows of V.
size_t sweep_smem_bytes(int m) {
  const size_t R = (size_t)(m + kEigCtas - 1) / kEigCtas;
  return 3 * R * (size_t)(m | 1) * sizeof(double);
}

__device__ __forceinline__ double block_sum_c(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kEigThreads / 32; ++w) t += red[w];
  return t;
}

// Cyclic Jacobi on the symmetric m x m matrix in Cg (row-major, leading
// dimension m), V accumulating the rotations from I. On return evals[i] =
// the final diagonal entry i (unsorted) and Cg holds V (column i belongs to
// evals[i]). Rotation rule and stop test of the single-CTA FP64 sweeps: a sweep starts
// only while the squared off-diagonal norm exceeds stop times the squared
// Frobenius norm, and a sweep that rotates nothing ends the iteration.
__global__ void __cluster_dims__(kEigCtas, 1, 1) __launch_bounds__(kEigThreads)
k_eig_sweeps(int m, double *__restrict__ Cg, double *__restrict__ evals, int max_sweeps,
             double stop) {
  cg::cluster_group cl = cg::this_cluster();
  const int g = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int R = (m + kEigCtas - 1) / kEigCtas;
  const int ld = m | 1;
  const int r0 = g * R, nr = max(0, min(m, r0 + R) - r0);
  const int mp = m + (m & 1), npairs = mp / 2;
  extern __shared__ double sm[];
  double *Cbuf = sm;                        // [2][R][ld]
  double *V = sm + 2 * (size_t)R * ld;      // [R][ld]
  __shared__ double rc[kMaxM0 / 2], rs[kMaxM0 / 2];
  __shared__ int ra[kMaxM0 / 2], rb[kMaxM0 / 2];
  __shared__ double self_c[kMaxM0], part_c[kMaxM0];
  __shared__ int partner[kMaxM0];
  __shared__ double red[kEigThreads / 32];
  __shared__ double norms[2];  // this CTA's squared off-diagonal and whole norms
  __shared__ double totals[2];
  __shared__ int any_rot;

  for (int e = tid; e < nr * m; e += kEigThreads) {
    const int li = e / m, k = e % m;
    Cbuf[(size_t)li * ld + k] = Cg[(size_t)(r0 + li) * m + k];
    V[(size_t)li * ld + k] = (r0 + li == k) ? 1.0 : 0.0;
  }
  cl.sync();  // every CTA of the cluster runs and holds its rows
  int cur = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    const double *C = Cbuf + (size_t)cur * R * ld;
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < nr * m; e += kEigThreads) {
      const int li = e / m, k = e % m;
      const double v = C[(size_t)li * ld + k] * C[(size_t)li * ld + k];
      tot += v;
      if (r0 + li != k) off += v;
    }
    off = block_sum_c(off, red);
    tot = block_sum_c(tot, red);
    if (tid == 0) {
      norms[0] = off;
      norms[1] = tot;
    }
    cl.sync();
    if (tid == 0) {  // the same sums, in rank order, in every CTA
      double so = 0.0, st = 0.0;
      for (int r = 0; r < kEigCtas; ++r) {
        const double *p = cl.map_shared_rank(norms, r);
        so += p[0];
        st += p[1];
      }
      totals[0] = so;
      totals[1] = st;
      any_rot = 0;
    }
    cl.sync();  // norms read everywhere before they change or a CTA exits
    if (!(totals[0] > stop * totals[1])) break;
    // rotation angles in FP32 while the off-diagonal part is large, exact FP64
    // angles for the final sweeps (their quadratic convergence)
    const bool coarse = totals[0] > kCoarseAngles * totals[1];
    for (int round = 0; round < mp - 1; ++round) {
      const double *Cc = Cbuf + (size_t)cur * R * ld;
      double *Cn = Cbuf + (size_t)(cur ^ 1) * R * ld;
      // 1. the round's rotations (all of them, in every CTA)
      for (int p = tid; p < npairs; p += kEigThreads) {
        const int pa = p, pb = mp - 1 - p;
        int a = pa == 0 ? 0 : 1 + (pa - 1 + round) % (mp - 1);
        int b = pb == 0 ? 0 : 1 + (pb - 1 + round) % (mp - 1);
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        double c = 1.0, s = 0.0;
        if (b < m) {
          const double *ca = cl.map_shared_rank(Cc, a / R) + (size_t)(a % R) * ld;
          const double *cb = cl.map_shared_rank(Cc, b / R) + (size_t)(b % R) * ld;
          const double apq = ca[b], app = ca[a], aqq = cb[b];
          if (fabs(apq) > 1e-300 && fabs(apq) > DBL_EPSILON * sqrt(fabs(app * aqq))) {
            double t;
            // (FP32 only where tau stays a normal FP32 number)
            if (coarse && fabs(apq) > 1e-30 && fabs(aqq - app) < 1e30) {
              // t = tan(theta) in FP32 (~1e-7 relative: the rotation then leaves
              // ~1e-7 of C[a][b], far below the off-diagonal mass of a coarse
              // sweep); c = (1 + t^2)^-1/2 from rsqrtf and two FP64 Newton
              // steps, so that c^2 + s^2 = 1 to FP64 rounding
              const float tau = (float)(aqq - app) / (2.f * (float)apq);
              const float tf = (tau >= 0.f ? 1.f : -1.f) /
                               (fabsf(tau) + (fabsf(tau) < 1e18f ? sqrtf(1.f + tau * tau) : fabsf(tau)));
              t = tf;
              const double x = 1.0 + t * t;
              double y = rsqrtf((float)x);
              y = y * (1.5 - 0.5 * x * y * y);
              y = y * (1.5 - 0.5 * x * y * y);
              c = y;
            } else {
              const double tau = (aqq - app) / (2.0 * apq);
              t = (tau >= 0.0 ? 1.0 : -1.0) /
                  (fabs(tau) + (fabs(tau) < 1e150 ? sqrt(1.0 + tau * tau) : fabs(tau)));
              c = 1.0 / sqrt(1.0 + t * t);
            }
            s = t * c;
            if (s != 0.0) any_rot = 1;  // every writer stores the same value
          }
        }
        ra[p] = a;
        rb[p] = b < m ? b : a;
        rc[p] = c;
        rs[p] = s;
        const bool rot = b < m && s != 0.0;
        partner[a] = rot ? b : -1;
        self_c[a] = c;
        part_c[a] = -s;
        if (b < m) {
          partner[b] = rot ? a : -1;
          self_c[b] = c;
          part_c[b] = s;
        }
      }
      __syncthreads();
      // 2. rows: C <- J^T C into the other buffer (partner rows from their
      // owners; a thread's remote loads are all issued before they are used)
      for (int e0 = 0; e0 < nr * m; e0 += kRowBatch * kEigThreads) {
        double xp[kRowBatch];
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
          const int e = e0 + u * kEigThreads + tid;
          xp[u] = 0.0;
          if (e < nr * m) {
            const int li = e / m, k = e % m, pr = partner[r0 + li];
            if (pr >= 0) xp[u] = cl.map_shared_rank(Cc, pr / R)[(size_t)(pr % R) * ld + k];
          }
        }
#pragma unroll
        for (int u = 0; u < kRowBatch; ++u) {
          const int e = e0 + u * kEigThreads + tid;
          if (e < nr * m) {
            const int li = e / m, k = e % m, i = r0 + li;
            const double x = Cc[(size_t)li * ld + k];
            Cn[(size_t)li * ld + k] = partner[i] >= 0 ? self_c[i] * x + part_c[i] * xp[u] : x;
          }
        }
      }
      cl.sync();  // all new rows written, all reads of the old buffer done
      // 3. columns: C <- C J, V <- V J on this CTA's rows
      for (int e = tid; e < nr * npairs; e += kEigThreads) {
        const int li = e / npairs, p = e % npairs;
        const int a = ra[p], b = rb[p];
        const double s = rs[p];
        if (a == b || s == 0.0) continue;
        const double c = rc[p];
        double *row = Cn + (size_t)li * ld;
        const double x = row[a], y = row[b];
        row[a] = c * x - s * y;
        row[b] = s * x + c * y;
        double *vr = V + (size_t)li * ld;
        const double u = vr[a], v = vr[b];
        vr[a] = c * u - s * v;
        vr[b] = s * u + c * v;
      }
      cur ^= 1;
      cl.sync();  // the round is complete in every CTA
    }
    if (!any_rot) break;
  }
  const double *C = Cbuf + (size_t)cur * R * ld;
  for (int li = tid; li < nr; li += kEigThreads) evals[r0 + li] = C[(size_t)li * ld + r0 + li];
  for (int e = tid; e < nr * m; e += kEigThreads) {
    const int li = e / m, k = e % m;
    Cg[(size_t)(r0 + li) * m + k] = V[(size_t)li * ld + k];
  }
}

}  // namespace

bool eig_cluster_supported(int m) { return m >= kEigMinM && m <= kMaxM0; }

cudaError_t eig_cluster_init() {
  return cudaFuncSetAttribute(k_eig_sweeps, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_smem_bytes(kMaxM0));
}

cudaError_t eig_sweeps_launch(int m, double *C, double *evals, cudaStream_t st) {
  if (!eig_cluster_supported(m)) return cudaErrorInvalidValue;
  k_eig_sweeps<<<kEigCtas, kEigThreads, sweep_smem_bytes(m), st>>>(m, C, evals, 60, 1e-28);
  return cudaGetLastError();
}

}  // namespace ifeast
