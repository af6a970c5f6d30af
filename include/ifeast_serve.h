/*
 * ifeast_serve.h -- continuous serving of many IFEAST solves on one GPU.
 *
 * A server accepts eigen-requests (matrix, interval, subspace size, options,
 * initial subspace) at any time and runs them with overlapping work on the
 * device: every admitted request gets its own handle (ifeast.h), its own CUDA
 * stream and a worker thread that drives its outer iterations, so the kernels
 * of different requests interleave on the GPU. A request is admitted, in
 * arrival order, as soon as its device workspace fits in the remaining memory
 * budget and an execution slot is free; its memory returns to the budget when
 * it finishes. Each request's subspace and Krylov state stay resident in its
 * workspace across its outer iterations.
 *
 * Every kernel of a solve uses fixed-order reductions, so a request's result
 * does not depend on which other requests share the GPU.
 *
 * All functions return an ifeast_status code. Host pointers only; inputs are
 * copied at submit time.
 */
#ifndef IFEAST_SERVE_H
#define IFEAST_SERVE_H

#include "ifeast.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifeast_server *ifeast_server_t;

typedef struct {
  size_t mem_budget_bytes;  /* device memory the admitted requests may hold together */
  int max_active;           /* requests running at once (worker threads), >= 1      */
  int device;               /* CUDA device ordinal                                  */
} ifeast_server_opts;

typedef struct {
  int status;               /* ifeast_status of the solve                           */
  int found;                /* eigenpairs inside the interval                       */
  int outer_iters;
  double RF;
  double submit_to_start_ms;  /* queueing delay (admission wait)                    */
  double submit_to_done_ms;   /* latency                                            */
  size_t workspace_bytes;
} ifeast_request_info;

int ifeast_server_create(const ifeast_server_opts *o, ifeast_server_t *out);

/* Queues one request. A (host CSR) and X0 (n x m0 row-major host array) are
 * copied before the call returns. *id receives the request id (>= 0).
 * INVALID_ARG / UNSUPPORTED as ifeast_create; OOM if the request's workspace
 * alone exceeds the whole budget. */
int ifeast_server_submit(ifeast_server_t s, const ifeast_csr *A, const ifeast_contour *c, int m0,
                         const ifeast_opts *o, const double *X0, int64_t *id);

/* Blocks until request id has finished, then copies its results like
 * ifeast_eigenpairs (host outputs, any may be NULL; evecs n x cap row-major)
 * and its record into *info (may be NULL). Each id can be waited for once;
 * the results are released afterwards. Returns the request's solve status,
 * or INVALID_ARG for an unknown id. */
int ifeast_server_wait(ifeast_server_t s, int64_t id, int cap, int *m_found, double *evals,
                       double *evecs, double *resid, ifeast_request_info *info);

/* Waits for every queued request and stops the worker threads. */
void ifeast_server_destroy(ifeast_server_t s);

#ifdef __cplusplus
}
#endif
#endif
