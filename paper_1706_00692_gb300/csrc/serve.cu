// Continuous serving of IFEAST solves (include/ifeast_serve.h): FIFO admission
// under a device-memory budget, one handle + stream + worker thread per running
// request, results kept until the caller waits for them.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ifeast_serve.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  int64_t n = 0, nnz = 0;
  std::vector<int32_t> rowptr, colidx;
  std::vector<double> val;
  ifeast_contour contour{};
  std::vector<double> user_zw;  // IFEAST_USER nodes (contour.user_zw points here)
  ifeast_opts opts{};
  int m0 = 0;
  std::vector<double> X0;
  size_t ws_bytes = 0;
  Clock::time_point t_submit, t_start, t_done;
  bool done = false;
  int status = IFEAST_OK;
  ifeast_stats_t stats{};
  int found = 0;
  std::vector<double> evals, evecs, resid;  // evecs n x found row-major
};

}  // namespace

struct ifeast_server {
  ifeast_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv;  // admission and completion
  std::deque<std::shared_ptr<Request>> pending;
  std::map<int64_t, std::shared_ptr<Request>> requests;
  size_t used = 0;
  bool stopping = false;
  int64_t next_id = 0;
  std::vector<std::thread> workers;
};

namespace {

void run_request(const ifeast_server_opts &so, Request &r) {
  if (cudaSetDevice(so.device) != cudaSuccess) {
    r.status = IFEAST_ERR_CUDA;
    return;
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    r.status = IFEAST_ERR_CUDA;
    return;
  }
  void *ws = nullptr;
  if (cudaMallocAsync(&ws, r.ws_bytes, st) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(st);
    r.status = IFEAST_ERR_OOM;
    return;
  }
  ifeast_csr A{r.n, r.nnz, r.rowptr.data(), r.colidx.data(), r.val.data()};
  ifeast_t h = nullptr;
  int rc = ifeast_create(&A, nullptr, &r.contour, r.m0, &r.opts, ws, r.ws_bytes, st, &h);
  if (rc == IFEAST_OK) {
    rc = ifeast_solve(h, r.X0.data(), 0, 0, nullptr);
    ifeast_stats(h, &r.stats);
    if (rc == IFEAST_OK || rc == IFEAST_ERR_NOT_CONVERGED || rc == IFEAST_ERR_M0_TOO_SMALL) {
      int m = 0;
      if (ifeast_eigenpairs(h, 0, &m, nullptr, nullptr, nullptr, 0) == IFEAST_OK && m > 0) {
        r.evals.resize(m);
        r.resid.resize(m);
        r.evecs.resize((size_t)r.n * m);
        ifeast_eigenpairs(h, m, &m, r.evals.data(), r.evecs.data(), r.resid.data(), 0);
      }
      r.found = m;
    }
    ifeast_destroy(h);
  }
  cudaFreeAsync(ws, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  r.X0.clear();
  r.X0.shrink_to_fit();
  r.status = rc;
}

void worker_loop(ifeast_server *s) {
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [s] {
        if (!s->pending.empty() && s->used + s->pending.front()->ws_bytes <= s->opts.mem_budget_bytes)
          return true;
        return s->stopping && s->pending.empty();
      });
      if (s->pending.empty()) return;  // stopping
      r = s->pending.front();
      s->pending.pop_front();
      s->used += r->ws_bytes;
      r->t_start = Clock::now();
    }
    s->cv.notify_all();  // the next request in line may fit as well
    run_request(s->opts, *r);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->used -= r->ws_bytes;
      r->t_done = Clock::now();
      r->done = true;
    }
    s->cv.notify_all();
  }
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

extern "C" {

int ifeast_server_create(const ifeast_server_opts *o, ifeast_server_t *out) {
  if (!o || !out || o->max_active < 1 || o->mem_budget_bytes == 0 || o->device < 0)
    return IFEAST_ERR_INVALID_ARG;
  *out = nullptr;
  ifeast_server *s = new (std::nothrow) ifeast_server();
  if (!s) return IFEAST_ERR_OOM;
  s->opts = *o;
  for (int i = 0; i < o->max_active; ++i) s->workers.emplace_back(worker_loop, s);
  *out = s;
  return IFEAST_OK;
}

int ifeast_server_submit(ifeast_server_t s, const ifeast_csr *A, const ifeast_contour *c, int m0,
                         const ifeast_opts *o, const double *X0, int64_t *id) {
  if (!s || !A || !c || !o || !X0 || !id || !A->rowptr || A->n < 1 || A->nnz < 0)
    return IFEAST_ERR_INVALID_ARG;
  size_t bytes = 0;
  int rc = ifeast_workspace_bytes(A->n, A->nnz, m0, c, o, &bytes);
  if (rc) return rc;
  if (bytes > s->opts.mem_budget_bytes) return IFEAST_ERR_OOM;
  auto r = std::make_shared<Request>();
  r->n = A->n;
  r->nnz = A->nnz;
  r->rowptr.assign(A->rowptr, A->rowptr + A->n + 1);
  if (A->nnz > 0) {
    if (!A->colidx || !A->val) return IFEAST_ERR_INVALID_ARG;
    r->colidx.assign(A->colidx, A->colidx + A->nnz);
    r->val.assign(A->val, A->val + A->nnz);
  }
  r->contour = *c;
  if (c->rule == IFEAST_USER) {  // the caller's node array may be freed on return
    r->user_zw.assign(c->user_zw, c->user_zw + 4 * (size_t)c->nc);
    r->contour.user_zw = r->user_zw.data();
  }
  r->opts = *o;
  r->m0 = m0;
  r->X0.assign(X0, X0 + (size_t)A->n * m0);
  r->ws_bytes = bytes;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->requests[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
  }
  s->cv.notify_all();
  return IFEAST_OK;
}

int ifeast_server_wait(ifeast_server_t s, int64_t id, int cap, int *m_found, double *evals,
                       double *evecs, double *resid, ifeast_request_info *info) {
  if (!s || cap < 0) return IFEAST_ERR_INVALID_ARG;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->requests.find(id);
    if (it == s->requests.end()) return IFEAST_ERR_INVALID_ARG;
    r = it->second;
    s->cv.wait(lk, [&r] { return r->done; });
    s->requests.erase(id);
  }
  const int m = r->found;
  if (m_found) *m_found = m;
  const int cnt = m < cap ? m : cap;
  for (int q = 0; q < cnt; ++q) {
    if (evals) evals[q] = r->evals[q];
    if (resid) resid[q] = r->resid[q];
  }
  if (evecs)
    for (int64_t i = 0; i < r->n; ++i)
      for (int q = 0; q < cnt; ++q) evecs[(size_t)i * cap + q] = r->evecs[(size_t)i * m + q];
  if (info) {
    info->status = r->status;
    info->found = m;
    info->outer_iters = r->stats.outer_iters;
    info->RF = r->stats.RF;
    info->submit_to_start_ms = ms_between(r->t_submit, r->t_start);
    info->submit_to_done_ms = ms_between(r->t_submit, r->t_done);
    info->workspace_bytes = r->ws_bytes;
  }
  return r->status;
}

void ifeast_server_destroy(ifeast_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto &t : s->workers) t.join();
  delete s;
}

}  // extern "C"
