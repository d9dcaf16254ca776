// Request server: continuous batching of decompositions of different N, L
// and k as they arrive (the serving pattern around Algorithms 1-3).
//
// Requests wait in arrival order.  A request whose series fits the batched
// engine goes to the batch queue; the rest go to the single-series queue.
// Worker threads, each with its own non-blocking CUDA stream, take work as
// soon as they are idle and the device-memory budget admits it:
//   * batch workers pack up to max_batch queued requests into one
//     ssa_decompose_batch launch (one persistent kernel over all of them);
//   * single workers run ssa_embed_plan + ssa_decompose for one request,
//     keeping its spectrum and Lanczos state on the device until it is done.
// Requests that arrive while others run are admitted as workers and memory
// free up, and their kernels overlap on the device with the running ones.
// Admission is strictly first-come-first-served within each queue; the
// memory held by a running request is the estimate of budget.h.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ssa.h"
#include "budget.h"
#include "prof.h"

using ssa::host_set_error;

namespace {

struct Req {
  int64_t id = 0;
  std::vector<double> f;
  int64_t N = 0, L = 0;
  int k = 0;
  int outputs = 0;
  int64_t mem = 0;
  bool batched = false;
  bool done = false;
  int status = SSA_OK;
  char err[256] = {0};
  int converged = 0, restarts = 0;
  int64_t matvecs = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::vector<double> sigma, resid, U, V;
};

}  // namespace

struct ssa_server_s {
  ssa_serve_opts_t o{};
  int dev = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;       // work available / memory freed / stop
  std::condition_variable cv_done;  // a request finished
  std::deque<Req*> q_single, q_batch;
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_id = 1;
  int grid_cap = 0;  // ssa_opts_t.grid_cap of the single-series requests
  int64_t mem_in_use = 0, mem_peak = 0;
  int64_t submitted = 0, completed = 0, running = 0, batches = 0, batched_requests = 0;
  bool stop = false;
  std::vector<std::thread> threads;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  bool fits(int64_t bytes) const { return mem_in_use == 0 || mem_in_use + bytes <= o.mem_budget; }
  void admit(int64_t bytes) {
    mem_in_use += bytes;
    mem_peak = std::max(mem_peak, mem_in_use);
  }
};

namespace {

void finish(ssa_server_s* S, Req* r, int64_t mem) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->mem_in_use -= mem;
    --S->running;
    ++S->completed;
    r->t_done = S->now();
    r->done = true;
  }
  S->cv.notify_all();
  S->cv_done.notify_all();
}

void fail(Req* r, int rc) {
  r->status = rc;
  std::snprintf(r->err, sizeof r->err, "%s", ssa_last_error());
}

void run_single(ssa_server_s* S, Req* r, cudaStream_t st) {
  ssa_opts_t o;
  ssa_default_opts(&o);
  o.precision = S->o.precision;
  o.tol = S->o.tol;
  o.stream = st;
  o.grid_cap = S->grid_cap;
  ssa_plan_t plan = nullptr;
  int rc = ssa_embed_plan(r->N, r->L, &o, &plan);
  if (rc) return fail(r, rc);
  ssa_decomp_t d = nullptr;
  rc = ssa_decompose(plan, r->f.data(), r->k, &d);
  if (rc != SSA_OK && rc != SSA_ENOCONV) {
    fail(r, rc);
    ssa_plan_destroy(plan);
    return;
  }
  const int64_t K = r->N - r->L + 1;
  r->sigma.resize(r->k);
  r->resid.resize(r->k);
  if (r->outputs & SSA_SERVE_VECTORS) {
    r->U.resize((size_t)r->L * r->k);
    r->V.resize((size_t)K * r->k);
  }
  int rc2 = ssa_decomp_get(d, r->sigma.data(), r->U.empty() ? nullptr : r->U.data(),
                           r->V.empty() ? nullptr : r->V.data(), r->resid.data());
  int k = 0, kd = 0;
  ssa_decomp_info(d, &k, &r->converged, &r->restarts, &r->matvecs, &kd);
  ssa_decomp_destroy(d);
  ssa_plan_destroy(plan);
  if (rc2) return fail(r, rc2);
  r->status = rc;
  if (rc == SSA_ENOCONV) std::snprintf(r->err, sizeof r->err, "did not converge within max_restarts");
}

void run_batch(ssa_server_s* S, std::vector<Req*>& rs, cudaStream_t st) {
  const int n = (int)rs.size();
  std::vector<int64_t> off(n + 1, 0), Ls(n);
  std::vector<int32_t> ks(n);
  for (int i = 0; i < n; ++i) {
    off[i + 1] = off[i] + rs[i]->N;
    Ls[i] = rs[i]->L;
    ks[i] = rs[i]->k;
  }
  std::vector<double> f((size_t)off[n]);
  for (int i = 0; i < n; ++i) std::memcpy(f.data() + off[i], rs[i]->f.data(), rs[i]->N * sizeof(double));
  ssa_opts_t o;
  ssa_default_opts(&o);
  o.precision = S->o.precision;
  o.tol = S->o.tol;
  o.stream = st;
  ssa_batch_t b = nullptr;
  int rc = ssa_decompose_batch(n, f.data(), off.data(), Ls.data(), ks.data(), &o, &b);
  if (rc != SSA_OK && rc != SSA_ENOCONV && rc != SSA_ENUMERIC) {
    for (Req* r : rs) fail(r, rc);
    return;
  }
  for (int i = 0; i < n; ++i) {
    Req* r = rs[i];
    const int64_t K = r->N - r->L + 1;
    r->sigma.resize(r->k);
    r->resid.resize(r->k);
    if (r->outputs & SSA_SERVE_VECTORS) {
      r->U.resize((size_t)r->L * r->k);
      r->V.resize((size_t)K * r->k);
    }
    int k = 0, conv = 0, rs_ = 0;
    int64_t mv = 0;
    ssa_batch_info(b, i, &k, &conv, &rs_, &mv);
    int rc2 = ssa_batch_get(b, i, r->sigma.data(), r->U.empty() ? nullptr : r->U.data(),
                            r->V.empty() ? nullptr : r->V.data(), r->resid.data());
    r->converged = conv;
    r->restarts = rs_;
    r->matvecs = mv;
    if (rc2) fail(r, rc2);
    else if (!conv) {
      r->status = SSA_ENOCONV;
      std::snprintf(r->err, sizeof r->err, "did not converge within max_restarts");
    }
  }
  ssa_batch_destroy(b);
}

void single_worker(ssa_server_s* S) {
  cudaSetDevice(S->dev);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || (!S->q_single.empty() && S->fits(S->q_single.front()->mem)); });
      if (S->stop) break;
      r = S->q_single.front();
      S->q_single.pop_front();
      S->admit(r->mem);
      ++S->running;
      r->t_start = S->now();
    }
    run_single(S, r, st);
    finish(S, r, r->mem);
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

void batch_worker(ssa_server_s* S) {
  cudaSetDevice(S->dev);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<ssa::BatchItem> items;
  for (;;) {
    std::vector<Req*> take;
    int64_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) break;
        // first come, first served: pack from the front while the budget admits
        items.clear();
        take.clear();
        bytes = 0;
        for (Req* r : S->q_batch) {
          if ((int)take.size() >= S->o.max_batch) break;
          items.push_back({r->N, r->L, r->k});
          const int64_t nb = ssa::batch_path_bytes(items, 0);
          if (!take.empty() && S->mem_in_use + nb > S->o.mem_budget) break;
          if (take.empty() && !S->fits(nb)) break;
          take.push_back(r);
          bytes = nb;
        }
        if (!take.empty()) break;
        S->cv.wait(lk);
      }
      if (S->stop) break;
      S->q_batch.erase(S->q_batch.begin(), S->q_batch.begin() + take.size());
      S->admit(bytes);
      S->running += (int64_t)take.size();
      ++S->batches;
      S->batched_requests += (int64_t)take.size();
      const double t = S->now();
      for (Req* r : take) r->t_start = t;
    }
    run_batch(S, take, st);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->mem_in_use -= bytes;
      S->running -= (int64_t)take.size();
      S->completed += (int64_t)take.size();
      const double t = S->now();
      for (Req* r : take) {
        r->t_done = t;
        r->done = true;
      }
    }
    S->cv.notify_all();
    S->cv_done.notify_all();
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" void ssa_serve_default_opts(ssa_serve_opts_t* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = SSA_PREC_F32C;
  o->tol = 0.0;
  o->mem_budget = (int64_t)40 << 30;
  // measured on the serving workload (N log-uniform [1e3, 1e6], k U{2..64}): more single-series
  // workers or batch workers, or larger batches, left the batched engine less of the device and
  // the capacity for the whole mix lower (16 / 2 / 512: ~50 requests/s; 4-8 / 1 / 64-256: 70-74)
  o->workers = 8;
  o->batch_workers = 1;
  o->max_batch = 128;
  o->batch_max_n = 0;
}

extern "C" int ssa_serve_create(const ssa_serve_opts_t* opts, ssa_server_t* out) {
  if (!out) {
    host_set_error("out is NULL");
    return SSA_EINVAL;
  }
  *out = nullptr;
  ssa_serve_opts_t o;
  ssa_serve_default_opts(&o);
  if (opts) {
    o = *opts;
    ssa_serve_opts_t d;
    ssa_serve_default_opts(&d);
    if (o.mem_budget <= 0) o.mem_budget = d.mem_budget;
    if (o.workers <= 0) o.workers = d.workers;
    if (o.batch_workers < 0) o.batch_workers = 0;
    if (o.max_batch <= 0) o.max_batch = d.max_batch;
  }
  if (o.precision != SSA_PREC_F64 && o.precision != SSA_PREC_F32C) {
    host_set_error("unknown precision");
    return SSA_EINVAL;
  }
  if (o.workers > 64 || o.batch_workers > 16) {
    host_set_error("at most 64 single-series workers and 16 batch workers");
    return SSA_EINVAL;
  }
  if (o.grid_cap < 0) {
    host_set_error("grid_cap must be >= 0");
    return SSA_EINVAL;
  }
  ssa_server_s* S = new (std::nothrow) ssa_server_s();
  if (!S) return SSA_ENOMEM;
  S->o = o;
  cudaGetDevice(&S->dev);
  S->grid_cap = o.grid_cap;
  S->t0 = std::chrono::steady_clock::now();
  // keep freed stream-ordered memory in the pool so that per-request
  // allocations are served without returning to the CUDA driver
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, S->dev) == cudaSuccess) {
    uint64_t thr = (uint64_t)o.mem_budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  ssa::lib_pool_keep((uint64_t)o.mem_budget);  // the single-series path allocates from this one
  for (int i = 0; i < o.workers; ++i) S->threads.emplace_back(single_worker, S);
  for (int i = 0; i < o.batch_workers; ++i) S->threads.emplace_back(batch_worker, S);
  *out = S;
  return SSA_OK;
}

extern "C" int ssa_serve_submit(ssa_server_t S, const double* f, int64_t N, int64_t L, int k, int outputs,
                                int64_t* id) {
  if (!S || !f || !id) {
    host_set_error("NULL argument");
    return SSA_EINVAL;
  }
  const int64_t K = N - L + 1;
  if (N <= 2 || L <= 1 || L >= N || k < 1 || k > std::min(L, K)) {
    host_set_error("need N > 2, 1 < L < N and 1 <= k <= min(L, K)");
    return SSA_EINVAL;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) return SSA_ENOMEM;
  r->N = N;
  r->L = L;
  r->k = k;
  r->outputs = outputs;
  const int64_t nlim = S->o.batch_max_n;
  r->batched = S->o.batch_workers > 0 && nlim >= 0 && (nlim == 0 || N <= nlim) &&
               ssa::batch_eligible(N, L, k, S->o.precision);
  r->mem = r->batched ? ssa::batch_path_bytes({{N, L, k}}, 0) : ssa::plan_path_bytes(N, L, k, S->o.precision);
  if (r->mem > S->o.mem_budget) {
    delete r;
    host_set_error("the request needs more device memory than the server's budget");
    return SSA_ENOMEM;
  }
  r->f.assign(f, f + N);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = S->now();
    S->reqs[r->id] = r;
    (r->batched ? S->q_batch : S->q_single).push_back(r);
    ++S->submitted;
  }
  S->cv.notify_all();
  *id = r->id;
  return SSA_OK;
}

extern "C" int ssa_serve_poll(ssa_server_t S, int64_t id, double timeout_s, int* done) {
  if (!S || !done) {
    host_set_error("NULL argument");
    return SSA_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) {
    host_set_error("unknown request id");
    return SSA_EINVAL;
  }
  Req* r = it->second;
  if (!r->done && timeout_s > 0)
    S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  *done = r->done ? 1 : 0;
  return SSA_OK;
}

extern "C" int ssa_serve_take(ssa_server_t S, int64_t id, double* sigma, double* U, double* V, double* resid,
                              ssa_serve_info_t* info) {
  if (!S) {
    host_set_error("server is NULL");
    return SSA_EINVAL;
  }
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) {
      host_set_error("unknown request id");
      return SSA_EINVAL;
    }
    if (!it->second->done) {
      host_set_error("request not finished (ssa_serve_poll)");
      return SSA_EINVAL;
    }
    if ((U || V) && !(it->second->outputs & SSA_SERVE_VECTORS)) {
      host_set_error("vectors were not requested at submission");
      return SSA_EINVAL;
    }
    r = it->second;
    S->reqs.erase(it);
  }
  if (info) {
    info->status = r->status;
    info->converged = r->converged;
    info->restarts = r->restarts;
    info->matvecs = r->matvecs;
    info->batched = r->batched ? 1 : 0;
    info->t_submit = r->t_submit;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
  }
  const int rc = r->status;
  if (rc == SSA_OK || rc == SSA_ENOCONV) {
    if (sigma) std::memcpy(sigma, r->sigma.data(), r->k * sizeof(double));
    if (resid) std::memcpy(resid, r->resid.data(), r->k * sizeof(double));
    if (U) std::memcpy(U, r->U.data(), r->U.size() * sizeof(double));
    if (V) std::memcpy(V, r->V.data(), r->V.size() * sizeof(double));
  }
  if (rc != SSA_OK) host_set_error(r->err);
  delete r;
  return rc;
}

extern "C" int ssa_serve_stats(ssa_server_t S, ssa_serve_stats_t* st) {
  if (!S || !st) {
    host_set_error("NULL argument");
    return SSA_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->queued = (int64_t)(S->q_single.size() + S->q_batch.size());
  st->running = S->running;
  st->mem_in_use = S->mem_in_use;
  st->mem_peak = S->mem_peak;
  st->batches = S->batches;
  st->batched_requests = S->batched_requests;
  return SSA_OK;
}

extern "C" void ssa_serve_destroy(ssa_server_t S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (std::thread& t : S->threads) t.join();
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}
