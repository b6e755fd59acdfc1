// Projection server: a request loop with continuous batching (sip_server_*).
//
// Requests (a grid, a set list and a model in host memory) arrive at any
// time from any thread.  One worker thread owns the device side:
//  - admission: queued requests are grouped into a cohort when the HBM
//    budget has room for the cohort's whole state (its arena size is
//    computed before anything is allocated, so the budget is never
//    exceeded); a cohort forms when `max_batch` requests wait, when the
//    oldest has waited `max_wait_ms`, or when the device is idle;
//  - execution: a cohort is a batched plan (every launch covers all of its
//    requests) on its own CUDA stream, so cohorts admitted at different times
//    overlap on the device; it advances `check_every` iterations per chunk,
//    replayed from a CUDA graph; every request keeps x, y_i, v_i, rho_i and
//    its CG state resident in the cohort's arena until it finishes;
//  - completion: after each chunk the done flags come back asynchronously;
//    a request is delivered (result copied to its host buffer, latency
//    recorded) as soon as its own stopping rule holds, and the cohort's
//    memory returns to the budget when its last request is delivered.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "sip.h"
#include "sip_dev.cuh"
#include "sip_host.h"
#include "sip_kernels.h"

using namespace sip;

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id = 0;
  sip_grid grid;
  std::vector<sip_set> sets;
  std::vector<unsigned char> m;  // model, host copy
  void *x_user = nullptr;        // caller's result buffer (host)
  int64_t n = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 running, 2 delivered, 3 failed
  sip_status status = SIP_OK;
  sip_info info;
};

struct Cohort {
  Plan P;
  cudaStream_t st = nullptr, cap = nullptr;
  cudaEvent_t ev_flags = nullptr, ev_out = nullptr;
  std::vector<Request *> reqs;
  int32_t *flags = nullptr;        // pinned: done flag per instance
  unsigned char *xout = nullptr;   // pinned: results of the instances being delivered
  InstScal *scal_out = nullptr;    // pinned: their scalars (info)
  std::vector<int> delivering;     // instances whose results are in flight to xout
  std::vector<char> delivered;
  int iters_run = 0;
  int phase = 0;  // 0 idle, 1 chunk + flags in flight, 2 results in flight
  int64_t bytes = 0;
  int remaining = 0;
};

}  // namespace

struct sip_server {
  sip_server_config cfg;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request *> queue;
  std::unordered_map<int64_t, Request *> reqs;
  std::vector<Cohort *> active;
  int64_t used = 0, peak_used = 0;
  int64_t next_id = 1;
  int64_t completed = 0, failed = 0;
  std::vector<double> latency;
  double t_first = -1, t_last = 0;
  bool stop = false;
  std::thread worker;
  std::string err;
};

namespace {

size_t esz(int dtype) { return dtype == SIP_F64 ? 8 : 4; }

void release(Cohort *c) {
  c->P.release();
  if (c->st) cudaStreamDestroy(c->st);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->ev_flags) cudaEventDestroy(c->ev_flags);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->flags) cudaFreeHost(c->flags);
  if (c->xout) cudaFreeHost(c->xout);
  if (c->scal_out) cudaFreeHost(c->scal_out);
  delete c;
}

void finish_request(sip_server *S, Request *r, sip_status st) {
  r->status = st;
  r->t_done = now_ms();
  r->state = st == SIP_OK ? 2 : 3;
  if (st == SIP_OK) {
    ++S->completed;
    S->latency.push_back(r->t_done - r->t_submit);
    S->t_last = r->t_done;
  } else {
    ++S->failed;
  }
}

// Build and start a cohort from the queue head (called with the lock held).
// Returns false when nothing could be admitted.
bool admit(sip_server *S) {
  if (S->queue.empty() || (int)S->active.size() >= S->cfg.max_cohorts) return false;
  const double wait = now_ms() - S->queue.front()->t_submit;
  const bool idle = S->active.empty();
  if (!idle && (int)S->queue.size() < S->cfg.max_batch && wait < S->cfg.max_wait_ms) return false;
  // size-aware grouping: a cohort takes requests within a factor 4 of the
  // oldest request's grid size (so small requests do not iterate at the pace
  // of large ones), at most max_points grid points and max_batch requests
  std::vector<Request *> take;
  std::vector<InstLayout> L;
  int64_t bytes = 0, points = 0;
  const int64_t n0 = S->queue.front()->n;
  for (Request *r : S->queue) {
    if ((int)take.size() >= S->cfg.max_batch) break;
    if (r->n * 4 < n0 || r->n > n0 * 4) continue;
    if (!take.empty() && points + r->n > S->cfg.max_points) break;
    std::vector<InstLayout> L2 = L;
    L2.push_back(make_layout(grid_desc(r->grid), r->sets.data(), (int)r->sets.size(), S->cfg.opts));
    const int64_t b = plan_bytes(L2, S->cfg.opts.dtype, true, true);
    if (b < 0 || S->used + b > S->cfg.budget_bytes) break;
    L = std::move(L2);
    bytes = b;
    points += r->n;
    take.push_back(r);
  }
  if (take.empty()) {
    // the head request alone exceeds what is free: if nothing runs it can
    // never fit, so reject it instead of waiting forever
    if (idle) {
      Request *r = S->queue.front();
      S->queue.pop_front();
      finish_request(S, r, SIP_ERR_BUDGET);
      S->cv.notify_all();
      return true;
    }
    return false;
  }
  Cohort *c = new Cohort();
  c->reqs = take;
  c->delivered.assign(take.size(), 0);
  c->remaining = (int)take.size();
  auto bail = [&](sip_status st) {
    for (Request *r : take) finish_request(S, r, st);
    release(c);
  };
  for (Request *r : take) S->queue.erase(std::find(S->queue.begin(), S->queue.end(), r));
  const int dtype = S->cfg.opts.dtype;
  if (plan_build(c->P, L, dtype, true, true) != SIP_OK) {
    bail(SIP_ERR_OOM);
    S->cv.notify_all();
    return true;
  }
  c->bytes = c->P.arena_bytes;
  const size_t W = esz(dtype);
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_flags, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&c->flags, take.size() * sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&c->xout, (size_t)c->P.pack_off.back() * W) != cudaSuccess ||
      cudaMallocHost(&c->scal_out, take.size() * sizeof(InstScal)) != cudaSuccess) {
    cudaGetLastError();
    bail(SIP_ERR_CUDA);
    S->cv.notify_all();
    return true;
  }
  // models in, state reset, first chunk
  const double t0 = now_ms();
  bool ok = true;
  for (size_t i = 0; i < take.size() && ok; ++i) {
    take[i]->state = 1;
    take[i]->t_start = t0;
    ok = cudaMemcpyAsync((char *)c->P.m_pack + c->P.pack_off[i] * W, take[i]->m.data(), take[i]->m.size(),
                         cudaMemcpyHostToDevice, c->st) == cudaSuccess;
  }
  if (!ok || plan_prepare(c->P, c->st, false) != SIP_OK) {
    cudaStreamSynchronize(c->st);
    bail(SIP_ERR_CUDA);
    S->cv.notify_all();
    return true;
  }
  S->used += c->bytes;
  S->peak_used = std::max(S->peak_used, S->used);
  S->active.push_back(c);
  return true;
}

// Advance one cohort by one step of its state machine.  Returns true when
// it made progress.
bool advance(sip_server *S, Cohort *c) {
  const int dtype = S->cfg.opts.dtype;
  const size_t W = esz(dtype);
  const int n = (int)c->reqs.size();
  if (c->phase == 0) {
    // next chunk, then the done flags (strided out of the instance scalars)
    const int chunk = std::max(1, S->cfg.opts.check_every);
    sip_status st = run_iterations(c->P, c->st, c->cap, chunk, false, nullptr, nullptr);
    c->iters_run += chunk;
    if (st == SIP_OK &&
        cudaMemcpy2DAsync(c->flags, sizeof(int32_t), &c->P.d_scal[0].done, sizeof(InstScal), sizeof(int32_t), n,
                          cudaMemcpyDeviceToHost, c->st) == cudaSuccess &&
        cudaEventRecord(c->ev_flags, c->st) == cudaSuccess) {
      c->phase = 1;
    } else {
      for (int i = 0; i < n; ++i)
        if (!c->delivered[i]) finish_request(S, c->reqs[i], SIP_ERR_CUDA);
      c->remaining = 0;
    }
    return true;
  }
  if (c->phase == 1) {
    if (cudaEventQuery(c->ev_flags) != cudaSuccess) return false;
    c->delivering.clear();
    for (int i = 0; i < n; ++i)
      if (!c->delivered[i] && c->flags[i])
        c->delivering.push_back(i);
    if (c->delivering.empty()) {
      c->phase = 0;
      return true;
    }
    for (int i : c->delivering) {
      cudaMemcpyAsync(c->xout + c->P.pack_off[i] * W, (const char *)c->P.x_pack + c->P.pack_off[i] * W,
                      (size_t)(c->P.pack_off[i + 1] - c->P.pack_off[i]) * W, cudaMemcpyDeviceToHost, c->st);
      cudaMemcpyAsync(&c->scal_out[i], &c->P.d_scal[i], sizeof(InstScal), cudaMemcpyDeviceToHost, c->st);
    }
    cudaEventRecord(c->ev_out, c->st);
    c->phase = 2;
    return true;
  }
  if (cudaEventQuery(c->ev_out) != cudaSuccess) return false;
  for (int i : c->delivering) {
    Request *r = c->reqs[i];
    memcpy(r->x_user, c->xout + c->P.pack_off[i] * W, (size_t)r->n * W);
    const InstScal &sc = c->scal_out[i];
    sip_info &f = r->info;
    memset(&f, 0, sizeof f);
    f.iters = sc.iters;
    f.cg_steps_total = sc.cg_total;
    f.stop_reason = sc.stop_reason;
    f.window_hits = sc.win_hits;
    f.nblocks = c->P.h_insts[i].nb;
    f.r_evol = sc.r_evol;
    for (int b = 0; b < c->P.h_insts[i].p; ++b) {
      f.r_feas[b] = sc.r_feas[b];
      f.sigma[b] = sc.sigma[b];
      f.k[b] = sc.kcard[b];
    }
    for (int b = 0; b < f.nblocks; ++b) {
      f.rho[b] = sc.rho[b];
      f.gamma[b] = sc.gamma[b];
    }
    finish_request(S, r, sc.stop_reason < 0 ? SIP_ERR_NONFINITE : SIP_OK);
    f.ms = (float)(r->t_done - r->t_start);
    c->delivered[i] = 1;
    --c->remaining;
  }
  c->phase = 0;
  S->cv.notify_all();
  return true;
}

void worker_loop(sip_server *S) {
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool progress = false;
    while (admit(S)) progress = true;
    for (size_t j = 0; j < S->active.size();) {
      Cohort *c = S->active[j];
      progress |= advance(S, c);  // asynchronous CUDA calls only; lock held for the bookkeeping
      if (c->remaining == 0 && c->phase == 0) {
        S->used -= c->bytes;
        S->active.erase(S->active.begin() + j);
        lk.unlock();
        cudaStreamSynchronize(c->st);
        release(c);
        lk.lock();
        progress = true;
        S->cv.notify_all();
      } else {
        ++j;
      }
    }
    if (S->stop && S->active.empty() && S->queue.empty()) break;
    if (!progress) S->cv.wait_for(lk, std::chrono::microseconds(100));
  }
}

}  // namespace

extern "C" {

void sip_server_config_default(sip_server_config *c) {
  if (!c) return;
  memset(c, 0, sizeof *c);
  sip_options_default(&c->opts);
  c->opts.stop = 2;
  c->opts.max_iter = 500;
  c->budget_bytes = (int64_t)120 << 30;
  c->max_batch = 64;
  c->max_cohorts = 8;
  c->max_wait_ms = 2.0;
  c->max_points = (int64_t)1 << 24;
}

sip_status sip_server_create(const sip_server_config *cfg, sip_server **out) {
  if (!cfg || !out) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->budget_bytes <= 0 || cfg->max_batch < 1 || cfg->max_cohorts < 1 || !(cfg->max_wait_ms >= 0.0) ||
      cfg->max_points < 1)
    return fail(SIP_ERR_INVALID_ARG, "bad server configuration");
  if (cfg->opts.levels != 1 || cfg->opts.rho_schedule || cfg->opts.gamma_schedule || cfg->opts.trace)
    return fail(SIP_ERR_INVALID_ARG, "served projections are single-level without schedules or traces");
  sip_set s;
  memset(&s, 0, sizeof s);
  s.type = SIP_SET_BOUNDS;
  s.hi = 1.0;
  sip_grid g;
  memset(&g, 0, sizeof g);
  g.ndim = 2;
  g.n[0] = g.n[1] = 2;
  g.h[0] = g.h[1] = 1.0;
  if (sip_status st = validate(&g, &s, 1, &cfg->opts)) return st;
  if (cfg->opts.store_bf16) return fail(SIP_ERR_INVALID_ARG, "the server does not run the BF16 storage trial");
  if (cfg->opts.tune) return fail(SIP_ERR_INVALID_ARG, "the server's cohorts are not tuned");
  sip_server *S = new (std::nothrow) sip_server();
  if (!S) return fail(SIP_ERR_OOM, "host allocation failed");
  S->cfg = *cfg;
  // cohorts run concurrently on their own streams: no persistent
  // (cooperative) kernels, whose grid barriers could wait on CTAs that
  // another cohort's grid keeps from becoming resident
  S->cfg.opts.exec = SIP_EXEC_GRAPH;
  int dev = 0;
  cudaGetDevice(&dev);
  S->worker = std::thread([S, dev]() {
    cudaSetDevice(dev);
    worker_loop(S);
  });
  *out = S;
  return SIP_OK;
}

sip_status sip_server_submit(sip_server *S, const sip_grid *grid, const sip_set *sets, int nsets, const void *m_host,
                             void *x_host, int64_t *req_id) {
  if (!S || !m_host || !x_host || !req_id) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  if (sip_status st = validate(grid, sets, nsets, &S->cfg.opts)) return st;
  for (int i = 0; i < nsets; ++i)
    if (sets[i].lo_vec || sets[i].hi_vec || sets[i].center_vec || sets[i].op == SIP_OP_BLUR)
      return fail(SIP_ERR_INVALID_ARG, "set %d: per-entry vectors and blur tables are not served", i);
  Request *r = new (std::nothrow) Request();
  if (!r) return fail(SIP_ERR_OOM, "host allocation failed");
  r->grid = *grid;
  r->sets.assign(sets, sets + nsets);
  r->n = grid_desc(*grid).N();
  const size_t bytes = (size_t)r->n * esz(S->cfg.opts.dtype);
  r->m.assign((const unsigned char *)m_host, (const unsigned char *)m_host + bytes);
  r->x_user = x_host;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) {
    delete r;
    return fail(SIP_ERR_INVALID_ARG, "server is shutting down");
  }
  r->id = S->next_id++;
  if (S->t_first < 0) S->t_first = r->t_submit;
  S->reqs[r->id] = r;
  S->queue.push_back(r);
  *req_id = r->id;
  S->cv.notify_all();
  return SIP_OK;
}

sip_status sip_server_wait(sip_server *S, int64_t id, double timeout_ms, sip_info *info, double *latency_ms) {
  if (!S) return fail(SIP_ERR_INVALID_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(SIP_ERR_INVALID_ARG, "unknown request %lld", (long long)id);
  Request *r = it->second;
  const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
  while (r->state < 2) {
    if (timeout_ms >= 0 && S->cv.wait_until(lk, until) == std::cv_status::timeout && r->state < 2)
      return fail(SIP_ERR_TIMEOUT, "request %lld still running", (long long)id);
    if (timeout_ms < 0) S->cv.wait(lk);
  }
  if (info) *info = r->info;
  if (latency_ms) *latency_ms = r->t_done - r->t_submit;
  const sip_status st = r->status;
  S->reqs.erase(it);
  delete r;
  if (st != SIP_OK) return fail(st, "request %lld failed", (long long)id);
  return SIP_OK;
}

sip_status sip_server_query_stats(sip_server *S, sip_server_stats *out) {
  if (!S || !out) return fail(SIP_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof *out);
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (int64_t)S->queue.size();
  out->running_cohorts = (int)S->active.size();
  out->hbm_in_use = S->used;
  out->hbm_peak = S->peak_used;
  std::vector<double> l = S->latency;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) { return l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    const double span = (S->t_last - S->t_first) / 1000.0;
    out->projections_per_s = span > 0 ? (double)S->completed / span : 0.0;
  }
  return SIP_OK;
}

sip_status sip_server_destroy(sip_server *S) {
  if (!S) return SIP_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  for (auto &kv : S->reqs) delete kv.second;
  delete S;
  return SIP_OK;
}

}  // extern "C"
