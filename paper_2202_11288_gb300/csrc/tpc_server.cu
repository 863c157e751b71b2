// Request server: continuous batching of independent solves on one GPU.
//
// A worker thread owns every handle. Requests (problem description + host buffers) are queued
// by tpc_server_submit; the worker admits them while a slot (max_inflight) and device memory
// (the HBM budget) are free, keeps level hierarchies resident keyed by the problem (dimension,
// variant, kernel, transfer, outer iteration, horizon, mesh size, precision) and reuses an idle one when the key
// repeats (a request whose
// key's hierarchies are all busy waits for one, unless the key may have another; later
// requests of other keys go ahead), evicting idle hierarchies least-recently-used first when
// the budget requires. Every admitted solve runs on
// its handle's own stream as an ordinary tpc_solve (same arithmetic, same result as solving it
// alone); the worker polls them without blocking, so requests that arrive while others are on
// the GPU start as soon as a slot and memory free up and their work overlaps on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tpc_internal.h"

namespace tpc {
void set_host_error(const std::string& s);
}

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long ticket = 0;
  tpc_request r{};
  Clock::time_point t_submit;
};

struct Entry {
  int dim = 1, variant = 0, precision = 0, kernel = 0, transfer = 0, outer = 0;
  double delta = 0.0, h = 0.0, kernel_a = 0.0;
  tpc_handle* H = nullptr;        // 1-D requests
  tpc2d_handle* H2 = nullptr;     // 2-D requests
  size_t bytes = 0;
  bool busy = false;
  unsigned long long last_use = 0;
};

struct Active {
  Entry* entry = nullptr;
  Request req;
  tpc::AsyncSolve* a = nullptr;
  tpc::AsyncSolve2* a2 = nullptr;
  Clock::time_point t_start;
};

}  // namespace

struct tpc_server {
  tpc_server_config cfg{};
  tpc_params prm{};
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Request> pending;           // guarded by mu
  std::vector<tpc_server_result> done;   // guarded by mu
  long long next_ticket = 1;             // guarded by mu
  std::atomic<long long> outstanding{0};  // submitted and not yet finished
  // worker-owned (entries are heap objects so that active solves keep valid pointers)
  std::vector<Entry*> cache;
  std::vector<Active> active;
  size_t used_bytes = 0;
  unsigned long long tick = 0;
  std::string worker_err;
  tpc_server_stats stats{};              // guarded by mu
  Clock::time_point t_stats, t_last;     // start of the statistics, last worker update
};

namespace {

int req_dim(const tpc_request& r) { return r.dim == 2 ? 2 : 1; }

// The transfer a request asks for (the server's parameters' unless the request names one).
int req_transfer(const tpc_server* S, const tpc_request& r) {
  if (r.transfer == TPC_REQUEST_TRANSFER_PAPER) return TPC_TRANSFER_PAPER;
  if (r.transfer == TPC_REQUEST_TRANSFER_GEOMETRIC) return TPC_TRANSFER_GEOMETRIC;
  return S->prm.transfer;
}

// The outer iteration a request asks for (the server's parameters' unless it names one).
int req_outer(const tpc_server* S, const tpc_request& r) {
  if (r.outer == TPC_REQUEST_OUTER_VCYCLE) return TPC_OUTER_VCYCLE;
  if (r.outer == TPC_REQUEST_OUTER_FGMRES) return TPC_OUTER_FGMRES;
  return S->prm.outer;
}

bool same_key(const tpc_server* S, const Entry& e, const tpc_request& r, int precision) {
  return e.dim == req_dim(r) && e.variant == r.variant && e.precision == precision &&
         e.delta == r.delta && e.h == r.h && e.kernel == r.kernel && e.kernel_a == r.kernel_a &&
         e.transfer == req_transfer(S, r) && e.outer == req_outer(S, r);
}

void destroy_entry(Entry* e) {
  if (e->H) tpc_destroy(e->H);
  if (e->H2) tpc2d_destroy(e->H2);
  delete e;
}

size_t entry_bytes(const Entry* e) {
  return e->H2 ? tpc::handle2d_device_bytes(e->H2) : tpc::handle_device_bytes(e->H);
}

// Device bytes a hierarchy of this key needs: the size of a resident one with the same
// dimension, mesh size, variant and precision if there is one, else an estimate from the level
// sizes (1-D: spectra, twiddles, vectors over all levels, about 220 bytes per unknown in FP64,
// 320 with the FP32 copy; 2-D: the level vectors, about 160 and 240 bytes per unknown), plus
// the fixed tables.
size_t estimate_bytes(const tpc_server* S, const tpc_request& r) {
  const int dim = req_dim(r);
  for (const Entry* e : S->cache)
    if (e->dim == dim && e->h == r.h && e->precision == S->cfg.precision &&
        e->variant == r.variant)
      return e->bytes;
  const double n1 = 2.0 / r.h;
  const bool mixed = S->cfg.precision == TPC_MIXED;
  if (dim == 2)
    return (size_t)(n1 * n1 * (mixed ? 240.0 : 160.0) + n1 * 320.0) + (size_t(1) << 20);
  return (size_t)(n1 * (mixed ? 320.0 : 220.0)) + (size_t(256) << 10);
}

void finish_request(tpc_server* S, Active& act, int status, int iters, double relres) {
  tpc_server_result res{};
  res.ticket = act.req.ticket;
  res.status = status;
  res.iters = iters;
  res.relres = relres;
  res.latency_s = std::chrono::duration<double>(Clock::now() - act.req.t_submit).count();
  res.queue_s = std::chrono::duration<double>(act.t_start - act.req.t_submit).count();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(res);
  }
  S->outstanding.fetch_sub(1);
  S->cv.notify_all();
}

// Try to start the request; returns false if it must wait (for a slot, for memory, or for
// a busy hierarchy of its key when the key already has max_handles_per_key of them).
bool admit(tpc_server* S, Request& req) {
  if ((int)S->active.size() >= S->cfg.max_inflight) return false;
  const int prec = S->cfg.precision;
  Entry* ent = nullptr;
  int same = 0;
  for (Entry* e : S->cache) {
    if (!same_key(S, *e, req.r, prec)) continue;
    ++same;
    if (!e->busy) {
      ent = e;
      break;
    }
  }
  if (!ent && same >= S->cfg.max_handles_per_key) return false;
  Active act;
  act.req = req;
  act.t_start = Clock::now();
  if (!ent) {
    const size_t need = estimate_bytes(S, req.r);
    // evict idle hierarchies, least recently used first, until the new one fits
    while (S->used_bytes + need > S->cfg.hbm_budget_bytes) {
      int lru = -1;
      for (size_t i = 0; i < S->cache.size(); ++i)
        if (!S->cache[i]->busy &&
            (lru < 0 || S->cache[i]->last_use < S->cache[lru]->last_use))
          lru = (int)i;
      if (lru < 0) break;
      S->used_bytes -= S->cache[lru]->bytes;
      destroy_entry(S->cache[lru]);
      S->cache.erase(S->cache.begin() + lru);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        ++S->stats.evictions;
      }
    }
    if (S->used_bytes + need > S->cfg.hbm_budget_bytes) {
      if (!S->active.empty()) return false;  // wait for memory to free up
      finish_request(S, act, TPC_ENOMEM, 0, 0.0);  // larger than the whole budget
      return true;
    }
    tpc_params p = S->prm;
    p.variant = req.r.variant;
    p.kernel = req.r.kernel;
    p.kernel_a = req.r.kernel_a;
    p.transfer = req_transfer(S, req.r);
    p.outer = req_outer(S, req.r);
    tpc_handle* H = nullptr;
    tpc2d_handle* H2 = nullptr;
    const int rc = req_dim(req.r) == 2 ? tpc2d_setup(&p, req.r.delta, req.r.h, nullptr, &H2)
                                       : tpc_setup(&p, req.r.delta, req.r.h, 0, nullptr, &H);
    if (rc != TPC_OK) {
      finish_request(S, act, rc, 0, 0.0);
      return true;
    }
    ent = new Entry();
    ent->dim = req_dim(req.r);
    ent->variant = req.r.variant;
    ent->precision = prec;
    ent->delta = req.r.delta;
    ent->h = req.r.h;
    ent->kernel = req.r.kernel;
    ent->kernel_a = req.r.kernel_a;
    ent->transfer = p.transfer;
    ent->outer = p.outer;
    ent->H = H;
    ent->H2 = H2;
    ent->bytes = entry_bytes(ent);
    S->used_bytes += ent->bytes;
    S->cache.push_back(ent);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      ++S->stats.setups;
    }
  }
  act.entry = ent;
  const long long n = ent->H2 ? tpc2d_level_size(ent->H2, tpc2d_finest_level(ent->H2))
                              : tpc_level_size(ent->H, tpc_finest_level(ent->H));
  if (req.r.n != n) {
    finish_request(S, act, TPC_EINVAL, 0, 0.0);
    return true;
  }
  const int rc = ent->H2
                     ? tpc::async2d_begin_host(ent->H2, req.r.b_host, req.r.x_host, req.r.tol, &act.a2)
                     : tpc::async_begin_host(ent->H, req.r.b_host, req.r.x_host, req.r.tol, &act.a);
  if (rc != TPC_OK) {
    finish_request(S, act, rc, 0, 0.0);
    return true;
  }
  // the staging buffers of the first host solve are allocated then: count them
  const size_t now_bytes = entry_bytes(ent);
  S->used_bytes += now_bytes - ent->bytes;
  ent->bytes = now_bytes;
  ent->busy = true;
  S->active.push_back(act);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->stats.admitted;
  }
  return true;
}

void worker_main(tpc_server* S) {
  cudaSetDevice(S->device);
  std::deque<Request> queue;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // occupancy statistics: the time since the last update counted with the solves that
      // were on the GPU during it
      const Clock::time_point now = Clock::now();
      const double dt = std::chrono::duration<double>(now - S->t_last).count();
      S->t_last = now;
      const int na = (int)S->active.size();
      if (na > 0) S->stats.busy_s += dt;
      S->stats.inflight_s += dt * na;
      S->stats.max_inflight_seen = std::max(S->stats.max_inflight_seen, na);
      S->stats.resident_bytes = S->used_bytes;
      if (queue.empty() && S->active.empty() && S->pending.empty() && !S->stop)
        S->cv.wait_for(lk, std::chrono::milliseconds(1));
      if (S->stop && S->pending.empty() && queue.empty() && S->active.empty()) break;
      while (!S->pending.empty()) {
        queue.push_back(S->pending.front());
        S->pending.pop_front();
      }
    }
    // admit in arrival order, passing over requests that must wait for their key, while
    // slots and memory allow
    for (auto it = queue.begin(); it != queue.end() && (int)S->active.size() < S->cfg.max_inflight;) {
      if (admit(S, *it))
        it = queue.erase(it);
      else
        ++it;
    }
    // advance the solves on the GPU
    bool progressed = false;
    for (size_t i = 0; i < S->active.size();) {
      Active& act = S->active[i];
      int fin = 0;
      const int rc = act.a2 ? tpc::async2d_poll(act.a2, &fin) : tpc::async_poll(act.a, &fin);
      if (rc != TPC_OK || fin) {
        int status = rc, iters = 0;
        double rel = 0.0;
        if (rc == TPC_OK) {
          if (act.a2) tpc::async2d_result(act.a2, &status, &iters, &rel);
          else tpc::async_result(act.a, &status, &iters, &rel);
        }
        if (act.a2) tpc::async2d_free(act.a2);
        else tpc::async_free(act.a);
        act.entry->busy = false;
        act.entry->last_use = ++S->tick;
        finish_request(S, act, status, iters, rel);
        S->active.erase(S->active.begin() + i);
        progressed = true;
        continue;
      }
      ++i;
    }
    if (!progressed && !S->active.empty()) std::this_thread::yield();
  }
  for (Entry* e : S->cache) destroy_entry(e);
  S->cache.clear();
}

}  // namespace

extern "C" {

void tpc_server_default_config(tpc_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->hbm_budget_bytes = (size_t)150 << 30;
  c->max_inflight = 32;
  c->precision = TPC_MIXED;
  c->max_handles_per_key = 1;
}

int tpc_server_create(const tpc_server_config* cfg, const tpc_params* p, tpc_server** out) {
  if (!cfg || !out || cfg->max_inflight < 1 || cfg->hbm_budget_bytes == 0 ||
      cfg->max_handles_per_key < 1 ||
      (cfg->precision != TPC_FP64 && cfg->precision != TPC_MIXED)) {
    tpc::set_host_error("bad argument to tpc_server_create");
    return TPC_EINVAL;
  }
  *out = nullptr;
  tpc_server* S = new (std::nothrow) tpc_server();
  if (!S) return TPC_ENOMEM;
  S->cfg = *cfg;
  if (p)
    S->prm = *p;
  else
    tpc_default_params(&S->prm);
  S->prm.precision = cfg->precision;
  S->t_stats = S->t_last = Clock::now();
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    (void)cudaGetLastError();
    delete S;
    tpc::set_host_error("tpc_server_create: no CUDA device");
    return TPC_ECUDA;
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return TPC_OK;
}

int tpc_server_submit(tpc_server* S, const tpc_request* r, long long* ticket) {
  if (!S || !r || !r->b_host || !r->x_host || !(r->tol >= 0.0) || r->n <= 0 || r->dim < 0 ||
      r->dim > 2 || r->transfer < TPC_REQUEST_TRANSFER_DEFAULT ||
      r->transfer > TPC_REQUEST_TRANSFER_GEOMETRIC || r->outer < TPC_REQUEST_OUTER_DEFAULT ||
      r->outer > TPC_REQUEST_OUTER_FGMRES) {
    tpc::set_host_error("bad argument to tpc_server_submit");
    return TPC_EINVAL;
  }
  Request q;
  q.r = *r;
  q.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    q.ticket = S->next_ticket++;
    S->pending.push_back(q);
    S->outstanding.fetch_add(1);
  }
  S->cv.notify_all();
  if (ticket) *ticket = q.ticket;
  return TPC_OK;
}

int tpc_server_poll(tpc_server* S, tpc_server_result* out, int cap, int wait_ms) {
  if (!S || (cap > 0 && !out) || cap < 0) return TPC_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->done.empty() && wait_ms > 0)
    S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !S->done.empty(); });
  const int k = std::min<int>(cap, (int)S->done.size());
  for (int i = 0; i < k; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + k);
  return k;
}

long long tpc_server_outstanding(tpc_server* S) { return S ? S->outstanding.load() : 0; }

int tpc_server_get_stats(tpc_server* S, tpc_server_stats* out, int reset) {
  if (!S || !out) return TPC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  const Clock::time_point now = Clock::now();
  *out = S->stats;
  out->elapsed_s = std::chrono::duration<double>(now - S->t_stats).count();
  if (reset) {
    const size_t resident = S->stats.resident_bytes;
    S->stats = tpc_server_stats{};
    S->stats.resident_bytes = resident;
    S->t_stats = S->t_last = now;
  }
  return TPC_OK;
}

void tpc_server_destroy(tpc_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  delete S;
}

}  // extern "C"
