// Serving form: a request loop with continuous batching.  A worker thread
// owns a BatchEngine whose arena (allocated once) bounds device memory.
// Between Lanczos steps it admits queued requests in arrival order while a
// slot is free and the request's tables and Krylov vectors fit in the
// arena, steps every admitted request together (one captured graph per
// step), completes the ones whose energy has converged, frees their arena
// range, and wakes their waiters.  Requests keep their Krylov state on the
// device from admission to completion.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>

#include "batch.h"

using namespace edk;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  ed_model_desc m{};
  std::vector<int> bi, bj;
  std::vector<double> jxy, jz, t, U, eps;
  size_t bytes = 0;
  int slot = -1;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 cancelled, 4 failed
  ed_status status = ED_OK;
  std::string msg;  // error text of a failed request (set on the worker thread)
  Clock::time_point t_submit, t_admit, t_done;
  double e0 = 0.0;
  int iterations = 0;
  int converged = 0;
  bool cancel = false;
};

}  // namespace

struct ed_server {
  BatchEngine eng;
  ed_server_opts opts{};
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<double> latencies;
  uint64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0, failed = 0;
  int inject_left = 0;
  bool stop = false;
  bool have_first = false;
  Clock::time_point t_first;
  Clock::time_point t_last;
  uint64_t slot_owner[4096];
  int64_t free_cache = 0;  // arena bytes free, refreshed by the worker under mu
};

extern "C" void ed_server_default_opts(ed_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->device_bytes = (int64_t)1 << 30;
  o->max_slots = 256;
  o->max_iter = 400;
  o->check_every = 5;
  o->tol = 1e-7;
  o->seed = 20260507ULL;
  o->inject_alloc_failures = 0;
}

static void worker_loop(ed_server* S) {
  std::vector<int> done;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      int admitted = 0;  // device work lists are rebuilt once for all admissions of this round
      // admission in arrival order while a slot is free and the arena fits
      while (!S->stop && !S->queue.empty()) {
        Request& r = S->reqs[S->queue.front()];
        if (r.cancel) {
          r.state = 3;
          r.status = ED_ECANCELLED;
          r.t_done = Clock::now();
          S->queue.pop_front();
          S->cv_done.notify_all();
          continue;
        }
        if (S->eng.active_count() >= S->opts.max_slots || r.bytes + 4096 > S->eng.arena_free()) break;
        S->queue.pop_front();
        if (S->inject_left > 0) {  // host-side fault injection: the admission's allocation "fails"
          --S->inject_left;
          r.state = 4;
          r.status = ED_ENOMEM;
          r.t_done = Clock::now();
          ++S->failed;
          S->cv_done.notify_all();
          continue;
        }
        int slot = -1;
        lk.unlock();
        // CSR or tensor-core form: the choice cached for the shape by a
        // tuned batch of this process, else the dense form
        ed_status st = S->eng.add(r.m, S->opts.seed, &slot, false);
        lk.lock();
        if (st != ED_OK) {
          r.state = 4;
          r.status = st;
          r.msg = ed_last_error();
          r.t_done = Clock::now();
          ++S->failed;
          S->cv_done.notify_all();
          continue;
        }
        r.slot = slot;
        r.state = 1;
        r.t_admit = Clock::now();
        S->slot_owner[slot] = r.ticket;
        S->free_cache = (int64_t)S->eng.arena_free();
        ++admitted;
      }
      if (admitted > 0) {
        lk.unlock();
        const ed_status st = S->eng.rebuild_active();
        lk.lock();
        if (st != ED_OK) {
          const std::string msg = ed_last_error();
          for (auto& kv : S->reqs)
            if (kv.second.state == 1) {
              kv.second.state = 4;
              kv.second.status = st;
              kv.second.msg = msg;
              kv.second.t_done = Clock::now();
              ++S->failed;
            }
          S->stop = true;
          S->cv_done.notify_all();
          break;
        }
      }
      if (S->stop) break;
      if (S->eng.active_count() == 0) {
        S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
    }
    // one group of Lanczos steps over every admitted request
    ed_status st = S->eng.steps(S->opts.check_every);
    done.clear();
    if (st == ED_OK) st = S->eng.poll(S->opts.tol, S->opts.check_every, &done);
    std::lock_guard<std::mutex> lk(S->mu);
    if (st != ED_OK) {
      // device error: fail every running request and stop serving
      const std::string msg = ed_last_error();
      for (auto& kv : S->reqs)
        if (kv.second.state == 1) {
          kv.second.state = 4;
          kv.second.status = st;
          kv.second.msg = msg;
          kv.second.t_done = Clock::now();
          ++S->failed;
        }
      S->stop = true;
      S->cv_done.notify_all();
      break;
    }
    for (int slot : done) {
      Request& r = S->reqs[S->slot_owner[slot]];
      r.e0 = S->eng.energy(slot);
      r.iterations = S->eng.iterations(slot);
      r.converged = S->eng.converged(slot) ? 1 : 0;
      r.state = 2;
      r.status = r.converged ? ED_OK : ED_ENOCONV;
      r.t_done = Clock::now();
      S->eng.remove(slot, false);
      r.slot = -1;
      S->latencies.push_back(std::chrono::duration<double>(r.t_done - r.t_submit).count());
      ++S->completed;
      S->t_last = r.t_done;
    }
    // cancelled running requests leave between steps
    for (auto& kv : S->reqs) {
      Request& r = kv.second;
      if (r.state == 1 && r.cancel) {
        S->eng.remove(r.slot);
        r.slot = -1;
        r.state = 3;
        r.status = ED_ECANCELLED;
        r.t_done = Clock::now();
      }
    }
    S->free_cache = (int64_t)S->eng.arena_free();
    if (!done.empty()) S->cv_done.notify_all();
  }
}

extern "C" ed_status ed_server_create(const ed_server_opts* opts, ed_server** out) {
  if (!out) { set_error("out is NULL"); return ED_EINVAL; }
  *out = nullptr;
  ed_server_opts o;
  ed_server_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_slots < 1 || o.max_slots > 4096 || o.device_bytes < (1 << 20) || o.max_iter < 2 || o.check_every < 1) {
    set_error("bad server options");
    return ED_EINVAL;
  }
  ed_server* S = new (std::nothrow) ed_server();
  if (!S) { set_error("host allocation failed"); return ED_ENOMEM; }
  S->opts = o;
  S->inject_left = o.inject_alloc_failures;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = 0; }
  ed_status st = S->eng.init(dev, (size_t)o.device_bytes, o.max_slots, o.max_iter, true);
  if (st != ED_OK) { delete S; return st; }
  S->free_cache = (int64_t)S->eng.arena_free();
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return ED_OK;
}

extern "C" ed_status ed_server_submit(ed_server* S, const ed_model_desc* m, uint64_t* ticket) {
  if (!S || !m || !ticket) { set_error("NULL argument"); return ED_EINVAL; }
  size_t bytes = 0;
  int64_t dim = 0;
  ED_TRY(BatchEngine::instance_bytes(*m, true, &bytes, &dim));
  Request r;
  r.bi.assign(m->bi, m->bi + m->n_bonds);
  r.bj.assign(m->bj, m->bj + m->n_bonds);
  auto cp = [](const double* p, int n) { return p ? std::vector<double>(p, p + n) : std::vector<double>(n, 0.0); };
  r.jxy = cp(m->jxy, m->n_bonds);
  r.jz = cp(m->jz, m->n_bonds);
  r.t = cp(m->t, m->n_bonds);
  r.U = cp(m->U, m->n_sites);
  r.eps = cp(m->eps, m->n_sites);
  r.m = *m;
  r.bytes = bytes;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) { set_error("server stopped"); return ED_ECUDA; }
  if (bytes + 4096 > S->eng.arena_size()) { set_error("request needs %zu bytes, server budget %zu", bytes, S->eng.arena_size()); return ED_ENOMEM; }
  r.ticket = S->next_ticket++;
  r.t_submit = Clock::now();
  if (!S->have_first) { S->have_first = true; S->t_first = r.t_submit; }
  Request& stored = S->reqs[r.ticket];
  stored = std::move(r);
  // the descriptor points at the request's own copies
  stored.m.bi = stored.bi.data();
  stored.m.bj = stored.bj.data();
  stored.m.jxy = stored.jxy.data();
  stored.m.jz = stored.jz.data();
  stored.m.t = stored.t.data();
  stored.m.U = stored.U.data();
  stored.m.eps = stored.eps.data();
  S->queue.push_back(stored.ticket);
  ++S->submitted;
  *ticket = stored.ticket;
  S->cv_work.notify_one();
  return ED_OK;
}

extern "C" ed_status ed_server_wait(ed_server* S, uint64_t ticket, int timeout_ms, ed_result* res) {
  if (!S || !res) { set_error("NULL argument"); return ED_EINVAL; }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return ED_EINVAL; }
  auto finished = [&] { return it->second.state >= 2; };
  if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), finished)) {
    set_error("ticket %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
    return ED_ETIMEOUT;
  }
  const Request& r = it->second;
  std::memset(res, 0, sizeof(*res));
  res->e0 = r.e0;
  res->iterations = r.iterations;
  res->converged = r.converged;
  res->status = r.status;
  if (r.status != ED_OK && r.status != ED_ENOCONV && !r.msg.empty()) set_error("%s", r.msg.c_str());
  res->latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
  if (r.state == 2 || (r.state == 3 && r.t_admit.time_since_epoch().count() != 0)) {
    res->queue_s = std::chrono::duration<double>(r.t_admit - r.t_submit).count();
    res->run_s = std::chrono::duration<double>(r.t_done - r.t_admit).count();
  }
  return r.status == ED_ENOCONV ? ED_OK : r.status;
}

extern "C" ed_status ed_server_cancel(ed_server* S, uint64_t ticket) {
  if (!S) { set_error("NULL server"); return ED_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) { set_error("unknown ticket"); return ED_EINVAL; }
  if (it->second.state < 2) it->second.cancel = true;
  S->cv_work.notify_one();
  return ED_OK;
}

static double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  double pos = p * (v.size() - 1);
  size_t i = (size_t)pos;
  double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

extern "C" ed_status ed_server_get_stats(ed_server* S, ed_server_stats* out) {
  if (!S || !out) { set_error("NULL argument"); return ED_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (int64_t)S->queue.size();
  int64_t running = 0;
  for (auto& kv : S->reqs) running += kv.second.state == 1 ? 1 : 0;
  out->running = running;
  out->p50_s = percentile(S->latencies, 0.50);
  out->p99_s = percentile(S->latencies, 0.99);
  double sum = 0.0;
  for (double v : S->latencies) sum += v;
  out->mean_s = S->latencies.empty() ? 0.0 : sum / S->latencies.size();
  const double span = S->completed ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
  out->throughput_rps = span > 0 ? S->completed / span : 0.0;
  out->device_bytes = (int64_t)S->eng.arena_size();
  out->device_bytes_free = S->free_cache;
  return ED_OK;
}

extern "C" void ed_server_destroy(ed_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  delete S;
}
