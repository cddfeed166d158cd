// server.cu -- continuous-batching serving loop for pricing / hedging
// requests (bsde_server_* of include/bsde.h).
//
// A worker thread admits queued requests while slots and the device-memory
// budget allow.  Each admitted request gets a resident Problem (its points,
// basis matrix, Gram matrix, coefficients and Philox key stay on the device
// for all its Picard iterations) and a stream of its own; its whole solve is
// one captured CUDA graph, so the iterations of all admitted requests run
// concurrently on the GPU.  When a request's completion event fires, the
// worker builds its report, records its latency (submit -> completion),
// frees its memory and admits the next request in the queue.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "runtime.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t id = 0;
  ModelHost model;
  GridHost grid;
  bsde_solve_params prm;
  double t_submit = 0.0, t_done = 0.0;
  size_t bytes = 0;
  double work = 0.0;  // K_it n M N, the shortest-first key
  int prio = 0;       // 1: admitted on a high-priority stream
  std::unique_ptr<Problem> prob;
  cudaStream_t stream = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bsde_report rep;
  int rc = 0;
};

}  // namespace

struct bsde_server {
  bsde_server_opts opts;
  Allocator al;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<std::unique_ptr<Req>> queue;
  std::vector<std::unique_ptr<Req>> running;
  std::map<uint64_t, std::unique_ptr<Req>> done;
  // streams of finished requests, by priority: requests with less work than
  // the average so far run on high-priority streams, so that their kernels
  // take the next free CTA slots ahead of the long requests' path kernels
  std::vector<cudaStream_t> free_streams[2];  // [0] normal, [1] high priority
  double work_sum = 0.0;
  uint64_t work_count = 0;
  int large_running = 0;  // running requests on normal-priority streams
  size_t used_bytes = 0;
  std::vector<uint64_t> admitting;  // ids popped from the queue, not yet in running/done
  std::vector<double> latencies_ms;
  double path_steps = 0.0, busy_s = 0.0, busy_since = -1.0;
  uint64_t completed = 0;
  std::string err;

  void loop();
  bool admit_one(std::unique_lock<std::mutex>& lk);
};

bool bsde_server::admit_one(std::unique_lock<std::mutex>& lk) {
  if (queue.empty() || (int)running.size() >= opts.max_slots) return false;
  // next request: the oldest (FIFO), the one with the least work, or the
  // one with the highest response ratio (wait + service) / service
  size_t pick = 0;
  if (opts.policy == BSDE_POLICY_SHORTEST) {
    for (size_t q = 1; q < queue.size(); ++q)
      if (queue[q]->work < queue[pick]->work) pick = q;
  } else if (opts.policy == BSDE_POLICY_SIZE_LANES) {
    // arrival order, but a request with at least the average work waits
    // while large_slots such requests run; smaller ones pass it
    const double sum = work_sum, cnt = (double)work_count;
    bool found = false;
    for (size_t q = 0; q < queue.size(); ++q) {
      const double w = queue[q]->work;
      const bool large = w >= (sum + w) / (cnt + 1.0);
      if (!large || large_running < (opts.large_slots > 0 ? opts.large_slots : 2)) {
        pick = q;
        found = true;
        break;
      }
    }
    if (!found) return false;
  } else if (opts.policy == BSDE_POLICY_RESPONSE_RATIO) {
    // service estimate: path-steps at the throughput measured so far (a
    // GB300-scale default until a second of busy time has been seen)
    const double t = now_s();
    const double busy = busy_s + (busy_since >= 0 ? t - busy_since : 0.0);
    const double rate = busy > 1.0 && path_steps > 0 ? path_steps / busy : 5e10;
    double best = -1.0;
    for (size_t q = 0; q < queue.size(); ++q) {
      const double svc = queue[q]->work / rate + 1e-4;
      const double ratio = (t - queue[q]->t_submit + svc) / svc;
      if (ratio > best) {
        best = ratio;
        pick = q;
      }
    }
  }
  Req* r = queue[pick].get();
  if (opts.mem_budget && used_bytes + r->bytes > opts.mem_budget && !running.empty()) return false;
  std::unique_ptr<Req> req = std::move(queue[pick]);
  queue.erase(queue.begin() + pick);
  used_bytes += req->bytes;
  if (busy_since < 0) busy_since = now_s();
  cudaStream_t st;
  work_sum += req->work;
  ++work_count;
  const int hi = req->work < work_sum / (double)work_count ? 1 : 0;
  if (!free_streams[hi].empty()) {
    st = free_streams[hi].back();
    free_streams[hi].pop_back();
  } else {
    int lo_p = 0, hi_p = 0;
    cudaDeviceGetStreamPriorityRange(&lo_p, &hi_p);
    cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi ? hi_p : lo_p);
  }
  req->prio = hi;
  if (!hi) ++large_running;
  req->stream = st;
  admitting.push_back(req->id);
  lk.unlock();
  // device work outside the lock: allocation, capture, graph launch
  req->prob.reset(new Problem());
  Problem& P = *req->prob;
  P.mixed = (opts.precision == BSDE_PREC_MIXED);
  P.model = req->model;
  P.grid = req->grid;
  P.has_model = P.has_grid = true;
  cudaEventCreate(&req->e0);
  cudaEventCreate(&req->e1);
  req->rc = P.start(req->prm, al, 0, st, req->e0, req->e1);
  lk.lock();
  admitting.erase(std::find(admitting.begin(), admitting.end(), req->id));
  if (req->rc != BSDE_OK) {
    // failed before reaching the device: complete immediately
    memset(&req->rep, 0, sizeof(req->rep));
    req->rep.status = req->rc;
    req->t_done = now_s();
    P.release(al, st);
    used_bytes -= req->bytes;
    if (!req->prio) --large_running;
    free_streams[req->prio].push_back(st);
    done[req->id] = std::move(req);
    cv_done.notify_all();
    return true;
  }
  running.push_back(std::move(req));
  return true;
}

void bsde_server::loop() {
  cudaSetDevice(opts.device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    while (admit_one(lk)) {
    }
    // completions
    bool progressed = false;
    for (size_t i = 0; i < running.size();) {
      Req* r = running[i].get();
      if (cudaEventQuery(r->e1) == cudaErrorNotReady) {
        ++i;
        continue;
      }
      lk.unlock();
      r->rc = r->prob->complete(r->prm, r->stream, r->e0, r->e1, &r->rep);
      r->rep.status = r->rc;
      r->t_done = now_s();
      r->prob->release(al, r->stream);
      cudaStreamSynchronize(r->stream);
      cudaEventDestroy(r->e0);
      cudaEventDestroy(r->e1);
      r->e0 = r->e1 = nullptr;
      lk.lock();
      used_bytes -= r->bytes;
      if (!r->prio) --large_running;
      free_streams[r->prio].push_back(r->stream);
      latencies_ms.push_back((r->t_done - r->t_submit) * 1e3);
      if (r->rc == BSDE_OK) path_steps += r->rep.path_steps;
      ++completed;
      r->prob.reset();
      done[r->id] = std::move(running[i]);
      running.erase(running.begin() + i);
      progressed = true;
      cv_done.notify_all();
    }
    if (running.empty() && busy_since >= 0) {
      busy_s += now_s() - busy_since;
      busy_since = -1.0;
    }
    if (!progressed) {
      if (running.empty() && queue.empty() && admitting.empty())
        cv.wait(lk);
      else
        cv.wait_for(lk, std::chrono::microseconds(200));
    }
  }
}

extern "C" {

int bsde_server_create(bsde_server** out, const bsde_server_opts* o) {
  if (!out || !o || o->max_slots < 1 || o->max_slots > 64 || o->large_slots < 0 ||
      o->large_slots > 64 ||
      (o->precision != BSDE_PREC_FP64 && o->precision != BSDE_PREC_MIXED) ||
      (o->policy != BSDE_POLICY_FIFO && o->policy != BSDE_POLICY_SHORTEST &&
       o->policy != BSDE_POLICY_RESPONSE_RATIO && o->policy != BSDE_POLICY_SIZE_LANES))
    return BSDE_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o->device < 0 || o->device >= ndev) {
    cudaGetLastError();
    return BSDE_ERR_CUDA;
  }
  try {
    bsde_server* s = new bsde_server();
    s->opts = *o;
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return BSDE_OK;
  } catch (...) {
    return BSDE_ERR_NOMEM;
  }
}

int bsde_server_submit(bsde_server* s, const bsde_request* rq, uint64_t* id) {
  if (!s || !rq || !id) return BSDE_ERR_INVALID_ARG;
  try {
    std::unique_ptr<Req> r(new Req());
    std::string e;
    int rc = bsde_set_model_impl(r->model, &rq->sigma, rq->r, &rq->payoff, &rq->penalty, e);
    if (rc == BSDE_OK)
      rc = bsde_set_grid_impl(r->grid, r->model.d, rq->n, rq->lo, rq->hi, 1, e);
    if (rc != BSDE_OK) {
      std::lock_guard<std::mutex> g(s->mu);
      s->err = e;
      return rc;
    }
    r->prm = rq->params;
    int p = 0;
    rc = bsde_basis_size(r->model.d, r->prm.eta, r->prm.q, &p);
    if (rc != BSDE_OK) return rc;
    const int tpb = s->opts.precision == BSDE_PREC_MIXED ? 128 : 64;
    const bool qr = r->prm.ls_mode == 1;
    r->bytes = Problem::estimate_bytes(r->model.d, rq->n, p, r->prm.M, r->prm.N_steps,
                                       s->opts.precision == BSDE_PREC_MIXED, tpb, 4, 0, 0, qr,
                                       Problem::fact_group(p, r->prm.K_it, true, qr));
    r->work = (double)r->prm.K_it * rq->n * (double)r->prm.M * r->prm.N_steps;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> g(s->mu);
    if (s->opts.mem_budget && r->bytes > s->opts.mem_budget) {
      s->err = "submit: request larger than the server's memory budget";
      return BSDE_ERR_NOMEM;
    }
    r->id = s->next_id++;
    *id = r->id;
    s->queue.push_back(std::move(r));
    s->cv.notify_all();
    return BSDE_OK;
  } catch (...) {
    return BSDE_ERR_NOMEM;
  }
}

int bsde_server_poll(bsde_server* s, uint64_t id, bsde_report* rep) {
  if (!s) return BSDE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->done.find(id);
  if (it == s->done.end()) {
    for (auto& r : s->queue)
      if (r->id == id) return 0;
    for (auto& r : s->running)
      if (r->id == id) return 0;
    if (std::find(s->admitting.begin(), s->admitting.end(), id) != s->admitting.end()) return 0;
    s->err = "poll: unknown request id";
    return BSDE_ERR_INVALID_ARG;
  }
  if (rep) *rep = it->second->rep;
  s->done.erase(it);
  return 1;
}

int bsde_server_drain(bsde_server* s, double timeout_ms) {
  if (!s) return BSDE_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto pred = [s] { return s->queue.empty() && s->running.empty() && s->admitting.empty(); };
  if (timeout_ms > 0) {
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred))
      return BSDE_ERR_TIMEOUT;
  } else {
    s->cv_done.wait(lk, pred);
  }
  return BSDE_OK;
}

int bsde_server_stats_get(bsde_server* s, bsde_server_stats* st) {
  if (!s || !st) return BSDE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  memset(st, 0, sizeof(*st));
  st->completed = s->completed;
  st->queued = s->queue.size();
  st->running = s->running.size() + s->admitting.size();
  std::vector<double> l = s->latencies_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    size_t idx = (size_t)(q * (double)(l.size() - 1) + 0.5);
    return l[std::min(idx, l.size() - 1)];
  };
  st->p50_ms = pct(0.50);
  st->p99_ms = pct(0.99);
  st->path_steps = s->path_steps;
  double busy = s->busy_s + (s->busy_since >= 0 ? now_s() - s->busy_since : 0.0);
  st->busy_s = busy;
  st->path_steps_per_s = busy > 0 ? s->path_steps / busy : 0.0;
  return BSDE_OK;
}

void bsde_server_destroy(bsde_server* s) {
  if (!s) return;
  bsde_server_drain(s, 0);
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->worker.join();
  cudaSetDevice(s->opts.device);
  for (auto& pool : s->free_streams)
    for (auto st : pool) cudaStreamDestroy(st);
  delete s;
}

const char* bsde_server_last_error(const bsde_server* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
