// Request server over the public plan API (helm.h): a FIFO of independent
// solve requests, a device-memory-budgeted plan cache, one scheduler thread
// that starts requests on a pool of CUDA streams as slots and plans free up,
// so independent requests overlap on the GPU, and one builder thread that
// makes new plans meanwhile (a plan build works on the legacy stream and the
// slots' streams are non-blocking, so builds and solves overlap too).  The
// paper's method has no counterpart: this is the serving layer around its
// solver.
//
// Only the scheduler and the builder make CUDA calls after creation;
// submitters and waiters touch the queue and the results under the server
// mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "helm.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

struct PlanKey {
  int32_t dim, dtype, residual, max_iter;
  int64_t n[3];
  double h[3], omega, tol;
  bool operator==(const PlanKey& o) const {
    return dim == o.dim && dtype == o.dtype && residual == o.residual && max_iter == o.max_iter &&
           n[0] == o.n[0] && n[1] == o.n[1] && n[2] == o.n[2] && h[0] == o.h[0] && h[1] == o.h[1] &&
           h[2] == o.h[2] && omega == o.omega && tol == o.tol;
  }
};

PlanKey key_of(const helm_request& r) {
  PlanKey k{};
  k.dim = r.dim;
  k.dtype = r.dtype;
  const bool refined = r.dtype == HELM_C64_REFINED;
  k.residual = refined ? r.residual : 0;
  k.max_iter = refined ? r.max_iter : 0;
  k.tol = refined ? r.tol : 0.0;
  k.n[0] = r.n[0];
  k.n[1] = r.n[1];
  k.n[2] = r.dim == 3 ? r.n[2] : 1;
  k.h[0] = r.h[0];
  k.h[1] = r.h[1];
  k.h[2] = r.dim == 3 ? r.h[2] : 0.0;
  k.omega = r.omega;
  return k;
}

int64_t unknowns(const helm_request& r) { return r.n[0] * r.n[1] * (r.dim == 3 ? r.n[2] : 1); }

// Device memory of a plan before it exists, for admission: per unknown, above
// what the plans of these modes were measured to hold (2D complex64 refined
// with the float-float residual 79 B, complex128 191 B; 3D 96 B and 112 B),
// plus a fixed allowance for the O(n) tables.
size_t plan_bytes_estimate(const helm_request& r) {
  const double N = (double)unknowns(r);
  double per;
  if (r.dim == 2) per = r.dtype == HELM_C128 ? 200.0 : 100.0;
  else per = r.dtype == HELM_C128 ? 128.0 : 112.0;
  return (size_t)(per * N) + ((size_t)64 << 20);
}

struct PlanEntry {
  PlanKey key;
  helm_plan_t plan = nullptr;
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_use = 0;
};

struct Request {
  int64_t ticket = 0;
  helm_request spec{};
  Clock::time_point t_submit, t_start, t_done;
  bool started = false, done = false;
  int status = HELM_OK;
  int plan_reused = 0;
  size_t reserve = 0;  // device memory reserved while its plan is built
  bool fresh = false;  // its plan was built for it (not a reuse)
  int iterations = 0, converged = 1;
  double residual = 0.0;
  std::string error;  // what failed, for a request that did not complete
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Request* req = nullptr;
  PlanEntry* plan = nullptr;
};

int check_request(const helm_request* r) {
  if (!r || (r->dim != 2 && r->dim != 3) || r->nrhs < 1 || !r->f || !r->u) return HELM_EINVAL;
  const int nd = r->dim;
  for (int k = 0; k < nd; ++k)
    if (r->n[k] < 3 || !(r->h[k] > 0) || !std::isfinite(r->h[k])) return HELM_EINVAL;
  if (!(r->omega > 0) || !std::isfinite(r->omega)) return HELM_EINVAL;
  if (r->dtype != HELM_C128 && r->dtype != HELM_C64_RAW && r->dtype != HELM_C64_REFINED) return HELM_EINVAL;
  if (r->dtype == HELM_C64_REFINED) {
    if (r->residual != HELM_RESID_FP64 && r->residual != HELM_RESID_FF) return HELM_EINVAL;
    if (!(r->tol >= 0) || r->max_iter < 1 || r->max_iter > 15) return HELM_EINVAL;
  }
  // f and u must not overlap
  const size_t eb = r->dtype == HELM_C64_RAW ? 8 : 16;
  const size_t bytes = (size_t)unknowns(*r) * (size_t)r->nrhs * eb;
  const char* f = static_cast<const char*>(r->f);
  const char* u = static_cast<const char*>(r->u);
  if (f < u + bytes && u < f + bytes) return HELM_EINVAL;
  return HELM_OK;
}

}  // namespace

struct helm_server {
  int device = 0;
  size_t budget = 0, in_use = 0, peak = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // scheduler: a request arrived, or stop
  std::condition_variable cv_done;  // waiters: a request finished
  std::deque<Request*> pending;     // FIFO, not yet started
  std::unordered_map<int64_t, std::unique_ptr<Request>> requests;
  std::vector<std::unique_ptr<PlanEntry>> cache;
  std::vector<Slot> slots;
  int64_t next_ticket = 1;
  uint64_t use_clock = 0;
  bool stop = false;
  int64_t submitted = 0, completed = 0, failed = 0, built = 0, reused = 0, evicted = 0;
  double unknowns_solved = 0.0;
  bool any_submit = false;
  Clock::time_point t_first, t_last;
  std::vector<double> latencies;
  std::thread worker;
  // plan builds: requests waiting for the builder, the operators being built
  std::deque<Request*> build_queue;
  std::vector<PlanKey> building;
  int builds_in_flight = 0;
  bool stop_build = false;
  // bumped (under the mutex) by every event that may let a waiting request
  // start: a submission, a finished build, stop
  uint64_t wake = 0;
  std::condition_variable cv_build;
  std::thread builder;

  void run();
  void build_loop();
  bool being_built(const PlanKey& k) const {
    for (const PlanKey& b : building)
      if (b == k) return true;
    return false;
  }
  bool builds_pending() const { return builds_in_flight > 0 || !build_queue.empty(); }
  bool start_one(std::unique_lock<std::mutex>& lk);
  void finish(Slot& sl, cudaError_t q);
  void fail(Request* r, int status, const std::string& why);
  bool running() const {
    for (const Slot& s : slots)
      if (s.req) return true;
    return false;
  }
};

namespace {

// the plan's settings for a request (refined modes).  Server plans launch
// kernel by kernel: a CUDA graph capture in the scheduler thread would make
// any device-wide synchronisation by another thread of the process fail
// while it lasts.
int configure(helm_plan_t p, const helm_request& r) {
  int rc = helm_set_graphs(p, 0);
  if (rc || r.dtype != HELM_C64_REFINED) return rc;
  rc = helm_set_residual(p, r.residual);
  if (!rc) rc = helm_set_refinement(p, r.tol, r.max_iter);
  return rc;
}

}  // namespace

void helm_server::fail(Request* r, int status, const std::string& why) {
  r->status = status;
  r->error = why;
  r->done = true;
  r->t_done = Clock::now();
  ++failed;
  cv_done.notify_all();
}

void helm_server::finish(Slot& sl, cudaError_t q) {
  Request* r = sl.req;
  if (q != cudaSuccess && r->status == HELM_OK) {
    r->status = HELM_ECUDA;
    r->error = std::string("completion event: ") + cudaGetErrorString(q);
  }
  if (r->status == HELM_OK) {
    helm_info info;
    int rc = helm_get_info(sl.plan->plan, &info);  // the slot's work is complete
    const bool filled = rc == HELM_OK || rc == HELM_ENOTCONV;  // ENOTCONV: info is filled
    if (filled) {
      // a plan's first solve may add buffers (the float-float vectors)
      in_use = in_use - std::min(in_use, sl.plan->bytes) + info.device_bytes;
      sl.plan->bytes = info.device_bytes;
      peak = std::max(peak, in_use);
    }
    if (!filled) {
      r->status = rc;
      r->error = std::string("helm_get_info: ") + helm_status_string(rc) + ": " + helm_last_error(sl.plan->plan);
    } else if (r->spec.dtype == HELM_C64_REFINED) {
      r->iterations = info.iterations;
      r->converged = info.converged;
      r->residual = info.residual[info.iterations];
      if (!info.converged) r->status = HELM_ENOTCONV;
    }
  }
  r->t_done = Clock::now();
  r->done = true;
  t_last = r->t_done;
  if (r->status == HELM_OK || r->status == HELM_ENOTCONV) {
    ++completed;
    unknowns_solved += (double)unknowns(r->spec) * (double)r->spec.nrhs;
    latencies.push_back(seconds_between(r->t_submit, r->t_done));
  } else {
    ++failed;
  }
  sl.plan->busy = false;
  sl.plan->last_use = ++use_clock;
  sl.req = nullptr;
  sl.plan = nullptr;
  cv_done.notify_all();
}

// Start the oldest pending request that can start now.  Returns true if the
// queue changed (a request started or failed).
bool helm_server::start_one(std::unique_lock<std::mutex>& lk) {
  Slot* slot = nullptr;
  for (Slot& s : slots)
    if (!s.req) {
      slot = &s;
      break;
    }
  if (!slot || pending.empty()) return false;
  bool memory_blocked = false;  // an older request waits for memory: later ones may only reuse plans
  for (size_t qi = 0; qi < pending.size(); ++qi) {
    Request* r = pending[qi];
    const PlanKey key = key_of(r->spec);
    PlanEntry* pe = nullptr;
    bool found_busy = false;
    for (auto& e : cache)
      if (e->key == key) {
        if (!e->busy) pe = e.get();
        else found_busy = true;
        if (pe) break;
      }
    bool reuse = pe != nullptr && !r->fresh;
    if (!pe) {
      // its plan is busy or being built (one instance per operator), or an
      // older request waits for memory
      if (found_busy || memory_blocked || being_built(key)) continue;
      const size_t est = plan_bytes_estimate(r->spec);
      if (est > budget) {
        pending.erase(pending.begin() + (std::ptrdiff_t)qi);
        fail(r, HELM_ENOMEM, "the plan's estimate exceeds the device budget");
        return true;
      }
      // evict idle plans, least recently used first, until the estimate fits
      while (in_use + est > budget) {
        PlanEntry* lru = nullptr;
        size_t lru_i = 0;
        for (size_t i = 0; i < cache.size(); ++i)
          if (!cache[i]->busy && (!lru || cache[i]->last_use < lru->last_use)) {
            lru = cache[i].get();
            lru_i = i;
          }
        if (!lru) break;
        helm_destroy(lru->plan);
        in_use -= std::min(in_use, lru->bytes);
        cache.erase(cache.begin() + (std::ptrdiff_t)lru_i);
        ++evicted;
      }
      if (in_use + est > budget) {
        if (!running() && !builds_pending()) {  // nothing will free memory: it can never fit
          pending.erase(pending.begin() + (std::ptrdiff_t)qi);
          fail(r, HELM_ENOMEM, "the plan does not fit the device budget beside the cached plans");
          return true;
        }
        memory_blocked = true;
        continue;
      }
      // the builder thread makes the plan; the scheduler goes on with other
      // requests, and this one returns to the front of the queue when built
      pending.erase(pending.begin() + (std::ptrdiff_t)qi);
      in_use += est;  // reserved while building
      r->reserve = est;
      building.push_back(key);
      build_queue.push_back(r);
      cv_build.notify_one();
      return true;
    } else {
      pending.erase(pending.begin() + (std::ptrdiff_t)qi);
      if (reuse) ++reused;
    }
    // launch its right-hand sides on the slot's stream
    pe->busy = true;
    pe->last_use = ++use_clock;
    r->started = true;
    r->plan_reused = reuse ? 1 : 0;
    r->t_start = Clock::now();
    const size_t eb = r->spec.dtype == HELM_C64_RAW ? 8 : 16;
    const size_t stride = (size_t)unknowns(r->spec) * eb;
    int rc = helm_set_stream(pe->plan, slot->stream);
    (void)stride;
    // the request's right-hand sides, several at once on the plan's workspaces
    if (!rc) rc = helm_solve_many(pe->plan, r->spec.nrhs, r->spec.f, r->spec.u);
    if (rc) {
      r->status = rc;
      r->error = std::string("solve: ") + helm_status_string(rc) + ": " + helm_last_error(pe->plan);
    }
    cudaEventRecord(slot->done, slot->stream);
    slot->req = r;
    slot->plan = pe;
    return true;
  }
  return false;
}

void helm_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    const uint64_t seen = wake;
    bool progress = false;
    for (Slot& sl : slots)
      if (sl.req) {
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        finish(sl, q);
        progress = true;
      }
    while (start_one(lk)) progress = true;
    const bool busy = running();
    if (stop && pending.empty() && !busy && !builds_pending()) break;
    if (progress) continue;
    // nothing started: sleep until a slot may have finished (polled) or
    // something else changed; requests that wait for a plan being built
    // must not keep the mutex from the builder
    if (busy) cv_work.wait_for(lk, std::chrono::microseconds(50));
    else cv_work.wait(lk, [&] { return wake != seen; });
  }
}

// The builder: plans for the requests the scheduler queued, one at a time,
// with the lock released while building.  A built plan joins the cache idle
// and its request goes back to the front of the queue.
void helm_server::build_loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv_build.wait(lk, [&] { return stop_build || !build_queue.empty(); });
    if (build_queue.empty()) break;  // stop_build
    Request* r = build_queue.front();
    build_queue.pop_front();
    ++builds_in_flight;
    const helm_request sp = r->spec;
    const PlanKey key = key_of(sp);
    lk.unlock();
    helm_plan_t plan = nullptr;
    int rc = sp.dim == 2 ? helm_plan_2d(&plan, sp.n[0], sp.n[1], sp.h[0], sp.h[1], sp.omega, sp.dtype)
                         : helm_plan_3d(&plan, sp.n[0], sp.n[1], sp.n[2], sp.h[0], sp.h[1], sp.h[2], sp.omega,
                                        sp.dtype);
    if (!rc) rc = configure(plan, sp);
    helm_info info;
    if (!rc) {
      rc = helm_get_info(plan, &info);
      if (rc == HELM_ENOTCONV) rc = HELM_OK;  // the state of the plan's trial solves: info is filled
    }
    std::string why;
    if (rc) {
      why = std::string("plan build: ") + helm_status_string(rc);
      if (plan) why += std::string(": ") + helm_last_error(plan);
    }
    if (rc && plan) {
      helm_destroy(plan);
      plan = nullptr;
    }
    lk.lock();
    --builds_in_flight;
    in_use -= std::min(in_use, r->reserve);
    r->reserve = 0;
    for (size_t i = 0; i < building.size(); ++i)
      if (building[i] == key) {
        building.erase(building.begin() + (std::ptrdiff_t)i);
        break;
      }
    if (rc) {
      fail(r, rc, why);
    } else {
      auto e = std::make_unique<PlanEntry>();
      e->key = key;
      e->plan = plan;
      e->bytes = info.device_bytes;
      e->last_use = ++use_clock;
      in_use += e->bytes;
      peak = std::max(peak, in_use);
      cache.push_back(std::move(e));
      ++built;
      r->fresh = true;
      pending.push_front(r);
    }
    ++wake;
    cv_work.notify_one();
  }
}

namespace {

// waits on `cv` until pred() holds; timeout_s < 0: no limit.  True if pred holds.
template <typename Pred>
bool wait_until(std::condition_variable& cv, std::unique_lock<std::mutex>& lk, double timeout_s, Pred pred) {
  if (timeout_s < 0) {
    cv.wait(lk, pred);
    return true;
  }
  return cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = (size_t)std::ceil(q * (double)v.size());  // nearest rank
  return v[std::min(v.size() - 1, i > 0 ? i - 1 : 0)];
}

}  // namespace

extern "C" {

int helm_server_create(helm_server_t* out, int32_t nslots, size_t device_budget_bytes) {
  if (!out) return HELM_EINVAL;
  *out = nullptr;
  if (nslots < 1 || nslots > 16 || device_budget_bytes == 0) return HELM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HELM_ECUDA;
  }
  auto s = std::make_unique<helm_server>();
  s->device = dev;
  s->budget = device_budget_bytes;
  s->slots.resize((size_t)nslots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (Slot& t : s->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.done) cudaEventDestroy(t.done);
      }
      return HELM_ECUDA;
    }
  }
  helm_server* raw = s.release();
  raw->worker = std::thread([raw] { raw->run(); });
  raw->builder = std::thread([raw] { raw->build_loop(); });
  *out = raw;
  return HELM_OK;
}

int helm_server_submit(helm_server_t s, const helm_request* req, int64_t* ticket) {
  if (!s || !ticket) return HELM_EINVAL;
  *ticket = 0;
  const int rc = check_request(req);
  if (rc) return rc;
  auto r = std::make_unique<Request>();
  r->spec = *req;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return HELM_EINVAL;
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    if (!s->any_submit) {
      s->any_submit = true;
      s->t_first = r->t_submit;
    }
    ++s->submitted;
    ++s->wake;
    s->pending.push_back(r.get());
    s->requests.emplace(r->ticket, std::move(r));
  }
  s->cv_work.notify_one();
  return HELM_OK;
}

int helm_server_wait(helm_server_t s, int64_t ticket, double timeout_s, helm_request_result* res) {
  if (!s) return HELM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return HELM_EINVAL;
  Request* r = it->second.get();
  const bool done = wait_until(s->cv_done, lk, timeout_s, [&] { return r->done; });
  if (res) {
    std::memset(res, 0, sizeof(*res));
    res->done = r->done ? 1 : 0;
    res->status = r->status;
    res->plan_reused = r->plan_reused;
    res->iterations = r->iterations;
    res->converged = r->converged;
    res->residual = r->residual;
    if (r->started) res->queue_s = seconds_between(r->t_submit, r->t_start);
    if (r->done) res->latency_s = seconds_between(r->t_submit, r->t_done);
  }
  return done ? HELM_OK : HELM_ETIMEOUT;
}

const char* helm_server_error(helm_server_t s, int64_t ticket) {
  if (!s) return "";
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  return it == s->requests.end() ? "" : it->second->error.c_str();
}

int helm_server_drain(helm_server_t s, double timeout_s) {
  if (!s) return HELM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = wait_until(s->cv_done, lk, timeout_s, [&] { return s->completed + s->failed == s->submitted; });
  return ok ? HELM_OK : HELM_ETIMEOUT;
}

int helm_server_get_stats(helm_server_t s, helm_server_stats* st) {
  if (!s || !st) return HELM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->plans_built = s->built;
  st->plans_reused = s->reused;
  st->plans_evicted = s->evicted;
  st->unknowns_solved = s->unknowns_solved;
  st->elapsed_s = s->any_submit && s->completed > 0 ? seconds_between(s->t_first, s->t_last) : 0.0;
  st->latency_p50_s = percentile(s->latencies, 0.50);
  st->latency_p99_s = percentile(s->latencies, 0.99);
  double sum = 0.0;
  for (double v : s->latencies) sum += v;
  st->latency_mean_s = s->latencies.empty() ? 0.0 : sum / (double)s->latencies.size();
  st->device_bytes_in_use = s->in_use;
  st->device_bytes_peak = s->peak;
  return HELM_OK;
}

int helm_server_destroy(helm_server_t s) {
  if (!s) return HELM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    ++s->wake;
  }
  s->cv_work.notify_one();
  if (s->worker.joinable()) s->worker.join();  // after every queued request, builds included
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_build = true;
  }
  s->cv_build.notify_one();
  if (s->builder.joinable()) s->builder.join();
  cudaSetDevice(s->device);
  for (auto& e : s->cache) helm_destroy(e->plan);
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  delete s;
  return HELM_OK;
}

}  // extern "C"
