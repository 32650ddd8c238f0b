// Serving loop: continuous batching of CC3 triples requests on one GPU.
//
// Requests (a residual, Algorithm 1, or a Jacobian transformation of trial
// vectors, for problems of any (no, nv)) are copied at submit and queued.
// The server owns max_slots worker threads, each with its own non-blocking
// CUDA stream.  A free worker admits the first queued request whose device
// footprint fits the remaining HBM budget (first fit; once the oldest queued
// request has waited longer than the aging limit, only it may be admitted, so
// that large requests are not starved by a stream of small ones).  An
// admitted request keeps its integrals and amplitudes resident in its own
// context for its whole evaluation; the batches of triples of all admitted
// requests are issued on their own streams and interleave on the device.
//
// Failure isolation: a request that fails (bad input, vanishing denominator,
// out of memory, a bounded device wait that gave up) completes with its
// status and does not disturb the others.  A sticky CUDA error (one that
// invalidates the device context) cannot be isolated: every later request
// then fails with CC3_ERR_CUDA.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cc3_internal.h"
#include "split.h"

namespace {

using Clock = std::chrono::steady_clock;
double secs(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double>(b - a).count();
}

enum ReqState { PENDING = 0, RUNNING = 1, DONE = 2 };

struct Req {
  uint64_t ticket = 0;
  cc3_request q{};  // sizes and user output pointers
  std::vector<double> eps_o, eps_v, t2, vvvo, ooov, ovov, F, chol, omega, R1, R2;
  std::vector<double> o1, o2, e, rho1, rho2;
  size_t footprint = 0;
  int state = PENDING;
  int status = CC3_OK;
  bool cancel = false;
  double nominal = 0.0;
  Clock::time_point t_submit, t_start, t_done;
};

constexpr double kAgingSeconds = 10.0;
constexpr size_t kMargin = 64u << 20;  // CUDA plan tables, rounding of allocations

size_t request_footprint(const cc3_request &q) {
  const int ntri = q.no * (q.no + 1) * (q.no + 2) / 6;
  size_t b = cc3::ctx_footprint(q.no, q.nv, q.naux, ntri, true);
  if (q.flags & CC3_DETERMINISTIC) b += 16 * ((size_t)q.no * q.nv * (1 + (size_t)q.no * q.nv));
  if (q.prec == CC3_SPLIT_BF16) b += cc3::split_footprint(q.no, q.nv, 6, ntri);
  if (q.kind == 1) b += cc3::jacobian_footprint(q.no, q.nv, q.naux, q.nvec, ntri, true);
  if (q.kind == 1 && q.prec == CC3_SPLIT_BF16)
    b += cc3::split_jacobian_footprint(q.no, q.nv, 6, q.nvec);
  return b + kMargin;
}

int validate(const cc3_request &q) {
  if (q.kind != 0 && q.kind != 1) return CC3_ERR_ARG;
  if (q.prec != CC3_FP64 && q.prec != CC3_SPLIT_BF16 && q.prec != CC3_SPLIT_INT8)
    return CC3_ERR_ARG;
  if (q.no < 1 || q.nv < 1 || q.no > 256 || q.nv > 1024 || q.naux < 0) return CC3_ERR_ARG;
  if (!q.eps_o || !q.eps_v || !q.t2 || !q.g_vvvo || !q.g_ooov || !q.g_ovov || !q.F_ov)
    return CC3_ERR_ARG;
  if (q.naux > 0 && !q.chol_L) return CC3_ERR_ARG;
  if (q.kind == 1 && (q.nvec < 1 || !q.omega || !q.R1 || !q.R2 || q.naux < 1 || !q.rho1 ||
                      !q.rho2))
    return CC3_ERR_ARG;
  if (q.flags & ~CC3_DETERMINISTIC) return CC3_ERR_ARG;
  if ((q.flags & CC3_DETERMINISTIC) && q.kind == 1) return CC3_ERR_UNSUPPORTED;
  return CC3_OK;
}

template <class T>
void copy_in(std::vector<T> &dst, const T *src, size_t n) {
  if (src) dst.assign(src, src + n);
}

}  // namespace

struct cc3_server {
  int device = 0;
  size_t budget = 0, in_use = 0, peak = 0;
  int max_slots = 1;
  std::mutex mu;
  std::condition_variable cv_work;  // workers: a request was queued or memory freed
  std::condition_variable cv_done;  // waiters: a request completed
  std::deque<Req *> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  std::vector<std::thread> workers;
  bool stopping = false;
  uint64_t next_ticket = 1;
  long long submitted = 0, admitted = 0, completed = 0, rejected = 0, cancelled = 0;
  std::vector<double> lat_ms;
  double nominal = 0.0;
  int running = 0;
  double busy_total = 0.0;
  Clock::time_point t0, busy_since;
};

namespace {

// Under the lock: the next request to admit, removed from the queue.
Req *pick(cc3_server *S) {
  if (S->pending.empty()) return nullptr;
  const auto now = Clock::now();
  const bool head_aged = secs(S->pending.front()->t_submit, now) > kAgingSeconds;
  for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
    Req *r = *it;
    if (S->in_use + r->footprint <= S->budget) {
      S->pending.erase(it);
      return r;
    }
    if (head_aged) break;
  }
  return nullptr;
}

int execute(Req *r, cudaStream_t st) {
  const cc3_request &q = r->q;
  cc3_ctx *ctx = nullptr;
  int rc = cc3_ctx_create(&ctx, q.no, q.nv, r->eps_o.data(), r->eps_v.data(), r->t2.data(),
                          r->vvvo.data(), r->ooov.data(), r->ovov.data(), r->F.data(),
                          q.naux > 0 ? r->chol.data() : nullptr, q.naux, q.flags, st);
  if (rc != CC3_OK) return rc;
  const size_t n1 = (size_t)q.no * q.nv, nt2 = n1 * q.no * q.nv;
  if (q.kind == 0) {
    r->o1.resize(n1);
    r->o2.resize(nt2);
    r->e.resize(1);
    rc = cc3_omega_triples(ctx, q.prec, r->o1.data(), r->o2.data(), r->e.data(), st);
  } else {
    r->rho1.resize(n1 * q.nvec);
    r->rho2.resize(nt2 * q.nvec);
    rc = cc3_jacobian_triples(ctx, q.prec, q.nvec, r->omega.data(), r->R1.data(), r->R2.data(),
                              r->rho1.data(), r->rho2.data(), st);
  }
  cc3_counters cnt{};
  cc3_ctx_counters(ctx, &cnt);
  r->nominal = cnt.nominal_flop;
  cc3_ctx_destroy(ctx);
  cudaStreamSynchronize(st);
  return rc;
}

void release_inputs(Req *r) {
  for (auto *v : {&r->eps_o, &r->eps_v, &r->t2, &r->vvvo, &r->ooov, &r->ovov, &r->F, &r->chol,
                  &r->omega, &r->R1, &r->R2}) {
    v->clear();
    v->shrink_to_fit();
  }
}

void worker_main(cc3_server *S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;
  }
  for (;;) {
    Req *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stopping || (r = pick(S)) != nullptr; });
      if (!r) break;
      r->state = RUNNING;
      r->t_start = Clock::now();
      S->in_use += r->footprint;
      S->peak = std::max(S->peak, S->in_use);
      S->admitted++;
      if (S->running++ == 0) S->busy_since = r->t_start;
    }
    const int rc = st ? execute(r, st) : CC3_ERR_CUDA;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->t_done = Clock::now();
      r->status = r->cancel ? CC3_ERR_CANCELLED : rc;
      r->state = DONE;
      S->in_use -= r->footprint;
      if (--S->running == 0) S->busy_total += secs(S->busy_since, r->t_done);
      if (r->cancel) {
        S->cancelled++;
      } else {
        S->completed++;
        S->lat_ms.push_back(1e3 * secs(r->t_submit, r->t_done));
        if (rc == CC3_OK) S->nominal += r->nominal;
      }
      release_inputs(r);
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p * (v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int cc3_serve_footprint(const cc3_request *req, size_t *bytes) {
  if (!req || !bytes) return CC3_ERR_ARG;
  const int rc = validate(*req);
  if (rc != CC3_OK) return rc;
  *bytes = request_footprint(*req);
  return CC3_OK;
}

int cc3_serve_start(cc3_server **out, size_t hbm_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 64) return CC3_ERR_ARG;
  *out = nullptr;
  cc3_server *S = new (std::nothrow) cc3_server();
  if (!S) return CC3_ERR_OOM;
  cudaGetDevice(&S->device);
  if (hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      delete S;
      return CC3_FAIL(CC3_ERR_CUDA, "cudaMemGetInfo");
    }
    hbm_budget_bytes = fr / 10 * 9;
  }
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  S->t0 = Clock::now();
  try {
    for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker_main, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stopping = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers) t.join();
    delete S;
    return CC3_ERR_OOM;
  }
  *out = S;
  return CC3_OK;
}

int cc3_serve_submit(cc3_server *S, const cc3_request *req, uint64_t *ticket) {
  if (!S || !req || !ticket) return CC3_ERR_ARG;
  const cc3_request &q = *req;
  int rc = validate(q);
  if (rc != CC3_OK) return rc;
  if (q.prec == CC3_SPLIT_INT8) return CC3_ERR_UNSUPPORTED;
  std::unique_ptr<Req> r(new (std::nothrow) Req());
  if (!r) return CC3_ERR_OOM;
  r->q = q;
  r->footprint = request_footprint(q);
  const size_t no = q.no, nv = q.nv, n = no + nv, nt2 = no * no * nv * nv;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return CC3_ERR_CANCELLED;
    S->submitted++;
    if (r->footprint > S->budget) {
      S->rejected++;
      return CC3_FAIL(CC3_ERR_BUSY, "request footprint exceeds the server's HBM budget");
    }
  }
  try {
    copy_in(r->eps_o, q.eps_o, no);
    copy_in(r->eps_v, q.eps_v, nv);
    copy_in(r->t2, q.t2, nt2);
    copy_in(r->vvvo, q.g_vvvo, nv * nv * nv * no);
    copy_in(r->ooov, q.g_ooov, no * no * no * nv);
    copy_in(r->ovov, q.g_ovov, nt2);
    copy_in(r->F, q.F_ov, no * nv);
    if (q.naux > 0) copy_in(r->chol, q.chol_L, (size_t)q.naux * n * n);
    if (q.kind == 1) {
      copy_in(r->omega, q.omega, (size_t)q.nvec);
      copy_in(r->R1, q.R1, (size_t)q.nvec * no * nv);
      copy_in(r->R2, q.R2, (size_t)q.nvec * nt2);
    }
  } catch (...) {
    return CC3_FAIL(CC3_ERR_OOM, "host copy of the request");
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return CC3_ERR_CANCELLED;
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    *ticket = r->ticket;
    S->pending.push_back(r.get());
    S->reqs.emplace(r->ticket, std::move(r));
  }
  S->cv_work.notify_one();
  return CC3_OK;
}

int cc3_serve_poll(cc3_server *S, uint64_t ticket, int *done) {
  if (!S || !done) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return CC3_ERR_NOT_FOUND;
  *done = it->second->state == DONE;
  return CC3_OK;
}

int cc3_serve_wait(cc3_server *S, uint64_t ticket, double timeout_s) {
  if (!S) return CC3_ERR_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return CC3_ERR_NOT_FOUND;
  Req *r = it->second.get();
  auto ready = [&] { return r->state == DONE; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return CC3_ERR_TIMEOUT;
  }
  const int status = r->status;
  if (status == CC3_OK) {
    const cc3_request &q = r->q;
    if (q.kind == 0) {
      if (q.Omega1) std::memcpy(q.Omega1, r->o1.data(), r->o1.size() * sizeof(double));
      if (q.Omega2) std::memcpy(q.Omega2, r->o2.data(), r->o2.size() * sizeof(double));
      if (q.E_T) *q.E_T = r->e[0];
    } else {
      std::memcpy(q.rho1, r->rho1.data(), r->rho1.size() * sizeof(double));
      std::memcpy(q.rho2, r->rho2.data(), r->rho2.size() * sizeof(double));
    }
  }
  S->reqs.erase(it);
  return status;
}

int cc3_serve_cancel(cc3_server *S, uint64_t ticket) {
  if (!S) return CC3_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return CC3_ERR_NOT_FOUND;
    Req *r = it->second.get();
    if (r->state == PENDING) {
      S->pending.erase(std::find(S->pending.begin(), S->pending.end(), r));
      r->state = DONE;
      r->status = CC3_ERR_CANCELLED;
      r->t_done = Clock::now();
      S->cancelled++;
      release_inputs(r);
    } else if (r->state == RUNNING) {
      r->cancel = true;  // the evaluation finishes; its result is dropped
    }
  }
  S->cv_done.notify_all();
  return CC3_OK;
}

int cc3_serve_stats(cc3_server *S, cc3_stats *out) {
  if (!S || !out) return CC3_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const auto now = Clock::now();
  std::memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->cancelled = S->cancelled;
  out->p50_ms = percentile(S->lat_ms, 0.50);
  out->p99_ms = percentile(S->lat_ms, 0.99);
  double sum = 0.0;
  for (double x : S->lat_ms) sum += x;
  out->mean_ms = S->lat_ms.empty() ? 0.0 : sum / S->lat_ms.size();
  out->busy_s = S->busy_total + (S->running ? secs(S->busy_since, now) : 0.0);
  out->wall_s = secs(S->t0, now);
  out->nominal_flop = S->nominal;
  out->hbm_in_use = S->in_use;
  out->hbm_peak = S->peak;
  return CC3_OK;
}

int cc3_serve_stop(cc3_server *S) {
  if (!S) return CC3_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
    for (Req *r : S->pending) {
      r->state = DONE;
      r->status = CC3_ERR_CANCELLED;
      S->cancelled++;
    }
    S->pending.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto &t : S->workers) t.join();
  delete S;
  return CC3_OK;
}

}  // extern "C"
