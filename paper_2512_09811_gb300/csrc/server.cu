// Serving loop (declared in include/pp.h as pp_server_*): window-solve requests for
// several dots, continuously batched.
//
// Each registered dot keeps host copies of its inputs.  A dot becomes resident (its
// context and window slots on the device) when a request for it is scheduled and its
// estimated device footprint fits the budget next to the resident dots; otherwise the
// least recently used idle dots are evicted first, and when nothing idle can be evicted
// the dot waits.  A pool of worker threads advances resident dots one solver step at a
// time: before every step the dot's queued requests are admitted into free window slots,
// so a request that arrives while others run joins their sigma batches at the next
// iteration, and a finished window leaves at once, freeing its slot.  Different dots run
// on their own streams from different workers, so their work overlaps on the device.
#include "pp_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SrvReq {
  unsigned long long id = 0;
  int dot = 0;
  double omega0 = 0, delta = 0;
  int k = 0;
  double t_submit = 0, t_start = -1, t_done = -1;
  bool done = false;
  int status = PP_OK;
  std::string err;
  WindowResult res;
};

struct SrvDot {
  int o = 0, v = 0, Q = 0, dtype = 0;
  std::vector<double> eps, mu;
  std::vector<unsigned char> B;
  bool has_mu = false;
  pp_ctx *ctx = nullptr;
  WindowBatch *wb = nullptr;
  bool claimed = false;   // a worker is creating, stepping or evicting it
  bool creating = false;  // claimed for creation: its estimate counts against the budget
  size_t est = 0, actual = 0;
  double last_used = 0;
  std::deque<unsigned long long> queue;
  std::vector<unsigned long long> slot_req;
  int active = 0;
};

// Device bytes a resident dot will hold: resident integrals and intermediates, the
// tensor-core plan with the sigma workspace for the largest batch a step can form, and
// the window slots.  Mirrors the allocation rules of the context, the plan and the slots.
size_t estimate_bytes(long long o, long long v, long long Q, const pp_options &opt, int slots) {
  const long long ov = o * v, n = o + v, L = 2 * ov;
  auto pad = [](long long x) { return std::max<long long>(64, (x + 63) / 64 * 64); };
  // FP64 blocks Boo, Bov, Bvv, BooT, GB, Gamma and the small intermediates; the permuted Bvv
  // only in the FP64 form
  long long total = 8 * (Q * (o * o + ov + v * v) + Q * o * o + 3 * Q * ov + 8 * ov + 2 * o * o + 2 * v * v + n);
  if (opt.prec == PP_FP64) total += 8 * Q * v * v;
  const long long rows_max = 2LL * 32 * slots;  // half-vectors of the largest step batch
  if (opt.prec != PP_FP64) {
    const long long ldq = pad(Q), ldT = pad(ov), vp = pad(v), Qp = pad(Q);
    total += 4 * (n + Q * ov + 2 * o * o + 2 * v * v);  // FP32 eps, Bov and pair sums
    total += 4 * (ov * ldq + Q * v * vp + 2 * Q * o * vp + v * v * Qp + o * o * Qp + v * pad(Q * v));
    const long long per_half = 4 * (7 * ov + Q) + 4 * (o * vp + v * pad(o) + o * pad(Q * v) + o * pad(2 * Q * o)) +
                               4 * Q * ldT + 8 * ov * Qp;
    const long long ws = (long long)(opt.workspace_gb * (1LL << 30));
    long long R = std::max<long long>(2, std::min<long long>(ws / std::max<long long>(per_half, 1), 64));
    R = std::min(R & ~1LL, rows_max);
    total += per_half * R + 4 * (64LL << 20);
  } else {
    const long long per_half = 8 * (3 * Q * ov + 2 * Q * o * o + 8 * ov + Q);
    long long R = std::max<long long>(2, std::min<long long>((6LL << 30) / std::max<long long>(per_half, 1), 64));
    R = std::min(R & ~1LL, rows_max);
    total += per_half * R + 2 * (256LL << 20);
  }
  const long long m_max = std::min<long long>(std::min(opt.m_max, 112), L);
  const long long mm = 112 * 112;
  total += slots * (8 * L * (3 * m_max + 3 * 64 + 3 * 32) + 8 * 26 * mm + 3 * 32 * 8 * L) + 8 * 296 * mm;
  return (size_t)total;
}

}  // namespace

struct pp_server {
  size_t budget = 0;
  pp_options opt{};
  int slots = 4;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<std::unique_ptr<SrvDot>> dots;
  std::unordered_map<unsigned long long, std::unique_ptr<SrvReq>> reqs;
  unsigned long long next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::string err;
  pp_server_stats_t st{};
  int running = 0;

  size_t freeing = 0;  // bytes of evicted dots still being freed

  size_t resident_bytes() const {
    size_t n = freeing;
    for (const auto &d : dots)
      if (d->ctx || d->creating) n += std::max(d->est, d->actual);
    return n;
  }
  bool has_work(const SrvDot &d) const { return !d.queue.empty() || d.active > 0; }

  void complete(SrvReq &r, int status, const std::string &msg) {
    r.status = status;
    r.err = msg;
    r.done = true;
    r.t_done = now_ms();
    if (status == PP_OK || status == PP_ENOTCONV) ++st.completed;
    else ++st.failed;
  }

  // drop a resident dot's device state (caller holds the claim, not the lock)
  static void release_device(SrvDot &d) {
    if (d.wb) window_batch_destroy(d.wb);
    d.wb = nullptr;
    if (d.ctx) pp_destroy(d.ctx);
    d.ctx = nullptr;
  }

  void fail_dot(SrvDot &d, int status, const std::string &msg) {
    for (auto &id : d.slot_req)
      if (id) {
        complete(*reqs[id], status, msg);
        id = 0;
      }
    while (!d.queue.empty()) {
      complete(*reqs[d.queue.front()], status, msg);
      d.queue.pop_front();
    }
    d.active = 0;
  }

  void worker() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
      // the dot with work that was served least recently among those that can run now: a
      // resident dot, or one whose footprint fits once idle resident dots are evicted
      SrvDot *d = nullptr;
      {
        size_t evictable = 0;
        bool any_resident = false;
        for (auto &p : dots) {
          any_resident = any_resident || p->ctx || p->creating;
          if (p->ctx && !p->claimed && !has_work(*p)) evictable += std::max(p->est, p->actual);
        }
        const size_t held = resident_bytes();
        for (auto &p : dots) {
          if (p->claimed || !has_work(*p)) continue;
          // resident, or fits once idle dots are evicted, or would be alone on the device then
          const size_t kept = held - std::min(held, evictable);
          const bool can_run = p->ctx || !any_resident || kept + p->est <= budget || kept == freeing;
          if (can_run && (!d || p->last_used < d->last_used)) d = p.get();
        }
      }
      if (!d) {
        cv.wait(lk);
        continue;
      }
      d->claimed = true;  // before the lock is released anywhere below
      if (!d->ctx) {
        // admission by device footprint; evict idle resident dots, least recently used first
        while (resident_bytes() + d->est > budget) {
          SrvDot *victim = nullptr;
          for (auto &p : dots)
            if (p->ctx && !p->claimed && !has_work(*p) && (!victim || p->last_used < victim->last_used))
              victim = p.get();
          if (!victim) break;
          // detach under the lock, free outside it; the bytes count until they are freed
          const size_t vbytes = std::max(victim->est, victim->actual);
          SrvDot detached;
          detached.ctx = victim->ctx;
          detached.wb = victim->wb;
          victim->ctx = nullptr;
          victim->wb = nullptr;
          victim->actual = 0;
          freeing += vbytes;
          lk.unlock();
          release_device(detached);
          lk.lock();
          freeing -= vbytes;
          ++st.ctx_evicted;
        }
        bool any_resident = false;
        for (auto &p : dots) any_resident = any_resident || p->ctx || (p->creating && p.get() != d);
        if (resident_bytes() + d->est > budget && any_resident) {
          d->claimed = false;
          cv.wait(lk);  // wait until a resident dot goes idle or finishes
          continue;
        }
        d->creating = true;
        lk.unlock();
        pp_ctx *ctx = nullptr;
        WindowBatch *wb = nullptr;
        std::string msg;
        pp_status cst = pp_create(d->o, d->v, d->Q, d->eps.data(), d->B.data(), d->dtype,
                                  d->has_mu ? d->mu.data() : nullptr, &opt, &ctx);
        if (cst != PP_OK) {
          msg = pp_last_error(nullptr);
        } else {
          try {
            wb = window_batch_new(ctx, slots, false);
          } catch (const PPError &e) {
            cst = e.st;
            msg = e.msg;
          } catch (...) {
            cst = PP_ECUDA;
            msg = "window slots could not be created";
          }
        }
        lk.lock();
        d->creating = false;
        if (cst != PP_OK) {
          if (ctx) pp_destroy(ctx);
          fail_dot(*d, cst, msg);
          d->claimed = false;
          cv.notify_all();
          continue;
        }
        d->ctx = ctx;
        d->wb = wb;
        d->slot_req.assign(slots, 0);
        ++st.ctx_created;
      }
      // admit queued requests into free slots (continuous batching)
      while (!d->queue.empty()) {
        SrvReq &r = *reqs[d->queue.front()];
        int slot = -1;
        try {
          slot = window_batch_add(d->wb, r.omega0, r.delta, r.k);
        } catch (const PPError &e) {
          complete(r, e.st, e.msg);
          d->queue.pop_front();
          continue;
        }
        if (slot < 0) break;
        d->slot_req[slot] = r.id;
        r.t_start = now_ms();
        d->queue.pop_front();
        ++d->active;
      }
      ++running;
      st.max_concurrent_dots = std::max(st.max_concurrent_dots, running);
      st.max_windows_per_step = std::max(st.max_windows_per_step, d->active);
      ++st.steps;
      lk.unlock();
      int est = PP_OK;
      std::string emsg;
      if (d->active > 0) {
        try {
          window_batch_step(d->wb);
        } catch (const PPError &e) {
          est = e.st;
          emsg = e.msg;
        } catch (...) {
          est = PP_ECUDA;
          emsg = "unexpected error in a solver step";
        }
      }
      const size_t actual = ctx_device_bytes(d->ctx) + window_batch_bytes(d->wb);
      lk.lock();
      --running;
      if (est != PP_OK) {
        for (int s = 0; s < slots; ++s)
          if (d->slot_req[s]) window_batch_release(d->wb, s);
        for (auto &id : d->slot_req)
          if (id) {
            complete(*reqs[id], est, emsg);
            id = 0;
          }
        d->active = 0;
      } else {
        for (int s = 0; s < slots; ++s) {
          if (!d->slot_req[s] || !window_batch_finished(d->wb, s)) continue;
          SrvReq &r = *reqs[d->slot_req[s]];
          r.res = window_batch_take(d->wb, s);
          complete(r, r.res.status, r.res.status == PP_OK ? "" : "window did not converge");
          d->slot_req[s] = 0;
          --d->active;
        }
      }
      d->actual = actual;
      d->last_used = now_ms();
      d->claimed = false;
      cv.notify_all();
    }
  }
};

extern "C" pp_status pp_server_create(size_t hbm_budget, const pp_options *opt, int slots_per_dot, int nworkers,
                                      pp_server **out) {
  if (out) *out = nullptr;
  if (!out || hbm_budget == 0 || slots_per_dot < 1 || slots_per_dot > 16 || nworkers < 0 || nworkers > 16)
    return PP_EINVAL;
  pp_options o;
  if (opt) o = *opt;
  else pp_default_options(&o);
  if (o.cuda_stream) return PP_EINVAL;  // every dot gets its own stream
  if (!(o.workspace_gb > 0)) o.workspace_gb = 12.0;  // a fixed share per dot: the budget is per dot
  pp_server *S = new (std::nothrow) pp_server();
  if (!S) return PP_ENOMEM;
  S->budget = hbm_budget;
  S->opt = o;
  S->slots = slots_per_dot;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return PP_ECUDA;
  }
  const int nw = nworkers > 0 ? nworkers : 4;
  for (int w = 0; w < nw; ++w) S->workers.emplace_back([S] { S->worker(); });
  *out = S;
  return PP_OK;
}

extern "C" pp_status pp_server_add_dot(pp_server *S, int nocc, int nvir, int naux, const double *eps,
                                       const void *B, int B_dtype, const double *mu, int *dot_id) {
  if (!S || !dot_id || !eps || (!B && naux > 0) || nocc < 1 || nvir < 1 || naux < 0 ||
      (B_dtype != 0 && B_dtype != 1))
    return PP_EINVAL;
  auto d = std::make_unique<SrvDot>();
  d->o = nocc;
  d->v = nvir;
  d->Q = naux;
  d->dtype = B_dtype;
  const long long n = nocc + nvir;
  d->eps.assign(eps, eps + n);
  const size_t bbytes = (size_t)naux * n * n * (B_dtype == 0 ? sizeof(double) : sizeof(float));
  if (bbytes) {
    d->B.resize(bbytes);
    std::memcpy(d->B.data(), B, bbytes);
  }
  if (mu) {
    d->mu.assign(mu, mu + 3LL * nocc * nvir);
    d->has_mu = true;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  d->est = estimate_bytes(nocc, nvir, naux, S->opt, S->slots);
  // a dot whose footprint alone exceeds the whole budget could never be admitted
  if (d->est > S->budget) {
    S->err = "pp_server_add_dot: estimated device footprint " + std::to_string(d->est) +
             " bytes exceeds the serving budget of " + std::to_string(S->budget) + " bytes";
    return PP_ENOMEM;
  }
  *dot_id = (int)S->dots.size();
  S->dots.push_back(std::move(d));
  return PP_OK;
}

extern "C" pp_status pp_server_submit(pp_server *S, int dot_id, double omega0, double delta, int k,
                                      unsigned long long *req_id) {
  if (!S || !req_id || k < 1 || !(delta >= 0.0) || !std::isfinite(omega0)) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (dot_id < 0 || dot_id >= (int)S->dots.size()) return PP_EINVAL;
  auto r = std::make_unique<SrvReq>();
  r->id = S->next_id++;
  r->dot = dot_id;
  r->omega0 = omega0;
  r->delta = delta;
  r->k = k;
  r->t_submit = now_ms();
  *req_id = r->id;
  S->dots[dot_id]->queue.push_back(r->id);
  S->reqs.emplace(r->id, std::move(r));
  ++S->st.submitted;
  S->cv.notify_all();
  return PP_OK;
}

extern "C" pp_status pp_server_wait(pp_server *S, unsigned long long req_id, int timeout_ms, double *omega,
                                    double *osc, double *resid, int *nfound, double *latency_ms) {
  if (!S || !nfound) return PP_EINVAL;
  *nfound = 0;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(req_id);
  if (it == S->reqs.end()) return PP_EINVAL;
  SrvReq *r = it->second.get();
  if (!r->done) {
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) S->cv.wait(lk, pred);
    else if (!S->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return PP_ETIMEOUT;
  }
  const int nf = (int)r->res.omega.size();
  *nfound = nf;
  for (int t = 0; t < nf; ++t) {
    if (omega) omega[t] = r->res.omega[t];
    if (osc) osc[t] = r->res.osc[t];
    if (resid) resid[t] = r->res.resid[t];
  }
  if (latency_ms) latency_ms[0] = r->t_done - r->t_submit;
  if (latency_ms) latency_ms[1] = r->t_start >= 0 ? r->t_start - r->t_submit : 0.0;
  const int status = r->status;
  S->err = r->err;
  S->reqs.erase(it);
  return (pp_status)status;
}

extern "C" pp_status pp_server_stats(pp_server *S, pp_server_stats_t *out) {
  if (!S || !out) return PP_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  int res = 0;
  for (auto &d : S->dots) res += d->ctx ? 1 : 0;
  out->resident_dots = res;
  out->resident_bytes = (long long)S->resident_bytes();
  return PP_OK;
}

extern "C" const char *pp_server_last_error(const pp_server *S) { return S ? S->err.c_str() : ""; }

extern "C" void pp_server_destroy(pp_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto &t : S->workers) t.join();
  for (auto &d : S->dots) pp_server::release_device(*d);
  delete S;
}
