// Request loop: continuous batching of probability and sampling requests.
//
// gbs_submit copies a request into a host queue and returns a ticket.  A worker
// thread owned by the context admits queued requests in arrival order while
// their device footprint fits a fixed device arena (the HBM budget of the
// loop): a sampling request needs one trajectory block (its conditioned Sigma,
// 32 M^2 bytes plus a little), a probability request only the shared tree
// workspace.  Every iteration of the loop
//   1. evaluates all newly admitted probability requests as one tree batch, and
//   2. advances every active sampling trajectory by one measured mode, all of
//      their subset trees (of whatever state, size and step) in shared batches,
// so requests that arrive while others are on the GPU join at the next step
// and their work shares the same kernel launches.  A finished request frees its
// arena block at once, which admits the next queued one.  gbs_poll waits on a
// condition variable with a caller-given bound.  No device code ever waits on
// the host: the queue is host memory and every wait is a bounded host wait.
//
// Determinism: each tree is reduced on its own in a fixed order and each
// trajectory's precision depends only on its own history, so a request's result
// is bitwise the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gbs_internal.h"

namespace gbs {

gbs_status probs_batch(gbs_ctx* ctx, int nreq, const gbs_state* const* states, const int* const* modes, const int* N,
                       int prec, int basis, double rel_tol, gbs_prob* out);

namespace {

using clock_t_ = std::chrono::steady_clock;

// Longest wait of gbs_poll when the caller passes a negative bound (10 minutes).
constexpr int64_t kPollDefaultUs = 600LL * 1000 * 1000;

// A sampling request runs up to `width` postselection attempts at once, one per
// trajectory slot.  outcome[a] records attempt a (0 unknown, 1 rejected,
// 2 accepted with its clicks); the request's result is the lowest accepted
// attempt once every attempt below it is known to be rejected -- exactly what
// attempts run one after the other give.
struct Req {
  uint64_t ticket = 0;
  gbs_request r{};
  std::vector<int> modes;
  clock_t_::time_point t_submit, t_admit;
  size_t footprint = 0;
  long long arena_off = -1;
  std::vector<Trajectory> slots;
  std::vector<int> slot_attempt;  // attempt running in each slot, -1 = idle
  std::vector<signed char> outcome;
  std::map<int, std::vector<int>> accepted_clicks;
  int next_attempt = 0;
  bool admitted = false, done = false;
  gbs_result res{};
};

// First-fit allocator over the arena's byte range.
struct ArenaAlloc {
  size_t cap = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void reset(size_t c) {
    cap = c;
    free_.clear();
    if (c) free_[0] = c;
  }
  long long take(size_t n) {
    n = (n + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const size_t off = it->first, sz = it->second;
        free_.erase(it);
        if (sz > n) free_[off + n] = sz - n;
        return (long long)off;
      }
    }
    return -1;
  }
  void give(size_t off, size_t n) {
    n = (n + 255) / 256 * 256;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t in_use() const {
    size_t f = 0;
    for (auto& kv : free_) f += kv.second;
    return cap - f;
  }
};

struct Server {
  gbs_ctx* ctx = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::vector<Req*> active;  // admitted sampling requests
  std::unordered_map<uint64_t, Req*> table;
  bool stop = false;
  uint64_t next_ticket = 1;
  DevBuf arena;
  ArenaAlloc alloc;
  int max_active = 64;
  int width = 1;  // postselection attempts run at once per sampling request
  int max_prob_batch = 4096;
  gbs_status fatal = GBS_OK;
  // statistics
  long long submitted = 0, completed = 0, refused = 0;
  std::vector<double> latencies;
  double busy_s = 0.0;
  clock_t_::time_point t_start;
};

int width_of(const Server* sv, const gbs_request& r) {
  return std::max(1, std::min(sv->width, r.max_attempts));
}

size_t footprint_of(const Server* sv, const gbs_request& r) {
  return r.kind == GBS_REQ_SAMPLE ? (size_t)width_of(sv, r) * ((traj_bytes(r.state->M) + 255) / 256 * 256) : 0;
}

// Start attempt `a` of request q in slot k.
gbs_status start_attempt(gbs_ctx* ctx, Req* q, int k, int a) {
  Trajectory& tj = q->slots[k];
  tj.seed = q->r.seed;
  tj.sample = q->r.sample_index;
  tj.attempt = a;
  tj.N_post = q->r.N;
  tj.want_p0 = false;
  q->slot_attempt[k] = a;
  return traj_start(ctx, tj);
}

// Lowest attempt whose outcome is not "rejected": its index and outcome.
int first_open(const Req* q, int* oc) {
  int a = 0;
  while (a < (int)q->outcome.size() && q->outcome[a] == 1) ++a;
  *oc = a < (int)q->outcome.size() ? q->outcome[a] : 1;
  return a;
}

void finish(Server* sv, Req* q, gbs_status st) {
  q->res.status = st;
  q->res.kind = q->r.kind;
  q->res.latency_s = std::chrono::duration<double>(clock_t_::now() - q->t_submit).count();
  q->res.queue_s = std::chrono::duration<double>(q->t_admit - q->t_submit).count();
  q->done = true;
  sv->completed++;
  sv->latencies.push_back(q->res.latency_s);
  if (q->arena_off >= 0) {
    sv->alloc.give((size_t)q->arena_off, q->footprint);
    q->arena_off = -1;
  }
}

void worker_loop(Server* sv) {
  gbs_ctx* ctx = sv->ctx;
  cudaSetDevice(ctx->device);
  for (;;) {
    std::vector<Req*> probs, fresh;
    std::vector<Req*> active;
    bool idle;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      idle = sv->active.empty();
    }
    if (idle) {
      // nothing running: the stream is idle for want of work, not because the
      // host is slow, so that time is no host gap
      std::lock_guard<std::mutex> g(ctx->mu);
      ctx->gap_open = false;
    }
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(20),
                           [&] { return sv->stop || !sv->pending.empty() || !sv->active.empty(); });
      if (sv->stop) return;
      // admission in arrival order while the footprint fits
      while (!sv->pending.empty()) {
        Req* q = sv->pending.front();
        if (q->r.kind == GBS_REQ_PROB) {
          if ((int)probs.size() >= sv->max_prob_batch) break;
          probs.push_back(q);
        } else {
          if ((int)sv->active.size() >= sv->max_active) break;
          const long long off = sv->alloc.take(q->footprint);  // all attempt slots in one block
          if (off < 0) break;  // wait for memory to free up (first in, first out)
          q->arena_off = off;
          sv->active.push_back(q);
          fresh.push_back(q);
        }
        q->admitted = true;
        q->t_admit = clock_t_::now();
        sv->pending.pop_front();
      }
      active = sv->active;
    }
    if (probs.empty() && active.empty()) continue;
    const auto t0 = clock_t_::now();
    std::vector<Req*> finished;
    std::vector<gbs_status> fin_status;
    {
      std::lock_guard<std::mutex> g(ctx->mu);
      // 1. probability requests: one batch per precision request kind
      if (!probs.empty()) {
        std::map<std::pair<int, int>, std::vector<Req*>> groups;
        for (Req* q : probs) groups[{q->r.prec, q->r.basis}].push_back(q);
        for (auto& kv : groups) {
          auto& v = kv.second;
          std::vector<const gbs_state*> sts(v.size());
          std::vector<const int*> mp(v.size());
          std::vector<int> Ns(v.size());
          std::vector<gbs_prob> out(v.size());
          for (size_t i = 0; i < v.size(); ++i) {
            sts[i] = v[i]->r.state;
            mp[i] = v[i]->modes.data();
            Ns[i] = v[i]->r.N;
          }
          gbs_status st = probs_batch(ctx, (int)v.size(), sts.data(), mp.data(), Ns.data(), kv.first.first,
                                      kv.first.second, v[0]->r.rel_tol, out.data());
          for (size_t i = 0; i < v.size(); ++i) {
            v[i]->res.prob = out[i];
            finished.push_back(v[i]);
            const gbs_status rs = (st == GBS_OK || st == GBS_EPRECISION || st == GBS_ENOTPD) ? out[i].status : st;
            fin_status.push_back(rs == GBS_OK && st == GBS_EPRECISION ? GBS_EPRECISION : rs);
          }
        }
      }
      // 2. sampling: start the new ones, advance every running attempt by one mode
      for (Req* q : fresh) {
        const int w = width_of(sv, q->r);
        const size_t stride = (traj_bytes(q->r.state->M) + 255) / 256 * 256;
        q->slots.assign(w, Trajectory());
        q->slot_attempt.assign(w, -1);
        q->outcome.assign(q->r.max_attempts, 0);
        gbs_status st = GBS_OK;
        for (int k = 0; k < w && !st; ++k) {
          traj_bind(q->slots[k], const_cast<gbs_state*>(q->r.state),
                    (unsigned char*)sv->arena.ptr + q->arena_off + k * stride);
          st = start_attempt(ctx, q, k, q->next_attempt++);
        }
        if (st) {
          sv->fatal = st;
          for (auto& tj : q->slots) tj.state = -1;  // failed: completed below with the error
          finished.push_back(q);
          fin_status.push_back(st);
        }
      }
      // one advance per precision setting (requests normally all use AUTO)
      std::map<int, std::vector<Req*>> by_prec;
      for (Req* q : active)
        for (auto& tj : q->slots)
          if (tj.state == Trajectory::kRunning) {
            by_prec[q->r.prec].push_back(q);
            break;
          }
      for (auto& kv : by_prec) {
        std::vector<Trajectory*> tjs;
        for (Req* q : kv.second)
          for (auto& tj : q->slots)
            if (tj.state == Trajectory::kRunning) tjs.push_back(&tj);
        gbs_sample_stats stt{};
        const gbs_status st = sampler_advance(ctx, tjs, kv.first, stt);
        if (st) sv->fatal = st;
        for (Req* q : kv.second) {
          if (st) {
            finished.push_back(q);
            fin_status.push_back(st);
            continue;
          }
          // record the attempts that ended in this step
          for (size_t k = 0; k < q->slots.size(); ++k) {
            Trajectory& tj = q->slots[k];
            const int a = q->slot_attempt[k];
            if (a < 0 || tj.state == Trajectory::kRunning) continue;
            if (tj.state == Trajectory::kDone) {
              q->outcome[a] = 2;
              q->accepted_clicks[a] = tj.S;
            } else {
              q->outcome[a] = 1;
            }
            q->slot_attempt[k] = -1;
          }
          int oc = 0;
          const int a0 = first_open(q, &oc);
          if (a0 == (int)q->outcome.size()) {  // every attempt rejected
            q->res.attempts = a0;
            finished.push_back(q);
            fin_status.push_back(GBS_EREJECT);
            continue;
          }
          if (oc == 2) {  // the lowest attempt not rejected was accepted
            const std::vector<int>& S = q->accepted_clicks[a0];
            q->res.n_clicks = (int)S.size();
            for (int c = 0; c < (int)S.size() && c < 64; ++c) q->res.clicks[c] = S[c];
            q->res.attempts = a0 + 1;
            finished.push_back(q);
            fin_status.push_back(GBS_OK);
            continue;
          }
          // attempts above an accepted one can no longer matter: stop them
          const int best = q->accepted_clicks.empty() ? (int)q->outcome.size() : q->accepted_clicks.begin()->first;
          gbs_status e2 = GBS_OK;
          for (size_t k = 0; k < q->slots.size() && !e2; ++k) {
            if (q->slot_attempt[k] > best) {
              q->slots[k].state = Trajectory::kRejected;
              q->slot_attempt[k] = -1;
            }
            if (q->slot_attempt[k] < 0 && q->next_attempt < best) e2 = start_attempt(ctx, q, (int)k, q->next_attempt++);
          }
          if (e2) {
            finished.push_back(q);
            fin_status.push_back(e2);
          }
        }
      }
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->busy_s += std::chrono::duration<double>(clock_t_::now() - t0).count();
      for (size_t i = 0; i < finished.size(); ++i) {
        Req* q = finished[i];
        if (q->r.kind == GBS_REQ_SAMPLE)
          sv->active.erase(std::remove(sv->active.begin(), sv->active.end(), q), sv->active.end());
        finish(sv, q, fin_status[i]);
      }
    }
    if (!finished.empty()) sv->cv_done.notify_all();
  }
}

Server* server_of(gbs_ctx* ctx) { return (Server*)ctx->server; }

gbs_status validate(gbs_ctx* ctx, const gbs_request* r, std::vector<int>& modes) {
  if (!r->state || r->state->ctx != ctx) return set_error(ctx, GBS_EINVAL, "request: state of another context");
  if (r->kind == GBS_REQ_PROB) {
    if (r->N < 0 || r->N > 32) return set_error(ctx, GBS_EINVAL, "request: N must be in [0, 32]");
    if (r->N > 0 && !r->modes) return set_error(ctx, GBS_EINVAL, "request: modes is NULL");
    if (r->prec < GBS_PREC_AUTO || r->prec > kPrecLast) return set_error(ctx, GBS_EINVAL, "request: prec");
    modes.assign(r->modes, r->modes + r->N);
    std::vector<int> s = modes;
    std::sort(s.begin(), s.end());
    for (int i = 0; i < r->N; ++i) {
      if (s[i] < 0 || s[i] >= r->state->M) return set_error(ctx, GBS_EINVAL, "request: mode out of range");
      if (i && s[i] == s[i - 1]) return set_error(ctx, GBS_EINVAL, "request: repeated mode");
    }
    return GBS_OK;
  }
  if (r->kind == GBS_REQ_SAMPLE) {
    if (r->N < 0 || r->N > 31) return set_error(ctx, GBS_EINVAL, "request: N_post must be in [0, 31]");
    if (r->max_attempts < 1) return set_error(ctx, GBS_EINVAL, "request: max_attempts must be >= 1");
    if (r->prec != GBS_PREC_AUTO && r->prec != GBS_PREC_FP64 && r->prec != GBS_PREC_DD && r->prec != GBS_PREC_TD &&
        !is_fixed_point(r->prec))
      return set_error(ctx, GBS_EINVAL, "request: prec");
    if (r->sample_index < 0 || r->sample_index >= (1 << 20)) return set_error(ctx, GBS_EINVAL, "request: sample index");
    return GBS_OK;
  }
  return set_error(ctx, GBS_EINVAL, "request: unknown kind");
}

}  // namespace

void server_shutdown(gbs_ctx* ctx) {
  Server* sv = server_of(ctx);
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  sv->cv_done.notify_all();
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, sv->arena);
  }
  for (auto& kv : sv->table) delete kv.second;
  for (Req* q : sv->pending)
    if (!sv->table.count(q->ticket)) delete q;
  delete sv;
  ctx->server = nullptr;
}

}  // namespace gbs

using namespace gbs;

extern "C" {

gbs_status gbs_server_start(gbs_ctx* ctx, size_t arena_bytes, int max_active, int attempt_width) {
  if (!ctx || arena_bytes == 0 || max_active < 1 || attempt_width < 1 || attempt_width > 64) return GBS_EINVAL;
  if (ctx->server) return set_error(ctx, GBS_EINVAL, "request loop already running");
  Server* sv = new Server();
  sv->ctx = ctx;
  sv->max_active = max_active;
  sv->width = attempt_width;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaSetDevice(ctx->device);
    gbs_status e = dev_alloc(ctx, sv->arena, arena_bytes);
    if (e) {
      delete sv;
      return e;
    }
  }
  sv->alloc.reset(arena_bytes);
  sv->t_start = clock_t_::now();
  ctx->server = sv;
  sv->worker = std::thread(worker_loop, sv);
  return GBS_OK;
}

gbs_status gbs_server_stop(gbs_ctx* ctx) {
  if (!ctx) return GBS_EINVAL;
  server_shutdown(ctx);
  return GBS_OK;
}

gbs_status gbs_submit(gbs_ctx* ctx, const gbs_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return GBS_EINVAL;
  Server* sv = server_of(ctx);
  if (!sv) return set_error(ctx, GBS_EINVAL, "request loop not running (gbs_server_start)");
  Req* q = new Req();
  q->r = *req;
  gbs_status e = validate(ctx, req, q->modes);
  if (e) {
    delete q;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->refused++;
    return e;
  }
  q->r.modes = nullptr;
  q->footprint = footprint_of(sv, q->r);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (q->footprint > sv->alloc.cap) {
      sv->refused++;
      delete q;
      return set_error(ctx, GBS_ENOMEM, "request larger than the loop's device arena");
    }
    q->ticket = sv->next_ticket++;
    q->t_submit = clock_t_::now();
    sv->pending.push_back(q);
    sv->table[q->ticket] = q;
    sv->submitted++;
    *ticket = q->ticket;
  }
  sv->cv_work.notify_one();
  return GBS_OK;
}

gbs_status gbs_poll(gbs_ctx* ctx, uint64_t ticket, gbs_result* out, int64_t timeout_us) {
  if (!ctx || !out) return GBS_EINVAL;
  Server* sv = server_of(ctx);
  if (!sv) return GBS_ENOTFOUND;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->table.find(ticket);
  if (it == sv->table.end()) return GBS_ENOTFOUND;
  Req* q = it->second;
  if (!q->done && timeout_us != 0) {
    auto pred = [&] { return q->done || sv->stop; };
    // a negative bound still ends: after kPollDefaultUs the call gives up
    const int64_t us = timeout_us < 0 ? kPollDefaultUs : timeout_us;
    sv->cv_done.wait_for(lk, std::chrono::microseconds(us), pred);
    if (!q->done && timeout_us < 0) return GBS_ETIMEDOUT;
  }
  if (!q->done) return GBS_PENDING;
  *out = q->res;
  sv->table.erase(it);
  delete q;
  return GBS_OK;
}

gbs_status gbs_server_stats_get(gbs_ctx* ctx, gbs_server_stats* out) {
  if (!ctx || !out) return GBS_EINVAL;
  Server* sv = server_of(ctx);
  if (!sv) return GBS_ENOTFOUND;
  std::lock_guard<std::mutex> lk(sv->mu);
  memset(out, 0, sizeof *out);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->refused = sv->refused;
  out->active = (long long)sv->active.size();
  out->queued = (long long)sv->pending.size();
  std::vector<double> l = sv->latencies;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    out->p50_s = pct(0.50);
    out->p99_s = pct(0.99);
    double s = 0;
    for (double x : l) s += x;
    out->mean_s = s / l.size();
  }
  out->busy_s = sv->busy_s;
  out->wall_s = std::chrono::duration<double>(clock_t_::now() - sv->t_start).count();
  out->arena_bytes = sv->alloc.cap;
  out->arena_in_use = sv->alloc.in_use();
  out->last_error = sv->fatal;
  return GBS_OK;
}

}  // extern "C"
