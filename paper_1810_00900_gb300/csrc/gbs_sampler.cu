// Chain-rule click sampler (the paper's Sec. II update rule, in closed form).
//
// Modes are measured from the last to the first.  Each trajectory keeps its
// own Sigma' = Sigma conditioned on vacuum at every mode that stayed dark so
// far, in the real x/p basis, on the device.  At step k, with clicks S so far:
//
//   D  = sum_{W subset S} (-1)^|W| det(Sigma'_W)^(-1/2)
//   Nn = sum_{W subset S} (-1)^|W| det(Sigma'_{W u k})^(-1/2)
//   p0 = Nn / D   (probability that mode k stays dark)
//
// Both sums come from one subset tree over S u {k} with k last (the batched
// engine): in its sign convention F_inc = (-1)^m Nn and F_exc = (-1)^(m+1) D,
// so p0 = -F_inc / F_exc.  After a dark step only half of that tree is new:
// det Sigma'_{W u k} = det Sigma'_k det (Sigma'|k)_W gives
//   Nn_k = det(Sigma'_k)^(-1/2) (-1)^m Tor_k,  Tor_k = tree over S of Sigma'|k,
// and the next step's D is exactly (-1)^m Tor_k (conditioning on k is the same
// Schur step), so a "half" step evaluates 2^m instead of 2^(m+1) terms.  The
// full tree runs at the first step, after a click and when a step's error
// check asks for a wider precision.  A device kernel draws u from SplitMix64 (output
// 1 + step + 2^20 (attempt + 2^12 sample) of the stream with state `seed`),
// keeps the mode dark iff u < p0 (or applies the forced outcome), and a dark
// mode is conditioned away by the Schur complement
//   Sigma' <- Sigma'_AA - Sigma'_Ak Sigma'_kk^-1 Sigma'_kA
// (the paper's Eq. 4a in Sigma form), a rank-2 update of the active block.
//
// Precision: the cancellation ratio grows with every click, so each
// trajectory's tree runs in the cheapest of FP64 / double-double /
// triple-double whose error bound keeps |delta p0| below 5e-10 (half the 1e-9
// near-tie threshold), predicted from its previous step and verified
// (escalated to a full tree at a wider precision) after the fact.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "gbs_internal.h"
#include "gbs_num.cuh"
#include "gbs_tree.cuh"

namespace gbs {

namespace {

constexpr int kMaxClicks = 31;  // tree size m + 1 <= 32

// Sigma = V + I/2 (complex, block order) -> real x/p basis, full 2M x 2M.
__global__ void sigma_real_kernel(const cplx<double>* __restrict__ V, int M, double* __restrict__ S) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * M) return;
  const int j = (int)(t / M), k = (int)(t % M);
  const long long D = 2LL * M;
  cplx<double> h00 = V[j * D + k], h01 = V[j * D + k + M];
  cplx<double> h10 = V[(j + M) * D + k], h11 = V[(j + M) * D + k + M];
  if (j == k) {
    h00.re += 0.5;
    h11.re += 0.5;
  }
  // q^+ h q with q = [[1, i], [1, -i]]/sqrt2 (columns x, p)
  const long long r0 = 2LL * j, c0 = 2LL * k;
  S[r0 * D + c0] = 0.5 * (h00.re + h01.re + h10.re + h11.re);
  S[(r0 + 1) * D + c0] = 0.5 * ((h00.im + h01.im) - (h10.im + h11.im));
  S[(r0 + 1) * D + c0 + 1] = 0.5 * ((h00.re - h01.re) - (h10.re - h11.re));
  S[r0 * D + c0 + 1] = -0.5 * (h00.im - h01.im + h10.im - h11.im);
}

struct GatherItem {
  const double* sig;
  const int* clicks;
  double* s0;  // half mode: out, det(Sigma'_k)^(-1/2)
  long long root_off;
  int m, k, M, half;
};

// Full mode: root = Sigma'[S u {k}] (k last).  Half mode: root = (Sigma'|k)[S],
// the Schur complement of mode k restricted to the clicked modes.  Packed lower
// triangle, one block per item.
__global__ void gather_kernel(const GatherItem* __restrict__ items, double* __restrict__ roots) {
  const GatherItem it = items[blockIdx.x];
  const int n = it.half ? it.m : it.m + 1, d = 2 * n;
  const long long D = 2LL * it.M;
  const long long rk = 2LL * it.k;
  double q00 = 0, q10 = 0, q11 = 0;
  if (it.half) {
    const double p00 = it.sig[rk * D + rk], p10 = it.sig[(rk + 1) * D + rk], p11 = it.sig[(rk + 1) * D + rk + 1];
    const double det = p00 * p11 - p10 * p10;
    const double inv = 1.0 / det;
    q00 = p11 * inv;
    q10 = -p10 * inv;
    q11 = p00 * inv;
    if (threadIdx.x == 0) *it.s0 = rsqrt(det);
  }
  for (int e = threadIdx.x; e < d * (d + 1) / 2; e += blockDim.x) {
    int a = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while (a * (a + 1) / 2 > e) --a;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    const int b = e - a * (a + 1) / 2;
    const int ma = (a >> 1) < it.m ? it.clicks[a >> 1] : it.k;
    const int mb = (b >> 1) < it.m ? it.clicks[b >> 1] : it.k;
    const long long ra = 2LL * ma + (a & 1), rb = 2LL * mb + (b & 1);
    double x = it.sig[ra * D + rb];
    if (it.half) {
      const double ua0 = it.sig[ra * D + rk], ua1 = it.sig[ra * D + rk + 1];
      const double ub0 = it.sig[rk * D + rb], ub1 = it.sig[(rk + 1) * D + rb];
      const double l0 = fma(ua0, q00, ua1 * q10), l1 = fma(ua0, q10, ua1 * q11);
      x = fma(-l0, ub0, fma(-l1, ub1, x));
    }
    roots[it.root_off + e] = x;
  }
}

struct DecideItem {
  double inc[3], exc[3];  // full: tree sums; half: inc = Tor_k over S, exc unused
  double* sig;            // Sigma' of the trajectory
  int* clicks;
  double* pinv;           // out: scaled inverse of the 2x2 pivot block (3 values)
  double* dcarry;         // in (half) / out: D of the next step, triple-double
  const double* s0;       // half: det(Sigma'_k)^(-1/2)
  unsigned long long seed;
  int m, k, step, sample, attempt, forced, half, M;
};

struct DecideOut {
  double p0;
  int click, near_tie;
};

__device__ __forceinline__ double splitmix_u(unsigned long long seed, unsigned long long n) {
  unsigned long long z = seed + n * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-53;
}

__global__ void decide_kernel(const DecideItem* __restrict__ items, int nitems, DecideOut* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nitems) return;
  const DecideItem it = items[i];
  const int M = it.M;
  const unsigned long long seed = it.seed;
  const double sgn = (it.m & 1) ? -1.0 : 1.0;  // (-1)^m
  // Nn (a) and D (b) in triple-double, then p0 = a/b by two correction steps
  td a, b, xnext;
  if (it.half) {
    const td tor{it.inc[0], it.inc[1], it.inc[2]};
    xnext = tor * sgn;  // (-1)^m Tor_k: D of the next step if k stays dark
    a = xnext * (*it.s0);
    b = td{it.dcarry[0], it.dcarry[1], it.dcarry[2]};
  } else {
    a = td{it.inc[0], it.inc[1], it.inc[2]} * sgn;
    b = td{it.exc[0], it.exc[1], it.exc[2]} * (-sgn);
  }
  const double q0 = a.x0 / b.x0;
  const td r1 = a - b * q0;
  const double q1 = r1.x0 / b.x0;
  const td r2 = r1 - b * q1;
  const double q2 = r2.x0 / b.x0;
  const double p0 = q0 + (q1 + q2);
  int click;
  int near = 0;
  if (it.forced >= 0) {
    click = it.forced;
  } else {
    const unsigned long long n =
        1ull + (unsigned long long)it.step +
        (1ull << 20) * ((unsigned long long)it.attempt + (1ull << 12) * (unsigned long long)it.sample);
    const double u = splitmix_u(seed, n);
    click = !(u < p0);
    near = fabs(u - p0) < 1e-9;
  }
  out[i] = DecideOut{p0, click, near};
  if (click) {
    it.clicks[it.m] = it.k;
  } else {
    // pivot block P = Sigma'[k, k] (2 x 2), its inverse for the conditioning
    const long long D = 2LL * M;
    const long long r = 2LL * it.k;
    const double p00 = it.sig[r * D + r], p10 = it.sig[(r + 1) * D + r], p11 = it.sig[(r + 1) * D + r + 1];
    const double det = p00 * p11 - p10 * p10;
    const double inv = 1.0 / det;
    it.pinv[0] = p11 * inv;   // (P^-1)_00
    it.pinv[1] = -p10 * inv;  // (P^-1)_10
    it.pinv[2] = p00 * inv;   // (P^-1)_11
    // D of the next step = Nn_k / det(P)^(-1/2)
    if (!it.half) xnext = a * sqrt(det);
    it.dcarry[0] = xnext.x0;
    it.dcarry[1] = xnext.x1;
    it.dcarry[2] = xnext.x2;
  }
}

struct CondItem {
  double* sig;
  const int* clicks;
  const double* pinv;
  double* L;       // 2 x A scratch: L row i at L[2i], L[2i+1]
  long long entry_begin;
  int m, k, A, M;  // A = 2k + 2m active rows
};

__device__ __forceinline__ long long active_row(int i, int k, const int* clicks) {
  return i < 2 * k ? (long long)i : 2LL * clicks[(i - 2 * k) >> 1] + ((i - 2 * k) & 1);
}

// L_i = Sigma'[i, k-block] P^-1 for every active row i.
__global__ void cond_L_kernel(const CondItem* __restrict__ items) {
  const CondItem it = items[blockIdx.y];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= it.A) return;
  const long long D = 2LL * it.M;
  const long long ri = active_row(i, it.k, it.clicks);
  const double u0 = it.sig[ri * D + 2LL * it.k], u1 = it.sig[ri * D + 2LL * it.k + 1];
  it.L[2 * i] = fma(u0, it.pinv[0], u1 * it.pinv[1]);
  it.L[2 * i + 1] = fma(u0, it.pinv[1], u1 * it.pinv[2]);
}

// Sigma'[i, j] -= L_i . Sigma'[k-block, j] over the active block.
__global__ void cond_update_kernel(const CondItem* __restrict__ items, int nitems, long long total) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].entry_begin <= t) lo = mid; else hi = mid - 1;
  }
  const CondItem it = items[lo];
  const long long e = t - it.entry_begin;
  const int i = (int)(e / it.A), j = (int)(e % it.A);
  const long long D = 2LL * it.M;
  const long long ri = active_row(i, it.k, it.clicks), rj = active_row(j, it.k, it.clicks);
  const double w0 = it.sig[(2LL * it.k) * D + rj], w1 = it.sig[(2LL * it.k + 1) * D + rj];
  double* x = it.sig + ri * D + rj;
  *x = fma(-it.L[2 * i], w0, fma(-it.L[2 * i + 1], w1, *x));
}

}  // namespace

gbs_status ensure_sigma_real(gbs_ctx* ctx, gbs_state* st) {
  if (st->sig_real.ptr) return GBS_OK;
  const long long M = st->M;
  gbs_status e;
  if ((e = ensure_V(ctx, st))) return e;
  if ((e = dev_alloc(ctx, st->sig_real, (size_t)(4 * M * M) * sizeof(double)))) return e;
  sigma_real_kernel<<<(unsigned)((M * M + 255) / 256), 256, 0, ctx->stream>>>((const cplx<double>*)st->V.ptr,
                                                                              (int)M, (double*)st->sig_real.ptr);
  count_launch(ctx);
  return check_cuda(ctx, cudaGetLastError(), "sigma real");
}

double unit_of(int prec) {
  switch (prec) {
    case GBS_PREC_FP64: return 0x1p-53;
    case GBS_PREC_DD: return 0x1p-102;
    case GBS_PREC_FXN: return 0x1p-108;
    case GBS_PREC_FX: return 0x1p-140;
    case GBS_PREC_FXW: return 0x1p-158;  // limited by the three-double tree output
  }
  return 0x1p-152;
}

namespace {
// Slot of a precision in gbs_sample_stats.trees / tree_seconds.
int stat_slot(int prec) {
  return prec == GBS_PREC_FX ? 3 : prec == GBS_PREC_FXW ? 4 : prec == GBS_PREC_FXN ? 5 : prec - 1;
}
}  // namespace


size_t traj_bytes(int M) {
  return (size_t)4 * M * M * sizeof(double) + 64 * sizeof(int) + 8 * sizeof(double) +
         ((size_t)4 * M + 256) * sizeof(double);
}

void traj_bind(Trajectory& tj, gbs_state* st, unsigned char* mem) {
  tj.st = st;
  tj.M = st->M;
  const size_t sig_bytes = (size_t)4 * tj.M * tj.M * sizeof(double);
  tj.sig = (double*)mem;
  tj.clicks = (int*)(mem + sig_bytes);
  tj.pinv = (double*)(mem + sig_bytes + 64 * sizeof(int));  // [0..2] P^-1, [3] s0
  tj.dcarry = tj.pinv + 4;
  tj.L = tj.pinv + 8;
}

gbs_status traj_start(gbs_ctx* ctx, Trajectory& tj) {
  gbs_status e;
  if ((e = ensure_sigma_real(ctx, tj.st))) return e;
  if ((e = check_cuda(ctx, cudaMemcpyAsync(tj.sig, tj.st->sig_real.ptr, (size_t)4 * tj.M * tj.M * sizeof(double),
                                           cudaMemcpyDeviceToDevice, ctx->stream),
                      "init trajectory")))
    return e;
  tj.step = 0;
  tj.m = 0;
  tj.S.clear();
  tj.kappa_prev = 1.0;
  tj.relD = 0.0;
  tj.need_full = 1;
  tj.state = Trajectory::kRunning;
  if (tj.want_p0) tj.p0.assign(tj.M, 0.0);
  return GBS_OK;
}

namespace {
struct StepTree {
  Trajectory* tj;
  int half;      // 1: tree over S of Sigma'|k; 0: tree over S u {k}
  int n;         // modes of the tree (0 = no tree: Tor = 1)
  int prec;
  long long root_off;
  ProbOut res;
};
}  // namespace

// Advance every running trajectory of `jobs` by one measured mode.  The jobs may
// belong to different states, sizes and step positions; all their trees of a
// given precision run as one batch.  A trajectory that finishes becomes kDone,
// one abandoned by postselection kRejected (the caller restarts or drops it).
gbs_status sampler_advance(gbs_ctx* ctx, const std::vector<Trajectory*>& jobs, int prec, gbs_sample_stats& stt) {
  std::vector<Trajectory*> act;
  for (Trajectory* t : jobs)
    if (t->state == Trajectory::kRunning) act.push_back(t);
  if (act.empty()) return GBS_OK;
  gbs_status e;
  // Bound on |delta p0|: half the near-tie threshold, so that a decision can
  // differ from an exact evaluation only for draws already counted as near ties.
  const double TOL = 5e-10;
  // AUTO ladder: FP64, fixed point with 128, 160 then 192 fraction bits (when
  // the state bounds the tree), triple-double.  The prediction from the
  // previous step keeps a factor 4 of margin for FP64 and 2 for the narrow
  // fixed point (a miss there costs ~0.7 of the next rung); the wider
  // fixed-point trees are cheap enough relative to the next rung that they are
  // tried without margin (the check after the tree escalates it when needed).
  auto pick = [&](const Trajectory* t, double kp, int n) {
    if (prec != GBS_PREC_AUTO) return prec;
    const int ladder[5] = {GBS_PREC_FP64, GBS_PREC_FXN, GBS_PREC_FX, GBS_PREC_FXW, GBS_PREC_TD};
    const double margin[4] = {4.0, 2.0, 1.0, 1.0};
    for (int l = 0; l < 4; ++l) {
      if (is_fixed_point(ladder[l]) && !fx_ok_sigma(t->st, n)) continue;
      if (err_factor(ladder[l], n) * unit_of(ladder[l]) * kp * margin[l] < TOL) return ladder[l];
    }
    return (int)GBS_PREC_TD;
  };
  // The next rung after a failed check; the wide fixed point is the last one
  // where the state allows it (triple-double's bound is looser), so a half
  // tree there is only redone as a full tree in the same precision.
  auto wider = [&](const Trajectory* t, int p, int n) {
    if ((p == GBS_PREC_FP64 || p == GBS_PREC_FXN) && fx_ok_sigma(t->st, n)) return (int)GBS_PREC_FX;
    if ((p == GBS_PREC_FX || p == GBS_PREC_FXW) && fx_ok_sigma(t->st, n)) return (int)GBS_PREC_FXW;
    return (int)GBS_PREC_TD;
  };
  auto last_rung = [&](const StepTree& q) {
    return !q.half && (q.prec == GBS_PREC_TD || q.prec == GBS_PREC_FXW);
  };
  if ((e = stage_begin(ctx, act.size() * (2 * sizeof(GatherItem) + sizeof(DecideItem) + sizeof(CondItem) + 4 * 16384) +
                                (1 << 16))))
    return e;
  std::vector<StepTree> trees(act.size());
  std::vector<size_t> todo(act.size());
  for (size_t i = 0; i < act.size(); ++i) {
    Trajectory* t = act[i];
    StepTree& q = trees[i];
    q.tj = t;
    q.half = t->need_full ? 0 : 1;
    q.n = q.half ? t->m : t->m + 1;
    q.prec = pick(t, t->kappa_prev * (q.half ? 1.5 : 8.0), q.n);
    if (is_fixed_point(q.prec) && !fx_ok_sigma(t->st, q.n))
      return set_error(ctx, GBS_EPRECISION, "sampler: the state does not bound the fixed-point tree");
    todo[i] = i;
  }
  for (int round = 0; round < 4 && !todo.empty(); ++round) {
    std::vector<GatherItem> gi;
    long long ent = 0;
    for (size_t i : todo) {
      StepTree& q = trees[i];
      Trajectory* t = q.tj;
      q.root_off = ent;
      gi.push_back(GatherItem{t->sig, t->clicks, t->pinv + 3, ent, t->m, t->M - 1 - t->step, t->M, q.half});
      const int d = 2 * std::max(q.n, 1);
      ent += (long long)d * (d + 1) / 2;
    }
    if ((e = dev_reserve(ctx, ctx->hbuf, (size_t)ent * sizeof(double)))) return e;
    const void* dgi = nullptr;
    if ((e = stage(ctx, gi.data(), gi.size() * sizeof(GatherItem), &dgi))) return e;
    gather_kernel<<<(unsigned)gi.size(), 128, 0, ctx->stream>>>((const GatherItem*)dgi, (double*)ctx->hbuf.ptr);
    count_launch(ctx);
    for (int pv : {GBS_PREC_FP64, GBS_PREC_DD, GBS_PREC_FXN, GBS_PREC_FX, GBS_PREC_FXW, GBS_PREC_TD}) {
      std::vector<size_t> grp;
      for (size_t i : todo)
        if (trees[i].prec == pv && trees[i].n > 0) grp.push_back(i);
      if (grp.empty()) continue;
      std::vector<BatchTree> sub(grp.size());
      std::vector<double> zero(grp.size(), 0.0);
      for (size_t j = 0; j < grp.size(); ++j) sub[j] = BatchTree{trees[grp[j]].n, trees[grp[j]].root_off};
      std::vector<ProbOut> r(grp.size());
      const auto tb = std::chrono::steady_clock::now();
      if ((e = batch_eval(ctx, pv, true, (int)grp.size(), sub.data(), ctx->hbuf.ptr, zero.data(), r.data())))
        return e;
      stt.tree_seconds[stat_slot(pv)] += std::chrono::duration<double>(std::chrono::steady_clock::now() - tb).count();
      stt.trees[stat_slot(pv)] += (long long)grp.size();
      stt.steps += (long long)grp.size();
      for (size_t j = 0; j < grp.size(); ++j) trees[grp[j]].res = r[j];
    }
    std::vector<size_t> next;
    for (size_t i : todo) {
      StepTree& q = trees[i];
      if (q.n == 0) {  // half step with no clicks yet: Tor = 1 exactly
        memset(&q.res, 0, sizeof(ProbOut));
        q.res.tor[0] = 1.0;
        q.res.abs_sum = 1.0;
      }
      if (q.res.status == kStatusRange && prec == GBS_PREC_AUTO) {  // fixed point out of range: redo in TD
        q.half = 0;
        q.n = q.tj->m + 1;
        q.prec = GBS_PREC_TD;
        next.push_back(i);
        stt.escalations++;
        continue;
      }
      if (q.res.status == kStatusRange)
        return set_error(ctx, GBS_EPRECISION, "sampler: a fixed-point tree left its range");
      if (q.res.status) return set_error(ctx, GBS_ENOTPD, "sampler: a pivot block is not positive definite");
      const double u = unit_of(q.prec), n = err_factor(q.prec, q.n) / 4.0;
      double dp;
      if (q.half) {
        const double tor = fabs(q.res.tor[0]);
        dp = (q.n ? 4.0 * n * u * q.res.abs_sum / std::max(tor, 1e-300) : 0.0) + 2e-16 + q.tj->relD;
      } else {
        const double exc = fabs(q.res.exc[0]), inc = fabs(q.res.inc[0]);
        const double p0 = exc > 0 ? inc / exc : INFINITY;
        dp = 4.0 * n * u * q.res.abs_sum * (1.0 + p0) / std::max(exc, 1e-300);
      }
      if (!(dp < TOL) && (prec != GBS_PREC_AUTO || last_rung(q))) stt.uncertified++;
      if (prec == GBS_PREC_AUTO && !(dp < TOL) && !last_rung(q)) {
        q.half = 0;
        q.n = q.tj->m + 1;
        q.prec = wider(q.tj, q.prec, q.n);
        next.push_back(i);
        stt.escalations++;
      }
    }
    todo.swap(next);
  }
  // ---- decide on the device
  std::vector<DecideItem> di(act.size());
  for (size_t i = 0; i < act.size(); ++i) {
    const StepTree& q = trees[i];
    Trajectory* t = q.tj;
    DecideItem d{};
    for (int c = 0; c < 3; ++c) {
      d.inc[c] = q.half ? q.res.tor[c] : q.res.inc[c];  // half: the whole Torontonian of the tree over S
      d.exc[c] = q.res.exc[c];
    }
    const int k = t->M - 1 - t->step;
    d.sig = t->sig;
    d.clicks = t->clicks;
    d.pinv = t->pinv;
    d.dcarry = t->dcarry;
    d.s0 = t->pinv + 3;
    d.seed = t->seed;
    d.m = t->m;
    d.k = k;
    d.step = t->step;
    d.sample = t->sample;
    d.attempt = t->attempt;
    d.forced = t->forced.empty() ? -1 : (int)t->forced[k];
    d.half = q.half;
    d.M = t->M;
    di[i] = d;
    const double u = unit_of(q.prec), n = err_factor(q.prec, q.n) / 4.0;
    if (q.half) {
      const double tor = fabs(q.res.tor[0]);
      t->kappa_prev = q.res.abs_sum / std::max(tor, 1e-300);
      t->relD = 4.0 * n * u * t->kappa_prev + 2e-16;  // the carried D is (-1)^m Tor_k
    } else {
      const double exc = fabs(q.res.exc[0]), inc = fabs(q.res.inc[0]);
      t->kappa_prev = q.res.abs_sum / std::max(std::min(exc, inc), 1e-300);
      t->relD = 4.0 * n * u * q.res.abs_sum / std::max(inc, 1e-300) + 4e-16;
    }
  }
  const void* ddi = nullptr;
  if ((e = stage(ctx, di.data(), di.size() * sizeof(DecideItem), &ddi))) return e;
  if ((e = dev_reserve(ctx, ctx->out, act.size() * sizeof(DecideOut) + 64))) return e;
  DecideOut* dout = (DecideOut*)ctx->out.ptr;
  decide_kernel<<<(unsigned)((act.size() + 63) / 64), 64, 0, ctx->stream>>>((const DecideItem*)ddi, (int)act.size(),
                                                                            dout);
  count_launch(ctx);
  std::vector<DecideOut> dec(act.size());
  if ((e = check_cuda(ctx, cudaMemcpyAsync(dec.data(), dout, act.size() * sizeof(DecideOut), cudaMemcpyDeviceToHost,
                                           ctx->stream),
                      "decide readback")) ||
      (e = stream_sync(ctx)))
    return e;
  // ---- bookkeeping, postselection, conditioning of the dark modes
  std::vector<CondItem> ci;
  long long entries = 0;
  for (size_t i = 0; i < act.size(); ++i) {
    Trajectory* t = act[i];
    const int k = t->M - 1 - t->step;
    if (t->want_p0) t->p0[t->step] = dec[i].p0;
    stt.near_ties += dec[i].near_tie;
    t->need_full = dec[i].click;
    if (dec[i].click) {
      t->S.push_back(k);
      t->m++;
    }
    const bool free_run = t->forced.empty();
    if ((t->N_post > 0 && free_run && (t->m > t->N_post || t->m + k < t->N_post)) ||
        (free_run && t->m > kMaxClicks)) {
      t->state = Trajectory::kRejected;
      stt.rejections++;
      continue;
    }
    if (!dec[i].click && k > 0) {
      const int A = 2 * k + 2 * t->m;
      ci.push_back(CondItem{t->sig, t->clicks, t->pinv, t->L, entries, t->m, k, A, t->M});
      entries += (long long)A * A;
    }
    t->step++;
    if (k == 0) t->state = Trajectory::kDone;
  }
  if (!ci.empty()) {
    const void* dci = nullptr;
    if ((e = stage(ctx, ci.data(), ci.size() * sizeof(CondItem), &dci))) return e;
    int amax = 0;
    for (const CondItem& c : ci) amax = std::max(amax, c.A);
    dim3 gl((amax + 255) / 256, (unsigned)ci.size());
    cond_L_kernel<<<gl, 256, 0, ctx->stream>>>((const CondItem*)dci);
    cond_update_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, ctx->stream>>>((const CondItem*)dci,
                                                                                   (int)ci.size(), entries);
    count_launch(ctx, 2);
    if ((e = check_cuda(ctx, cudaGetLastError(), "conditioning"))) return e;
  }
  return GBS_OK;
}

}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_sample(gbs_ctx* ctx, const gbs_state* cst, int n_samples, uint64_t seed, int N_post,
                                 int max_attempts, const int* forced_clicks, int prec, uint8_t* patterns,
                                 double* p0_out, gbs_sample_stats* stats) {
  if (!ctx || !cst || !patterns || n_samples < 1) return GBS_EINVAL;
  if (N_post < 0 || N_post > kMaxClicks || (forced_clicks && N_post < 1)) return GBS_EINVAL;
  if (prec != GBS_PREC_AUTO && prec != GBS_PREC_FP64 && prec != GBS_PREC_DD && prec != GBS_PREC_TD &&
      !is_fixed_point(prec))
    return GBS_EINVAL;
  if (max_attempts < 1) max_attempts = 1;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  gbs_state* st = const_cast<gbs_state*>(cst);
  const int M = st->M;
  if (forced_clicks) {
    for (long long i = 0; i < (long long)n_samples * N_post; ++i)
      if (forced_clicks[i] < 0 || forced_clicks[i] >= M) return set_error(ctx, GBS_EINVAL, "forced click out of range");
  }
  const auto t_start = std::chrono::steady_clock::now();
  const int T = n_samples;
  const size_t per = traj_bytes(M);
  DevBuf work;
  gbs_status e;
  if ((e = dev_alloc(ctx, work, per * T))) return e;
  auto fail = [&](gbs_status code) {
    dev_free(ctx, work);
    return code;
  };
  std::vector<Trajectory> tr(T);
  std::vector<Trajectory*> ptrs(T);
  for (int t = 0; t < T; ++t) {
    traj_bind(tr[t], st, (unsigned char*)work.ptr + per * t);
    tr[t].seed = seed;
    tr[t].sample = t;
    tr[t].attempt = 0;
    tr[t].N_post = N_post;
    tr[t].want_p0 = p0_out != nullptr;
    if (forced_clicks) {
      tr[t].forced.assign(M, 0);
      for (int c = 0; c < N_post; ++c) tr[t].forced[forced_clicks[(long long)t * N_post + c]] = 1;
    }
    if ((e = traj_start(ctx, tr[t]))) return fail(e);
    ptrs[t] = &tr[t];
  }
  gbs_sample_stats stt{};
  memset(patterns, 0xFF, (size_t)T * M);
  for (;;) {
    bool any = false;
    for (Trajectory& t : tr) {
      if (t.state == Trajectory::kRejected && t.attempt + 1 < max_attempts) {
        t.attempt++;
        if ((e = traj_start(ctx, t))) return fail(e);
      }
      any |= t.state == Trajectory::kRunning;
    }
    if (!any) break;
    if ((e = sampler_advance(ctx, ptrs, prec, stt))) return fail(e);
  }
  if ((e = stream_sync(ctx))) return fail(e);
  dev_free(ctx, work);
  bool all = true;
  for (int t = 0; t < T; ++t) {
    if (tr[t].state == Trajectory::kDone) {
      uint8_t* row = patterns + (size_t)t * M;
      memset(row, 0, M);
      for (int c : tr[t].S) row[c] = 1;
      if (p0_out) memcpy(p0_out + (size_t)t * M, tr[t].p0.data(), M * sizeof(double));
    } else {
      all = false;
    }
  }
  stt.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  stt.cond_seconds = stt.seconds;
  for (double t : stt.tree_seconds) stt.cond_seconds -= t;
  if (stats) *stats = stt;
  if (!all) return set_error(ctx, GBS_EREJECT, "postselection attempts exhausted for some samples");
  return GBS_OK;
}

// ------------------------------------------------- seed-drawn click positions --
namespace {
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

extern "C" gbs_status gbs_draw_click_positions(int M, int n_clicks, uint64_t seed, int n_samples, int* out) {
  if (M < 1 || n_clicks < 0 || n_clicks > M || n_clicks > kMaxClicks || n_samples < 0 || (!out && n_samples))
    return GBS_EINVAL;
  // stream "clicks" (identifier 6) of the workload seed, then output n = start + 1, start + 2, ...
  const uint64_t s = mix64(seed * kGamma + 6ull * 0xD1B54A32D192ED03ull);
  std::vector<int> perm(M);
  for (int i = 0; i < n_samples; ++i) {
    for (int j = 0; j < M; ++j) perm[j] = j;
    const uint64_t start = (uint64_t)i * (uint64_t)n_clicks;
    for (int c = 0; c < n_clicks; ++c) {
      const double u = (double)(mix64(s + (start + (uint64_t)c + 1ull) * kGamma) >> 11) * 0x1p-53;
      const int j = c + (int)(u * (double)(M - c));
      std::swap(perm[c], perm[j]);
    }
    std::sort(perm.begin(), perm.begin() + n_clicks);
    for (int c = 0; c < n_clicks; ++c) out[(long long)i * n_clicks + c] = perm[c];
  }
  return GBS_OK;
}

extern "C" gbs_status gbs_sample_forced_random(gbs_ctx* ctx, const gbs_state* st, int n_samples, uint64_t seed,
                                               int n_clicks, int prec, uint8_t* patterns, double* p0_out,
                                               gbs_sample_stats* stats) {
  if (!ctx || !st || n_samples < 1 || n_clicks < 1) return GBS_EINVAL;
  std::vector<int> pos((size_t)n_samples * n_clicks);
  gbs_status e = gbs_draw_click_positions(st->M, n_clicks, seed, n_samples, pos.data());
  if (e) return e;
  return gbs_sample(ctx, st, n_samples, seed, n_clicks, 1, pos.data(), prec, patterns, p0_out, stats);
}
