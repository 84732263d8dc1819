// Batched probabilities: staging arena, batched click blocks, per-tree finish,
// the precision ladder over a batch, and gbs_torontonian_batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <set>
#include <vector>

#include "gbs_batch_driver.cuh"
#include "gbs_internal.h"

namespace gbs {

gbs_status stage_begin(gbs_ctx* ctx, size_t bytes) {
  bytes = (bytes + 4096 + 255) / 256 * 256;
  if (bytes > ctx->stage_cap) {
    gbs_status st;
    if ((st = stream_sync(ctx))) return st;
    size_t cap = std::max(bytes, ctx->stage_cap * 2);
    cap = std::max(cap, (size_t)1 << 20);
    if (ctx->stage_host) cudaFreeHost(ctx->stage_host);
    ctx->stage_host = nullptr;
    ctx->stage_cap = 0;
    if ((st = check_cuda(ctx, cudaMallocHost(&ctx->stage_host, cap), "pinned staging"))) return st;
    dev_free(ctx, ctx->stage_dev);
    if ((st = dev_alloc(ctx, ctx->stage_dev, cap))) return st;
    ctx->stage_cap = cap;
  }
  ctx->stage_off = 0;
  return GBS_OK;
}

gbs_status stage(gbs_ctx* ctx, const void* data, size_t bytes, const void** dev) {
  const size_t off = (ctx->stage_off + 255) / 256 * 256;
  if (off + bytes > ctx->stage_cap) return set_error(ctx, GBS_ENOMEM, "staging arena too small for this call");
  unsigned char* h = (unsigned char*)ctx->stage_host + off;
  unsigned char* d = (unsigned char*)ctx->stage_dev.ptr + off;
  if (bytes) memcpy(h, data, bytes);
  ctx->stage_off = off + bytes;
  *dev = d;
  if (!bytes) return GBS_OK;
  return check_cuda(ctx, cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, ctx->stream), "stage copy");
}

const BatchTune& batch_tune_for(gbs_ctx* ctx, int prec, bool real) {
  return ctx->tune[prec < 0 || prec > kPrecLast ? 1 : prec][real ? 1 : 0];
}

// Every value of a tree over n modes of (Sigma^-1)_S fits the fixed-point
// range: Sigma >= I/2 bounds the entries by 2, the pivot determinants lie in
// [1/sigma_max^2, 4] (so the scaled pivot inverses and the products formed with
// them stay below 2^23, inside the entries' 31-bit integer part), each included
// pivot multiplies s by at most sigma_max, and the sums are bounded by
// (1 + sigma_max)^n (inside the 63-bit integer part of s and the sums).
bool fx_ok_inverse(const gbs_state* st, int n) {
  const double sm = st->sigma_max;
  return sm > 0.0 && sm <= 1024.0 && n * std::log2(1.0 + sm) < 60.0;
}
// A tree over a conditioned Sigma' (sampler): Sigma' >= I/2 bounds the pivot
// determinants below by 1/4, so s <= 2^n and the sums <= 3^n; entries and
// determinants are bounded by sigma_max and sigma_max^2.
bool fx_ok_sigma(const gbs_state* st, int n) {
  const double sm = st->sigma_max;
  return sm > 0.0 && sm < 64.0 && n <= 36;
}

// ------------------------------------------------------- click blocks ---
struct ClickReq {
  const cplx<double>* U;      // factor form (or null)
  const double* alpha;
  const double* beta;
  const cplx<double>* Sinv;   // dense form (when U is null)
  long long pair_begin;
  long long root_off;
  int M, N;
  ModeList S;
};

// One warp per (request, mode pair j >= k); writes the packed lower triangle.
__global__ void batch_click_block_kernel(const ClickReq* __restrict__ reqs, int nreq, long long total_pairs,
                                         int real_basis, void* __restrict__ roots) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= total_pairs) return;
  int lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (reqs[mid].pair_begin <= w) lo = mid; else hi = mid - 1;
  }
  const ClickReq& q = reqs[lo];
  const int p = (int)(w - q.pair_begin);
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= p) ++j;
  const int k = p - j * (j + 1) / 2;
  const int M = q.M;
  double ar = 0, ai = 0, br = 0, bi = 0;  // A = (Sigma^-1)_{a_j a_k}, B = (Sigma^-1)_{a_j a^+_k}
  cplx<double> h10{0, 0}, h11{0, 0};
  if (q.U) {
    const cplx<double>* uj = q.U + (long long)q.S.m[j] * M;
    const cplx<double>* uk = q.U + (long long)q.S.m[k] * M;
    for (int l = lane; l < M; l += 32) {
      const cplx<double> x = uj[l], y = uk[l];
      const double pr = x.re * y.re + x.im * y.im, pi = x.im * y.re - x.re * y.im;
      const double qr = x.re * y.re - x.im * y.im, qi = x.re * y.im + x.im * y.re;
      ar = fma(pr, q.alpha[l], ar);
      ai = fma(pi, q.alpha[l], ai);
      br = fma(qr, q.beta[l], br);
      bi = fma(qi, q.beta[l], bi);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      ar += __shfl_down_sync(0xffffffffu, ar, off);
      ai += __shfl_down_sync(0xffffffffu, ai, off);
      br += __shfl_down_sync(0xffffffffu, br, off);
      bi += __shfl_down_sync(0xffffffffu, bi, off);
    }
    h10 = {br, -bi};
    h11 = {ar, -ai};
  } else if (lane == 0) {
    const long long D = 2LL * M;
    const long long rj = q.S.m[j], rk = q.S.m[k];
    const cplx<double> h00 = q.Sinv[rj * D + rk], h01 = q.Sinv[rj * D + rk + M];
    h10 = q.Sinv[(rj + M) * D + rk];
    h11 = q.Sinv[(rj + M) * D + rk + M];
    ar = h00.re; ai = h00.im; br = h01.re; bi = h01.im;
  }
  if (lane != 0) return;
  if (j == k) { ai = 0.0; h11.im = 0.0; }
  const int a0 = 2 * j, b0 = 2 * k;
  auto T3 = [](int a, int b) { return a * (a + 1) / 2 + b; };
  if (real_basis) {
    // q^+ h q with q = [[1, i], [1, -i]]/sqrt2, h = [[h00, h01], [h10, h11]]
    double* o = (double*)roots + q.root_off;
    o[T3(a0, b0)] = 0.5 * (ar + br + h10.re + h11.re);
    o[T3(a0 + 1, b0)] = 0.5 * ((ai + bi) - (h10.im + h11.im));
    o[T3(a0 + 1, b0 + 1)] = 0.5 * ((ar - br) - (h10.re - h11.re));
    if (j != k) o[T3(a0, b0 + 1)] = -0.5 * (ai - bi + h10.im - h11.im);
  } else {
    cplx<double>* o = (cplx<double>*)roots + q.root_off;
    o[T3(a0, b0)] = {ar, ai};
    o[T3(a0 + 1, b0)] = h10;
    o[T3(a0 + 1, b0 + 1)] = h11;
    if (j != k) o[T3(a0, b0 + 1)] = {br, bi};
  }
}

// A-priori cancellation estimate of each tree: the ratio sum|t| / |Tor| the
// modes would have if they were independent, prod_j (g_j + 1) / |g_j - 1| with
// g_j = det(P_j)^(-1/2) of the mode's diagonal 2x2 block of the root (exact
// for independent modes; on Haar-random states it lies 0.3 to 17 orders of
// magnitude above the true ratio).  Output: log10 of it per tree (inf when a
// block has g = 1 or is not positive definite).
__global__ void kappa_estimate_kernel(const BatchTree* __restrict__ trees, int ntrees, const void* __restrict__ roots,
                                      int real_basis, double* __restrict__ log10_kappa) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntrees) return;
  const BatchTree tr = trees[t];
  double lk = 0.0;
  for (int j = 0; j < tr.n; ++j) {
    const long long a = (long long)(2 * j) * (2 * j + 1) / 2 + 2 * j;        // tri(2j, 2j)
    const long long b = (long long)(2 * j + 1) * (2 * j + 2) / 2 + 2 * j;    // tri(2j+1, 2j)
    double det;
    if (real_basis) {
      const double* r = (const double*)roots + tr.root_off;
      det = r[a] * r[b + 1] - r[b] * r[b];
    } else {
      const cplx<double>* r = (const cplx<double>*)roots + tr.root_off;
      det = r[a].re * r[b + 1].re - (r[b].re * r[b].re + r[b].im * r[b].im);
    }
    const double g = det > 0.0 ? rsqrt(det) : 0.0;
    lk += det > 0.0 && g != 1.0 ? log10((g + 1.0) / fabs(g - 1.0)) : INFINITY;
  }
  log10_kappa[t] = lk;
}

__global__ void batch_finish_kernel(const TreeOut* __restrict__ outs, const int* __restrict__ status,
                                    const double* __restrict__ logdet, const int* __restrict__ nmodes, double u,
                                    double extra, int ntrees, ProbOut* __restrict__ po) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntrees) return;
  const TreeOut& o = outs[t];
  const td a{o.inc[0], o.inc[1], o.inc[2]};
  const td b{o.exc[0], o.exc[1], o.exc[2]};
  const td tor = a + b;
  const double sc = exp(-0.5 * logdet[t]);
  const td p = tor * sc;
  ProbOut r;
  r.p_hi = p.x0;
  r.p_lo = p.x1 + p.x2;
  r.tor[0] = tor.x0; r.tor[1] = tor.x1; r.tor[2] = tor.x2;
  r.abs_sum = o.abs;
  const double tv = tor.x0 + (tor.x1 + tor.x2);
  r.kappa = tv != 0.0 ? o.abs / fabs(tv) : INFINITY;
  r.err = (4.0 * (nmodes[t] > 0 ? nmodes[t] : 1) + extra) * u * o.abs * sc;
  for (int i = 0; i < 3; ++i) { r.inc[i] = o.inc[i]; r.exc[i] = o.exc[i]; }
  r.status = status[t];
  r.pad = 0;
  po[t] = r;
}

static double unit_roundoff_b(int prec) {
  switch (prec) {
    case GBS_PREC_FP64:
    case GBS_PREC_FP64P: return ldexp(1.0, -53);
    case GBS_PREC_DD: return ldexp(1.0, -102);
    case GBS_PREC_TD: return ldexp(1.0, -152);
    case GBS_PREC_FP32_DIAG: return ldexp(1.0, -24);
    case GBS_PREC_FXN: return ldexp(1.0, -108);
    case GBS_PREC_FX: return ldexp(1.0, -140);
    case GBS_PREC_FXW: return ldexp(1.0, -158);  // the three-double output, not the 2^-192 resolution, limits it
  }
  return 1.0;
}

static gbs_status batch_variant(gbs_ctx* ctx, int prec, bool real, int nt, const BatchTree* tr, const void* roots,
                                TreeOut* outs, int* status) {
  const BatchTune& tu = batch_tune_for(ctx, prec, real);
  switch (prec) {
    case GBS_PREC_FP64: return real ? batch_fp64_real(ctx, nt, tr, roots, outs, status, tu)
                                    : batch_fp64_cplx(ctx, nt, tr, roots, outs, status, tu);
    case GBS_PREC_DD: return real ? batch_dd_real(ctx, nt, tr, roots, outs, status, tu)
                                  : batch_dd_cplx(ctx, nt, tr, roots, outs, status, tu);
    case GBS_PREC_TD: return real ? batch_td_real(ctx, nt, tr, roots, outs, status, tu)
                                  : batch_td_cplx(ctx, nt, tr, roots, outs, status, tu);
    case GBS_PREC_FP32_DIAG: return real ? batch_fp32_real(ctx, nt, tr, roots, outs, status, tu)
                                         : batch_fp32_cplx(ctx, nt, tr, roots, outs, status, tu);
    case GBS_PREC_FX: return real ? batch_fx_real(ctx, nt, tr, roots, outs, status, tu)
                                  : set_error(ctx, GBS_EINVAL, "the fixed-point precision needs the real basis");
    case GBS_PREC_FXW: return real ? batch_fxw_real(ctx, nt, tr, roots, outs, status, tu)
                                   : set_error(ctx, GBS_EINVAL, "the fixed-point precision needs the real basis");
    case GBS_PREC_FXN: return real ? batch_fxn_real(ctx, nt, tr, roots, outs, status, tu)
                                   : set_error(ctx, GBS_EINVAL, "the fixed-point precision needs the real basis");
    case GBS_PREC_FP64P: return real ? batch_fp64p_real(ctx, nt, tr, roots, outs, status, tu)
                                     : set_error(ctx, GBS_EINVAL, "the paired FP64 precision needs the real basis");
  }
  return set_error(ctx, GBS_EINVAL, "unknown precision");
}

gbs_status batch_eval(gbs_ctx* ctx, int prec, bool real, int ntrees, const BatchTree* trees, const void* roots_dev,
                      const double* logdet, ProbOut* host_out) {
  if (ntrees <= 0) return GBS_OK;
  gbs_status st;
  // too large for one plan: the two halves in turn (a tree's result does not depend
  // on the rest of its batch, so the split changes no value)
  auto split = [&]() -> gbs_status {
    const int h = ntrees / 2;
    gbs_status s2 = batch_eval(ctx, prec, real, h, trees, roots_dev, logdet, host_out);
    if (s2) return s2;
    return batch_eval(ctx, prec, real, ntrees - h, trees + h, roots_dev, logdet + h, host_out + h);
  };
  const size_t n = (size_t)ntrees;
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t bytes = r256(n * sizeof(TreeOut)) + r256(n * sizeof(ProbOut)) + r256(n * sizeof(int));
  if ((st = dev_reserve(ctx, ctx->aux_dev, bytes))) return st;
  unsigned char* base = (unsigned char*)ctx->aux_dev.ptr;
  TreeOut* outs = (TreeOut*)base;
  ProbOut* po = (ProbOut*)(base + ((n * sizeof(TreeOut) + 255) / 256) * 256);
  int* status = (int*)((unsigned char*)po + ((n * sizeof(ProbOut) + 255) / 256) * 256);
  std::vector<int> nm(n);
  for (size_t t = 0; t < n; ++t) nm[t] = trees[t].n;
  const void *d_logdet = nullptr, *d_n = nullptr;
  if ((st = stage(ctx, logdet, n * sizeof(double), &d_logdet)) || (st = stage(ctx, nm.data(), n * sizeof(int), &d_n)))
    return st;
  if ((st = check_cuda(ctx, cudaMemsetAsync(status, 0, n * sizeof(int), ctx->stream), "memset"))) return st;
  ctx->batch_split = false;
  if ((st = batch_variant(ctx, prec, real, ntrees, trees, roots_dev, outs, status))) {
    if (st == GBS_ENOMEM && ctx->batch_split) {
      ctx->batch_split = false;
      return split();
    }
    return st;
  }
  batch_finish_kernel<<<(ntrees + 127) / 128, 128, 0, ctx->stream>>>(
      outs, status, (const double*)d_logdet, (const int*)d_n, unit_roundoff_b(prec),
      err_factor(prec, 1) - err_factor(GBS_PREC_TD, 1), ntrees, po);
  count_launch(ctx);
  if ((st = check_cuda(ctx, cudaGetLastError(), "finish"))) return st;
  if ((st = check_cuda(ctx, cudaMemcpyAsync(host_out, po, n * sizeof(ProbOut), cudaMemcpyDeviceToHost, ctx->stream),
                       "readback")) ||
      (st = stream_sync(ctx)))
    return st;
  if (ctx->timing && ctx->leaf_timer.pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->leaf_timer.start, ctx->leaf_timer.stop);
    ctx->leaf_timer.total_ms += ms;
    ctx->leaf_timer.count += 1;
    ctx->leaf_timer.pending = false;
  }
  return GBS_OK;
}

// Click blocks of several (state, modes) requests into ctx->hbuf; fills trees[].
gbs_status batch_click_blocks(gbs_ctx* ctx, int nreq, const gbs_state* const* states, const int* const* modes,
                              const int* N, bool real, std::vector<BatchTree>& trees) {
  std::vector<ClickReq> reqs;
  trees.resize(nreq);
  long long pairs = 0, ent = 0;
  for (int i = 0; i < nreq; ++i) {
    ClickReq q{};
    const gbs_state* st = states[i];
    q.U = st->has_factors ? (const cplx<double>*)st->U.ptr : nullptr;
    q.alpha = (const double*)st->alpha.ptr;
    q.beta = (const double*)st->beta.ptr;
    q.Sinv = (const cplx<double>*)st->Sinv.ptr;
    q.M = st->M;
    q.N = N[i];
    for (int j = 0; j < 32; ++j) q.S.m[j] = j < N[i] ? modes[i][j] : 0;
    q.pair_begin = pairs;
    q.root_off = ent;
    trees[i] = BatchTree{N[i], ent};
    pairs += (long long)N[i] * (N[i] + 1) / 2;
    ent += (long long)N[i] * (2 * N[i] + 1);  // sym(2N)
    if (N[i] > 0) reqs.push_back(q);
  }
  gbs_status st;
  if ((st = dev_reserve(ctx, ctx->hbuf, (size_t)std::max(1LL, ent) * (real ? 8 : 16)))) return st;
  if (reqs.empty()) return GBS_OK;
  const void* d = nullptr;
  if ((st = stage(ctx, reqs.data(), reqs.size() * sizeof(ClickReq), &d))) return st;
  const long long threads = pairs * 32;
  batch_click_block_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(
      (const ClickReq*)d, (int)reqs.size(), pairs, real ? 1 : 0, ctx->hbuf.ptr);
  count_launch(ctx);
  return check_cuda(ctx, cudaGetLastError(), "click blocks");
}

static void fill(gbs_prob* out, const ProbOut& r, int prec, bool real, double logdet) {
  out->p_hi = r.p_hi;
  out->p_lo = r.p_lo;
  for (int i = 0; i < 3; ++i) out->tor[i] = r.tor[i];
  out->abs_sum = r.abs_sum;
  out->kappa = r.kappa;
  out->err_bound = r.err;
  out->logdet_sigma = logdet;
  out->prec_used = prec;
  out->basis_used = real ? GBS_BASIS_REAL : GBS_BASIS_COMPLEX;
  out->status = r.status == kStatusNotPD ? GBS_ENOTPD : r.status == kStatusRange ? GBS_EPRECISION : GBS_OK;
}

// Probabilities of a batch of requests with the precision ladder; out[] per request.
gbs_status probs_batch(gbs_ctx* ctx, int nreq, const gbs_state* const* states, const int* const* modes, const int* N,
                       int prec, int basis, double rel_tol, gbs_prob* out) {
  const bool real = basis != GBS_BASIS_COMPLEX;
  gbs_status st;
  if ((st = stage_begin(ctx, (size_t)nreq * 8192 + (1 << 16)))) return st;
  std::vector<BatchTree> trees;
  if ((st = batch_click_blocks(ctx, nreq, states, modes, N, real, trees))) return st;
  const double tol = rel_tol > 0 ? rel_tol : 1e-10;
  // requests still to evaluate (N == 0 needs no tree: Tor = 1)
  std::vector<int> todo;
  for (int i = 0; i < nreq; ++i) {
    if (N[i] == 0) {
      memset(&out[i], 0, sizeof(gbs_prob));
      out[i].p_hi = exp(-0.5 * states[i]->logdet_sigma);
      out[i].tor[0] = 1.0;
      out[i].abs_sum = 1.0;
      out[i].kappa = 1.0;
      out[i].logdet_sigma = states[i]->logdet_sigma;
      out[i].prec_used = prec == GBS_PREC_AUTO ? GBS_PREC_FP64 : prec;
      out[i].basis_used = real ? GBS_BASIS_REAL : GBS_BASIS_COMPLEX;
    } else {
      todo.push_back(i);
    }
  }
  // AUTO: FP64; then FP64 with the last two levels cancellation-free (real
  // basis) for the requests whose FP64 estimate missed rel_tol by at most
  // kPairReach (the grouping's estimate is 1e1 to 1e3 below FP64's on the
  // states it was measured on); then fixed point (160, then 192 fraction bits) where the
  // state bounds the tree (real basis), then triple-double.  A request moves
  // on while its error estimate misses rel_tol or its fixed-point tree left the
  // range.  The narrow fixed point (128 fraction bits) comes before FX for the
  // requests whose earlier rungs bound |p| away from zero well enough to
  // predict its estimate (FP64's scaled by 2^-55) within rel_tol with a factor
  // 2 of margin; without such a bound a miss would cost ~0.7 of FX on top.
  // Trees of kSkip64 or more modes skip FP64 unless the a-priori cancellation
  // estimate (kappa_estimate_kernel) leaves it within kPairReach of rel_tol:
  // there FP64 almost never certifies and costs ~0.2 of FX for nothing.  The
  // estimate is exact for independent modes but runs up to 17 orders of
  // magnitude high on correlated ones, so smaller trees keep the FP64 rung
  // (cheap, and the bound on |p| it gives admits them to the narrow fixed
  // point); a tree that skipped FP64 goes to the narrow fixed point only when
  // the estimate itself predicts success.  Only trees of kSkip64 or more modes
  // consult the estimate, so it is computed only when the batch holds one, and
  // a request's rungs never depend on what it is batched with.
  constexpr double kPairReach = 1e3;
  constexpr int kSkip64 = 16;
  const int ladder[6] = {GBS_PREC_FP64, GBS_PREC_FP64P, GBS_PREC_FXN, GBS_PREC_FX, GBS_PREC_FXW, GBS_PREC_TD};
  const int steps = prec == GBS_PREC_AUTO ? 6 : 1;
  bool uncertified = false;
  std::vector<double> err64(nreq, INFINITY), p_low(nreq, 0.0);  // FP64 estimate, lower bound on |p|
  std::vector<double> lk(nreq, INFINITY);  // log10 of the a-priori cancellation estimate
  bool need_estimate = false;  // only trees of kSkip64+ modes use it (to skip FP64, and then for FXN)
  for (int i : todo) need_estimate |= N[i] >= kSkip64;
  if (prec == GBS_PREC_AUTO && need_estimate) {
    std::vector<BatchTree> tt(todo.size());
    for (size_t i = 0; i < todo.size(); ++i) tt[i] = trees[todo[i]];
    std::vector<double> est(todo.size(), 0.0);
    const void *d_tt = nullptr, *d_est = nullptr;
    if ((st = stage(ctx, tt.data(), tt.size() * sizeof(BatchTree), &d_tt)) ||
        (st = stage(ctx, est.data(), est.size() * sizeof(double), &d_est)))
      return st;
    kappa_estimate_kernel<<<(unsigned)((todo.size() + 127) / 128), 128, 0, ctx->stream>>>(
        (const BatchTree*)d_tt, (int)todo.size(), ctx->hbuf.ptr, real ? 1 : 0, (double*)d_est);
    count_launch(ctx);
    if ((st = check_cuda(ctx, cudaMemcpyAsync(est.data(), d_est, est.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                              ctx->stream),
                         "kappa estimate")) ||
        (st = stream_sync(ctx)))
      return st;
    for (size_t i = 0; i < todo.size(); ++i) lk[todo[i]] = est[i];
  }
  std::vector<char> ran64(nreq, 0);
  for (int k = 0; k < steps && !todo.empty(); ++k) {
    const int pr = prec == GBS_PREC_AUTO ? ladder[k] : prec;
    std::vector<int> run, next;
    for (int i : todo) {
      const double l4n = std::log10(4.0 * std::max(N[i], 1));
      if (prec == GBS_PREC_AUTO && pr == GBS_PREC_FP64 && N[i] >= kSkip64 &&
          !(l4n - 53.0 * std::log10(2.0) + lk[i] <= std::log10(kPairReach * tol))) {
        next.push_back(i);
        continue;
      }
      if (prec == GBS_PREC_AUTO && pr == GBS_PREC_FP64P &&
          !(real && ran64[i] && out[i].err_bound <= kPairReach * tol * fabs(out[i].p_hi))) {
        next.push_back(i);
        continue;
      }
      if (prec == GBS_PREC_AUTO && pr == GBS_PREC_FXN && !(2.0 * err64[i] * 0x1p-55 <= tol * p_low[i]) &&
          !(N[i] >= kSkip64 && std::log10(2.0) + l4n - 108.0 * std::log10(2.0) + lk[i] <= std::log10(tol))) {
        next.push_back(i);
        continue;
      }
      if (is_fixed_point(pr) && !(real && fx_ok_inverse(states[i], N[i]))) {
        if (prec == GBS_PREC_AUTO) {
          next.push_back(i);
          continue;
        }
        return set_error(ctx, GBS_EPRECISION, "the state does not bound the fixed-point tree (or basis not real)");
      }
      run.push_back(i);
    }
    std::vector<BatchTree> sub(run.size());
    std::vector<double> ld(run.size());
    for (size_t i = 0; i < run.size(); ++i) {
      sub[i] = trees[run[i]];
      ld[i] = states[run[i]]->logdet_sigma;
    }
    std::vector<ProbOut> res(run.size());
    if ((st = batch_eval(ctx, pr, real, (int)run.size(), sub.data(), ctx->hbuf.ptr, ld.data(), res.data())))
      return st;
    for (size_t i = 0; i < run.size(); ++i) {
      fill(&out[run[i]], res[i], pr, real, ld[i]);
      if (prec != GBS_PREC_AUTO) continue;
      if (pr == GBS_PREC_FP64) {
        err64[run[i]] = res[i].err;
        ran64[run[i]] = 1;
      }
      if (res[i].status == 0) p_low[run[i]] = std::max(p_low[run[i]], fabs(res[i].p_hi) - res[i].err);
      const bool missed = res[i].status == 0 && !(res[i].err <= tol * fabs(res[i].p_hi));
      // triple-double (u = 2^-152) cannot improve on a wide fixed-point result
      // (2^-158): such a request stops here, uncertified
      if (missed && pr == GBS_PREC_FXW)
        uncertified = true;
      else if (res[i].status == kStatusRange || missed)
        next.push_back(run[i]);
    }
    std::sort(next.begin(), next.end());
    todo.swap(next);
    if (k == steps - 1 && !todo.empty()) uncertified = true;
  }
  for (int i = 0; i < nreq; ++i) {
    if (out[i].status == GBS_ENOTPD) return set_error(ctx, GBS_ENOTPD, "a pivot block is not positive definite");
    if (out[i].status) return set_error(ctx, out[i].status, "a fixed-point tree left its range");
  }
  if (uncertified) return set_error(ctx, GBS_EPRECISION, "the triple-double error estimate exceeds rel_tol");
  return GBS_OK;
}

}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_autotune(gbs_ctx* ctx, int prec, int basis, int n, int n_trees, char* report,
                                   size_t report_len) {
  if (!ctx || prec < GBS_PREC_FP64 || prec > kPrecLast || n < 6 || n > 28 || n_trees < 1 || n_trees > 64)
    return GBS_EINVAL;
  if (prec >= GBS_PREC_FX && basis == GBS_BASIS_COMPLEX) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  const bool real = basis != GBS_BASIS_COMPLEX;
  // A synthetic well-conditioned positive-definite root (the timing does not
  // depend on the values): identity plus a small symmetric perturbation.
  const int D = 2 * n, ne = D * (D + 1) / 2;
  std::vector<double> root(ne * (real ? 1 : 2), 0.0);
  unsigned long long x = 0x9E3779B97F4A7C15ull;
  for (int a = 0; a < D; ++a)
    for (int b = 0; b <= a; ++b) {
      const int t = a * (a + 1) / 2 + b;
      x ^= x << 13; x ^= x >> 7; x ^= x << 17;
      const double v = (a == b) ? 1.0 : 0.02 * ((double)(x >> 11) * 0x1p-53 - 0.5);
      if (real) root[t] = v; else { root[2 * t] = v; root[2 * t + 1] = (a == b) ? 0.0 : 0.5 * v; }
    }
  gbs_status st;
  // n_trees trees of n, n-1, ... modes (at least 6), all on leading blocks of the one root
  std::vector<BatchTree> trees(n_trees);
  for (int i = 0; i < n_trees; ++i) trees[i] = BatchTree{std::max(6, n - i), 0};
  const std::vector<double> zeros(n_trees, 0.0);
  std::vector<ProbOut> outs(n_trees);
  const BatchTune saved = ctx->tune[prec][real ? 1 : 0];
  BatchTune best = saved;
  double best_ms = 1e30;
  std::string rep = "[";
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int subs[] = {0, 2, 3, 4, 5, 6, 7};
  const int tops[] = {6, 8, 9, 10};
  const int grids[] = {0, 8};
  const long long lts[] = {1LL << 17, 1LL << 19};
  const int mids[] = {0, 4, 5};
  for (int me : mids)
  for (int qd = 0; qd < 2; ++qd)
  for (int se : subs)
    for (int dt : tops)
      for (int gr : grids)
        for (long long lt : lts) {
          BatchTune cand;
          cand.sub_e = se;
          cand.d_top = dt;
          cand.leaf_grid_per_sm = gr;
          cand.level_threads = lt;
          cand.q_drop = qd;
          cand.mid_e = me;
          ctx->tune[prec][real ? 1 : 0] = cand;
          float ms_best = 1e30f;
          for (int rep_i = 0; rep_i < 3; ++rep_i) {
            if ((st = stage_begin(ctx, root.size() * 8 + (1 << 16)))) goto done;
            const void* d = nullptr;
            if ((st = stage(ctx, root.data(), root.size() * 8, &d))) goto done;
            cudaEventRecord(e0, ctx->stream);
            if ((st = batch_eval(ctx, prec, real, n_trees, trees.data(), d, zeros.data(), outs.data()))) goto done;
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep_i > 0 && ms < ms_best) ms_best = ms;  // the first run warms up
          }
          char buf[192];
          snprintf(buf, sizeof buf,
                   "%s{\"sub_e\":%d,\"d_top\":%d,\"grid_per_sm\":%d,\"level_threads\":%lld,\"q_drop\":%d,"
                   "\"mid_e\":%d,\"ms\":%.4f}",
                   rep.size() > 1 ? "," : "", se, dt, gr, lt, qd, me, ms_best);
          rep += buf;
          if (ms_best < best_ms) {
            best_ms = ms_best;
            best = cand;
          }
        }
  st = GBS_OK;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->tune[prec][real ? 1 : 0] = st == GBS_OK ? best : saved;
  if (st == GBS_OK) ctx->tuned[prec][real ? 1 : 0] = true;
  rep += "]";
  if (report && report_len) {
    snprintf(report, report_len, "%s", rep.c_str());
  }
  return st;
}

extern "C" gbs_status gbs_get_tuning(gbs_ctx* ctx, int prec, int basis, int* sub_e, int* d_top, int* grid_per_sm,
                                     long long* level_threads, int* q_drop, int* mid_e) {
  if (!ctx || prec < GBS_PREC_FP64 || prec > kPrecLast) return GBS_EINVAL;
  const BatchTune& t = ctx->tune[prec][basis != GBS_BASIS_COMPLEX ? 1 : 0];
  if (sub_e) *sub_e = t.sub_e;
  if (d_top) *d_top = t.d_top;
  if (grid_per_sm) *grid_per_sm = t.leaf_grid_per_sm;
  if (level_threads) *level_threads = t.level_threads;
  if (q_drop) *q_drop = t.q_drop;
  if (mid_e) *mid_e = t.mid_e;
  return GBS_OK;
}

extern "C" gbs_status gbs_set_tuning(gbs_ctx* ctx, int prec, int basis, int sub_e, int d_top, int grid_per_sm,
                                     long long level_threads, int q_drop, int mid_e) {
  if (!ctx || prec < GBS_PREC_FP64 || prec > kPrecLast || sub_e < 0 || sub_e > 7 ||
      d_top < 0 ||
      d_top > 16 || grid_per_sm < 0 || level_threads < 1 || q_drop < 0 || q_drop > 2 || mid_e < 0 || mid_e > 8)
    return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  BatchTune& t = ctx->tune[prec][basis != GBS_BASIS_COMPLEX ? 1 : 0];
  t.sub_e = sub_e;
  t.d_top = d_top;
  t.leaf_grid_per_sm = grid_per_sm;
  t.level_threads = level_threads;
  t.q_drop = q_drop;
  t.mid_e = mid_e;
  return GBS_OK;
}

extern "C" gbs_status gbs_torontonian_batch(gbs_ctx* ctx, int n_req, const gbs_state* const* states,
                                            const int* modes, const int* N_per, int prec, int basis, double rel_tol,
                                            gbs_prob* out) {
  if (!ctx || n_req < 0 || (n_req > 0 && (!states || !N_per || !out))) return GBS_EINVAL;
  if (prec < GBS_PREC_AUTO || prec > kPrecLast) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  std::vector<const int*> mp(n_req);
  long long off = 0;
  for (int i = 0; i < n_req; ++i) {
    if (!states[i] || states[i]->ctx != ctx) return set_error(ctx, GBS_EINVAL, "state of another context");
    if (N_per[i] < 0 || N_per[i] > 32) return set_error(ctx, GBS_EINVAL, "N must be in [0, 32]");
    if (N_per[i] > 0 && !modes) return set_error(ctx, GBS_EINVAL, "modes is NULL");
    mp[i] = modes ? modes + off : nullptr;
    std::set<int> seen;
    for (int j = 0; j < N_per[i]; ++j) {
      const int m = mp[i][j];
      if (m < 0 || m >= states[i]->M) return set_error(ctx, GBS_EINVAL, "mode out of range");
      if (!seen.insert(m).second) return set_error(ctx, GBS_EINVAL, "repeated mode");
    }
    off += N_per[i];
  }
  if (n_req == 0) return GBS_OK;
  return probs_batch(ctx, n_req, states, mp.data(), N_per, prec, basis, rel_tol, out);
}
