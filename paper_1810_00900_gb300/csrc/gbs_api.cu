// C ABI entry points: context, memory ledger, states, probabilities.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <vector>

#include "gbs_internal.h"
#include "gbs_num.cuh"
#include "gbs_tree.cuh"

namespace gbs {

gbs_status set_error(gbs_ctx* ctx, gbs_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

gbs_status check_cuda(gbs_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GBS_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return set_error(ctx, GBS_ECUDA, buf);
}

gbs_status dev_alloc(gbs_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget)
    return set_error(ctx, GBS_ENOMEM, "device memory budget of the context exceeded");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, GBS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b.ptr = p;
  b.bytes = bytes;
  ctx->in_use += bytes;
  return GBS_OK;
}

void dev_free(gbs_ctx* ctx, DevBuf& b) {
  if (b.ptr) {
    cudaFree(b.ptr);
    ctx->in_use -= b.bytes;
  }
  b.ptr = nullptr;
  b.bytes = 0;
}

gbs_status dev_reserve(gbs_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.ptr && b.bytes >= bytes) return GBS_OK;
  if (b.ptr) {
    // the previous contents are not kept; make sure no queued work still uses them
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, b);
  }
  return dev_alloc(ctx, b, bytes);
}

// p = Tor exp(-logdet/2), kappa, error model; Tor = inc + exc in triple-double.
struct ProbOut {
  double p_hi, p_lo;
  double tor[3];
  double abs_sum, kappa, err;
  double inc[3], exc[3];
  int status;
};

__global__ void finish_kernel(const TreeOut* __restrict__ t, const int* __restrict__ status, double logdet, double u,
                              int n, ProbOut* __restrict__ out) {
  if (threadIdx.x != 0) return;
  const td a{t->inc[0], t->inc[1], t->inc[2]};
  const td b{t->exc[0], t->exc[1], t->exc[2]};
  const td tor = a + b;
  const double sc = exp(-0.5 * logdet);
  const td p = tor * sc;
  out->p_hi = p.x0;
  out->p_lo = p.x1 + p.x2;
  out->tor[0] = tor.x0;
  out->tor[1] = tor.x1;
  out->tor[2] = tor.x2;
  out->abs_sum = t->abs;
  const double tv = tor.x0 + (tor.x1 + tor.x2);
  out->kappa = tv != 0.0 ? t->abs / fabs(tv) : INFINITY;
  out->err = 4.0 * (n > 0 ? n : 1) * u * t->abs * sc;
  for (int i = 0; i < 3; ++i) {
    out->inc[i] = t->inc[i];
    out->exc[i] = t->exc[i];
  }
  out->status = *status;
}

static double unit_roundoff(int prec) {
  switch (prec) {
    case GBS_PREC_FP64: return ldexp(1.0, -53);
    case GBS_PREC_DD: return ldexp(1.0, -102);
    case GBS_PREC_TD: return ldexp(1.0, -152);
    case GBS_PREC_FP32_DIAG: return ldexp(1.0, -24);
  }
  return 1.0;
}

static gbs_status run_variant(gbs_ctx* ctx, int prec, bool real, const void* G, int n, TreeOut* out) {
  switch (prec) {
    case GBS_PREC_FP64: return real ? tree_fp64_real(ctx, G, n, out) : tree_fp64_cplx(ctx, G, n, out);
    case GBS_PREC_DD: return real ? tree_dd_real(ctx, G, n, out) : tree_dd_cplx(ctx, G, n, out);
    case GBS_PREC_TD: return real ? tree_td_real(ctx, G, n, out) : tree_td_cplx(ctx, G, n, out);
    case GBS_PREC_FP32_DIAG: return real ? tree_fp32_real(ctx, G, n, out) : tree_fp32_cplx(ctx, G, n, out);
  }
  return set_error(ctx, GBS_EINVAL, "unknown precision");
}

// Run the tree over the packed root already in ctx->hbuf (n modes) and read back.
static gbs_status eval_tree(gbs_ctx* ctx, int prec, bool real, int n, double logdet, ProbOut* host) {
  gbs_status st;
  if ((st = dev_reserve(ctx, ctx->out, sizeof(TreeOut) + sizeof(ProbOut) + 64))) return st;
  TreeOut* tout = (TreeOut*)ctx->out.ptr;
  ProbOut* pout = (ProbOut*)((char*)ctx->out.ptr + ((sizeof(TreeOut) + 15) / 16) * 16);
  if ((st = run_variant(ctx, prec, real, ctx->hbuf.ptr, n, tout))) return st;
  finish_kernel<<<1, 32, 0, ctx->stream>>>(tout, (const int*)ctx->status.ptr, logdet, unit_roundoff(prec), n, pout);
  count_launch(ctx);
  if ((st = check_cuda(ctx, cudaGetLastError(), "finish"))) return st;
  if ((st = check_cuda(ctx, cudaMemcpyAsync(ctx->host_out, pout, sizeof(ProbOut), cudaMemcpyDeviceToHost, ctx->stream),
                       "readback")))
    return st;
  if ((st = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync"))) return st;
  if (ctx->timing && ctx->leaf_timer.pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->leaf_timer.start, ctx->leaf_timer.stop);
    ctx->leaf_timer.total_ms += ms;
    ctx->leaf_timer.count += 1;
    ctx->leaf_timer.pending = false;
  }
  memcpy(host, ctx->host_out, sizeof(ProbOut));
  if (host->status == kStatusNotPD) return set_error(ctx, GBS_ENOTPD, "a pivot block is not positive definite");
  return GBS_OK;
}

static gbs_status validate_modes(gbs_ctx* ctx, const int* modes, int N, int M) {
  if (N < 0 || N > 32) return set_error(ctx, GBS_EINVAL, "N must be in [0, 32]");
  if (N > 0 && !modes) return set_error(ctx, GBS_EINVAL, "modes is NULL");
  std::set<int> seen;
  for (int i = 0; i < N; ++i) {
    if (modes[i] < 0 || modes[i] >= M) return set_error(ctx, GBS_EINVAL, "mode out of range");
    if (!seen.insert(modes[i]).second) return set_error(ctx, GBS_EINVAL, "repeated mode");
  }
  return GBS_OK;
}

static void fill_prob(gbs_prob* out, const ProbOut& r, int prec, bool real, double logdet) {
  out->p_hi = r.p_hi;
  out->p_lo = r.p_lo;
  for (int i = 0; i < 3; ++i) out->tor[i] = r.tor[i];
  out->abs_sum = r.abs_sum;
  out->kappa = r.kappa;
  out->err_bound = r.err;
  out->logdet_sigma = logdet;
  out->prec_used = prec;
  out->basis_used = real ? GBS_BASIS_REAL : GBS_BASIS_COMPLEX;
}

}  // namespace gbs

using namespace gbs;

extern "C" {

const char* gbs_status_string(gbs_status st) {
  switch (st) {
    case GBS_OK: return "ok";
    case GBS_EINVAL: return "invalid argument";
    case GBS_ENOMEM: return "device memory budget exceeded";
    case GBS_ENOTPD: return "matrix not positive definite";
    case GBS_EPRECISION: return "requested accuracy not certified";
    case GBS_EREJECT: return "postselection attempts exhausted";
    case GBS_ETIMEDOUT: return "timed out";
    case GBS_ECUDA: return "CUDA error";
    case GBS_PENDING: return "pending";
    case GBS_ENOTFOUND: return "unknown ticket";
  }
  return "unknown status";
}

gbs_status gbs_ctx_create(gbs_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return GBS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GBS_EINVAL;
  }
  gbs_ctx* ctx = new gbs_ctx();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  gbs_status st;
  if ((st = check_cuda(ctx, cudaSetDevice(device), "cudaSetDevice")) ||
      (st = check_cuda(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "stream")) ||
      (st = check_cuda(ctx, cudaMallocHost(&ctx->host_out, 4096), "pinned"))) {
    delete ctx;
    return st;
  }
  ctx->own_stream = true;
  cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  *out = ctx;
  return GBS_OK;
}

void gbs_ctx_destroy(gbs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  server_shutdown(ctx);
  cudaStreamSynchronize(ctx->stream);
  DevBuf* bufs[] = {&ctx->lvl[0], &ctx->lvl[1], &ctx->sbuf[0], &ctx->sbuf[1], &ctx->partials,
                    &ctx->out,    &ctx->status, &ctx->hbuf};
  for (DevBuf* b : bufs) dev_free(ctx, *b);
  if (ctx->leaf_timer.start) {
    cudaEventDestroy(ctx->leaf_timer.start);
    cudaEventDestroy(ctx->leaf_timer.stop);
  }
  if (ctx->host_out) cudaFreeHost(ctx->host_out);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

gbs_status gbs_ctx_set_stream(gbs_ctx* ctx, void* stream) {
  if (!ctx) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  ctx->stream = (cudaStream_t)stream;
  ctx->own_stream = false;
  return GBS_OK;
}

const char* gbs_ctx_last_error(const gbs_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }
size_t gbs_ctx_bytes_in_use(const gbs_ctx* ctx) { return ctx ? ctx->in_use.load() : 0; }
long long gbs_ctx_launch_count(const gbs_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

gbs_status gbs_ctx_enable_timing(gbs_ctx* ctx, int enable) {
  if (!ctx) return GBS_EINVAL;
  ctx->timing = enable != 0;
  return GBS_OK;
}

gbs_status gbs_ctx_kernel_time(gbs_ctx* ctx, double* total_ms, long long* launches) {
  if (!ctx) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  if (total_ms) *total_ms = ctx->leaf_timer.total_ms;
  if (launches) *launches = ctx->leaf_timer.count;
  ctx->leaf_timer.total_ms = 0.0;
  ctx->leaf_timer.count = 0;
  return GBS_OK;
}

gbs_status gbs_build_state(gbs_ctx* ctx, int M, const double* U, const double* r, double eta, double* V_out,
                           gbs_state** st) {
  if (!ctx) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  return state_build(ctx, M, U, r, eta, V_out, st);
}

gbs_status gbs_state_from_V(gbs_ctx* ctx, int M, const double* V, gbs_state** st) {
  if (!ctx) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  return state_from_V(ctx, M, V, st);
}

void gbs_state_free(gbs_state* st) {
  if (!st) return;
  gbs_ctx* ctx = st->ctx;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  DevBuf* bufs[] = {&st->U, &st->r, &st->alpha, &st->beta, &st->V, &st->Sinv};
  for (DevBuf* b : bufs) dev_free(ctx, *b);
  delete st;
}

gbs_status gbs_state_info(const gbs_state* st, int* M, double* logdet) {
  if (!st) return GBS_EINVAL;
  if (M) *M = st->M;
  if (logdet) *logdet = st->logdet_sigma;
  return GBS_OK;
}

gbs_status gbs_sigma_inv_block(gbs_ctx* ctx, const gbs_state* st, const int* modes, int N, int basis,
                               double* H_out) {
  if (!ctx || !st || !H_out) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  gbs_status e;
  if ((e = validate_modes(ctx, modes, N, st->M))) return e;
  if (N == 0) return GBS_OK;
  const bool real = basis != GBS_BASIS_COMPLEX;
  const int D = 2 * N, ne = D * (D + 1) / 2;
  const size_t esz = real ? 8 : 16;
  if ((e = dev_reserve(ctx, ctx->hbuf, ne * esz))) return e;
  if ((e = click_block(ctx, st, modes, N, real ? 1 : 0, ctx->hbuf.ptr))) return e;
  std::vector<double> packed(ne * (real ? 1 : 2));
  if ((e = check_cuda(ctx, cudaMemcpyAsync(packed.data(), ctx->hbuf.ptr, ne * esz, cudaMemcpyDeviceToHost, ctx->stream),
                      "readback")) ||
      (e = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync")))
    return e;
  // unpack the lower triangle into the full Hermitian / symmetric matrix
  for (int a = 0; a < D; ++a)
    for (int b = 0; b <= a; ++b) {
      const int t = a * (a + 1) / 2 + b;
      if (real) {
        H_out[a * D + b] = packed[t];
        H_out[b * D + a] = packed[t];
      } else {
        H_out[2 * (a * D + b)] = packed[2 * t];
        H_out[2 * (a * D + b) + 1] = packed[2 * t + 1];
        H_out[2 * (b * D + a)] = packed[2 * t];
        H_out[2 * (b * D + a) + 1] = -packed[2 * t + 1];
      }
    }
  return GBS_OK;
}

gbs_status gbs_torontonian(gbs_ctx* ctx, const gbs_state* st, const int* modes, int N, int prec, int basis,
                           double rel_tol, gbs_prob* out) {
  if (!ctx || !st || !out) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  gbs_status e;
  if ((e = validate_modes(ctx, modes, N, st->M))) return e;
  if (prec < GBS_PREC_AUTO || prec > GBS_PREC_FP32_DIAG) return set_error(ctx, GBS_EINVAL, "bad precision");
  const bool real = basis != GBS_BASIS_COMPLEX;
  const double logdet = st->logdet_sigma;
  if (N == 0) {
    // Only the empty subset: Tor = 1, p = vacuum probability of every mode.
    memset(out, 0, sizeof *out);
    const double p = exp(-0.5 * logdet);
    out->p_hi = p;
    out->tor[0] = 1.0;
    out->abs_sum = 1.0;
    out->kappa = 1.0;
    out->logdet_sigma = logdet;
    out->prec_used = prec == GBS_PREC_AUTO ? GBS_PREC_FP64 : prec;
    out->basis_used = real ? GBS_BASIS_REAL : GBS_BASIS_COMPLEX;
    return GBS_OK;
  }
  const int D = 2 * N, ne = D * (D + 1) / 2;
  if ((e = dev_reserve(ctx, ctx->hbuf, ne * (real ? 8 : 16)))) return e;
  if ((e = click_block(ctx, st, modes, N, real ? 1 : 0, ctx->hbuf.ptr))) return e;
  const double tol = rel_tol > 0 ? rel_tol : 1e-10;
  ProbOut r;
  if (prec != GBS_PREC_AUTO) {
    if ((e = eval_tree(ctx, prec, real, N, logdet, &r))) return e;
    fill_prob(out, r, prec, real, logdet);
    return GBS_OK;
  }
  const int ladder[3] = {GBS_PREC_FP64, GBS_PREC_DD, GBS_PREC_TD};
  for (int i = 0; i < 3; ++i) {
    if ((e = eval_tree(ctx, ladder[i], real, N, logdet, &r))) return e;
    fill_prob(out, r, ladder[i], real, logdet);
    const double p = fabs(r.p_hi);
    if (r.err <= tol * p) return GBS_OK;
  }
  return set_error(ctx, GBS_EPRECISION, "the triple-double error estimate exceeds rel_tol");
}

gbs_status gbs_subset_sum(gbs_ctx* ctx, int n, const double* G, int basis, int prec, double* inc, double* exc,
                          double* tor, double* abs_sum) {
  if (!ctx || !G || n < 1 || n > 32) return GBS_EINVAL;
  if (prec < GBS_PREC_FP64 || prec > GBS_PREC_FP32_DIAG) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  const bool real = basis != GBS_BASIS_COMPLEX;
  const int D = 2 * n, ne = D * (D + 1) / 2;
  std::vector<double> packed(ne * (real ? 1 : 2));
  for (int a = 0; a < D; ++a)
    for (int b = 0; b <= a; ++b) {
      const int t = a * (a + 1) / 2 + b;
      if (real) {
        packed[t] = G[a * D + b];
      } else {
        packed[2 * t] = G[2 * (a * D + b)];
        packed[2 * t + 1] = a == b ? 0.0 : G[2 * (a * D + b) + 1];
      }
    }
  gbs_status e;
  if ((e = dev_reserve(ctx, ctx->hbuf, packed.size() * 8))) return e;
  if ((e = check_cuda(ctx, cudaMemcpyAsync(ctx->hbuf.ptr, packed.data(), packed.size() * 8, cudaMemcpyHostToDevice,
                                           ctx->stream),
                      "copy G")))
    return e;
  ProbOut r;
  if ((e = eval_tree(ctx, prec, real, n, 0.0, &r))) return e;
  for (int i = 0; i < 3; ++i) {
    if (inc) inc[i] = r.inc[i];
    if (exc) exc[i] = r.exc[i];
    if (tor) tor[i] = r.tor[i];
  }
  if (abs_sum) *abs_sum = r.abs_sum;
  return GBS_OK;
}

}  // extern "C"
