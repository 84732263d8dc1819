// C ABI entry points: context, memory ledger, states, probabilities.
#include <algorithm>
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

gbs_status stream_sync(gbs_ctx* ctx) {
  const gbs_status st = check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
  ctx->gap_since = std::chrono::steady_clock::now();
  ctx->gap_open = true;
  ctx->gap_waits++;
  return st;
}

gbs_status check_cuda(gbs_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return GBS_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return set_error(ctx, GBS_ECUDA, buf);
}

// Give every cached block back to CUDA (cudaFree; they leave in_use with it).
void cache_release(gbs_ctx* ctx) {
  std::lock_guard<std::mutex> g(ctx->cache_mu);
  for (auto& kv : ctx->cache) {
    cudaFree(kv.second);
    ctx->in_use -= kv.first;
  }
  ctx->cache.clear();
  ctx->cached = 0;
}

gbs_status dev_alloc(gbs_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  {
    // reuse a cached block of at least the size and at most twice it
    std::lock_guard<std::mutex> g(ctx->cache_mu);
    auto it = ctx->cache.lower_bound(bytes);
    if (it != ctx->cache.end() && it->first <= 2 * bytes) {
      b.ptr = it->second;
      b.bytes = it->first;
      ctx->cached -= it->first;
      ctx->cache.erase(it);
      return GBS_OK;
    }
  }
  if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget) cache_release(ctx);
  if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget)
    return set_error(ctx, GBS_ENOMEM, "device memory budget of the context exceeded");
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cache_release(ctx);  // CUDA may have been short of memory held in the cache
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return set_error(ctx, GBS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  b.ptr = p;
  b.bytes = bytes;
  ctx->in_use += bytes;
  return GBS_OK;
}

void dev_free(gbs_ctx* ctx, DevBuf& b) {
  if (b.ptr) {
    std::lock_guard<std::mutex> g(ctx->cache_mu);
    if (ctx->cached + b.bytes <= ((size_t)1 << 30)) {  // keep up to 1 GiB of freed blocks
      ctx->cache.emplace(b.bytes, b.ptr);
      ctx->cached += b.bytes;
    } else {
      cudaFree(b.ptr);
      ctx->in_use -= b.bytes;
    }
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

// gbs_batch_api.cu
gbs_status probs_batch(gbs_ctx* ctx, int nreq, const gbs_state* const* states, const int* const* modes, const int* N,
                       int prec, int basis, double rel_tol, gbs_prob* out);

// Smallest and largest eigenvalue of the symmetric D x D matrix whose lower
// triangle is G (row-major): cyclic Jacobi rotations on a host copy.  Returns
// false if they do not converge.
bool sym_eig_range(const double* G, int D, double& lmin, double& lmax) {
  std::vector<double> A((size_t)D * D);
  for (int a = 0; a < D; ++a)
    for (int b = 0; b <= a; ++b) A[(size_t)a * D + b] = A[(size_t)b * D + a] = G[(size_t)a * D + b];
  for (int sweep = 0;; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int a = 0; a < D; ++a) {
      diag += A[(size_t)a * D + a] * A[(size_t)a * D + a];
      for (int b = 0; b < a; ++b) off += A[(size_t)a * D + b] * A[(size_t)a * D + b];
    }
    if (off <= 1e-30 * diag) break;
    if (sweep == 60) return false;
    for (int p = 0; p < D; ++p)
      for (int q = p + 1; q < D; ++q) {
        const double apq = A[(size_t)p * D + q];
        if (apq == 0.0) continue;
        // rotation zeroing A[p][q]: tan of the angle is the smaller root of t^2 + 2 theta t - 1
        const double theta = (A[(size_t)q * D + q] - A[(size_t)p * D + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < D; ++k) {
          const double akp = A[(size_t)k * D + p], akq = A[(size_t)k * D + q];
          A[(size_t)k * D + p] = c * akp - sn * akq;
          A[(size_t)k * D + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < D; ++k) {
          const double apk = A[(size_t)p * D + k], aqk = A[(size_t)q * D + k];
          A[(size_t)p * D + k] = c * apk - sn * aqk;
          A[(size_t)q * D + k] = sn * apk + c * aqk;
        }
      }
  }
  lmin = lmax = A[0];
  for (int a = 1; a < D; ++a) {
    lmin = std::min(lmin, A[(size_t)a * D + a]);
    lmax = std::max(lmax, A[(size_t)a * D + a]);
  }
  return true;
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
  {
    // tree workspace of one batch: a quarter of the device (or half the budget)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      total_b = (size_t)16 << 30;
    }
    ctx->batch_cap_bytes = total_b / 4;
    if (hbm_budget_bytes) ctx->batch_cap_bytes = std::min(ctx->batch_cap_bytes, hbm_budget_bytes / 2);
  }
  // Launch shapes before any autotuning: wider arithmetic makes the redundant
  // prefix elimination of the top kernel dearer, so it stops earlier.
  for (int b = 0; b < 2; ++b) {
    ctx->tune[GBS_PREC_FP64][b].sub_e = 6;
    ctx->tune[GBS_PREC_FP64][b].d_top = 8;
    ctx->tune[GBS_PREC_FP32_DIAG][b].sub_e = 6;
    ctx->tune[GBS_PREC_FP32_DIAG][b].d_top = 8;
    ctx->tune[GBS_PREC_DD][b].sub_e = 6;
    ctx->tune[GBS_PREC_DD][b].d_top = 5;
    ctx->tune[GBS_PREC_TD][b].sub_e = 6;
    ctx->tune[GBS_PREC_TD][b].d_top = 4;
    ctx->tune[GBS_PREC_FX][b].sub_e = 6;
    ctx->tune[GBS_PREC_FX][b].d_top = 6;
    ctx->tune[GBS_PREC_FXW][b].sub_e = 6;
    ctx->tune[GBS_PREC_FXW][b].d_top = 6;
    ctx->tune[GBS_PREC_FP64P][b].sub_e = 6;
    ctx->tune[GBS_PREC_FP64P][b].d_top = 8;
    ctx->tune[GBS_PREC_FXN][b].sub_e = 6;
    ctx->tune[GBS_PREC_FXN][b].d_top = 6;
  }
  *out = ctx;
  return GBS_OK;
}

void gbs_ctx_destroy(gbs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  server_shutdown(ctx);
  cudaStreamSynchronize(ctx->stream);
  DevBuf* bufs[] = {&ctx->lvl[0], &ctx->lvl[1], &ctx->sbuf[0], &ctx->sbuf[1], &ctx->partials,
                    &ctx->out,    &ctx->status, &ctx->hbuf,    &ctx->stage_dev, &ctx->aux_dev};
  for (DevBuf* b : bufs) dev_free(ctx, *b);
  cache_release(ctx);
  if (ctx->leaf_timer.start) {
    cudaEventDestroy(ctx->leaf_timer.start);
    cudaEventDestroy(ctx->leaf_timer.stop);
  }
  if (ctx->host_out) cudaFreeHost(ctx->host_out);
  if (ctx->stage_host) cudaFreeHost(ctx->stage_host);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

gbs_status gbs_ctx_set_stream(gbs_ctx* ctx, void* stream) {
  if (!ctx) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cache_release(ctx);  // cached blocks were last used on the old stream
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

gbs_status gbs_ctx_host_gaps(gbs_ctx* ctx, double* seconds, long long* waits) {
  if (!ctx) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  if (seconds) *seconds = ctx->gap_s;
  if (waits) *waits = ctx->gap_waits;
  ctx->gap_s = 0.0;
  ctx->gap_waits = 0;
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
  DevBuf* bufs[] = {&st->U, &st->r, &st->alpha, &st->beta, &st->V, &st->Sinv, &st->sig_real};
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
      (e = stream_sync(ctx)))
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
  if (prec < GBS_PREC_AUTO || prec > kPrecLast) return set_error(ctx, GBS_EINVAL, "bad precision");
  const int* mp[1] = {modes};
  const int Nv[1] = {N};
  return probs_batch(ctx, 1, &st, mp, Nv, prec, basis, rel_tol, out);
}

gbs_status gbs_subset_sum(gbs_ctx* ctx, int n, const double* G, int basis, int prec, double* inc, double* exc,
                          double* tor, double* abs_sum) {
  if (!ctx || !G || n < 1 || n > 32) return GBS_EINVAL;
  if (prec < GBS_PREC_FP64 || prec > kPrecLast) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  const bool real = basis != GBS_BASIS_COMPLEX;
  if (is_fixed_point(prec)) {
    double lmin = 0.0, lmax = 0.0;
    // entries and their scaled pivot inverses stay below 2^31: eigenvalues in [2^-8, 64]
    if (!real || !sym_eig_range(G, 2 * n, lmin, lmax) || !(lmin >= 0x1p-8 && lmax <= 64.0) ||
        !(n * std::log2(1.0 + 1.0 / lmin) < 60.0))
      return set_error(ctx, GBS_EPRECISION, "gbs_subset_sum: matrix outside the fixed-point range");
  }
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
  if ((e = stage_begin(ctx, packed.size() * 8 + (1 << 16)))) return e;
  const void* G_dev = nullptr;
  if ((e = stage(ctx, packed.data(), packed.size() * 8, &G_dev))) return e;
  const BatchTree tree{n, 0};
  const double zero = 0.0;
  ProbOut r;
  if ((e = batch_eval(ctx, prec, real, 1, &tree, G_dev, &zero, &r))) return e;
  if (r.status == kStatusRange) return set_error(ctx, GBS_EPRECISION, "a fixed-point tree left its range");
  if (r.status) return set_error(ctx, GBS_ENOTPD, "a pivot block is not positive definite");
  for (int i = 0; i < 3; ++i) {
    if (inc) inc[i] = r.inc[i];
    if (exc) exc[i] = r.exc[i];
    if (tor) tor[i] = r.tor[i];
  }
  if (abs_sum) *abs_sum = r.abs_sum;
  return GBS_OK;
}

}  // extern "C"
