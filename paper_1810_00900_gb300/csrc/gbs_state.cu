// State construction and Sigma^-1 click blocks.
//
//  - state_params_kernel / build_V_kernel: the covariance of squeezed vacuum
//    followed by an interferometer and loss (paper Sec. II, Eq. 1; inputs as in
//    Sec. III; loss as in Sec. IV):
//        V = S S^+ / 2,  S = [[U ch R, U sh R], [U* sh R, U* ch R]]
//    blockwise A = U diag(cosh 2r) U^+ / 2, B = U diag(sinh 2r) U^T / 2,
//    V = [[A, B], [B*, A*]], then V <- eta V + (1 - eta) I/2.
//  - Closed-form inverse: with E = blockdiag(U, U*) P, P mixing (a_l, a_l^+)
//    into (1, +-1)/sqrt2, Sigma = V + I/2 = E diag(d+, d-) E^+ with
//    d+- = (eta e^{+-2r} + 2 - eta)/2, hence
//        (Sigma^-1)_{a_j a_k}   = sum_l U_jl conj(U_kl) alpha_l
//        (Sigma^-1)_{a_j a^+_k} = sum_l U_jl U_kl beta_l
//    with alpha = (1/d+ + 1/d-)/2, beta = (1/d+ - 1/d-)/2, and
//    log det Sigma = sum_l log(d+ d-).  O(N^2 M) per click block.
//  - States given only by V: Sigma is inverted by Gauss-Jordan elimination
//    (no pivoting; Sigma is Hermitian positive definite), one launch per pivot,
//    ping-pong buffers; log det Sigma is the sum of the logs of the pivots.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gbs_internal.h"
#include "gbs_num.cuh"

namespace gbs {

// packed lower-triangle index of entry (a, b), a >= b
static __host__ __device__ constexpr int tri(int a, int b) { return a * (a + 1) / 2 + b; }

__global__ void state_params_kernel(const double* __restrict__ r, double eta, int M, double* __restrict__ alpha,
                                    double* __restrict__ beta, double* __restrict__ ch2, double* __restrict__ sh2,
                                    double* __restrict__ logd) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= M) return;
  const double e = exp(2.0 * r[l]);
  const double dp = 0.5 * (eta * e + 2.0 - eta);
  const double dm = 0.5 * (eta / e + 2.0 - eta);
  alpha[l] = 0.5 * (1.0 / dp + 1.0 / dm);
  beta[l] = 0.5 * (1.0 / dp - 1.0 / dm);
  ch2[l] = 0.5 * cosh(2.0 * r[l]);
  sh2[l] = 0.5 * sinh(2.0 * r[l]);
  logd[l] = log(dp) + log(dm);
}

// Fixed-order double-double sum of x[0..n) by one block.
__global__ void sum_dd_kernel(const double* __restrict__ x, int n, double* __restrict__ out) {
  // strided per-thread sums, then a fixed-order shuffle tree within each warp
  // and across the (at most 32) warps: deterministic, and no serial loop
  dd acc = dd_make(0.0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = acc + x[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    acc = acc + dd{__shfl_down_sync(0xffffffffu, acc.hi, off), __shfl_down_sync(0xffffffffu, acc.lo, off)};
  __shared__ dd sh[32];
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    dd t = lane < nw ? sh[lane] : dd_make(0.0);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      t = t + dd{__shfl_down_sync(0xffffffffu, t.hi, off), __shfl_down_sync(0xffffffffu, t.lo, off)};
    if (lane == 0) out[0] = t.hi + t.lo;
  }
}

// One thread per (j, k) of the M x M blocks.
__global__ void build_V_kernel(const cplx<double>* __restrict__ U, const double* __restrict__ ch2,
                               const double* __restrict__ sh2, double eta, int M, cplx<double>* __restrict__ V) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)M * M) return;
  const int j = (int)(t / M), k = (int)(t % M);
  double ar = 0, ai = 0, br = 0, bi = 0;
  for (int l = 0; l < M; ++l) {
    const cplx<double> x = U[(long long)j * M + l], y = U[(long long)k * M + l];
    // x conj(y) cosh(2r)/2 and x y sinh(2r)/2
    const double pr = x.re * y.re + x.im * y.im, pi = x.im * y.re - x.re * y.im;
    const double qr = x.re * y.re - x.im * y.im, qi = x.re * y.im + x.im * y.re;
    ar = fma(pr, ch2[l], ar);
    ai = fma(pi, ch2[l], ai);
    br = fma(qr, sh2[l], br);
    bi = fma(qi, sh2[l], bi);
  }
  const double diag = (j == k) ? 0.5 * (1.0 - eta) : 0.0;
  const long long D = 2LL * M;
  V[(long long)j * D + k] = {eta * ar + diag, eta * ai};
  V[(long long)j * D + k + M] = {eta * br, eta * bi};
  V[(long long)(j + M) * D + k] = {eta * br, -eta * bi};
  V[(long long)(j + M) * D + k + M] = {eta * ar + diag, -eta * ai};
}

// Click block from the factors: one warp per mode pair (j >= k).  Output packed
// lower triangle of the 2N x 2N matrix (entry (a, b), a >= b, at tri(a, b)).
__global__ void sigma_inv_block_kernel(const cplx<double>* __restrict__ U, const double* __restrict__ alpha,
                                       const double* __restrict__ beta, int M, ModeList S, int N, int real_basis,
                                       void* __restrict__ out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int npairs = N * (N + 1) / 2;
  if (warp >= npairs) return;
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= warp) ++j;
  const int k = warp - j * (j + 1) / 2;
  const cplx<double>* uj = U + (long long)S.m[j] * M;
  const cplx<double>* uk = U + (long long)S.m[k] * M;
  double ar = 0, ai = 0, br = 0, bi = 0;
  for (int l = lane; l < M; l += 32) {
    const cplx<double> x = uj[l], y = uk[l];
    const double pr = x.re * y.re + x.im * y.im, pi = x.im * y.re - x.re * y.im;
    const double qr = x.re * y.re - x.im * y.im, qi = x.re * y.im + x.im * y.re;
    ar = fma(pr, alpha[l], ar);
    ai = fma(pi, alpha[l], ai);
    br = fma(qr, beta[l], br);
    bi = fma(qi, beta[l], bi);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, off);
    ai += __shfl_down_sync(0xffffffffu, ai, off);
    br += __shfl_down_sync(0xffffffffu, br, off);
    bi += __shfl_down_sync(0xffffffffu, bi, off);
  }
  if (lane != 0) return;
  if (j == k) ai = 0.0;  // A is Hermitian: real diagonal
  const int a0 = 2 * j, b0 = 2 * k;
  if (real_basis) {
    double* o = (double*)out;
    // q^+ [[A, B], [B*, A*]] q with q = [[1, i], [1, -i]]/sqrt2 (columns x, p)
    o[tri(a0, b0)] = ar + br;
    o[tri(a0 + 1, b0)] = ai + bi;
    o[tri(a0 + 1, b0 + 1)] = ar - br;
    if (j != k) o[tri(a0, b0 + 1)] = bi - ai;
  } else {
    cplx<double>* o = (cplx<double>*)out;
    o[tri(a0, b0)] = {ar, ai};
    o[tri(a0 + 1, b0)] = {br, -bi};
    o[tri(a0 + 1, b0 + 1)] = {ar, -ai};
    if (j != k) o[tri(a0, b0 + 1)] = {br, bi};
  }
}

// Click block from a dense Sigma^-1 (block order): one thread per mode pair.
__global__ void gather_inv_block_kernel(const cplx<double>* __restrict__ Si, int M, ModeList S, int N,
                                        int real_basis, void* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N * (N + 1) / 2) return;
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= p) ++j;
  const int k = p - j * (j + 1) / 2;
  const long long D = 2LL * M;
  const int rj = S.m[j], rk = S.m[k];
  cplx<double> h00 = Si[rj * D + rk], h01 = Si[rj * D + rk + M];
  cplx<double> h10 = Si[(rj + M) * D + rk], h11 = Si[(rj + M) * D + rk + M];
  const int a0 = 2 * j, b0 = 2 * k;
  if (real_basis) {
    double* o = (double*)out;
    o[tri(a0, b0)] = 0.5 * (h00.re + h01.re + h10.re + h11.re);
    o[tri(a0 + 1, b0)] = 0.5 * ((h00.im + h01.im) - (h10.im + h11.im));
    o[tri(a0 + 1, b0 + 1)] = 0.5 * ((h00.re - h01.re) - (h10.re - h11.re));
    if (j != k) o[tri(a0, b0 + 1)] = -0.5 * (h00.im - h01.im + h10.im - h11.im);
  } else {
    cplx<double>* o = (cplx<double>*)out;
    if (j == k) { h00.im = 0.0; h11.im = 0.0; }
    o[tri(a0, b0)] = h00;
    o[tri(a0 + 1, b0)] = h10;
    o[tri(a0 + 1, b0 + 1)] = h11;
    if (j != k) o[tri(a0, b0 + 1)] = h01;
  }
}

__global__ void sigma_from_V_kernel(const cplx<double>* __restrict__ V, long long D, cplx<double>* __restrict__ X) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * D) return;
  cplx<double> v = V[t];
  if (t / D == t % D) v.re += 0.5;
  X[t] = v;
}

// One Gauss-Jordan step on pivot k, X -> Y (no pivoting).
__global__ void gauss_jordan_step_kernel(const cplx<double>* __restrict__ X, long long D, int k,
                                         cplx<double>* __restrict__ Y, double* __restrict__ piv,
                                         int* __restrict__ status) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= D * D) return;
  const long long i = t / D, j = t % D;
  const cplx<double> p = X[k * D + k];
  const double pr = p.re;  // Hermitian PD: the pivot is real and positive
  if (!(pr > 0.0)) {
    if (t == 0) atomicExch(status, (int)3);
    return;
  }
  const double ip = 1.0 / pr;
  cplx<double> y;
  if (i == k && j == k) {
    y = {ip, 0.0};
    piv[k] = pr;
  } else if (i == k) {
    const cplx<double> x = X[k * D + j];
    y = {x.re * ip, x.im * ip};
  } else if (j == k) {
    const cplx<double> x = X[i * D + k];
    y = {-x.re * ip, -x.im * ip};
  } else {
    const cplx<double> a = X[i * D + k], b = X[k * D + j], x = X[i * D + j];
    // x - a b / p
    y.re = x.re - (a.re * b.re - a.im * b.im) * ip;
    y.im = x.im - (a.re * b.im + a.im * b.re) * ip;
  }
  Y[t] = y;
}

__global__ void log_kernel(const double* __restrict__ x, int n, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = log(x[i]);
}


// ------------------------------------------------------------ host side --

static gbs_status alloc_state(gbs_ctx* ctx, int M, gbs_state** out) {
  gbs_state* st = new gbs_state();
  st->ctx = ctx;
  st->M = M;
  *out = st;
  return GBS_OK;
}

// The covariance V of a factor-built state, on first use (sampling, V_out).
gbs_status ensure_V(gbs_ctx* ctx, gbs_state* st) {
  if (st->V.ptr) return GBS_OK;
  const int M = st->M;
  const size_t MM = (size_t)M * M;
  DevBuf tmp;
  gbs_status e;
  if ((e = dev_alloc(ctx, st->V, 4 * MM * 16)) || (e = dev_alloc(ctx, tmp, (3 * (size_t)M + 1) * 8))) {
    dev_free(ctx, tmp);
    return e;
  }
  double* ch2 = (double*)tmp.ptr;
  double* sh2 = ch2 + M;
  double* logd = sh2 + M;
  cudaStream_t s = ctx->stream;
  // alpha/beta are already in place: rewrite them with identical values
  state_params_kernel<<<(M + 127) / 128, 128, 0, s>>>((const double*)st->r.ptr, st->eta, M, (double*)st->alpha.ptr,
                                                      (double*)st->beta.ptr, ch2, sh2, logd);
  const long long nt = (long long)M * M;
  build_V_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>((const cplx<double>*)st->U.ptr, ch2, sh2, st->eta, M,
                                                                (cplx<double>*)st->V.ptr);
  count_launch(ctx, 2);
  if ((e = check_cuda(ctx, cudaGetLastError(), "build V")) ||
      (e = stream_sync(ctx))) {
    dev_free(ctx, tmp);
    return e;
  }
  dev_free(ctx, tmp);
  return GBS_OK;
}

gbs_status state_build(gbs_ctx* ctx, int M, const double* U, const double* r, double eta, double* V_out,
                       gbs_state** out) {
  if (M < 1 || !U || !r || !out) return set_error(ctx, GBS_EINVAL, "gbs_build_state: bad arguments");
  if (!(eta > 0.0 && eta <= 1.0)) return set_error(ctx, GBS_EINVAL, "gbs_build_state: eta must be in (0, 1]");
  for (int l = 0; l < M; ++l)
    if (!std::isfinite(r[l])) return set_error(ctx, GBS_EINVAL, "gbs_build_state: non-finite squeezing");
  for (long long i = 0; i < 2LL * M * M; ++i)
    if (!std::isfinite(U[i])) return set_error(ctx, GBS_EINVAL, "gbs_build_state: non-finite U");
  gbs_state* st = nullptr;
  alloc_state(ctx, M, &st);
  st->has_factors = true;
  st->eta = eta;
  // largest eigenvalue of Sigma: max over modes of d+ = (eta e^(2|r|) + 2 - eta) / 2
  for (int l = 0; l < M; ++l)
    st->sigma_max = std::max(st->sigma_max, 0.5 * (eta * std::exp(2.0 * std::fabs(r[l])) + 2.0 - eta));
  const size_t MM = (size_t)M * M;
  DevBuf tmp;
  gbs_status e;
  auto fail = [&](gbs_status code) {
    dev_free(ctx, tmp);
    gbs_state_free(st);
    return code;
  };
  if ((e = dev_alloc(ctx, st->U, MM * 16)) || (e = dev_alloc(ctx, st->r, M * 8)) ||
      (e = dev_alloc(ctx, st->alpha, M * 8)) || (e = dev_alloc(ctx, st->beta, M * 8)) ||
      (e = dev_alloc(ctx, tmp, (3 * (size_t)M + 1) * 8)))
    return fail(e);
  cudaStream_t s = ctx->stream;
  if ((e = check_cuda(ctx, cudaMemcpyAsync(st->U.ptr, U, MM * 16, cudaMemcpyHostToDevice, s), "copy U")) ||
      (e = check_cuda(ctx, cudaMemcpyAsync(st->r.ptr, r, M * 8, cudaMemcpyHostToDevice, s), "copy r")))
    return fail(e);
  double* ch2 = (double*)tmp.ptr;
  double* sh2 = ch2 + M;
  double* logd = sh2 + M;
  double* ld_out = logd + M;
  state_params_kernel<<<(M + 127) / 128, 128, 0, s>>>((const double*)st->r.ptr, eta, M, (double*)st->alpha.ptr,
                                                      (double*)st->beta.ptr, ch2, sh2, logd);
  sum_dd_kernel<<<1, 256, 0, s>>>(logd, M, ld_out);
  count_launch(ctx, 2);
  if ((e = check_cuda(ctx, cudaGetLastError(), "state kernels"))) return fail(e);
  if ((e = check_cuda(ctx, cudaMemcpyAsync(&st->logdet_sigma, ld_out, 8, cudaMemcpyDeviceToHost, s), "copy logdet")))
    return fail(e);
  if ((e = stream_sync(ctx))) return fail(e);
  dev_free(ctx, tmp);
  if (V_out) {
    if ((e = ensure_V(ctx, st))) return fail(e);
    if ((e = check_cuda(ctx, cudaMemcpyAsync(V_out, st->V.ptr, 4 * MM * 16, cudaMemcpyDeviceToHost, s), "copy V")) ||
        (e = stream_sync(ctx)))
      return fail(e);
  }
  *out = st;
  return GBS_OK;
}

gbs_status state_from_V(gbs_ctx* ctx, int M, const double* V, gbs_state** out) {
  if (M < 1 || !V || !out) return set_error(ctx, GBS_EINVAL, "gbs_state_from_V: bad arguments");
  const long long D = 2LL * M;
  for (long long i = 0; i < 2 * D * D; ++i)
    if (!std::isfinite(V[i])) return set_error(ctx, GBS_EINVAL, "gbs_state_from_V: non-finite V");
  gbs_state* st = nullptr;
  alloc_state(ctx, M, &st);
  // Gershgorin bound on the largest eigenvalue of Sigma = V + I/2
  for (long long i = 0; i < D; ++i) {
    double row = 0.5;
    for (long long j = 0; j < D; ++j) row += std::hypot(V[2 * (i * D + j)], V[2 * (i * D + j) + 1]);
    st->sigma_max = std::max(st->sigma_max, row);
  }
  DevBuf X2, piv;
  gbs_status e;
  auto fail = [&](gbs_status code) {
    dev_free(ctx, X2);
    dev_free(ctx, piv);
    gbs_state_free(st);
    return code;
  };
  if ((e = dev_alloc(ctx, st->V, D * D * 16)) || (e = dev_alloc(ctx, st->Sinv, D * D * 16)) ||
      (e = dev_alloc(ctx, X2, D * D * 16)) || (e = dev_alloc(ctx, piv, (2 * D + 2) * 8)) ||
      (e = dev_reserve(ctx, ctx->status, sizeof(int))))
    return fail(e);
  cudaStream_t s = ctx->stream;
  int* status = (int*)ctx->status.ptr;
  if ((e = check_cuda(ctx, cudaMemcpyAsync(st->V.ptr, V, D * D * 16, cudaMemcpyHostToDevice, s), "copy V")) ||
      (e = check_cuda(ctx, cudaMemsetAsync(status, 0, sizeof(int), s), "memset")))
    return fail(e);
  const long long nt = D * D;
  const unsigned nb = (unsigned)((nt + 255) / 256);
  cplx<double>* bufs[2] = {(cplx<double>*)st->Sinv.ptr, (cplx<double>*)X2.ptr};
  sigma_from_V_kernel<<<nb, 256, 0, s>>>((const cplx<double>*)st->V.ptr, D, bufs[0]);
  double* pv = (double*)piv.ptr;
  for (int k = 0; k < D; ++k)
    gauss_jordan_step_kernel<<<nb, 256, 0, s>>>(bufs[k & 1], D, k, bufs[(k + 1) & 1], pv, status);
  // D is even, so the inverse ends in bufs[0] == Sinv.
  log_kernel<<<(unsigned)((D + 255) / 256), 256, 0, s>>>(pv, (int)D, pv + D);
  sum_dd_kernel<<<1, 256, 0, s>>>(pv + D, (int)D, pv + 2 * D);
  count_launch(ctx, D + 3);
  if ((e = check_cuda(ctx, cudaGetLastError(), "gauss-jordan"))) return fail(e);
  int hstatus = 0;
  if ((e = check_cuda(ctx, cudaMemcpyAsync(&st->logdet_sigma, pv + 2 * D, 8, cudaMemcpyDeviceToHost, s), "copy")) ||
      (e = check_cuda(ctx, cudaMemcpyAsync(&hstatus, status, 4, cudaMemcpyDeviceToHost, s), "copy")) ||
      (e = stream_sync(ctx)))
    return fail(e);
  if (hstatus) return fail(set_error(ctx, GBS_ENOTPD, "gbs_state_from_V: Sigma = V + I/2 is not positive definite"));
  dev_free(ctx, X2);
  dev_free(ctx, piv);
  *out = st;
  return GBS_OK;
}

// Enqueue the packed click block (Sigma^-1)_S into dev_out.
gbs_status click_block(gbs_ctx* ctx, const gbs_state* st, const int* modes, int N, int real_basis, void* dev_out) {
  ModeList S;
  for (int i = 0; i < 32; ++i) S.m[i] = i < N ? modes[i] : 0;
  cudaStream_t s = ctx->stream;
  if (st->has_factors) {
    const int npairs = N * (N + 1) / 2;
    const int threads = 32 * npairs;
    sigma_inv_block_kernel<<<(threads + 255) / 256, 256, 0, s>>>(
        (const cplx<double>*)st->U.ptr, (const double*)st->alpha.ptr, (const double*)st->beta.ptr, st->M, S, N,
        real_basis, dev_out);
  } else {
    const int npairs = N * (N + 1) / 2;
    gather_inv_block_kernel<<<(npairs + 127) / 128, 128, 0, s>>>((const cplx<double>*)st->Sinv.ptr, st->M, S, N,
                                                                   real_basis, dev_out);
  }
  count_launch(ctx);
  return check_cuda(ctx, cudaGetLastError(), "click block");
}

}  // namespace gbs
