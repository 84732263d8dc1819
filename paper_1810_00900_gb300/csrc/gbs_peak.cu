// Peak microbenchmarks, the roofline denominators of the subset-determinant
// kernels:
//   FP64   independent chains of dependent DFMAs in every thread of a full grid;
//          the FP64 pipe is the only unit it loads.
//   FX     independent chains of dependent 192-bit fixed-point products (the
//          entry type of the FX trees, gbs_fx.cuh): the integer multiply-add
//          and carry work that bounds the fixed-point trees.
#include "gbs_internal.h"
#include "gbs_fx.cuh"

namespace gbs {

template <int ILP>
__global__ void dfma_chain_kernel(double* out, int iters, double a, double b) {
  double x[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) x[i] = threadIdx.x * 1e-9 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < ILP; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < ILP; ++i) s += x[i];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int ILP>
__global__ void fx_product_chain_kernel(uint32_t* out, int iters, uint32_t seed) {
  fx x[ILP], y[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      x[i].w[k] = seed * (threadIdx.x + 7 * i + 13 * k + 1) + blockIdx.x;
      y[i].w[k] = (seed ^ 0x9e3779b9u) * (threadIdx.x + 3 * i + 5 * k + 1);
    }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < ILP; ++i) x[i] = x[i] * y[i];
  }
  uint32_t acc = 0u;
#pragma unroll
  for (int i = 0; i < ILP; ++i)
#pragma unroll
    for (int k = 0; k < 6; ++k) acc ^= x[i].w[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace gbs

using namespace gbs;

extern "C" gbs_status gbs_measure_fx_peak(gbs_ctx* ctx, double* products_per_s) {
  if (!ctx || !products_per_s) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  // 16 warps per SM, four independent product chains per thread
  const int threads = 128, blocks = 4 * ctx->sm_count, iters = 2048;
  constexpr int ILP = 4;
  DevBuf buf;
  gbs_status st;
  if ((st = dev_alloc(ctx, buf, (size_t)threads * blocks * sizeof(uint32_t)))) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    fx_product_chain_kernel<ILP><<<blocks, threads, 0, ctx->stream>>>((uint32_t*)buf.ptr, iters, 12345u + rep);
    cudaEventRecord(e1, ctx->stream);
    count_launch(ctx);
    if ((st = check_cuda(ctx, cudaEventSynchronize(e1), "fx peak"))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(ctx, buf);
  if (st) return st;
  *products_per_s = (double)iters * ILP * (double)threads * blocks / (best * 1e-3);
  return GBS_OK;
}

extern "C" gbs_status gbs_measure_fp64_peak(gbs_ctx* ctx, double* gflops) {
  if (!ctx || !gflops) return GBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  cudaSetDevice(ctx->device);
  const int threads = 256, blocks = 4 * ctx->sm_count, iters = 8192;
  constexpr int ILP = 8;
  DevBuf buf;
  gbs_status st;
  if ((st = dev_alloc(ctx, buf, (size_t)threads * blocks * sizeof(double)))) return st;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    dfma_chain_kernel<ILP><<<blocks, threads, 0, ctx->stream>>>((double*)buf.ptr, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, ctx->stream);
    count_launch(ctx);
    if ((st = check_cuda(ctx, cudaEventSynchronize(e1), "fp64 peak"))) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(ctx, buf);
  if (st) return st;
  *gflops = 2.0 * iters * ILP * (double)threads * blocks / (best * 1e-3) / 1e9;
  return GBS_OK;
}
