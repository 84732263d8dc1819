// FP64 peak microbenchmark: independent chains of dependent DFMAs in every
// thread of a full grid; the FP64 pipe is the only unit it loads.  Used as the
// roofline denominator of the FP64-bound subset-determinant kernels.
#include "gbs_internal.h"

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

}  // namespace gbs

using namespace gbs;

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
