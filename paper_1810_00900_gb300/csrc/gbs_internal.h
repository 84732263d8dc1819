// Internal C++ interfaces shared by the translation units of libgbs.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gbs.h"

namespace gbs {

// The largest gbs_prec value.
constexpr int kPrecLast = GBS_PREC_FXN;

// The fixed-point precisions (real basis; need a state that bounds the tree).
constexpr bool is_fixed_point(int prec) {
  return prec == GBS_PREC_FXN || prec == GBS_PREC_FX || prec == GBS_PREC_FXW;
}

struct TreeOut;

// One tree of a batch: n modes, packed FP64 root starting at entry root_off.
struct BatchTree {
  int n;
  long long root_off;
};

// Launch parameters of the batched engine (chosen by the autotuner).
struct BatchTune {
  int d_top = 10;                       // depth the top kernel reaches per tree (at most)
  int top_threads = 256;                // CTA size of the top kernel
  long long level_threads = 1LL << 18;  // target threads per breadth-first level launch
  int leaf_grid_per_sm = 0;             // 0: one CTA per work unit; k > 0: persistent, k CTAs per SM
  int sub_e = 5;                        // levels each subtree CTA expands in shared memory (0: plain leaf)
  int q_drop = 0;                       // register depth-first levels below the variant's maximum (fewer
                                        // registers per thread, more warps per SM)
  int mid_e = 0;                        // levels each top CTA expands in shared memory after its prefix
};

// Device memory obtained by the library, accounted against the context budget.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct KernelTimer {
  cudaEvent_t start = nullptr, stop = nullptr;
  double total_ms = 0.0;
  long long count = 0;
  bool pending = false;
};

}  // namespace gbs

struct gbs_ctx {
  int device = 0;
  size_t budget = 0;
  std::atomic<size_t> in_use{0};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  std::mutex mu;  // serialises calls that use the shared workspace
  // Freed device blocks kept for reuse (stream-ordered: every use of a block is
  // queued on the context's one stream, so a later allocation may take it at
  // once); they stay counted in in_use, and are released when an allocation
  // would exceed the budget, when the stream changes and at destruction.
  std::mutex cache_mu;
  std::multimap<size_t, void*> cache;
  size_t cached = 0;

  // tree workspace (grown on demand)
  gbs::DevBuf lvl[2], sbuf[2], partials, out, status, hbuf;
  // batched engine: small tables staged host -> device through a bump arena
  // (pinned host + device, reset at the start of each synchronous call) and
  // the per-tree results
  gbs::DevBuf stage_dev, aux_dev;
  void* stage_host = nullptr;
  size_t stage_cap = 0, stage_off = 0;
  // host-pinned readback
  void* host_out = nullptr;

  // instrumentation
  bool timing = false;
  gbs::KernelTimer leaf_timer;
  std::atomic<long long> launches{0};
  int sm_count = 0;
  // host gaps: time from the return of a host wait on the stream (stream_sync)
  // to the next kernel launch, while the stream sits empty
  bool gap_open = false;
  std::chrono::steady_clock::time_point gap_since;
  double gap_s = 0.0;
  long long gap_waits = 0;

  // batched-engine launch parameters per (precision, basis): [prec][real]
  gbs::BatchTune tune[gbs::kPrecLast + 1][2];  // [gbs_prec][basis is real]
  bool tuned[gbs::kPrecLast + 1][2] = {};

  // request loop (see gbs_server.cu)
  void* server = nullptr;

  // A batch whose tree workspace (level buffers, s values, partials) would
  // exceed batch_cap_bytes is refused by the planner before anything is
  // allocated or launched (batch_split set) and evaluated in parts instead.
  size_t batch_cap_bytes = 0;
  bool batch_split = false;
};

struct gbs_state {
  gbs_ctx* ctx = nullptr;
  int M = 0;
  bool has_factors = false;  // built from (U, r, eta): closed-form Sigma^-1 blocks available
  double eta = 1.0;
  double logdet_sigma = 0.0;
  double sigma_max = 0.0;  // upper bound on the largest eigenvalue of Sigma (0 = unknown)
  gbs::DevBuf U;      // M x M complex (interleaved), row-major
  gbs::DevBuf r;      // M doubles
  gbs::DevBuf alpha;  // M doubles: (1/d+ + 1/d-)/2
  gbs::DevBuf beta;   // M doubles: (1/d+ - 1/d-)/2
  gbs::DevBuf V;      // 2M x 2M complex covariance, block order (a, a^+); built on first use
  gbs::DevBuf Sinv;   // 2M x 2M complex Sigma^-1 (states given by V only)
  gbs::DevBuf sig_real;  // 2M x 2M Sigma in the real x/p basis (built by the first gbs_sample)
};

namespace gbs {

// error helpers (gbs_api.cu)
gbs_status set_error(gbs_ctx* ctx, gbs_status st, const std::string& msg);
gbs_status check_cuda(gbs_ctx* ctx, cudaError_t e, const char* what);
gbs_status dev_alloc(gbs_ctx* ctx, DevBuf& b, size_t bytes);
gbs_status dev_reserve(gbs_ctx* ctx, DevBuf& b, size_t bytes);  // grow-only
void dev_free(gbs_ctx* ctx, DevBuf& b);
void cache_release(gbs_ctx* ctx);  // return cached device blocks to CUDA (cudaFree)
inline void count_launch(gbs_ctx* ctx, long long n = 1) {
  ctx->launches += n;
  if (ctx->gap_open) {
    ctx->gap_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - ctx->gap_since).count();
    ctx->gap_open = false;
  }
}
// Wait for the context stream to drain (to read results back) and start a host gap.
gbs_status stream_sync(gbs_ctx* ctx);

// Staging arena: stage_begin() makes room for `bytes` (synchronising first if it
// must grow) and resets it; stage() copies host data into the next region and
// queues the host -> device copy on the context stream.  (gbs_batch_api.cu)
gbs_status stage_begin(gbs_ctx* ctx, size_t bytes);
gbs_status stage(gbs_ctx* ctx, const void* data, size_t bytes, const void** dev);

// Per-tree result after the finishing kernel (device and host layout).
struct ProbOut {
  double p_hi, p_lo;
  double tor[3];
  double abs_sum, kappa, err;
  double inc[3], exc[3];
  int status;
  int pad;
};

gbs_status batch_fp64_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fp64_cplx(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_dd_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_dd_cplx(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_td_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_td_cplx(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fx_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fxw_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fp64p_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fxn_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fp32_real(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);
gbs_status batch_fp32_cplx(gbs_ctx*, int, const BatchTree*, const void*, TreeOut*, int*, const BatchTune&);

// Evaluate ntrees trees whose packed FP64 roots are already in roots_dev
// (entries at trees[t].root_off); logdet[t] (host) scales p = Tor exp(-logdet/2).
// Synchronous: fills host_out[0..ntrees).  (gbs_batch_api.cu)
gbs_status batch_eval(gbs_ctx* ctx, int prec, bool real, int ntrees, const BatchTree* trees, const void* roots_dev,
                      const double* logdet, ProbOut* host_out);
// The tuning in force for (prec, basis) -- the autotuner's choice when one was made.
const BatchTune& batch_tune_for(gbs_ctx* ctx, int prec, bool real);

// One chain-rule trajectory (gbs_sampler.cu): host bookkeeping plus device
// buffers inside a block of traj_bytes(M) bytes bound by traj_bind().
struct Trajectory {
  enum { kRunning = 0, kDone = 1, kRejected = 2 };
  gbs_state* st = nullptr;
  int M = 0;
  unsigned long long seed = 0;
  int sample = 0, attempt = 0, N_post = 0;
  std::vector<char> forced;  // empty: free draws; else 1 where the outcome is a click
  bool want_p0 = false;
  // device
  double* sig = nullptr;  // conditioned Sigma' (2M x 2M, real x/p basis)
  int* clicks = nullptr;
  double* pinv = nullptr;
  double* dcarry = nullptr;
  double* L = nullptr;
  // host
  int step = 0, m = 0, need_full = 1, state = kRunning;
  std::vector<int> S;
  double kappa_prev = 1.0, relD = 0.0;
  std::vector<double> p0;
};
size_t traj_bytes(int M);
void traj_bind(Trajectory& tj, gbs_state* st, unsigned char* mem);
gbs_status traj_start(gbs_ctx* ctx, Trajectory& tj);
gbs_status ensure_sigma_real(gbs_ctx* ctx, gbs_state* st);
gbs_status sampler_advance(gbs_ctx* ctx, const std::vector<Trajectory*>& jobs, int prec, gbs_sample_stats& stt);
double unit_of(int prec);
// Fixed-point eligibility (gbs_batch_api.cu): a tree over n modes of
// (Sigma^-1)_S, resp. of a conditioned Sigma', keeps every value in range.
bool fx_ok_inverse(const gbs_state* st, int n);
bool fx_ok_sigma(const gbs_state* st, int n);

// Error model of a subset tree over n modes in precision prec: |dTor| <=
// err_factor * unit * sum|terms|, with 4 n units per term (n rank-2 Schur steps
// and one inverse square root) and, for the FP64 family, 24 more for the FP64
// sums of the non-negative sign-split partials (up to 15 within a thread's
// register subtree, 5 across a warp, margin for the double-double stages).
inline double err_factor(int prec, int n) {
  const double base = 4.0 * (n > 1 ? n : 1);
  return (prec == GBS_PREC_FP64 || prec == GBS_PREC_FP64P || prec == GBS_PREC_FP32_DIAG) ? base + 24.0 : base;
}

// Up to 32 click modes passed by value as a kernel argument.
struct ModeList {
  int m[32];
};

// Request loop (gbs_server.cu): stop and free it, if running.
void server_shutdown(gbs_ctx* ctx);

// States (gbs_state.cu)
gbs_status state_build(gbs_ctx* ctx, int M, const double* U, const double* r, double eta, double* V_out,
                       gbs_state** out);
gbs_status state_from_V(gbs_ctx* ctx, int M, const double* V, gbs_state** out);
// Build the covariance V of a factor-built state if it is not there yet.
gbs_status ensure_V(gbs_ctx* ctx, gbs_state* st);
// Enqueue the packed lower triangle of (Sigma^-1)_S (FP64; complex entries as
// (re, im) pairs, or real x/p entries) into dev_out on the context stream.
gbs_status click_block(gbs_ctx* ctx, const gbs_state* st, const int* modes, int N, int real_basis, void* dev_out);
}  // namespace gbs
