// A variant of the FP64 real-basis subset tree that allocates nothing.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree.  cudaFree
// synchronises the whole device, so a latency-critical loop that runs other
// streams concurrently loses its overlap; callers whose device memory is owned
// by another allocator (a framework's caching allocator, a memory pool with a
// fixed budget) cannot accept hidden allocations; and code that has already
// sized all its memory up front cannot afford an allocation that may fail
// later.  This entry point takes device input and output buffers from the
// caller and keeps its intermediate data (tree levels, per-block partial sums,
// status word) in one file-scope __device__ array of fixed size, created when
// the library's device code is loaded and held by every GPU that loads it
// until the process exits.
//
// The array is shared by every call: calls whose work overlaps on the GPU (on
// different streams without ordering between them) race on it.  Each call
// clears the status word it reads; everything else it reads was written by the
// same call.  The array's device address is looked up once per device (first
// call on it) and kept for the life of the process, so the entry point must not
// be used on a device after cudaDeviceReset of that device in the same process.
#include <mutex>

#include "gbs_internal.h"
#include "gbs_tree.cuh"

namespace gbs {
namespace {

constexpr int kStaticQ = 5;  // register depth of the leaf kernel (as the FP64 real tree)
constexpr int kStaticMaxN = GBS_STATIC_MAX_N;

constexpr size_t level_entries_max(int n, int Q) {
  size_t best = 0;
  for (int l = 0; l <= n - Q; ++l) {
    const size_t v = ((size_t)1 << l) * (size_t)sym(2 * (n - l));
    best = v > best ? v : best;
  }
  return best;
}
constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kLevelBytes = round256(level_entries_max(kStaticMaxN, kStaticQ) * sizeof(double));
constexpr size_t kLeaves = (size_t)1 << (kStaticMaxN - kStaticQ);
constexpr size_t kSBytes = round256(kLeaves * sizeof(double));
constexpr size_t kBlocks = (kLeaves + 127) / 128;
constexpr size_t kPartBytes = round256(kBlocks * sizeof(Partial<dd>));
constexpr size_t kOutBytes = round256(sizeof(TreeOut) + sizeof(int));
constexpr size_t kScratchBytes = 2 * kLevelBytes + 2 * kSBytes + kPartBytes + kOutBytes;
static_assert(kScratchBytes <= GBS_STATIC_SCRATCH_BYTES, "static scratch too small for GBS_STATIC_MAX_N");

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[GBS_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Lower triangle of the caller's full 2n x 2n row-major matrix -> packed root.
__global__ void static_pack_kernel(const double* __restrict__ G, int n, double* __restrict__ root,
                                   double* __restrict__ s, int* __restrict__ status) {
  const int d = 2 * n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < sym(d)) {
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= i) ++a;
    const int b = i - a * (a + 1) / 2;
    root[i] = G[(long long)a * d + b];
  }
  if (i == 0) {
    s[0] = 1.0;
    *status = 0;
  }
}

// out = {tor_hi, tor_lo, inc_hi, inc_lo, exc_hi, exc_lo, abs_sum, status}
__global__ void static_emit_kernel(const TreeOut* __restrict__ t, const int* __restrict__ status,
                                   double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  const dd inc{t->inc[0], t->inc[1]}, exc{t->exc[0], t->exc[1]};
  const dd tor = inc + exc;
  out[0] = tor.hi;
  out[1] = tor.lo;
  out[2] = inc.hi;
  out[3] = inc.lo;
  out[4] = exc.hi;
  out[5] = exc.lo;
  out[6] = t->abs;
  out[7] = (double)*status;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

// Errors of this call's own launches are read right after each launch; an
// error that earlier work left pending is found before anything is queued and
// reported as GBS_ECUDA without being cleared.
#define GBS_STATIC_LAUNCHED()                               \
  do {                                                      \
    if (cudaGetLastError() != cudaSuccess) return GBS_ECUDA; \
  } while (0)

extern "C" gbs_status gbs_subset_sum_static(const double* G_dev, int n, double* out_dev, void* cuda_stream) {
  if (n < 1 || n > kStaticMaxN || !G_dev || !out_dev) return GBS_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return GBS_ECUDA;
  unsigned char* base = nullptr;
  if (scratch_address((void**)&base) != cudaSuccess) return GBS_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* lv[2] = {(double*)base, (double*)(base + kLevelBytes)};
  double* sv[2] = {(double*)(base + 2 * kLevelBytes), (double*)(base + 2 * kLevelBytes + kSBytes)};
  Partial<dd>* parts = (Partial<dd>*)(base + 2 * kLevelBytes + 2 * kSBytes);
  TreeOut* tout = (TreeOut*)(base + 2 * kLevelBytes + 2 * kSBytes + kPartBytes);
  int* status = (int*)(tout + 1);

  const int Q = n < kStaticQ ? n : kStaticQ;
  const int depth = n - Q;
  const long long leaves = 1LL << depth;
  const int blocks = (int)((leaves + 127) / 128);
  const int nent = sym(2 * n);
  static_pack_kernel<<<(nent + 255) / 256, 256, 0, s>>>(G_dev, n, lv[0], sv[0], status);
  GBS_STATIC_LAUNCHED();
  int cur = 0;
  for (int l = 0; l < depth; ++l) {
    const long long count = 1LL << l;
    const int q = n - l;
    const long long threads = count * (2 * q - 2);
    tree_level_kernel<double><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(lv[cur], sv[cur], count, q,
                                                                               lv[cur ^ 1], sv[cur ^ 1], status);
    GBS_STATIC_LAUNCHED();
    cur ^= 1;
  }
  switch (Q) {
    case 1: tree_leaf_kernel<double, 1><<<blocks, 128, 0, s>>>(lv[cur], sv[cur], leaves, depth, parts, status); break;
    case 2: tree_leaf_kernel<double, 2><<<blocks, 128, 0, s>>>(lv[cur], sv[cur], leaves, depth, parts, status); break;
    case 3: tree_leaf_kernel<double, 3><<<blocks, 128, 0, s>>>(lv[cur], sv[cur], leaves, depth, parts, status); break;
    case 4: tree_leaf_kernel<double, 4><<<blocks, 128, 0, s>>>(lv[cur], sv[cur], leaves, depth, parts, status); break;
    default: tree_leaf_kernel<double, 5><<<blocks, 128, 0, s>>>(lv[cur], sv[cur], leaves, depth, parts, status); break;
  }
  GBS_STATIC_LAUNCHED();
  tree_final_kernel<dd><<<1, 256, 0, s>>>(parts, blocks, tout);
  GBS_STATIC_LAUNCHED();
  static_emit_kernel<<<1, 32, 0, s>>>(tout, status, out_dev);
  GBS_STATIC_LAUNCHED();
  return GBS_OK;
}
#undef GBS_STATIC_LAUNCHED
