// Same-precision CPU baseline of the subset enumeration: the decision tree of
// shared-prefix Schur complements in plain FP64, depth-first per thread, OpenMP
// over subtrees.  Bench comparator only: it shares no code with the CUDA
// library or with the oracle.
//
// For a 2n x 2n real symmetric positive-definite G (mode i on rows 2i, 2i+1)
// it returns Tor = sum over mode subsets Z of (-1)^(n - |Z|) det(G_Z)^(-1/2)
// and the sum of |terms|.  Every term is one of the paper's vacuum
// probabilities (Eq. 5); the decision tree reuses the elimination step behind
// its no-click update (Eq. 4a): deciding mode j either drops its two rows
// (excluded) or replaces the undecided block by its Schur complement with
// respect to the 2 x 2 pivot block of j (included), det(G_Z) being the product
// of the included pivots' determinants.
//
// Storage: each node is a dense (2q x 2q) block addressed through a leading
// dimension, so the excluded child is the parent's trailing block (no copy);
// only the lower triangle is read and written.
#include <omp.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

struct Acc {
  double pos = 0.0, neg = 0.0;  // terms with sign +1 and -1, summed separately
};

// Per-thread work space: one (2q x 2q) block per depth of the walk.
struct Walker {
  int n;
  std::vector<std::vector<double>> buf;  // buf[q]: block of an included child with q undecided modes
  std::vector<double> l0, l1, u0, u1;
  Acc acc;
  explicit Walker(int n_) : n(n_), buf(n_ + 1), l0(2 * n_), l1(2 * n_), u0(2 * n_), u1(2 * n_) {
    for (int q = 0; q <= n; ++q) buf[q].assign((size_t)(2 * q) * (2 * q) + 1, 0.0);
  }

  // Node with q undecided modes: block C (leading dimension ld), scale s, sign of its
  // terms (+1 / -1 for an even / odd number of exclusions so far).
  void walk(const double* C, int ld, int q, double s, int sign) {
    if (q == 0) {
      if (sign > 0) acc.pos += s; else acc.neg += s;
      return;
    }
    const double a = C[0], b = C[ld], c = C[ld + 1];
    const double det = a * c - b * b;
    const double g = 1.0 / std::sqrt(det);
    const int d = 2 * q - 2;
    if (d > 0) {
      double* D = buf[q - 1].data();
      const double ia = a / det, ic = c / det, ib = b / det;
      for (int i = 0; i < d; ++i) {
        const double x0 = C[(i + 2) * ld], x1 = C[(i + 2) * ld + 1];
        u0[i] = x0;
        u1[i] = x1;
        l0[i] = x0 * ic - x1 * ib;  // row i of U P^-1
        l1[i] = x1 * ia - x0 * ib;
      }
      for (int i = 0; i < d; ++i) {
        const double* src = C + (i + 2) * ld + 2;
        double* dst = D + i * d;
        const double li0 = l0[i], li1 = l1[i];
        for (int j = 0; j <= i; ++j) dst[j] = src[j] - li0 * u0[j] - li1 * u1[j];
      }
      walk(D, d, q - 1, s * g, sign);
    } else {
      walk(nullptr, 0, 0, s * g, sign);
    }
    walk(q > 1 ? C + 2 * ld + 2 : nullptr, ld, q - 1, s, -sign);  // excluded: the trailing block as it is
  }
};

}  // namespace

extern "C" {

// Tor and sum|terms| of G (row-major 2n x 2n, lower triangle read) with `threads`
// OpenMP threads (<= 0: all).  The first `split` modes are decided by a loop over
// 2^split prefixes shared out among the threads.  Returns 0, or 1 if a pivot was
// not positive definite (the sums are then NaN), 2 on bad arguments.
int cpu_tree_fp64(int n, const double* G, int threads, int split, double* tor, double* abs_sum, double* seconds) {
  if (n < 1 || n > 40 || !G) return 2;
  if (threads <= 0) threads = omp_get_max_threads();
  if (split < 0) split = 0;
  if (split > n) split = n;
  const int D = 2 * n;
  const auto t0 = std::chrono::steady_clock::now();
  double pos = 0.0, neg = 0.0;
  const long long prefixes = 1LL << split;
#pragma omp parallel num_threads(threads) reduction(+ : pos, neg)
  {
    Walker w(n);
    std::vector<double> A((size_t)D * D), B((size_t)D * D);
#pragma omp for schedule(dynamic, 1)
    for (long long pf = 0; pf < prefixes; ++pf) {
      // decide the first `split` modes as the bits of pf (bit split-1-i for mode i: 1 = included)
      std::memcpy(A.data(), G, sizeof(double) * D * D);
      double* C = A.data();
      double* T = B.data();
      int ld = D, q = n, sign = 1;
      double s = 1.0;
      bool ok = true;
      for (int i = 0; i < split && ok; ++i) {
        if (!((pf >> (split - 1 - i)) & 1)) {
          C += 2 * ld + 2;
          --q;
          sign = -sign;
          continue;
        }
        const double a = C[0], b = C[ld], c = C[ld + 1];
        const double det = a * c - b * b;
        const double ia = a / det, ic = c / det, ib = b / det;
        const int d = 2 * q - 2;
        for (int r = 0; r < d; ++r)
          for (int col = 0; col <= r; ++col) {
            const double x0 = C[(r + 2) * ld], x1 = C[(r + 2) * ld + 1];
            const double y0 = C[(col + 2) * ld], y1 = C[(col + 2) * ld + 1];
            T[r * d + col] = C[(r + 2) * ld + col + 2] - (x0 * ic - x1 * ib) * y0 - (x1 * ia - x0 * ib) * y1;
          }
        s /= std::sqrt(det);
        std::swap(A, B);
        C = A.data();
        T = B.data();
        ld = d;
        --q;
      }
      w.acc = Acc();
      w.walk(q > 0 ? C : nullptr, ld, q, s, sign);
      pos += w.acc.pos;
      neg += w.acc.neg;
    }
  }
  const auto t1 = std::chrono::steady_clock::now();
  *tor = pos - neg;
  *abs_sum = pos + neg;
  if (seconds) *seconds = std::chrono::duration<double>(t1 - t0).count();
  return std::isfinite(pos + neg) ? 0 : 1;
}

int cpu_tree_max_threads(void) { return omp_get_max_threads(); }

}  // extern "C"
