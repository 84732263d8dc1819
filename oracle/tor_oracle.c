/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * legs may load this code.  It shares nothing with the GPU path.
 *
 * What it computes: signed sums of inverse square roots of principal-minor
 * determinants of a 2n x 2n complex Hermitian positive-definite matrix G whose
 * rows/columns 2i, 2i+1 belong to "mode" i:
 *
 *     S = sum over W subset of F of  sign(W) * det(G[W u X])^(-1/2)
 *
 * with F a list of free modes, X a list of modes always included, and
 * sign(W) = (-1)^(|F|-|W|) (Torontonian convention) or (-1)^|W| (inclusion-
 * exclusion over clicked modes).  Every term is a vacuum probability of the
 * paper's Eq. (5) (q = 2/sqrt(det(V_B + 1)) = 1/sqrt(det Sigma_B)), and the
 * alternating sums are the click/no-click bookkeeping of Eqs. (6)-(7) written
 * in closed form; with G = (Sigma^-1)_S, F = S, X empty and the Torontonian
 * sign this is Tor(O_S) with O = 1 - Sigma^-1.
 *
 * Two independent evaluations:
 *   O1 (orc_sum_bruteforce): the definition -- every subset separately, its
 *      determinant by Gaussian elimination with partial pivoting.
 *   O2 (orc_sum_tree): the same sum by a binary decision tree over the free
 *      modes, using det [[P, B], [B^H, D]] = det P * det(D - B^H P^-1 B)
 *      (the Schur-complement identity behind the paper's Eq. (4a)) to reuse
 *      the elimination of a shared prefix.  O2 exists because O1 cannot finish
 *      2^24 subsets; tests pin O2 to O1.
 *
 * Arithmetic: "qd" numbers, unevaluated sums of four doubles with about 212
 * bits of precision, built only from error-free transformations:
 *   TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971) and TwoProd via a
 *   fused multiply-add.  Normalisation repeats an error-free VecSum pass
 *   (Ogita, Rump, Oishi 2005) until the components stop changing, which leaves
 *   them non-overlapping and decreasing; the sum is exact until the final
 *   truncation to four components.  Division is long division, the inverse
 *   square root Newton's iteration.  This is deliberately simple and slow.
 *
 * Build with -ffp-contract=off: every rounding must be the one written here.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QK 4 /* components per number */

typedef struct { double c[QK]; } qd;
typedef struct { qd re, im; } cqd;

/* ---------------------------------------------------------------- EFTs --- */

static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *e = (a - av) + (b - bv);
  *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/* Repeated VecSum until a fixed point, then keep the QK leading components.
 * t[] is overwritten.  At the fixed point adding t[i] to t[i-1] no longer
 * changes t[i-1], i.e. |t[i]| <= ulp(t[i-1])/2, and zeros sit at the end. */
static qd normalize(double *t, int n) {
  for (int pass = 0; pass < 4 * n + 8; ++pass) {
    int changed = 0;
    for (int i = n - 1; i >= 1; --i) {
      double s, e;
      two_sum(t[i - 1], t[i], &s, &e);
      if (s != t[i - 1] || e != t[i]) changed = 1;
      t[i - 1] = s;
      t[i] = e;
    }
    if (!changed) break;
  }
  qd r;
  /* Zeros may remain between nonzero components only if a component is 0
   * while a later one is not, which the fixed point excludes; still compact. */
  int k = 0;
  for (int i = 0; i < n && k < QK; ++i)
    if (t[i] != 0.0) r.c[k++] = t[i];
  for (; k < QK; ++k) r.c[k] = 0.0;
  return r;
}

static inline qd qd_from(double a) { qd r = {{a, 0.0, 0.0, 0.0}}; return r; }
static inline double qd_hi(qd a) { return a.c[0]; }

static qd qd_add(qd a, qd b) {
  double t[2 * QK];
  /* interleave by weight so one pass already moves most of the mass */
  for (int i = 0; i < QK; ++i) { t[2 * i] = a.c[i]; t[2 * i + 1] = b.c[i]; }
  return normalize(t, 2 * QK);
}

static qd qd_neg(qd a) { for (int i = 0; i < QK; ++i) a.c[i] = -a.c[i]; return a; }
static qd qd_sub(qd a, qd b) { return qd_add(a, qd_neg(b)); }

/* Product: all a_i*b_j with i+j <= QK-1 exactly (TwoProd), the i+j = QK terms
 * rounded; the dropped terms are below 2^-(53*QK) |a b| * QK^2. */
static qd qd_mul(qd a, qd b) {
  double t[2 * QK * QK];
  int n = 0;
  for (int s = 0; s <= QK; ++s) {
    for (int i = 0; i <= s && i < QK; ++i) {
      int j = s - i;
      if (j >= QK) continue;
      if (s < QK) {
        two_prod(a.c[i], b.c[j], &t[n], &t[n + 1]);
        n += 2;
      } else {
        t[n++] = a.c[i] * b.c[j];
      }
    }
  }
  return normalize(t, n);
}

static qd qd_mul_d(qd a, double b) {
  double t[2 * QK];
  for (int i = 0; i < QK; ++i) two_prod(a.c[i], b, &t[2 * i], &t[2 * i + 1]);
  return normalize(t, 2 * QK);
}

/* Long division: q_k = (remainder)_hi / b_hi, remainder -= q_k * b. */
static qd qd_div(qd a, qd b) {
  double q[QK + 1];
  qd r = a;
  for (int k = 0; k <= QK; ++k) {
    q[k] = r.c[0] / b.c[0];
    r = qd_sub(r, qd_mul_d(b, q[k]));
  }
  return normalize(q, QK + 1);
}

/* 1/sqrt(a), a > 0: Newton x <- x + x (1 - a x^2) / 2 from the double guess;
 * each step doubles the correct bits (53 -> 106 -> 212), a third one settles. */
static qd qd_rsqrt(qd a) {
  qd x = qd_from(1.0 / sqrt(a.c[0]));
  for (int it = 0; it < 3; ++it) {
    qd ax2 = qd_mul(a, qd_mul(x, x));
    qd corr = qd_sub(qd_from(1.0), ax2);
    x = qd_add(x, qd_mul_d(qd_mul(x, corr), 0.5));
  }
  return x;
}

static inline int qd_is_neg(qd a) { return a.c[0] < 0.0; }

/* ------------------------------------------------------------- complex --- */

static inline cqd cq_from(double re, double im) { cqd z; z.re = qd_from(re); z.im = qd_from(im); return z; }
static inline cqd cq_add(cqd a, cqd b) { cqd z; z.re = qd_add(a.re, b.re); z.im = qd_add(a.im, b.im); return z; }
static inline cqd cq_sub(cqd a, cqd b) { cqd z; z.re = qd_sub(a.re, b.re); z.im = qd_sub(a.im, b.im); return z; }
static inline cqd cq_mul(cqd a, cqd b) {
  cqd z;
  z.re = qd_sub(qd_mul(a.re, b.re), qd_mul(a.im, b.im));
  z.im = qd_add(qd_mul(a.re, b.im), qd_mul(a.im, b.re));
  return z;
}
static inline cqd cq_conj(cqd a) { a.im = qd_neg(a.im); return a; }
static inline qd cq_abs2(cqd a) { return qd_add(qd_mul(a.re, a.re), qd_mul(a.im, a.im)); }
static cqd cq_div(cqd a, cqd b) {
  qd den = cq_abs2(b);
  cqd num = cq_mul(a, cq_conj(b));
  cqd z; z.re = qd_div(num.re, den); z.im = qd_div(num.im, den);
  return z;
}
static inline double cq_abs2_d(cqd a) { return a.re.c[0] * a.re.c[0] + a.im.c[0] * a.im.c[0]; }

/* --------------------------------------------------- O1: brute force ----- */

/* Determinant of the d x d complex matrix A (row-major, overwritten) by
 * Gaussian elimination with partial pivoting.  Returns the determinant. */
static cqd det_lu(cqd *A, int d) {
  cqd det = cq_from(1.0, 0.0);
  for (int k = 0; k < d; ++k) {
    int p = k;
    double best = cq_abs2_d(A[k * d + k]);
    for (int i = k + 1; i < d; ++i) {
      double v = cq_abs2_d(A[i * d + k]);
      if (v > best) { best = v; p = i; }
    }
    if (p != k) {
      for (int j = 0; j < d; ++j) { cqd t = A[k * d + j]; A[k * d + j] = A[p * d + j]; A[p * d + j] = t; }
      det.re = qd_neg(det.re); det.im = qd_neg(det.im);
    }
    cqd piv = A[k * d + k];
    det = cq_mul(det, piv);
    for (int i = k + 1; i < d; ++i) {
      cqd f = cq_div(A[i * d + k], piv);
      for (int j = k + 1; j < d; ++j) A[i * d + j] = cq_sub(A[i * d + j], cq_mul(f, A[k * d + j]));
    }
  }
  return det;
}

typedef struct {
  int n;              /* G is 2n x 2n */
  const double *G;    /* interleaved (re, im), row-major */
  int nf; const int *F;
  int nx; const int *X;
  int sign_mode;      /* 0: (-1)^(nf-|W|), 1: (-1)^|W| */
  /* work split */
  uint64_t begin, end;
  /* results */
  qd sum; qd abs_sum; int status;
} bf_task;

static void *bf_worker(void *arg) {
  bf_task *t = (bf_task *)arg;
  int dmax = 2 * (t->nf + t->nx);
  int *rows = (int *)malloc(sizeof(int) * (dmax > 0 ? dmax : 1));
  cqd *A = (cqd *)malloc(sizeof(cqd) * (dmax > 0 ? dmax * dmax : 1));
  qd sum = qd_from(0.0), asum = qd_from(0.0);
  t->status = 0;
  for (uint64_t w = t->begin; w < t->end; ++w) {
    int d = 0, card = 0;
    for (int i = 0; i < t->nf; ++i)
      if ((w >> i) & 1u) { rows[d++] = 2 * t->F[i]; rows[d++] = 2 * t->F[i] + 1; ++card; }
    for (int i = 0; i < t->nx; ++i) { rows[d++] = 2 * t->X[i]; rows[d++] = 2 * t->X[i] + 1; }
    qd term;
    if (d == 0) {
      term = qd_from(1.0);
    } else {
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
          const double *g = t->G + 2 * ((size_t)rows[a] * 2 * t->n + rows[b]);
          A[a * d + b] = cq_from(g[0], g[1]);
        }
      cqd det = det_lu(A, d);
      if (qd_is_neg(det.re) || det.re.c[0] == 0.0) { t->status = 1; break; }
      term = qd_rsqrt(det.re);
    }
    int neg = t->sign_mode == 0 ? ((t->nf - card) & 1) : (card & 1);
    asum = qd_add(asum, term);
    sum = neg ? qd_sub(sum, term) : qd_add(sum, term);
  }
  t->sum = sum; t->abs_sum = asum;
  free(rows); free(A);
  return NULL;
}

static void qd_store(qd v, double *out) { for (int i = 0; i < QK; ++i) out[i] = v.c[i]; }

/* Returns 0 on success, 1 if some minor is not positive, 2 on bad arguments. */
int orc_sum_bruteforce(int n, const double *G, int nf, const int *F, int nx, const int *X,
                       int sign_mode, int nthreads, double *out_sum, double *out_abs) {
  if (n < 0 || nf < 0 || nx < 0 || nf > 40 || nf + nx > n) return 2;
  uint64_t total = (uint64_t)1 << nf;
  if (nthreads < 1) nthreads = 1;
  if ((uint64_t)nthreads > total) nthreads = (int)total;
  bf_task *tasks = (bf_task *)calloc(nthreads, sizeof(bf_task));
  pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
  for (int i = 0; i < nthreads; ++i) {
    bf_task *t = &tasks[i];
    t->n = n; t->G = G; t->nf = nf; t->F = F; t->nx = nx; t->X = X; t->sign_mode = sign_mode;
    t->begin = total * i / nthreads; t->end = total * (i + 1) / nthreads;
    pthread_create(&th[i], NULL, bf_worker, t);
  }
  qd sum = qd_from(0.0), asum = qd_from(0.0);
  int status = 0;
  for (int i = 0; i < nthreads; ++i) {
    pthread_join(th[i], NULL);
    sum = qd_add(sum, tasks[i].sum);
    asum = qd_add(asum, tasks[i].abs_sum);
    if (tasks[i].status) status = 1;
  }
  qd_store(sum, out_sum);
  *out_abs = asum.c[0];
  free(tasks); free(th);
  return status;
}

/* ------------------------------------------------ O2: decision tree ------ */

typedef struct {
  int nf, sign_mode, depth_top;
  const cqd *C0;     /* Schur complement on the free modes after the fixed ones, (2nf)^2 */
  qd s0;             /* det(G_X)^(-1/2) */
  int task_begin, task_end;
  qd *task_sum, *task_abs;
  int status;
} tree_ctx;

/* Include the first mode (rows 0,1) of the q-mode matrix C: returns the
 * (q-1)-mode Schur complement in Cn and det(P)^(-1/2) in *g. */
static int tree_include(const cqd *C, int q, cqd *Cn, qd *g) {
  int d = 2 * q, dn = d - 2;
  cqd p00 = C[0], p01 = C[1], p10 = C[d], p11 = C[d + 1];
  /* det P = p00 p11 - p01 p10 (real for Hermitian P) */
  cqd det = cq_sub(cq_mul(p00, p11), cq_mul(p01, p10));
  if (qd_is_neg(det.re) || det.re.c[0] == 0.0) return 1;
  *g = qd_rsqrt(det.re);
  /* P^-1 = [[p11, -p01], [-p10, p00]] / det */
  cqd inv00 = cq_div(p11, det), inv01 = cq_div(cq_sub(cq_from(0, 0), p01), det);
  cqd inv10 = cq_div(cq_sub(cq_from(0, 0), p10), det), inv11 = cq_div(p00, det);
  for (int a = 0; a < dn; ++a) {
    cqd ua0 = C[(a + 2) * d + 0], ua1 = C[(a + 2) * d + 1];
    cqd l0 = cq_add(cq_mul(ua0, inv00), cq_mul(ua1, inv10));
    cqd l1 = cq_add(cq_mul(ua0, inv01), cq_mul(ua1, inv11));
    for (int b = 0; b < dn; ++b) {
      cqd v = C[(a + 2) * d + (b + 2)];
      v = cq_sub(v, cq_mul(l0, C[0 * d + (b + 2)]));
      v = cq_sub(v, cq_mul(l1, C[1 * d + (b + 2)]));
      Cn[a * dn + b] = v;
    }
  }
  return 0;
}

static void tree_exclude(const cqd *C, int q, cqd *Cn) {
  int d = 2 * q, dn = d - 2;
  for (int a = 0; a < dn; ++a)
    for (int b = 0; b < dn; ++b) Cn[a * dn + b] = C[(a + 2) * d + (b + 2)];
}

/* Depth-first sum below a node with q undecided modes. ninc = included so far,
 * nexc = excluded so far.  scratch holds q levels of matrices. */
static int tree_dfs(const cqd *C, int q, qd s, int ninc, int nexc, int sign_mode, cqd *scratch,
                    qd *sum, qd *asum) {
  if (q == 0) {
    int neg = sign_mode == 0 ? (nexc & 1) : (ninc & 1);
    *asum = qd_add(*asum, s);
    *sum = neg ? qd_sub(*sum, s) : qd_add(*sum, s);
    return 0;
  }
  cqd *Cn = scratch;
  cqd *next = scratch + (size_t)(2 * q - 2) * (2 * q - 2);
  qd g;
  if (tree_include(C, q, Cn, &g)) return 1;
  if (tree_dfs(Cn, q - 1, qd_mul(s, g), ninc + 1, nexc, sign_mode, next, sum, asum)) return 1;
  tree_exclude(C, q, Cn);
  return tree_dfs(Cn, q - 1, s, ninc, nexc + 1, sign_mode, next, sum, asum);
}

static void *tree_worker(void *arg) {
  tree_ctx *t = (tree_ctx *)arg;
  int nf = t->nf;
  size_t cap = 0;
  for (int q = nf; q >= 0; --q) cap += (size_t)(2 * q) * (2 * q);
  cqd *buf = (cqd *)malloc(sizeof(cqd) * (cap + 1));
  cqd *root = (cqd *)malloc(sizeof(cqd) * ((size_t)4 * nf * nf + 1));
  cqd *tmp = (cqd *)malloc(sizeof(cqd) * ((size_t)4 * nf * nf + 1));
  t->status = 0;
  for (int task = t->task_begin; task < t->task_end; ++task) {
    /* decisions for the first depth_top modes: bit (depth_top-1-i) of task = include mode i */
    memcpy(root, t->C0, sizeof(cqd) * 4 * nf * nf);
    qd s = t->s0;
    int q = nf, ninc = 0, nexc = 0, bad = 0;
    for (int i = 0; i < t->depth_top; ++i) {
      int inc = (task >> (t->depth_top - 1 - i)) & 1;
      if (inc) {
        qd g;
        if (tree_include(root, q, tmp, &g)) { bad = 1; break; }
        s = qd_mul(s, g);
        ++ninc;
      } else {
        tree_exclude(root, q, tmp);
        ++nexc;
      }
      --q;
      memcpy(root, tmp, sizeof(cqd) * 4 * q * q);
    }
    qd sum = qd_from(0.0), asum = qd_from(0.0);
    if (bad || tree_dfs(root, q, s, ninc, nexc, t->sign_mode, buf, &sum, &asum)) { t->status = 1; break; }
    t->task_sum[task] = sum;
    t->task_abs[task] = asum;
  }
  free(buf); free(root); free(tmp);
  return NULL;
}

int orc_sum_tree(int n, const double *G, int nf, const int *F, int nx, const int *X, int sign_mode,
                 int nthreads, double *out_sum, double *out_abs) {
  if (n < 0 || nf < 0 || nx < 0 || nf > 40 || nf + nx > n) return 2;
  /* Gather the fixed modes first, then the free modes, and eliminate the fixed
   * block: C0 = Schur complement on F, s0 = det(G_X)^(-1/2). */
  int q = nx + nf, d = 2 * q;
  cqd *A = (cqd *)malloc(sizeof(cqd) * ((size_t)d * d + 1));
  cqd *B = (cqd *)malloc(sizeof(cqd) * ((size_t)d * d + 1));
  int *rows = (int *)malloc(sizeof(int) * (d + 1));
  int k = 0;
  for (int i = 0; i < nx; ++i) { rows[k++] = 2 * X[i]; rows[k++] = 2 * X[i] + 1; }
  for (int i = 0; i < nf; ++i) { rows[k++] = 2 * F[i]; rows[k++] = 2 * F[i] + 1; }
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      const double *g = G + 2 * ((size_t)rows[a] * 2 * n + rows[b]);
      A[a * d + b] = cq_from(g[0], g[1]);
    }
  qd s0 = qd_from(1.0);
  int status = 0;
  for (int i = 0; i < nx; ++i) {
    qd g;
    if (tree_include(A, q, B, &g)) { status = 1; break; }
    s0 = qd_mul(s0, g);
    --q;
    memcpy(A, B, sizeof(cqd) * 4 * q * q);
  }
  if (status) { free(A); free(B); free(rows); return status; }
  int depth_top = nf < 8 ? nf : 8;
  int ntask = 1 << depth_top;
  qd *task_sum = (qd *)calloc(ntask, sizeof(qd));
  qd *task_abs = (qd *)calloc(ntask, sizeof(qd));
  if (nthreads < 1) nthreads = 1;
  if (nthreads > ntask) nthreads = ntask;
  tree_ctx *ctx = (tree_ctx *)calloc(nthreads, sizeof(tree_ctx));
  pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
  for (int i = 0; i < nthreads; ++i) {
    tree_ctx *t = &ctx[i];
    t->nf = nf; t->sign_mode = sign_mode; t->depth_top = depth_top; t->C0 = A; t->s0 = s0;
    t->task_begin = ntask * i / nthreads; t->task_end = ntask * (i + 1) / nthreads;
    t->task_sum = task_sum; t->task_abs = task_abs;
    pthread_create(&th[i], NULL, tree_worker, t);
  }
  for (int i = 0; i < nthreads; ++i) {
    pthread_join(th[i], NULL);
    if (ctx[i].status) status = 1;
  }
  qd sum = qd_from(0.0), asum = qd_from(0.0);
  for (int i = 0; i < ntask; ++i) { sum = qd_add(sum, task_sum[i]); asum = qd_add(asum, task_abs[i]); }
  qd_store(sum, out_sum);
  *out_abs = asum.c[0];
  free(task_sum); free(task_abs); free(ctx); free(th); free(A); free(B); free(rows);
  return status;
}

/* ------------------------------------------- exported arithmetic probes -- */
/* For the tests that pin the qd arithmetic against exact rationals. */
void orc_qd_op(int op, const double *a, const double *b, double *out) {
  qd x, y, r;
  for (int i = 0; i < QK; ++i) { x.c[i] = a[i]; y.c[i] = b[i]; }
  switch (op) {
    case 0: r = qd_add(x, y); break;
    case 1: r = qd_mul(x, y); break;
    case 2: r = qd_div(x, y); break;
    case 3: r = qd_rsqrt(x); break;
    default: r = qd_sub(x, y); break;
  }
  qd_store(r, out);
}

/* Normalise an arbitrary list of doubles into a qd (exact up to truncation). */
void orc_qd_normalize(const double *t_in, int n, double *out) {
  double *t = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  memcpy(t, t_in, sizeof(double) * n);
  qd r = normalize(t, n);
  qd_store(r, out);
  free(t);
}

/* Determinant of a d x d complex matrix (interleaved re/im, row-major) in qd. */
void orc_det(int d, const double *M, double *out_re, double *out_im) {
  cqd *A = (cqd *)malloc(sizeof(cqd) * ((size_t)d * d + 1));
  for (int i = 0; i < d * d; ++i) A[i] = cq_from(M[2 * i], M[2 * i + 1]);
  cqd det = d > 0 ? det_lu(A, d) : cq_from(1.0, 0.0);
  qd_store(det.re, out_re);
  qd_store(det.im, out_im);
  free(A);
}
