/*
 * gbs.h -- C ABI of libgbs: exact threshold-detector Gaussian Boson Sampling
 * (click probabilities via Torontonians and chain-rule click sampling) on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Gupt, Arrazola, Quesada, Bromley, "Classical benchmarking of Gaussian
 * Boson Sampling on the Titan supercomputer", arXiv:1810.00900.  Sec. II gives
 * the sequential-measurement algorithm: a Gaussian state (Eq. 1), the
 * no-click update V_A' = V_A - V_AB (V_B + 1)^-1 V_AB^T (Eq. 4a), the vacuum
 * probability q = 2 / sqrt(det(V_B + 1)) of a measured mode (Eq. 5) and the
 * click / no-click mixture updates (Eqs. 6-7).  Summing that mixture in closed
 * form gives the threshold click probability of a pattern S (clicks on S,
 * vacuum elsewhere) as
 *
 *     p(S) = Tor(O_S) / sqrt(det Sigma),
 *     Tor(O_S) = sum over Z subset S of (-1)^(|S|-|Z|) / sqrt(det(1 - O_Z)),
 *
 * with Sigma = V + 1/2 (complex basis, vacuum V = 1/2) and O = 1 - Sigma^-1, so
 * that every term is a vacuum probability of Eq. (5).
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  - Modes are 0-based.  M = number of modes of a state, N = number of clicks.
 *  - Complex numbers are interleaved (re, im) doubles.  Matrices are row-major.
 *  - Complex basis: (a_1..a_M, a_1^+..a_M^+) ("block order"); covariance V is
 *    2M x 2M complex with vacuum V = I/2.  The paper's real basis is
 *    (x_1, p_1, ..., x_M, p_M) with hbar = 2; a = (x + i p)/2.
 *  - Status: every function returns a gbs_status (0 = GBS_OK).  No exceptions
 *    cross the ABI.  On error the outputs are left unspecified and a message
 *    is available from gbs_ctx_last_error().
 *  - Ownership: the caller owns every array it passes (host memory unless a
 *    parameter says "device"); the library copies what it keeps.  Handles
 *    (gbs_ctx, gbs_state) are owned by the caller and freed explicitly; every
 *    state must be freed before the context it was created on.
 *  - Thread safety: calls on one context are serialised internally; the
 *    request loop (gbs_submit / gbs_poll) may be used from any thread.
 */
#ifndef GBS_H_
#define GBS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gbs_status;
#define GBS_OK 0
#define GBS_EINVAL 1      /* invalid argument */
#define GBS_ENOMEM 2      /* device memory budget of the context exceeded */
#define GBS_ENOTPD 3      /* a matrix that must be positive definite is not */
#define GBS_EPRECISION 4  /* the requested accuracy cannot be certified */
#define GBS_EREJECT 5     /* postselection attempts exhausted */
#define GBS_ETIMEDOUT 6   /* a bounded wait ran out */
#define GBS_ECUDA 7       /* a CUDA runtime call failed */
#define GBS_PENDING 8     /* request not finished yet (gbs_poll) */
#define GBS_ENOTFOUND 9   /* unknown ticket */

/* Per-term arithmetic of the subset enumeration. */
typedef enum {
  GBS_PREC_AUTO = 0,       /* cheapest of FP64 / FP64P / FXN / FX / FXW / TD whose error estimate
                              meets rel_tol (FP64P only where FP64 missed by <= 1e3) */
  GBS_PREC_FP64 = 1,       /* IEEE double */
  GBS_PREC_DD = 2,         /* double-double, ~106-bit significand */
  GBS_PREC_TD = 3,         /* triple-double, ~159-bit significand */
  GBS_PREC_FP32_DIAG = 4,  /* FP32 terms, FP64 sums: diagnostic only */
  GBS_PREC_FX = 5,         /* fixed point, 224-bit integers on the integer pipe:
                              160 fraction bits, range +-2^63; real basis only, and
                              only where the state bounds every value of the tree
                              (otherwise GBS_EPRECISION, or TD under AUTO) */
  GBS_PREC_FXW = 6,        /* wide fixed point, 256-bit integers: 192 fraction bits,
                              same range and conditions as GBS_PREC_FX */
  GBS_PREC_FP64P = 7,      /* FP64 with the last two levels of the subset tree summed
                              in a cancellation-free form: each group of four subsets
                              that differ only in the last two modes adds one value
                              whose factors carry small relative errors, so the
                              error estimate follows the groups' magnitudes instead of
                              the terms' (1e2..1e3 smaller on Haar states).  Real
                              basis; Torontonians only (not the sampler's split sums).
                              abs_sum / kappa then refer to the group magnitudes. */
  GBS_PREC_FXN = 8         /* narrow fixed point, 160-bit integers: 128 fraction bits,
                              same range and conditions as GBS_PREC_FX, ~0.7x its
                              integer work; tried before FX where a prediction of the
                              cancellation says it suffices */
} gbs_prec;

/* Basis of the matrices the enumeration factors.  Both give identical
 * determinants (the per-mode change of basis is unitary); the real one needs
 * a quarter of the floating-point work. */
typedef enum { GBS_BASIS_AUTO = 0, GBS_BASIS_REAL = 1, GBS_BASIS_COMPLEX = 2 } gbs_basis;

typedef struct gbs_ctx gbs_ctx;
typedef struct gbs_state gbs_state;

/* Result of a probability evaluation. */
typedef struct {
  double p_hi, p_lo;     /* p(S) = p_hi + p_lo */
  double tor[3];         /* Tor(O_S) = tor[0] + tor[1] + tor[2] */
  double abs_sum;        /* sum over the 2^N subsets of |term| */
  double kappa;          /* cancellation ratio abs_sum / |Tor| */
  double err_bound;      /* estimated absolute error of p (model: 4 N u abs_sum / sqrt(det Sigma)) */
  double logdet_sigma;   /* log det Sigma of the state */
  int prec_used;         /* gbs_prec that produced the value */
  int basis_used;        /* gbs_basis that produced the value */
  int status;            /* GBS_OK, or GBS_ENOTPD for this request */
} gbs_prob;

/* ------------------------------------------------------------ context -- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the device
 * memory the context may hold (0 = no bound); allocations beyond it fail with
 * GBS_ENOMEM.  The context owns a CUDA stream unless gbs_ctx_set_stream is used. */
gbs_status gbs_ctx_create(gbs_ctx** ctx, int device, size_t hbm_budget_bytes);
void gbs_ctx_destroy(gbs_ctx* ctx);
/* Run all later work of the context on `cuda_stream` (a cudaStream_t, borrowed). */
gbs_status gbs_ctx_set_stream(gbs_ctx* ctx, void* cuda_stream);
const char* gbs_ctx_last_error(const gbs_ctx* ctx);
const char* gbs_status_string(gbs_status st);
/* Device bytes currently held by the context and its states. */
size_t gbs_ctx_bytes_in_use(const gbs_ctx* ctx);
/* Kernel launches made by the context so far (all entry points). */
long long gbs_ctx_launch_count(const gbs_ctx* ctx);
/* When enabled, the subset-enumeration kernel of every Torontonian is bracketed
 * by CUDA events on the context stream; gbs_ctx_kernel_time returns the summed
 * device time (ms) and the number of timed launches, and resets them. */
gbs_status gbs_ctx_enable_timing(gbs_ctx* ctx, int enable);
gbs_status gbs_ctx_kernel_time(gbs_ctx* ctx, double* total_ms, long long* launches);
/* Host gaps of the context: the summed wall time (s) from the return of each
 * host wait on the context stream (a synchronisation to read results back)
 * to the next kernel launch, while the stream sits empty, and the number of
 * such waits; both reset on read.  A lower bound on the device idle time the
 * host side causes (launches slower than the kernels they follow add more).
 * The paper has no counterpart. */
gbs_status gbs_ctx_host_gaps(gbs_ctx* ctx, double* seconds, long long* waits);

/* FP64 throughput of this GPU, measured now: a full grid of independent
 * dependent-FMA chains (no memory traffic), best of three timed launches on the
 * context stream.  *gflops receives the rate in GFLOP/s (one FMA = 2 flops).
 * The denominator of the FP64 roofline of the subset enumeration.  The paper
 * has no GPU counterpart; it reports CPU walltimes only (Sec. III, Table II). */
gbs_status gbs_measure_fp64_peak(gbs_ctx* ctx, double* gflops);

/* Fixed-point product throughput of this GPU, measured now: a full grid (16
 * warps per SM) of four independent chains of dependent products per thread,
 * in the FX entry type (six 32-bit limbs, 160 fraction bits: 26 partial
 * products of 32 x 32 bits each), no memory traffic, best of three timed
 * launches on the context stream.  *products_per_s receives products per
 * second.  The denominator of the integer-pipe roofline of the fixed-point
 * trees, whose work is counted in these products (the paper's quadruple
 * precision of Sec. III A, carried out in integer arithmetic here). */
gbs_status gbs_measure_fx_peak(gbs_ctx* ctx, double* products_per_s);

/* -------------------------------------------------------------- states -- */

/* Build the state of M single-mode squeezers r[0..M-1] followed by the M x M
 * interferometer U (complex, row-major) and uniform loss with transmissivity
 * eta in (0, 1].  Paper Sec. II (Eq. 1) for the state, Sec. III ("8 dB of
 * squeezing", Haar-random unitaries) for the inputs, Sec. IV for losses.
 *   V = S S^+ / 2,  S = [[U ch R, U sh R], [U* sh R, U* ch R]],  R = diag(r),
 *   then V <- eta V + (1 - eta) I/2.
 * V_out (may be NULL): caller-owned 2M x 2M complex, receives V in block order.
 * *st receives a library-owned handle keeping U, r, eta on the device (16 M^2
 * bytes); V itself (64 M^2 bytes) is built on the device when first needed
 * (V_out, sampling).
 * Errors: GBS_EINVAL (M < 1, eta outside (0, 1], non-finite input),
 * GBS_ENOMEM, GBS_ECUDA. */
gbs_status gbs_build_state(gbs_ctx* ctx, int M, const double* U, const double* r, double eta, double* V_out,
                           gbs_state** st);

/* A state given only by its 2M x 2M complex covariance V (block order, host).
 * Sigma = V + I/2 is inverted once on the device (Gauss-Jordan, FP64).
 * Errors: GBS_EINVAL, GBS_ENOTPD (Sigma not positive definite), GBS_ENOMEM. */
gbs_status gbs_state_from_V(gbs_ctx* ctx, int M, const double* V, gbs_state** st);
void gbs_state_free(gbs_state* st);
/* Number of modes and log det Sigma of a state. */
gbs_status gbs_state_info(const gbs_state* st, int* M, double* logdet_sigma);

/* (Sigma^-1)_S for the N modes `modes` (distinct, in [0, M)), mode-interleaved:
 * rows/columns 2i, 2i+1 belong to modes[i].  basis GBS_BASIS_COMPLEX gives the
 * (a_j, a_j^+) rows, 2N x 2N complex (8 N^2 doubles); GBS_BASIS_REAL the
 * (x_j, p_j) rows, 2N x 2N real (4 N^2 doubles).  H_out is caller-owned host
 * memory.  For states built from (U, r, eta) this is the closed form
 * Sigma^-1 = E diag(1/d) E^+ restricted to S (O(N^2 M) work). */
gbs_status gbs_sigma_inv_block(gbs_ctx* ctx, const gbs_state* st, const int* modes, int N, int basis,
                               double* H_out);

/* --------------------------------------------------------- probabilities -- */

/* Click probability of the pattern "clicks on modes[0..N-1], no click on every
 * other mode of the state", p = Tor(O_S)/sqrt(det Sigma).  The 2^N subset
 * determinants run on the GPU (decision tree with shared-prefix Schur
 * complements), the alternating sum is accumulated in double-double (or
 * triple-double).  prec: gbs_prec; basis: gbs_basis; out: caller-owned.
 * rel_tol (<= 0 means 1e-10) is the target relative error for GBS_PREC_AUTO.
 * Errors: GBS_EINVAL (N < 0 or N > 32, repeated or out-of-range modes),
 * GBS_ENOTPD, GBS_EPRECISION (AUTO could not meet rel_tol even on its last rung --
 * FXW where the state bounds the fixed-point tree, TD otherwise; *out then holds
 * that value), GBS_ENOMEM, GBS_ECUDA. */
gbs_status gbs_torontonian(gbs_ctx* ctx, const gbs_state* st, const int* modes, int N, int prec, int basis,
                           double rel_tol, gbs_prob* out);

/* Click probabilities of n_req requests in one batch: request i asks for the
 * pattern modes[off_i .. off_i + N_per[i]) on states[i] (off_i = sum of the
 * earlier N_per).  The requests may differ in state, M, N and loss; all their
 * subset trees run together (one plan, one launch per tree level over the whole
 * batch), and each result is bitwise the same as when evaluated alone.
 * prec, basis, rel_tol as for gbs_torontonian (AUTO escalates per request).
 * out: caller-owned array of n_req results; out[i].status flags GBS_ENOTPD per
 * request.  Returns the first error; GBS_EPRECISION if some request stayed
 * above rel_tol in TD (its result is still filled in). */
gbs_status gbs_torontonian_batch(gbs_ctx* ctx, int n_req, const gbs_state* const* states, const int* modes,
                                 const int* N_per, int prec, int basis, double rel_tol, gbs_prob* out);

/* ------------------------------------------------------------ sampling -- */

typedef struct {
  long long steps;        /* no-click probabilities evaluated (one subset tree each) */
  long long escalations;  /* trees repeated at a wider precision after the error check */
  long long near_ties;    /* coin draws with |u - p0| < 1e-9 */
  long long rejections;   /* trajectories abandoned by postselection (each may retry) */
  double seconds;         /* wall time of the call */
  long long trees[6];     /* subset trees evaluated in FP64, DD, TD, FX, FXW, FXN */
  double tree_seconds[6]; /* wall time spent in those tree batches */
  double cond_seconds;    /* wall time of gathers, decisions and conditioning */
  long long uncertified;  /* steps whose p0 error bound stayed above 5e-10 even in TD */
} gbs_sample_stats;

/* Chain-rule threshold-detector samples (the paper's Sec. II algorithm in
 * closed form).  Modes are measured from M-1 down to 0; at each step the
 * probability p0 that the mode stays dark given the outcomes so far is one
 * subset tree over the clicked modes plus the current one (on Sigma conditioned
 * on the dark modes, Eq. 4a in Sigma form), and the mode stays dark iff
 * u < p0 with u = (SplitMix64 output 1 + step + 2^20 (attempt + 2^12 sample) of
 * the stream with state `seed`) >> 11 * 2^-53, where step = M-1-mode.
 *   n_samples      number of samples (trajectories run together);
 *   N_post         0: no postselection; > 0: keep only samples with exactly N_post
 *                  clicks -- a trajectory is abandoned as soon as it has more, or
 *                  can no longer reach N_post, and restarts with attempt + 1;
 *   max_attempts   attempts per sample (>= 1); a sample that exhausts them is
 *                  left as 0xFF in `patterns` and the call returns GBS_EREJECT;
 *   forced_clicks  NULL, or n_samples x N_post click modes: the paper's forced-
 *                  outcome benchmark (Sec. III B) -- the outcome of every step is
 *                  preset (click iff the mode is listed) while p0 is still
 *                  evaluated at every step;
 *   prec           GBS_PREC_AUTO (per trajectory and step, the cheapest of FP64 /
 *                  FX / FXW / TD keeping the estimated error of p0 below 5e-10,
 *                  half the near-tie threshold) or a fixed FP64 / DD / TD / FX / FXW;
 *   patterns       caller-owned n_samples x M bytes (1 = click);
 *   p0_out         NULL or caller-owned n_samples x M doubles, p0 of step s of
 *                  sample i at [i * M + s] (last attempt);
 *   stats          NULL or caller-owned.
 * At most 31 clicks per trajectory (a free trajectory that exceeds it is treated
 * as rejected).  Device memory: 32 M^2 bytes per sample for its conditioned
 * Sigma.  Errors: GBS_EINVAL, GBS_EREJECT, GBS_ENOMEM, GBS_ENOTPD, GBS_ECUDA. */
gbs_status gbs_sample(gbs_ctx* ctx, const gbs_state* st, int n_samples, uint64_t seed, int N_post, int max_attempts,
                      const int* forced_clicks, int prec, uint8_t* patterns, double* p0_out,
                      gbs_sample_stats* stats);

/* The paper's forced-outcome benchmark with the click positions drawn from the
 * seed (Sec. III B: the walltime runs force the clicks on chosen modes and time
 * the chain, which still evaluates p0 at every step): sample i is forced to
 * click on the n_clicks modes gbs_draw_click_positions gives for it, then run as
 * gbs_sample with those positions (one attempt).  Arguments and errors as for
 * gbs_sample (1 <= n_clicks <= 31). */
gbs_status gbs_sample_forced_random(gbs_ctx* ctx, const gbs_state* st, int n_samples, uint64_t seed, int n_clicks,
                                    int prec, uint8_t* patterns, double* p0_out, gbs_sample_stats* stats);

/* The click positions gbs_sample_forced_random uses (host only, no GPU): for
 * sample i, n_clicks distinct modes of M from a partial Fisher-Yates shuffle
 * driven by outputs i*n_clicks + 1 .. (i+1)*n_clicks of the SplitMix64 stream
 * (Steele, Lea, Flood 2014) with state mix64(seed * 0x9E3779B97F4A7C15 +
 * 6 * 0xD1B54A32D192ED03): draw c picks index c + floor(u (M - c)), u the top 53
 * bits of the output times 2^-53; each sample's modes are returned sorted.
 * out: caller-owned n_samples x n_clicks ints.  Errors: GBS_EINVAL. */
gbs_status gbs_draw_click_positions(int M, int n_clicks, uint64_t seed, int n_samples, int* out);

/* ---------------------------------------------------------- request loop -- */

typedef enum { GBS_REQ_PROB = 0, GBS_REQ_SAMPLE = 1 } gbs_req_kind;

typedef struct {
  int kind;                /* gbs_req_kind */
  const gbs_state* state;  /* must stay alive until the request is polled */
  int N;                   /* PROB: click count; SAMPLE: N_post (0 = no postselection) */
  const int* modes;        /* PROB: the N click modes (copied by gbs_submit) */
  uint64_t seed;           /* SAMPLE: coin stream seed (as gbs_sample) */
  int sample_index;        /* SAMPLE: sample index of the coin counter, 0 <= index < 2^20 */
  int max_attempts;        /* SAMPLE: postselection attempts (>= 1) */
  int prec;                /* gbs_prec (SAMPLE: AUTO, FP64, DD, TD, FX or FXW) */
  int basis;               /* PROB: gbs_basis */
  double rel_tol;          /* PROB: as gbs_torontonian */
} gbs_request;

typedef struct {
  int status;              /* GBS_OK, GBS_EREJECT (attempts exhausted), GBS_EPRECISION, GBS_ENOTPD, ... */
  int kind;
  gbs_prob prob;           /* PROB */
  int n_clicks;            /* SAMPLE: clicked modes (at most 31) */
  int clicks[64];
  int attempts;            /* SAMPLE: attempts used */
  double latency_s;        /* submit -> completion */
  double queue_s;          /* submit -> admission */
} gbs_result;

typedef struct {
  long long submitted, completed, refused, active, queued;
  double p50_s, p99_s, mean_s;  /* latency percentiles of completed requests */
  double busy_s, wall_s;        /* time the loop spent working / since start */
  size_t arena_bytes, arena_in_use;
  int last_error;
} gbs_server_stats;

/* Start the context's request loop: a worker thread that admits submitted
 * requests in arrival order while their device footprint fits an arena of
 * arena_bytes (allocated now; a sampling request needs 32 M^2 bytes plus about
 * 32 M per attempt slot, a probability request only the shared tree
 * workspace) and at most max_active sampling requests run at once.  Each loop
 * iteration evaluates all newly admitted probability requests as one batch and
 * advances every running sampling attempt by one measured mode, all their
 * subset trees batched together, so late arrivals join running work at the
 * next step.  attempt_width (1..64): postselection attempts a sampling request
 * runs at once (attempts a, a+1, ... on separate trajectories); its result is
 * still the lowest accepted attempt, the one attempts run one after another
 * give, so a result is bitwise the same alone, in any mix and at any width.
 * While the loop runs, direct calls on the same context still work (they
 * interleave with loop iterations).
 * The paper has no counterpart (its runs were single jobs, Sec. III-IV). */
gbs_status gbs_server_start(gbs_ctx* ctx, size_t arena_bytes, int max_active, int attempt_width);
/* Stop the loop (waits for the current iteration); unpolled results are dropped. */
gbs_status gbs_server_stop(gbs_ctx* ctx);
/* Queue a request; *ticket identifies it.  Errors: GBS_EINVAL (loop not running,
 * bad descriptor), GBS_ENOMEM (footprint larger than the whole arena). */
gbs_status gbs_submit(gbs_ctx* ctx, const gbs_request* req, uint64_t* ticket);
/* Wait up to timeout_us microseconds for a ticket (0: do not wait; < 0: until
 * done, but at most 10 minutes).  GBS_OK: *out holds the result (its own status
 * in out->status) and the ticket is consumed; GBS_PENDING: not finished within
 * a bound the caller gave; GBS_ETIMEDOUT: not finished within the 10 minutes of
 * a negative bound (the ticket stays valid); GBS_ENOTFOUND: unknown or already
 * consumed ticket. */
gbs_status gbs_poll(gbs_ctx* ctx, uint64_t ticket, gbs_result* out, int64_t timeout_us);
gbs_status gbs_server_stats_get(gbs_ctx* ctx, gbs_server_stats* out);

/* Launch shape of the batched enumeration, per (precision, basis):
 *   sub_e          0..7: levels a subtree CTA (2^sub_e threads, at least one
 *                  warp, so 32 >> sub_e roots at once below 5) expands in
 *                  shared memory before its threads run the register
 *                  depth-first leaves (0 = no in-CTA expansion, one thread per
 *                  leaf root);
 *   d_top          prefix depth the first kernel reaches by eliminating each
 *                  node's included prefix modes in shared memory;
 *   grid_per_sm    0 = one CTA per work unit; k > 0 = persistent grid of k CTAs
 *                  per SM looping over the work units;
 *   level_threads  target threads per breadth-first level launch (sets how
 *                  many rows of a node one thread updates);
 *   q_drop         0..2: register depth-first levels below the variant's
 *                  maximum (fewer registers per thread, more warps per SM);
 *   mid_e          0..8: levels each first-kernel CTA goes on expanding in
 *                  shared memory after its prefix (replacing that many
 *                  breadth-first level launches; reduced to fit 200 KB).
 * gbs_autotune times candidate shapes on a synthetic batch of n_trees (1..64)
 * trees of n, n-1, ... modes (6 <= n <= 28; a workload of uneven trees tunes
 * best on a batch that resembles it)
 * on the context stream and keeps the fastest for later calls; report (may be
 * NULL) receives the timings as a JSON array, truncated to report_len bytes.
 * The paper has no counterpart (its Titan runs used MPI + OpenMP, Sec. III). */
gbs_status gbs_autotune(gbs_ctx* ctx, int prec, int basis, int n, int n_trees, char* report, size_t report_len);
gbs_status gbs_get_tuning(gbs_ctx* ctx, int prec, int basis, int* sub_e, int* d_top, int* grid_per_sm,
                          long long* level_threads, int* q_drop, int* mid_e);
gbs_status gbs_set_tuning(gbs_ctx* ctx, int prec, int basis, int sub_e, int d_top, int grid_per_sm,
                          long long level_threads, int q_drop, int mid_e);

/* Signed subset sum of an explicit matrix, the enumeration alone:
 *   tor = sum over Z subset {0..n-1} of (-1)^(n-|Z|) det(G_Z)^(-1/2)
 * split as tor = inc + exc by whether Z contains mode n-1, and abs_sum =
 * sum of |terms|.  G: host, 2n x 2n, mode i on rows/columns 2i, 2i+1; complex
 * interleaved (basis GBS_BASIS_COMPLEX) or real (GBS_BASIS_REAL), Hermitian /
 * symmetric positive definite (only the lower triangle is read).
 * inc, exc, tor: caller-owned double[3] each (may be NULL), unevaluated sums.
 * prec must not be GBS_PREC_AUTO; GBS_PREC_FX / FXW need the real basis and a matrix
 * whose eigenvalues lie in [2^-8, 64] with (1 + 1/lambda_min)^n < 2^60
 * (checked on the host; otherwise GBS_EPRECISION).  GBS_PREC_FP64P (real basis)
 * returns the whole sum in inc and zero in exc, and abs_sum is the sum of the
 * group magnitudes.
 * Errors: GBS_EINVAL, GBS_ENOTPD, GBS_EPRECISION, GBS_ECUDA. */
gbs_status gbs_subset_sum(gbs_ctx* ctx, int n, const double* G, int basis, int prec, double* inc, double* exc,
                          double* tor, double* abs_sum);

/* ------------------------------------------------------- no allocation -- */

/* Largest n accepted by gbs_subset_sum_static, and the size of the device
 * array it works in. */
#define GBS_STATIC_MAX_N 19
#define GBS_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

/* gbs_subset_sum for FP64, real basis, that allocates no memory at all.
 * The paper has no counterpart; this exists for callers that cannot call
 * cudaMalloc / cudaFree: cudaFree synchronises the whole device (fatal to a
 * loop that overlaps work on several streams), memory owned by another
 * allocator or a fixed pool must not be bypassed, and memory sized up front
 * must not hit an allocation that can fail later.  The caller passes device
 * buffers; the intermediate data (tree levels, partial sums, a status word)
 * live in one file-scope __device__ array of GBS_STATIC_SCRATCH_BYTES, which
 * every GPU that loads this library holds until the process exits.
 *   G_dev   device, 2n x 2n real symmetric positive definite, row-major, mode i
 *           on rows/columns 2i, 2i+1 (the lower triangle is read);
 *   n       number of modes, 1 <= n <= GBS_STATIC_MAX_N (larger n: GBS_EINVAL,
 *           nothing is launched);
 *   out_dev device, 8 doubles: {tor_hi, tor_lo, inc_hi, inc_lo, exc_hi, exc_lo,
 *           abs_sum, status}, with tor = inc + exc as in gbs_subset_sum and
 *           status 0, or 3 (GBS_ENOTPD) when a pivot block was not positive
 *           definite (then the sums are meaningless);
 *   cuda_stream  the cudaStream_t the work is queued on (0 = legacy default).
 * The call is asynchronous: it returns after queueing (GBS_OK), GBS_EINVAL or
 * GBS_ECUDA (one of its launches failed, or the device array could not be
 * located).  A CUDA error that earlier work left pending is reported as
 * GBS_ECUDA before anything is queued, and is not cleared.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life
 * of the process; make that first call before any stream capture, and do not
 * call this entry point on a device after a cudaDeviceReset of it.  All calls
 * share the one array and each leaves its data there: calls that can overlap
 * on the GPU race and must be ordered by the caller (one stream, or events). */
gbs_status gbs_subset_sum_static(const double* G_dev, int n, double* out_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GBS_H_ */
