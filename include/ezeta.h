/*
 * ezeta.h -- C ABI of the GB300 (sm_103a) Epstein zeta library.
 *
 * Implements the data-parallel path of "Epstein zeta method for many-body
 * lattice sums" (Buchheit & Busse): the Epstein zeta function evaluated by its
 * incomplete-gamma splitting, the n-body zeta function through the Epstein
 * representation theorem with the Duffy transformation, the singular split of
 * Sec. 3 with its eps-split/Taylor/Hadamard meromorphic continuation, and the
 * ATM energy of the Proposition in Sec. 2.
 *
 * General rules for every entry point:
 *  - Lattice matrices are row-major d x d (A[i*d+j] = component i of basis
 *    vector j); the lattice is A Z^d and the reciprocal lattice A^{-T} Z^d
 *    (Def. "Lattices").  1 <= d <= 3 for the lattice sums (Duffy nodes, near part,
 *    serving); the Epstein zeta function alone takes 1 <= d <= 6 (Sec. 6: the method
 *    holds in any dimension).
 *  - Pointers marked "host or device" may point to host memory or to device
 *    memory of the current CUDA device; the library detects which.  The caller
 *    owns every input and output buffer.  Library handles own their own device
 *    tables and scratch.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  When an output
 *    is host memory the call synchronises that stream before returning; when all
 *    outputs are device memory the call is asynchronous on `stream`.
 *  - Return value: EZ_OK or one of the error codes below; ez_last_error()
 *    returns a thread-local message for the last failure.  No C++ exception
 *    crosses the ABI and no device code traps or asserts.
 *  - A handle may be used by one host thread at a time.
 */
#ifndef EZETA_H
#define EZETA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EZ_OK 0
#define EZ_EINVAL 1        /* bad argument: d, singular A, n, node counts, NULL pointer */
#define EZ_EDOMAIN 2       /* pole: Gamma(nu/2) pole (nu in -2N0), y in Lambda* with nu <= d,  \
                              or a Hadamard exponent mu + 2k = 0 */
#define EZ_EUNSUPPORTED 3  /* a feature this entry point does not have (e.g. EZ_MIXED in ez_epstein_zeta) */
#define EZ_ENOMEM 4        /* device allocation failed */
#define EZ_ECUDA 5         /* CUDA runtime error */
#define EZ_ETIMEOUT 6      /* a bounded device or host wait ran out */
#define EZ_EBUSY 7         /* serving queue full */

#define EZ_MAX_NU 8   /* distinct exponents per sum */
#define EZ_MAX_PROD 4 /* products per sum (ATM uses 3) */

typedef struct ez_lattice_s* ez_lattice;

typedef enum {
  EZ_FP64 = 0,  /* every operation in IEEE binary64 */
  EZ_MIXED = 1  /* Gaussian-decaying tail terms in binary32 with compensated sums;
                   leading terms, singular parts and reductions in binary64 */
} ez_precision;

/* Quadrature and truncation of one lattice sum.  Zero fields take the defaults. */
typedef struct {
  int n_u;        /* u_rule 1: Gauss-Legendre nodes on [0, 1/2];
                     u_rule 2: nodes per graded panel [eps,2eps],[2eps,4eps],..,[.,1/2] */
  int n_v;        /* Gauss-Legendre nodes per v axis, v in [0,1]^{d-1} (ignored for d=1) */
  int u_rule;     /* 0: 2 if some nu_i < d or nu_i - d in 2N0, else 1 */
  double eps;     /* split point of the near part (default 1e-2, Sec. 4.1) */
  int ell;        /* Taylor order 2*ell of Z^reg in the near part (default 4, Sec. 4.1) */
  double lambda;  /* splitting parameter of the incomplete-gamma form; 0 = default: 2 V (d = 1),
                     3 V^{1/2} (d = 2), 4.5 V^{1/3} (d = 3, EZ_FP64) or 4 V^{1/3} (d = 3, EZ_MIXED),
                     lowered if needed so that the real-space box half-width stays <= 16.  The sum
                     does not depend on it (Crandall's formula, Sec. 2); ez_epstein_zeta uses V^{1/d} */
  double r_real;  /* real-space cutoff |z| <= r_real (default sqrt(T/pi) lambda, T = 45 for
                     EZ_FP64, 36 for EZ_MIXED) */
  double r_recip; /* reciprocal cutoff |g + k| <= r_recip (default sqrt(T/pi) / lambda) */
  int prec;       /* ez_precision */
  int dedupe;     /* 1: one Epstein zeta evaluation per distinct nu and node (default);
                     0: one evaluation per factor (n <= EZ_MAX_NU) */
  int part;       /* n_parts > 1: only part `part` (0 <= part < n_parts) of the sum: a contiguous
                     range of its Duffy lines (sector, u node) for d <= 2, of its line groups
                     (the four sectors 4 j .. 4 j + 3 of one axis j, u node) for d = 3, the
                     near part in part 0.  The values of the n_parts parts add up to the whole
                     sum (to rounding), so one sum can be split over several GPUs or streams;
                     0 and 0 (or n_parts <= 1): the whole sum */
  int n_parts;
} ez_quadrature;

/* Fills *q with the defaults (n_u = 32, n_v = 32, u_rule 0, eps 1e-2, ell 4, lambda 0,
 * cutoffs 0, EZ_FP64, dedupe 1, the whole sum). */
void ez_quadrature_default(ez_quadrature* q);

/* One lattice sum: product p = prod_j Z_{nu_j}(k)^{expo[p][j]} integrated over the
 * Brillouin zone (Thm "Epstein representation"): value_p = V int_BZ product_p dk. */
typedef struct {
  int n_distinct;
  double nu[EZ_MAX_NU];
  int n_prod;
  int expo[EZ_MAX_PROD][EZ_MAX_NU];
} ez_sum_spec;

/* --- lattices (Def. "Lattices") ------------------------------------------------ */
/* Creates the lattice (scale A) Z^d from A (host, d*d doubles, row-major as above) and the
 * lattice constant scale > 0 (1 for A itself; the presets of the paper are given at unit
 * density and scaled by it).  EZ_EINVAL if d is not in 1..6, scale is not a positive finite
 * number or A is singular.  The handle keeps the scaled matrix, its inverse and volume.
 * Every lattice-sum entry point (ez_lattice_sums, ez_batch_create, ez_lattice_sum_nbody,
 * ez_lattice_sum_adaptive, ez_atm_energy, ez_plan_describe) and ez_epstein_zeta_static
 * return EZ_EUNSUPPORTED for a lattice with d > 3. */
int ez_lattice_create(int d, const double* A, double scale, ez_lattice* out);
int ez_lattice_destroy(ez_lattice lat);

/* --- Epstein zeta function (Def. "Epstein zeta function") -------------------- */
/* Z_{Lambda,nu}(x, y_i) for i < m, by the incomplete-gamma splitting with
 * parameter lambda = V^{1/d}: re[i] + i im[i] = sum'_{z} e^{-2 pi i z.y_i} |z - x|^{-nu},
 * meromorphically continued in nu.  nu is any real number (orders a = nu/2 and (d - nu)/2
 * of Gamma(a, t) need not be half-integers); nu in -2N0 is EZ_EDOMAIN.  prec must be EZ_FP64: this entry point has no
 * mixed-precision form, and EZ_MIXED returns EZ_EUNSUPPORTED (any other value EZ_EINVAL).
 *   x  : host, d doubles.
 *   y  : host or device, m*d doubles (point i at y[i*d .. i*d+d-1]).
 *   re, im : host or device, m doubles each (im may be NULL).
 * y_i in Lambda* with nu <= d is a pole: re[i] = im[i] = NaN and the call returns
 * EZ_EDOMAIN after finishing the other points.  m = 0 is a no-op.
 * d = 4..6: cutoffs pi |z - x|^2 / lambda^2 <= 45 and pi lambda^2 |g + y|^2 <= 45 (the
 * neglected terms are below e^{-45} ~ 3e-20 of the nearest ones); the real-space ball is
 * enumerated once per call and the reciprocal ball per point, and the call synchronises
 * `stream` once more to size its tables.  EZ_EINVAL if the bounding box of a ball needs
 * more than 63 lattice points along an axis (a very skewed basis; reduce it first). */
int ez_epstein_zeta(ez_lattice lat, double nu, const double* x, const double* y, size_t m,
                    double* re, double* im, int prec, void* stream);

/* Same values as ez_epstein_zeta, computed without allocating anything.  The paper
 * has no counterpart: this serves callers that cannot allocate device memory when
 * they need a value -- code running inside an allocator or a memory-pool callback,
 * real-time threads that must stay out of the driver's allocator (cudaMalloc can
 * synchronise the device and take locks), processes whose device memory is fully
 * reserved by another framework.  All scratch (descriptors, reciprocal-lattice
 * list, real-space box, Phi table, pole flag) lives in one static device array of
 * 256 KiB that every GPU loading this library holds until the process exits.
 *   y, re, im : DEVICE buffers only (EZ_EINVAL otherwise); x : host, d doubles.
 * A lattice/exponent whose tables exceed 256 KiB is rejected with EZ_EINVAL and a
 * message giving the size (use ez_epstein_zeta for it).  The first call on each
 * device resolves the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  Every call reuses the same array and leaves its
 * contents behind (the pole flag is cleared at the start of each call); calls that
 * overlap on the GPU -- other streams or other host threads -- race on it.  The call
 * synchronises `stream` to read the pole flag. */
int ez_epstein_zeta_static(ez_lattice lat, double nu, const double* x, const double* y, size_t m,
                           double* re, double* im, void* stream);

/* --- n-body zeta function (Def. "Many-body zeta function") ------------------- */
/* zeta^(n)_Lambda(nu_1..nu_n) through the Epstein representation and the Duffy
 * transformation (Cor. "Duffy transformation"), with the eps-split meromorphic
 * continuation of Sec. 3 when u_rule is 2.
 *   nu      : host, n real exponents (1 <= n <= 64; not in -2N0).  Unless every nu_i - d is a
 *             positive odd integer the default u rule is the eps-split (u_rule 2), whose near
 *             part integrates u^{mu-1} log^m in closed form; a product with some mu + 2k = 0
 *             (a pole of the closed form; the paper gives no formula for it) is EZ_EDOMAIN.
 *   value   : host or device, 1 double.
 *   err_est : host or device, 1 double, or NULL.  When given, the same sum is also
 *             computed on the embedded coarse rule -- ceil(n_u/2) u nodes per panel and
 *             ceil(n_v/2) v nodes per axis, same panels, near part, splitting parameter
 *             and cutoffs -- in the same launch, and *err_est = |value - coarse value|.
 *             Both Gauss-Legendre rules converge geometrically, so this bounds the far-
 *             field quadrature error of the coarse rule and overstates that of value; it
 *             does not include the lattice-sum truncation (below e^{-45}, or e^{-36} in the
 *             mixed form) or the near part's Taylor truncation (order 2 ell).  Costs about
 *             2^{-d} of the sum again.  NULL: no extra work.
 * Synchronises `stream`. */
int ez_lattice_sum_nbody(ez_lattice lat, const double* nu, int n, const ez_quadrature* q,
                         double* value, double* err_est, void* stream);

/* The far-field u integral by adaptive quadrature (Sec. 3: standard adaptive quadrature with
 * recursive interval subdivision), global and in rounds of one batched launch each.  Round 0
 * applies the q->n_u-point Gauss-Legendre rule to every starting panel: the graded panels
 * [eps, 2 eps], ..., [., 1/2] with the near part on (0, eps) when the u rule is the eps-split
 * (u_rule 2, or 0 resolving to it), else [0, 1/4] and [1/4, 1/2] (u_rule 1: the paper's plain
 * adaptive integration of the full u interval, for nu_i >= d).  Each later round evaluates the
 * two halves of every open panel; a panel closes with the value of its halves when
 * |Q(panel) - Q(halves)| <= tol x |running total| x (panel length / interval length) for every
 * product, else both halves stay open.  The v rule (q->n_v per axis), cutoffs, splitting
 * parameter, precision and near part are those of q (part/n_parts must be 0/1).
 *   tol        : relative tolerance in (0, 1);  max_rounds : 2..60 (open panels left after the
 *                last round count with their values and carried estimates)
 *   value      : host, spec->n_prod doubles;  err_est : host, spec->n_prod doubles or NULL
 *                (sum over closed panels of |Q(panel) - Q(halves)|: the coarse panels' errors)
 *   n_u_used   : host or NULL, u nodes evaluated over all rounds.
 * Synchronises `stream`; every round rebuilds the sum's tables. */
int ez_lattice_sum_adaptive(ez_lattice lat, const ez_sum_spec* spec, const ez_quadrature* q, double tol,
                            int max_rounds, double* value, double* err_est, long long* n_u_used, void* stream);

/* --- ATM cohesive energy (Prop. in Sec. 2) ------------------------------------ */
/* E = zeta(3,3,3)/24 - 3 zeta(-1,5,5)/16 + 3 zeta(1,3,5)/8; the three zeta^(3) are
 * computed in one pass over the nodes (distinct nu = -1, 1, 3, 5).
 *   energy : host, 1 double; parts : host, 3 doubles (may be NULL). */
int ez_atm_energy(ez_lattice lat, const ez_quadrature* q, double* energy, double* parts,
                  void* stream);

/* --- batched lattice sums ----------------------------------------------------- */
/* n_req sums in one pass: sum r uses lats[r], specs[r], quads[r] and writes
 * out[r*EZ_MAX_PROD + p] for p < specs[r].n_prod (host or device).
 * lines (optional, host or device): per-line partial sums, EZ_MAX_PROD doubles per
 * line; the lines of sum r are line_offsets[r] .. line_offsets[r+1]-1: first the
 * far-field lines in the order (sector, u node), then, for the eps-split rule, one
 * near-part line per sector.  The value of product p is the sum of its lines.
 * line_offsets (optional, host, n_req+1 entries).  Synchronises `stream`. */
int ez_lattice_sums(int n_req, const ez_lattice* lats, const ez_sum_spec* specs,
                    const ez_quadrature* quads, double* out, double* lines, long long* line_offsets,
                    void* stream);

/* A batch keeps the plans of n_req sums and the device memory of all their tables
 * and partial sums resident.  ez_batch_create plans, allocates (cudaMalloc and
 * pinned host staging, owned by the batch) and uploads the descriptors on
 * `stream`; it also creates a second CUDA stream and two events of its own, on which
 * the near part's setup of each run overlaps the rest of the setup (every run stays
 * ordered on the caller's stream; without them everything runs on it).  ez_batch_run launches every kernel of the path and writes
 * out[r*EZ_MAX_PROD + p] (host or device; with host memory
 * the call synchronises `stream`, with device memory it is asynchronous).
 * ez_batch_lines copies the per-line partial sums of the last run (layout as in
 * ez_lattice_sums); ez_batch_n_lines gives their count.  A batch may be run any
 * number of times, on one stream at a time.  Every run rebuilds the lattice tables
 * (reciprocal lists, real-space boxes, Taylor tensors); the tables of Phi_a(t), which
 * depend on the orders a alone, are filled by the first run and kept by the batch. */
typedef struct ez_batch_s* ez_batch;
int ez_batch_create(int n_req, const ez_lattice* lats, const ez_sum_spec* specs,
                    const ez_quadrature* quads, void* stream, ez_batch* out);
int ez_batch_run(ez_batch b, double* out, void* stream);
long long ez_batch_n_lines(ez_batch b);
int ez_batch_lines(ez_batch b, double* lines, long long* line_offsets, void* stream);
int ez_batch_destroy(ez_batch b);

/* Timing of batch runs with CUDA events recorded on the run's stream: after
 * ez_batch_timing(b, 1, ...) every run records events around its setup kernels,
 * its far-field kernels and its near-part/reduction kernels.  A later call
 * (enable 0 or 1) returns, for the last run, the milliseconds of the far-field
 * kernels (far_ms) and of the whole launch sequence (total_ms); it waits for
 * that run's last event. */
int ez_batch_timing(ez_batch b, int enable, float* far_ms, float* total_ms);

/* Algorithmic FP64 flops of the far-field kernels of the last run: every in-range
 * reciprocal term costs 3d - 1 flops for |g + k|^2 plus, per distinct exponent,
 * 2n + 1 for its Phi polynomial of n coefficients (n counted on the device: the
 * tables keep 4..16 coefficients per interval as accuracy needs), plus the fixed
 * per-node and per-block costs of the real-space contraction and bookkeeping.
 * terms / coefs (optional) receive the device counts.  Synchronous. */
int ez_batch_far_flops(ez_batch b, double* flops, long long* terms, long long* coefs);

/* Bytes of device memory owned by the batch and of its host staging (the bytes
 * uploaded by ez_batch_create and by every ez_lattice_sums call of the same sums). */
int ez_batch_sizes(ez_batch b, long long* device_bytes, long long* staging_bytes);

/* --- serving: continuous batching of lattice sums ---------------------------- */
/* A server owns a worker thread that turns a stream of requests into batched
 * launches.  Each "tick" is one batch (ez_batch semantics: all kernels of the path
 * for every admitted request, their nodes mixed in the same launches) on one of
 * n_streams CUDA streams with its own device memory; several ticks run on the GPU
 * at once.  Requests are admitted in FIFO order whenever a stream is free and the
 * device memory of all running ticks plus the new one fits mem_budget_bytes;
 * requests that arrive while others run are admitted into the next tick, so their
 * work overlaps with the running ones.  A request's result does not depend on which
 * other requests share its tick (every sum's items and reductions are its own).
 * Server time is CLOCK_MONOTONIC seconds. */
#define EZ_REQ_ERR_EST 1 /* ez_request.flags: also return an error estimate (see ez_result) */

typedef struct {
  int d;
  double A[9];            /* row-major d x d */
  ez_sum_spec spec;
  ez_quadrature quad;
  unsigned long long tag; /* caller's label, returned with the result */
  int flags;              /* 0 or EZ_REQ_ERR_EST */
} ez_request;

typedef struct {
  unsigned long long ticket, tag;
  int status;                 /* EZ_OK, or the error of this request (EZ_EDOMAIN, EZ_ENOMEM, ...) */
  double value[EZ_MAX_PROD];  /* value of each product of the spec */
  double t_submit, t_start, t_done;  /* submit, launch of its tick, completion seen by the worker */
  double err_est[EZ_MAX_PROD];  /* with EZ_REQ_ERR_EST: |value - value on the embedded coarse rule|,
                                   as ez_lattice_sum_nbody's err_est (the coarse sum runs in the same
                                   tick); NaN otherwise.  The mixed form's rounding adds at most its
                                   stated bound, 1e-10 relative. */
} ez_result;

typedef struct {
  long long submitted, completed, failed, ticks, max_batch_seen;
  double busy_seconds;        /* union of the intervals with at least one tick in flight */
  long long peak_device_bytes;
  /* resident tables: the incomplete-gamma table of each order a (Phi_a, tabulated in t, the
   * same for every lattice) is built once, by the first tick that needs it, and read by every
   * later tick: tables built and (tick, table) reuses */
  long long phi_tables_built, phi_tables_reused;
} ez_serve_stats;

#define EZ_SERVER_DRYRUN 1 /* plan and schedule without touching the GPU (values NaN) */

/* Device memory: every tick allocates its tables from a memory pool owned by the server, in
 * stream order, and returns them in stream order when its results have been copied out, so the
 * worker never synchronises the device; the pool keeps up to mem_budget_bytes for reuse.
 * Requests are planned by ez_server_submit on the caller's thread; the worker only launches.
 * mem_budget_bytes: device memory the server may hold for running ticks (> 0);
 * n_streams: concurrent ticks (1..16); max_batch: requests per tick (1..65536);
 * max_pending: queue capacity (ez_server_submit returns EZ_EBUSY beyond it). */
typedef struct ez_server_s* ez_server;
int ez_server_create(size_t mem_budget_bytes, int n_streams, int max_batch, int max_pending, int flags,
                     ez_server* out);
/* Copies the request (non-blocking).  Invalid d or singular A fail here (EZ_EINVAL);
 * other per-request errors come back in the result's status. */
int ez_server_submit(ez_server s, const ez_request* req, unsigned long long* ticket);
/* Moves up to max_results completed results into out (oldest first); *n_out gets the count. */
int ez_server_poll(ez_server s, ez_result* out, int max_results, int* n_out);
/* Waits up to timeout_ms for one ticket (EZ_ETIMEOUT if it has not completed; EZ_EINVAL for an
 * unknown or already collected ticket).  The result is removed from the server. */
int ez_server_wait(ez_server s, unsigned long long ticket, int timeout_ms, ez_result* out);
int ez_server_stats(ez_server s, ez_serve_stats* out);
/* Waits (bounded by timeout_ms) for the running ticks, then frees everything; pending
 * requests that never started are dropped.  EZ_ETIMEOUT if ticks were still running. */
int ez_server_destroy(ez_server s, int timeout_ms);

/* Number of Duffy sectors (d 2^{d-1}) and far-field u nodes for (d, q). */
int ez_layout(int d, const ez_sum_spec* spec, const ez_quadrature* q, int* n_sectors,
              int* n_u_total, int* u_rule_used);

/* Diagnostic (no counterpart in the paper): the plan the library makes for one sum --
 * splitting parameter, cutoffs, real-space box, block decomposition, this part's range of
 * far lines, mixed-form thresholds -- computed on the host (no GPU needed).  EZ_EINVAL /
 * EZ_EDOMAIN as ez_lattice_sums would return for the same arguments. */
typedef struct {
  double lambda, r_real, r_recip;
  int M[3];                 /* real-space box half-widths */
  int m_hp[3];              /* mixed form: terms with |m_i| >= m_hp[i] summed in plain binary32 */
  int n_sectors, n_u_total, u_rule;
  int vchunk, n_chunks;     /* d = 3: v2 rows per far-field block, blocks per line group */
  long long line_lo, line_hi; /* this part's far lines (d <= 2) or line groups (d = 3) */
  long long n_far_items;    /* far-field blocks of this part */
  size_t far_smem_bytes;    /* dynamic shared memory of one far-field block */
  float t_mix, t_mid;       /* mixed form: binary32 tails beyond t_mix, binary32 polynomial
                               beyond t_mid (3e38 in the FP64 form) */
  int n_alpha;              /* u_rule 2: Taylor multi-indices alpha of the near part (even
                               |alpha| <= 2 ell; only all-even alpha on a lattice that every
                               axis reflection x_i -> -x_i maps onto itself); 0 otherwise */
} ez_plan_info;
int ez_plan_describe(ez_lattice lat, const ez_sum_spec* spec, const ez_quadrature* q, ez_plan_info* out);

/* Diagnostic (no counterpart in the paper): sustained FP64 FMA throughput of the
 * current device in TFLOP/s, from a DFMA loop on every SM timed with CUDA events. */
int ez_diag_fp64_peak(double* tflops, void* stream);
/* The same for binary32 FMA (the pipe of the mixed form's tails and float-float arithmetic). */
int ez_diag_fp32_peak(double* tflops, void* stream);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* ez_last_error(void);

/* Number of kernels launched by this library on the calling thread since the
 * last reset (reset = 1 clears it). */
long long ez_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* EZETA_H */
