/*
 * hc.h — C-ABI of the GB300 homotopy-continuation path tracker (libhc.so).
 *
 * The library tracks many independent solution paths x(t) of a homotopy
 * H(x, t) from t = 0 to t = 1 on one GPU, the data-parallel method of
 * Chien et al., "GPU-Based Homotopy Continuation for Minimal Problems in
 * Computer Vision" (arXiv 2112.03444):
 *   - Sec. 3, Eq. 1: H(x,t) = (1-t) G(x) + t F(x); here (1-t) gamma G + t F
 *     with a random unit gamma for total-degree homotopies, or the parameter
 *     homotopy H(x,t) = F(x; (1-t) p0 + t p1) of Sec. 6 / Sec. 7 (start
 *     solutions at a generic parameter point p0, target parameters p1).
 *   - Sec. 3, Eqs. 2-4: predictor on dx/dt = -(dH/dx)^-1 dH/dt, with the
 *     4th-order Runge-Kutta method the paper names.
 *   - Sec. 3, Eqs. 5-6: Newton corrector at t + dt.
 *   - Sec. 6: per path, evaluation of H, dH/dx, dH/dt from the terms of the
 *     equations (each term's value and all its derivatives from one pass of
 *     prefix and suffix products), and a fused solve of the small dense
 *     complex system on the augmented matrix [A b] kept in registers, one
 *     matrix row per lane.
 *
 * The problem statement follows Sec. 3: N polynomial equations in N unknowns
 * (square systems), a start system whose solutions are all known, and the
 * homotopy joining them.  Inputs are coefficients or parameters, start
 * solutions and tracker settings; outputs are endpoints and per-path status.
 *
 * Threading: calls on different problems may come from different threads; a
 * single hc_problem or hc_batch must not be used from two threads at once.
 * All complex numbers are interleaved (re, im) pairs of double.
 */
#ifndef HC_H
#define HC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes of every call. */
typedef enum hc_status {
  HC_OK = 0,                /* success (for hc_poll: the batch is done)              */
  HC_PENDING = 1,           /* hc_poll: the batch is still running                   */
  HC_ERR_INVALID = -1,      /* a descriptor field is out of range or inconsistent    */
  HC_ERR_OOM = -2,          /* device or host allocation failed                      */
  HC_ERR_CUDA = -3,         /* a CUDA runtime call failed (see hc_last_error)         */
  HC_ERR_TIMEOUT = -4,      /* hc_poll: device step budget exhausted                 */
  HC_ERR_NUMERIC = -5,      /* non-finite coefficients or parameters in the input     */
  HC_ERR_BUSY = -6,         /* admission refused (memory cap) and blocking not asked */
  HC_ERR_UNSUPPORTED = -7   /* a problem shape this build has no kernel for          */
} hc_status;

/* Homotopy kinds (hc_problem_desc.kind). */
enum {
  HC_TOTAL_DEGREE = 0,  /* H = (1-t) gamma G + t F, G_i = x_i^{d_i} - 1, d_i = deg F_i */
  HC_PARAMETER = 1,     /* H = F(x; (1-t) p0 + t p1), start solutions given at p0      */
  HC_COEFFICIENT = 2    /* H = sum_k ((1-t) c_k(p0) + t c_k(p1)) x^a_k, c_k(p) the term
                           coefficient at parameters p: the coefficients themselves
                           interpolated, as Sec. 6 states; same inputs as
                           HC_PARAMETER (the two agree when every coefficient is
                           linear in the parameters)                              */
};

/* Tracking precision (hc_settings.precision). */
enum {
  HC_PREC_FP64 = 0,   /* every step in complex FP64 (the plain reference form)         */
  HC_PREC_MIXED = 1,  /* complex FP32 predictor and corrector; FP64 state x in the
                         endgame (t > t_endgame) with double-float corrector
                         residuals (FP64 after a rejected step there), FP64
                         residuals in the final Newton refinement; colliding
                         endpoints (path jumps) and failed paths re-tracked with
                         high-precision residuals, then in the precision
                         retrack_precision names                               */
  HC_PREC_DF = 2      /* FP64 state, time and step control as HC_PREC_FP64; the
                         evaluation of H, Hx, Ht and the solve in complex
                         double-float arithmetic (pairs of FP32 numbers, about
                         48 significant bits, FP32's exponent range) on the
                         FP32 pipe; the corrector's residual from that
                         evaluation until a step of the path is rejected, in
                         FP64 after; FP64 refinement residuals and backward
                         error.  Dense systems track one path per warp.       */
};

/* Per-path status codes (hc_batch_desc.status_out).  HC_PATH_REAL is or-ed
 * into HC_PATH_FINITE when the endpoint is real within real_tol. */
enum {
  HC_PATH_NONE = 0,          /* not tracked (step budget exhausted)            */
  HC_PATH_FINITE = 1,        /* nonsingular finite endpoint, backward error ok */
  HC_PATH_DIVERGED = 2,      /* |x|_inf exceeded r_inf                          */
  HC_PATH_FAIL_STEP = 3,     /* step size fell below dt_min                     */
  HC_PATH_FAIL_MAXSTEPS = 4, /* max_steps reached                               */
  HC_PATH_FAIL_NAN = 5,      /* non-finite state                                */
  HC_PATH_SINGULAR = 6,      /* endpoint found but cond_1(dF/dx) > singular_cond */
  HC_PATH_FAIL_REFINE = 7,   /* refinement left backward error > finite_tol     */
  HC_PATH_REAL = 0x80
};

/* Flags of hc_batch_desc.flags. */
enum {
  HC_DEVICE_PTRS = 1u << 0,  /* coef/p1 and every output pointer are device memory
                                on the current device; otherwise they are host memory
                                and the library stages the copies on the stream     */
  HC_BLOCKING_ADMIT = 1u << 1 /* wait for memory instead of returning HC_ERR_BUSY    */
};

/*
 * Tracker settings.  The paper (Sec. 3) fixes the predictor and corrector but
 * is silent on step control, tolerances, the endgame and classification; these
 * fields are this library's reading.  Defaults: hc_default_settings().
 *
 * Step rule: a step of size h from t is accepted iff Newton at t + h
 * converges (|dx|_inf <= newton_tol * (1 + |x|_inf)) within max_newton
 * iterations and the first correction is at most max_first_corr * (1 + |x|);
 * after grow_after consecutive accepts dt doubles (capped at dt_max); on a
 * reject dt halves; dt < dt_min fails the path.
 */
typedef struct hc_settings {
  double dt_min;          /* 1e-6 */
  double dt_max;          /* 0.05 */
  double dt_init;         /* 0.01 */
  double newton_tol;      /* FP64 corrector tolerance, 1e-8 */
  double newton_tol_fp32; /* FP32 corrector tolerance (mixed precision), 1e-4 */
  double max_first_corr;  /* 0.1 */
  double refine_tol;      /* endpoint refinement target, 1e-13 */
  double r_inf;           /* divergence radius, 1e8 */
  double finite_tol;      /* backward-error bound for a finite root, 1e-10 */
  double real_tol;        /* |Im x|_inf <= real_tol * max(1, |x|_inf), 1e-8 */
  double singular_cond;   /* cond_1 bound, 1e12 */
  double t_endgame;       /* mixed precision: FP64 residuals for t > t_endgame, 0.95 */
  double dt_min_fp32;     /* mixed precision: a path whose FP32 step falls below this
                             continues with FP64 state and FP64 residuals, 1e-4 */
  double max_first_corr_fp32; /* first-correction bound of the FP32 tier, 0.01 */
  int32_t max_steps_fp32; /* mixed precision: FP32-state steps before that switch, 2000 */
  int32_t max_newton;     /* 3 */
  int32_t max_steps;      /* 100000 (also the device step budget of one path) */
  int32_t grow_after;     /* 3 */
  int32_t refine_iters;   /* 8 */
  int32_t precision;      /* HC_PREC_MIXED */
  int32_t escalate;       /* 1: mixed-precision paths that fail or whose endpoints
                             collide are re-tracked (FP64 residuals, then FP64)     */
  int32_t lanes;          /* mixed precision: 0 = default group width (next power of two
                             >= n, at least 4), 32 = one path per warp (n <= 16)   */
  int32_t max_newton_ir;  /* mixed precision: corrector iterations allowed in the
                             FP64-residual mode, 6.  Its iterations solve with the
                             FP32 Jacobian and contract only linearly (about
                             cond * 6e-8 per iteration), so one exact Newton step
                             is worth about two of them                         */
  int32_t block_threads;  /* threads per block of the main tracking launch: 0 (the
                             default, 128), 32, 64 or 128; paths per block =
                             threads / lanes (the autotuner's block axis)       */
  /* Power-series endgame (Morgan, Sommese & Wampler 1992; the paper is
   * silent on endgames), off by default.  Past t = 1 - eg_s0 the step control
   * lands on the sample times 1 - eg_s0 eg_ratio^k (k < eg_samples); the cycle
   * number c (<= eg_cmax) comes from the ratio of successive sample
   * differences, and the endpoint is predicted by cubic Hermite
   * extrapolation to s = 0 in w = (1 - t)^(1/c) while the samples converge.
   * Two agreeing predictions with c > 1 end the path at the prediction,
   * HC_PATH_SINGULAR if its backward error passes; a step-size failure inside
   * the endgame takes the last such prediction.  Paths with c = 1 (nonsingular
   * endpoints) are tracked to t = 1 as without the endgame.  It runs in the
   * FP64-state kernels (precisions FP64 and DF, and the last re-tracking tier
   * of the mixed pipeline, which receives the paths that fail near their end). */
  int32_t endgame;        /* 0: off, 1: power-series endgame */
  int32_t eg_cmax;        /* 8 */
  int32_t eg_samples;     /* 40 */
  int32_t retrack_precision; /* precision of the last re-tracking tier of the mixed
                             pipeline: HC_PREC_DF (the default; GB300 issues FP64
                             at a small fraction of its FP32 rate) or
                             HC_PREC_FP64.  With the endgame on, that tier runs
                             in FP64 whatever this says: the endgame's
                             extrapolation uses dx/ds at its samples, which a
                             double-float solve near a multiple root gives
                             with about five bits less                       */
  double eg_s0;           /* 0.1 */
  double eg_ratio;        /* 0.5 */
  double eg_tol;          /* agreement of two predictions, relative: 1e-8 */
} hc_settings;

/*
 * Problem description (deep-copied by hc_create_problem; the caller may free
 * every buffer as soon as the call returns).
 *
 * The target system F is a list of n_terms terms; term k contributes
 *   term_coef[k] * prod_f p[term_param[k][f]] * x^term_exp[k]
 * to equation term_eq[k].  For HC_TOTAL_DEGREE the coefficients are given per
 * instance in hc_batch_desc.coef (term order) and term_coef is the default.
 */
typedef struct hc_problem_desc {
  int32_t n;                   /* unknowns = equations, 1..32                      */
  int32_t n_terms;             /* T >= n                                            */
  const int32_t* term_eq;      /* [T] equation index in [0, n)                     */
  const double* term_coef;     /* [T][2] complex scalar                             */
  const uint8_t* term_exp;     /* [T][n] exponents (total degree of a term <= 15)   */
  int32_t max_pfac;            /* parameter factors per term (0 for total degree)  */
  const int32_t* term_param;   /* [T][max_pfac] index in [0, n_params) or -1; may be
                                  NULL when max_pfac == 0                           */
  int32_t n_params;            /* HC_PARAMETER: length of p0 / p1                   */
  int32_t kind;                /* HC_TOTAL_DEGREE or HC_PARAMETER                   */
  double gamma[2];             /* HC_TOTAL_DEGREE: the constant gamma (unit modulus)*/
  const double* p0;            /* HC_PARAMETER: [n_params][2] start parameters      */
  int64_t n_start;             /* HC_PARAMETER: number of start solutions           */
  const double* start;         /* HC_PARAMETER: [n_start][n][2] start solutions     */
  hc_settings settings;
  /* HC_PARAMETER, optional: sign symmetries.  Symmetry k negates the unknowns
   * whose bits are set in sym_mask[k].  Allowed when every term has even
   * total degree in the unknowns of every mask (then H(D x, t) = H(x, t)
   * and the path from D s is D times the path from s, exactly in floating
   * point: negation is exact and the evaluation and the solve treat the
   * negated columns alike).  The start set must be closed under the masks.
   * The library then tracks one start per orbit and writes every orbit
   * member's endpoint as the signed image of its representative's; the
   * duplicate check compares endpoints up to the signs.  A batch with a
   * start subset tracks its starts without the reduction. */
  int32_t n_sym;               /* 0..4                                              */
  uint32_t sym_mask[4];
} hc_problem_desc;

typedef struct hc_problem hc_problem;  /* opaque */
typedef struct hc_batch hc_batch;      /* opaque */

/*
 * One batch (paper Sec. 3: the target systems F -- their coefficients, or the
 * target parameters p1 of Sec. 6 -- tracked from the start solutions of G;
 * Sec. 6: every path an independent work item): n_instances systems of the
 * problem's family tracked together in one persistent launch.
 *   HC_TOTAL_DEGREE: coef = [n_instances][T][2] doubles (NULL: every instance
 *                    uses the problem's term_coef); paths = prod_i d_i.
 *   HC_PARAMETER:    p1 = [n_instances][n_params][2] doubles (required);
 *                    paths = n_start.
 * Optional start subset: with n_subset > 0, instance k tracks only the
 * starts path_ids[k][0 .. n_subset) (host int64, each in [0, paths)) and
 * its outputs hold n_subset paths, in that order (P below = n_subset).
 * Optional step budget: with step_budget > 0 the batch starts no new path
 * once the paths it has finished took that many steps (accepted + rejected,
 * all tiers) in total; paths never started keep HC_PATH_NONE and hc_poll
 * returns HC_ERR_TIMEOUT (results of the finished paths are valid).  A path
 * that has started always finishes (its own limit is settings.max_steps).
 * Outputs (written by the library until hc_poll returns HC_OK), P = paths:
 *   x_out      [n_instances][P][n][2] double  endpoints after refinement
 *   status_out [n_instances][P] uint8         HC_PATH_* codes
 *   steps_out  [n_instances][P][3] int32      accepted, rejected steps,
 *                                              Newton iterations (optional)
 *   be_out     [n_instances][P] double        backward error (optional)
 * Without HC_DEVICE_PTRS the host buffers must stay valid until hc_poll
 * returns HC_OK; the library copies through device staging buffers on the
 * batch's stream.  path_ids is copied before hc_track_batch returns.
 */
typedef struct hc_batch_desc {
  int32_t n_instances;
  uint32_t flags;
  const double* coef;
  const double* p1;
  void* stream;                /* cudaStream_t; NULL = the legacy default stream */
  double* x_out;
  uint8_t* status_out;
  int32_t* steps_out;
  double* be_out;
  int64_t step_budget;         /* 0: none                                        */
  int32_t n_subset;            /* 0: every start path                             */
  int32_t reserved;            /* 0                                               */
  const int64_t* path_ids;     /* [n_instances][n_subset] (host), or NULL        */
} hc_batch_desc;

/* Summary filled by hc_poll when the batch is done. */
typedef struct hc_batch_result {
  int64_t paths;               /* n_instances * paths per instance            */
  int64_t finite, real, diverged, singular, failed;
  int64_t escalated;           /* mixed-precision re-tracks (both tiers)        */
  int64_t steps_accepted, steps_rejected, newton_iters;  /* all tiers        */
  int64_t esc_accepted, esc_rejected, esc_newton;        /* FP64 tier part   */
  double device_ms;            /* stream time from first copy to last copy      */
  double track_ms;             /* stream time of the tracking launch             */
  double escalate_ms;          /* stream time of the re-tracking launches        */
  int64_t untracked;           /* paths never started (step budget exhausted)    */
  int64_t steps_total;         /* steps counted against the step budget          */
} hc_batch_result;

/* Static description of an error code; never NULL.  (Library utility; the
 * paper defines no error reporting.) */
const char* hc_status_string(int32_t status);

/* Last CUDA or validation error message of the calling thread ("" if none).
 * (Library utility.) */
const char* hc_last_error(void);

/* Default settings (values listed in the hc_settings comments): the step
 * rule, tolerances and classification thresholds on which Sec. 3 is silent,
 * read by this library. */
hc_settings hc_default_settings(void);

/*
 * Sec. 3 (the square system F, the start system G with known solutions and
 * the homotopy H joining them) and Sec. 6 (the terms of the equations as the
 * evaluator's input): validate and deep-copy a problem; upload its encoded
 * form (term tables or dense coefficient maps) to the current device.  On
 * error *out is left untouched.  Errors: HC_ERR_INVALID (index
 * out of range, n outside 1..32, missing start data, unsupported degree),
 * HC_ERR_NUMERIC (non-finite data), HC_ERR_OOM, HC_ERR_CUDA.
 */
hc_status hc_create_problem(const hc_problem_desc* d, hc_problem** out);

/* Paths per instance of a problem (prod d_i, the Bezout number of the
 * total-degree start system, or n_start); -1 for NULL. */
int64_t hc_problem_paths(const hc_problem* p);

/* Static facts of a problem, for callers that size buffers or admit work
 * (library utility). */
typedef struct hc_problem_info {
  int32_t n;                  /* unknowns                                        */
  int32_t kind;               /* HC_TOTAL_DEGREE or HC_PARAMETER                 */
  int32_t inputs_per_instance;/* complex inputs per instance: n_terms (coef) or
                                 n_params (p1)                                   */
  int32_t lanes;              /* lanes per path of its kernels                   */
  int64_t paths;              /* paths per instance                              */
  int64_t device_bytes_per_instance; /* device memory one instance of a batch
                                 needs (inputs, encoded data, outputs, scratch)  */
} hc_problem_info;

hc_status hc_problem_query(const hc_problem* p, hc_problem_info* out);

/*
 * Continuous admission (not in the paper, which tracks the paths of one
 * system per run; serving systems as they arrive is this library's): a
 * stream holds `slots` instance slots of a problem
 * on the device and a resident tracking launch whose lane groups take the
 * next path of the next submitted instance as soon as they free up, instead
 * of each batch waiting for a launch of its own.  The launch polls a
 * host-published counter in mapped memory with sleeps between polls and
 * ends after idle_us without work (the next submit or poll starts it
 * again); a slot whose paths are done gets the re-tracking tiers of the
 * mixed pipeline on a side stream, as hc_track_batch runs them for a batch.
 * Results are those of hc_track_batch on the same inputs, path for path.
 * One thread at a time may use a stream.  Streams track in mixed precision
 * with the default group width (settings.lanes is not applied; other
 * precisions return HC_ERR_UNSUPPORTED), and apply no sign symmetries
 * (every start is tracked).
 *   hc_stream_create  slots 1..4096, idle_us 1..1e7; allocates the ring
 *                     (inputs, tables, outputs, lists per slot) and mapped
 *                     control words; the problem must outlive the stream.
 *   hc_stream_submit  inputs as one instance of hc_batch_desc (coef [T] for
 *                     total degree, NULL: the problem's own; p1 [n_params]
 *                     otherwise), host memory; copies and stages them,
 *                     publishes the instance's paths and returns its ticket
 *                     (0, 1, 2, ...).  HC_ERR_BUSY when the ticket's slot
 *                     (ticket mod slots) still holds an uncollected request.
 *   hc_stream_poll    waits up to timeout_us (< 0: no limit, 0: check once)
 *                     for ticket's results and copies them to the host
 *                     buffers (x_out [paths][n] complex, status_out
 *                     [paths], optional steps_out [paths][3] and be_out
 *                     [paths]); HC_ERR_TIMEOUT if not done yet; the slot is
 *                     free again after a successful poll.
 *   hc_stream_destroy stops the resident launch (its groups leave after
 *                     their current paths), waits for it and frees the stream.
 */
typedef struct hc_stream hc_stream;
hc_status hc_stream_create(hc_problem* p, int32_t slots, int64_t idle_us, hc_stream** out);
hc_status hc_stream_submit(hc_stream* s, const double* inputs, int64_t* ticket);
hc_status hc_stream_poll(hc_stream* s, int64_t ticket, int64_t timeout_us, double* x_out,
                         uint8_t* status_out, int32_t* steps_out, double* be_out);
hc_status hc_stream_destroy(hc_stream* s);

/*
 * Sec. 6 ("Parallel Evaluations of the Jacobian and Vectors": dH/dx, dH/dt
 * and H evaluated together from the terms of the equations) and Sec. 3 (H):
 * evaluate the problem's homotopy at n_points points with the tracker's own
 * device evaluator, in FP64 (HC_PREC_FP64), FP32 (HC_PREC_MIXED) or
 * double-float (HC_PREC_DF) arithmetic.
 *   inputs   host, the instances' data as in hc_batch_desc: total degree
 *            coef [n_instances][T] complex (NULL: the problem's own
 *            coefficients), parameter and coefficient-interpolation
 *            homotopies p1 [n_instances][n_params] complex (required)
 *   instance host [n_points], each in [0, n_instances)
 *   x        host [n_points][n] complex; t host [n_points]
 *   H, Ht    host out [n_points][n] complex; Hx host out [n_points][n][n]
 *            complex, row-major (Hx[k][i][j] = dH_i/dx_j at point k)
 * Synchronous; allocates its device buffers per call on the problem's
 * device.  Returns HC_ERR_INVALID for bad arguments or an out-of-range
 * instance index, HC_ERR_UNSUPPORTED for a shape without an evaluation
 * kernel, HC_ERR_OOM / HC_ERR_CUDA for device failures.
 */
hc_status hc_evaluate(const hc_problem* p, int32_t precision, int32_t n_instances,
                      const double* inputs, int64_t n_points, const int64_t* instance,
                      const double* x, const double* t, double* H, double* Hx, double* Ht);

/*
 * Sec. 3 (predictor-corrector tracking of every start path from t = 0 to
 * t = 1, Eqs. 2-6) run as Sec. 6 lays the work out on the GPU (each path an
 * independent track, evaluation and the fused solve per path): enqueue one
 * batch on b->stream and return at once with *out set.  Staging of
 * coefficients, the tracking launch and the result copies all run on the
 * stream.  Admission: with a device-memory cap set (hc_set_memory_cap), a
 * batch whose device memory would take the batches in flight on the device
 * past the cap returns HC_ERR_BUSY, or with HC_BLOCKING_ADMIT waits for
 * earlier batches to finish (a batch larger than the cap on its own is
 * admitted when nothing else is in flight).  Errors: HC_ERR_INVALID,
 * HC_ERR_OOM, HC_ERR_CUDA, HC_ERR_BUSY.
 */
hc_status hc_track_batch(hc_problem* p, const hc_batch_desc* b, hc_batch** out);

/*
 * Admission cap for hc_track_batch on the current device: the device bytes
 * (inputs, encoded tables, outputs, scratch) of the batches in flight may
 * not exceed max_device_bytes (0: no cap, the default).  A batch counts as
 * in flight until its completion is observed (hc_poll, hc_destroy or a later
 * admission check).  (Library utility; the paper tracks one system at a
 * time.)  Errors: HC_ERR_INVALID (negative), HC_ERR_CUDA.
 */
hc_status hc_set_memory_cap(int64_t max_device_bytes);

/*
 * The output side of Sec. 3 (endpoints and their classification): wait at
 * most timeout_us microseconds (< 0: without limit, 0: just test) for the
 * batch.  HC_OK: done, *r filled (r may be NULL).  HC_ERR_TIMEOUT: done, but
 * the batch's step budget ran out before every path started (*r filled,
 * r->untracked > 0).  HC_PENDING: still running.  Never blocks beyond the
 * timeout.
 */
hc_status hc_poll(hc_batch* b, int64_t timeout_us, hc_batch_result* r);

/* Free a problem, a batch, a plan or a server (waits for running work
 * first).  NULL is a no-op.  A problem must outlive its batches and plans.
 * (Library utility.) */
void hc_destroy(void* handle);

/*
 * Plans: a batch shape replayed as one CUDA graph (no counterpart in the
 * paper, which launches one system at a time; Sec. 6 only asks that data
 * transfer be avoided).  A batch of hc_track_batch is a fixed sequence of
 * launches; a plan records that sequence once -- coefficient staging, the
 * tracking launch, the re-tracking tiers on a high-priority branch, the
 * summary -- with device buffers allocated for good, so each later batch of
 * the same size costs one graph launch plus its input and output copies, and
 * no allocation.  Plans take no start subset and no step budget.
 *
 * hc_plan_create: fixes the problem's current settings, n_instances and the
 * device (the current one).  Errors: HC_ERR_INVALID, HC_ERR_OOM, HC_ERR_CUDA,
 * HC_ERR_UNSUPPORTED.
 *
 * hc_plan_run: *b as for hc_track_batch, with b->n_instances equal to the
 * plan's (else HC_ERR_INVALID); coef NULL means the problem's own
 * coefficients.  Host or device pointers are both accepted
 * (HC_DEVICE_PTRS is not needed).  Returns a batch handle for hc_poll and
 * hc_destroy at once.  Runs of one plan are ordered on the device (each
 * starts after the previous run's last copy, on whatever stream); the
 * batch's track_ms and escalate_ms report the plan's most recent run.
 * The plan owns its device buffers: free it with hc_destroy after its
 * batches are done.
 */
typedef struct hc_plan hc_plan;  /* opaque */
hc_status hc_plan_create(hc_problem* p, int32_t n_instances, hc_plan** out);
hc_status hc_plan_run(hc_plan* plan, const hc_batch_desc* b, hc_batch** out);

/*
 * Autotuner (no counterpart in the paper, which fixes one warp per path in
 * Sec. 6).  Runs the caller's representative batch (*sample, as for
 * hc_track_batch; its outputs are overwritten) under each candidate
 * configuration -- all-FP64; mixed precision with lanes per path (the default
 * width or one path per warp), paths per block (block_threads 128 or 64) and
 * the FP32 first-correction bound (0.01 or 0.1) -- twice each, and keeps in
 * the problem's settings the candidate with the shortest device time among
 * those that recover at least as many finite roots as the all-FP64 run.
 * *report (may be NULL) lists what was tried.
 */
typedef struct hc_tune_report {
  int32_t n_candidates;
  int32_t best;                /* index into the arrays below                    */
  int32_t cached;              /* hc_autotune_cached: 1 if the cache answered     */
  int32_t reserved;
  double ms[16];               /* device time of each candidate's second run     */
  int64_t finite[16];          /* finite roots found by each candidate           */
  hc_settings tried[16];
} hc_tune_report;

hc_status hc_autotune(hc_problem* p, const hc_batch_desc* sample, hc_tune_report* report);

/*
 * The autotuner with a cache file: cache_path is a JSON object mapping a key
 * of the problem's shape and precision -- kind, n, total degree, term count,
 * parameter count, symmetries, precision -- to the chosen lanes,
 * block_threads, max_first_corr_fp32 and precision.  A key already in the
 * file is applied to the problem's settings without tracking
 * (report->cached = 1, n_candidates = 0); otherwise hc_autotune runs and its
 * choice is added to the file (created if absent; other keys are kept).
 * Errors: those of hc_autotune, HC_ERR_INVALID for an unreadable or
 * unwritable cache file.
 */
hc_status hc_autotune_cached(hc_problem* p, const hc_batch_desc* sample, const char* cache_path,
                             hc_tune_report* report);

/*
 * Continuous-batching server (serving form of the tracker; no counterpart in
 * the paper, which tracks one system per launch).  Requests -- one system instance each: the
 * coefficients (HC_TOTAL_DEGREE) or target parameters (HC_PARAMETER) of one
 * problem -- are queued per problem.  A dispatcher thread forms a batch from
 * whatever is pending for a problem as soon as one of n_streams streams is
 * free and the device memory of the in-flight batches plus the new one stays
 * within max_device_bytes (a request that alone exceeds the cap runs when
 * nothing else is in flight).  Requests that arrive while others run are
 * admitted as streams and memory free up, so their work overlaps on the
 * device.  Results are the same whether a request runs alone or in a batch:
 * every path is computed independently.
 */
typedef struct hc_server hc_server;  /* opaque */

typedef struct hc_server_config {
  int32_t n_streams;           /* concurrent batches (streams), default 4; while
                                  several problems wait, one problem holds at most
                                  half of them                                     */
  int32_t max_batch_instances; /* instances per batch, default 64                    */
  int64_t max_device_bytes;    /* admission cap on in-flight batches, default 8 GiB  */
} hc_server_config;

typedef struct hc_request_info {
  int64_t paths;               /* paths of the request                               */
  int64_t finite, real;        /* status counts                                      */
  double queue_us;             /* submit -> dispatch                                 */
  double latency_us;           /* submit -> result on the host                       */
  int32_t batch_instances;     /* size of the batch it ran in                        */
  int32_t reserved;
} hc_request_info;

/* Default configuration. */
hc_server_config hc_server_default_config(void);

/* Start a server on the current device (creates its streams and thread).
 * Errors: HC_ERR_INVALID, HC_ERR_CUDA, HC_ERR_OOM. */
hc_status hc_server_create(const hc_server_config* cfg, hc_server** out);

/* Queue one request: input = host [inputs_per_instance][2] doubles (copied
 * before return).  *request_id identifies it.  The problem must outlive the
 * server.  Errors: HC_ERR_INVALID. */
hc_status hc_server_submit(hc_server* s, hc_problem* p, const double* input,
                           uint64_t* request_id);

/* Wait at most timeout_us (< 0: without limit) for a request; on HC_OK copy
 * its endpoints (host [paths][n][2] doubles, may be NULL) and statuses (host
 * [paths] uint8, may be NULL), fill *info (may be NULL) and release the
 * request.  HC_PENDING if not done within the timeout; HC_ERR_INVALID for an
 * unknown id; a batch error is returned as its status. */
hc_status hc_server_wait(hc_server* s, uint64_t request_id, int64_t timeout_us, double* x_out,
                         uint8_t* status_out, hc_request_info* info);

/* Counters since creation: [0] requests done [1] batches [2] max batches in
 * flight at once [3] max in-flight device bytes [4] max instances in a batch. */
hc_status hc_server_stats(hc_server* s, int64_t* out5);

/*
 * Sec. 6, the fused batched linear solver (LU with partial pivoting on the
 * augmented matrix [A b], the triangular solve folded into the same kernel,
 * data held in registers), measured standalone as in the paper's Fig. 3:
 * solves A_k x_k = b_k for k < batch, n x n complex systems, one lane group
 * per system, one matrix row per lane (the tracker's own solve).  The
 * elimination is Gauss-Jordan (it also clears above the pivot), which with
 * one row per lane replaces the back substitution at no extra latency.
 *   n       1..32
 *   batch   >= 0 (0: nothing to do)
 *   fp32    0: complex double (interleaved re, im doubles);
 *           1: complex float (interleaved re, im floats)
 *   A       device [batch][n][n] complex, row-major, system after system
 *   b       device [batch][n] complex
 *   x       device [batch][n] complex (output; may not alias A or b)
 *   info    device [batch] int32 (optional): 0, or 1 if a pivot was zero or
 *           non-finite (x is then not a solution)
 *   stream  cudaStream_t (NULL: the legacy default stream)
 * Enqueues one launch and returns.  Pivot: largest |Re| + |Im|, lowest row
 * on ties.  Errors: HC_ERR_INVALID, HC_ERR_CUDA.
 */
hc_status hc_batched_solve(int32_t n, int64_t batch, int32_t fp32, const void* A, const void* b,
                           void* x, int32_t* info, void* stream);

/*
 * Sec. 7: the start systems of the parameter homotopies come from monodromy
 * (Macaulay2 in the paper) -- all isolated solutions of F(x; p0) at a
 * generic complex parameter point p0.  This call computes them on the GPU
 * from one seed solution: the known solutions are carried around triangle
 * loops p0 -> pa -> pb -> p0 through random complex parameter points
 * (parameter homotopies tracked by hc_track_batch), and endpoints not yet
 * known (relative infinity distance > 1e-6) are added, until stall_loops
 * consecutive loops add nothing.  A round runs loops_per_round loops; their
 * first legs share one batch.  With sign symmetries in the family
 * (n_sym > 0) the sign images of every new solution are added too and the
 * legs track one start per orbit.
 *   family          HC_PARAMETER description; its p0, n_start and start are
 *                   ignored (the call sets them per leg); its settings apply
 *   x0, p0          host [n][2] and [n_params][2]: a solution of F(x0; p0) = 0
 *   seed            seeds the loop points (splitmix64 + Box-Muller)
 *   out             host [max_solutions][n][2] doubles: the solutions found
 * *n_solutions receives the count (also when it exceeds max_solutions, in
 * which case HC_ERR_INVALID is returned and out is not written); *info
 * (may be NULL) the loops, rounds, tracked paths and wall time.  Errors:
 * HC_ERR_INVALID and those of hc_create_problem / hc_track_batch.
 */
typedef struct hc_monodromy_desc {
  const hc_problem_desc* family;
  const double* x0;
  const double* p0;
  uint64_t seed;
  int32_t stall_loops;         /* e.g. 10                                          */
  int32_t max_loops;           /* e.g. 400                                         */
  int32_t loops_per_round;     /* e.g. 4                                           */
  int32_t reserved;            /* 0                                                */
  int64_t max_solutions;
  double* out;
} hc_monodromy_desc;

typedef struct hc_monodromy_info {
  int32_t loops, rounds;
  int64_t paths_tracked;
  double seconds;
} hc_monodromy_info;

hc_status hc_monodromy_solve(const hc_monodromy_desc* d, int64_t* n_solutions,
                             hc_monodromy_info* info);

/*
 * Measurement utility (no counterpart in the paper): FMA throughput of the
 * current device's CUDA cores, FP32 (fp64 = 0) or FP64 (fp64 = 1), from one
 * timed launch of independent FMA chains on every SM; iters sets the length
 * (each thread issues iters * 128 FMAs).  *flops_per_s = 2 * FMAs / time.
 * Used for the roofline of the ALU-bound tracker.  Errors: HC_ERR_INVALID,
 * HC_ERR_OOM, HC_ERR_CUDA.
 */
hc_status hc_measure_fma_peak(int32_t fp64, int32_t iters, double* flops_per_s, double* ms);

/*
 * Tracking without allocation (no counterpart in the paper).  For callers
 * that cannot allocate device memory when they track: code inside a pool or
 * arena that owns the device, real-time loops that must not enter the CUDA
 * allocator (it can synchronize the device), hosts whose allocator belongs to
 * another framework.  Runs the same dense total-degree kernels as
 * hc_track_batch on one batch, allocating nothing: every buffer besides the
 * caller's inputs and outputs lives in one fixed 16 MiB device array that
 * each GPU loading the library holds until exit.
 *   n, degree   dense system: every monomial of degree <= degree in each of
 *               the n equations; degree 2 with n <= 12 or degree 3 with n <= 8
 *   gamma       host [2] unit-modulus homotopy constant
 *   settings    host hc_settings (precision, tolerances, escalation)
 *   coef        device [n_instances][n][M][2] doubles, M = C(n+degree, degree),
 *               monomials in graded order (degree 0 first; inside a degree the
 *               sorted variable tuple in lexicographic order)
 *   x_out, status_out, steps_out (required), be_out (optional): device
 *               buffers laid out as in hc_batch_desc
 *   stream      cudaStream_t (NULL = legacy default stream)
 * Enqueues on the stream and returns; completion is the stream's.  The first
 * call on a device looks up the array's device address (make it before any
 * stream capture).  Calls share the array: calls that overlap on the GPU
 * race and must be serialized by the caller.  A batch whose scratch exceeds
 * the array returns HC_ERR_INVALID (hc_last_error says how much it needs);
 * also HC_ERR_INVALID for bad arguments, HC_ERR_CUDA for launch errors.
 */
hc_status hc_track_dense_noalloc(int32_t n, int32_t degree, const double* gamma,
                                 const hc_settings* settings, int32_t n_instances,
                                 const double* coef, double* x_out, uint8_t* status_out,
                                 int32_t* steps_out, double* be_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HC_H */
