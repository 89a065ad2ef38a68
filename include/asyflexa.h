/*
 * asyflexa.h -- C ABI of the GB300 (sm_103a) AsyFLEXA block-update library.
 *
 * The library solves
 *
 *     minimise  F(x) = f(x) + lambda * ||x||_1   subject to  lo <= x <= hi      (eq. 1)
 *
 * with f one of
 *     ASYFLEXA_LOSS_LASSO :  f(x) = 0.5 * ||A x - b||^2          (Section 4.2)
 *     ASYFLEXA_LOSS_NCQUAD:  f(x) = ||A x - b||^2 - c * ||x||^2  (Section 4.3, nonconvex)
 *     ASYFLEXA_LOSS_DC_LOG / DC_EXP: ||A x - b||^2 + lambda * H(x) with a nonconvex
 *                            regulariser H (Section 4.3), see asyflexa_loss
 * by the fixed-stepsize AsyFLEXA iteration (Algorithm 1): a block of w columns reads a
 * possibly stale residual r = A x - b, forms its gradient, takes the closed-form best
 * response of the proximal-linear surrogate (eq. 2; soft-threshold then clip to the
 * box) and steps  x_i <- x_i + gamma * (xhat_i - x_i)  (step S.4), after which
 * r += A_i * Delta_i.
 *
 * Data layout: A is m x n column-major with leading dimension lda (elements); lda must
 * be >= m and lda * sizeof(element) a multiple of 16 bytes, A itself 16-byte aligned.
 * Vectors are dense and contiguous.
 *
 * Ownership: every pointer in asyflexa_problem and the x passed to solve/step/check are
 * caller-owned DEVICE memory, borrowed (never freed) for the lifetime of the handle;
 * the caller must keep them alive and unmodified (except x through this API) until
 * asyflexa_destroy.  The handle owns its residual, weights and scratch.
 *
 * Streams: every call enqueues work on the stream given to asyflexa_create.
 * asyflexa_step is asynchronous with respect to the host; asyflexa_solve,
 * asyflexa_check and the getters synchronise that stream.
 *
 * Errors: every function returns an asyflexa_status.  Nothing throws across the ABI.
 * A CUDA error or a device-side timeout is latched in the handle; asyflexa_last_error
 * gives a message (per handle, or thread-local for a NULL handle).
 */
#ifndef ASYFLEXA_H
#define ASYFLEXA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ASYFLEXA_ABI_VERSION 1

typedef struct asyflexa_s* asyflexa_t;

typedef enum {
    ASYFLEXA_OK = 0,
    ASYFLEXA_ENOTCONV = 1,      /* solve stopped at max_sweeps before meeting the tolerances */
    ASYFLEXA_EINVAL = -1,       /* bad argument (null, misaligned, out of range, wrong dtype) */
    ASYFLEXA_ECUDA = -2,        /* a CUDA runtime error (message in asyflexa_last_error) */
    ASYFLEXA_ENOMEM = -3,       /* device allocation failed */
    ASYFLEXA_ETIMEOUT = -4,     /* a bounded device-side wait expired; results invalid */
    ASYFLEXA_ENONFINITE = -5,   /* NaN/Inf found in the objective or residual */
    ASYFLEXA_EUNSUPPORTED = -6  /* valid request this build does not implement */
} asyflexa_status;

typedef enum {
    ASYFLEXA_LOSS_LASSO = 0,    /* f = 0.5 ||Ax - b||^2 */
    ASYFLEXA_LOSS_NCQUAD = 1,   /* f = ||Ax - b||^2 - c ||x||^2 */
    ASYFLEXA_LOSS_DC_LOG = 2,   /* F = ||Ax - b||^2 + lambda sum_j h(x_j), h = log(1+theta|x|)/log(1+theta) */
    ASYFLEXA_LOSS_DC_EXP = 3    /* F = ||Ax - b||^2 + lambda sum_j h(x_j), h = 1 - exp(-theta|x|) */
} asyflexa_loss;
/* The DC losses (Section 4.3, nonconvex sparse learning) split h = eta|x| - h-(x) with h-
 * convex and smooth (eta = theta / log(1+theta) for log, theta for exp) and run the method on
 * f = ||Ax - b||^2 - lambda sum_j h-(x_j), G = lambda eta ||x||_1: the best response keeps
 * the quadratic's coordinate curvature 2||a_j||^2 and linearises -lambda h- at the current
 * point.  theta > 0 is passed in asyflexa_problem.c. */

/* SYNC: deterministic Jacobi sweeps (every block from the same x; bit-reproducible).
 * ASYNC: persistent CTAs, each owning a fixed set of blocks (Assumption D4), reading the
 *        shared residual without locks and updating it with atomics (Algorithm 1 with
 *        delays bounded by the number of updates in flight, Assumption D1). */
typedef enum { ASYFLEXA_SYNC = 0, ASYFLEXA_ASYNC = 1 } asyflexa_mode;

typedef enum {
    ASYFLEXA_F64 = 0,
    ASYFLEXA_F32 = 1,
    ASYFLEXA_BF16 = 2,          /* A only, with per-column FP32 scales */
    ASYFLEXA_FP8E4M3 = 3        /* A only, with per-column FP32 scales */
} asyflexa_dtype;

/* Problem data (eq. 1).  All pointers are device pointers owned by the caller. */
typedef struct {
    int64_t m;                  /* rows of A (>= 1) */
    int64_t n;                  /* columns of A = number of variables (>= 1) */
    int64_t lda;                /* leading dimension of A in elements (see layout above) */
    int32_t a_dtype;            /* asyflexa_dtype of A */
    int32_t x_dtype;            /* ASYFLEXA_F64 or ASYFLEXA_F32: type of x, b, lo, hi */
    const void* A;              /* m x n column-major */
    const float* col_scale;     /* length n: a_j = col_scale[j] * stored_j; BF16/FP8 only, else NULL */
    const void* b;              /* length m */
    const void* lo;             /* length n lower bounds, or NULL for -inf */
    const void* hi;             /* length n upper bounds, or NULL for +inf */
    double lambda;              /* weight of ||x||_1 (of H for the DC losses), >= 0 */
    double c;                   /* NCQUAD concavity weight; theta of the DC losses; ignored for LASSO */
    int32_t loss;               /* asyflexa_loss */
    int32_t reserved0;
    const void* A_master;       /* optional FP32 copy of A (m x n, leading dimension lda_master), only
                                   with BF16/FP8 storage: exact residual refreshes and checks use it, and
                                   solve ends with FP32 "polish" sweeps on it (see asyflexa_solve) */
    int64_t lda_master;
    const void* lin;            /* optional linear term (length n, x_dtype): f(x) += lin^T x, so
                                   grad_j f gains lin_j; NULL = 0.  With lambda = 0 and b = 0 the method
                                   then solves A^T A x = -lin (used by the adjoint of the solution map) */
} asyflexa_problem;

/* Method parameters.  Fill with asyflexa_opts_default, then override. */
typedef struct {
    int32_t block_w;            /* columns per block, 1..128 (last block may be shorter) */
    int32_t mode;               /* asyflexa_mode */
    double gamma;               /* fixed step (Algorithm 1, S.4), > 0 */
    double tau;                 /* proximal weight: surrogate curvature d_j = (1+tau_rel)*kappa_j + tau */
    double tau_rel;             /* relative proximal weight (see tau); both >= 0 */
    int32_t refresh_every;      /* recompute r = A x - b exactly every this many sweeps (>= 1) */
    int32_t check_every;        /* solve: evaluate F every this many sweeps (>= 1) */
    int32_t max_sweeps;         /* solve: sweep budget (>= 1) */
    int32_t num_ctas;           /* CTAs of the sweep kernels; 0 = one per SM */
    double tol_gap;             /* solve: stop when (F - f_star)/|f_star| <= tol_gap ... */
    double tol_stat;            /* ... and ||xhat(x) - x||_inf / max(1,||x||_inf) <= tol_stat */
    double f_star;              /* optimal value if known, else NaN (then only tol_stat is used) */
    uint64_t seed;              /* reserved */
    int32_t profile;            /* 1: time every sweep-kernel launch with CUDA events (see
                                   asyflexa_read_counters); 0: off */
    int32_t variant;            /* async kernel: 0 = automatic (2 for FP32 with m > 12288 and
                                   BF16/FP8 with m > 16384, 3 for smaller m, 1 where neither
                                   applies), 1 = staged residual tile (any m, any dtype),
                                   2 = register increment with the residual snapshot in shared
                                   memory, each thread holding its rows of the current column in
                                   registers (16 warps that also refill the ring), 3 = the same
                                   with a producer warp and the column read from shared memory
                                   twice (variants 2 and 3: FP32/BF16/FP8, m up to 24576 rows;
                                   EUNSUPPORTED otherwise).  exact_grad 1 runs the form of 3 */
    double switch_tol;          /* with A_master: solve leaves the low-precision phase when a check
                                   interval lowers F by less than switch_tol * |F| (default 1e-7) */
    double gamma_mu;            /* 0 (default): fixed step gamma (Algorithm 1).  > 0: the diminishing
                                   rule of the experiments of Section 4, gamma^0 = gamma and
                                   gamma^{k+1} = gamma^k (1 - gamma_mu gamma^k), k counting block
                                   updates from the start of asyflexa_solve (or of the handle /
                                   asyflexa_reset_counters for asyflexa_step).  Async: update k is the
                                   one that read the residual after k completed updates (exact for a
                                   single CTA); sync: block i of the s-th sweep is update s N + i. */
    int32_t tau_adapt;          /* 1: solve adapts the proximal weight between checks (a rule in the
                                   spirit of FLEXA's, which the paper does not restate): when a check
                                   interval raised F, every d_j grows by tau_extra (doubled; the first
                                   time 0.05 * mean d_j); after 5 intervals in a row that lowered F it
                                   shrinks by half.  Restarts at 0 in every solve.  0 (default): off */
    int32_t exact_grad;         /* gradient arithmetic of the asynchronous register kernel (kernel
                                   variants 2 and 3): 0 (default) FP32 accumulation; 1: compensated (Dot2)
                                   accumulation, as accurate as FP64 accumulation of the FP32
                                   residual snapshot, about 1.6x the sweep time (FP32 storage only:
                                   EUNSUPPORTED otherwise, or when the register kernel does not
                                   apply).  The batched and multi-lane forms ignore it */
    int32_t delay_ns;           /* test-only staleness widener (0 = off, the default): in the
                                   asynchronous single-problem kernels with several CTAs, every
                                   odd-numbered CTA sleeps this many ns (__nanosleep, at most
                                   1000000) before each block's scatter, so that the other CTAs'
                                   reads miss its updates for longer (Assumption D1's delays grow;
                                   the staleness histogram shows it).  EINVAL outside [0, 1000000] */
    int32_t reserved2;
} asyflexa_opts;

/* Results and counters.  Optimality fields are FP64 and computed from an exact
 * residual (FP64 accumulation) and a compensated gradient (see asyflexa_check). */
typedef struct {
    int64_t sweeps;             /* sweeps performed by the last solve (or since create for check) */
    int64_t block_updates;      /* block updates performed (each sweep updates every block once) */
    double F;                   /* objective at x */
    double rel_gap;             /* (F - f_star)/|f_star|, NaN if f_star unknown */
    double stat_xhat;           /* ||xhat(x) - x||_inf / max(1, ||x||_inf)   (Section 4.3 merit) */
    double stat_mf;             /* ||M_F(x)||_inf / max(1, ||x||_inf)        (Section 3 measure) */
    double kkt_viol;            /* LASSO without box: max KKT residual; NaN otherwise */
    int64_t nnz;                /* nonzeros of x */
    double seconds;             /* device time of the last solve (CUDA events) */
    double hbm_bytes;           /* algorithmic bytes of A streamed by the sweeps of the last solve */
    uint64_t staleness_hist[32];/* async: histogram of updates completed between a block's read
                                   of r and its own update; bucket k holds delays in [2^k-1, 2^(k+1)-1) */
    int64_t kernel_launches;    /* kernels launched by this handle so far */
    double sweep_kernel_seconds;/* profile=1: summed device time of the sweep-kernel launches */
    int64_t sweep_kernel_launches; /* profile=1: number of sweep-kernel launches timed */
    int64_t sweep_kernel_sweeps;   /* profile=1: sweeps performed by those launches */
    int32_t status;             /* asyflexa_status of the last solve/check */
    int32_t checked;            /* 1 if the stat_* / kkt fields were evaluated */
    int64_t polish_sweeps;      /* with A_master: sweeps of the last solve run on the FP32 copy;
                                   multi-lane form: sweeps of the single-lane finish of a lane */
    double polish_seconds;      /* with A_master: device time of that FP32 phase */
    int32_t block_w;            /* batched solve: block width used (given or autotuned) */
    int32_t kernel_variant;     /* async sweep kernel this handle launches (1, 2 or 3, see
                                   asyflexa_opts.variant); set by solve, check, read_counters */
    double dual_gap;            /* plain LASSO (no box, no linear term): (P(x) - D(nu)) / max(1, |P(x)|)
                                   with the feasible dual point nu = theta r, theta = min(1, lambda /
                                   ||A^T r||_inf) -- an upper bound of the relative optimality gap
                                   that needs no optimum; NaN for other problems.  Reported, not a
                                   stopping test: with FP32 iterates ||A^T r||_inf carries the
                                   rounding of the heaviest column, which loosens the bound. */
    double tau_extra;           /* solve with tau_adapt: the proximal weight added at the end */
    int32_t batch_form;         /* batched solve: ASYFLEXA_BATCH_FORM_ASYNC, _GS or _MULTI */
    int32_t ctas_per_sm;        /* batched solve, Gauss-Seidel form: CTAs resident per SM (autotuned) */
    int32_t handed_over;        /* batched solve, Gauss-Seidel form: problems that ran in more than
                                   one launch (total), or the further launches it ran in (per
                                   problem) */
    int32_t reserved1;
} asyflexa_stats;

/* Library version (ASYFLEXA_ABI_VERSION).  Never fails. */
int asyflexa_version(void);

/* Human-readable name of a status code.  Never fails. */
const char* asyflexa_status_string(int status);

/* Default options: block_w 32, SYNC, gamma 0.9, tau 0, tau_rel 0, refresh_every 10,
 * check_every 10, max_sweeps 1000, num_ctas 0, tol_gap 1e-6, tol_stat 1e-6, f_star NaN. */
void asyflexa_opts_default(asyflexa_opts* opts);

/* Validate the problem and options, compute the surrogate weights
 * d_j = (1+tau_rel)*kappa_j + tau (kappa_j the curvature of f along coordinate j:
 * ||a_j||^2 for LASSO, 2||a_j||^2 - 2c for NCQUAD; Section 4 surrogates) and allocate
 * the handle's state on the current device.  cuda_stream is a cudaStream_t (NULL =
 * legacy default stream).  EINVAL if any d_j < 0 (nonconvex curvature not compensated
 * by tau).  On success *h is a new handle; on failure *h is NULL. */
int asyflexa_create(asyflexa_t* h, const asyflexa_problem* prob, const asyflexa_opts* opts,
                    void* cuda_stream);

/* Release the handle's device memory (after synchronising its stream).  NULL is a no-op. */
int asyflexa_destroy(asyflexa_t h);

/* r = A x - b with FP64 accumulation over the nonzero columns of x (x: length n device
 * vector of x_dtype).  The residual is the handle's internal FP64 vector. */
int asyflexa_residual_refresh(asyflexa_t h, const void* x);

/* n_sweeps sweeps of the configured mode on x (in place).  Each sweep updates every
 * block once.  The residual must describe x: it does after create+refresh, solve, step
 * or check on the same x; a first step after create refreshes it automatically.  If x is
 * changed outside this API, call asyflexa_residual_refresh first.  The residual is
 * recomputed exactly every refresh_every sweeps and at the end of the call.
 * Asynchronous: returns after enqueueing. */
int asyflexa_step(asyflexa_t h, void* x, int32_t n_sweeps);

/* Run sweeps from the given x (in place) until the stopping rule of the options holds
 * or max_sweeps is reached (ENOTCONV).  Every check_every sweeps F is evaluated from an
 * exact residual; once (F - f_star)/|f_star| <= tol_gap (or always, if f_star is NaN) the
 * stationarity ||xhat(x) - x||_inf / max(1, ||x||_inf) is evaluated and the solve stops when
 * it is <= tol_stat.  A stationarity check that fails within 2 tol_stat is repeated after
 * 2 sweeps instead of check_every (at most check_every times; not with A_master or
 * tau_adapt): near tol_stat the stationarity of FP32 iterates fluctuates from sweep to sweep.
 * The stopping decision and the returned stats come from the same exact check.
 * With A_master set, these sweeps run on the BF16/FP8 matrix while
 * F, the residual refreshes and the stationarity are those of the FP32 problem; when a check
 * interval lowers F by less than switch_tol * |F|, or (f_star known) F comes within
 * max(tol_gap, u^2) of f_star relative (u the storage's unit roundoff: 2^-8 BF16, 2^-4 FP8
 * e4m3; about how far the stored problem's optimal F lies) without the tolerances holding,
 * the solve continues with FP32 sweeps on A_master ("polish") until the same stopping rule
 * holds.  Fills *out (may be NULL);
 * out->block_updates counts this solve's updates.  Synchronises. */
int asyflexa_solve(asyflexa_t h, void* x, asyflexa_stats* out);

/* Evaluate F, rel_gap, the stationarity measures, KKT and nnz at x, after an exact
 * residual refresh.  Fills *out.  Synchronises. */
int asyflexa_check(asyflexa_t h, const void* x, asyflexa_stats* out);

/* Counters accumulated since create or the last asyflexa_reset_counters: fills sweeps,
 * block_updates, staleness_hist, kernel_launches and (profile=1) the sweep_kernel_* fields
 * of *out (other fields untouched).  Synchronises. */
int asyflexa_read_counters(asyflexa_t h, asyflexa_stats* out);

/* Zero the update counters, the staleness histogram and the sweep-kernel timers. */
int asyflexa_reset_counters(asyflexa_t h);

/* Copy the handle's residual (FP64, length m) into a caller device buffer.  Synchronises. */
int asyflexa_get_residual(asyflexa_t h, double* r_out);

/* Copy the surrogate weights d_j (FP64, length n) into a caller device buffer.  Synchronises. */
int asyflexa_get_weights(asyflexa_t h, double* d_out);

/* r_out = A x - b for the problem *prob at x, without a handle and without allocating
 * any device memory.  (The paper has no counterpart; this is a service entry point.)
 *
 * For callers that cannot allocate device memory when they need the residual: a plugin or
 * library inside a host application that hands it a fixed device-memory budget and owns every
 * allocation itself, or a latency-sensitive loop in which cudaMalloc / cudaFree would
 * synchronise the device and stall the other streams.  The result equals
 * asyflexa_residual_refresh on a handle for the same problem and x up to the grouping of
 * partial sums: the same ordered compaction of the nonzeros of x, the same compensated
 * products and the same fixed-order FP64 reduction, through the register-batched gather
 * kernel instead of the handle's pipelined one.
 *
 * prob: as for asyflexa_create (device pointers A, b, col_scale; lo, hi, lambda, c, loss
 * are ignored).  x: length n device vector of x_dtype.  r_out: caller-owned device buffer
 * of m doubles.  cuda_stream: the stream the kernels are enqueued on (NULL = legacy
 * default stream); the call does not synchronise.
 *
 * Limits: n <= 262144 and m <= 654848 (the row limit is what fits one FP64 partial sum per
 * row in the scratch).
 * Larger problems return ASYFLEXA_EINVAL with a message naming the limit; other argument
 * errors also return ASYFLEXA_EINVAL.  Messages: asyflexa_last_error(NULL), per thread.
 *
 * Scratch: one file-scope 8 MiB device array, held by every GPU that loads the library
 * until the process exits.  Its device address is looked up (cudaGetSymbolAddress) by the
 * first call on each device, with that device current, so make that first call before any
 * stream capture.  The address is then cached per device index for the life of the process:
 * this assumes the device's primary context throughout (after cudaDeviceReset, or from a
 * different context on that device, the cached address is not valid).  Every call shares the
 * array: calls that overlap on the GPU (e.g. on two streams) race and must be serialised by
 * the caller.  The array keeps the last call's contents; every scratch value a call reads is
 * written earlier in the same call, so nothing needs clearing. */
int asyflexa_residual_noalloc(const asyflexa_problem* prob, const void* x, double* r_out, void* cuda_stream);

/* Diagnostic: run the kernels' own number conversions over an array.  The kernels convert
 * the FP64 residual to its FP32 snapshot (step S.2 of Algorithm 1) and each FP32 scatter
 * increment to the FP64 reduction operand with integer operations on the IEEE 754 fields
 * instead of the conversion instructions, and decode BF16 / FP8-e4m3 storage of A to FP32;
 * this entry point exposes exactly those functions so that a test can compare them bit for
 * bit with round-to-nearest-even and with the storage formats' definitions.
 *
 * dir 0: in = n doubles, out = n floats (FP64 -> FP32, round to nearest even);
 * dir 1: in = n floats, out = n doubles (FP32 -> FP64, exact);
 * dir 2: in = n FP8-e4m3 bytes, out = n floats (exact; the NaN codes 0x7f / 0xff give NaN);
 * dir 3: in = n BF16 values, out = n floats (exact).
 * For dir 2 and 3, n is a multiple of 16 and 8 (whole 16-byte units) and `in` is 16-byte
 * aligned.  in, out: caller-owned device buffers; cuda_stream: the stream the kernel is
 * enqueued on (NULL = legacy default stream); the call does not synchronise.  Returns
 * ASYFLEXA_OK, or ASYFLEXA_EINVAL (bad dir, n < 0, n not a whole number of units, NULL
 * buffers with n > 0, misaligned `in`) / ASYFLEXA_ECUDA (launch failure) with a message in
 * asyflexa_last_error(NULL). */
int asyflexa_convert_check(int dir, const void* in, void* out, int64_t n, void* cuda_stream);

/* Diagnostic: run the kernels' bounded wait on a shared-memory mbarrier that expects one
 * arrival.  Every wait of the sweep kernels gives up after a time limit (2 s of the GPU's
 * global timer), records a timeout for the host and returns, instead of spinning; this entry
 * point runs that same wait with a caller's limit in a one-thread kernel.  arrive_first = 1:
 * the thread arrives before waiting, so the wait completes at once; 0: nothing ever
 * arrives, so the wait runs out after limit_ns nanoseconds (1e3 <= limit_ns <= 1e9).
 * result: host array of 4 ints, written on return: [1 if the wait completed else 0, the
 * recorded error (0, or ASYFLEXA_ETIMEOUT), the CTA's abort flag, elapsed microseconds].
 * Synchronous (allocates 16 bytes of device memory, legacy default stream).  Returns
 * ASYFLEXA_OK if the wait completed, ASYFLEXA_ETIMEOUT if it ran out (the context stays
 * usable), ASYFLEXA_EINVAL / ENOMEM / ECUDA otherwise. */
int asyflexa_wait_check(int arrive_first, int64_t limit_ns, int* result);

/* Per-column scaled low-precision storage of an FP32 matrix, for the BF16/FP8 form of the
 * method: Q[:, j] = round(A[:, j] / scale[j]) in `dtype` (ASYFLEXA_BF16 or ASYFLEXA_FP8E4M3,
 * round-to-nearest, FP8 saturating to finite values), with scale[j] = max_i |A[i, j]| / qmax
 * (qmax = 448 for FP8, 1 for BF16; 1 for a zero column), so that a_j ~= scale[j] * Q[:, j].
 * A: m x n FP32 column-major (lda >= m).  Q: output, ldq >= m with ldq * element size a
 * multiple of 16 bytes (rows m..ldq-1 are written as 0).  scale: output, n floats.  All
 * device pointers, caller-owned.  Enqueued on cuda_stream; does not synchronise.
 * EINVAL on bad arguments (message: asyflexa_last_error(NULL)). */
int asyflexa_quantize(const float* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* Q, int64_t ldq,
                      float* scale, void* cuda_stream);

/* out[:, c] = A[:, idx[c]] for c < k: the column submatrix A_S of an m x n column-major
 * matrix of `dtype` (asyflexa_dtype), e.g. the columns on the support of a solution for the
 * adjoint of the solution map.  Rows m..ldo-1 of out are written as 0.  A (lda), out (ldo):
 * device, 16-byte aligned, column strides multiples of 16 bytes; idx: k device int32 indices
 * in [0, n) (not checked).  Enqueued on cuda_stream.  EINVAL on bad arguments. */
int asyflexa_gather_columns(const void* A, int64_t lda, int32_t dtype, int64_t m, const int32_t* idx, int64_t k,
                            void* out, int64_t ldo, void* cuda_stream);

/* Adjoint of the LASSO solution map x*(lambda, b) (system form 3; not in the paper, derived
 * from the LASSO optimality conditions of eq. 1 with f = 0.5||Ax - b||^2, Section 4.2).  On
 * the support S = { j : |x_j| > rel_tol * max(1, ||x||_inf) } with signs s = sign(x_S), the
 * conditions A_S^T (A_S x_S - b) + lambda s = 0 are smooth in (lambda, b); for a loss with
 * v = dL/dx* and w solving (A_S^T A_S) w = v_S:
 *     *out_dlam = dL/dlambda = -s^T w,        out_db = dL/db = A_S w.
 * w is computed by the library's block update on the gathered columns A_S (an internal
 * handle with b = 0, lambda = 0 and linear term -v_S, whose minimiser solves that system);
 * out_db is that handle's exact residual at w.
 *
 * A: m x n column-major, F64 or F32 storage (EUNSUPPORTED otherwise), lda as for
 * asyflexa_create.  x (the solution) and v: device, n entries of A's type.  rel_tol >= 0.
 * opts: the support solve's options (NULL = async, one CTA, block_w 8, gamma 1, tol_stat
 * 1e-7, max_sweeps 2000); f_star is ignored.  out_dlam: host double.  out_db: device, m
 * doubles.  out_support (host, may be NULL): |S|.  out_stats (host, may be NULL): the
 * support solve's statistics.  An empty support gives 0 and db = 0.
 *
 * Allocates (and frees) device memory for A_S and its vectors; enqueued on cuda_stream and
 * synchronises it.  Returns OK, ENOTCONV (the support solve hit max_sweeps; the results are
 * those of its last iterate), or EINVAL / EUNSUPPORTED / ENOMEM / ECUDA / ENONFINITE with a
 * message in asyflexa_last_error(NULL). */
int asyflexa_adjoint(const void* A, int64_t lda, int32_t a_dtype, int64_t m, int64_t n, const void* x,
                     const void* v, double rel_tol, const asyflexa_opts* opts, double* out_dlam, double* out_db,
                     int64_t* out_support, asyflexa_stats* out_stats, void* cuda_stream);

/* ---------------------------------------------------------------- batched problems
 * Many independent problems (e.g. LASSO instances of uneven sizes, or one matrix with many
 * lambda values) solved together, in one of two forms:
 *
 *   ASYFLEXA_BATCH_FORM_GS (Gauss-Seidel form): ONE persistent launch for the whole batch.
 *     Each CTA takes the next problem from a queue (largest first), runs Algorithm 1 on it
 *     alone -- a single owner for every block, so exact cyclic block Gauss-Seidel (blocks of
 *     w <= 4 columns; w = 1 is the scalar blocks of Section 4.1) with the fixed step of S.4
 *     and the best response of eq. 2 -- with
 *     the residual held in registers, and runs its own stopping test (exact residual, F,
 *     gap, and the Section 4.3 merit) before taking the next problem.  FP32 problems with
 *     m <= 8192.  The launch is captured in a CUDA graph and replayed by later solves.
 *   ASYFLEXA_BATCH_FORM_ASYNC (rounds of the asynchronous kernel): every round of
 *     refresh_every sweeps is one persistent launch covering the blocks of every problem
 *     (each block still has a single owning CTA, Assumption D4), followed by exact residual
 *     refreshes, objectives and a device-side convergence test, the round replayed as a
 *     captured CUDA graph.  FP32 problems with m <= 24576.
 *
 * A problem the Gauss-Seidel form has not finished after 300 sweeps leaves the launch and
 * continues, from its current iterate, in a further Gauss-Seidel launch over the problems left
 * (its own launch shape, tuned on them for the longest per-problem time), which hands its own
 * unfinished problems on after 600 sweeps, and so on with the handoff doubling: the first
 * launch ends with the bulk of the batch, and the last few problems run under a shape of
 * their own.  When at most 16 problems are left after a launch, they are finished instead,
 * side by side, by the single-problem async solver (asyflexa_solve on their own handles, each
 * on a stream and a host thread of its own) with max(1, m / (2 * block_w)) CTAs each, so
 * that they do not each hold one SM while the rest idle; their stats then carry batch_form
 * ASYFLEXA_BATCH_FORM_ASYNC.
 *
 *   ASYFLEXA_BATCH_FORM_MULTI (multi-lane form): problems that share A (a lambda path or
 *     several data vectors; LASSO, no box or linear term, at most 64) are the lanes of one
 *     multi-lane handle (asyflexa_multi_*): every block update is done for all of them at once
 *     on the tensor cores, and every lane is confirmed by an exact check.
 *
 * The form is chosen at create (flags) or automatically: the multi-lane form when the problems
 * fit it and ASYFLEXA_BATCH_SHARED_A is set, else the Gauss-Seidel form when every problem fits
 * it and there are at least as many problems as SMs, else the async rounds.  An
 * autotuner then picks the form's launch shape at the first solve by timing one sweep of
 * every problem per candidate -- Gauss-Seidel form: 7 or 15 consumer warps per CTA (2 or 1
 * CTAs per SM), the block width and ring slot -- 1, 2 or 4 columns with 16 KB slots, 4 or 8
 * with 32 KB slots (a slot holds up to 8 columns; a problem whose columns do not fit w to a
 * slot takes as many as fit) -- and the ring depth that fits; the tuning sweeps are undone
 * (the iterates are saved and restored), so they count neither as sweeps nor against
 * max_sweeps; async rounds: the block width 16, 32
 * or 64 (real sweeps, counted) -- and caches the choice per batch shape (problem count, total
 * size, largest m, flags) for the life of the process. */
typedef struct asyflexa_batch_s* asyflexa_batch_t;

/* flags for asyflexa_batch_create */
#define ASYFLEXA_BATCH_SHARED_A 1     /* problems share A: normal L2 priority for its reads (and,
                                         in the async rounds, blocks interleaved across problems
                                         so that their reads of the same panel hit L2) */
#define ASYFLEXA_BATCH_FORM_ASYNC 2   /* force the async rounds form */
#define ASYFLEXA_BATCH_FORM_GS 4      /* force the Gauss-Seidel form (EUNSUPPORTED if a problem
                                         does not fit it) */
#define ASYFLEXA_BATCH_FORM_MULTI 8   /* force the multi-lane form (EUNSUPPORTED if the problems
                                         do not fit it) */

/* probs: count FP32 problems (as for asyflexa_create; LASSO or NCQUAD loss).  opts: shared
 * method parameters: gamma, tau, tau_rel, tol_gap, tol_stat, max_sweeps, num_ctas (0 = all
 * SMs; in the Gauss-Seidel form the most CTAs that run problems at once), check_every
 * (Gauss-Seidel form: sweeps between stopping tests), refresh_every (async rounds: sweeps per
 * round), switch_tol, block_w (async rounds: 16 .. 128, 0 lets the autotuner pick 16, 32 or
 * 64; Gauss-Seidel form: 1 .. 8 fixes the block width, any other value lets the autotuner pick
 * 1, 2, 4 or 8).  All problems and
 * their device buffers must outlive the batch.  Errors: asyflexa_last_error(NULL). */
int asyflexa_batch_create(asyflexa_batch_t* hb, const asyflexa_problem* probs, int32_t count,
                          const asyflexa_opts* opts, int32_t flags, void* cuda_stream);

/* Solve every problem from its iterate xs[k] (device, in place).  f_star: count optimal values
 * or NULL.  Problem k is done when ||xhat(x) - x||_inf / max(1, ||x||_inf) <= tol_stat and, if
 * f_star[k] is a number, (F_k - f_star[k]) / |f_star[k]| <= tol_gap.  Gauss-Seidel form: both
 * are evaluated by the problem's CTA every check_every sweeps (every 2 sweeps once the merit is
 * within 2 tol_stat).  Async rounds: a problem leaves the rounds when its gap meets tol_gap
 * (without f_star: when a round lowers F_k by no more than switch_tol * |F_k|); the exact
 * stationarity check then runs for it, and a problem that fails it rejoins the rounds.
 * per (count entries, may be NULL): each problem's F, rel_gap, stat_xhat, nnz, sweeps,
 * block_updates and status (ENOTCONV at max_sweeps, ENONFINITE if F became non-finite) as the
 * stopping test saw them, and block_w (Gauss-Seidel form: the tuned width, or as many columns
 * as one ring slot holds if fewer); Gauss-Seidel form also: seconds (the time its CTA worked
 * on it, global timer, plus the time of its async finish if it had one), kernel_variant and
 * ctas_per_sm (of the launch that finished it; 0 after an async finish), batch_form
 * (ASYFLEXA_BATCH_FORM_ASYNC after an async finish) and handed_over; for the exact check of
 * asyflexa_check use asyflexa_batch_check.
 * total: sweeps (the largest number of sweeps of any problem; async rounds: tuning sweeps
 * included),
 * block_updates (all problems), seconds (CUDA events around the solve), block_w, batch_form,
 * ctas_per_sm, kernel_variant (Gauss-Seidel form: consumer warps per CTA), status (OK if all
 * done). */
int asyflexa_batch_solve(asyflexa_batch_t hb, void* const* xs, const double* f_star, asyflexa_stats* per,
                         asyflexa_stats* total);

/* The exact check of asyflexa_check (exact residual, F, gap with f_star[k], stat_xhat,
 * stat_mf, KKT, nnz) for every problem at xs[k]; f_star may be NULL.  per: count entries.
 * Synchronises.  Returns the first error, else OK. */
int asyflexa_batch_check(asyflexa_batch_t hb, void* const* xs, const double* f_star, asyflexa_stats* per);

/* Release the batch and its internal handles.  NULL is a no-op. */
int asyflexa_batch_destroy(asyflexa_batch_t hb);

/* Last error message of the handle (or of the calling thread for NULL).  Never NULL. */
/* ---------------------------------------------------------------- multi-lane form
 * k LASSO problems ("lanes") that share A and differ in b and lambda -- a lambda path or
 * several data vectors -- solved together: every block update of Algorithm 1 is done for all
 * lanes at once, its two products G = A_i^T R~ (w x k) and R += A_i Delta_i (m x k) on the
 * tensor cores (TF32 with a hi/lo split, FP32-grade products, FP64 residuals), so each byte of
 * A serves k lanes.  Blocks of w = 32 columns; async mode.  By default every solve starts with
 * max(1, 2m / 32) CTAs (at most 2 per SM), i.e. up to 2m columns of each lane in flight, and
 * halves the grid whenever a check interval raises some lane's F (too many updates in flight);
 * opts.num_ctas > 0 fixes the grid.
 *
 * prob:    FP32 A (m x n, lda) and FP32 vectors; LASSO loss; no box, linear term or master
 *          copy (EUNSUPPORTED otherwise).  prob->b and prob->lambda are ignored.
 * k:       1..64 lanes.  B: device FP32, lane l's b at B + l * ldb (ldb >= m).
 * lambdas: host, k weights.  opts: gamma, tau, tau_rel, refresh_every (exact residual
 *          recomputation), check_every, max_sweeps, tol_gap, tol_stat, switch_tol (stall test
 *          for lanes without f_star), num_ctas.
 * Borrowed like asyflexa_create's pointers; the handle owns its residuals and iterates. */
typedef struct asyflexa_multi_s* asyflexa_multi_t;
int asyflexa_multi_create(asyflexa_multi_t* h, const asyflexa_problem* prob, int32_t k, const void* B, int64_t ldb,
                          const double* lambdas, const asyflexa_opts* opts, void* cuda_stream);
/* Solve all lanes from the iterates in X (device FP32, lane l's x at X + l * ldx, ldx >= n),
 * written back in place.  A lane is done when (F - f_star[l]) / |f_star[l]| <= tol_gap (or,
 * with f_star NULL or NaN, when a check interval lowers F by <= switch_tol |F|) and its
 * ||xhat(x) - x||_inf / max(1, ||x||_inf) <= tol_stat.  The in-loop test uses the tensor-core
 * gradients; when every lane has passed it, every lane is checked exactly at its returned
 * iterate (r = A x - b and A^T r of all lanes with error-free FP32 products and sums, as
 * accurate as FP64 accumulation), and a lane that fails that check is finished from its
 * iterate by the single-lane solver (FP32 products, exact checks; per[l].polish_sweeps counts
 * its sweeps) within the sweeps left.  per (k entries; F, gap, stationarity and nnz of the
 * exact check, or the finishing solve's statistics) and total may be NULL.  B (the
 * data vectors, lane l's b at B + l * ldb) must stay valid for the life of the handle.
 * Returns OK when every lane is done, ENOTCONV at max_sweeps, or an error. */
int asyflexa_multi_solve(asyflexa_multi_t h, void* X, int64_t ldx, const double* f_star, asyflexa_stats* per,
                         asyflexa_stats* total);
int asyflexa_multi_destroy(asyflexa_multi_t h);

const char* asyflexa_last_error(asyflexa_t h);

#ifdef __cplusplus
}
#endif

#endif /* ASYFLEXA_H */
