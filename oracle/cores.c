/* Multi-core CPU form of Algorithm 1 for LASSO, in FP64: the shared-memory setup of the
 * experiments in Section 4 (variables partitioned among the cores, one core per partition,
 * no locks), used to time the method against the number of cores as Section 4.2 does.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests and by the CPU timing leg of the benchmark,
 * never by the product path.  Plain C, no blocking or vectorisation beyond
 * what the compiler does on its own; the GPU library shares nothing with it.
 *
 * Problem (Section 4.2): F(x) = 0.5 ||Ax - b||^2 + lam ||x||_1 over R^n, A m x n stored in
 * FP32 column-major (column j at At + j * lda), converted to FP64 element by element.
 *
 * Each thread owns the contiguous range of blocks [t N / c, (t + 1) N / c) of the N blocks of
 * w columns (Assumption D4: no other thread writes those x_j).  For each of its blocks, in
 * order, it
 *   S.2  reads the shared state (a stale, possibly inconsistent read: other threads write it
 *        meanwhile) and forms the block's partial gradients g_j;
 *   eq. 2  computes the best response x^_j = soft(x_j - g_j / d_j, lam / d_j) with
 *        d_j = ||a_j||^2 + tau (x^_j = 0 when d_j = 0);
 *   S.4  steps x_j <- x_j + gamma (x^_j - x_j).
 * Two forms of the shared state:
 *   residual form (Q == NULL): the threads share r = Ax - b; g_j = a_j^T r, and a step adds
 *        a_j Delta_j to r element by element with a lock-free compare-and-swap (a plain add
 *        with one thread) -- the form the GPU library uses;
 *   Gram form: the threads share x; g_j = (Q x)_j - q_j with Q = A^T A and q = A^T b given
 *        precomputed (the paper's experiments precompute both offline), and a step writes
 *        only x_j.
 * After every sweep of all threads a barrier lets thread 0 evaluate F and stop once
 * (F - F*) / |F*| < tol: the relative error of Section 4.2.  With one thread the iteration is
 * the cyclic block Gauss-Seidel method.
 */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

typedef struct {
    int64_t m, n, lda;
    const float* At;
    const double *b, *Q, *q; /* Q n x n row-major, q length n (Gram form) or NULL */
    double lam, gamma, f_star, tol;
    const double* d;
    uint64_t* x; /* FP64 bit patterns: written by the owner, read by all (Gram form) */
    uint64_t* r; /* FP64 bit patterns, read and added to atomically (residual form) */
    double* rr;  /* thread 0's scratch for the Gram form's check */
    int w, threads, max_sweeps;
    pthread_barrier_t bar;
    int stop, sweeps;
    double F, check_seconds;
    long long updates;
} shared_t;

typedef struct {
    shared_t* s;
    int t;
} arg_t;

static double bits_to_f64(uint64_t u) {
    double v;
    memcpy(&v, &u, sizeof v);
    return v;
}

static uint64_t f64_to_bits(double v) {
    uint64_t u;
    memcpy(&u, &v, sizeof u);
    return u;
}

static double load_r(const uint64_t* r, int64_t i) {
    return bits_to_f64(__atomic_load_n(&r[i], __ATOMIC_RELAXED));
}

static void store_x(uint64_t* x, int64_t j, double v) {
    __atomic_store_n(&x[j], f64_to_bits(v), __ATOMIC_RELAXED);
}

static double seconds_between(const struct timespec* a, const struct timespec* b) {
    return (double)(b->tv_sec - a->tv_sec) + 1e-9 * (double)(b->tv_nsec - a->tv_nsec);
}

/* r = Ax - b formed anew in FP64 over the nonzero x_j */
static void residual_anew(int64_t m, int64_t n, int64_t lda, const float* At, const double* b, const uint64_t* x,
                          double* rr) {
    for (int64_t i = 0; i < m; ++i) rr[i] = -b[i];
    for (int64_t j = 0; j < n; ++j) {
        const double xj = load_r(x, j);
        if (xj != 0.0)
            for (int64_t i = 0; i < m; ++i) rr[i] += (double)At[j * lda + i] * xj;
    }
}

static void add_r(uint64_t* r, int64_t i, double v, int shared) {
    if (!shared) {
        r[i] = f64_to_bits(bits_to_f64(r[i]) + v);
        return;
    }
    uint64_t old = __atomic_load_n(&r[i], __ATOMIC_RELAXED);
    for (;;) {
        const uint64_t nw = f64_to_bits(bits_to_f64(old) + v);
        if (__atomic_compare_exchange_n(&r[i], &old, nw, 1, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) return;
    }
}

static double soft(double v, double t) {
    const double a = fabs(v) - t;
    return a > 0.0 ? copysign(a, v) : 0.0;
}

/* F(x) = 0.5 ||r||^2 + lam ||x||_1 from the maintained residual (residual form) or from r
 * formed anew (Gram form) */
static double objective_now(const shared_t* s) {
    double rr = 0.0, l1 = 0.0;
    if (s->Q) residual_anew(s->m, s->n, s->lda, s->At, s->b, s->x, s->rr);
    for (int64_t i = 0; i < s->m; ++i) {
        const double v = s->Q ? s->rr[i] : load_r(s->r, i);
        rr += v * v;
    }
    for (int64_t j = 0; j < s->n; ++j) l1 += fabs(load_r(s->x, j));
    return 0.5 * rr + s->lam * l1;
}

static void* worker(void* p) {
    arg_t* a = (arg_t*)p;
    shared_t* s = a->s;
    const int64_t nb = (s->n + s->w - 1) / s->w;
    const int64_t b0 = (int64_t)a->t * nb / s->threads, b1 = (int64_t)(a->t + 1) * nb / s->threads;
    const int shared = s->threads > 1;
    double* g = (double*)malloc(sizeof(double) * (size_t)s->w);
    double* dl = (double*)malloc(sizeof(double) * (size_t)s->w);
    long long updates = 0;
    for (int sweep = 0; sweep < s->max_sweeps; ++sweep) {
        for (int64_t blk = b0; blk < b1; ++blk) {
            const int64_t j0 = blk * s->w;
            const int64_t j1 = j0 + s->w < s->n ? j0 + s->w : s->n;
            for (int64_t j = j0; j < j1; ++j) { /* S.2: gradient at the read of r, or of x */
                double acc = 0.0;
                if (s->Q) {
                    const double* qj = s->Q + j * s->n;
                    for (int64_t k = 0; k < s->n; ++k) acc += qj[k] * load_r(s->x, k);
                    acc -= s->q[j];
                } else {
                    const float* aj = s->At + j * s->lda;
                    for (int64_t i = 0; i < s->m; ++i) acc += (double)aj[i] * load_r(s->r, i);
                }
                g[j - j0] = acc;
            }
            for (int64_t j = j0; j < j1; ++j) { /* eq. 2 and S.4 */
                const double dj = s->d[j], xj = load_r(s->x, j);
                const double xh = dj > 0.0 ? soft(xj - g[j - j0] / dj, s->lam / dj) : 0.0;
                const double delta = s->gamma * (xh - xj);
                store_x(s->x, j, xj + delta);
                dl[j - j0] = delta;
            }
            if (s->Q) {
                ++updates;
                continue;
            }
            for (int64_t j = j0; j < j1; ++j) { /* r += a_j Delta_j */
                const double delta = dl[j - j0];
                if (delta == 0.0) continue;
                const float* aj = s->At + j * s->lda;
                for (int64_t i = 0; i < s->m; ++i) add_r(s->r, i, (double)aj[i] * delta, shared);
            }
            ++updates;
        }
        pthread_barrier_wait(&s->bar);
        if (a->t == 0) { /* the check; the other threads wait, so its time is left out */
            struct timespec c0, c1;
            clock_gettime(CLOCK_MONOTONIC, &c0);
            s->sweeps = sweep + 1;
            s->F = objective_now(s);
            if (s->f_star == s->f_star && (s->F - s->f_star) / fabs(s->f_star) < s->tol) s->stop = 1;
            clock_gettime(CLOCK_MONOTONIC, &c1);
            s->check_seconds += seconds_between(&c0, &c1);
        }
        pthread_barrier_wait(&s->bar);
        if (s->stop) break;
    }
    __atomic_fetch_add(&s->updates, updates, __ATOMIC_RELAXED);
    free(g);
    free(dl);
    return NULL;
}

/* Runs the partitioned method from x (in/out, length n) until the relative error of F drops
 * below tol (f_star NaN: never) or max_sweeps sweeps are done.  Q (n x n row-major, A^T A)
 * and q (A^T b), both FP64, select the Gram form; pass NULL for the residual form.
 * out[0] sweeps, out[1] F(x) recomputed from r = Ax - b formed anew in FP64, out[2] wall
 * seconds of the iteration (threads started to threads joined) without the checks, out[3]
 * block updates, out[4] F at the last check, out[5] seconds spent in the checks.  Returns 0,
 * or -1 on bad arguments or a failed allocation. */
int oracle_cores_lasso(int64_t m, int64_t n, int64_t lda, const float* At, const double* b, const double* Q,
                       const double* q, double lam, double gamma, double tau, int w, int threads, int max_sweeps,
                       double f_star, double tol, double* x, double* out) {
    if (m <= 0 || n <= 0 || lda < m || w <= 0 || threads <= 0 || max_sweeps < 0 || !At || !b || !x || !out ||
        (Q == NULL) != (q == NULL))
        return -1;
    shared_t s;
    memset(&s, 0, sizeof s);
    s.m = m;
    s.n = n;
    s.lda = lda;
    s.At = At;
    s.b = b;
    s.Q = Q;
    s.q = q;
    s.lam = lam;
    s.gamma = gamma;
    s.f_star = f_star;
    s.tol = tol;
    s.w = w;
    s.threads = threads;
    s.max_sweeps = max_sweeps;
    double* d = (double*)malloc(sizeof(double) * (size_t)n);
    uint64_t* xb = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t* r = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)m);
    double* rr = (double*)malloc(sizeof(double) * (size_t)m);
    pthread_t* tid = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    arg_t* args = (arg_t*)malloc(sizeof(arg_t) * (size_t)threads);
    int rc = -1, started = 0;
    if (!d || !xb || !r || !rr || !tid || !args) goto done;
    /* d_j = ||a_j||^2 + tau (Section 4.2 surrogate: exact coordinate curvature plus tau) */
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < m; ++i) acc += (double)At[j * lda + i] * (double)At[j * lda + i];
        d[j] = acc + tau;
    }
    for (int64_t j = 0; j < n; ++j) xb[j] = f64_to_bits(x[j]);
    residual_anew(m, n, lda, At, b, xb, rr);
    for (int64_t i = 0; i < m; ++i) r[i] = f64_to_bits(rr[i]);
    s.d = d;
    s.x = xb;
    s.r = r;
    s.rr = rr;
    if (pthread_barrier_init(&s.bar, NULL, (unsigned)threads) != 0) goto done;
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    for (int t = 0; t < threads; ++t) {
        args[t].s = &s;
        args[t].t = t;
        if (pthread_create(&tid[t], NULL, worker, &args[t]) != 0) break;
        ++started;
    }
    if (started < threads) {
        /* the started threads would wait at the barrier for ever: the process cannot recover */
        abort();
    }
    for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
    clock_gettime(CLOCK_MONOTONIC, &t1);
    pthread_barrier_destroy(&s.bar);
    for (int64_t j = 0; j < n; ++j) x[j] = bits_to_f64(xb[j]);
    /* F(x) with r formed anew */
    residual_anew(m, n, lda, At, b, xb, rr);
    double qq = 0.0, l1 = 0.0;
    for (int64_t i = 0; i < m; ++i) qq += rr[i] * rr[i];
    for (int64_t j = 0; j < n; ++j) l1 += fabs(x[j]);
    out[0] = (double)s.sweeps;
    out[1] = 0.5 * qq + lam * l1;
    out[2] = seconds_between(&t0, &t1) - s.check_seconds;
    out[3] = (double)s.updates;
    out[4] = s.F;
    out[5] = s.check_seconds;
    rc = 0;
done:
    free(d);
    free(xb);
    free(r);
    free(rr);
    free(tid);
    free(args);
    return rc;
}
