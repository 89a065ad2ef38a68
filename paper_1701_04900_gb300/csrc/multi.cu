// Multi-right-hand-side form of the block update (C ABI asyflexa_multi_*): k LASSO problems
// sharing A (a lambda path, or several data vectors), every block update done for all lanes at
// once by the tensor-core kernel of sweep_multi.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "sweep_multi.cuh"

namespace asyflexa_internal {
void set_thread_error(const std::string& msg);
}  // namespace asyflexa_internal

namespace {

// Two CUDA events destroyed with the scope (error returns included).
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

int mfail(const std::string& m, int code = ASYFLEXA_EINVAL) {
    asyflexa_internal::set_thread_error(m);
    return code;
}

#define MCK(call, where)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            (void)cudaGetLastError();                                                            \
            return mfail(std::string(where) + ": " + cudaGetErrorString(e_), ASYFLEXA_ECUDA);     \
        }                                                                                        \
    } while (0)

template <int KP>
const void* multi_kernel() { return reinterpret_cast<const void*>(asyflexa::sweep_multi_kernel<KP>); }

}  // namespace

struct asyflexa_multi_s {
    asyflexa_t base = nullptr;  // single-lane handle on lane 0: weights d_j, geometry, stream
    int k = 0, kp = 0, grid = 0;
    int grid_start = 0;     // the grid every solve starts from
    bool grid_auto = false; // num_ctas 0: the grid halves when a check interval raises some lane's F
    int64_t m = 0, n = 0;
    asyflexa_opts opts{};
    cudaStream_t stream = nullptr;
    std::vector<double> lam;
    double* lam_d = nullptr;
    const float* B = nullptr;  // the caller's k x ldb data vectors (lane l at B + l ldb)
    int64_t ldb = 0;
    double* Bm = nullptr;     // m x kp: -b of every lane (initial residual)
    double* R = nullptr;      // m x kp
    float* X = nullptr;       // n x kp
    float* G = nullptr;       // n x kp (checks)
    double* Rx = nullptr;     // m x kp: exact residuals (checks)
    float2* Rhl = nullptr;    // m x kp: the same as FP32 (hi, lo) pairs
    double* Gx = nullptr;     // n x kp: exact gradients (checks)
    float* dinv = nullptr;    // n: 1/d_j (FP32)
    float* thr = nullptr;     // n x kp: lam_l / d_j (FP32)
    double* norms = nullptr;  // 3 kp
    unsigned long long* meas = nullptr;  // 2 kp
    unsigned long long* counters = nullptr;
    unsigned long long* hist = nullptr;
    size_t smem = 0;
    long long launches = 0;
};

namespace {

int launch_multi(asyflexa_multi_s& H, int mode, int sweeps) {
    asyflexa::MultiParams p{};
    const asyflexa_problem& P = H.base->prob;
    p.A = static_cast<const float*>(P.A);
    p.lda = P.lda;
    p.m = H.m;
    p.n = H.n;
    p.R = H.R;
    p.X = H.X;
    p.dw = H.base->dw;
    p.lam = H.lam_d;
    p.dinv = H.dinv;
    p.thr = H.thr;
    p.gamma = H.opts.gamma;
    p.kp = H.kp;
    p.nblocks = static_cast<int>((H.n + asyflexa::kMW - 1) / asyflexa::kMW);
    p.sweeps = sweeps;
    p.mode = mode;
    p.G = H.G;
    p.counters = H.counters;
    p.hist = H.hist;
    const void* fn = H.kp == 8    ? multi_kernel<8>()
                     : H.kp == 16 ? multi_kernel<16>()
                     : H.kp == 32 ? multi_kernel<32>()
                                  : multi_kernel<64>();
    void* args[] = {&p};
    // the refresh and the gradient pass make no step, so they may use every SM
    const int grid = mode == 0 ? H.grid : std::min(p.nblocks, H.base->sm_count * 2);
    MCK(cudaLaunchKernel(fn, dim3(grid), dim3(asyflexa::kMThreads), args, H.smem, H.stream), "multi sweep launch");
    ++H.launches;
    return ASYFLEXA_OK;
}

// R = -B + A X (exact up to the FP32-grade products, FP64 accumulation)
int multi_refresh(asyflexa_multi_s& H) {
    MCK(cudaMemcpyAsync(H.R, H.Bm, H.m * H.kp * sizeof(double), cudaMemcpyDeviceToDevice, H.stream), "reset R");
    return launch_multi(H, 1, 1);
}

template <int KP>
void launch_norms(asyflexa_multi_s& H, const double* R) {
    asyflexa::multi_norms_kernel<KP><<<H.base->sm_count * 2, 256, 0, H.stream>>>(R, H.m, H.X, H.n, H.norms);
}

// Per-lane F = 0.5 ||r||^2 + lam ||x||_1 and nnz from the residuals R (the sweeps' by default).
// Synchronises.
int multi_objective(asyflexa_multi_s& H, std::vector<double>& F, std::vector<double>& nnz, const double* R = nullptr) {
    if (!R) R = H.R;
    MCK(cudaMemsetAsync(H.norms, 0, 3 * H.kp * sizeof(double), H.stream), "clear norms");
    switch (H.kp) {
        case 8: launch_norms<8>(H, R); break;
        case 16: launch_norms<16>(H, R); break;
        case 32: launch_norms<32>(H, R); break;
        default: launch_norms<64>(H, R); break;
    }
    ++H.launches;
    MCK(cudaGetLastError(), "norms launch");
    std::vector<double> v(3 * H.kp);
    MCK(cudaMemcpyAsync(v.data(), H.norms, v.size() * sizeof(double), cudaMemcpyDeviceToHost, H.stream), "read norms");
    MCK(cudaStreamSynchronize(H.stream), "synchronize");
    F.assign(H.k, 0.0);
    nnz.assign(H.k, 0.0);
    for (int l = 0; l < H.k; ++l) {
        F[l] = 0.5 * v[l] + H.lam[l] * v[H.kp + l];
        nnz[l] = v[2 * H.kp + l];
    }
    return ASYFLEXA_OK;
}

template <int KP>
void launch_stat(asyflexa_multi_s& H) {
    asyflexa::multi_stat_kernel<KP><<<H.base->sm_count * 4, 256, 0, H.stream>>>(H.G, H.X, H.base->dw, H.lam_d, H.n,
                                                                                H.meas);
}

// Per-lane ||xhat(x) - x||_inf / max(1, ||x||_inf) from the gradients of the current R.
int multi_stationarity(asyflexa_multi_s& H, std::vector<double>& stat) {
    int rc = launch_multi(H, 2, 1);
    if (rc) return rc;
    MCK(cudaMemsetAsync(H.meas, 0, 2 * H.kp * sizeof(unsigned long long), H.stream), "clear measures");
    switch (H.kp) {
        case 8: launch_stat<8>(H); break;
        case 16: launch_stat<16>(H); break;
        case 32: launch_stat<32>(H); break;
        default: launch_stat<64>(H); break;
    }
    ++H.launches;
    MCK(cudaGetLastError(), "stationarity launch");
    std::vector<unsigned long long> v(2 * H.kp);
    MCK(cudaMemcpyAsync(v.data(), H.meas, v.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, H.stream),
        "read measures");
    MCK(cudaStreamSynchronize(H.stream), "synchronize");
    stat.assign(H.k, 0.0);
    for (int l = 0; l < H.k; ++l) {
        double dx, ax;
        std::memcpy(&dx, &v[l], sizeof dx);
        std::memcpy(&ax, &v[H.kp + l], sizeof ax);
        stat[l] = dx / std::max(1.0, ax);
    }
    return ASYFLEXA_OK;
}

template <int KP>
void launch_exact(asyflexa_multi_s& H) {
    const int gr = static_cast<int>((H.m + asyflexa::kXT - 1) / asyflexa::kXT);
    const int gg = static_cast<int>((H.n + asyflexa::kXT - 1) / asyflexa::kXT);
    const float* A = static_cast<const float*>(H.base->prob.A);
    asyflexa::multi_exact_residual_kernel<KP><<<gr, 256, 0, H.stream>>>(A, H.base->prob.lda, H.m, H.n, H.X, H.B,
                                                                        H.ldb, H.k, H.Rx, H.Rhl);
    asyflexa::multi_exact_grad_kernel<KP><<<gg, 256, 0, H.stream>>>(A, H.base->prob.lda, H.m, H.n, H.Rhl, H.Gx);
    asyflexa::multi_stat64_kernel<KP><<<H.base->sm_count * 4, 256, 0, H.stream>>>(H.Gx, H.X, H.base->dw, H.lam_d,
                                                                                   H.n, H.meas);
}

// The exact check of every lane at the current iterates: R = A X - B and G = A^T R with
// error-free FP32 products and sums (FP64-grade), then per lane F, nnz and
// ||xhat(x) - x||_inf / max(1, ||x||_inf).  Synchronises.
int multi_exact_check(asyflexa_multi_s& H, std::vector<double>& F, std::vector<double>& nnz,
                      std::vector<double>& stat) {
    MCK(cudaMemsetAsync(H.meas, 0, 2 * H.kp * sizeof(unsigned long long), H.stream), "clear measures");
    switch (H.kp) {
        case 8: launch_exact<8>(H); break;
        case 16: launch_exact<16>(H); break;
        case 32: launch_exact<32>(H); break;
        default: launch_exact<64>(H); break;
    }
    H.launches += 3;
    MCK(cudaGetLastError(), "exact check launch");
    int rc = multi_objective(H, F, nnz, H.Rx);
    if (rc) return rc;
    std::vector<unsigned long long> v(2 * H.kp);
    MCK(cudaMemcpyAsync(v.data(), H.meas, v.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, H.stream),
        "read measures");
    MCK(cudaStreamSynchronize(H.stream), "synchronize");
    stat.assign(H.k, 0.0);
    for (int l = 0; l < H.k; ++l) {
        double dx, ax;
        std::memcpy(&dx, &v[l], sizeof dx);
        std::memcpy(&ax, &v[H.kp + l], sizeof ax);
        stat[l] = dx / std::max(1.0, ax);
    }
    return ASYFLEXA_OK;
}

// Finishes lane l from its iterate x_l (the caller's layout) with the single-lane solver (FP32
// products, exact checks), at most max_sweeps sweeps: for a lane whose tensor-core iterate the
// exact check rejects.  st: the solve's statistics.
int multi_lane_polish(asyflexa_multi_s& H, int l, float* x_l, double f_star_l, int max_sweeps, asyflexa_stats* st) {
    asyflexa_s& b = *H.base;
    b.prob.b = H.B + static_cast<int64_t>(l) * H.ldb;
    b.prob.lambda = H.lam[l];
    b.opts.f_star = f_star_l;
    b.opts.max_sweeps = max_sweeps;
    b.r_valid = false;
    std::memset(st, 0, sizeof *st);
    const int rc = asyflexa_solve(H.base, x_l, st);
    b.prob.b = H.B;
    b.prob.lambda = H.lam[0];
    b.opts.f_star = NAN;
    b.opts.max_sweeps = H.opts.max_sweeps;
    b.r_valid = false;
    if (rc < 0) return mfail(std::string("lane polish: ") + asyflexa_last_error(H.base), rc);
    return ASYFLEXA_OK;
}

}  // namespace

extern "C" {

int asyflexa_multi_destroy(asyflexa_multi_t H) {
    if (!H) return ASYFLEXA_OK;
    if (H->stream) cudaStreamSynchronize(H->stream);
    void* ptrs[] = {H->lam_d, H->Bm, H->R, H->X, H->G, H->norms, H->meas, H->counters, H->hist, H->dinv, H->thr, H->Rx, H->Rhl, H->Gx};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (H->base) asyflexa_destroy(H->base);
    delete H;
    return ASYFLEXA_OK;
}

int asyflexa_multi_create(asyflexa_multi_t* out, const asyflexa_problem* prob, int32_t k, const void* B, int64_t ldb,
                          const double* lambdas, const asyflexa_opts* opts, void* stream) {
    if (!out) return mfail("out is NULL");
    *out = nullptr;
    if (!prob || !B || !lambdas || !opts) return mfail("prob, B, lambdas or opts is NULL");
    if (k < 1 || k > asyflexa::kMKMax) return mfail("k must be in [1, 64]");
    if (prob->a_dtype != ASYFLEXA_F32 || prob->x_dtype != ASYFLEXA_F32)
        return mfail("the multi-lane form takes FP32 A and vectors", ASYFLEXA_EUNSUPPORTED);
    if (prob->loss != ASYFLEXA_LOSS_LASSO || prob->lo || prob->hi || prob->lin || prob->A_master)
        return mfail("the multi-lane form solves plain LASSO lanes (no box, linear term or master copy)",
                     ASYFLEXA_EUNSUPPORTED);
    if (ldb < prob->m) return mfail("ldb must be >= m");
    for (int l = 0; l < k; ++l)
        if (!(lambdas[l] >= 0.0) || !std::isfinite(lambdas[l])) return mfail("every lambda must be finite and >= 0");
    auto* H = new (std::nothrow) asyflexa_multi_s();
    if (!H) return mfail("host allocation failed", ASYFLEXA_ENOMEM);
    auto fail = [&](int rc) {
        asyflexa_multi_destroy(H);
        return rc;
    };
    // the single-lane handle of lane 0 validates the problem and computes the weights d_j
    asyflexa_problem p0 = *prob;
    p0.b = B;
    p0.lambda = lambdas[0];
    asyflexa_opts o = *opts;
    o.mode = ASYFLEXA_ASYNC;
    o.block_w = asyflexa::kMW;
    o.profile = 0;
    o.exact_grad = 0;  // the multi-lane kernel has its own split-TF32 arithmetic
    int rc = asyflexa_create(&H->base, &p0, &o, stream);
    if (rc) return fail(mfail(std::string("lane 0: ") + asyflexa_last_error(nullptr), rc));
    H->opts = o;
    H->stream = static_cast<cudaStream_t>(stream);
    H->B = static_cast<const float*>(B);
    H->ldb = ldb;
    H->k = k;
    H->kp = k <= 8 ? 8 : k <= 16 ? 16 : k <= 32 ? 32 : 64;
    H->m = prob->m;
    H->n = prob->n;
    H->lam.assign(lambdas, lambdas + k);
    const int nblocks = static_cast<int>((H->n + asyflexa::kMW - 1) / asyflexa::kMW);
    // updates in flight: every lane has grid * w columns in flight.  The default starts at up to
    // 2 m (2 CTAs per SM at most: a lambda path converged as fast in sweeps as with m, a single
    // problem diverged at 2.4 m) and halves the grid whenever a check interval raises some
    // lane's F, the sign of too many updates in flight
    const int cap = static_cast<int>(std::max<int64_t>(1, 2 * H->m / asyflexa::kMW));
    H->grid_auto = opts->num_ctas <= 0;
    H->grid = opts->num_ctas > 0 ? opts->num_ctas : std::min(cap, H->base->sm_count * 2);
    H->grid = std::max(1, std::min(H->grid, nblocks));
    H->grid_start = H->grid;
    std::vector<double> lp(H->kp, INFINITY);
    for (int l = 0; l < k; ++l) lp[l] = lambdas[l];
    cudaError_t e = cudaMalloc(&H->lam_d, H->kp * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->Bm, H->m * H->kp * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->R, H->m * H->kp * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->X, H->n * H->kp * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&H->G, H->n * H->kp * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&H->dinv, H->n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&H->Rx, H->m * H->kp * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->Rhl, H->m * H->kp * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&H->Gx, H->n * H->kp * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->thr, H->n * H->kp * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&H->norms, 3 * H->kp * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&H->meas, 2 * H->kp * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&H->counters, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&H->hist, 32 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(mfail(std::string("multi allocation: ") + cudaGetErrorString(e), ASYFLEXA_ENOMEM));
    }
    H->smem = sizeof(asyflexa::MultiSmem);
    const void* fns[] = {multi_kernel<8>(), multi_kernel<16>(), multi_kernel<32>(), multi_kernel<64>()};
    for (const void* f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(H->smem));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(mfail(std::string("multi smem attribute: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
        }
    }
    e = cudaMemcpyAsync(H->lam_d, lp.data(), H->kp * sizeof(double), cudaMemcpyHostToDevice, H->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(H->counters, 0, 4 * sizeof(unsigned long long), H->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(H->hist, 0, 32 * sizeof(unsigned long long), H->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(mfail(std::string("multi set-up: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
    }
    // the elementwise step's coefficient tables
    {
        const int grid = H->base->sm_count * 4;
        switch (H->kp) {
            case 8: asyflexa::multi_coef_kernel<8><<<grid, 256, 0, H->stream>>>(H->base->dw, H->lam_d, H->n, H->dinv, H->thr); break;
            case 16: asyflexa::multi_coef_kernel<16><<<grid, 256, 0, H->stream>>>(H->base->dw, H->lam_d, H->n, H->dinv, H->thr); break;
            case 32: asyflexa::multi_coef_kernel<32><<<grid, 256, 0, H->stream>>>(H->base->dw, H->lam_d, H->n, H->dinv, H->thr); break;
            default: asyflexa::multi_coef_kernel<64><<<grid, 256, 0, H->stream>>>(H->base->dw, H->lam_d, H->n, H->dinv, H->thr); break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(mfail(std::string("multi set-up: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
    }
    // Bm = -B laid out m x kp
    asyflexa::multi_transpose_kernel<float, double><<<H->base->sm_count * 2, 256, 0, H->stream>>>(
        static_cast<const float*>(B), ldb, H->Bm, 0, H->m, k, H->kp, 0, -1.0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(mfail(std::string("multi set-up: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
    *out = H;
    return ASYFLEXA_OK;
}

int asyflexa_multi_solve(asyflexa_multi_t H, void* X, int64_t ldx, const double* f_star, asyflexa_stats* per,
                         asyflexa_stats* total) {
    if (!H || !X) return mfail("handle or X is NULL");
    if (ldx < H->n) return mfail("ldx must be >= n");
    EventPair ev_e0;
    MCK(cudaEventCreate(&ev_e0.a), "event");
    MCK(cudaEventCreate(&ev_e0.b), "event");
    cudaEvent_t e0 = ev_e0.a, e1 = ev_e0.b;
    MCK(cudaEventRecord(e0, H->stream), "event record");
    asyflexa::multi_transpose_kernel<float, float><<<H->base->sm_count * 2, 256, 0, H->stream>>>(
        static_cast<const float*>(X), ldx, H->X, 0, H->n, H->k, H->kp, 0, 1.0);
    MCK(cudaGetLastError(), "gather iterates");
    int rc = multi_refresh(*H);
    if (rc) return rc;
    const int k = H->k;
    std::vector<int> done(k, 0);
    std::vector<long long> conv_sweeps(k, -1);
    std::vector<double> F, Fprev(k, NAN), nnz, stat(k, NAN);
    long long sweeps = 0;
    int since_refresh = 0;
    const int step = std::max(1, std::min(H->opts.check_every, H->opts.refresh_every));
    H->grid = H->grid_start;
    std::vector<double> Flast(k, NAN);  // every lane's F at the previous check (grid control)
    // A lane that the in-loop test (tensor-core gradients) passes is confirmed by the exact check
    // at its returned iterate.  The split-TF32 products put the multi-lane fixed point up to
    // about 1e-6 away in that measure, so a lane the exact check rejects is finished by the
    // single-lane solver from its iterate (its FP32 products and exact checks).
    std::vector<asyflexa_stats> exact(k);
    std::vector<long long> polish(k, 0);
    while (sweeps < H->opts.max_sweeps) {
        const int ks = static_cast<int>(std::min<long long>(step, H->opts.max_sweeps - sweeps));
        rc = launch_multi(*H, 0, ks);
        if (rc) return rc;
        sweeps += ks;
        since_refresh += ks;
        if (since_refresh >= H->opts.refresh_every) {
            rc = multi_refresh(*H);
            if (rc) return rc;
            since_refresh = 0;
        }
        rc = multi_objective(*H, F, nnz);
        if (rc) return rc;
        if (H->grid_auto && H->grid > 1) {
            bool rose = false;
            for (int l = 0; l < k; ++l)
                rose |= std::isfinite(Flast[l]) && F[l] > Flast[l] + 1e-12 * std::fabs(Flast[l]);
            if (rose) H->grid = std::max(1, H->grid / 2);
        }
        Flast = F;
        bool need_stat = false;
        for (int l = 0; l < k; ++l) {
            if (!std::isfinite(F[l])) return mfail("objective is not finite", ASYFLEXA_ENONFINITE);
            if (done[l]) continue;
            const bool known = f_star && std::isfinite(f_star[l]);
            const bool gap_ok = known ? (F[l] - f_star[l]) / std::fabs(f_star[l]) <= H->opts.tol_gap
                                      : std::isfinite(Fprev[l]) &&
                                            Fprev[l] - F[l] <= H->opts.switch_tol * std::fabs(F[l]);
            if (gap_ok) need_stat = true;
            Fprev[l] = F[l];
        }
        if (need_stat) {
            rc = multi_stationarity(*H, stat);
            if (rc) return rc;
            for (int l = 0; l < k; ++l) {
                if (done[l]) continue;
                const bool known = f_star && std::isfinite(f_star[l]);
                const bool gap_ok =
                    !known || (F[l] - f_star[l]) / std::fabs(f_star[l]) <= H->opts.tol_gap;
                if (gap_ok && stat[l] <= H->opts.tol_stat) {
                    done[l] = 1;
                    conv_sweeps[l] = sweeps;
                }
            }
        }
        if (std::all_of(done.begin(), done.end(), [](int d) { return d != 0; })) break;
    }
    // the exact check of every lane at its iterate; a lane the in-loop test passed but the exact
    // check rejects is finished by the single-lane solver
    std::vector<double> Fx, nnzx, statx;
    rc = multi_exact_check(*H, Fx, nnzx, statx);
    if (rc) return rc;
    asyflexa::multi_transpose_kernel<float, float><<<H->base->sm_count * 2, 256, 0, H->stream>>>(
        H->X, 0, static_cast<float*>(X), ldx, H->n, H->k, H->kp, 1, 1.0);
    MCK(cudaGetLastError(), "scatter iterates");
    for (int l = 0; l < k; ++l) {
        const double fsl = f_star ? f_star[l] : NAN;
        asyflexa_stats& q = exact[l];
        std::memset(&q, 0, sizeof q);
        q.F = Fx[l];
        q.rel_gap = std::isfinite(fsl) ? (Fx[l] - fsl) / std::fabs(fsl) : NAN;
        q.stat_xhat = statx[l];
        q.stat_mf = q.kkt_viol = q.dual_gap = NAN;
        q.nnz = static_cast<long long>(nnzx[l]);
        q.checked = 1;
        const bool gap_ok = !std::isfinite(fsl) || q.rel_gap <= H->opts.tol_gap;
        if (!done[l] || (gap_ok && q.stat_xhat <= H->opts.tol_stat)) continue;
        const long long left = H->opts.max_sweeps - sweeps;
        if (left <= 0) {
            done[l] = 0;
            continue;
        }
        asyflexa_stats ps;
        float* xl = static_cast<float*>(X) + static_cast<int64_t>(l) * ldx;
        rc = multi_lane_polish(*H, l, xl, fsl, static_cast<int>(left), &ps);
        if (rc) return rc;
        polish[l] = ps.sweeps;
        q = ps;
        done[l] = ps.status == ASYFLEXA_OK ? 1 : 0;
    }
    MCK(cudaEventRecord(e1, H->stream), "event record");
    MCK(cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const long long nblocks = (H->n + asyflexa::kMW - 1) / asyflexa::kMW;
    int worst = ASYFLEXA_OK;
    for (int l = 0; l < k; ++l) {
        const int st = done[l] ? ASYFLEXA_OK : ASYFLEXA_ENOTCONV;
        if (st != ASYFLEXA_OK) worst = st;
        if (per) {
            asyflexa_stats s;
            std::memset(&s, 0, sizeof s);
            s = exact[l];  // F, gap, stationarity, KKT measures and nnz of the exact check
            s.sweeps = (conv_sweeps[l] >= 0 ? conv_sweeps[l] : sweeps) + polish[l];
            s.polish_sweeps = polish[l];
            s.block_updates = s.sweeps * nblocks;
            s.seconds = 0.0;
            s.status = st;
            s.checked = 1;
            s.block_w = asyflexa::kMW;
            per[l] = s;
        }
    }
    if (total) {
        std::memset(total, 0, sizeof *total);
        total->sweeps = sweeps;
        total->block_updates = sweeps * nblocks * k;
        total->seconds = ms * 1e-3;
        total->status = worst;
        total->kernel_launches = H->launches;
        total->block_w = asyflexa::kMW;
        unsigned long long hist[32];
        MCK(cudaMemcpy(hist, H->hist, sizeof hist, cudaMemcpyDeviceToHost), "read hist");
        for (int b = 0; b < 32; ++b) total->staleness_hist[b] = hist[b];
    }
    return worst;
}

}  // extern "C"
