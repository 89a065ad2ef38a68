// asyflexa_adjoint: the backward pass of the LASSO solution map x*(lambda, b).
//
// Not in the paper; derived from the LASSO optimality conditions.  On the support S of x*
// with signs s = sign(x*_S), A_S^T (A_S x_S - b) + lambda s = 0, which is smooth in
// (lambda, b) while S and s stay fixed.  For a loss L(x*) with v = dL/dx*, and w the solution
// of (A_S^T A_S) w = v_S:
//     dL/dlambda = -s^T w,        dL/db = A_S w.
// w minimises 0.5 ||A_S w||^2 - v_S^T w, i.e. the same problem class as the forward solve
// with b = 0, lambda = 0 and the linear term lin = -v_S, so the library computes it with its
// own block update (an internal handle on the gathered columns A_S); the handle's exact
// residual at w is A_S w - 0 = dL/db.
//
// Every step runs in the kernels below or in the library's other kernels: the support
// selection |x_j| > rel_tol * max(1, ||x||_inf) and the gathered -v_S and s (one ordered
// pass), the column gather, the solve for w, and the reduction -s^T w.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "../../include/asyflexa.h"

namespace asyflexa_internal {
void set_thread_error(const std::string& msg);
}  // namespace asyflexa_internal

namespace {

constexpr int kSelThreads = 1024;

// One block: t = rel_tol * max(1, ||x||_inf); then, in increasing j, every j with |x_j| > t
// appends (j, -v_j, sign(x_j)) to (idx, lin, sgn); *count = |S|.  A block-wide exclusive scan
// per chunk of 1024 entries keeps the order (and so the result) deterministic.
template <typename T>
__global__ void __launch_bounds__(kSelThreads) support_select_kernel(const T* x, const T* v, int64_t n,
                                                                     double rel_tol, int32_t* idx, T* lin, T* sgn,
                                                                     int64_t* count) {
    __shared__ double red[kSelThreads / 32];
    __shared__ int wsum[kSelThreads / 32];
    __shared__ int64_t base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double mx = 0.0;
    for (int64_t j = tid; j < n; j += kSelThreads) mx = fmax(mx, fabs(static_cast<double>(x[j])));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    if (tid == 0) base = 0;
    __syncthreads();
    if (warp == 0) {
        double t = red[lane];
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    const double thr = rel_tol * fmax(1.0, red[0]);
    for (int64_t j0 = 0; j0 < n; j0 += kSelThreads) {
        const int64_t j = j0 + tid;
        const double xj = j < n ? static_cast<double>(x[j]) : 0.0;
        const bool in = j < n && fabs(xj) > thr;
        const unsigned ball = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wsum[warp] = __popc(ball);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) {
            before += w < warp ? wsum[w] : 0;
            total += wsum[w];
        }
        if (in) {
            const int64_t pos = base + before + __popc(ball & ((1u << lane) - 1u));
            idx[pos] = static_cast<int32_t>(j);
            lin[pos] = -v[j];
            sgn[pos] = xj > 0.0 ? T(1) : T(-1);
        }
        __syncthreads();
        if (tid == 0) base += total;
        __syncthreads();
    }
    if (tid == 0) *count = base;
}

// out = -sum_k sgn[k] w[k] in FP64, fixed order (one block).
template <typename T>
__global__ void __launch_bounds__(kSelThreads) neg_signed_sum_kernel(const T* sgn, const T* w, int64_t k,
                                                                     double* out) {
    __shared__ double part[kSelThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double s = 0.0;
    for (int64_t i = tid; i < k; i += kSelThreads) s += static_cast<double>(sgn[i]) * static_cast<double>(w[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[warp] = s;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < kSelThreads / 32; ++i) t += part[i];
        *out = -t;
    }
}

int afail(int code, const std::string& m) {
    asyflexa_internal::set_thread_error(m);
    return code;
}

}  // namespace

extern "C" int asyflexa_adjoint(const void* A, int64_t lda, int32_t a_dtype, int64_t m, int64_t n, const void* x,
                                const void* v, double rel_tol, const asyflexa_opts* opts, double* out_dlam,
                                double* out_db, int64_t* out_support, asyflexa_stats* out_stats, void* cuda_stream) {
    if (a_dtype != ASYFLEXA_F64 && a_dtype != ASYFLEXA_F32)
        return afail(ASYFLEXA_EUNSUPPORTED, "asyflexa_adjoint: A must be F64 or F32 storage");
    if (!A || !x || !v || !out_dlam || !out_db) return afail(ASYFLEXA_EINVAL, "asyflexa_adjoint: NULL argument");
    if (m < 1 || n < 1 || lda < m) return afail(ASYFLEXA_EINVAL, "asyflexa_adjoint: need m, n >= 1 and lda >= m");
    if (!(rel_tol >= 0.0) || !std::isfinite(rel_tol)) return afail(ASYFLEXA_EINVAL, "asyflexa_adjoint: rel_tol must be finite and >= 0");
    const bool f64 = a_dtype == ASYFLEXA_F64;
    const size_t ex = f64 ? 8 : 4;
    if ((lda * static_cast<int64_t>(ex)) % 16 != 0 || (reinterpret_cast<uintptr_t>(A) & 15u))
        return afail(ASYFLEXA_EINVAL, "asyflexa_adjoint: A must be 16-byte aligned with lda * element size a multiple of 16");
    if (n > (int64_t(1) << 31) - 1) return afail(ASYFLEXA_EINVAL, "asyflexa_adjoint: n too large");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    asyflexa_opts o;
    if (opts) {
        o = *opts;
    } else {
        // one CTA: exact cyclic Gauss-Seidel on the (small) support problem
        asyflexa_opts_default(&o);
        o.mode = ASYFLEXA_ASYNC;
        o.num_ctas = 1;
        o.block_w = 8;
        o.gamma = 1.0;
        o.max_sweeps = 2000;
        o.check_every = 5;
        o.refresh_every = 5;
        o.tol_stat = 1e-7;
    }
    o.f_star = std::nan("");

    int32_t* idx = nullptr;
    void *lin = nullptr, *sgn = nullptr, *AS = nullptr, *b0 = nullptr, *w = nullptr;
    int64_t* d_count = nullptr;
    double* d_dlam = nullptr;
    asyflexa_t h = nullptr;
    int rc = ASYFLEXA_OK;
    auto cleanup = [&]() {
        if (h) asyflexa_destroy(h);
        void* ptrs[] = {idx, lin, sgn, AS, b0, w, d_count, d_dlam};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    };
#define ACK(call, where)                                                                      \
    do {                                                                                      \
        const cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                              \
            (void)cudaGetLastError();                                                         \
            cleanup();                                                                        \
            return afail(e_ == cudaErrorMemoryAllocation ? ASYFLEXA_ENOMEM : ASYFLEXA_ECUDA,  \
                         std::string("asyflexa_adjoint: ") + where + ": " + cudaGetErrorString(e_)); \
        }                                                                                     \
    } while (0)

    ACK(cudaMalloc(&idx, n * sizeof(int32_t)), "alloc support");
    ACK(cudaMalloc(&lin, n * ex), "alloc linear term");
    ACK(cudaMalloc(&sgn, n * ex), "alloc signs");
    ACK(cudaMalloc(&d_count, sizeof(int64_t)), "alloc count");
    ACK(cudaMalloc(&d_dlam, sizeof(double)), "alloc result");
    if (f64)
        support_select_kernel<double><<<1, kSelThreads, 0, st>>>(static_cast<const double*>(x),
                                                                 static_cast<const double*>(v), n, rel_tol, idx,
                                                                 static_cast<double*>(lin), static_cast<double*>(sgn),
                                                                 d_count);
    else
        support_select_kernel<float><<<1, kSelThreads, 0, st>>>(static_cast<const float*>(x),
                                                                static_cast<const float*>(v), n, rel_tol, idx,
                                                                static_cast<float*>(lin), static_cast<float*>(sgn),
                                                                d_count);
    ACK(cudaGetLastError(), "support selection");
    int64_t k = 0;
    ACK(cudaMemcpyAsync(&k, d_count, sizeof k, cudaMemcpyDeviceToHost, st), "read support size");
    ACK(cudaStreamSynchronize(st), "synchronize");
    if (out_support) *out_support = k;
    if (out_stats) std::memset(out_stats, 0, sizeof *out_stats);
    if (k == 0) {
        // empty support: x* does not move with (lambda, b)
        *out_dlam = 0.0;
        ACK(cudaMemsetAsync(out_db, 0, m * sizeof(double), st), "clear db");
        ACK(cudaStreamSynchronize(st), "synchronize");
        cleanup();
        return ASYFLEXA_OK;
    }
    const int64_t per = 16 / static_cast<int64_t>(ex);
    const int64_t ldS = (m + per - 1) / per * per;
    ACK(cudaMalloc(&AS, static_cast<size_t>(k) * ldS * ex), "alloc A_S");
    ACK(cudaMalloc(&b0, ldS * ex), "alloc b");
    ACK(cudaMalloc(&w, k * ex), "alloc w");
    ACK(cudaMemsetAsync(b0, 0, ldS * ex, st), "clear b");
    ACK(cudaMemsetAsync(w, 0, k * ex, st), "clear w");
    rc = asyflexa_gather_columns(A, lda, a_dtype, m, idx, k, AS, ldS, cuda_stream);
    if (rc) {
        cleanup();
        return rc;
    }
    asyflexa_problem P;
    std::memset(&P, 0, sizeof P);
    P.m = m;
    P.n = k;
    P.lda = ldS;
    P.a_dtype = a_dtype;
    P.x_dtype = a_dtype;
    P.A = AS;
    P.b = b0;
    P.lambda = 0.0;
    P.loss = ASYFLEXA_LOSS_LASSO;
    P.lin = lin;
    rc = asyflexa_create(&h, &P, &o, cuda_stream);
    if (rc) {
        const std::string why = asyflexa_last_error(nullptr);
        h = nullptr;
        cleanup();
        return afail(rc, "asyflexa_adjoint: support problem: " + why);
    }
    asyflexa_stats sst;
    std::memset(&sst, 0, sizeof sst);
    rc = asyflexa_solve(h, w, &sst);
    if (out_stats) *out_stats = sst;
    if (rc < 0) {
        const std::string why = asyflexa_last_error(h);
        cleanup();
        return afail(rc, "asyflexa_adjoint: support solve: " + why);
    }
    // dL/db = A_S w (the handle's exact residual at w, b = 0); dL/dlambda = -s^T w
    const int grc = asyflexa_get_residual(h, out_db);
    if (grc) {
        const std::string why = asyflexa_last_error(h);
        cleanup();
        return afail(grc, "asyflexa_adjoint: " + why);
    }
    if (f64)
        neg_signed_sum_kernel<double><<<1, kSelThreads, 0, st>>>(static_cast<const double*>(sgn),
                                                                 static_cast<const double*>(w), k, d_dlam);
    else
        neg_signed_sum_kernel<float><<<1, kSelThreads, 0, st>>>(static_cast<const float*>(sgn),
                                                                static_cast<const float*>(w), k, d_dlam);
    ACK(cudaGetLastError(), "signed sum");
    ACK(cudaMemcpyAsync(out_dlam, d_dlam, sizeof(double), cudaMemcpyDeviceToHost, st), "read dlambda");
    ACK(cudaStreamSynchronize(st), "synchronize");
#undef ACK
    cleanup();
    return rc;  // OK, or ENOTCONV when the support solve hit max_sweeps
}
