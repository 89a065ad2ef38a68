// Host-side launch code for one storage type of A.  Included by exactly one translation
// unit per type (inst_*.cu), which instantiates Launcher<TA>.
#pragma once

#include "aux.cuh"
#include "handle.h"
#include "sweep.cuh"

namespace asyflexa {

template <typename TA>
int Launcher<TA>::set_smem_attrs(asyflexa_s& h) {
    cudaError_t e;
    e = cudaFuncSetAttribute(sweep_kernel<TA, kJacobi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(h.sweep_smem));
    if (e != cudaSuccess) return static_cast<int>(e);
    e = cudaFuncSetAttribute(sweep_kernel<TA, kAsync>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(h.sweep_smem));
    if (e != cudaSuccess) return static_cast<int>(e);
    if (h.check_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(check_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(h.check_smem));
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    return 0;
}

template <typename TA>
cudaError_t Launcher<TA>::colnorm(asyflexa_s& h) {
    const auto& P = h.prob;
    const bool lasso = P.loss == ASYFLEXA_LOSS_LASSO;
    const int grid = h.sm_count * 4;
    colnorm_kernel<TA><<<grid, kAuxThreads, 0, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, P.m, P.n, P.col_scale, lasso ? 1.0 : 2.0, lasso ? 0.0 : 2.0 * P.c,
        h.opts.tau, h.opts.tau_rel, h.dw, h.flag);
    ++h.launches;
    return cudaGetLastError();
}

template <typename TA>
cudaError_t Launcher<TA>::sweep(asyflexa_s& h, void* x, int mode, int sweeps) {
    const auto& P = h.prob;
    const bool lasso = P.loss == ASYFLEXA_LOSS_LASSO;
    SweepParams p;
    p.A = P.A;
    p.lda = P.lda;
    p.m = P.m;
    p.mcopy = h.mcopy;
    p.n = P.n;
    p.scale = P.col_scale;
    p.r = h.r;
    p.x = x;
    p.lo = P.lo;
    p.hi = P.hi;
    p.dw = h.dw;
    p.lam = P.lambda;
    p.gamma = h.opts.gamma;
    p.s_loss = lasso ? 1.0 : 2.0;
    p.c2 = lasso ? 0.0 : 2.0 * P.c;
    p.w = h.opts.block_w;
    p.nblocks = h.nblocks;
    p.sweeps = sweeps;
    p.tile_rows = h.tile_rows;
    p.ntiles = h.ntiles;
    p.chunk_rows = h.chunk_rows;
    p.stages = h.stages;
    p.delta = h.delta;
    p.counters = h.counters;
    p.hist = h.hist;
    p.err = h.err;
    if (mode == ASYFLEXA_ASYNC)
        sweep_kernel<TA, kAsync><<<h.sweep_ctas, kSweepThreads, h.sweep_smem, h.stream>>>(p);
    else
        sweep_kernel<TA, kJacobi><<<h.sweep_ctas, kSweepThreads, h.sweep_smem, h.stream>>>(p);
    ++h.launches;
    return cudaGetLastError();
}

// Deterministic r += A * delta over the nonzero entries of delta.
template <typename TA>
cudaError_t Launcher<TA>::jacobi_apply(asyflexa_s& h) {
    using TC = typename ATraits<TA>::TC;
    using TX = typename XType<TA>::T;
    static_assert(sizeof(TC) == sizeof(TX), "list values share the x buffer type");
    const auto& P = h.prob;
    const TC* d = static_cast<const TC*>(h.delta);
    count_nonzero_kernel<TC><<<h.compact_tiles, kAuxThreads, 0, h.stream>>>(d, P.n, h.tilecnt);
    compact_kernel<TC><<<h.compact_tiles, kAuxThreads, 0, h.stream>>>(d, P.n, h.tilecnt, h.compact_tiles, h.list_idx,
                                                                      static_cast<TC*>(h.list_val), h.count);
    dim3 g(h.gemv_rowtiles, h.nseg);
    gather_gemv_kernel<TA, TC, TC><<<g, kAuxThreads, 0, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, h.mcopy, P.col_scale, h.list_idx, static_cast<const TC*>(h.list_val),
        h.count, static_cast<TC*>(h.partial));
    const int rg = static_cast<int>((h.mcopy + kAuxThreads - 1) / kAuxThreads);
    reduce_partials_kernel<TC, TX><<<rg, kAuxThreads, 0, h.stream>>>(h.r, static_cast<const TC*>(h.partial), h.nseg,
                                                                      P.m, h.mcopy, static_cast<const TX*>(P.b), 0);
    h.launches += 4;
    return cudaGetLastError();
}

// r = A x - b with FP64 accumulation over the nonzero columns of x.
template <typename TA>
cudaError_t Launcher<TA>::refresh(asyflexa_s& h, const void* xv) {
    using TX = typename XType<TA>::T;
    const auto& P = h.prob;
    const TX* x = static_cast<const TX*>(xv);
    count_nonzero_kernel<TX><<<h.compact_tiles, kAuxThreads, 0, h.stream>>>(x, P.n, h.tilecnt);
    compact_kernel<TX><<<h.compact_tiles, kAuxThreads, 0, h.stream>>>(x, P.n, h.tilecnt, h.compact_tiles, h.list_idx,
                                                                      static_cast<TX*>(h.list_val), h.count);
    dim3 g(h.gemv_rowtiles, h.nseg);
    gather_gemv_kernel<TA, TX, double><<<g, kAuxThreads, 0, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, h.mcopy, P.col_scale, h.list_idx, static_cast<const TX*>(h.list_val),
        h.count, static_cast<double*>(h.partial));
    const int rg = static_cast<int>((h.mcopy + kAuxThreads - 1) / kAuxThreads);
    reduce_partials_kernel<double, TX><<<rg, kAuxThreads, 0, h.stream>>>(
        h.r, static_cast<const double*>(h.partial), h.nseg, P.m, h.mcopy, static_cast<const TX*>(P.b), 1);
    h.launches += 4;
    return cudaGetLastError();
}

template <typename TA>
cudaError_t Launcher<TA>::norms(asyflexa_s& h, const void* xv) {
    using TX = typename XType<TA>::T;
    norms_kernel<TX><<<kNormsGrid, kAuxThreads, 0, h.stream>>>(h.r, h.prob.m, static_cast<const TX*>(xv), h.prob.n,
                                                                h.norms_part);
    finalize_norms_kernel<double><<<1, 32, 0, h.stream>>>(h.norms_part, kNormsGrid, h.norms_out);
    h.launches += 2;
    return cudaGetLastError();
}

template <typename TA>
cudaError_t Launcher<TA>::check(asyflexa_s& h, const void* xv) {
    using TX = typename XType<TA>::T;
    const auto& P = h.prob;
    const bool lasso = P.loss == ASYFLEXA_LOSS_LASSO;
    const int lasso_nobox = lasso && P.lo == nullptr && P.hi == nullptr;
    check_kernel<TA><<<h.check_ctas, kAuxThreads, h.check_use_smem ? h.check_smem : 0, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, P.m, P.n, P.col_scale, h.r, static_cast<const TX*>(xv),
        static_cast<const TX*>(P.lo), static_cast<const TX*>(P.hi), h.dw, P.lambda, lasso ? 1.0 : 2.0,
        lasso ? 0.0 : 2.0 * P.c, lasso_nobox, h.check_use_smem ? 1 : 0, h.meas);
    ++h.launches;
    return cudaGetLastError();
}

}  // namespace asyflexa

#define ASYFLEXA_INSTANTIATE(TA) template struct asyflexa::Launcher<TA>;
