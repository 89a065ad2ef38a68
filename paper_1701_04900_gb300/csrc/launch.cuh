// Host-side launch code for one storage type of A.  Included by exactly one translation
// unit per type (inst_*.cu), which instantiates Launcher<TA>.
#pragma once

#include <type_traits>

#include "aux.cuh"
#include "handle.h"
#include "sweep.cuh"
#include "sweep_async.cuh"

namespace asyflexa {

// Register-increment async kernel instances: CPC = 16 KB stages per column (1..6).
template <typename TA, int CPC>
constexpr bool reg_fits() {
    return kRegKpc * CPC * ATraits<TA>::kVec <= kRegMaxRowsPerThread;
}

template <typename TA, bool EXACT>
const void* reg_kernel_inst(int cpc) {
    switch (cpc) {
        case 1:
            if constexpr (reg_fits<TA, 1>()) return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 1, false, EXACT>);
            break;
        case 2:
            if constexpr (reg_fits<TA, 2>()) return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 2, false, EXACT>);
            break;
        case 3:
            if constexpr (reg_fits<TA, 3>()) return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 3, false, EXACT>);
            break;
        case 4:
            if constexpr (reg_fits<TA, 4>()) return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 4, false, EXACT>);
            break;
        case 5:
            if constexpr (reg_fits<TA, 5>()) return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 5, false, EXACT>);
            break;
        case 6:
            if constexpr (reg_fits<TA, 6>()) return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 6, false, EXACT>);
            break;
        default: break;
    }
    return nullptr;
}

// The register-increment kernel instance for CPC stages per column; exact: the compensated
// gradient form (FP32 storage only; nullptr otherwise).
template <typename TA>
const void* reg_kernel(int cpc, bool exact = false) {
    if constexpr (sizeof(typename ATraits<TA>::TC) != 4) {
        return nullptr;  // FP64 problems use the staged kernel
    } else if constexpr (std::is_same<TA, float>::value) {
        return exact ? reg_kernel_inst<TA, true>(cpc) : reg_kernel_inst<TA, false>(cpc);
    } else {
        return exact ? nullptr : reg_kernel_inst<TA, false>(cpc);
    }
}

// Instances holding fewer units per thread than 2 per stage, for columns whose last stage is
// only partly filled: FP8 columns of up to 24576 rows (1536 units of 16 rows) span 2 stages
// but need 3 units per thread; BF16 columns of up to 20480 rows need 5 of the 6.  Returns the
// instance for cpc stages and at most `upt` units per thread (its unit count in *upt_out), or
// nullptr.
template <typename TA>
const void* reg_kernel_partial(int cpc, int upt, int* upt_out) {
    if constexpr (std::is_same<TA, __nv_fp8_e4m3>::value) {
        if (cpc == 2 && upt <= 3) {
            *upt_out = 3;
            return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 2, false, false, 3>);
        }
    }
    if constexpr (std::is_same<TA, __nv_bfloat16>::value) {
        if (cpc == 3 && upt <= 5) {
            *upt_out = 5;
            return reinterpret_cast<const void*>(sweep_async_reg_kernel<TA, 3, false, false, 5>);
        }
    }
    (void)cpc;
    (void)upt;
    (void)upt_out;
    return nullptr;
}

// The column-in-registers instance (sweep_async_rc_kernel) for cpc stages and upt units per
// thread, or nullptr.
template <typename TA, int CPC>
const void* rc_inst() {
    if constexpr (reg_fits<TA, CPC>())
        return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, CPC>);
    else
        return nullptr;
}

// Columns per barrier of the column-in-registers form by storage type: BF16 and FP8 columns
// are short in bytes but not in rows, so their per-column barrier, warp sums and residual reads
// are shared by 2 and 4 columns; FP32 keeps 1.
template <typename TA>
constexpr int rc_group() {
    if constexpr (std::is_same<TA, __nv_bfloat16>::value) return 2;
    if constexpr (std::is_same<TA, __nv_fp8_e4m3>::value) return 4;
    return 1;
}

// The instance of the column-in-registers form for cpc stages, upt units per thread and g
// columns per barrier (g = 1, or rc_group<TA>() and its half for the short-column types, at
// the column lengths the automatic choice gives them: more than 16384 rows), or nullptr.
template <typename TA>
const void* rc_kernel(int cpc, int upt, int g = 1) {
    if constexpr (sizeof(typename ATraits<TA>::TC) != 4) {
        return nullptr;
    } else {
        if (g != 1) {
            constexpr int G = rc_group<TA>();
            if constexpr (G >= 2) {
                if constexpr (std::is_same<TA, __nv_bfloat16>::value) {
                    if (g == 2 && cpc == 2 && upt == 4) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 2, 0, 2>);
                    if (g == 2 && cpc == 3 && upt == 6) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 3, 0, 2>);
                    if (g == 2 && cpc == 3 && upt == 5) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 3, 5, 2>);
                }
                if constexpr (std::is_same<TA, __nv_fp8_e4m3>::value) {
                    if (cpc == 2 && upt == 3) {
                        if (g == 4) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 2, 3, 4>);
                        if (g == 2) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 2, 3, 2>);
                    }
                }
            }
            return nullptr;
        }
        if (upt != kRegKpc * cpc) {
            if constexpr (std::is_same<TA, __nv_fp8_e4m3>::value)
                if (cpc == 2 && upt == 3) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 2, 3>);
            if constexpr (std::is_same<TA, __nv_bfloat16>::value)
                if (cpc == 3 && upt == 5) return reinterpret_cast<const void*>(sweep_async_rc_kernel<TA, 3, 5>);
            return nullptr;
        }
        switch (cpc) {
            case 1: return rc_inst<TA, 1>();
            case 2: return rc_inst<TA, 2>();
            case 3: return rc_inst<TA, 3>();
            case 4: return rc_inst<TA, 4>();
            case 5: return rc_inst<TA, 5>();
            case 6: return rc_inst<TA, 6>();
            default: return nullptr;
        }
    }
}

// Choose the register-increment kernel instance that covers the column (sets h.reg_*).
// Returns 0 if none applies (the staged kernel is used), 1 if chosen, or a negative
// cudaError_t if setting its shared-memory attribute failed.  The ring must hold one
// column plus at least one 16 KB stage of prefetch (more stages when they fit).
template <typename TA>
int Launcher<TA>::choose_reg(asyflexa_s& h) {
    h.reg_upt = h.reg_cpc = h.reg_stages = 0;
    h.reg_exact_ok = h.reg_rc_ok = false;
    h.reg_smem = 0;
    const int64_t units = h.mcopy / h.vec;
    const int cpc = static_cast<int>((units + kRegStageUnits - 1) / kRegStageUnits);
    if (cpc < 1 || cpc > 6) return 0;
    const int upt_needed = static_cast<int>((units + kRegConsThreads - 1) / kRegConsThreads);
    // the instance holding the fewest units per thread that covers the column
    int upt = kRegKpc * cpc;
    const void* fn = reg_kernel_partial<TA>(cpc, upt_needed, &upt);
    if (!fn) fn = reg_kernel<TA>(cpc);
    if (!fn) return 0;
    const int rt_rows = static_cast<int>(h.mcopy);
    const RegLayout L0 = make_reg_layout(rt_rows, 0);
    if (L0.total + 512 + static_cast<size_t>(cpc + 1) * L0.stage_bytes > h.smem_optin) return 0;
    int stages = static_cast<int>((h.smem_optin - L0.total - 512) / L0.stage_bytes);
    if (stages > 16) stages = 16;
    h.reg_upt = upt;
    h.reg_cpc = cpc;
    h.reg_stages = stages;
    h.reg_smem = make_reg_layout(rt_rows, stages).total;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(h.smem_optin));
    if (e != cudaSuccess) return -static_cast<int>(e);
    const void* fx = reg_kernel<TA>(cpc, true);
    h.reg_exact_ok = fx != nullptr;
    if (fx) {
        e = cudaFuncSetAttribute(fx, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(h.smem_optin));
        if (e != cudaSuccess) return -static_cast<int>(e);
    }
    // the column-in-registers form: the most columns per barrier whose stages fit the ring with
    // one column's stages to spare for the prefetch (and one refilling warp per stage)
    h.reg_g = 1;
    for (int g = rc_group<TA>(); g > 1; g /= 2) {
        if (g * cpc + cpc > stages || g * cpc > kRegConsWarps) continue;
        if (make_reg_layout(rt_rows, stages, g).total > h.smem_optin || !rc_kernel<TA>(cpc, upt, g)) continue;
        h.reg_g = g;
        break;
    }
    h.rc_smem = make_reg_layout(rt_rows, stages, h.reg_g).total;
    const void* fr = rc_kernel<TA>(cpc, upt, h.reg_g);
    h.reg_rc_ok = fr != nullptr;
    if (fr) {
        e = cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(h.smem_optin));
        if (e != cudaSuccess) return -static_cast<int>(e);
    }
    return 1;
}

// Geometry of the pipelined gather (refresh and Jacobi scatter): row tiles of
// kAuxThreads * kPipeElems rows, and as many list segments as fill the resident blocks of
// every SM once (at most 64).  Sets the kernels' shared-memory attribute.
template <typename TA>
int Launcher<TA>::setup_pipe(asyflexa_s& h) {
    using TX = typename XType<TA>::T;
    using TC = typename ATraits<TA>::TC;
    constexpr int U = kPipeElems / ATraits<TA>::kVec;
    h.pipe_smem = static_cast<size_t>(kPipeStages) * U * kAuxThreads * sizeof(uint4);
    const int64_t units = h.mcopy / h.vec;
    const int64_t per_cta = static_cast<int64_t>(kAuxThreads) * U;
    h.pipe_rowtiles = static_cast<int>((units + per_cta - 1) / per_cta);
    const void* fns[2] = {reinterpret_cast<const void*>(gather_gemv_pipe_kernel<TA, TX, true>),
                          reinterpret_cast<const void*>(gather_gemv_pipe_kernel<TA, TC, false>)};
    int bps = 64;
    for (const void* fn : fns) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(h.smem_optin));
        if (e != cudaSuccess) return static_cast<int>(e);
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kAuxThreads, h.pipe_smem);
        if (e != cudaSuccess) return static_cast<int>(e);
        bps = b < bps ? b : bps;
    }
    if (bps < 1) bps = 1;
    const int nseg = static_cast<int>((static_cast<int64_t>(bps) * h.sm_count) / h.pipe_rowtiles);
    h.pipe_nseg = nseg < 1 ? 1 : (nseg > 64 ? 64 : nseg);
    return 0;
}

// A kernel's shared-memory limit is an attribute of the kernel function, shared by every handle
// (and batch) in the process, while each launch asks for its own size (which alone sets the
// occupancy).  Every such attribute is therefore set to the device's opt-in maximum: set to one
// handle's size, it would be lowered by a handle created later for a smaller problem, and the
// first handle's launches would then fail.
template <typename TA>
int Launcher<TA>::set_smem_attrs(asyflexa_s& h) {
    cudaError_t e;
    e = cudaFuncSetAttribute(sweep_kernel<TA, kJacobi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(h.smem_optin));
    if (e != cudaSuccess) return static_cast<int>(e);
    e = cudaFuncSetAttribute(sweep_kernel<TA, kAsync>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(h.smem_optin));
    if (e != cudaSuccess) return static_cast<int>(e);
    if (h.check_use_smem && h.check_smem > 48 * 1024) {
        e = cudaFuncSetAttribute(check_kernel<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(h.smem_optin));
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    return 0;
}

template <typename TA>
cudaError_t Launcher<TA>::colnorm(asyflexa_s& h) {
    const auto& P = h.prob;
    const int grid = h.sm_count * 4;
    colnorm_kernel<TA><<<grid, kAuxThreads, 0, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, P.m, P.n, P.col_scale, loss_s(P), loss_c2(P), h.opts.tau,
        h.opts.tau_rel, h.dw, h.flag);
    ++h.launches;
    return cudaGetLastError();
}

template <typename TA>
cudaError_t Launcher<TA>::sweep(asyflexa_s& h, void* x, int mode, int sweeps) {
    const auto& P = h.prob;
    SweepParams p{};
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
    p.lin = P.lin;
    p.lam = loss_l1(P);
    p.dc = loss_dc(P);
    p.gamma = h.opts.gamma;
    p.s_loss = loss_s(P);
    p.c2 = loss_c2(P);
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
    p.delay_ns = mode == ASYFLEXA_ASYNC ? h.opts.delay_ns : 0;
    if (h.opts.gamma_mu > 0.0) {
        p.gtab = h.gtab;
        p.gtab_len = static_cast<long long>(sweeps) * h.nblocks;
        p.k_base = static_cast<unsigned long long>(h.sched_k);
    }
    if (mode == ASYFLEXA_ASYNC && h.reg_upt > 0) {
        p.stages = h.reg_stages;
        p.tile_rows = static_cast<int>(h.mcopy);
        void* args[] = {&p};
        const bool exact = h.reg_exact_ok && h.opts.exact_grad == 1;
        if (!exact && h.reg_rc_ok && !h.reg_rc_off) {  // the column-in-registers form
            const cudaError_t e = cudaLaunchKernel(rc_kernel<TA>(h.reg_cpc, h.reg_upt, h.reg_g), dim3(h.sweep_ctas),
                                                   dim3(kRcThreads), args, h.rc_smem, h.stream);
            ++h.launches;
            return e != cudaSuccess ? e : cudaGetLastError();
        }
        int upt_unused = 0;
        const void* fn = h.reg_upt == kRegKpc * h.reg_cpc ? reg_kernel<TA>(h.reg_cpc, exact)
                                                          : reg_kernel_partial<TA>(h.reg_cpc, h.reg_upt, &upt_unused);
        const cudaError_t e = cudaLaunchKernel(fn,
                                               dim3(h.sweep_ctas), dim3(kRegThreads), args,
                                               h.reg_smem, h.stream);
        ++h.launches;
        return e != cudaSuccess ? e : cudaGetLastError();
    }
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
    dim3 g(h.pipe_rowtiles, h.pipe_nseg);
    gather_gemv_pipe_kernel<TA, TC, false><<<g, kAuxThreads, h.pipe_smem, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, h.mcopy, P.col_scale, h.list_idx, static_cast<const TC*>(h.list_val),
        h.count, h.partial);
    const int rg = static_cast<int>((h.mcopy + kAuxThreads - 1) / kAuxThreads);
    reduce_partials_kernel<TC, TX><<<rg, kAuxThreads, 0, h.stream>>>(h.r, static_cast<const TC*>(h.partial),
                                                                      h.pipe_nseg, P.m, h.mcopy,
                                                                      static_cast<const TX*>(P.b), 0);
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
    dim3 g(h.pipe_rowtiles, h.pipe_nseg);
    gather_gemv_pipe_kernel<TA, TX, true><<<g, kAuxThreads, h.pipe_smem, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, h.mcopy, P.col_scale, h.list_idx, static_cast<const TX*>(h.list_val),
        h.count, h.partial);
    const int rg = static_cast<int>((h.mcopy + kAuxThreads - 1) / kAuxThreads);
    reduce_partials_kernel<double, TX><<<rg, kAuxThreads, 0, h.stream>>>(
        h.r, static_cast<const double*>(h.partial), h.pipe_nseg, P.m, h.mcopy, static_cast<const TX*>(P.b), 1);
    h.launches += 4;
    return cudaGetLastError();
}

template <typename TA>
cudaError_t Launcher<TA>::norms(asyflexa_s& h, const void* xv) {
    using TX = typename XType<TA>::T;
    norms_kernel<TX><<<kNormsGrid, kAuxThreads, 0, h.stream>>>(h.r, static_cast<const TX*>(h.prob.b), h.prob.m,
                                                                static_cast<const TX*>(xv), h.prob.n,
                                                                static_cast<const TX*>(h.prob.lin), loss_dc(h.prob),
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
    check_kernel<TA><<<h.check_ctas, kCheckThreads, h.check_use_smem ? h.check_smem : 0, h.stream>>>(
        static_cast<const TA*>(P.A), P.lda, P.m, P.n, P.col_scale, h.r, static_cast<const TX*>(xv),
        static_cast<const TX*>(P.lo), static_cast<const TX*>(P.hi), h.dw, static_cast<const TX*>(P.lin), loss_l1(P),
        loss_s(P), loss_c2(P), loss_dc(P), lasso_nobox, h.check_use_smem ? 1 : 0, h.meas);
    ++h.launches;
    return cudaGetLastError();
}

template <typename TA>
cudaError_t Launcher<TA>::shift_weights(asyflexa_s& h, double delta) {
    shift_weights_kernel<double><<<h.sm_count * 2, kAuxThreads, 0, h.stream>>>(h.dw, h.prob.n, delta);
    ++h.launches;
    return cudaGetLastError();
}

}  // namespace asyflexa

#define ASYFLEXA_INSTANTIATE(TA) template struct asyflexa::Launcher<TA>;
