// Asynchronous sweep kernel with a register-resident block increment (FP32/BF16/FP8
// storage; m up to 24576 rows).
//
// Same method step as sweep.cuh (Algorithm 1, S.1-S.5; eq. 2 best response; Section 4
// surrogate), organised so that A is read from HBM exactly once per sweep even when many
// coordinates move (the generic kernel re-reads every moving column for its scatter):
//
//   * at the start of a block the consumers stage the FP64 residual, converted to FP32, in
//     shared memory (the stale read r~ of step S.2), together with the block's x_j, bounds,
//     column scales, 1/d_j and lam/d_j;
//   * every consumer thread owns the same 16-byte units u = k*512 + tid (k < 2*CPC) of
//     every column.  A column arrives in CPC ring stages of 1024 units (16 KB, 1-D bulk TMA
//     copies).  Consumers form a_j^T r~ from shared memory and publish per-warp partial
//     sums; after one barrier every consumer thread evaluates the closed-form best
//     response and fixed step for column j itself (identical FP32 arithmetic in every
//     thread, so they all agree; the surrogate is diagonal, so Delta_j only needs
//     a_j^T r~);
//   * while the column is still in shared memory every thread adds a_j * Delta_j to its
//     register copy of the block increment, then releases the column's stages;
//   * after the block's w columns the increment is added to r with one FP64 atomic per row
//     (lock-free).  All columns of the block used the same snapshot r~, so this is exactly
//     the block update r += A_i Delta_i.
//
// BATCHED = true runs many independent problems in one launch: the blocks of every problem
// form one global list (p.blk_inst / p.blk_local), each CTA owns the global blocks
// blockIdx.x, blockIdx.x + gridDim.x, ... (so each problem's blocks still have a single
// owner, Assumption D4), and each block reads its problem's matrix, residual, iterate and
// weights from the table p.batch.  Problems whose `active` flag is 0 are skipped (the flag is
// only changed between launches).
#pragma once

#include "convert.cuh"
#include "ptx.cuh"
#include "sweep.cuh"
#include "types.cuh"

namespace asyflexa {

constexpr int kRegConsWarps = 16;
constexpr int kRegConsThreads = kRegConsWarps * 32;
constexpr int kRegThreads = kRegConsThreads + 32;
constexpr int kRegKpc = 2;                                   // units per thread per stage
constexpr int kRegStageUnits = kRegKpc * kRegConsThreads;    // 1024 units = 16 KB
constexpr int kRegMaxRowsPerThread = 48;
constexpr int kRcGMax = 4;  // columns per barrier of the column-in-registers form

struct RegLayout {
    int stages;
    size_t stage_bytes;
    size_t off_ring, off_rt, off_colpart, off_coef, off_bars, off_misc, total;
};

// Per-column coefficients staged at the start of a block.
struct ColCoef {
    float x, lo, hi, dinv, thr, scale;  // x_j, bounds, 1/d_j (0 if d_j <= 0), lam/d_j, column scale
    float lin, pad0;                    // linear term of f (0 if none)
};

// g: columns whose partial sums one barrier publishes (1 for the other register kernels).
__host__ __device__ inline RegLayout make_reg_layout(int rt_rows, int stages, int g = 1) {
    RegLayout L;
    L.stages = stages;
    L.stage_bytes = static_cast<size_t>(kRegStageUnits) * 16;
    size_t o = 0;
    L.off_ring = o;
    o += L.stage_bytes * stages;
    L.off_rt = o;
    o = align_up_sz(o + static_cast<size_t>(rt_rows) * sizeof(float), 16);
    L.off_colpart = o;  // two buffers of per-warp partial sums (FP32 pairs in the compensated form,
                        // or the partials of g columns)
    o = align_up_sz(o + 2 * kRegConsWarps * (g > 2 ? g : 2) * sizeof(float), 16);
    L.off_coef = o;
    o = align_up_sz(o + kWMax * sizeof(ColCoef), 16);
    L.off_bars = o;
    o = align_up_sz(o + 2 * stages * sizeof(uint64_t), 16);
    L.off_misc = o;  // abort flag
    o += 16;
    L.total = align_up_sz(o, 128);
    return L;
}

// What one block update needs to know about its problem.
template <typename TA>
struct BlockView {
    using TX = typename XType<TA>::T;
    const TA* A;
    int64_t lda, m, mcopy, c0;
    double* r;
    TX* x;
    const TX* lo;
    const TX* hi;
    const TX* lin;
    const double* dw;
    const float* scale;
    double lam;
    float s_loss, c2;
    int wb;
    bool skip;
    DcTerm dc;
};

template <typename TA, bool BATCHED>
__device__ __forceinline__ BlockView<TA> block_view(const SweepParams& p, int b) {
    using TX = typename XType<TA>::T;
    BlockView<TA> v;
    if constexpr (BATCHED) {
        const int ii = p.blk_inst[b];
        if (ii < 0) {  // padding entry of the block list: nothing to do
            v.skip = true;
            return v;
        }
        const BatchInst& I = p.batch[ii];
        v.A = static_cast<const TA*>(I.A);
        v.lda = I.lda;
        v.m = I.m;
        v.mcopy = I.mcopy;
        v.c0 = static_cast<int64_t>(p.blk_local[b]) * I.w;
        v.wb = static_cast<int>(min64(I.w, I.n - v.c0));
        v.r = I.r;
        v.x = static_cast<TX*>(I.x);
        v.lo = static_cast<const TX*>(I.lo);
        v.hi = static_cast<const TX*>(I.hi);
        v.lin = static_cast<const TX*>(I.lin);
        v.dw = I.dw;
        v.scale = I.scale;
        v.lam = I.lam;
        v.s_loss = static_cast<float>(I.s_loss);
        v.c2 = static_cast<float>(I.c2);
        v.skip = I.active == 0;
        v.dc = DcTerm{0, 0.0, 0.0, 0.0};
    } else {
        v.A = static_cast<const TA*>(p.A);
        v.lda = p.lda;
        v.m = p.m;
        v.mcopy = p.mcopy;
        v.c0 = static_cast<int64_t>(b) * p.w;
        v.wb = static_cast<int>(min64(p.w, p.n - v.c0));
        v.r = p.r;
        v.x = static_cast<TX*>(p.x);
        v.lo = static_cast<const TX*>(p.lo);
        v.hi = static_cast<const TX*>(p.hi);
        v.lin = static_cast<const TX*>(p.lin);
        v.dw = p.dw;
        v.scale = p.scale;
        v.lam = p.lam;
        v.s_loss = static_cast<float>(p.s_loss);
        v.c2 = static_cast<float>(p.c2);
        v.skip = false;
        v.dc = p.dc;
    }
    return v;
}

// Compensated sum of the 16 warp partials (s, c) in a fixed pairwise order; every thread
// evaluates it and gets the same value.
__device__ __forceinline__ float sum_pairs_16(const float2* q) {
    float s[8], c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float e;
        two_sum(q[2 * i].x, q[2 * i + 1].x, s[i], e);
        c[i] = (q[2 * i].y + q[2 * i + 1].y) + e;
    }
#pragma unroll
    for (int w = 4; w >= 1; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; ++i) {
            float t, e;
            two_sum(s[2 * i], s[2 * i + 1], t, e);
            c[i] = (c[2 * i] + c[2 * i + 1]) + e;
            s[i] = t;
        }
    return s[0] + c[0];
}

// ---------------------------------------------------------------------------------------
// Pieces shared by the register-increment kernels (one block update, Algorithm 1).
// ---------------------------------------------------------------------------------------

// S.2 stale read: the FP64 residual rows [0, mcopy) rounded to FP32 into shared memory (rows
// >= m hold 0), kB independent 16-byte L2 loads in flight per thread.
template <int kThreads>
__device__ __forceinline__ void stage_residual(const double* r, int64_t mcopy, float* rt, int tid) {
    constexpr int kB = 8;
    const double2* rsrc = reinterpret_cast<const double2*>(r);
    float2* rdst = reinterpret_cast<float2*>(rt);
    const int pairs = static_cast<int>(mcopy / 2);
    for (int i0 = tid; i0 < pairs; i0 += kB * kThreads) {
        double2 v[kB];
#pragma unroll
        for (int t = 0; t < kB; ++t) {
            const int i = i0 + t * kThreads;
            v[t] = i < pairs ? __ldcg(rsrc + i) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int t = 0; t < kB; ++t) {
            const int i = i0 + t * kThreads;
            if (i < pairs) rdst[i] = make_float2(f64_to_f32(v[t].x), f64_to_f32(v[t].y));
        }
    }
}

// The per-column data of a block coordinate j = c0 + jl: loaded first (so that the loads
// overlap the residual reload), then turned into the epilogue's FP32 coefficients.
struct CoefLoads {
    double dw, x, lo, hi, lin;
    float scale;
};

template <typename TA>
__device__ __forceinline__ CoefLoads load_coef(const BlockView<TA>& bv, int jl) {
    const int64_t j = bv.c0 + jl;
    CoefLoads c;
    c.dw = bv.dw[j];
    c.x = static_cast<double>(bv.x[j]);
    c.lo = bv.lo ? static_cast<double>(bv.lo[j]) : -INFINITY;
    c.hi = bv.hi ? static_cast<double>(bv.hi[j]) : INFINITY;
    c.lin = bv.lin ? static_cast<double>(bv.lin[j]) : 0.0;
    c.scale = bv.scale ? bv.scale[j] : 1.f;
    return c;
}

template <typename TA>
__device__ __forceinline__ ColCoef finish_coef(const BlockView<TA>& bv, const CoefLoads& c) {
    ColCoef cf;
    cf.x = static_cast<float>(c.x);
    cf.lo = static_cast<float>(c.lo);
    cf.hi = static_cast<float>(c.hi);
    cf.dinv = c.dw > 0.0 ? static_cast<float>(1.0 / c.dw) : 0.f;
    cf.thr = c.dw > 0.0 ? static_cast<float>(bv.lam / c.dw) : 0.f;
    cf.scale = c.scale;
    // linear coefficient of the surrogate: lin_j, minus lam h-'(x_j) for the DC losses (the
    // concave part is linearised at the block's snapshot of x_j)
    double lj = c.lin;
    if (bv.dc.kind) lj -= bv.dc.lam * dc_hminus_grad(bv.dc, c.x);
    cf.lin = static_cast<float>(lj);
    cf.pad0 = 0.f;
    return cf;
}

// Sum of the 16 warp partials of g_j in a fixed order (every thread gets the same value).
__device__ __forceinline__ float sum_partials_16(const float* cp) {
    const float4* cp4 = reinterpret_cast<const float4*>(cp);
    const float4 q0 = cp4[0], q1 = cp4[1], q2 = cp4[2], q3 = cp4[3];
    return (((q0.x + q0.y) + (q0.z + q0.w)) + ((q1.x + q1.y) + (q1.z + q1.w))) +
           (((q2.x + q2.y) + (q2.z + q2.w)) + ((q3.x + q3.y) + (q3.z + q3.w)));
}

// Best response (eq. 2) and fixed step (S.4) of coordinate j from g_j = a_j^T r~, in FP32:
// returns the new x_j.
template <typename TA>
__device__ __forceinline__ float best_response_step(const BlockView<TA>& bv, const ColCoef& cf, float g,
                                                    float gamma) {
    const float grad = bv.s_loss * g * cf.scale - bv.c2 * cf.x + cf.lin;
    float xh = 0.f;
    if (cf.dinv > 0.f) {
        const float vv = fmaf(-grad, cf.dinv, cf.x);
        const float av = fabsf(vv) - cf.thr;
        xh = av > 0.f ? copysignf(av, vv) : 0.f;
    }
    xh = fminf(fmaxf(xh, cf.lo), cf.hi);
    return fmaf(gamma, xh - cf.x, cf.x);
}

// r += A_i Delta_i from the register increments: one FP64 atomic per row (skipping exact
// zeros).  The warp's units k*kThreads + 32*warp + l (l < 32) cover 32 V consecutive rows; a
// thread holds V consecutive ones.  Transposed through shuffles, so that in round q lane l
// adds row 32 q + l of that span (element l mod V of the unit held by lane q 32/V + l/V):
// every red instruction then covers 32 consecutive doubles (8 whole sectors) instead of 32
// rows 8 V bytes apart.
template <int V, int UPT, int kThreads>
__device__ __forceinline__ void scatter_increment(const float (&inc)[UPT][V], double* r, int64_t m, int warp,
                                                  int lane) {
    static_assert(32 % V == 0, "units of at most 32 rows");
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
        const int64_t row0 = (static_cast<int64_t>(k) * kThreads + warp * 32) * V;
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int src = q * (32 / V) + lane / V;
            const int esel = lane % V;
            float v = 0.f;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const float t = __shfl_sync(0xffffffffu, inc[k][e], src);
                v = e == esel ? t : v;
            }
            const int64_t row = row0 + q * 32 + lane;
            if (row < m && v != 0.f) red_add_f64(r + row, f32_to_f64(v));
        }
    }
    // A single CTA runs its blocks strictly in order (cyclic Gauss-Seidel), so its next read
    // of r must see this scatter.  With several CTAs the next read may miss it: that is one
    // more update in flight, within the bounded-delay model (Assumption D1), so no fence is
    // spent there.
    if (gridDim.x == 1) __threadfence();
}

// Block-end accounting (S.5, one thread): the global update counter, and the staleness of
// this update (updates completed between its read of r and its own completion) in a log2
// histogram.
__device__ __forceinline__ void account_block(const SweepParams& p, unsigned long long u_read, bool any,
                                              unsigned long long& my_updates, unsigned long long& my_active) {
    ++my_updates;
    if (any) ++my_active;
    const unsigned long long u1 = atomicAdd(&p.counters[0], 1ull);
    const unsigned long long dly = u1 - u_read;
    int bucket = 63 - __clzll(static_cast<long long>(dly + 1ull));
    bucket = bucket > 31 ? 31 : bucket;
    atomicAdd(&p.hist[bucket], 1ull);
}

// EXACT = true forms each block gradient g_j = a_j^T r~ with compensated arithmetic (Dot2 of
// Ogita, Rump and Oishi per accumulation chain, TwoSum in the warp and cross-warp sums), as
// accurate as FP64 accumulation of the FP32 snapshot r~; the plain form accumulates in FP32.
// At the 20000-row LASSO workload the compensated form lowers the level at which
// ||xhat(x) - x|| stops falling (the FP32 snapshot and staleness set the rest of it) and,
// above all, its sweep-to-sweep spikes, at about 1.6x the sweep time.
// UPTX > 0: this thread's units per column when fewer than the 2 per stage of CPC stages
// (the column's last stage only partly filled), so that fewer increment registers are held.
template <typename TA, int CPC, bool BATCHED = false, bool EXACT = false, int UPTX = 0>
__global__ void __launch_bounds__(kRegThreads, 1) sweep_async_reg_kernel(const SweepParams p) {
    using TC = typename ATraits<TA>::TC;
    static_assert(sizeof(TC) == 4, "register kernel computes in FP32");
    using TX = typename XType<TA>::T;
    static_assert(sizeof(TX) == 4, "register kernel updates FP32 x");
    constexpr int V = ATraits<TA>::kVec;
    constexpr int UPT = UPTX > 0 ? UPTX : kRegKpc * CPC;
    static_assert(UPT <= kRegKpc * CPC, "units beyond the column's stages");
    static_assert(UPT * V <= kRegMaxRowsPerThread, "too many rows per thread");

    extern __shared__ __align__(128) unsigned char smem[];
    const RegLayout L = make_reg_layout(p.tile_rows, p.stages);
    unsigned char* ring = smem + L.off_ring;
    float* rt = reinterpret_cast<float*>(smem + L.off_rt);
    float* colpart = reinterpret_cast<float*>(smem + L.off_colpart);
    ColCoef* coef = reinterpret_cast<ColCoef*>(smem + L.off_coef);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.off_bars);
    uint64_t* empty = full + p.stages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.off_misc);
    float* s_gamma = reinterpret_cast<float*>(smem + L.off_misc + 8);  // step of the current block

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int nblk = BATCHED ? p.total_blocks : p.nblocks;

    if (tid == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kRegConsWarps);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    // ------------------------------------------------------------------ producer
    if (warp == kRegConsWarps) {
        if (lane != 0) return;
        // A is streamed once per sweep (evict first) unless several batched problems share it
        const uint64_t pol = (BATCHED && p.keep_a_in_l2) ? l2_policy_evict_normal() : l2_policy_evict_first();
        uint32_t stage = 0, phase = 0;
        long long issued = 0;
        for (int s = 0; s < p.sweeps; ++s) {
            for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
                const BlockView<TA> bv = block_view<TA, BATCHED>(p, b);
                if (bv.skip) continue;
                const int64_t units = bv.mcopy / V;
                for (int jl = 0; jl < bv.wb; ++jl) {
                    const TA* col = bv.A + (bv.c0 + jl) * bv.lda;
                    for (int c = 0; c < CPC; ++c) {
                        const int64_t u0 = static_cast<int64_t>(c) * kRegStageUnits;
                        if (u0 >= units) break;
                        const uint32_t nbytes = static_cast<uint32_t>(min64(kRegStageUnits, units - u0) * 16);
                        if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, p.err)) goto drain;
                        mbar_arrive_expect_tx(&full[stage], nbytes);
                        bulk_load(ring + stage * L.stage_bytes, col + u0 * V, nbytes, &full[stage], pol);
                        ++issued;
                        if (++stage == static_cast<uint32_t>(p.stages)) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
        }
        return;
    drain: {
        const long long first = issued > p.stages ? issued - p.stages : 0;
        for (long long i = first; i < issued; ++i) {
            const uint32_t st = static_cast<uint32_t>(i % p.stages);
            const uint32_t ph = static_cast<uint32_t>((i / p.stages) & 1);
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(&full[st], ph)) {
                if (global_timer_ns() - t0 > kWaitLimitNs) break;
            }
        }
    }
        return;
    }

    // ------------------------------------------------------------------ consumers
    uint32_t stage = 0, phase = 0;
    unsigned long long u_read = 0, my_updates = 0, my_active = 0;

    float inc[UPT][V];
    int buf = 0;

    for (int s = 0; s < p.sweeps; ++s) {
        for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
            const BlockView<TA> bv = block_view<TA, BATCHED>(p, b);
            if (bv.skip) continue;  // uniform across the CTA and the producer
            const int64_t units = bv.mcopy / V;
            const int64_t units_full = bv.m / V;  // units whose rows are all < m
            int nchunks = 0;                      // stages per column actually present
            for (int c = 0; c < CPC; ++c)
                if (static_cast<int64_t>(c) * kRegStageUnits < units) ++nchunks;
            // S.2: stale read of the residual into shared memory, and the block's per-column
            // coefficients (the barrier that ended the previous block guarantees nobody still
            // reads rt or coef).  The coefficient loads go out before the residual reload, and
            // the last consumer thread reads the update counter, so that neither latency waits
            // behind the other.
            CoefLoads cl{};
            if (tid < bv.wb) cl = load_coef(bv, tid);
            if (tid == kRegConsThreads - 1) {
                u_read = ld_relaxed_u64(&p.counters[0]);
                // step of this block update (the update index is the number of updates
                // completed before this read of the residual)
                *s_gamma = static_cast<float>(launch_step(p, static_cast<long long>(u_read - p.k_base)));
            }
            stage_residual<kRegConsThreads>(bv.r, bv.mcopy, rt, tid);
            if (tid < bv.wb) coef[tid] = finish_coef(bv, cl);
#pragma unroll
            for (int k = 0; k < UPT; ++k)
#pragma unroll
                for (int e = 0; e < V; ++e) inc[k][e] = 0.f;
            bool any = false;
            named_bar_sync(1, kRegConsThreads);
            const float gamma = *s_gamma;

            for (int jl = 0; jl < bv.wb; ++jl) {
                // ---- dot a_j^T r~ over this thread's rows
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
                DFAcc dacc0, dacc1, dacc2, dacc3;  // compensated chains (EXACT)
                uint32_t st_c = stage, ph_c = phase;
                bool ok = !*abort_flag;
#pragma unroll 1
                for (int c = 0; c < CPC; ++c) {
                    if (c < nchunks) {
                        if (ok) ok = mbar_wait_bounded(&full[st_c], ph_c, abort_flag, p.err);
                        // a stage whose units all hold rows < m (every stage but a column's last
                        // when m is not a multiple of the stage rows) needs no per-unit checks
                        const bool whole = static_cast<int64_t>(c + 1) * kRegStageUnits <= units_full;
                        if (ok && whole && !EXACT) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + st_c * L.stage_bytes);
#pragma unroll
                            for (int kk = 0; kk < kRegKpc; ++kk) {
                                const int64_t u = static_cast<int64_t>(c * kRegKpc + kk) * kRegConsThreads + tid;
                                float a[V];
                                ATraits<TA>::unpack(src[kk * kRegConsThreads + tid], a);
                                const float* rv = rt + u * V;
#pragma unroll
                                for (int e = 0; e < V; e += 4) {
                                    const float4 r4 = *reinterpret_cast<const float4*>(rv + e);
                                    acc0 = fmaf(a[e], r4.x, acc0);
                                    acc1 = fmaf(a[e + 1], r4.y, acc1);
                                    acc2 = fmaf(a[e + 2], r4.z, acc2);
                                    acc3 = fmaf(a[e + 3], r4.w, acc3);
                                }
                            }
                        } else if (ok) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + st_c * L.stage_bytes);
#pragma unroll
                            for (int kk = 0; kk < kRegKpc; ++kk) {
                                const int64_t u = static_cast<int64_t>(c * kRegKpc + kk) * kRegConsThreads + tid;
                                if (u < units) {
                                    float a[V];
                                    ATraits<TA>::unpack(src[kk * kRegConsThreads + tid], a);
                                    const float* rv = rt + u * V;
                                    if (u < units_full) {
#pragma unroll
                                        for (int e = 0; e < V; e += 4) {
                                            const float4 r4 = *reinterpret_cast<const float4*>(rv + e);
                                            if constexpr (EXACT) {
                                                dacc0.add_prod(a[e], r4.x);
                                                dacc1.add_prod(a[e + 1], r4.y);
                                                dacc2.add_prod(a[e + 2], r4.z);
                                                dacc3.add_prod(a[e + 3], r4.w);
                                            } else {
                                                acc0 = fmaf(a[e], r4.x, acc0);
                                                acc1 = fmaf(a[e + 1], r4.y, acc1);
                                                acc2 = fmaf(a[e + 2], r4.z, acc2);
                                                acc3 = fmaf(a[e + 3], r4.w, acc3);
                                            }
                                        }
                                    } else {
                                        const int valid = static_cast<int>(bv.m - u * V);
#pragma unroll
                                        for (int e = 0; e < V; ++e) {
                                            if (e < valid) {
                                                if constexpr (EXACT)
                                                    dacc0.add_prod(a[e], rv[e]);
                                                else
                                                    acc0 = fmaf(a[e], rv[e], acc0);
                                            }
                                        }
                                    }
                                }
                            }
                        }
                        if (++st_c == static_cast<uint32_t>(p.stages)) {
                            st_c = 0;
                            ph_c ^= 1u;
                        }
                    }
                }
                static_assert(kRegConsWarps == 16, "the sums below read 16 warp partials");
                float* cp = colpart + buf * kRegConsWarps * (EXACT ? 2 : 1);
                if constexpr (EXACT) {
                    float ts, tc;
                    {
                        float t1, e1, t2, e2, e;
                        two_sum(dacc0.s, dacc1.s, t1, e1);
                        two_sum(dacc2.s, dacc3.s, t2, e2);
                        two_sum(t1, t2, ts, e);
                        tc = ((dacc0.c + dacc1.c) + (dacc2.c + dacc3.c)) + ((e1 + e2) + e);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {  // both lanes of a pair form the same exact sum
                        const float so = __shfl_xor_sync(0xffffffffu, ts, o);
                        const float co = __shfl_xor_sync(0xffffffffu, tc, o);
                        float t, e;
                        two_sum(ts, so, t, e);
                        tc = (tc + co) + e;
                        ts = t;
                    }
                    if (lane == 0) reinterpret_cast<float2*>(cp)[warp] = make_float2(ts, tc);
                } else {
                    const float v = warp_sum((acc0 + acc1) + (acc2 + acc3));
                    if (lane == 0) cp[warp] = v;
                }
                const ColCoef cf = coef[jl];  // written before the block's first barrier
                named_bar_sync(1, kRegConsThreads);
                // ---- best response (eq. 2) + fixed step (S.4): every consumer thread sums the 16
                // warp partials in the same fixed order, so all agree on g and Delta_j
                float g;
                if constexpr (EXACT)
                    g = sum_pairs_16(reinterpret_cast<const float2*>(cp));
                else
                    g = sum_partials_16(cp);
                buf ^= 1;
                const float xn = best_response_step(bv, cf, g, gamma);
                const float dlt = xn - cf.x;
                float dj = 0.f;
                if (!*abort_flag) {
                    if (tid == 0) bv.x[bv.c0 + jl] = static_cast<TX>(xn);
                    dj = dlt * cf.scale;
                    any |= dlt != 0.f;
                }
                // ---- fold a_j * Delta_j into the register increment, then release the stages
                st_c = stage;
                ph_c = phase;
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    if (c < nchunks) {
                        if (dj != 0.f) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + st_c * L.stage_bytes);
                            if (static_cast<int64_t>(c + 1) * kRegStageUnits <= units) {  // every unit present
#pragma unroll
                                for (int kk = 0; kk < kRegKpc; ++kk) {
                                    const int k = c * kRegKpc + kk;
                                    if (k < UPT) {  // compile-time: units k >= UPT lie past the column
                                        float a[V];
                                        ATraits<TA>::unpack(src[kk * kRegConsThreads + tid], a);
#pragma unroll
                                        for (int e = 0; e < V; ++e) inc[k][e] = fmaf(a[e], dj, inc[k][e]);
                                    }
                                }
                            } else {
#pragma unroll
                                for (int kk = 0; kk < kRegKpc; ++kk) {
                                    const int k = c * kRegKpc + kk;
                                    const int64_t u = static_cast<int64_t>(k) * kRegConsThreads + tid;
                                    if (k < UPT && u < units) {
                                        float a[V];
                                        ATraits<TA>::unpack(src[kk * kRegConsThreads + tid], a);
#pragma unroll
                                        for (int e = 0; e < V; ++e) inc[k][e] = fmaf(a[e], dj, inc[k][e]);
                                    }
                                }
                            }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[st_c]);
                        if (++st_c == static_cast<uint32_t>(p.stages)) {
                            st_c = 0;
                            ph_c ^= 1u;
                        }
                    }
                }
                stage = st_c;
                phase = ph_c;
            }
            // ---- r += A_i Delta_i : one FP64 atomic per row (skipping exact zeros)
            // (the abort flag is read once per warp: the FP32 path below shuffles within the warp)
            const bool aborted = __shfl_sync(0xffffffffu, *abort_flag != 0, 0);
            if (!BATCHED && p.delay_ns > 0 && (blockIdx.x & 1u)) __nanosleep(static_cast<unsigned>(p.delay_ns));
            if (any && !aborted) scatter_increment<V, UPT, kRegConsThreads>(inc, bv.r, bv.m, warp, lane);
            named_bar_sync(1, kRegConsThreads);  // scatter issued; rt and coef free
            if (tid == kRegConsThreads - 1) account_block(p, u_read, any, my_updates, my_active);
        }
    }
    if (tid == kRegConsThreads - 1) {
        atomicAdd(&p.counters[1], my_updates);
        atomicAdd(&p.counters[2], my_active);
    }
}


// ---------------------------------------------------------------------------------------
// Column-in-registers form of the same kernel (one problem, plain FP32 accumulation).
//
// 16 warps and no producer warp: with 16 warps (4 per SM sub-partition) a thread may hold 128
// registers instead of 96, which is room for its units of the current column next to its
// block increment.  Each thread keeps the units it read for a_j^T r~ in registers and forms
// the increment a_j * Delta_j from them, so a column is read from shared memory once instead
// of twice.
//
// The ring is refilled at the column barrier.  The stages of the CTA's columns form one
// sequence (sweep, owned block, column, stage), and item k lives in slot k mod S.  Every warp
// has read all stages of column j before it arrives at the column's barrier, so right after
// that barrier warp c (c < nchunks) refills the slot of the column's stage c with the item S
// further on: no release barriers or waits, one copy per warp.  Column j + 1's items are then
// issued before its gradient pass starts (nchunks <= S), so no wait forms a cycle.
// ---------------------------------------------------------------------------------------

constexpr int kRcThreads = kRegConsThreads;

// Position of a ring item in the CTA's sequence: sweep, owned block, column in the block,
// stage in the column.
struct RcPos {
    int s, b, jl, c;
};

// Advances q by `steps` items (stages per column: nchunks); false past the CTA's last item.
__device__ __forceinline__ bool rc_next(RcPos& q, int steps, const SweepParams& p, int nchunks) {
    q.c += steps;
    while (q.c >= nchunks) {
        q.c -= nchunks;
        const int wb = static_cast<int>(min64(p.w, p.n - static_cast<int64_t>(q.b) * p.w));
        if (++q.jl >= wb) {
            q.jl = 0;
            q.b += gridDim.x;
            if (q.b >= p.nblocks) {
                q.b = blockIdx.x;
                if (++q.s >= p.sweeps) return false;
            }
        }
    }
    return true;
}

// Issues the bulk copy of item q into ring slot st (one thread); fills[st] counts the copies
// ever issued into the slot, for the drain at exit.
template <typename TA>
__device__ __forceinline__ void rc_issue(const SweepParams& p, const RcPos& q, int st, unsigned char* ring,
                                         size_t stage_bytes, uint64_t* full, uint32_t* fills, int64_t units) {
    constexpr int V = ATraits<TA>::kVec;
    const int64_t u0 = static_cast<int64_t>(q.c) * kRegStageUnits;
    const uint32_t nbytes = static_cast<uint32_t>(min64(kRegStageUnits, units - u0) * 16);
    const TA* col = static_cast<const TA*>(p.A) + (static_cast<int64_t>(q.b) * p.w + q.jl) * p.lda;
    fills[st] += 1u;
    fence_proxy_async_smem();  // the slot's earlier generic reads before the copy's async writes
    mbar_arrive_expect_tx(&full[st], nbytes);
    bulk_load(ring + st * stage_bytes, col + u0 * V, nbytes, &full[st], l2_policy_evict_first());
}

template <typename TA, int CPC, int UPTX = 0, int G = 1>
__global__ void __launch_bounds__(kRcThreads, 1) sweep_async_rc_kernel(const SweepParams p) {
    using TC = typename ATraits<TA>::TC;
    static_assert(sizeof(TC) == 4, "register kernel computes in FP32");
    using TX = typename XType<TA>::T;
    static_assert(sizeof(TX) == 4, "register kernel updates FP32 x");
    constexpr int V = ATraits<TA>::kVec;
    constexpr int UPT = UPTX > 0 ? UPTX : kRegKpc * CPC;
    static_assert(UPT <= kRegKpc * CPC, "units beyond the column's stages");
    static_assert(UPT * V <= kRegMaxRowsPerThread, "too many rows per thread");
    static_assert(G >= 1 && G <= kRcGMax, "columns per barrier");

    extern __shared__ __align__(128) unsigned char smem[];
    const RegLayout L = make_reg_layout(p.tile_rows, p.stages, G);
    unsigned char* ring = smem + L.off_ring;
    float* rt = reinterpret_cast<float*>(smem + L.off_rt);
    float* colpart = reinterpret_cast<float*>(smem + L.off_colpart);
    ColCoef* coef = reinterpret_cast<ColCoef*>(smem + L.off_coef);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.off_bars);
    uint32_t* fills = reinterpret_cast<uint32_t*>(full + p.stages);  // in the layout's second barrier array
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.off_misc);
    float* s_gamma = reinterpret_cast<float*>(smem + L.off_misc + 8);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int S = p.stages;
    const int64_t units = p.mcopy / V;
    const int64_t units_full = p.m / V;  // units whose rows are all < m
    int nchunks = 0;                     // stages per column
    for (int c = 0; c < CPC; ++c)
        if (static_cast<int64_t>(c) * kRegStageUnits < units) ++nchunks;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            fills[s] = 0u;
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0 && static_cast<int>(blockIdx.x) < p.nblocks && p.sweeps > 0) {
        RcPos q{0, static_cast<int>(blockIdx.x), 0, 0};
        for (int i = 0; i < S; ++i) {
            rc_issue<TA>(p, q, i, ring, L.stage_bytes, full, fills, units);
            if (!rc_next(q, 1, p, nchunks)) break;
        }
    }

    uint32_t stage = 0, phase = 0;
    unsigned long long u_read = 0, my_updates = 0, my_active = 0;
    float inc[UPT][V];
    int buf = 0;

    for (int s = 0; s < p.sweeps; ++s) {
        for (int b = blockIdx.x; b < p.nblocks; b += gridDim.x) {
            const BlockView<TA> bv = block_view<TA, false>(p, b);
            // S.2: stale read of the residual into shared memory, and the block's per-column
            // coefficients (the barrier that ended the previous block guarantees nobody still
            // reads rt or coef).  The coefficient loads go out before the residual reload, and
            // the last thread reads the update counter, so that neither latency waits behind
            // the other.
            CoefLoads cl{};
            if (tid < bv.wb) cl = load_coef(bv, tid);
            if (tid == kRcThreads - 1) {
                u_read = ld_relaxed_u64(&p.counters[0]);
                *s_gamma = static_cast<float>(launch_step(p, static_cast<long long>(u_read - p.k_base)));
            }
            stage_residual<kRcThreads>(bv.r, bv.mcopy, rt, tid);
            if (tid < bv.wb) coef[tid] = finish_coef(bv, cl);
#pragma unroll
            for (int k = 0; k < UPT; ++k)
#pragma unroll
                for (int e = 0; e < V; ++e) inc[k][e] = 0.f;
            bool any = false;
            named_bar_sync(1, kRcThreads);
            const float gamma = *s_gamma;

            // groups of G columns (the block's last group may be shorter): their stages are
            // consecutive ring items, so G * nchunks <= S slots hold a whole group; each
            // thread reads its residual units once per group for all G dots, and one barrier
            // publishes the group's G partial sums
            for (int j0 = 0; j0 < bv.wb; j0 += G) {
                const int gn = G == 1 ? 1 : (bv.wb - j0 < G ? bv.wb - j0 : G);
                // ---- dots a_j^T r~ over this thread's rows; the units stay in registers
                constexpr int NACC = G == 1 ? 4 : 2;  // independent FMA chains per column
                float acc[G][NACC];
                uint4 colr[G][UPT];
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int q = 0; q < NACC; ++q) acc[g][q] = 0.f;
                bool ok = !*abort_flag;
                const uint32_t st0 = stage, ph0 = phase;  // slot and parity of the group's first stage
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    if (c < nchunks) {
                        const uint4* src[G];
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            src[g] = nullptr;
                            if (g < gn) {
                                uint32_t sl = st0 + static_cast<uint32_t>(g * nchunks + c), ph = ph0;
                                if (sl >= static_cast<uint32_t>(S)) {
                                    sl -= static_cast<uint32_t>(S);
                                    ph ^= 1u;
                                }
                                if (ok) ok = mbar_wait_bounded(&full[sl], ph, abort_flag, p.err);
                                src[g] = reinterpret_cast<const uint4*>(ring + sl * L.stage_bytes);
                            }
                        }
                        const bool whole = static_cast<int64_t>(c + 1) * kRegStageUnits <= units_full;
#pragma unroll
                        for (int kk = 0; kk < kRegKpc; ++kk) {
                            const int k = c * kRegKpc + kk;
                            if (k < UPT) {
                                const int64_t u = static_cast<int64_t>(k) * kRcThreads + tid;
                                const float* rv = rt + u * V;
                                const bool full_unit = whole || u < units_full;
                                float r[V];
                                if (full_unit) {
#pragma unroll
                                    for (int e = 0; e < V; e += 4) {
                                        const float4 r4 = *reinterpret_cast<const float4*>(rv + e);
                                        r[e] = r4.x;
                                        r[e + 1] = r4.y;
                                        r[e + 2] = r4.z;
                                        r[e + 3] = r4.w;
                                    }
                                } else {
                                    const int valid = u < units ? static_cast<int>(bv.m - u * V) : 0;
#pragma unroll
                                    for (int e = 0; e < V; ++e) r[e] = e < valid ? rv[e] : 0.f;
                                }
#pragma unroll
                                for (int g = 0; g < G; ++g) {
                                    colr[g][k] = (g < gn && ok && (whole || u < units)) ? src[g][kk * kRcThreads + tid]
                                                                                       : make_uint4(0u, 0u, 0u, 0u);
                                    float a[V];
                                    ATraits<TA>::unpack(colr[g][k], a);
#pragma unroll
                                    for (int e = 0; e < V; ++e) acc[g][e % NACC] = fmaf(a[e], r[e], acc[g][e % NACC]);
                                }
                            }
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < kRegKpc; ++kk)
#pragma unroll
                            for (int g = 0; g < G; ++g)
                                if (c * kRegKpc + kk < UPT) colr[g][c * kRegKpc + kk] = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
                {
                    uint32_t nx = st0 + static_cast<uint32_t>(gn * nchunks);
                    phase = ph0;
                    if (nx >= static_cast<uint32_t>(S)) {
                        nx -= static_cast<uint32_t>(S);
                        phase ^= 1u;
                    }
                    stage = nx;
                }
                static_assert(kRegConsWarps == 16, "the sums below read 16 warp partials");
                float* cp = colpart + buf * (kRegConsWarps * G);
                {
                    float v[G];
#pragma unroll
                    for (int g = 0; g < G; ++g)
                        v[g] = NACC == 4 ? (acc[g][0] + acc[g][1]) + (acc[g][NACC - 2] + acc[g][NACC - 1])
                                         : acc[g][0] + acc[g][1];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int g = 0; g < G; ++g) v[g] += __shfl_xor_sync(0xffffffffu, v[g], o);
                    if (lane == 0) {
#pragma unroll
                        for (int g = 0; g < G; ++g)
                            if (g < gn) cp[g * kRegConsWarps + warp] = v[g];
                    }
                }
                ColCoef cf[G];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (g < gn) cf[g] = coef[j0 + g];
                named_bar_sync(1, kRcThreads);
                // every warp has read the group's stages: warp c refills the slot of the group's
                // stage c with the item S further on
                if (warp < gn * nchunks && lane == 0 && !*abort_flag) {
                    RcPos q{s, b, j0, 0};
                    if (rc_next(q, S + warp, p, nchunks)) {
                        uint32_t st = st0 + static_cast<uint32_t>(warp);
                        if (st >= static_cast<uint32_t>(S)) st -= static_cast<uint32_t>(S);
                        rc_issue<TA>(p, q, static_cast<int>(st), ring, L.stage_bytes, full, fills, units);
                    }
                }
                // ---- best responses (eq. 2) + fixed step (S.4), identical in every thread
                float dj[G];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    dj[g] = 0.f;
                    if (g < gn) {
                        const float gs = sum_partials_16(cp + g * kRegConsWarps);
                        const float xn = best_response_step(bv, cf[g], gs, gamma);
                        const float dlt = xn - cf[g].x;
                        if (!*abort_flag) {
                            if (tid == 0) bv.x[bv.c0 + j0 + g] = static_cast<TX>(xn);
                            dj[g] = dlt * cf[g].scale;
                            any |= dlt != 0.f;
                        }
                    }
                }
                buf ^= 1;
                // ---- fold a_j * Delta_j into the register increment (units past the column
                // hold zeros)
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (dj[g] != 0.f) {
#pragma unroll
                        for (int k = 0; k < UPT; ++k) {
                            float a[V];
                            ATraits<TA>::unpack(colr[g][k], a);
#pragma unroll
                            for (int e = 0; e < V; ++e) inc[k][e] = fmaf(a[e], dj[g], inc[k][e]);
                        }
                    }
                }
            }
            // ---- r += A_i Delta_i
            const bool aborted = __shfl_sync(0xffffffffu, *abort_flag != 0, 0);
            if (p.delay_ns > 0 && (blockIdx.x & 1u)) __nanosleep(static_cast<unsigned>(p.delay_ns));
            if (any && !aborted) scatter_increment<V, UPT, kRcThreads>(inc, bv.r, bv.m, warp, lane);
            named_bar_sync(1, kRcThreads);  // scatter issued; rt and coef free
            if (tid == kRcThreads - 1) account_block(p, u_read, any, my_updates, my_active);
        }
    }
    // no bulk copy may still be writing shared memory when the CTA exits (only after an
    // abort can an issued item be left unconsumed): wait for the last copy into every slot
    if (tid == kRcThreads - 1) {
        atomicAdd(&p.counters[1], my_updates);
        atomicAdd(&p.counters[2], my_active);
    }
    __syncthreads();
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            const uint32_t f = fills[st];
            if (f == 0u) continue;
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(&full[st], (f - 1u) & 1u)) {
                if (global_timer_ns() - t0 > kWaitLimitNs) break;
            }
        }
    }
}

}  // namespace asyflexa
