// Batched Gauss-Seidel form: many independent FP32 problems solved in ONE persistent launch,
// one CTA per problem at a time.
//
// A CTA takes the next problem from a queue (problems ordered by decreasing size, so that
// the largest start first) and runs Algorithm 1 on it with a single owner for every block:
// with one CTA there are no updates in flight, so the iteration is exact cyclic block
// Gauss-Seidel (blocks of w <= 4 consecutive columns with the separable surrogate; w = 1 is
// the paper's scalar blocks, Section 4.1) with the fixed step of S.4 and the best response of
// eq. 2.  The CTA then runs its own stopping test (exact residual, F, gap, and the Section 4.3
// merit ||xhat(x) - x||_inf / max(1, ||x||_inf)) and goes on with the next problem, so the
// whole batch needs no host round trip.
//
//   * The residual r = A x - b lives in registers for the whole solve: consumer thread t
//     owns the 16-byte units u = k * T + t (k < UPT, 4 rows each) of every column, and holds
//     r for those rows as an unevaluated FP32 pair (hi, lo) so that small late increments
//     are not lost to FP32 rounding.  Because a thread reads and updates only its own rows,
//     the update r += A_i Delta_i needs no barrier before the next block's gradients.
//   * A producer warp streams the blocks HBM -> SMEM, one 1-D bulk (TMA) copy per block (its
//     columns are contiguous: stride lda), into a ring of S slots (full / empty mbarriers).
//     A bulk copy costs the SM about the same time whatever its size up to tens of KB, so
//     short columns are fetched several per copy.  The consumers load the block's
//     coefficients (x_j and the FP32 d_j, 1/d_j staged at create) themselves, while they
//     form the block's gradients.
//   * A named barrier per block publishes the per-warp partial sums of a_j^T r for the block's
//     columns; lane t of warp 0 then evaluates the FP32 best response of column t (gs_delta)
//     and writes x_j, a second barrier publishes the steps, and every consumer thread folds
//     a_j Delta_j into its rows, re-reading the block from its slot.
//   * Near the tolerance every gradient a_j^T r is a Dot2 sum (error-free products and sums) over
//     r's (hi, lo) pair and every update is error-free; before that the sweeps use plain FP32
//     FMAs (an exact refresh follows every sweep phase).
//   * Phases of one solve: REFRESH (r = -b + sum over x_j != 0 of a_j x_j with error-free
//     products and sums -- plain FP32 products while the gap is above kGsFarGap -- then F with
//     FP64 sums), SWEEP (k sweeps, k = check_every, 2 near the tolerance, kGsFarChecks
//     check_every far from the gap), MERIT (x^_j with unit step, the largest |x^_j - x_j|).  A problem stops
//     when its gap (if f_star is known) and its merit meet the tolerances (OK), when F is not
//     finite (ENONFINITE), at max_sweeps, or when, with the gap met and the merit within 100
//     tol_stat, five checks in a row do not lower the best merit by 10% (ENOTCONV: the
//     stationarity floor of the FP32 iterate).
#pragma once

#include <cmath>
#include <type_traits>

#include "ptx.cuh"
#include "sweep.cuh"
#include "types.cuh"

namespace asyflexa {

// One problem of the batched Gauss-Seidel launch (device table entry).
struct GsInst {
    const float* A;
    int64_t lda, m, n;
    float* x;
    const float* b;
    const float* lo;
    const float* hi;
    const float* lin;
    const float2* dd;           // (d_j, 1/d_j) in FP32; (0, 0) where d_j <= 0
    double lam, s_loss, c2, c;  // s_loss = 1 (LASSO) or 2 (NCQUAD); c2 = 2c; c: NCQUAD weight (for F)
    double f_star;              // NaN: no gap test, stop on the merit alone
    int loss, wpick;            // wpick: this problem's block width (0: the launch's)
    // written by the kernel
    double F, stat, xmax;
    long long sweeps, nnz;
    int status, checks, w_used, pad1;  // w_used: the block width (the tuned one, or as many as a slot holds)
    long long ns;                      // the problem's solve time on its CTA (global timer)
};

struct GsParams {
    GsInst* inst;
    const int* order;   // problems in the order the queue hands them out
    int count;
    int* queue;         // next position in `order` (0 before the launch)
    double gamma, tol_gap, tol_stat;
    int check_every, max_sweeps, stages;
    int w;              // block width, 1 .. kGsWMax, of the problems with wpick = 0
    int64_t slot_bytes; // ring slot (a multiple of 128 bytes, at least the longest column)
    int sweeps_only;    // 1: exactly max_sweeps sweeps per problem, no stopping test (autotuner)
    int handoff_sweeps; // > 0: a problem still short of its tolerances after this many sweeps stops
                        // with kGsHandoff (the host finishes it with a second launch)
    int keep_a_in_l2;   // 1: A shared by the problems (normal L2 priority)
    int* err;
};

constexpr int kGsMeta = 64;  // REFRESH item ring (a power of 2, >= the ring depth)
constexpr int kGsWMax = 8;   // largest block width of the Gauss-Seidel form

struct GsLayout {
    size_t slot_bytes, off_ring, off_meta, off_part, off_red, off_dls, off_bars, off_misc, total;
};

__host__ __device__ inline GsLayout make_gs_layout(int nw, size_t slot_bytes, int stages) {
    GsLayout L;
    L.slot_bytes = slot_bytes;
    size_t o = 0;
    L.off_ring = o;
    o += L.slot_bytes * stages;
    L.off_meta = o;  // first column of each REFRESH item (-1: end of the phase)
    o += sizeof(int) * kGsMeta;
    L.off_part = o;  // two buffers of per-warp (s, c) partial pairs for up to kGsWMax columns
    o += 2 * static_cast<size_t>(kGsWMax) * nw * 2 * sizeof(float);
    o = (o + 15) / 16 * 16;
    L.off_red = o;   // per-warp FP64 sums of the objective pieces
    o += static_cast<size_t>(nw) * 8 * sizeof(double);
    L.off_dls = o;   // the steps x_new - x of the current block's columns
    o += kGsWMax * sizeof(float);
    o = (o + 15) / 16 * 16;
    L.off_bars = o;
    o += 2 * static_cast<size_t>(stages) * sizeof(uint64_t);
    L.off_misc = o;  // abort flag, queue position, decision values
    o += 128;
    L.total = (o + 127) / 128 * 128;
    return L;
}

constexpr int kGsRefresh = 0, kGsSweep = 1, kGsMerit = 2;
constexpr double kGsFarGap = 1e-2;  // a relative gap above this is far from any tolerance
constexpr int kGsFarChecks = 4;     // check intervals between checks while far
constexpr int kGsHandoff = 2;  // status: left for the second launch (not an asyflexa_status)
constexpr int kGsFloorChecks = 5;
constexpr double kGsFloorBand = 100.0;  // the floor rule applies within 100 tol_stat

// Shared decision values (written by thread 0 before a CTA barrier, read by every thread).
struct GsMisc {
    int abort, qi, nonfinite, pad;
    double F, xmax, merit;
    long long nnz;
    // the solve's control state, kept and decided by thread 0
    long long sweeps;
    double stat_ref;  // best merit so far
    float stat_last;
    int phase, k_sweeps, status, checks, exact, flat, flat_plain, done, reset;
    int plain_refresh;  // the next refresh may use plain FP32 products (far from the gap)
    double gap_last;    // the relative gap at the last refresh (NaN: not known)
};
static_assert(sizeof(GsMisc) <= 128, "the layout reserves 128 bytes for the control state");

// The coefficients of column j that the best response needs (bounds and linear term apart).
struct GsCoef {
    float x, d, dinv;
};

// x^_j - x_j for the best response of eq. 2 (soft-threshold, then clip), in FP32, from the
// gradient pair (gh, gl) of a_j^T r.  With q = d x - grad the soft-threshold step is
//     q > lam:  -(grad + lam) / d,    q < -lam:  -(grad - lam) / d,    else:  -x,
// and near a stationary point grad + lam (or grad - lam) cancels: formed as (gh + lam) + gl it
// is exact up to the last rounding (Sterbenz), where x - grad/d loses the digits of a small
// difference of two numbers as large as lam / d.
__device__ __forceinline__ float gs_delta(const GsCoef& c, float lo, float hi, float lin, float lam, float gh, float gl,
                                         float s_loss, float c2) {
    // grad = s_loss * g - c2 x + lin as a pair (s_loss is 1 or 2: exact)
    float th, tl;
    two_sum(s_loss * gh, fmaf(-c2, c.x, lin), th, tl);
    tl += s_loss * gl;
    float e;
    if (c.dinv > 0.f) {
        const float q = fmaf(c.x, c.d, -th) - tl;
        if (q > lam)
            e = -((th + lam) + tl) * c.dinv;
        else if (q < -lam)
            e = -((th - lam) + tl) * c.dinv;
        else
            e = -c.x;
    } else {
        e = -c.x;  // d_j = 0: x^_j = clip(0)
    }
    // the box, if active; otherwise e itself (not x + e rounded to FP32 and minus x, which
    // would hide a step below half an ulp of x from the stopping test)
    const float xe = c.x + e;
    if (xe < lo) return lo - c.x;
    if (xe > hi) return hi - c.x;
    return e;
}

// (hi, lo) += a * v with TwoProduct (FMA) and TwoSum: exact up to the rounding of lo.
__device__ __forceinline__ void ff_add_prod(float& hi, float& lo, float a, float v) {
    const float p = a * v;
    const float ep = fmaf(a, v, -p);
    const float s = hi + p;
    const float z = s - hi;
    const float es = (hi - (s - z)) + (p - z);
    lo += es + ep;
    hi = s;
}

// NW consumer warps and one producer warp: NW = 7 (two CTAs per SM) or 15 (one) keeps 16 warps
// on an SM, 4 per sub-partition, so that a thread may hold up to 128 registers.
template <int NW, int UPT>
__global__ void __launch_bounds__((NW + 1) * 32, NW < 8 ? 2 : 1) batch_gs_kernel(const GsParams p) {
    constexpr int T = NW * 32;  // consumer threads
    extern __shared__ __align__(128) unsigned char smem[];
    const GsLayout L = make_gs_layout(NW, static_cast<size_t>(p.slot_bytes), p.stages);
    unsigned char* ring = smem + L.off_ring;
    int* meta = reinterpret_cast<int*>(smem + L.off_meta);
    float2* part = reinterpret_cast<float2*>(smem + L.off_part);
    double* red = reinterpret_cast<double*>(smem + L.off_red);
    float* dls = reinterpret_cast<float*>(smem + L.off_dls);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.off_bars);
    uint64_t* empty = full + p.stages;
    GsMisc* misc = reinterpret_cast<GsMisc*>(smem + L.off_misc);
    volatile int* abort_flag = &misc->abort;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const bool producer = warp == NW;
    const int S = p.stages;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        misc->abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const uint64_t pol = p.keep_a_in_l2 ? l2_policy_evict_normal() : l2_policy_evict_first();
    long long it = 0;   // ring items issued (producer) / consumed (consumers); identical sequences
    int pslot = 0, cslot = 0;        // slot of item `it` (it mod S), producer / consumer side
    uint32_t ppar = 0u, cpar = 0u;   // parity of that slot's use by item `it`
    int buf = 0;        // partial-sum buffer of the next block
    bool ok = true;     // this thread's waits all completed

    float rhi[UPT][4], rlo[UPT][4];

    for (;;) {
        if (tid == 0) misc->qi = atomicAdd(p.queue, 1);
        __syncthreads();
        const int qi = misc->qi;
        if (qi >= p.count || *abort_flag) break;
        const int ii = p.order[qi];
        const GsInst& I = p.inst[ii];
        const float* A = I.A;
        float* X = I.x;
        const float2* DD = I.dd;
        const float *LO = I.lo, *HI = I.hi, *LIN = I.lin;
        const int lda = static_cast<int>(I.lda), m = static_cast<int>(I.m), n = static_cast<int>(I.n);
        const int units = (m + 3) / 4;
        const float s_loss = static_cast<float>(I.s_loss), c2 = static_cast<float>(I.c2);
        const float lam = static_cast<float>(I.lam);
        const float gamma = static_cast<float>(p.gamma);
        // columns per block: the tuned width, as many as a slot holds
        const int wcap = static_cast<int>((p.slot_bytes - static_cast<int64_t>(units) * 16) /
                                          (static_cast<int64_t>(lda) * 4)) + 1;
        const int wsel = I.wpick > 0 ? I.wpick : p.w;
        const int w = wsel < wcap ? wsel : wcap;
        // this thread's units k < kmine hold rows of the column; unit klast (or -1) is the
        // column's last one, of which only its first vlast rows are < m
        const int kmine = tid < units ? (units - 1 - tid) / T + 1 : 0;
        const int klast = ((units - 1) % T == tid) ? (units - 1) / T : -1;
        const int vlast = m - 4 * (units - 1);

        auto reset_r = [&]() {
#pragma unroll
            for (int k = 0; k < UPT; ++k) {
                const int u = k * T + tid;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = u * 4 + e;
                    rhi[k][e] = row < m ? -I.b[row] : 0.f;
                    rlo[k][e] = 0.f;
                }
            }
        };
        if (!producer) reset_r();

        const uint64_t t_start = global_timer_ns();
        if (tid == 0) {
            misc->sweeps = 0;
            misc->status = ASYFLEXA_ENOTCONV;
            misc->checks = 0;
            misc->phase = kGsRefresh;
            misc->k_sweeps = 0;
            misc->stat_last = NAN;
            // stationarity floor: with the gap met and the merit within kGsFloorBand tol_stat,
            // kGsFloorChecks checks in a row that do not lower the best merit by 10% end the
            // solve (ENOTCONV): the FP32 iterate has stopped moving
            misc->stat_ref = INFINITY;
            misc->flat = 0;
            // the sweeps' arithmetic: plain FP32 until the solve is near its tolerance (the gap
            // test passed with a known f_star; without one, a merit within kGsFloorBand tol_stat,
            // or two checks in a row that did not lower the best merit by 10%), exact from then on
            misc->exact = 0;
            misc->plain_refresh = 0;
            misc->gap_last = NAN;
            misc->flat_plain = 0;
            misc->done = 0;
            misc->reset = 0;
        }
        __syncthreads();
        for (;;) {
            const int phase = misc->phase, k_sweeps = misc->k_sweeps;
            const bool exact = misc->exact != 0;
            const bool plain = misc->plain_refresh != 0 && !exact;
            // ================================================================ one phase
            if (producer) {
                // ---- issue the phase's items into the ring (lane 0), in consumption order.
                // Item `it` goes to slot `pslot` (= it mod S), whose previous use (item it - S) had
                // parity ppar ^ 1.
                auto wait_slot = [&]() -> bool {  // item it - S consumed: its slot is free
                    if (it < S) return true;
                    return mbar_wait_bounded(&empty[pslot], ppar ^ 1u, abort_flag, p.err);
                };
                auto issue = [&](int j0, int wb) {  // lane 0, after wait_slot: columns j0 .. j0 + wb - 1
                    if (wb > 0) {
                        const uint32_t bytes = static_cast<uint32_t>(
                            static_cast<int64_t>(wb - 1) * lda * 4 + static_cast<int64_t>(units) * 16);
                        mbar_arrive_expect_tx(&full[pslot], bytes);
                        bulk_load(ring + pslot * L.slot_bytes, A + static_cast<int64_t>(j0) * lda, bytes, &full[pslot],
                                  pol);
                    } else {
                        mbar_arrive(&full[pslot]);
                    }
                    ++it;
                    if (++pslot == S) {
                        pslot = 0;
                        ppar ^= 1u;
                    }
                };
                bool go = true;
                if (phase == kGsRefresh) {
                    // the blocks of up to w columns that hold a nonzero x_j, found 32 columns at a
                    // time by the whole warp; no block crosses a group of 32 (w need not divide
                    // 32).  meta[item] = (the block's first column) * 16 + its width
                    for (int j0 = 0; j0 < n && go; j0 += 32) {
                        const int j = j0 + lane;
                        const bool nz = j < n && X[j] != 0.f;
                        const unsigned mask = __ballot_sync(0xffffffffu, nz);
                        for (int b0 = 0; b0 < 32 && j0 + b0 < n && go; b0 += w) {
                            int wb = 32 - b0 < w ? 32 - b0 : w;
                            if (n - (j0 + b0) < wb) wb = n - (j0 + b0);
                            const unsigned bm = (mask >> b0) & ((1u << wb) - 1u);
                            if (bm == 0u) continue;
                            int okl = 1;
                            if (lane == 0) {
                                okl = wait_slot() ? 1 : 0;
                                if (okl) {
                                    meta[it & (kGsMeta - 1)] = (j0 + b0) * 16 + wb;
                                    issue(j0 + b0, wb);
                                }
                            }
                            go = __shfl_sync(0xffffffffu, okl, 0) != 0;
                        }
                    }
                    if (lane == 0 && go && wait_slot()) {
                        meta[it & (kGsMeta - 1)] = -1;
                        issue(0, 0);
                    }
                } else if (lane == 0) {
                    const int nsw = phase == kGsSweep ? k_sweeps : 1;
                    for (int sw = 0; sw < nsw && go; ++sw)
                        for (int j0 = 0; j0 < n; j0 += w) {
                            if (!wait_slot()) {
                                go = false;
                                break;
                            }
                            issue(j0, n - j0 < w ? n - j0 : w);
                        }
                }
                it = __shfl_sync(0xffffffffu, it, 0);
                pslot = __shfl_sync(0xffffffffu, pslot, 0);
                ppar = __shfl_sync(0xffffffffu, ppar, 0);
            } else if (phase == kGsRefresh) {
                // ---- r += a_j x_j over the nonzero columns (no barrier: every thread reads and
                // writes only its own rows)
                for (;;) {
                    const int slot = cslot;
                    ok = ok && !*abort_flag && mbar_wait_bounded(&full[slot], cpar, abort_flag, p.err);
                    if (!ok) break;
                    const int code = meta[it & (kGsMeta - 1)];
                    const int j0 = code >> 4;  // -1: the end of the refresh
                    if (code >= 0) {
                        const int wb = code & 15;
                        for (int t = 0; t < wb; ++t) {
                            const float xj = X[j0 + t];
                            if (xj == 0.f) continue;
                            if (plain) {
                                // far from the gap: plain FP32 products (the next refresh that
                                // could pass the gap test is exact)
                                const uint4* srcp = reinterpret_cast<const uint4*>(ring + slot * L.slot_bytes +
                                                                                   static_cast<size_t>(t) * lda * 4);
#pragma unroll
                                for (int k = 0; k < UPT; ++k) {
                                    if (k < kmine) {
                                        float a[4];
                                        ATraits<float>::unpack(srcp[k * T + tid], a);
                                        const int nv = k == klast ? vlast : 4;
#pragma unroll
                                        for (int e = 0; e < 4; ++e)
                                            if (e < nv) rhi[k][e] = fmaf(a[e], xj, rhi[k][e]);
                                    }
                                }
                                continue;
                            }
                            const uint4* src = reinterpret_cast<const uint4*>(ring + slot * L.slot_bytes +
                                                                              static_cast<size_t>(t) * lda * 4);
#pragma unroll
                            for (int k = 0; k < UPT; ++k) {
                                if (k < kmine) {
                                    float a[4];
                                    ATraits<float>::unpack(src[k * T + tid], a);
                                    const int nv = k == klast ? vlast : 4;
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (e < nv) ff_add_prod(rhi[k][e], rlo[k][e], a[e], xj);
                                }
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[slot]);
                    ++it;
                    if (++cslot == S) {
                        cslot = 0;
                        cpar ^= 1u;
                    }
                    if (j0 < 0) break;
                }
            } else {
                // ---- SWEEP (k sweeps of cyclic block updates) or MERIT (one pass, no update).
                // A block is wb <= w consecutive columns of a sweep (the last block of a sweep may
                // be shorter), fetched by one copy into one slot; its columns share the residual
                // r of the block's start (the separable surrogate of the block update), so their
                // dots and reductions overlap and one barrier publishes all wb partial sums.  The
                // update pass then re-reads the block from its slot, released at the block end.
                const bool merit = phase == kGsMerit;
                const bool ex = merit || exact;
                const int nsw = merit ? 1 : k_sweeps;
                float mmax = 0.f;
                bool bad = false;
                // a column unit into registers, the rows past m of the last unit zeroed
                auto load_unit = [&](const uint4* src, int k) -> uint4 {
                    uint4 v = (ok && k < kmine) ? src[k * T + tid] : make_uint4(0u, 0u, 0u, 0u);
                    if (k == klast) {
                        if (vlast < 4) v.w = 0u;
                        if (vlast < 3) v.z = 0u;
                        if (vlast < 2) v.y = 0u;
                    }
                    return v;
                };
                // Lane t of warp 0 owns the block's column t: it sums the column's warp partials,
                // evaluates its best response and writes x_j, so column j (always at position
                // j mod w of its block) is read and written by one thread.  Its coefficients are
                // loaded one block ahead (x_j was last written by this thread a sweep earlier, or,
                // when a sweep is a single block, in the block just done: then the new value).
                float cx = 0.f, cd = 0.f, cdi = 0.f;  // this block's column
                float nx = 0.f, nd = 0.f, ndi = 0.f;  // the next block's
                if (warp == 0 && lane < w && lane < n) {
                    const float2 dd = DD[lane];
                    nx = X[lane];
                    nd = dd.x;
                    ndi = dd.y;
                }
                for (int sw = 0; sw < nsw; ++sw) {
                    for (int j0 = 0; j0 < n; j0 += w) {
                        const int wb = n - j0 < w ? n - j0 : w;
                        const int slot = cslot;
                        const int jn = j0 + w < n ? j0 + w : 0;  // the next block (of this or the next sweep)
                        if (warp == 0) {
                            cx = nx;
                            cd = nd;
                            cdi = ndi;
                            if (lane < w && jn + lane < n) {
                                const float2 dd = DD[jn + lane];
                                nx = X[jn + lane];
                                nd = dd.x;
                                ndi = dd.y;
                            }
                        }
                        ok = ok && !*abort_flag && mbar_wait_bounded(&full[slot], cpar, abort_flag, p.err);
                        float2* cp = part + buf * (kGsWMax * NW);
                        // a_j^T r.  Exact arithmetic (the merit pass, and the sweeps once the solve
                        // is near its tolerance): Dot2 products on r's (hi, lo) pair -- a plain FP32
                        // dot of length m errs by about sqrt(m) eps ||a_j|| ||r||, which divided by
                        // d_j = ||a_j||^2 puts the plain iteration's fixed point up to 1e-5 away from
                        // stationarity.  Earlier sweeps use plain FP32 FMAs on r_hi (the columns of a
                        // block interleaved); the exact refresh after every sweep phase removes their
                        // drift.
                        if (ex) {
#pragma unroll 1
                            for (int t = 0; t < wb; ++t) {
                                const uint4* src = reinterpret_cast<const uint4*>(ring + slot * L.slot_bytes +
                                                                                  static_cast<size_t>(t) * lda * 4);
                                DFAcc dacc0, dacc1;
                                float lo_acc = 0.f;
#pragma unroll
                                for (int k = 0; k < UPT; ++k) {
                                    float a[4];
                                    ATraits<float>::unpack(load_unit(src, k), a);
                                    dacc0.add_prod(a[0], rhi[k][0]);
                                    dacc1.add_prod(a[1], rhi[k][1]);
                                    dacc0.add_prod(a[2], rhi[k][2]);
                                    dacc1.add_prod(a[3], rhi[k][3]);
#pragma unroll
                                    for (int e = 0; e < 4; ++e) lo_acc = fmaf(a[e], rlo[k][e], lo_acc);
                                }
                                float ts, tc;
                                two_sum(dacc0.s, dacc1.s, ts, tc);
                                tc += (dacc0.c + dacc1.c) + lo_acc;
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) {
                                    const float so = __shfl_xor_sync(0xffffffffu, ts, o);
                                    const float co = __shfl_xor_sync(0xffffffffu, tc, o);
                                    float tt, e;
                                    two_sum(ts, so, tt, e);
                                    tc = (tc + co) + e;
                                    ts = tt;
                                }
                                if (lane == 0) cp[t * NW + warp] = make_float2(ts, tc);
                            }
                        } else if (w == 1) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + slot * L.slot_bytes);
                            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll
                            for (int k = 0; k < UPT; ++k) {
                                float a[4];
                                ATraits<float>::unpack(load_unit(src, k), a);
                                acc0 = fmaf(a[0], rhi[k][0], acc0);
                                acc1 = fmaf(a[1], rhi[k][1], acc1);
                                acc2 = fmaf(a[2], rhi[k][2], acc2);
                                acc3 = fmaf(a[3], rhi[k][3], acc3);
                            }
                            const float v = warp_sum((acc0 + acc1) + (acc2 + acc3));
                            if (lane == 0) cp[warp] = make_float2(v, 0.f);
                        } else {
                            // WB >= w columns without branches, so that their load, FMA and
                            // shuffle chains interleave: a column past the block's end reads the
                            // block's first column and its result is not used
                            auto dots = [&](auto wbc) {
                                constexpr int WB = decltype(wbc)::value;
                                float acc[WB];
#pragma unroll
                                for (int t = 0; t < WB; ++t) {
                                    const uint4* src = reinterpret_cast<const uint4*>(
                                        ring + slot * L.slot_bytes + static_cast<size_t>(t < wb ? t : 0) * lda * 4);
                                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                                    for (int k = 0; k < UPT; ++k) {
                                        float a[4];
                                        ATraits<float>::unpack(load_unit(src, k), a);
                                        a0 = fmaf(a[0], rhi[k][0], a0);
                                        a1 = fmaf(a[1], rhi[k][1], a1);
                                        a0 = fmaf(a[2], rhi[k][2], a0);
                                        a1 = fmaf(a[3], rhi[k][3], a1);
                                    }
                                    acc[t] = a0 + a1;
                                }
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                                    for (int t = 0; t < WB; ++t) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
                                if (lane == 0) {
#pragma unroll
                                    for (int t = 0; t < WB; ++t) cp[t * NW + warp] = make_float2(acc[t], 0.f);
                                }
                            };
                            if (w <= 2)
                                dots(std::integral_constant<int, 2>{});
                            else if (w <= 4)
                                dots(std::integral_constant<int, 4>{});
                            else
                                dots(std::integral_constant<int, 8>{});
                        }
                        named_bar_sync(1, T);
                        if (warp == 0) {
                            if (lane < wb) {
                                // the column's partials in a fixed order: g = gh + gl
                                const float2* c2p = cp + lane * NW;
                                float gh, gl;
                                if (ex) {
                                    float sh = c2p[0].x, cc = c2p[0].y;
#pragma unroll
                                    for (int w2 = 1; w2 < NW; ++w2) {
                                        float tt, e;
                                        two_sum(sh, c2p[w2].x, tt, e);
                                        cc = (cc + c2p[w2].y) + e;
                                        sh = tt;
                                    }
                                    two_sum(sh, cc, gh, gl);
                                } else {
                                    float sh = 0.f;
#pragma unroll
                                    for (int w2 = 0; w2 < NW; ++w2) sh += c2p[w2].x;
                                    gh = sh;
                                    gl = 0.f;
                                }
                                const int j = j0 + lane;
                                const GsCoef c{cx, cd, cdi};
                                const float e = gs_delta(c, LO ? LO[j] : -INFINITY, HI ? HI[j] : INFINITY,
                                                         LIN ? LIN[j] : 0.f, lam, gh, gl, s_loss, c2);
                                if (merit) {
                                    // |x^_j - x_j| (unit step): the Section 4.3 merit
                                    mmax = fmaxf(mmax, fabsf(e));
                                    bad |= !(fabsf(gh) <= 3.0e38f);  // NaN or infinite gradient
                                } else {
                                    const float xn = fmaf(gamma, e, cx);
                                    if (ok) X[j] = xn;
                                    if (jn == j0) nx = xn;  // the sweep is this one block
                                    dls[lane] = ok ? xn - cx : 0.f;
                                }
                            } else if (lane < kGsWMax && !merit) {
                                dls[lane] = 0.f;  // no column at this position
                            }
                        }
                        buf ^= 1;
                        if (!merit) {
                            named_bar_sync(1, T);  // the block's steps are in dls
                            // the block's increment r += A_i Delta_i, each thread on its own rows,
                            // the columns read again from the slot
                            if (ex) {
#pragma unroll 1
                                for (int t = 0; t < wb; ++t) {
                                    const float dl = dls[t];
                                    if (dl != 0.f) {
                                        const uint4* src = reinterpret_cast<const uint4*>(
                                            ring + slot * L.slot_bytes + static_cast<size_t>(t) * lda * 4);
#pragma unroll
                                        for (int k = 0; k < UPT; ++k) {
                                            float a[4];
                                            ATraits<float>::unpack(load_unit(src, k), a);
#pragma unroll
                                            for (int e = 0; e < 4; ++e) ff_add_prod(rhi[k][e], rlo[k][e], a[e], dl);
                                        }
                                    }
                                }
                            } else {
                                // dls[t] = 0 for t >= wb (and for columns that did not move); the
                                // columns past the block's end read the block's first column
                                auto update = [&](auto wbc) {
                                    constexpr int WB = decltype(wbc)::value;
                                    float dl[WB];
                                    bool any = false;
#pragma unroll
                                    for (int t = 0; t < WB; ++t) {
                                        dl[t] = dls[t];
                                        any |= dl[t] != 0.f;
                                    }
                                    if (any) {
#pragma unroll
                                        for (int k = 0; k < UPT; ++k) {
#pragma unroll
                                            for (int t = 0; t < WB; ++t) {
                                                const uint4* src = reinterpret_cast<const uint4*>(
                                                    ring + slot * L.slot_bytes +
                                                    static_cast<size_t>(t < wb ? t : 0) * lda * 4);
                                                float a[4];
                                                ATraits<float>::unpack(load_unit(src, k), a);
#pragma unroll
                                                for (int e = 0; e < 4; ++e) rhi[k][e] = fmaf(a[e], dl[t], rhi[k][e]);
                                            }
                                        }
                                    }
                                };
                                if (w <= 2)
                                    update(std::integral_constant<int, 2>{});
                                else if (w <= 4)
                                    update(std::integral_constant<int, 4>{});
                                else
                                    update(std::integral_constant<int, 8>{});
                            }
                        }
                        __syncwarp();
                        if (lane == 0 && ok) mbar_arrive(&empty[slot]);
                        ++it;
                        if (++cslot == S) {
                            cslot = 0;
                            cpar ^= 1u;
                        }
                    }
                }
                if (merit && warp == 0) {
                    // the largest merit over warp 0's lanes
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        mmax = fmaxf(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
                        bad |= __shfl_xor_sync(0xffffffffu, bad ? 1 : 0, o) != 0;
                    }
                }
                if (merit && tid == 0) {
                    misc->merit = bad ? NAN : static_cast<double>(mmax);
                }
            }
            __syncthreads();  // phase done: x and the ring are quiescent

            // ================================================================ after the phase
            if (phase == kGsRefresh && !producer) {
                // F(x) from the exact residual: FP64 sums in a fixed order, one quantity at a
                // time (few registers live beside the residual)
                auto warp_put = [&](double v, int q) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) red[warp * 8 + q] = v;
                };
                {
                    double rr = 0.0;
#pragma unroll
                    for (int k = 0; k < UPT; ++k)
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const double v = static_cast<double>(rhi[k][e]) + static_cast<double>(rlo[k][e]);
                            rr += v * v;
                        }
                    warp_put(rr, 0);
                }
                {
                    double ax = 0.0, x2 = 0.0;
                    for (int j = tid; j < n; j += T) {
                        const double xj = static_cast<double>(X[j]);
                        ax += fabs(xj);
                        x2 += xj * xj;
                    }
                    warp_put(ax, 1);
                    warp_put(x2, 2);
                }
                {
                    double lx = 0.0;
                    if (LIN)
                        for (int j = tid; j < n; j += T) lx += static_cast<double>(LIN[j]) * static_cast<double>(X[j]);
                    warp_put(lx, 3);
                }
                {
                    int nz = 0;
                    float xm = 0.f;
                    for (int j = tid; j < n; j += T) {
                        const float xj = X[j];
                        nz += xj != 0.f ? 1 : 0;
                        xm = fmaxf(xm, fabsf(xj));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        nz += __shfl_xor_sync(0xffffffffu, nz, o);
                        xm = fmaxf(xm, __shfl_xor_sync(0xffffffffu, xm, o));
                    }
                    if (lane == 0) {
                        red[warp * 8 + 4] = static_cast<double>(nz);
                        red[warp * 8 + 5] = static_cast<double>(xm);
                    }
                }
                named_bar_sync(1, T);
                if (tid == 0) {
                    double sm[6] = {0, 0, 0, 0, 0, 0};
                    for (int w2 = 0; w2 < NW; ++w2) {
                        for (int q = 0; q < 5; ++q) sm[q] += red[w2 * 8 + q];
                        sm[5] = fmax(sm[5], red[w2 * 8 + 5]);
                    }
                    const double F = (I.loss == ASYFLEXA_LOSS_LASSO ? 0.5 * sm[0] : sm[0] - I.c * sm[2]) + sm[3] +
                                     I.lam * sm[1];
                    misc->F = F;
                    misc->nnz = static_cast<long long>(sm[4]);
                    misc->xmax = sm[5];
                    misc->nonfinite = isfinite(F) ? 0 : 1;
                }
            }
            __syncthreads();

            // ================================================================ next phase
            // (decided by thread 0 from the shared values; every thread follows after a barrier)
            if (tid == 0) {
                GsMisc& g = *misc;
                g.reset = 0;
                bool sweep_next = false;
                if (*abort_flag) {
                    g.done = 1;
                } else if (phase == kGsRefresh) {
                    const double fs = I.f_star;
                    const bool gap_ok = !isfinite(fs) || (g.F - fs) / fabs(fs) <= p.tol_gap;
                    if (g.nonfinite) {
                        g.status = ASYFLEXA_ENONFINITE;
                        g.done = 1;
                    } else if (p.sweeps_only) {
                        if (g.sweeps >= p.max_sweeps) {
                            g.done = 1;
                        } else {
                            g.k_sweeps = static_cast<int>(p.max_sweeps - g.sweeps);
                            g.phase = kGsSweep;
                        }
                    } else if (gap_ok && g.plain_refresh && isfinite(fs)) {
                        // a plain refresh passed the gap test: redo it exactly before trusting it
                        g.exact = 1;
                        g.plain_refresh = 0;
                        g.phase = kGsRefresh;
                        g.reset = 1;
                    } else {
                        if (gap_ok && isfinite(fs)) g.exact = 1;
                        g.gap_last = isfinite(fs) ? (g.F - fs) / fabs(fs) : NAN;
                        if (g.sweeps > 0 && gap_ok)
                            g.phase = kGsMerit;
                        else
                            sweep_next = true;
                    }
                } else if (phase == kGsMerit) {
                    ++g.checks;
                    const double st = g.merit / fmax(1.0, g.xmax);
                    g.stat_last = static_cast<float>(st);
                    if (!isfinite(g.merit)) {
                        g.status = ASYFLEXA_ENONFINITE;
                        g.done = 1;
                    } else if (st <= p.tol_stat) {
                        g.status = ASYFLEXA_OK;
                        g.done = 1;
                    } else {
                        const bool better = st < 0.9 * g.stat_ref;
                        if (better) g.stat_ref = st;
                        if (!g.exact) {
                            g.flat_plain = better ? 0 : g.flat_plain + 1;
                            if (st <= kGsFloorBand * p.tol_stat || g.flat_plain >= 2) g.exact = 1;
                        } else if (better) {
                            g.flat = 0;
                        } else if (st <= kGsFloorBand * p.tol_stat && ++g.flat >= kGsFloorChecks) {
                            g.done = 1;
                        }
                        sweep_next = !g.done;
                    }
                } else {
                    // sweeps done: exact residual and F next
                    g.sweeps += k_sweeps;
                    g.phase = kGsRefresh;
                    g.reset = 1;
                }
                if (sweep_next) {
                    if (g.sweeps >= p.max_sweeps) {
                        g.done = 1;
                    } else if (p.handoff_sweeps > 0 && g.sweeps >= p.handoff_sweeps) {
                        g.status = kGsHandoff;
                        g.done = 1;
                    } else {
                        // near the tolerance the next check comes after 2 sweeps; far from the gap
                        // (above 1e-2 with a known f_star) after 4 check intervals, with plain
                        // products in the refresh
                        const bool near = phase == kGsMerit && g.stat_last <= 2.0 * p.tol_stat;
                        const bool far = !g.exact && g.gap_last > kGsFarGap;
                        g.plain_refresh = far ? 1 : 0;
                        long long k = near ? 2 : (far ? kGsFarChecks * p.check_every : p.check_every);
                        if (k > p.max_sweeps - g.sweeps) k = p.max_sweeps - g.sweeps;
                        g.k_sweeps = static_cast<int>(k);
                        g.phase = kGsSweep;
                    }
                }
            }
            __syncthreads();
            if (misc->done) break;
            if (misc->reset && !producer) reset_r();
        }
        if (tid == 0) {
            GsInst& O = p.inst[ii];
            O.F = misc->F;
            O.stat = static_cast<double>(misc->stat_last);
            O.xmax = misc->xmax;
            O.sweeps = misc->sweeps;
            O.nnz = misc->nnz;
            O.status = *abort_flag ? kDevTimeout : misc->status;
            O.checks = misc->checks;
            O.w_used = w;
            O.ns = static_cast<long long>(global_timer_ns() - t_start);
        }
        __syncthreads();  // the results and misc are read before the next problem rewrites misc
    }
    // after an abort a bulk copy may still be writing a slot: wait (bounded) for the last
    // item issued into every slot before the CTA exits
    if (producer && lane == 0 && *abort_flag) {
        for (int s = 0; s < S; ++s) {
            long long last = -1;
            for (long long q = it - 1; q >= 0 && q >= it - S; --q)
                if (q % S == s) last = q;
            if (last < 0) continue;
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(&full[s], static_cast<uint32_t>((last / S) & 1))) {
                if (global_timer_ns() - t0 > kWaitLimitNs) break;
            }
        }
    }
}

}  // namespace asyflexa
