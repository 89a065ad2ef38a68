// Batched Gauss-Seidel form: many independent FP32 problems solved in ONE persistent launch,
// one CTA per problem at a time.
//
// A CTA takes the next problem from a queue (problems ordered by decreasing size, so that
// the largest start first) and runs Algorithm 1 on it with a single owner for every block:
// with one CTA there are no updates in flight, so the iteration is exact cyclic
// Gauss-Seidel over scalar blocks (the paper's own block choice, Section 4.1) with the fixed
// step of S.4 and the best response of eq. 2.  The CTA then runs its own stopping test
// (exact residual, F, gap, and the Section 4.3 merit ||xhat(x) - x||_inf / max(1, ||x||_inf))
// and goes on with the next problem, so the whole batch needs no host round trip.
//
//   * The residual r = A x - b lives in registers for the whole solve: consumer thread t
//     owns the 16-byte units u = k * T + t (k < UPT, 4 rows each) of every column, and holds
//     r for those rows as an unevaluated FP32 pair (hi, lo) so that small late increments
//     are not lost to FP32 rounding.  Because a thread reads and updates only its own rows,
//     the update r += a_j Delta_j needs no barrier before the next column's gradient.
//   * A producer warp streams the columns HBM -> SMEM with 1-D bulk (TMA) copies into a ring
//     of S slots (full / empty mbarriers).  With each copy it stages the column's
//     coefficients (x_j, 1/d_j, lam/d_j, bounds, linear term) next to the slot.
//   * One named barrier per column publishes the per-warp partial sums of a_j^T r; every
//     consumer thread then evaluates the same FP32 best response (gs_delta).
//   * Every gradient a_j^T r is a Dot2 sum (error-free products and sums) over r's (hi, lo) pair.
//   * Phases of one solve: REFRESH (r = -b + sum over x_j != 0 of a_j x_j with error-free
//     products and sums, then F with FP64 sums), SWEEP (k sweeps, k = check_every or 2 near
//     the tolerance), MERIT (x^_j with unit step, the largest |x^_j - x_j|).  A problem stops
//     when its gap (if f_star is known) and its merit meet the tolerances (OK), when F is not
//     finite (ENONFINITE), at max_sweeps, or when, with the gap met and the merit within 100
//     tol_stat, five checks in a row do not lower the best merit by 10% (ENOTCONV: the
//     stationarity floor of the FP32 iterate).
#pragma once

#include <cmath>

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
    const double* dw;
    double lam, s_loss, c2, c;  // s_loss = 1 (LASSO) or 2 (NCQUAD); c2 = 2c; c: NCQUAD weight (for F)
    double f_star;              // NaN: no gap test, stop on the merit alone
    int loss, pad0;
    // written by the kernel
    double F, stat, xmax;
    long long sweeps, nnz;
    int status, checks;
};

struct GsParams {
    GsInst* inst;
    const int* order;   // problems in the order the queue hands them out
    int count;
    int* queue;         // next position in `order` (0 before the launch)
    double gamma, tol_gap, tol_stat;
    int check_every, max_sweeps, stages;
    int64_t slot_bytes;   // ring slot: the longest column's 16-byte units, rounded up to 128 bytes
    int sweeps_only;    // 1: exactly max_sweeps sweeps per problem, no stopping test (autotuner)
    int keep_a_in_l2;   // 1: A shared by the problems (normal L2 priority)
    int* err;
};

// Coefficients of the column in a ring slot (j < 0: end of a REFRESH phase).
struct GsSlot {
    int j;
    float x, dinv, lam, lo, hi, lin, d;  // d = d_j and dinv = 1/d_j in FP32 (0 if d_j <= 0)
};

struct GsLayout {
    size_t slot_bytes, off_ring, off_meta, off_part, off_red, off_bars, off_misc, total;
};

// slot_bytes: the longest column of the batch (16-byte units, rounded up to 128 bytes).
__host__ __device__ inline GsLayout make_gs_layout(int nw, size_t slot_bytes, int stages) {
    GsLayout L;
    L.slot_bytes = slot_bytes;
    size_t o = 0;
    L.off_ring = o;
    o += L.slot_bytes * stages;
    L.off_meta = o;
    o += sizeof(GsSlot) * stages;
    L.off_part = o;  // two buffers of per-warp (s, c) partial pairs
    o += 2 * static_cast<size_t>(nw) * 2 * sizeof(float);
    o = (o + 15) / 16 * 16;
    L.off_red = o;   // per-warp FP64 sums of the objective pieces
    o += static_cast<size_t>(nw) * 8 * sizeof(double);
    L.off_bars = o;
    o += 2 * static_cast<size_t>(stages) * sizeof(uint64_t);
    L.off_misc = o;  // abort flag, queue position, decision values
    o += 64;
    L.total = (o + 127) / 128 * 128;
    return L;
}

constexpr int kGsRefresh = 0, kGsSweep = 1, kGsMerit = 2;
constexpr int kGsFloorChecks = 5;
constexpr double kGsFloorBand = 100.0;  // the floor rule applies within 100 tol_stat

// Shared decision values (written by thread 0 before a CTA barrier, read by every thread).
struct GsMisc {
    int abort, qi, nonfinite, pad;
    double F, xmax, merit;
    long long nnz;
};

// x^_j - x_j for the best response of eq. 2 (soft-threshold, then clip), in FP32, from the
// gradient pair (gh, gl) of a_j^T r.  With q = d x - grad the soft-threshold step is
//     q > lam:  -(grad + lam) / d,    q < -lam:  -(grad - lam) / d,    else:  -x,
// and near a stationary point grad + lam (or grad - lam) cancels: formed as (gh + lam) + gl it
// is exact up to the last rounding (Sterbenz), where x - grad/d loses the digits of a small
// difference of two numbers as large as lam / d.
__device__ __forceinline__ float gs_delta(const GsSlot& c, float gh, float gl, float s_loss, float c2) {
    // grad = s_loss * g - c2 x + lin as a pair (s_loss is 1 or 2: exact)
    float th, tl;
    two_sum(s_loss * gh, fmaf(-c2, c.x, c.lin), th, tl);
    tl += s_loss * gl;
    float e;
    if (c.dinv > 0.f) {
        const float q = fmaf(c.x, c.d, -th) - tl;
        if (q > c.lam)
            e = -((th + c.lam) + tl) * c.dinv;
        else if (q < -c.lam)
            e = -((th - c.lam) + tl) * c.dinv;
        else
            e = -c.x;
    } else {
        e = -c.x;  // d_j = 0: x^_j = clip(0)
    }
    // the box, if active; otherwise e itself (not x + e rounded to FP32 and minus x, which
    // would hide a step below half an ulp of x from the stopping test)
    const float xe = c.x + e;
    if (xe < c.lo) return c.lo - c.x;
    if (xe > c.hi) return c.hi - c.x;
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
    GsSlot* meta = reinterpret_cast<GsSlot*>(smem + L.off_meta);
    float2* part = reinterpret_cast<float2*>(smem + L.off_part);
    double* red = reinterpret_cast<double*>(smem + L.off_red);
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
    int buf = 0;        // partial-sum buffer of the next column
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
        const int64_t lda = I.lda, m = I.m, n = I.n;
        const int64_t units = (m + 3) / 4;
        const uint32_t col_bytes = static_cast<uint32_t>(units * 16);
        const float s_loss = static_cast<float>(I.s_loss), c2 = static_cast<float>(I.c2);
        const float gamma = static_cast<float>(p.gamma);

        if (!producer) {
#pragma unroll
            for (int k = 0; k < UPT; ++k) {
                const int64_t u = static_cast<int64_t>(k) * T + tid;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int64_t row = u * 4 + e;
                    rhi[k][e] = row < m ? -I.b[row] : 0.f;
                    rlo[k][e] = 0.f;
                }
            }
        }

        long long sweeps = 0;
        int status = ASYFLEXA_ENOTCONV, checks = 0, phase = kGsRefresh, k_sweeps = 0;
        float stat_last = NAN;
        // stationarity floor: with the gap met and the merit within kGsFloorBand tol_stat,
        // kGsFloorChecks checks in a row that do not lower the best merit by 10% end the solve
        // (ENOTCONV): the FP32 iterate has stopped moving
        double stat_ref = INFINITY;
        int flat = 0;
        for (;;) {
            // ================================================================ one phase
            if (producer) {
                // ---- issue the phase's columns into the ring (lane 0), in consumption order.
                // wait_free(q, lead): item q may be issued once item q - lead has been consumed
                auto wait_free = [&](long long q, long long lead_items) -> bool {
                    if (q < lead_items) return true;
                    const long long r0 = q - lead_items;
                    return mbar_wait_bounded(&empty[r0 % S], static_cast<uint32_t>((r0 / S) & 1), abort_flag, p.err);
                };
                auto put = [&](const GsSlot& c) {
                    const int slot = static_cast<int>(it % S);
                    meta[slot] = c;
                    if (c.j >= 0) {
                        mbar_arrive_expect_tx(&full[slot], col_bytes);
                        bulk_load(ring + slot * L.slot_bytes, A + static_cast<int64_t>(c.j) * lda, col_bytes,
                                  &full[slot], pol);
                    } else {
                        mbar_arrive(&full[slot]);
                    }
                    ++it;
                };
                auto coef = [&](int j, float xj) {
                    GsSlot c;
                    c.j = j;
                    c.x = xj;
                    const double dj = I.dw[j];
                    c.dinv = dj > 0.0 ? static_cast<float>(1.0 / dj) : 0.f;
                    c.d = dj > 0.0 ? static_cast<float>(dj) : 0.f;
                    c.lam = static_cast<float>(I.lam);
                    c.lo = I.lo ? I.lo[j] : -INFINITY;
                    c.hi = I.hi ? I.hi[j] : INFINITY;
                    c.lin = I.lin ? I.lin[j] : 0.f;
                    return c;
                };
                if (phase == kGsRefresh) {
                    // the nonzero columns of x, found 32 at a time by the whole warp
                    bool go = true;
                    for (int64_t j0 = 0; j0 < n && go; j0 += 32) {
                        const int64_t j = j0 + lane;
                        const float xv = j < n ? I.x[j] : 0.f;
                        unsigned mask = __ballot_sync(0xffffffffu, xv != 0.f);
                        while (mask && go) {
                            const int bit = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const float xj = __shfl_sync(0xffffffffu, xv, bit);
                            int okl = 1;
                            if (lane == 0) {
                                okl = wait_free(it, S) ? 1 : 0;
                                if (okl) {
                                    GsSlot c{};
                                    c.j = static_cast<int>(j0 + bit);
                                    c.x = xj;
                                    put(c);
                                }
                            }
                            go = __shfl_sync(0xffffffffu, okl, 0) != 0;
                        }
                    }
                    if (lane == 0 && go && wait_free(it, S)) {
                        GsSlot c{};
                        c.j = -1;
                        put(c);
                    }
                } else {
                    const bool sweep = phase == kGsSweep;
                    const long long cnt = sweep ? static_cast<long long>(k_sweeps) * n : n;
                    // x_j of a sweep is final once the column's previous update is consumed: with
                    // n >= S + 32 the slot-free wait of the first of 32 items guarantees it for all
                    // 32, whose coefficients the warp then loads at once; otherwise lane 0 loads
                    // them column by column, at most min(S, n) items ahead
                    const bool batch = !sweep || n >= S + 32;
                    if (batch) {
                        bool go = true;
                        for (long long q0 = 0; q0 < cnt && go; q0 += 32) {
                            int okl = 1;
                            if (lane == 0) okl = wait_free(it, S) ? 1 : 0;
                            go = __shfl_sync(0xffffffffu, okl, 0) != 0;
                            if (!go) break;
                            const long long q = q0 + lane;
                            GsSlot mine{};
                            if (q < cnt) {
                                const int j = static_cast<int>(q % n);
                                mine = coef(j, I.x[j]);
                            }
                            const int nb = static_cast<int>(cnt - q0 < 32 ? cnt - q0 : 32);
                            for (int l = 0; l < nb && go; ++l) {
                                GsSlot c;
                                c.j = __shfl_sync(0xffffffffu, mine.j, l);
                                c.x = __shfl_sync(0xffffffffu, mine.x, l);
                                c.dinv = __shfl_sync(0xffffffffu, mine.dinv, l);
                                c.lam = __shfl_sync(0xffffffffu, mine.lam, l);
                                c.lo = __shfl_sync(0xffffffffu, mine.lo, l);
                                c.hi = __shfl_sync(0xffffffffu, mine.hi, l);
                                c.lin = __shfl_sync(0xffffffffu, mine.lin, l);
                                c.d = __shfl_sync(0xffffffffu, mine.d, l);
                                if (lane == 0) {
                                    okl = wait_free(it, S) ? 1 : 0;
                                    if (okl) put(c);
                                }
                                go = __shfl_sync(0xffffffffu, okl, 0) != 0;
                            }
                        }
                    } else if (lane == 0) {
                        const long long lead = n < S ? n : S;
                        for (long long q = 0; q < cnt; ++q) {
                            if (!wait_free(it, lead)) break;
                            const int j = static_cast<int>(q % n);
                            put(coef(j, I.x[j]));
                        }
                    }
                }
                it = __shfl_sync(0xffffffffu, it, 0);
            } else if (phase == kGsRefresh) {
                // ---- r += a_j x_j over the nonzero columns (no barrier: every thread reads and
                // writes only its own rows)
                for (;;) {
                    const int slot = static_cast<int>(it % S);
                    ok = ok && !*abort_flag &&
                         mbar_wait_bounded(&full[slot], static_cast<uint32_t>((it / S) & 1), abort_flag, p.err);
                    if (!ok) break;
                    const GsSlot c = meta[slot];
                    if (c.j >= 0) {
                        const uint4* src = reinterpret_cast<const uint4*>(ring + slot * L.slot_bytes);
#pragma unroll
                        for (int k = 0; k < UPT; ++k) {
                            const int64_t u = static_cast<int64_t>(k) * T + tid;
                            if (u < units) {
                                float a[4];
                                ATraits<float>::unpack(src[k * T + tid], a);
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (u * 4 + e < m) ff_add_prod(rhi[k][e], rlo[k][e], a[e], c.x);
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[slot]);
                    ++it;
                    if (c.j < 0) break;
                }
            } else {
                // ---- SWEEP (k sweeps of cyclic coordinate updates) or MERIT (one pass, no update)
                const bool merit = phase == kGsMerit;
                const long long cnt = merit ? n : static_cast<long long>(k_sweeps) * n;
                float mmax = 0.f;
                bool bad = false;
                for (long long q = 0; q < cnt; ++q) {
                    const int slot = static_cast<int>(it % S);
                    ok = ok && !*abort_flag &&
                         mbar_wait_bounded(&full[slot], static_cast<uint32_t>((it / S) & 1), abort_flag, p.err);
                    const GsSlot c = meta[slot];
                    const uint4* src = reinterpret_cast<const uint4*>(ring + slot * L.slot_bytes);
                    // a_j^T r with Dot2 products on r's (hi, lo) pair in both phases: a plain FP32
                    // dot of length m errs by about sqrt(m) eps ||a_j|| ||r||, which divided by
                    // d_j = ||a_j||^2 would put the iteration's fixed point 1e-5 away from
                    // stationarity on columns of moderate norm
                    uint4 colr[UPT];
                    DFAcc dacc0, dacc1;
                    float lo_acc = 0.f;
#pragma unroll
                    for (int k = 0; k < UPT; ++k) {
                        const int64_t u = static_cast<int64_t>(k) * T + tid;
                        colr[k] = (ok && u < units) ? src[k * T + tid] : make_uint4(0u, 0u, 0u, 0u);
                        if (u == units - 1) {  // rows past m in the last unit
                            const int valid = static_cast<int>(m - u * 4);
                            if (valid < 4) colr[k].w = 0u;
                            if (valid < 3) colr[k].z = 0u;
                            if (valid < 2) colr[k].y = 0u;
                        }
                        float a[4];
                        ATraits<float>::unpack(colr[k], a);
                        dacc0.add_prod(a[0], rhi[k][0]);
                        dacc1.add_prod(a[1], rhi[k][1]);
                        dacc0.add_prod(a[2], rhi[k][2]);
                        dacc1.add_prod(a[3], rhi[k][3]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) lo_acc = fmaf(a[e], rlo[k][e], lo_acc);
                    }
                    float2* cp = part + buf * NW;
                    {
                        float ts, tc;
                        two_sum(dacc0.s, dacc1.s, ts, tc);
                        tc += (dacc0.c + dacc1.c) + lo_acc;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const float so = __shfl_xor_sync(0xffffffffu, ts, o);
                            const float co = __shfl_xor_sync(0xffffffffu, tc, o);
                            float t, e;
                            two_sum(ts, so, t, e);
                            tc = (tc + co) + e;
                            ts = t;
                        }
                        if (lane == 0) cp[warp] = make_float2(ts, tc);
                    }
                    named_bar_sync(1, T);
                    // the NW partial pairs in a fixed order: every thread gets the same g
                    float gh, gl;
                    {
                        float s = cp[0].x, cc = cp[0].y;
#pragma unroll
                        for (int w = 1; w < NW; ++w) {
                            float t, e;
                            two_sum(s, cp[w].x, t, e);
                            cc = (cc + cp[w].y) + e;
                            s = t;
                        }
                        two_sum(s, cc, gh, gl);
                    }
                    buf ^= 1;
                    const float e = gs_delta(c, gh, gl, s_loss, c2);
                    if (merit) {
                        // |x^_j - x_j| (unit step): the Section 4.3 merit
                        mmax = fmaxf(mmax, fabsf(e));
                        bad |= !(fabsf(gh) <= 3.0e38f);  // NaN or infinite gradient
                    } else {
                        const float xn = fmaf(gamma, e, c.x);
                        const float dlt = xn - c.x;
                        if (ok && tid == 0) I.x[c.j] = xn;
                        if (ok && dlt != 0.f) {
#pragma unroll
                            for (int k = 0; k < UPT; ++k) {
                                float a[4];
                                ATraits<float>::unpack(colr[k], a);
#pragma unroll
                                for (int e = 0; e < 4; ++e) ff_add_prod(rhi[k][e], rlo[k][e], a[e], dlt);
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0 && ok) mbar_arrive(&empty[slot]);
                    ++it;
                }
                if (merit && tid == 0) {
                    misc->merit = bad ? NAN : static_cast<double>(mmax);
                }
            }
            __syncthreads();  // phase done: x and the ring are quiescent

            // ================================================================ after the phase
            if (phase == kGsRefresh && !producer) {
                // F(x) from the exact residual: FP64 sums in a fixed order
                double rr = 0.0, ax = 0.0, x2 = 0.0, lx = 0.0, xm = 0.0, nz = 0.0;
#pragma unroll
                for (int k = 0; k < UPT; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const double v = static_cast<double>(rhi[k][e]) + static_cast<double>(rlo[k][e]);
                        rr += v * v;
                    }
                for (int64_t j = tid; j < n; j += T) {
                    const double xj = static_cast<double>(I.x[j]);
                    ax += fabs(xj);
                    x2 += xj * xj;
                    if (I.lin) lx += static_cast<double>(I.lin[j]) * xj;
                    xm = fmax(xm, fabs(xj));
                    nz += xj != 0.0 ? 1.0 : 0.0;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    rr += __shfl_xor_sync(0xffffffffu, rr, o);
                    ax += __shfl_xor_sync(0xffffffffu, ax, o);
                    x2 += __shfl_xor_sync(0xffffffffu, x2, o);
                    lx += __shfl_xor_sync(0xffffffffu, lx, o);
                    nz += __shfl_xor_sync(0xffffffffu, nz, o);
                    xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
                }
                if (lane == 0) {
                    double* rw = red + warp * 8;
                    rw[0] = rr;
                    rw[1] = ax;
                    rw[2] = x2;
                    rw[3] = lx;
                    rw[4] = nz;
                    rw[5] = xm;
                }
                named_bar_sync(1, T);
                if (tid == 0) {
                    double s[6] = {0, 0, 0, 0, 0, 0};
                    for (int w = 0; w < NW; ++w) {
                        for (int q = 0; q < 5; ++q) s[q] += red[w * 8 + q];
                        s[5] = fmax(s[5], red[w * 8 + 5]);
                    }
                    const double F = (I.loss == ASYFLEXA_LOSS_LASSO ? 0.5 * s[0] : s[0] - I.c * s[2]) + s[3] +
                                     I.lam * s[1];
                    misc->F = F;
                    misc->nnz = static_cast<long long>(s[4]);
                    misc->xmax = s[5];
                    misc->nonfinite = isfinite(F) ? 0 : 1;
                }
            }
            __syncthreads();

            // ================================================================ next phase
            // (the same decision in every thread, from the shared values)
            if (*abort_flag) break;
            if (phase == kGsRefresh) {
                if (misc->nonfinite) {
                    status = ASYFLEXA_ENONFINITE;
                    break;
                }
                if (p.sweeps_only) {
                    if (sweeps >= p.max_sweeps) break;
                    k_sweeps = static_cast<int>(p.max_sweeps - sweeps);
                    phase = kGsSweep;
                    continue;
                }
                const double fs = I.f_star;
                const bool gap_ok = !isfinite(fs) || (misc->F - fs) / fabs(fs) <= p.tol_gap;
                if (sweeps > 0 && gap_ok) {
                    phase = kGsMerit;
                    continue;
                }
            } else if (phase == kGsMerit) {
                ++checks;
                const double st = misc->merit / fmax(1.0, misc->xmax);
                stat_last = static_cast<float>(st);
                if (!isfinite(misc->merit)) {
                    status = ASYFLEXA_ENONFINITE;
                    break;
                }
                if (st <= p.tol_stat) {
                    status = ASYFLEXA_OK;
                    break;
                }
                if (st < 0.9 * stat_ref) {
                    stat_ref = st;
                    flat = 0;
                } else if (st <= kGsFloorBand * p.tol_stat && ++flat >= kGsFloorChecks) {
                    break;
                }
            } else {
                // sweeps done: exact residual and F next
                sweeps += k_sweeps;
                phase = kGsRefresh;
                if (!producer) {
#pragma unroll
                    for (int k = 0; k < UPT; ++k) {
                        const int64_t u = static_cast<int64_t>(k) * T + tid;
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int64_t row = u * 4 + e;
                            rhi[k][e] = row < m ? -I.b[row] : 0.f;
                            rlo[k][e] = 0.f;
                        }
                    }
                }
                continue;
            }
            if (sweeps >= p.max_sweeps) break;
            // near the tolerance the next check comes after 2 sweeps
            const bool near = phase == kGsMerit && stat_last <= 2.0 * p.tol_stat;
            int k = near ? 2 : p.check_every;
            if (k > p.max_sweeps - sweeps) k = static_cast<int>(p.max_sweeps - sweeps);
            k_sweeps = k;
            phase = kGsSweep;
        }
        if (tid == 0) {
            GsInst& O = p.inst[ii];
            O.F = misc->F;
            O.stat = static_cast<double>(stat_last);
            O.xmax = misc->xmax;
            O.sweeps = sweeps;
            O.nnz = misc->nnz;
            O.status = *abort_flag ? kDevTimeout : status;
            O.checks = checks;
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
