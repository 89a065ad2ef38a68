// The block-update sweep kernel (Algorithm 1, steps S.1-S.5) for both execution modes.
//
// One CTA = 1 producer warp + kConsWarps consumer warps.  Each CTA owns the blocks
// b = blockIdx.x, blockIdx.x + gridDim.x, ... (a fixed partition, Assumption D4) and
// processes them in that order once per sweep.  For a block of w columns:
//
//   (S.2 read)  r~ <- r (FP64 residual in L2, widened/narrowed to TC, staged in shared
//               memory; in async mode this is the possibly stale residual);
//   (S.2 grad)  g_j = a_j^T r~ for the block's columns.  The producer streams the
//               column panel through a ring of shared-memory stages with 1-D bulk
//               (TMA) copies; consumers read 16-byte units and reduce with warp
//               shuffles and a fixed-order cross-warp sum (deterministic);
//   (S.2 best response, eq. 2 with the Section 4 surrogate)
//               xhat_j = clip(soft(x_j - grad_j/d_j, lam/d_j), lo_j, hi_j);
//   (S.3/S.4)   x_j <- x_j + gamma (xhat_j - x_j), owner-exclusive (D4);
//   async:      r += A_i Delta_i with FP64 atomic adds (lock-free; the stale-read model
//               of the Appendix bounds the inconsistency by the updates in flight);
//   sync:       Delta_j is written out and applied to r by a separate deterministic
//               gather kernel after all blocks are done (Jacobi).
//
// Residual tiling: r~ holds tile_rows rows; when m is larger the panel is processed
// tile by tile (tile-major), accumulating per-warp partial sums across tiles.
#pragma once

#include "ptx.cuh"
#include "types.cuh"

namespace asyflexa {

constexpr int kConsWarps = 8;
constexpr int kConsThreads = kConsWarps * 32;
constexpr int kSweepThreads = kConsThreads + 32;
constexpr int kWMax = 128;

enum SweepMode : int { kJacobi = 0, kAsync = 1 };

struct SweepLayout {
    int stages;
    int chunk_rows;
    int tile_rows;
    size_t stage_bytes;
    size_t off_ring, off_rt, off_colsum, off_actj, off_actv, off_flag, off_bars, off_misc, total;
};

__host__ __device__ inline size_t align_up_sz(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SweepLayout make_sweep_layout(int elt_a, int elt_c, int stages, int chunk_rows,
                                                         int tile_rows) {
    SweepLayout L;
    L.stages = stages;
    L.chunk_rows = chunk_rows;
    L.tile_rows = tile_rows;
    L.stage_bytes = align_up_sz(static_cast<size_t>(chunk_rows) * elt_a, 128);
    size_t o = 0;
    L.off_ring = o;
    o += L.stage_bytes * stages;
    L.off_rt = o;
    o = align_up_sz(o + static_cast<size_t>(tile_rows) * elt_c, 16);
    L.off_colsum = o;
    o = align_up_sz(o + static_cast<size_t>(kConsWarps) * kWMax * elt_c, 16);
    L.off_actj = o;
    o = align_up_sz(o + kWMax * sizeof(int), 16);
    L.off_actv = o;
    o = align_up_sz(o + static_cast<size_t>(kWMax) * elt_c, 16);
    L.off_flag = o;
    o = align_up_sz(o + kWMax * sizeof(int), 16);
    L.off_bars = o;
    o = align_up_sz(o + 2 * stages * sizeof(uint64_t), 16);
    L.off_misc = o;
    o += 16;
    L.total = align_up_sz(o, 128);
    return L;
}

// One problem of a batched launch (see sweep_async.cuh).
struct BatchInst {
    const void* A;
    int64_t lda, m, mcopy, n;
    double* r;
    void* x;
    const void* lo;
    const void* hi;
    const void* lin;
    const double* dw;
    const float* scale;
    double lam, s_loss, c2;
    int w, nblocks, active, pad;
};

struct SweepParams {
    const void* A;
    int64_t lda, m, mcopy, n;
    const float* scale;      // per-column scale of A (quantised storage) or nullptr
    double* r;               // residual, FP64, mcopy entries (rows >= m kept at zero)
    void* x;                 // TX[n]
    const void* lo;          // TX[n] or nullptr
    const void* hi;          // TX[n] or nullptr
    const double* dw;        // surrogate weights d_j
    const void* lin;         // TX[n] linear term of f, or nullptr
    double lam, gamma, s_loss, c2;  // lam: weight of ||x||_1 in G (lam * eta for the DC losses)
    DcTerm dc;               // linearised concave part -lam H- of f (kind 0: none)
    const double* gtab;      // diminishing steps of this launch (nullptr: fixed step gamma)
    long long gtab_len;      // entries of gtab (sweeps * nblocks)
    unsigned long long k_base;  // update index of gtab[0] (async: value of counters[0] at launch)
    int w, nblocks, sweeps;
    int tile_rows, ntiles, chunk_rows, stages;
    void* delta;             // Jacobi: TC[n] applied step
    unsigned long long* counters;  // [0] global update counter, [1] block updates, [2] blocks with Delta != 0
    unsigned long long* hist;      // 32-bucket staleness histogram
    int* err;
    int delay_ns;                  // test-only: odd CTAs sleep this long before each scatter (0: off)
    // batched launches only
    const BatchInst* batch;        // problem table
    const int* blk_inst;           // global block -> problem
    const int* blk_local;          // global block -> block index within its problem
    int total_blocks;
    int keep_a_in_l2;              // 1: load A with normal L2 priority (several problems share A)
};

// Step of update index `idx` within this launch's table (clamped), or the fixed step.
__device__ __forceinline__ double launch_step(const SweepParams& p, long long idx) {
    if (!p.gtab) return p.gamma;
    idx = idx < 0 ? 0 : (idx >= p.gtab_len ? p.gtab_len - 1 : idx);
    return p.gtab[idx];
}

template <typename TC>
__device__ __forceinline__ TC warp_sum(TC v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Closed-form best response and fixed step for one coordinate, in FP64.
// Returns the applied change Delta = x_new - x_old (exact difference of the stored values).
template <typename TX>
__device__ __forceinline__ double coordinate_update(double g_atr, TX* x, const TX* lo, const TX* hi, int64_t j,
                                                    double dj, double lam, double gamma, double s_loss,
                                                    double c2, double linj, const DcTerm& dc) {
    const double xj = static_cast<double>(x[j]);
    const double grad = s_loss * g_atr - c2 * xj + linj - dc.lam * dc_hminus_grad(dc, xj);
    double xh = 0.0;
    if (dj > 0.0) {
        const double v = xj - grad / dj;
        const double t = lam / dj;
        const double av = fabs(v) - t;
        xh = av > 0.0 ? copysign(av, v) : 0.0;
    }
    if (lo) xh = fmax(xh, static_cast<double>(lo[j]));
    if (hi) xh = fmin(xh, static_cast<double>(hi[j]));
    const TX xn = static_cast<TX>(xj + gamma * (xh - xj));
    x[j] = xn;
    return static_cast<double>(xn) - xj;
}

template <typename TA, int MODE>
__global__ void __launch_bounds__(kSweepThreads, 1) sweep_kernel(const SweepParams p) {
    using TC = typename ATraits<TA>::TC;
    using TX = typename XType<TA>::T;
    constexpr int V = ATraits<TA>::kVec;

    extern __shared__ __align__(128) unsigned char smem[];
    const SweepLayout L = make_sweep_layout(sizeof(TA), sizeof(TC), p.stages, p.chunk_rows, p.tile_rows);
    unsigned char* ring = smem + L.off_ring;
    TC* rt = reinterpret_cast<TC*>(smem + L.off_rt);
    TC* colsum = reinterpret_cast<TC*>(smem + L.off_colsum);
    int* actj = reinterpret_cast<int*>(smem + L.off_actj);
    TC* actv = reinterpret_cast<TC*>(smem + L.off_actv);
    int* aflag = reinterpret_cast<int*>(smem + L.off_flag);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.off_bars);
    uint64_t* empty = full + p.stages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.off_misc);
    int* s_nact = reinterpret_cast<int*>(smem + L.off_misc + 4);
    unsigned long long* s_u0 = reinterpret_cast<unsigned long long*>(smem + L.off_misc + 8);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const TA* A = static_cast<const TA*>(p.A);
    const int64_t lda = p.lda;

    if (tid == 0) {
        for (int s = 0; s < p.stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsWarps);
        }
        *abort_flag = 0;
        *s_nact = 0;
        fence_barrier_init();
    }
    __syncthreads();

    // ------------------------------------------------------------------ producer
    if (warp == kConsWarps) {
        if (lane != 0) return;
        const uint64_t pol = l2_policy_evict_first();
        uint32_t stage = 0, phase = 0;
        long long issued = 0;
        for (int s = 0; s < p.sweeps; ++s) {
            for (int b = blockIdx.x; b < p.nblocks; b += gridDim.x) {
                const int64_t c0 = static_cast<int64_t>(b) * p.w;
                const int wb = static_cast<int>(min64(p.w, p.n - c0));
                for (int t = 0; t < p.ntiles; ++t) {
                    const int64_t row0 = static_cast<int64_t>(t) * p.tile_rows;
                    const int64_t rows = min64(p.tile_rows, p.mcopy - row0);
                    for (int jl = 0; jl < wb; ++jl) {
                        const TA* col = A + (c0 + jl) * lda + row0;
                        for (int64_t cr = 0; cr < rows; cr += p.chunk_rows) {
                            const uint32_t nbytes =
                                static_cast<uint32_t>(min64(p.chunk_rows, rows - cr) * sizeof(TA));
                            if (!mbar_wait_bounded(&empty[stage], phase ^ 1u, abort_flag, p.err)) goto drain;
                            mbar_arrive_expect_tx(&full[stage], nbytes);
                            bulk_load(ring + stage * L.stage_bytes, col + cr, nbytes, &full[stage], pol);
                            ++issued;
                            if (++stage == static_cast<uint32_t>(p.stages)) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                }
            }
        }
        return;
    drain:
        // Aborted: wait (bounded) until the copies this thread issued have landed so that
        // no bulk copy targets shared memory after the CTA exits.
        {
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
    bool rt_valid = false;
    unsigned long long u0 = 0;
    unsigned long long my_updates = 0, my_active = 0;
    TX* x = static_cast<TX*>(p.x);
    const TX* lo = static_cast<const TX*>(p.lo);
    const TX* hi = static_cast<const TX*>(p.hi);

    for (int s = 0; s < p.sweeps; ++s) {
        for (int b = blockIdx.x; b < p.nblocks; b += gridDim.x) {
            const int64_t c0 = static_cast<int64_t>(b) * p.w;
            const int wb = static_cast<int>(min64(p.w, p.n - c0));
            for (int t = 0; t < p.ntiles; ++t) {
                const int64_t row0 = static_cast<int64_t>(t) * p.tile_rows;
                const int64_t rows = min64(p.tile_rows, p.mcopy - row0);
                if (MODE == kAsync || p.ntiles > 1 || !rt_valid) {
                    named_bar_sync(1, kConsThreads);  // every consumer is done with the old tile
                    if (MODE == kAsync && t == 0 && tid == 0) {
                        u0 = ld_relaxed_u64(&p.counters[0]);
                        *s_u0 = u0;  // read by the epilogue threads (several barriers later)
                    }
                    const double2* rsrc = reinterpret_cast<const double2*>(p.r + row0);
                    for (int64_t i = tid; i < rows / 2; i += kConsThreads) {
                        const double2 v = __ldcg(rsrc + i);
                        rt[2 * i] = static_cast<TC>(v.x);
                        rt[2 * i + 1] = static_cast<TC>(v.y);
                    }
                    named_bar_sync(1, kConsThreads);
                    rt_valid = true;
                }
                for (int jl = 0; jl < wb; ++jl) {
                    TC acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
                    for (int64_t cr = 0; cr < rows; cr += p.chunk_rows) {
                        const int nrows = static_cast<int>(min64(p.chunk_rows, rows - cr));
                        const bool ok = !*abort_flag && mbar_wait_bounded(&full[stage], phase, abort_flag, p.err);
                        if (ok) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + stage * L.stage_bytes);
                            const TC* rr = rt + cr;
                            const int64_t grow0 = row0 + cr;  // global row of the chunk's first element
                            const int units = nrows / V;
                            // units whose rows are all < m
                            const int full_units =
                                grow0 + nrows <= p.m ? units : static_cast<int>((p.m - grow0) / V);
                            int u = tid;
                            for (; u + 3 * kConsThreads < full_units; u += 4 * kConsThreads) {
                                const uint4 q0 = src[u];
                                const uint4 q1 = src[u + kConsThreads];
                                const uint4 q2 = src[u + 2 * kConsThreads];
                                const uint4 q3 = src[u + 3 * kConsThreads];
                                TC a0[V], a1[V], a2[V], a3[V];
                                ATraits<TA>::unpack(q0, a0);
                                ATraits<TA>::unpack(q1, a1);
                                ATraits<TA>::unpack(q2, a2);
                                ATraits<TA>::unpack(q3, a3);
                                const TC* r0 = rr + static_cast<int64_t>(u) * V;
                                const TC* r1 = r0 + kConsThreads * V;
                                const TC* r2 = r1 + kConsThreads * V;
                                const TC* r3 = r2 + kConsThreads * V;
#pragma unroll
                                for (int e = 0; e < V; ++e) {
                                    acc0 = fmac(a0[e], r0[e], acc0);
                                    acc1 = fmac(a1[e], r1[e], acc1);
                                    acc2 = fmac(a2[e], r2[e], acc2);
                                    acc3 = fmac(a3[e], r3[e], acc3);
                                }
                            }
                            for (; u < full_units; u += kConsThreads) {
                                const uint4 q0 = src[u];
                                TC a0[V];
                                ATraits<TA>::unpack(q0, a0);
                                const TC* r0 = rr + static_cast<int64_t>(u) * V;
#pragma unroll
                                for (int e = 0; e < V; ++e) acc0 = fmac(a0[e], r0[e], acc0);
                            }
                            if (full_units < units && tid == full_units % kConsThreads && u == full_units) {
                                // the single unit straddling row m: mask the padding rows
                                const uint4 q0 = src[full_units];
                                TC a0[V];
                                ATraits<TA>::unpack(q0, a0);
                                const TC* r0 = rr + static_cast<int64_t>(full_units) * V;
                                const int valid = static_cast<int>(p.m - (grow0 + static_cast<int64_t>(full_units) * V));
#pragma unroll
                                for (int e = 0; e < V; ++e)
                                    if (e < valid) acc0 = fmac(a0[e], r0[e], acc0);
                            }
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[stage]);
                        if (++stage == static_cast<uint32_t>(p.stages)) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    TC v = (acc0 + acc1) + (acc2 + acc3);
                    v = warp_sum(v);
                    if (lane == 0) {
                        TC* cs = colsum + warp * kWMax + jl;
                        *cs = (t == 0) ? v : (*cs + v);
                    }
                }
            }
            named_bar_sync(1, kConsThreads);  // colsum complete

            // ---------------- best response + fixed step (one thread per column)
            const bool aborted = *abort_flag != 0;
            if (tid < wb) {
                int flag = 0;
                TC dv = 0;
                if (!aborted) {
                    double g = 0.0;
#pragma unroll
                    for (int k = 0; k < kConsWarps; ++k) g += static_cast<double>(colsum[k * kWMax + tid]);
                    const int64_t j = c0 + tid;
                    const double sc = p.scale ? static_cast<double>(p.scale[j]) : 1.0;
                    const double linj = p.lin ? static_cast<double>(static_cast<const TX*>(p.lin)[j]) : 0.0;
                    // step of this block update: the update index is the number of updates completed
                    // before its residual read (async) or its position in the sweep (Jacobi)
                    const double gam =
                        launch_step(p, MODE == kAsync ? static_cast<long long>(*s_u0 - p.k_base)
                                                      : static_cast<long long>(s) * p.nblocks + b);
                    const double delta = coordinate_update<TX>(g * sc, x, lo, hi, j, p.dw[j], p.lam, gam,
                                                               p.s_loss, p.c2, linj, p.dc);
                    flag = delta != 0.0;
                    if (MODE == kJacobi) {
                        static_cast<TC*>(p.delta)[j] = static_cast<TC>(delta);
                    } else {
                        dv = static_cast<TC>(delta * sc);
                    }
                }
                aflag[tid] = flag;
                actv[tid] = dv;
            }
            named_bar_sync(1, kConsThreads);  // epilogue done: colsum free, flags written
            if (MODE == kJacobi) {
                if (tid == 0) ++my_updates;
                continue;
            }

            // ---------------- async: scatter r += A_i Delta_i
            if (p.delay_ns > 0 && (blockIdx.x & 1u)) __nanosleep(static_cast<unsigned>(p.delay_ns));
            if (warp == 0) {
                int base_out = 0;
                for (int base = 0; base < wb; base += 32) {
                    const int jl = base + lane;
                    const int f = (jl < wb) ? aflag[jl] : 0;
                    const TC dvl = (jl < wb) ? actv[jl] : TC(0);
                    const unsigned bal = __ballot_sync(0xffffffffu, f);
                    __syncwarp();
                    if (f) {
                        const int pos = base_out + __popc(bal & ((1u << lane) - 1u));
                        actj[pos] = static_cast<int>(jl);
                        actv[pos] = dvl;  // pos <= jl: never overwrites an unread entry
                    }
                    __syncwarp();
                    base_out += __popc(bal);
                }
                if (lane == 0) *s_nact = base_out;
            }
            named_bar_sync(1, kConsThreads);
            const int nact = *s_nact;
            if (tid == 0) {
                ++my_updates;
                if (nact) ++my_active;
            }
            if (nact > 0 && !*abort_flag) {
                const int64_t units = p.mcopy / V;
                for (int64_t u = tid; u < units; u += kConsThreads) {
                    TC inc[V];
#pragma unroll
                    for (int e = 0; e < V; ++e) inc[e] = 0;
                    int k = 0;
                    for (; k + 1 < nact; k += 2) {
                        const uint4 qa = ld_stream_u4(A + (c0 + actj[k]) * lda + u * V);
                        const uint4 qb = ld_stream_u4(A + (c0 + actj[k + 1]) * lda + u * V);
                        TC a[V], bb[V];
                        ATraits<TA>::unpack(qa, a);
                        ATraits<TA>::unpack(qb, bb);
                        const TC da = actv[k], db = actv[k + 1];
#pragma unroll
                        for (int e = 0; e < V; ++e) inc[e] = fmac(bb[e], db, fmac(a[e], da, inc[e]));
                    }
                    if (k < nact) {
                        const uint4 qa = ld_stream_u4(A + (c0 + actj[k]) * lda + u * V);
                        TC a[V];
                        ATraits<TA>::unpack(qa, a);
                        const TC da = actv[k];
#pragma unroll
                        for (int e = 0; e < V; ++e) inc[e] = fmac(a[e], da, inc[e]);
                    }
                    const int64_t row = u * V;
#pragma unroll
                    for (int e = 0; e < V; ++e)
                        if (row + e < p.m && inc[e] != TC(0)) red_add_f64(p.r + row + e, static_cast<double>(inc[e]));
                }
                __threadfence();
            }
            named_bar_sync(1, kConsThreads);  // scatter of this block complete and visible
            if (tid == 0) {
                const unsigned long long u1 = atomicAdd(&p.counters[0], 1ull);
                const unsigned long long dly = u1 - u0;
                int bucket = 63 - __clzll(static_cast<long long>(dly + 1ull));
                bucket = bucket > 31 ? 31 : bucket;
                atomicAdd(&p.hist[bucket], 1ull);
            }
        }
    }
    if (tid == 0) {
        atomicAdd(&p.counters[1], my_updates);
        if (MODE == kAsync) atomicAdd(&p.counters[2], my_active);
    }
}

}  // namespace asyflexa
