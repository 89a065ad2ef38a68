// Asynchronous sweep kernel with the residual snapshot in registers (FP32/BF16/FP8 storage,
// at most 40 rows per thread: m <= 20480 for FP32, 16384 for BF16 and FP8).
//
// The method step is the one of sweep_async.cuh (Algorithm 1, S.1-S.5; eq. 2 best
// response; the Section 4 surrogate), with the same division of rows among threads: thread
// t owns the 16-byte units u = k*512 + t of every column.  A thread therefore only ever
// reads its own rows of the stale residual r~, so the snapshot taken at the start of a
// block (S.2) is held in registers next to the block increment, and shared memory holds
// nothing but the ring of column chunks (13 stages of 16 KB instead of 9).  The deeper ring
// keeps more HBM reads in flight while the CTA is busy with the per-column reduction, the
// best response and the increment of the column before.  Measured on GB300 it streams A
// more slowly than the register-increment kernel of sweep_async.cuh (whose copy warp
// keeps the ring full without taking issue slots from the consumers), so it runs only when
// asked for (asyflexa_opts.variant = 3).
//
// There is no separate copy warp: the 16 warps are all consumers (so each thread may use
// 128 registers).  A ring slot is refilled by the warp that releases it last (elected with a
// shared-memory counter), right when it becomes free, with the chunk S positions further
// along the CTA's sequence of column chunks; that chunk is found by walking forward from the
// released one.  No warp ever waits for a refill it has to issue itself: chunk q is issued
// when chunk q - S (an earlier column, S > chunks per column) has been released by every
// warp, and every warp releases the chunks of a column before it reaches the next column.
#pragma once

#include "ptx.cuh"
#include "sweep.cuh"
#include "sweep_async.cuh"
#include "types.cuh"

namespace asyflexa {

constexpr int kRRThreads = kRegConsThreads;
constexpr int kRRMaxRowsPerThread = 40;

// The CTA's sequence of column chunks: for every sweep, its blocks b = blockIdx.x +
// i * gridDim.x in order, the columns of each block, the nch chunks of each column.
struct ChunkPos {
    int s, b, jl, c;
};

// Move `k` chunks forward.  Returns false if that runs past the last sweep.
__device__ __forceinline__ bool chunk_advance(const SweepParams& p, int nch, ChunkPos& q, int k) {
    int cc = q.c + k;
    int jl = q.jl + cc / nch;
    q.c = cc % nch;
    int b = q.b, s = q.s;
    int wb = static_cast<int>(min64(p.w, p.n - static_cast<int64_t>(b) * p.w));
    while (jl >= wb) {
        jl -= wb;
        b += gridDim.x;
        if (b >= p.nblocks) {
            b = blockIdx.x;
            if (++s >= p.sweeps) return false;
        }
        wb = static_cast<int>(min64(p.w, p.n - static_cast<int64_t>(b) * p.w));
    }
    q.s = s;
    q.b = b;
    q.jl = jl;
    return true;
}

// Issue the copy of chunk q into ring slot `slot` (completion counted on full[slot]).
template <typename TA>
__device__ __forceinline__ void issue_chunk(const SweepParams& p, int64_t units, const ChunkPos& q, uint32_t slot,
                                            unsigned char* ring, uint32_t stage_bytes, uint64_t* full,
                                            uint64_t pol) {
    constexpr int V = ATraits<TA>::kVec;
    const int64_t col = static_cast<int64_t>(q.b) * p.w + q.jl;
    const int64_t u0 = static_cast<int64_t>(q.c) * kRegStageUnits;
    const uint32_t nbytes = static_cast<uint32_t>(min64(kRegStageUnits, units - u0) * 16);
    const TA* src = static_cast<const TA*>(p.A) + col * p.lda + u0 * V;
    mbar_arrive_expect_tx(&full[slot], nbytes);
    bulk_load(ring + slot * stage_bytes, src, nbytes, &full[slot], pol);
}

template <typename TA, int CPC>
__global__ void __launch_bounds__(kRRThreads, 1) sweep_async_rr_kernel(const SweepParams p) {
    using TC = typename ATraits<TA>::TC;
    static_assert(sizeof(TC) == 4, "register kernel computes in FP32");
    using TX = typename XType<TA>::T;
    static_assert(sizeof(TX) == 4, "register kernel updates FP32 x");
    constexpr int V = ATraits<TA>::kVec;
    constexpr int UPT = kRegKpc * CPC;
    static_assert(UPT * V <= kRRMaxRowsPerThread, "too many rows per thread");

    extern __shared__ __align__(128) unsigned char smem[];
    const RegLayout L = make_reg_layout(0, p.stages);
    unsigned char* ring = smem + L.off_ring;
    float* colpart = reinterpret_cast<float*>(smem + L.off_colpart);
    ColCoef* coef = reinterpret_cast<ColCoef*>(smem + L.off_coef);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.off_bars);
    uint64_t* empty = full + p.stages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L.off_misc);
    int* relcnt = reinterpret_cast<int*>(smem + L.off_misc + 16);  // releases per slot (<= 16 slots)
    // 1 + parity of the use that the last copy issued into each slot fills (0: none yet)
    unsigned char* lastpar = smem + L.off_misc + 80;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int S = p.stages;
    const uint32_t stage_bytes = static_cast<uint32_t>(L.stage_bytes);
    const int64_t units = p.mcopy / V;
    const int64_t units_full = p.m / V;  // units whose rows are all < m
    const int nch = static_cast<int>((units + kRegStageUnits - 1) / kRegStageUnits);  // chunks per column
    const uint64_t pol = l2_policy_evict_first();  // A is streamed once per sweep

    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRegConsWarps);
            relcnt[k] = 0;
            lastpar[k] = 0;
        }
        *abort_flag = 0;
        fence_barrier_init();
        // first fill: chunks 0 .. S-1 of the sequence
        if (blockIdx.x < p.nblocks && p.sweeps > 0) {
            ChunkPos q{0, static_cast<int>(blockIdx.x), 0, 0};
            for (int k = 0; k < S; ++k) {
                issue_chunk<TA>(p, units, q, static_cast<uint32_t>(k), ring, stage_bytes, full, pol);
                lastpar[k] = 1;
                if (!chunk_advance(p, nch, q, 1)) break;
            }
        }
    }
    __syncthreads();

    uint32_t stage = 0, phase = 0;  // ring slot of the next chunk to consume and its use parity
    unsigned long long u_read = 0, my_updates = 0, my_active = 0;
    const float gamma = static_cast<float>(p.gamma);
    TX* x = static_cast<TX*>(p.x);
    const TX* lo = static_cast<const TX*>(p.lo);
    const TX* hi = static_cast<const TX*>(p.hi);
    const TX* lin = static_cast<const TX*>(p.lin);
    const float s_loss = static_cast<float>(p.s_loss);
    const float c2 = static_cast<float>(p.c2);

    float rr[UPT][V];   // this thread's rows of the stale residual r~ (S.2)
    float inc[UPT][V];  // this thread's rows of A_i Delta_i
    int buf = 0;

    for (int s = 0; s < p.sweeps; ++s) {
        for (int b = blockIdx.x; b < p.nblocks; b += gridDim.x) {
            const int64_t c0 = static_cast<int64_t>(b) * p.w;
            const int wb = static_cast<int>(min64(p.w, p.n - c0));
            if (tid == 0) u_read = ld_relaxed_u64(&p.counters[0]);
            // S.2: stale read of this thread's rows of r (rows >= m hold 0); all loads in flight
#pragma unroll
            for (int k = 0; k < UPT; ++k) {
                const int64_t u = static_cast<int64_t>(k) * kRRThreads + tid;
                const double2* src = reinterpret_cast<const double2*>(p.r + u * V);
#pragma unroll
                for (int e = 0; e < V; e += 2) {
                    const double2 d = u < units ? __ldcg(src + e / 2) : make_double2(0.0, 0.0);
                    rr[k][e] = static_cast<float>(d.x);
                    rr[k][e + 1] = static_cast<float>(d.y);
                }
            }
            // the block's per-column coefficients; the barrier that ended the previous block
            // guarantees nobody still reads coef
            if (tid < wb) {
                const int64_t j = c0 + tid;
                const double dj = p.dw[j];
                ColCoef cf;
                cf.x = static_cast<float>(x[j]);
                cf.lo = lo ? static_cast<float>(lo[j]) : -INFINITY;
                cf.hi = hi ? static_cast<float>(hi[j]) : INFINITY;
                cf.dinv = dj > 0.0 ? static_cast<float>(1.0 / dj) : 0.f;
                cf.thr = dj > 0.0 ? static_cast<float>(p.lam / dj) : 0.f;
                cf.scale = p.scale ? p.scale[j] : 1.f;
                cf.lin = lin ? static_cast<float>(lin[j]) : 0.f;
                cf.pad0 = 0.f;
                coef[tid] = cf;
            }
#pragma unroll
            for (int k = 0; k < UPT; ++k)
#pragma unroll
                for (int e = 0; e < V; ++e) inc[k][e] = 0.f;
            bool any = false;
            named_bar_sync(1, kRRThreads);

            for (int jl = 0; jl < wb; ++jl) {
                // ---- dot a_j^T r~ over this thread's rows
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
                uint32_t st_c = stage, ph_c = phase;
                bool ok = !*abort_flag;
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    if (c < nch) {
                        if (ok) ok = mbar_wait_bounded(&full[st_c], ph_c, abort_flag, p.err);
                        if (ok) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + st_c * stage_bytes);
#pragma unroll
                            for (int kk = 0; kk < kRegKpc; ++kk) {
                                const int k = c * kRegKpc + kk;
                                const int64_t u = static_cast<int64_t>(k) * kRRThreads + tid;
                                if (u < units) {
                                    float a[V];
                                    ATraits<TA>::unpack(src[kk * kRRThreads + tid], a);
                                    if (u < units_full) {
#pragma unroll
                                        for (int e = 0; e < V; e += 4) {
                                            acc0 = fmaf(a[e], rr[k][e], acc0);
                                            acc1 = fmaf(a[e + 1], rr[k][e + 1], acc1);
                                            acc2 = fmaf(a[e + 2], rr[k][e + 2], acc2);
                                            acc3 = fmaf(a[e + 3], rr[k][e + 3], acc3);
                                        }
                                    } else {
                                        const int valid = static_cast<int>(p.m - u * V);
#pragma unroll
                                        for (int e = 0; e < V; ++e)
                                            if (e < valid) acc0 = fmaf(a[e], rr[k][e], acc0);
                                    }
                                }
                            }
                        }
                        if (++st_c == static_cast<uint32_t>(S)) {
                            st_c = 0;
                            ph_c ^= 1u;
                        }
                    }
                }
                const float v = warp_sum((acc0 + acc1) + (acc2 + acc3));
                float* cp = colpart + buf * kRegConsWarps;
                if (lane == 0) cp[warp] = v;
                named_bar_sync(1, kRRThreads);
                // ---- best response (eq. 2) + fixed step (S.4): the same FP32 arithmetic in
                // every thread (fixed summation order), so all agree on Delta_j
                static_assert(kRegConsWarps <= 32, "one partial per lane");
                const float g = warp_sum(lane < kRegConsWarps ? cp[lane] : 0.f);
                buf ^= 1;
                const ColCoef cf = coef[jl];
                const float grad = s_loss * g * cf.scale - c2 * cf.x + cf.lin;
                float xh = 0.f;
                if (cf.dinv > 0.f) {
                    const float vv = fmaf(-grad, cf.dinv, cf.x);
                    const float av = fabsf(vv) - cf.thr;
                    xh = av > 0.f ? copysignf(av, vv) : 0.f;
                }
                xh = fminf(fmaxf(xh, cf.lo), cf.hi);
                const float xn = fmaf(gamma, xh - cf.x, cf.x);
                const float dlt = xn - cf.x;
                float dj = 0.f;
                if (!*abort_flag) {
                    if (tid == 0) x[c0 + jl] = static_cast<TX>(xn);
                    dj = dlt * cf.scale;
                    any |= dlt != 0.f;
                }
                // ---- fold a_j * Delta_j into the register increment, then release the chunks;
                // the last warp to release a slot refills it with the chunk S positions on
                st_c = stage;
                ph_c = phase;
#pragma unroll
                for (int c = 0; c < CPC; ++c) {
                    if (c < nch) {
                        if (dj != 0.f) {
                            const uint4* src = reinterpret_cast<const uint4*>(ring + st_c * stage_bytes);
#pragma unroll
                            for (int kk = 0; kk < kRegKpc; ++kk) {
                                const int k = c * kRegKpc + kk;
                                const int64_t u = static_cast<int64_t>(k) * kRRThreads + tid;
                                if (u < units) {
                                    float a[V];
                                    ATraits<TA>::unpack(src[kk * kRRThreads + tid], a);
#pragma unroll
                                    for (int e = 0; e < V; ++e) inc[k][e] = fmaf(a[e], dj, inc[k][e]);
                                }
                            }
                        }
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&empty[st_c]);
                            if (atomicAdd(&relcnt[st_c], 1) == kRegConsWarps - 1) {
                                relcnt[st_c] = 0;
                                // every warp has arrived: this use of the slot is over
                                ChunkPos q{s, b, jl, c};
                                if (!*abort_flag && mbar_wait_bounded(&empty[st_c], ph_c, abort_flag, p.err) &&
                                    chunk_advance(p, nch, q, S)) {
                                    issue_chunk<TA>(p, units, q, st_c, ring, stage_bytes, full, pol);
                                    lastpar[st_c] = static_cast<unsigned char>(1u + (ph_c ^ 1u));
                                }
                            }
                        }
                        if (++st_c == static_cast<uint32_t>(S)) {
                            st_c = 0;
                            ph_c ^= 1u;
                        }
                    }
                }
                stage = st_c;
                phase = ph_c;
            }
            // ---- r += A_i Delta_i : one FP64 atomic per row (skipping exact zeros)
            if (any && !*abort_flag) {
#pragma unroll
                for (int k = 0; k < UPT; ++k) {
                    const int64_t u = static_cast<int64_t>(k) * kRRThreads + tid;
                    if (u < units) {
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            const int64_t row = u * V + e;
                            if (row < p.m && inc[k][e] != 0.f) red_add_f64(p.r + row, static_cast<double>(inc[k][e]));
                        }
                    }
                }
                // one CTA runs its blocks strictly in order (cyclic Gauss-Seidel), so its next
                // read of r must see this scatter; with several CTAs a missed scatter is one
                // more update in flight (Assumption D1) and no fence is spent
                if (gridDim.x == 1) __threadfence();
            }
            named_bar_sync(1, kRRThreads);  // scatter issued; coef free
            if (tid == 0) {
                ++my_updates;
                if (any) ++my_active;
                const unsigned long long u1 = atomicAdd(&p.counters[0], 1ull);
                const unsigned long long dly = u1 - u_read;
                int bucket = 63 - __clzll(static_cast<long long>(dly + 1ull));
                bucket = bucket > 31 ? 31 : bucket;
                atomicAdd(&p.hist[bucket], 1ull);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (*abort_flag) {
            // copies still in flight must land before the CTA exits (bounded): wait for the
            // phase that each slot's most recent copy completes
            for (int k = 0; k < S; ++k) {
                if (!lastpar[k]) continue;
                const uint32_t par = lastpar[k] - 1u;
                const uint64_t t0 = global_timer_ns();
                while (!mbar_try_wait(&full[k], par)) {
                    if (global_timer_ns() - t0 > kWaitLimitNs) break;
                }
            }
        }
        atomicAdd(&p.counters[1], my_updates);
        atomicAdd(&p.counters[2], my_active);
    }
}

}  // namespace asyflexa
