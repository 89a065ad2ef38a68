// Multi-right-hand-side asynchronous sweep: k problems ("lanes") that share the matrix A and
// differ in b and lambda (a lambda path, or several data vectors), LASSO loss, FP32 A.
//
// The block update of Algorithm 1 for every lane at once: for block i the lanes' gradients are
// the dense product G = A_i^T R~ (w x k, R~ the lanes' stale residuals, S.2), the best
// responses and fixed steps are elementwise (eq. 2, S.4), and the scatter is the dense product
// R += A_i Delta_i (m x k).  With k lanes every byte of A serves k products, so both products
// run on the tensor cores (mma.sync m16n8k8, TF32).  TF32 keeps 10 bits of mantissa, so every
// operand is split x = hi + lo (both TF32) and a*b is formed as hi*hi + hi*lo + lo*hi with FP32
// accumulation: the error of the dropped lo*lo term is about 2^-22 relative, FP32-grade.
//
// Layout: A column-major (column j = A + j*lda), R FP64 row-major m x kp (row i holds the kp
// lanes' residuals), X FP32 row-major n x kp, kp = lanes padded to a multiple of 8 (padding
// lanes have lambda = +inf, stay at 0 and get zero steps).  Each CTA owns the blocks b = cta,
// cta + grid, ... (Assumption D4) and streams its block in row tiles of kMT rows twice:
// gradient pass (row tiles of A and R~ through shared memory, G accumulated in registers) and,
// after the elementwise step, the scatter pass (the same A tiles, now mostly L2 hits, times
// Delta, added to R with FP64 atomics).
#pragma once

#include "convert.cuh"
#include "ptx.cuh"
#include "sweep.cuh"
#include "types.cuh"

namespace asyflexa {

constexpr int kMW = 32;               // block width (columns)
constexpr int kMT = 64;               // rows per tile
constexpr int kMThreads = 256;        // 8 warps
constexpr int kMWarps = kMThreads / 32;
constexpr int kMAR = kMW * kMT / kMThreads;  // rows of an A tile column per thread
constexpr int kMKMax = 64;            // lanes (padded) per launch
constexpr int kMAS = kMT + 4;         // A tile stride (floats): conflict-free fragment loads
constexpr int kMRS = kMKMax + 8;      // R tile / Delta stride (floats)

struct MultiParams {
    const float* A;
    int64_t lda, m, n;
    double* R;            // m x kp (row-major), FP64
    float* X;             // n x kp (row-major)
    const double* dw;     // n surrogate weights (shared by the lanes)
    const double* lam;    // kp (padding lanes: +inf)
    const float* dinv;    // n: 1/d_j rounded to FP32 (0 where d_j <= 0)
    const float* thr;     // n x kp: lam_l / d_j rounded to FP32 (0 where d_j <= 0)
    double gamma;
    int kp, nblocks, sweeps;
    int mode;             // 0: sweep; 1: refresh (R += A X, no step); 2: gradient only (G out)
    float* G;             // mode 2: n x kp gradients A^T R
    unsigned long long* counters;  // [0] update counter, [1] block updates
    unsigned long long* hist;      // staleness histogram
};

struct MultiSmem {
    float a_hi[kMW * kMAS], a_lo[kMW * kMAS];   // A tile, column-major (j * kMAS + t)
    float r_hi[kMT * kMRS], r_lo[kMT * kMRS];   // R~ tile, row-major (t * kMRS + lane)
    float g[kMW * kMRS];                        // G (j * kMRS + lane)
    float d_hi[kMW * kMRS], d_lo[kMW * kMRS];   // Delta (j * kMRS + lane)
};

// TwoSum (Knuth): s + e == a + b exactly, s = fl(a + b).  Accumulates the per-tile FP32 sums
// in a float-float pair (hi, lo) with about 44 significant bits, on the FP32 pipe.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    const uint32_t h = to_tf32(x);
    hi = __uint_as_float(h);
    lo = __uint_as_float(to_tf32(x - hi));
}

// D += A (16x8, row) * B (8x8, col), TF32 in, FP32 accumulate.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(__float_as_uint(a[0])), "r"(__float_as_uint(a[1])), "r"(__float_as_uint(a[2])),
          "r"(__float_as_uint(a[3])), "r"(__float_as_uint(b[0])), "r"(__float_as_uint(b[1])));
}

// The A tile rows [row0, row0 + kMT) of columns c0 .. c0 + wb - 1 (zeros elsewhere): thread t
// holds kMAR consecutive rows of column t / (kMT / kMAR).  fetch loads them into registers (the
// next tile's loads overlap the current tile's MMAs); store splits them into TF32 hi / lo in
// shared memory.
__device__ __forceinline__ void fetch_a_tile(const MultiParams& p, int64_t c0, int wb, int64_t row0,
                                             float (&v)[kMAR]) {
    const int j = threadIdx.x / (kMT / kMAR);
    const int t0 = (threadIdx.x % (kMT / kMAR)) * kMAR;
#pragma unroll
    for (int e = 0; e < kMAR; ++e) {
        const int64_t row = row0 + t0 + e;
        v[e] = (j < wb && row < p.m) ? __ldg(p.A + (c0 + j) * p.lda + row) : 0.f;
    }
}

__device__ __forceinline__ void store_a_tile(MultiSmem& s, const float (&v)[kMAR]) {
    const int j = threadIdx.x / (kMT / kMAR);
    const int t0 = (threadIdx.x % (kMT / kMAR)) * kMAR;
#pragma unroll
    for (int e = 0; e < kMAR; ++e) {
        float hi, lo;
        split_tf32(v[e], hi, lo);
        s.a_hi[j * kMAS + t0 + e] = hi;
        s.a_lo[j * kMAS + t0 + e] = lo;
    }
}

// The lanes' residual tile R~[row0 .. row0 + kMT) x KP: element i = tid + kMThreads * q.
template <int KP>
__device__ __forceinline__ void fetch_r_tile(const MultiParams& p, int64_t row0, float (&v)[kMT * KP / kMThreads]) {
#pragma unroll
    for (int q = 0; q < kMT * KP / kMThreads; ++q) {
        const int i = threadIdx.x + kMThreads * q;
        const int64_t row = row0 + i / KP;
        v[q] = row < p.m ? static_cast<float>(__ldcg(p.R + row * KP + i % KP)) : 0.f;
    }
}

template <int KP>
__device__ __forceinline__ void store_r_tile(MultiSmem& s, const float (&v)[kMT * KP / kMThreads]) {
#pragma unroll
    for (int q = 0; q < kMT * KP / kMThreads; ++q) {
        const int i = threadIdx.x + kMThreads * q;
        float hi, lo;
        split_tf32(v[q], hi, lo);
        s.r_hi[(i / KP) * kMRS + i % KP] = hi;
        s.r_lo[(i / KP) * kMRS + i % KP] = lo;
    }
}

template <int KP>
__global__ void __launch_bounds__(kMThreads) sweep_multi_kernel(const MultiParams p) {
    static_assert(KP % 8 == 0 && KP <= kMKMax, "lanes padded to a multiple of 8");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MultiSmem& s = *reinterpret_cast<MultiSmem*>(smem_raw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int grp = lane >> 2;  // groupID of the mma fragments
    const int tig = lane & 3;   // thread in group
    constexpr int kNT = KP / 8;                 // n tiles (lanes)
    constexpr int kP1 = (kMW / 16) * kNT;       // gradient pass: (m tile, n tile) pairs over j
    constexpr int kP1W = (kP1 + kMWarps - 1) / kMWarps;  // pairs per warp
    constexpr int kP2 = (kMT / 16) * kNT;       // scatter pass: pairs over rows
    constexpr int kP2W = (kP2 + kMWarps - 1) / kMWarps;
    __shared__ int s_any;
    __shared__ unsigned long long s_uread;

    for (int sw = 0; sw < p.sweeps; ++sw) {
        for (int b = blockIdx.x; b < p.nblocks; b += gridDim.x) {
            const int64_t c0 = static_cast<int64_t>(b) * kMW;
            const int wb = static_cast<int>(min64(kMW, p.n - c0));
            if (tid == 0) s_uread = ld_relaxed_u64(&p.counters[0]);
            // ---- gradient pass: G = A_i^T R~ (S.2: R~ is read tile by tile, a stale read)
            // per row tile FP32 accumulators (tensor cores; the three split products in separate
            // chains), summed over the tiles in float-float, so the FP32 rounding of G grows with
            // the tile (kMT rows), not with m
            float acc_hi[kP1W][4], acc_lo[kP1W][4];
#pragma unroll
            for (int q = 0; q < kP1W; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc_hi[q][e] = acc_lo[q][e] = 0.f;
            if (p.mode != 1) {
                float av[kMAR], rv[kMT * KP / kMThreads];
                fetch_a_tile(p, c0, wb, 0, av);
                fetch_r_tile<KP>(p, 0, rv);
                for (int64_t row0 = 0; row0 < p.m; row0 += kMT) {
                    __syncthreads();  // previous tile consumed
                    store_a_tile(s, av);
                    store_r_tile<KP>(s, rv);
                    if (row0 + kMT < p.m) {  // next tile's loads in flight during this tile's MMAs
                        fetch_a_tile(p, c0, wb, row0 + kMT, av);
                        fetch_r_tile<KP>(p, row0 + kMT, rv);
                    }
                    __syncthreads();
#pragma unroll
                    for (int q = 0; q < kP1W; ++q) {
                        const int pr = warp + kMWarps * q;
                        if (pr < kP1) {
                            const int mt = pr / kNT, nt = pr % kNT;
                            const int j0 = mt * 16 + grp;
                            float t_ab[4] = {0.f, 0.f, 0.f, 0.f}, t_ba[4] = {0.f, 0.f, 0.f, 0.f},
                                  t_hh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
                            for (int k0 = 0; k0 < kMT; k0 += 8) {
                                float ah[4], al[4], bh[2], bl[2];
                                ah[0] = s.a_hi[j0 * kMAS + k0 + tig];
                                ah[1] = s.a_hi[(j0 + 8) * kMAS + k0 + tig];
                                ah[2] = s.a_hi[j0 * kMAS + k0 + tig + 4];
                                ah[3] = s.a_hi[(j0 + 8) * kMAS + k0 + tig + 4];
                                al[0] = s.a_lo[j0 * kMAS + k0 + tig];
                                al[1] = s.a_lo[(j0 + 8) * kMAS + k0 + tig];
                                al[2] = s.a_lo[j0 * kMAS + k0 + tig + 4];
                                al[3] = s.a_lo[(j0 + 8) * kMAS + k0 + tig + 4];
                                bh[0] = s.r_hi[(k0 + tig) * kMRS + nt * 8 + grp];
                                bh[1] = s.r_hi[(k0 + tig + 4) * kMRS + nt * 8 + grp];
                                bl[0] = s.r_lo[(k0 + tig) * kMRS + nt * 8 + grp];
                                bl[1] = s.r_lo[(k0 + tig + 4) * kMRS + nt * 8 + grp];
                                mma_tf32(t_ab, al, bh);
                                mma_tf32(t_ba, ah, bl);
                                mma_tf32(t_hh, ah, bh);
                            }
#pragma unroll
                            for (int e = 0; e < 4; ++e) two_sum_acc(acc_hi[q][e], acc_lo[q][e], t_hh[e] + (t_ab[e] + t_ba[e]));
                        }
                    }
                }
            }
            __syncthreads();
            // G to shared memory (fragment rows = columns j, fragment columns = lanes)
#pragma unroll
            for (int q = 0; q < kP1W; ++q) {
                const int pr = warp + kMWarps * q;
                if (pr < kP1) {
                    const int mt = pr / kNT, nt = pr % kNT;
                    const int j0 = mt * 16 + grp, l0 = nt * 8 + 2 * tig;
                    s.g[j0 * kMRS + l0] = acc_hi[q][0] + acc_lo[q][0];
                    s.g[j0 * kMRS + l0 + 1] = acc_hi[q][1] + acc_lo[q][1];
                    s.g[(j0 + 8) * kMRS + l0] = acc_hi[q][2] + acc_lo[q][2];
                    s.g[(j0 + 8) * kMRS + l0 + 1] = acc_hi[q][3] + acc_lo[q][3];
                }
            }
            if (tid == 0) s_any = 0;
            __syncthreads();
            // ---- elementwise: best response (eq. 2) + fixed step (S.4) per (column, lane); in
            // refresh mode Delta = x (R += A X), in gradient mode G is written out
            int any = 0;
            for (int i = tid; i < kMW * KP; i += kMThreads) {
                const int j = i / KP, l = i % KP;
                float dlt = 0.f;
                if (j < wb) {
                    const int64_t jj = c0 + j;
                    if (p.mode == 1) {
                        dlt = p.X[jj * KP + l];
                    } else if (p.mode == 2) {
                        p.G[jj * KP + l] = s.g[j * kMRS + l];
                    } else {
                        // the FP32 coefficients 1/d_j and lam_l/d_j come from tables made once per
                        // handle (FP64 divisions are slow on GB300's narrow FP64 pipe)
                        const float dinv = p.dinv[jj];
                        const float x = p.X[jj * KP + l];
                        float xh = 0.f;
                        if (dinv > 0.f) {
                            const float thr = p.thr[jj * KP + l];  // +inf for padding lanes
                            const float v = fmaf(-s.g[j * kMRS + l], dinv, x);
                            const float av = fabsf(v) - thr;
                            xh = av > 0.f ? copysignf(av, v) : 0.f;
                        }
                        const float xn = fmaf(static_cast<float>(p.gamma), xh - x, x);
                        dlt = xn - x;
                        if (dlt != 0.f) p.X[jj * KP + l] = xn;
                    }
                }
                float hi, lo;
                split_tf32(dlt, hi, lo);
                s.d_hi[j * kMRS + l] = hi;
                s.d_lo[j * kMRS + l] = lo;
                any |= dlt != 0.f;
            }
            if (any) s_any = 1;
            __syncthreads();
            // ---- scatter pass: R += A_i Delta (FP64 atomics; rows >= m skipped)
            if (s_any && p.mode != 2) {
                float av[kMAR];
                fetch_a_tile(p, c0, wb, 0, av);
                for (int64_t row0 = 0; row0 < p.m; row0 += kMT) {
                    store_a_tile(s, av);
                    __syncthreads();
                    if (row0 + kMT < p.m) fetch_a_tile(p, c0, wb, row0 + kMT, av);
#pragma unroll
                    for (int q = 0; q < kP2W; ++q) {
                        const int pr = warp + kMWarps * q;
                        if (pr < kP2) {
                            const int mt = pr / kNT, nt = pr % kNT;
                            const int t0 = mt * 16 + grp;
                            float c_ab[4] = {0.f, 0.f, 0.f, 0.f}, c_ba[4] = {0.f, 0.f, 0.f, 0.f},
                                  c_hh[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                            for (int k0 = 0; k0 < kMW; k0 += 8) {
                                float ah[4], al[4], bh[2], bl[2];
                                // A operand (rows t, columns j) = A tile transposed
                                ah[0] = s.a_hi[(k0 + tig) * kMAS + t0];
                                ah[1] = s.a_hi[(k0 + tig) * kMAS + t0 + 8];
                                ah[2] = s.a_hi[(k0 + tig + 4) * kMAS + t0];
                                ah[3] = s.a_hi[(k0 + tig + 4) * kMAS + t0 + 8];
                                al[0] = s.a_lo[(k0 + tig) * kMAS + t0];
                                al[1] = s.a_lo[(k0 + tig) * kMAS + t0 + 8];
                                al[2] = s.a_lo[(k0 + tig + 4) * kMAS + t0];
                                al[3] = s.a_lo[(k0 + tig + 4) * kMAS + t0 + 8];
                                bh[0] = s.d_hi[(k0 + tig) * kMRS + nt * 8 + grp];
                                bh[1] = s.d_hi[(k0 + tig + 4) * kMRS + nt * 8 + grp];
                                bl[0] = s.d_lo[(k0 + tig) * kMRS + nt * 8 + grp];
                                bl[1] = s.d_lo[(k0 + tig + 4) * kMRS + nt * 8 + grp];
                                mma_tf32(c_ab, al, bh);
                                mma_tf32(c_ba, ah, bl);
                                mma_tf32(c_hh, ah, bh);
                            }
                            float c[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) c[e] = c_hh[e] + (c_ab[e] + c_ba[e]);
                            const int l0 = nt * 8 + 2 * tig;
                            const int64_t r0 = row0 + t0, r1 = row0 + t0 + 8;
                            if (r0 < p.m) {
                                if (c[0] != 0.f) red_add_f64(p.R + r0 * KP + l0, static_cast<double>(c[0]));
                                if (c[1] != 0.f) red_add_f64(p.R + r0 * KP + l0 + 1, static_cast<double>(c[1]));
                            }
                            if (r1 < p.m) {
                                if (c[2] != 0.f) red_add_f64(p.R + r1 * KP + l0, static_cast<double>(c[2]));
                                if (c[3] != 0.f) red_add_f64(p.R + r1 * KP + l0 + 1, static_cast<double>(c[3]));
                            }
                        }
                    }
                    __syncthreads();  // tile consumed before the next load
                }
                // a single CTA runs its blocks in order (cyclic Gauss-Seidel per lane): its next
                // read of R must see this scatter
                if (gridDim.x == 1) __threadfence();
            }
            __syncthreads();
            if (tid == 0 && p.mode == 0) {
                const unsigned long long u1 = atomicAdd(&p.counters[0], 1ull);
                const unsigned long long dly = u1 - s_uread;
                int bucket = 63 - __clzll(static_cast<long long>(dly + 1ull));
                bucket = bucket > 31 ? 31 : bucket;
                atomicAdd(&p.hist[bucket], 1ull);
                atomicAdd(&p.counters[1], 1ull);
            }
        }
    }
}

// The elementwise step's FP32 coefficients: dinv[j] = 1/d_j and thr[j KP + l] = lam_l / d_j,
// each the FP64 quotient rounded to FP32 (0 where d_j <= 0).
template <int KP>
__global__ void multi_coef_kernel(const double* dw, const double* lam, int64_t n, float* dinv, float* thr) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n * KP;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t j = i / KP;
        const int l = static_cast<int>(i % KP);
        const double d = dw[j];
        thr[i] = d > 0.0 ? static_cast<float>(lam[l] / d) : 0.f;
        if (l == 0) dinv[j] = d > 0.0 ? static_cast<float>(1.0 / d) : 0.f;
    }
}

// Per-lane objective pieces: out[l] += sum_i R[i][l]^2 (first KP entries), out[KP + l] +=
// sum_j |X[j][l]| and out[2 KP + l] += nnz of lane l, FP64 atomics.  The grid stride is a
// multiple of KP (256 threads, KP in {8, 16, 32, 64}), so each thread stays on one lane.
template <int KP>
__global__ void __launch_bounds__(256) multi_norms_kernel(const double* R, int64_t m, const float* X, int64_t n,
                                                          double* out) {
    static_assert(256 % KP == 0, "one lane per thread");
    __shared__ double sh[3 * KP];
    for (int l = threadIdx.x; l < 3 * KP; l += blockDim.x) sh[l] = 0.0;
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int l = threadIdx.x % KP;
    double rr = 0.0, ax = 0.0, nz = 0.0;
    for (int64_t e = t0; e < m * KP; e += stride) rr = fma(R[e], R[e], rr);
    for (int64_t e = t0; e < n * KP; e += stride) {
        const double v = static_cast<double>(X[e]);
        ax += fabs(v);
        nz += v != 0.0 ? 1.0 : 0.0;
    }
    atomicAdd(&sh[l], rr);
    atomicAdd(&sh[KP + l], ax);
    atomicAdd(&sh[2 * KP + l], nz);
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * KP; i += blockDim.x) atomicAdd(&out[i], sh[i]);
}

// Layout changes between the caller's per-lane vectors (lane l at src + l * lds, length len)
// and the row-major len x KP array; lanes >= k are zero.  dir 0: lanes -> rows; 1: back.
template <typename TS, typename TD>
__global__ void __launch_bounds__(256) multi_transpose_kernel(const TS* src, int64_t lds, TD* dst, int64_t ldd,
                                                              int64_t len, int k, int kp, int dir, double scale) {
    const int64_t total = len * kp;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = e / kp;
        const int l = static_cast<int>(e % kp);
        if (dir == 0) {
            dst[e] = l < k ? static_cast<TD>(scale * static_cast<double>(src[l * lds + i])) : TD(0);
        } else if (l < k) {
            dst[l * ldd + i] = static_cast<TD>(src[e]);
        }
    }
}

// Per-lane stationarity: out[l] = max_j |xhat_j - x_j| (FP64 bits, atomic max) and
// out[kp + l] = max_j |x_j|, from the gradients G = A^T R (gradient pass, mode 2).
template <int KP>
__global__ void __launch_bounds__(256) multi_stat_kernel(const float* G, const float* X, const double* dw,
                                                         const double* lam, int64_t n, unsigned long long* out) {
    const int64_t total = n * KP;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t j = i / KP;
        const int l = static_cast<int>(i % KP);
        const double x = X[i], d = dw[j], g = G[i];
        double xh = 0.0;
        if (d > 0.0) {
            const double v = x - g / d;
            const double av = fabs(v) - lam[l] / d;
            xh = av > 0.0 ? copysign(av, v) : 0.0;
        }
        const double dx = fabs(xh - x), ax = fabs(x);
        if (dx > 0.0) atomicMax(&out[l], static_cast<unsigned long long>(__double_as_longlong(dx)));
        if (ax > 0.0) atomicMax(&out[KP + l], static_cast<unsigned long long>(__double_as_longlong(ax)));
    }
}


// ---------------------------------------------------------------------------------------
// Exact checks of all lanes at once (CUDA cores, error-free FP32 products and sums: Dot2 of
// Ogita, Rump and Oishi), as accurate as FP64 accumulation: the multi-lane sweeps' split-TF32
// products are FP32-grade, which puts their stationarity measure up to ~1e-6 off.
// ---------------------------------------------------------------------------------------

constexpr int kXT = 32;  // rows (residual) or columns (gradient) per CTA of the exact checks

// R = A X - B for every lane: a CTA owns kXT rows and every lane (thread t: row t mod 32, lanes
// t/32 + 8 q); the columns whose lanes are all zero are skipped.  B: the caller's k x ldb data
// vectors (lanes >= k: 0).  R: m x KP, FP64; Rhl: the same as FP32 (hi, lo) pairs, R = hi + lo
// to about 2^-48 relative, for the gradient kernel.
template <int KP>
__global__ void __launch_bounds__(256) multi_exact_residual_kernel(const float* A, int64_t lda, int64_t m, int64_t n,
                                                                   const float* X, const float* B, int64_t ldb, int k,
                                                                   double* R, float2* Rhl) {
    constexpr int LPT = KP / 8;  // lanes per thread
    __shared__ float sA[kXT][kXT + 1];   // [column][row]
    __shared__ float sX[kXT][KP];        // [column][lane]
    __shared__ int sNz[kXT];
    const int tid = threadIdx.x;
    const int rl = tid & 31, lg = tid >> 5;
    const int64_t row0 = static_cast<int64_t>(blockIdx.x) * kXT;
    DFAcc acc[LPT];
    for (int64_t j0 = 0; j0 < n; j0 += kXT) {
        __syncthreads();  // previous chunk consumed
        for (int i = tid; i < kXT * KP; i += 256) {
            const int jc = i / KP, l = i % KP;
            sX[jc][l] = j0 + jc < n ? X[(j0 + jc) * KP + l] : 0.f;
        }
        for (int i = tid; i < kXT * kXT; i += 256) {
            const int jc = i / kXT, r = i % kXT;
            sA[jc][r] = (j0 + jc < n && row0 + r < m) ? A[(j0 + jc) * lda + row0 + r] : 0.f;
        }
        __syncthreads();
        if (tid < kXT) {
            int nz = 0;
            for (int l = 0; l < KP; ++l) nz |= sX[tid][l] != 0.f;
            sNz[tid] = nz;
        }
        __syncthreads();
        for (int jc = 0; jc < kXT; ++jc) {
            if (!sNz[jc]) continue;
            const float a = sA[jc][rl];
#pragma unroll
            for (int q = 0; q < LPT; ++q) acc[q].add_prod(a, sX[jc][lg + 8 * q]);
        }
    }
    const int64_t row = row0 + rl;
    if (row < m) {
#pragma unroll
        for (int q = 0; q < LPT; ++q) {
            const int l = lg + 8 * q;
            const double b = l < k ? static_cast<double>(B[static_cast<int64_t>(l) * ldb + row]) : 0.0;
            const double v = acc[q].value() - b;
            const float h = f64_to_f32(v);
            R[row * KP + l] = v;
            Rhl[row * KP + l] = make_float2(h, f64_to_f32(v - f32_to_f64(h)));
        }
    }
}

// G = A^T R for every lane: a CTA owns kXT columns (thread t: column t mod 32, lanes t/32 + 8 q)
// and walks the rows in tiles of 64, with R as its FP32 (hi, lo) pairs (a r = a r_hi + a r_lo,
// the first product error-free).  G: n x KP, FP64.
template <int KP>
__global__ void __launch_bounds__(256) multi_exact_grad_kernel(const float* A, int64_t lda, int64_t m, int64_t n,
                                                               const float2* Rhl, double* G) {
    constexpr int LPT = KP / 8;
    constexpr int RT = 64;
    __shared__ float sA[kXT][RT + 1];    // [column][row]
    __shared__ float sRh[RT][KP], sRl[RT][KP];
    const int tid = threadIdx.x;
    const int cl = tid & 31, lg = tid >> 5;
    const int64_t j0 = static_cast<int64_t>(blockIdx.x) * kXT;
    DFAcc acc[LPT];
    float lo_acc[LPT];
#pragma unroll
    for (int q = 0; q < LPT; ++q) lo_acc[q] = 0.f;
    for (int64_t r0 = 0; r0 < m; r0 += RT) {
        __syncthreads();
        for (int i = tid; i < kXT * RT; i += 256) {
            const int jc = i / RT, r = i % RT;
            sA[jc][r] = (j0 + jc < n && r0 + r < m) ? A[(j0 + jc) * lda + r0 + r] : 0.f;
        }
        for (int i = tid; i < RT * KP; i += 256) {
            const int r = i / KP, l = i % KP;
            const float2 v = r0 + r < m ? Rhl[(r0 + r) * KP + l] : make_float2(0.f, 0.f);
            sRh[r][l] = v.x;
            sRl[r][l] = v.y;
        }
        __syncthreads();
        for (int r = 0; r < RT; ++r) {
            const float a = sA[cl][r];
#pragma unroll
            for (int q = 0; q < LPT; ++q) {
                acc[q].add_prod(a, sRh[r][lg + 8 * q]);
                lo_acc[q] = fmaf(a, sRl[r][lg + 8 * q], lo_acc[q]);
            }
        }
    }
    const int64_t j = j0 + cl;
    if (j < n) {
#pragma unroll
        for (int q = 0; q < LPT; ++q) G[j * KP + lg + 8 * q] = acc[q].value() + static_cast<double>(lo_acc[q]);
    }
}

// Per-lane ||xhat(x) - x||_inf and ||x||_inf from FP64 gradients (same as multi_stat_kernel).
template <int KP>
__global__ void __launch_bounds__(256) multi_stat64_kernel(const double* G, const float* X, const double* dw,
                                                           const double* lam, int64_t n, unsigned long long* out) {
    const int64_t total = n * KP;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t j = i / KP;
        const int l = static_cast<int>(i % KP);
        const double x = X[i], d = dw[j], g = G[i];
        double xh = 0.0;
        if (d > 0.0) {
            const double v = x - g / d;
            const double av = fabs(v) - lam[l] / d;
            xh = av > 0.0 ? copysign(av, v) : 0.0;
        }
        const double dx = fabs(xh - x), ax = fabs(x);
        if (dx > 0.0) atomicMax(&out[l], static_cast<unsigned long long>(__double_as_longlong(dx)));
        if (ax > 0.0) atomicMax(&out[KP + l], static_cast<unsigned long long>(__double_as_longlong(ax)));
    }
}

}  // namespace asyflexa
