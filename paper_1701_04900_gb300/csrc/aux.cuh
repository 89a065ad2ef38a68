// Auxiliary kernels around the sweep:
//   * colnorm_kernel      surrogate weights d_j = (1+tau_rel) kappa_j + tau   (create time)
//   * count/compact       deterministic ordered list of the nonzero entries of a vector
//   * gather_gemv_pipe_kernel  partial[seg] = sum_{k in seg} a_{j_k} v_k  (fixed segmentation;
//                         compensated products for the exact refresh, plain ones for the
//                         Jacobi scatter); gather_gemv_exact_kernel is the register-batched
//                         form kept for the no-allocation residual
//   * reduce_partials     r = r + sum_seg partial  (Jacobi scatter)  or
//                         r = sum_seg partial - b  (exact residual refresh, FP64 accumulation)
//   * norms / finalize    ||r||^2, ||x||_1, ||x||^2, nnz with fixed-order reductions
//   * check_kernel        full gradient with compensated (error-free transformation)
//                         FP32 products, and the optimality measures of x
// Every reduction here has a fixed order for a fixed launch shape, so results are
// bit-reproducible run to run.
#pragma once

#include <type_traits>

#include "ptx.cuh"
#include "types.cuh"

namespace asyflexa {

constexpr int kAuxThreads = 256;
constexpr int kCompactPerThread = 16;
constexpr int kCompactTile = kAuxThreads * kCompactPerThread;
constexpr int kGemvUnits = 2;     // 16-byte units of A per thread in gather_gemv_exact
constexpr int kPipeStages = 6;    // list entries (columns) in flight per thread in gather_gemv_pipe
constexpr int kPipeElems = 16;    // elements of A per thread per column in gather_gemv_pipe
constexpr int kNormsGrid = 256;
constexpr int kCheckThreads = 1024;

template <typename T>
__device__ __forceinline__ T block_sum_256(T v, T* sh /* >= 8 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[w] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < kAuxThreads / 32; ++k) s += sh[k];
    }
    __syncthreads();
    return s;  // valid in thread 0
}

// ----------------------------------------------------------------------------- weights

// Accumulator of sums of products: FP64 FMAs for FP64 storage, the double-FP32 pair for
// FP32-widened storage.
template <typename TC>
struct ProdAcc;
template <>
struct ProdAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct ProdAcc<float> : DFAcc {};

// One warp per column: kappa_j = s_loss * ||a_j||^2 * scale_j^2 - c2, with the squares
// accumulated exactly (ProdAcc) and combined across lanes in FP64.
template <typename TA>
__global__ void colnorm_kernel(const TA* A, int64_t lda, int64_t m, int64_t n, const float* scale, double s_loss,
                               double c2, double tau, double tau_rel, double* dw, int* neg_flag) {
    using TC = typename ATraits<TA>::TC;
    constexpr int V = ATraits<TA>::kVec;
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw) {
        const TA* col = A + j * lda;
        ProdAcc<TC> pa;
        const int64_t units = (m + V - 1) / V;
        for (int64_t u = lane; u < units; u += 32) {
            const uint4 q = ld_stream_u4(col + u * V);
            TC a[V];
            ATraits<TA>::unpack(q, a);
#pragma unroll
            for (int e = 0; e < V; ++e)
                if (u * V + e < m) pa.add_prod(a[e], a[e]);
        }
        double acc = pa.value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double sc = scale ? static_cast<double>(scale[j]) : 1.0;
            const double kappa = s_loss * acc * sc * sc - c2;
            const double d = (1.0 + tau_rel) * kappa + tau;
            dw[j] = d;
            if (!(d >= 0.0)) atomicOr(neg_flag, 1);
        }
    }
}

// ----------------------------------------------------------------------------- compaction

template <typename TV>
__global__ void count_nonzero_kernel(const TV* v, int64_t n, int* tilecnt) {
    __shared__ int sh[kAuxThreads / 32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kCompactTile + static_cast<int64_t>(threadIdx.x) * kCompactPerThread;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kCompactPerThread; ++k) {
        const int64_t i = base + k;
        if (i < n && v[i] != TV(0)) ++c;
    }
    const int s = block_sum_256<int>(c, sh);
    if (threadIdx.x == 0) tilecnt[blockIdx.x] = s;
}

// Writes (index, value) of the nonzeros in increasing index order; count -> *count.
template <typename TV>
__global__ void compact_kernel(const TV* v, int64_t n, const int* tilecnt, int ntiles, int* idx, TV* val,
                               int* count) {
    __shared__ int sh[kAuxThreads / 32];
    __shared__ int s_off;
    __shared__ int s_warp[kAuxThreads / 32];
    // offset of this tile = sum of earlier tile counts (fixed order)
    int part = 0;
    for (int t = threadIdx.x; t < blockIdx.x; t += kAuxThreads) part += tilecnt[t];
    const int off = block_sum_256<int>(part, sh);
    if (threadIdx.x == 0) s_off = off;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kCompactTile + static_cast<int64_t>(threadIdx.x) * kCompactPerThread;
    int c = 0;
#pragma unroll
    for (int k = 0; k < kCompactPerThread; ++k) {
        const int64_t i = base + k;
        if (i < n && v[i] != TV(0)) ++c;
    }
    // exclusive scan of c over the block
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    int wofs = 0;
    for (int k = 0; k < w; ++k) wofs += s_warp[k];
    int pos = s_off + wofs + incl - c;
#pragma unroll
    for (int k = 0; k < kCompactPerThread; ++k) {
        const int64_t i = base + k;
        if (i < n) {
            const TV x = v[i];
            if (x != TV(0)) {
                idx[pos] = static_cast<int>(i);
                val[pos] = x;
                ++pos;
            }
        }
    }
    if (blockIdx.x == ntiles - 1 && threadIdx.x == kAuxThreads - 1) *count = pos;
}

// ----------------------------------------------------------------------------- gather GEMV

// grid = (row tiles of kAuxThreads * kPipeElems rows, nseg); dynamic shared memory
// kPipeStages * kAuxThreads * kPipeElems * sizeof(TA) bytes.
// partial[seg * mcopy + row] = sum over the seg-th slice of the list of
// a_{idx[k]}[row] * val[k] * scale[idx[k]], accumulated in list order: with compensated
// (error-free) FP32 products and an FP64 result when kExact (the exact residual), else in the
// compute type TC (the Jacobi scatter).  Each thread streams its own 16-byte units of the next
// kPipeStages - 1 columns into a shared-memory ring with cp.async while it accumulates the
// current one, and reads back only what it copied itself, so no barrier is needed.
template <typename TA, typename TV, bool kExact>
__global__ void __launch_bounds__(kAuxThreads) gather_gemv_pipe_kernel(const TA* A, int64_t lda, int64_t mcopy,
                                                                       const float* scale, const int* idx,
                                                                       const TV* val, const int* count,
                                                                       void* partial_out) {
    using TC = typename ATraits<TA>::TC;
    using TP = typename std::conditional<kExact, double, TC>::type;
    constexpr int V = ATraits<TA>::kVec;
    constexpr int U = kPipeElems / V;  // 16-byte units per thread per column
    static_assert(U >= 1 && U * V == kPipeElems, "whole units per thread");
    extern __shared__ __align__(16) uint4 ring[];  // [stage][U][kAuxThreads]
    const int cnt = *count;
    const int nseg = gridDim.y;
    const int seg = blockIdx.y;
    const int k0 = static_cast<int>((static_cast<int64_t>(cnt) * seg) / nseg);
    const int k1 = static_cast<int>((static_cast<int64_t>(cnt) * (seg + 1)) / nseg);
    const int64_t units = mcopy / V;
    int64_t uu[U];
#pragma unroll
    for (int q = 0; q < U; ++q) uu[q] = (static_cast<int64_t>(blockIdx.x) * U + q) * kAuxThreads + threadIdx.x;
    // copies of list entry kk into ring stage st (one commit group per entry, empty past k1)
    auto issue = [&](int kk, int st) {
        if (kk < k1) {
            const TA* col = A + static_cast<int64_t>(__ldg(idx + kk)) * lda;
#pragma unroll
            for (int q = 0; q < U; ++q)
                if (uu[q] < units) cp_async_16(&ring[(st * U + q) * kAuxThreads + threadIdx.x], col + uu[q] * V);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < kPipeStages - 1; ++t) issue(k0 + t, t);
    typename std::conditional<kExact, ProdAcc<TC>, TP>::type acc[U][V];
    if constexpr (!kExact) {
#pragma unroll
        for (int q = 0; q < U; ++q)
#pragma unroll
            for (int e = 0; e < V; ++e) acc[q][e] = TP(0);
    }
    int st = 0;
    for (int k = k0; k < k1; ++k) {
        issue(k + kPipeStages - 1, st == 0 ? kPipeStages - 1 : st - 1);
        cp_async_wait<kPipeStages - 1>();  // entry k's copies have landed
        TC vh, vl = TC(0);
        if constexpr (kExact) {
            double v = static_cast<double>(__ldg(val + k));
            if (scale) v *= static_cast<double>(__ldg(scale + __ldg(idx + k)));
            vh = static_cast<TC>(v);
            vl = static_cast<TC>(v - static_cast<double>(vh));
        } else {
            vh = static_cast<TC>(__ldg(val + k));
            if (scale) vh *= static_cast<TC>(__ldg(scale + __ldg(idx + k)));
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            if (uu[q] < units) {
                TC a[V];
                ATraits<TA>::unpack(ring[(st * U + q) * kAuxThreads + threadIdx.x], a);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    if constexpr (kExact) {
                        acc[q][e].add_prod(a[e], vh);
                        if (vl != TC(0)) acc[q][e].add_prod(a[e], vl);
                    } else {
                        acc[q][e] = fmac(a[e], vh, acc[q][e]);
                    }
                }
            }
        }
        st = st + 1 == kPipeStages ? 0 : st + 1;
    }
    cp_async_wait<0>();
    TP* out = static_cast<TP*>(partial_out) + static_cast<int64_t>(seg) * mcopy;
#pragma unroll
    for (int q = 0; q < U; ++q)
        if (uu[q] < units)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                if constexpr (kExact)
                    out[uu[q] * V + e] = acc[q][e].value();
                else
                    out[uu[q] * V + e] = acc[q][e];
            }
}

template <typename TA, typename TV>
__global__ void __launch_bounds__(kAuxThreads) gather_gemv_exact_kernel(const TA* A, int64_t lda, int64_t mcopy,
                                                                        const float* scale, const int* idx,
                                                                        const TV* val, const int* count,
                                                                        double* partial) {
    using TC = typename ATraits<TA>::TC;
    constexpr int V = ATraits<TA>::kVec;
    const int cnt = *count;
    const int nseg = gridDim.y;
    const int seg = blockIdx.y;
    const int k0 = static_cast<int>((static_cast<int64_t>(cnt) * seg) / nseg);
    const int k1 = static_cast<int>((static_cast<int64_t>(cnt) * (seg + 1)) / nseg);
    const int64_t units = mcopy / V;
    int64_t uu[kGemvUnits];
#pragma unroll
    for (int q = 0; q < kGemvUnits; ++q)
        uu[q] = (static_cast<int64_t>(blockIdx.x) * kGemvUnits + q) * kAuxThreads + threadIdx.x;
    ProdAcc<TC> acc[kGemvUnits][V];
    constexpr int KU = 4;  // list entries whose loads are in flight together
    for (int k = k0; k < k1; k += KU) {
        uint4 q4[KU][kGemvUnits];
        TC vh[KU], vl[KU];
#pragma unroll
        for (int t = 0; t < KU; ++t) {
            vh[t] = vl[t] = TC(0);
            if (k + t < k1) {
                const int j = __ldg(idx + k + t);
                double v = static_cast<double>(__ldg(val + k + t));
                if (scale) v *= static_cast<double>(__ldg(scale + j));
                vh[t] = static_cast<TC>(v);
                vl[t] = static_cast<TC>(v - static_cast<double>(vh[t]));
                const TA* col = A + static_cast<int64_t>(j) * lda;
#pragma unroll
                for (int q = 0; q < kGemvUnits; ++q)
                    if (uu[q] < units) q4[t][q] = ld_stream_u4(col + uu[q] * V);
            }
        }
#pragma unroll
        for (int t = 0; t < KU; ++t) {
            if (k + t < k1) {
#pragma unroll
                for (int q = 0; q < kGemvUnits; ++q) {
                    if (uu[q] < units) {
                        TC a[V];
                        ATraits<TA>::unpack(q4[t][q], a);
#pragma unroll
                        for (int e = 0; e < V; ++e) {
                            acc[q][e].add_prod(a[e], vh[t]);
                            if (vl[t] != TC(0)) acc[q][e].add_prod(a[e], vl[t]);
                        }
                    }
                }
            }
        }
    }
    double* out = partial + static_cast<int64_t>(seg) * mcopy;
#pragma unroll
    for (int q = 0; q < kGemvUnits; ++q)
        if (uu[q] < units)
#pragma unroll
            for (int e = 0; e < V; ++e) out[uu[q] * V + e] = acc[q][e].value();
}

// r[i] = (set ? -b[i] : r[i]) + sum_seg partial[seg][i]  for i < m (fixed order); r[i] = 0 for m <= i < mcopy.
template <typename TP, typename TB>
__global__ void reduce_partials_kernel(double* r, const TP* partial, int nseg, int64_t m, int64_t mcopy, const TB* b,
                                       int set_mode) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < mcopy;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (i >= m) {
            r[i] = 0.0;
            continue;
        }
        double s = 0.0;
        for (int k = 0; k < nseg; ++k) s += static_cast<double>(partial[static_cast<int64_t>(k) * mcopy + i]);
        r[i] = set_mode ? (s - static_cast<double>(b[i])) : (r[i] + s);
    }
}

// ----------------------------------------------------------------------------- proximal weight

// d_j += delta for every coordinate (the proximal weight tau of all surrogates changes by delta).
template <typename T>
__global__ void __launch_bounds__(kAuxThreads) shift_weights_kernel(T* dw, int64_t n, T delta) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kAuxThreads;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * kAuxThreads + threadIdx.x; j < n; j += stride) dw[j] += delta;
}

// ----------------------------------------------------------------------------- norms

constexpr int kNormsFields = 7;

// part[blk*7 + {0..6}] = {sum r_i^2, sum |x_j|, sum x_j^2, nnz(x), sum lin_j x_j, sum h(x_j),
// sum b_i r_i} over a fixed stride (lin may be null; field 5 is 0 unless dc.kind != 0).
template <typename TX>
__global__ void __launch_bounds__(kAuxThreads) norms_kernel(const double* r, const TX* b, int64_t m, const TX* x,
                                                            int64_t n, const TX* lin, DcTerm dc, double* part) {
    __shared__ double sh[kAuxThreads / 32];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * kAuxThreads;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kAuxThreads + threadIdx.x;
    double rr = 0.0, a1 = 0.0, a2 = 0.0, nz = 0.0, lx = 0.0, hs = 0.0, br = 0.0;
    for (int64_t i = i0; i < m; i += stride) {
        rr = fma(r[i], r[i], rr);
        br = fma(static_cast<double>(b[i]), r[i], br);
    }
    for (int64_t j = i0; j < n; j += stride) {
        const double v = static_cast<double>(x[j]);
        a1 += fabs(v);
        a2 = fma(v, v, a2);
        nz += (v != 0.0) ? 1.0 : 0.0;
        if (lin) lx = fma(static_cast<double>(lin[j]), v, lx);
        if (dc.kind) hs += dc_h(dc, v);
    }
    rr = block_sum_256<double>(rr, sh);
    a1 = block_sum_256<double>(a1, sh);
    a2 = block_sum_256<double>(a2, sh);
    nz = block_sum_256<double>(nz, sh);
    lx = block_sum_256<double>(lx, sh);
    hs = block_sum_256<double>(hs, sh);
    br = block_sum_256<double>(br, sh);
    if (threadIdx.x == 0) {
        double* o = part + blockIdx.x * kNormsFields;
        o[0] = rr;
        o[1] = a1;
        o[2] = a2;
        o[3] = nz;
        o[4] = lx;
        o[5] = hs;
        o[6] = br;
    }
}

template <typename T>
__global__ void finalize_norms_kernel(const T* part, int nparts, T* out) {
    // templated only so that every translation unit may instantiate it
    if (threadIdx.x < kNormsFields) {
        double s = 0.0;
        for (int k = 0; k < nparts; ++k) s += part[k * kNormsFields + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// ----------------------------------------------------------------------------- check

template <typename TA>
struct CheckDot;

// FP64 storage: FP64 products and accumulation.
template <>
struct CheckDot<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double rh, double /*rl*/) { s = fma(a, rh, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// FP32 compute: Dot2 with the residual split into hi + lo FP32 parts.
struct CheckDotF {
    float p = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float rh, float rl) {
        const float h = a * rh;
        const float eprod = fmaf(a, rh, -h);  // exact: a*rh = h + eprod
        float sum, esum;
        two_sum(p, h, sum, esum);
        p = sum;
        c += (esum + eprod) + a * rl;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(p) + static_cast<double>(c); }
};
template <>
struct CheckDot<float> : CheckDotF {};
template <>
struct CheckDot<__nv_bfloat16> : CheckDotF {};
template <>
struct CheckDot<__nv_fp8_e4m3> : CheckDotF {};

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
    atomicMax(p, static_cast<unsigned long long>(__double_as_longlong(v)));
}

// meas: [0] max|M_F|, [1] max|xhat - x|, [2] max KKT (LASSO w/o box), [3] max|x|, [4] nnz,
//       [5] nonfinite flag.  One warp per column.  The residual is staged in shared memory
//       as (hi, lo) pairs when it fits (use_smem), else read from global memory.
template <typename TA>
__global__ void __launch_bounds__(kCheckThreads) check_kernel(const TA* A, int64_t lda, int64_t m, int64_t n,
                                                            const float* scale, const double* r,
                                                            const typename XType<TA>::T* x,
                                                            const typename XType<TA>::T* lo,
                                                            const typename XType<TA>::T* hi, const double* dw,
                                                            const typename XType<TA>::T* lin, double lam,
                                                            double s_loss, double c2, DcTerm dc, int lasso_nobox,
                                                            int use_smem, unsigned long long* meas) {
    using TC = typename ATraits<TA>::TC;
    constexpr int V = ATraits<TA>::kVec;
    extern __shared__ __align__(16) unsigned char csm[];
    TC* rh_s = reinterpret_cast<TC*>(csm);
    const int64_t mc = (m + V - 1) / V * V;
    TC* rl_s = rh_s + mc;
    if (use_smem) {
        for (int64_t i = threadIdx.x; i < mc; i += blockDim.x) {
            const double v = i < m ? r[i] : 0.0;
            const TC h = static_cast<TC>(v);
            rh_s[i] = h;
            rl_s[i] = static_cast<TC>(v - static_cast<double>(h));
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    double mmf = 0.0, mxh = 0.0, mkkt = 0.0, mx = 0.0, matr = 0.0;
    unsigned long long nnz = 0;
    int nonfinite = 0;
    constexpr int kU = 4;  // independent 16-byte loads in flight per lane
    for (int64_t j = gw; j < n; j += nw) {
        const TA* col = A + j * lda;
        CheckDot<TA> acc;
        const int64_t units = mc / V;
        for (int64_t u0 = lane; u0 < units; u0 += 32 * kU) {
            uint4 q[kU];
#pragma unroll
            for (int t = 0; t < kU; ++t)
                if (u0 + 32 * t < units) q[t] = ld_stream_u4(col + (u0 + 32 * t) * V);
#pragma unroll
            for (int t = 0; t < kU; ++t) {
                const int64_t u = u0 + 32 * t;
                if (u < units) {
                    TC a[V];
                    ATraits<TA>::unpack(q[t], a);
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const int64_t i = u * V + e;
                        if (i < m) {
                            TC h, l;
                            if (use_smem) {
                                h = rh_s[i];
                                l = rl_s[i];
                            } else {
                                const double v = r[i];
                                h = static_cast<TC>(v);
                                l = static_cast<TC>(v - static_cast<double>(h));
                            }
                            acc.add(a[e], h, l);
                        }
                    }
                }
            }
        }
        double g = acc.value();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if (lane == 0) {
            const double sc = scale ? static_cast<double>(scale[j]) : 1.0;
            const double xj = static_cast<double>(x[j]);
            const double grad = s_loss * g * sc - c2 * xj + (lin ? static_cast<double>(lin[j]) : 0.0) -
                                dc.lam * dc_hminus_grad(dc, xj);
            const double l = lo ? static_cast<double>(lo[j]) : -INFINITY;
            const double h = hi ? static_cast<double>(hi[j]) : INFINITY;
            // M_F: unit-weight proximal step
            double v = xj - grad;
            double av = fabs(v) - lam;
            double y = av > 0.0 ? copysign(av, v) : 0.0;
            y = fmin(fmax(y, l), h);
            const double mf = fabs(xj - y);
            // xhat with the surrogate weight d_j
            const double dj = dw[j];
            double xh = 0.0;
            if (dj > 0.0) {
                v = xj - grad / dj;
                av = fabs(v) - lam / dj;
                xh = av > 0.0 ? copysign(av, v) : 0.0;
            }
            xh = fmin(fmax(xh, l), h);
            const double dx = fabs(xh - xj);
            double kkt = 0.0;
            if (lasso_nobox) kkt = xj == 0.0 ? fmax(fabs(grad) - lam, 0.0) : fabs(grad + copysign(lam, xj));
            if (!(isfinite(mf) && isfinite(dx) && isfinite(kkt) && isfinite(xj))) nonfinite = 1;
            mmf = fmax(mmf, mf);
            mxh = fmax(mxh, dx);
            mkkt = fmax(mkkt, kkt);
            mx = fmax(mx, fabs(xj));
            matr = fmax(matr, fabs(s_loss * g * sc));  // ||s A^T r||_inf, for the LASSO dual point
            nnz += (xj != 0.0);
        }
    }
    if (lane == 0) {
        if (mmf > 0.0) atomic_max_nonneg(&meas[0], mmf);
        if (mxh > 0.0) atomic_max_nonneg(&meas[1], mxh);
        if (mkkt > 0.0) atomic_max_nonneg(&meas[2], mkkt);
        if (mx > 0.0) atomic_max_nonneg(&meas[3], mx);
        if (nnz) atomicAdd(&meas[4], nnz);
        if (nonfinite) atomicOr(&meas[5], 1ull);
        if (matr > 0.0) atomic_max_nonneg(&meas[6], matr);
    }
}

}  // namespace asyflexa
