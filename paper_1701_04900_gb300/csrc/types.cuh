// Element traits for the storage type of A: how many rows one 16-byte unit holds and
// how to widen a unit to the compute type TC.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

namespace asyflexa {

template <typename TA>
struct ATraits;

template <>
struct ATraits<double> {
    using TC = double;
    static constexpr int kVec = 2;
    __device__ __forceinline__ static void unpack(const uint4& v, TC (&o)[kVec]) {
        o[0] = __hiloint2double(static_cast<int>(v.y), static_cast<int>(v.x));
        o[1] = __hiloint2double(static_cast<int>(v.w), static_cast<int>(v.z));
    }
};

template <>
struct ATraits<float> {
    using TC = float;
    static constexpr int kVec = 4;
    __device__ __forceinline__ static void unpack(const uint4& v, TC (&o)[kVec]) {
        o[0] = __uint_as_float(v.x);
        o[1] = __uint_as_float(v.y);
        o[2] = __uint_as_float(v.z);
        o[3] = __uint_as_float(v.w);
    }
};

template <>
struct ATraits<__nv_bfloat16> {
    using TC = float;
    static constexpr int kVec = 8;
    __device__ __forceinline__ static void unpack(const uint4& v, TC (&o)[kVec]) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // bf16 -> f32 is exact: the bf16 bits are the high half of the f32 bits.
            o[2 * i] = __uint_as_float(w[i] << 16);
            o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
};

template <>
struct ATraits<__nv_fp8_e4m3> {
    using TC = float;
    static constexpr int kVec = 16;
    __device__ __forceinline__ static void unpack(const uint4& v, TC (&o)[kVec]) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_fp8x2_storage_t lo2 = static_cast<__nv_fp8x2_storage_t>(w[i] & 0xffffu);
            __nv_fp8x2_storage_t hi2 = static_cast<__nv_fp8x2_storage_t>(w[i] >> 16);
            __half2_raw hl = __nv_cvt_fp8x2_to_halfraw2(lo2, __NV_E4M3);
            __half2_raw hh = __nv_cvt_fp8x2_to_halfraw2(hi2, __NV_E4M3);
            float2 fl = __half22float2(*reinterpret_cast<__half2*>(&hl));
            float2 fh = __half22float2(*reinterpret_cast<__half2*>(&hh));
            o[4 * i + 0] = fl.x;
            o[4 * i + 1] = fl.y;
            o[4 * i + 2] = fh.x;
            o[4 * i + 3] = fh.y;
        }
    }
};

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmac(double a, double b, double c) { return ::fma(a, b, c); }

// Sum of FP32 products carried as an unevaluated pair (s, c) of FP32 numbers using the
// error-free transformations TwoProduct (via FMA) and TwoSum (Knuth), as in the Dot2
// algorithm of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26(6), 2005).  The result is as accurate as a dot product computed in twice the
// working precision, without FP64 arithmetic in the loop (FP64 throughput on GB300 is a
// small fraction of FP32).
// TwoSum (Knuth): s = fl(a + b) and s + e = a + b exactly (Ogita, Rump, Oishi 2005).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float z = s - a;
    e = (a - (s - z)) + (b - z);
}

struct DFAcc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        const float ep = fmaf(a, b, -p);  // exact: a*b = p + ep
        const float t = s + p;
        const float z = t - s;
        const float es = (s - (t - z)) + (p - z);  // exact: s + p = t + es
        s = t;
        c += es + ep;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(s) + static_cast<double>(c); }
};

// x / b / bounds type: double for FP64 problems, float otherwise.
template <typename TA>
struct XType {
    using T = float;
};
template <>
struct XType<double> {
    using T = double;
};

// Nonconvex regulariser of the sparse-learning problem of Section 4.3, F = ||Ax-b||^2 + lam H(x)
// with H = sum_j h(x_j): kind 1 = log, h(x) = log(1 + theta|x|) / log(1 + theta); kind 2 =
// exp, h(x) = 1 - exp(-theta|x|).  h = eta|x| - h-(x) with h- convex and smooth; the method's
// smooth part f holds -lam H-, G = lam eta ||x||_1.  kind 0: no such term.
struct DcTerm {
    int kind;
    double lam, theta, eta;
};

// d/dx h-(x) = eta sign(x) - h'(x) (0 at x = 0).
__device__ __forceinline__ double dc_hminus_grad(const DcTerm& d, double x) {
    if (d.kind == 0 || x == 0.0) return 0.0;
    const double a = fabs(x);
    const double v = d.kind == 2 ? -d.theta * expm1(-d.theta * a) : d.eta * (d.theta * a) / (1.0 + d.theta * a);
    return copysign(v, x);
}

// h(x) itself (for the objective).
__device__ __forceinline__ double dc_h(const DcTerm& d, double x) {
    const double a = fabs(x);
    return d.kind == 2 ? -expm1(-d.theta * a) : log1p(d.theta * a) / log1p(d.theta);
}

}  // namespace asyflexa
