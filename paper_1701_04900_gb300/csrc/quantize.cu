// Storage utilities for the column-major matrix:
//
// asyflexa_quantize: per-column scaled BF16 / FP8-e4m3 storage of an FP32 matrix.  For the
// low-precision form of the method A is stored as codes q_j with one FP32 scale per column,
// a_j ~= scale_j * q_j; the sweeps then stream 2 (BF16) or 1 (FP8) bytes per entry instead
// of 4 and accumulate in FP32.  scale_j = max_i |a_ij| / qmax with qmax = 448 (the largest
// finite e4m3 value) for FP8 and 1 for BF16, so every code is finite.
//
// asyflexa_gather_columns: the column submatrix A_S (used for the adjoint of the solution
// map, which lives on the support S of the solution).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/asyflexa.h"

namespace asyflexa_internal {
void set_thread_error(const std::string& msg);
}  // namespace asyflexa_internal

namespace {

template <int KIND>
__global__ void quantize_kernel(const float* A, int64_t m, int64_t n, int64_t lda, void* Q, int64_t ldq,
                                float* scale) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t j = gw; j < n; j += nw) {
        const float* col = A + j * lda;
        float amax = 0.f;
        for (int64_t i = lane; i < m; i += 32) amax = fmaxf(amax, fabsf(col[i]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        const float qmax = KIND == ASYFLEXA_FP8E4M3 ? 448.f : 1.f;
        const float s = amax > 0.f ? amax / qmax : 1.f;
        const float inv = 1.f / s;
        if (lane == 0) scale[j] = s;
        if (KIND == ASYFLEXA_BF16) {
            __nv_bfloat16* q = static_cast<__nv_bfloat16*>(Q) + j * ldq;
            for (int64_t i = lane; i < ldq; i += 32) q[i] = __float2bfloat16_rn(i < m ? col[i] * inv : 0.f);
        } else {
            __nv_fp8_storage_t* q = static_cast<__nv_fp8_storage_t*>(Q) + j * ldq;
            for (int64_t i = lane; i < ldq; i += 32)
                q[i] = __nv_cvt_float_to_fp8(i < m ? col[i] * inv : 0.f, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// One warp per output column, 16-byte copies (both strides are multiples of 16 bytes).
__global__ void gather_columns_kernel(const uint4* A, int64_t lda16, const int32_t* idx, int64_t k, uint4* out,
                                      int64_t ldo16, int64_t units) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t c = gw; c < k; c += nw) {
        const uint4* src = A + static_cast<int64_t>(idx[c]) * lda16;
        uint4* dst = out + c * ldo16;
        for (int64_t u = lane; u < ldo16; u += 32) dst[u] = u < units ? src[u] : make_uint4(0, 0, 0, 0);
    }
}

}  // namespace

extern "C" int asyflexa_gather_columns(const void* A, int64_t lda, int32_t dtype, int64_t m, const int32_t* idx,
                                       int64_t k, void* out, int64_t ldo, void* cuda_stream) {
    auto fail = [](const std::string& msg) {
        asyflexa_internal::set_thread_error(msg);
        return static_cast<int>(ASYFLEXA_EINVAL);
    };
    int elt = 0;
    switch (dtype) {
        case ASYFLEXA_F64: elt = 8; break;
        case ASYFLEXA_F32: elt = 4; break;
        case ASYFLEXA_BF16: elt = 2; break;
        case ASYFLEXA_FP8E4M3: elt = 1; break;
        default: return fail("unknown dtype");
    }
    if (!A || !idx || !out) return fail("A, idx or out is NULL");
    if (m < 1 || k < 0 || lda < m || ldo < m) return fail("need m >= 1, k >= 0, lda >= m, ldo >= m");
    if ((lda * elt) % 16 || (ldo * elt) % 16 || (reinterpret_cast<uintptr_t>(A) & 15u) ||
        (reinterpret_cast<uintptr_t>(out) & 15u))
        return fail("A and out must be 16-byte aligned with 16-byte multiple column strides");
    if (k == 0) return ASYFLEXA_OK;
    const int64_t per = 16 / elt;
    const int64_t units = (m + per - 1) / per;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms > 0 ? 8 * sms : 1024;
    gather_columns_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        static_cast<const uint4*>(A), lda * elt / 16, idx, k, static_cast<uint4*>(out), ldo * elt / 16, units);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        asyflexa_internal::set_thread_error(std::string("gather launch: ") + cudaGetErrorString(e));
        return ASYFLEXA_ECUDA;
    }
    return ASYFLEXA_OK;
}

extern "C" int asyflexa_quantize(const float* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* Q,
                                 int64_t ldq, float* scale, void* cuda_stream) {
    auto fail = [](const std::string& msg) {
        asyflexa_internal::set_thread_error(msg);
        return static_cast<int>(ASYFLEXA_EINVAL);
    };
    if (!A || !Q || !scale) return fail("A, Q or scale is NULL");
    if (dtype != ASYFLEXA_BF16 && dtype != ASYFLEXA_FP8E4M3) return fail("dtype must be BF16 or FP8E4M3");
    if (m < 1 || n < 1 || lda < m || ldq < m) return fail("need m, n >= 1, lda >= m and ldq >= m");
    const int elt = dtype == ASYFLEXA_BF16 ? 2 : 1;
    if ((ldq * elt) % 16 != 0) return fail("ldq * element size must be a multiple of 16 bytes");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int grid = sms > 0 ? 8 * sms : 1024;
    if (dtype == ASYFLEXA_BF16)
        quantize_kernel<ASYFLEXA_BF16><<<grid, 256, 0, st>>>(A, m, n, lda, Q, ldq, scale);
    else
        quantize_kernel<ASYFLEXA_FP8E4M3><<<grid, 256, 0, st>>>(A, m, n, lda, Q, ldq, scale);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        asyflexa_internal::set_thread_error(std::string("quantize launch: ") + cudaGetErrorString(e));
        return ASYFLEXA_ECUDA;
    }
    return ASYFLEXA_OK;
}
