// Diagnostic entry points.  asyflexa_convert_check runs the kernels' own FP32 <-> FP64
// conversions (convert.cuh) and their decoding of BF16 / FP8-e4m3 storage (ATraits in
// types.cuh) over a caller's array, so that they can be compared bit for bit with IEEE 754
// conversions and the formats' definitions computed elsewhere.  asyflexa_wait_check runs the
// kernels' bounded mbarrier wait (ptx.cuh) on a barrier that is, or is never, arrived at, so
// that a test can see a wait give up with the timeout status and the context stay usable.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/asyflexa.h"
#include "convert.cuh"
#include "ptx.cuh"
#include "types.cuh"

namespace asyflexa_internal {
void set_thread_error(const std::string& msg);
}  // namespace asyflexa_internal

namespace {

__global__ void __launch_bounds__(256) convert_kernel(int dir, const void* in, void* out, int64_t n) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (dir == 0) {
            static_cast<float*>(out)[i] = asyflexa::f64_to_f32(static_cast<const double*>(in)[i]);
        } else {
            static_cast<double*>(out)[i] = asyflexa::f32_to_f64(static_cast<const float*>(in)[i]);
        }
    }
}

// One 16-byte unit of stored elements per thread, decoded by the same unpack the kernels use.
template <typename TA>
__global__ void __launch_bounds__(256) decode_kernel(const uint4* in, float* out, int64_t units) {
    constexpr int V = asyflexa::ATraits<TA>::kVec;
    for (int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; u < units;
         u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float a[V];
        asyflexa::ATraits<TA>::unpack(in[u], a);
#pragma unroll
        for (int k = 0; k < V; ++k) out[u * V + k] = a[k];
    }
}

// One thread: an mbarrier expecting one arrival, arrived at first or never, then the bounded
// wait.  out: [completed (1/0), err (0 or kDevTimeout), abort flag, elapsed microseconds].
__global__ void wait_check_kernel(int arrive_first, unsigned long long limit_ns, int* out) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    asyflexa::mbar_init(&bar, 1);
    abort_flag = 0;
    asyflexa::fence_barrier_init();
    out[1] = 0;
    if (arrive_first) asyflexa::mbar_arrive(&bar);
    const uint64_t t0 = asyflexa::global_timer_ns();
    const bool ok = asyflexa::mbar_wait_bounded_for(&bar, 0u, &abort_flag, out + 1, limit_ns);
    const uint64_t t1 = asyflexa::global_timer_ns();
    out[0] = ok ? 1 : 0;
    out[2] = abort_flag;
    out[3] = static_cast<int>((t1 - t0) / 1000u);
}

int fail(int code, const std::string& m) {
    asyflexa_internal::set_thread_error(m);
    return code;
}

}  // namespace

extern "C" int asyflexa_convert_check(int dir, const void* in, void* out, int64_t n, void* cuda_stream) {
    if (dir < 0 || dir > 3)
        return fail(ASYFLEXA_EINVAL, "dir must be 0 (FP64 -> FP32), 1 (FP32 -> FP64), 2 (FP8-e4m3 -> FP32) or "
                                     "3 (BF16 -> FP32)");
    if (n < 0) return fail(ASYFLEXA_EINVAL, "n must be >= 0");
    const int vec = dir == 2 ? 16 : dir == 3 ? 8 : 1;
    if (n % vec != 0) return fail(ASYFLEXA_EINVAL, "n must be a multiple of 16 (dir 2) or 8 (dir 3)");
    if (n == 0) return ASYFLEXA_OK;
    if (!in || !out) return fail(ASYFLEXA_EINVAL, "in or out is NULL");
    if (dir >= 2 && reinterpret_cast<uintptr_t>(in) % 16 != 0)
        return fail(ASYFLEXA_EINVAL, "in must be 16-byte aligned for dir 2 and 3");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t want = (n / vec + 255) / 256;
    const int blocks = static_cast<int>(want < 4096 ? want : 4096);
    if (dir == 2) {
        decode_kernel<__nv_fp8_e4m3><<<blocks, 256, 0, st>>>(static_cast<const uint4*>(in), static_cast<float*>(out),
                                                              n / vec);
    } else if (dir == 3) {
        decode_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<const uint4*>(in), static_cast<float*>(out),
                                                              n / vec);
    } else {
        convert_kernel<<<blocks, 256, 0, st>>>(dir, in, out, n);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ASYFLEXA_ECUDA, std::string("convert_check launch: ") + cudaGetErrorString(e));
    return ASYFLEXA_OK;
}

extern "C" int asyflexa_wait_check(int arrive_first, int64_t limit_ns, int* result) {
    if (!result) return fail(ASYFLEXA_EINVAL, "result is NULL");
    if (limit_ns < 1000 || limit_ns > 1000000000)
        return fail(ASYFLEXA_EINVAL, "limit_ns must be within [1e3, 1e9]");
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 4 * sizeof(int));
    if (e != cudaSuccess) return fail(ASYFLEXA_ENOMEM, std::string("wait_check: ") + cudaGetErrorString(e));
    wait_check_kernel<<<1, 1>>>(arrive_first ? 1 : 0, static_cast<unsigned long long>(limit_ns), d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(result, d, 4 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ASYFLEXA_ECUDA, std::string("wait_check: ") + cudaGetErrorString(e));
    return result[0] ? ASYFLEXA_OK : ASYFLEXA_ETIMEOUT;
}
