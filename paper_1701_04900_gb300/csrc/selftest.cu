// Diagnostic entry point asyflexa_convert_check: runs the kernels' own FP32 <-> FP64
// conversions (convert.cuh) over a caller's array, so that they can be compared bit for bit
// with IEEE 754 round-to-nearest-even conversions computed elsewhere.
#include <cuda_runtime.h>

#include <string>

#include "../../include/asyflexa.h"
#include "convert.cuh"

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

int fail(int code, const std::string& m) {
    asyflexa_internal::set_thread_error(m);
    return code;
}

}  // namespace

extern "C" int asyflexa_convert_check(int dir, const void* in, void* out, int64_t n, void* cuda_stream) {
    if (dir != 0 && dir != 1) return fail(ASYFLEXA_EINVAL, "dir must be 0 (FP64 -> FP32) or 1 (FP32 -> FP64)");
    if (n < 0) return fail(ASYFLEXA_EINVAL, "n must be >= 0");
    if (n == 0) return ASYFLEXA_OK;
    if (!in || !out) return fail(ASYFLEXA_EINVAL, "in or out is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t want = (n + 255) / 256;
    const int blocks = static_cast<int>(want < 4096 ? want : 4096);
    convert_kernel<<<blocks, 256, 0, st>>>(dir, in, out, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ASYFLEXA_ECUDA, std::string("convert_check launch: ") + cudaGetErrorString(e));
    return ASYFLEXA_OK;
}
