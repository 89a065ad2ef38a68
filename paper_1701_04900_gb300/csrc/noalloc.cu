// asyflexa_residual_noalloc: the exact residual r = A x - b without a handle and without
// any device allocation.
//
// Some callers cannot allocate device memory when they need this value: a plugin inside a
// host application that gives it a fixed device-memory budget and owns every allocation, or
// a latency-sensitive loop in which cudaMalloc / cudaFree would synchronise the device and
// stall every other stream.  This entry point takes its scratch from one file-scope device
// array of fixed size instead of handle-owned allocations, and computes what the residual
// refresh of a handle computes by the same steps (ordered compaction of the nonzeros of x,
// compensated products, fixed-order FP64 reduction) through the register-batched gather
// kernel (gather_gemv_exact_kernel) instead of the handle's pipelined one, so the two agree up
// to the grouping of partial sums.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/asyflexa.h"
#include "aux.cuh"

namespace asyflexa_internal {
// Sets the calling thread's message returned by asyflexa_last_error(NULL) (api.cu).
void set_thread_error(const std::string& msg);
}  // namespace asyflexa_internal

namespace {

using namespace asyflexa;

// Scratch capacity and the problem sizes it supports.
constexpr size_t kScratchBytes = size_t(8) << 20;           // 8 MiB per device, held until exit
constexpr int64_t kNoallocMaxN = int64_t(1) << 18;          // 262144 columns
constexpr size_t kListBytes = kNoallocMaxN * (sizeof(int) + sizeof(double));  // indices + values
constexpr size_t kTileBytes = 4096;                          // tile counts (<= 1024 ints) + count
constexpr size_t kPartialBytes = kScratchBytes - kListBytes - kTileBytes;
constexpr int kNoallocMaxSeg = 16;

// The scratch itself.  In host code this name is only a host-side stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress (see scratch_address).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

int fail(int code, const std::string& m) {
    asyflexa_internal::set_thread_error(m);
    return code;
}

// r[i] = sum_seg partial[seg * stride + i] - b[i] for i < m, in fixed segment order.
template <typename TB>
__global__ void noalloc_reduce_kernel(double* r, const double* partial, int nseg, int64_t m, int64_t stride,
                                      const TB* b) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < nseg; ++k) s += partial[static_cast<int64_t>(k) * stride + i];
        r[i] = s - static_cast<double>(b[i]);
    }
}

// Device address of g_noalloc_scratch on the current device, looked up once per device index
// and cached for the life of the process (the device's primary context is assumed throughout).
int scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return fail(ASYFLEXA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return ASYFLEXA_OK;
}

template <typename TA>
cudaError_t run(const asyflexa_problem& P, const void* xv, double* r_out, cudaStream_t st, unsigned char* scr,
                int sm_count) {
    using TX = typename XType<TA>::T;
    constexpr int V = ATraits<TA>::kVec;
    const int64_t m = P.m, n = P.n;
    const int64_t mcopy = (m + V - 1) / V * V;
    const TX* x = static_cast<const TX*>(xv);
    int* list_idx = reinterpret_cast<int*>(scr);
    TX* list_val = reinterpret_cast<TX*>(scr + kNoallocMaxN * sizeof(int));
    int* tilecnt = reinterpret_cast<int*>(scr + kListBytes);
    int* count = tilecnt + 1000;
    double* partial = reinterpret_cast<double*>(scr + kListBytes + kTileBytes);
    const int tiles = static_cast<int>((n + kCompactTile - 1) / kCompactTile);
    const int64_t units = mcopy / V;
    const int rowtiles = static_cast<int>((units + kAuxThreads * kGemvUnits - 1) / (kAuxThreads * kGemvUnits));
    int nseg = static_cast<int>(kPartialBytes / (static_cast<size_t>(mcopy) * sizeof(double)));
    const int want = (2 * sm_count + rowtiles - 1) / rowtiles;
    nseg = nseg < want ? nseg : want;
    nseg = nseg > kNoallocMaxSeg ? kNoallocMaxSeg : (nseg < 1 ? 1 : nseg);
    count_nonzero_kernel<TX><<<tiles, kAuxThreads, 0, st>>>(x, n, tilecnt);
    compact_kernel<TX><<<tiles, kAuxThreads, 0, st>>>(x, n, tilecnt, tiles, list_idx, list_val, count);
    gather_gemv_exact_kernel<TA, TX><<<dim3(rowtiles, nseg), kAuxThreads, 0, st>>>(
        static_cast<const TA*>(P.A), P.lda, mcopy, P.col_scale, list_idx, list_val, count, partial);
    // reduce into the caller's buffer of exactly m entries
    const int rg = static_cast<int>((m + kAuxThreads - 1) / kAuxThreads);
    noalloc_reduce_kernel<TX><<<rg, kAuxThreads, 0, st>>>(r_out, partial, nseg, m, mcopy, static_cast<const TX*>(P.b));
    return cudaGetLastError();
}

}  // namespace

extern "C" int asyflexa_residual_noalloc(const asyflexa_problem* P, const void* x, double* r_out,
                                         void* cuda_stream) {
    if (!P || !x || !r_out) return fail(ASYFLEXA_EINVAL, "problem, x or r_out is NULL");
    int ea = 0;
    switch (P->a_dtype) {
        case ASYFLEXA_F64: ea = 8; break;
        case ASYFLEXA_F32: ea = 4; break;
        case ASYFLEXA_BF16: ea = 2; break;
        case ASYFLEXA_FP8E4M3: ea = 1; break;
        default: return fail(ASYFLEXA_EINVAL, "unknown a_dtype");
    }
    if (P->x_dtype != (P->a_dtype == ASYFLEXA_F64 ? ASYFLEXA_F64 : ASYFLEXA_F32))
        return fail(ASYFLEXA_EINVAL, "x_dtype must be F64 for F64 A and F32 otherwise");
    if (P->m < 1 || P->n < 1) return fail(ASYFLEXA_EINVAL, "m and n must be >= 1");
    if (P->lda < P->m || (P->lda * ea) % 16 != 0 || !P->A || (reinterpret_cast<uintptr_t>(P->A) & 15u))
        return fail(ASYFLEXA_EINVAL, "A must be 16-byte aligned with lda >= m and lda * element size a multiple of 16");
    if (!P->b) return fail(ASYFLEXA_EINVAL, "b is NULL");
    const bool quant = P->a_dtype == ASYFLEXA_BF16 || P->a_dtype == ASYFLEXA_FP8E4M3;
    if (quant != (P->col_scale != nullptr)) return fail(ASYFLEXA_EINVAL, "col_scale is required exactly for BF16/FP8 storage");
    const int v = 16 / ea;
    const int64_t mcopy = (P->m + v - 1) / v * v;
    if (P->n > kNoallocMaxN)
        return fail(ASYFLEXA_EINVAL, "n = " + std::to_string(P->n) + " exceeds the no-allocation limit of " +
                                         std::to_string(kNoallocMaxN) + " columns");
    if (static_cast<size_t>(mcopy) * sizeof(double) > kPartialBytes)
        return fail(ASYFLEXA_EINVAL, "m = " + std::to_string(P->m) + " exceeds the no-allocation limit of " +
                                         std::to_string(kPartialBytes / sizeof(double)) + " rows");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ASYFLEXA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(ASYFLEXA_EINVAL, "device index out of range");
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(ASYFLEXA_ECUDA, std::string("SM count: ") + cudaGetErrorString(e));
    unsigned char* scr = nullptr;
    int rc = scratch_address(dev, &scr);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    switch (P->a_dtype) {
        case ASYFLEXA_F64: e = run<double>(*P, x, r_out, st, scr, sms); break;
        case ASYFLEXA_F32: e = run<float>(*P, x, r_out, st, scr, sms); break;
        case ASYFLEXA_BF16: e = run<__nv_bfloat16>(*P, x, r_out, st, scr, sms); break;
        default: e = run<__nv_fp8_e4m3>(*P, x, r_out, st, scr, sms); break;
    }
    if (e != cudaSuccess) return fail(ASYFLEXA_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return ASYFLEXA_OK;
}
