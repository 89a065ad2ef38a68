// Batched form: many independent problems (uneven sizes, or one matrix with many lambda
// values) solved together, in one of two forms.
//
// Gauss-Seidel form (batch_gs.cuh): ONE persistent launch for the whole batch; each CTA
// solves whole problems from a queue (largest first), one at a time, by exact cyclic
// Gauss-Seidel with its own stopping test.  The launch is captured in a CUDA graph.
//
// Async rounds: one persistent asynchronous sweep launch per round covers the blocks of
// every problem; each round (sweeps, exact residual refreshes, objectives, device-side
// convergence test) is replayed as a captured CUDA graph.  The sweep kernel is the
// register-increment async kernel of sweep_async.cuh in its BATCHED form: the blocks of all
// problems form one global list, CTA c owns the global blocks c, c + G, ..., and a converged
// problem's blocks are skipped from the next round on.
//
// Every problem keeps its own internal handle for the surrogate weights, the FP64 residual
// and the refresh / objective / check kernels.  An autotuner picks the launch shape of the
// chosen form by timing one real sweep per candidate and caches it per batch shape.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"
#include "sweep_async.cuh"
#include "batch_gs.cuh"

extern template struct asyflexa::Launcher<float>;

namespace asyflexa_internal {
void set_thread_error(const std::string& msg);
}  // namespace asyflexa_internal

using asyflexa::BatchInst;
using asyflexa::Launcher;

namespace {

struct ConvState {
    const double* norms;  // the problem's objective partials (internal handle)
    double lam, c, f_star, F, F_prev;
    int loss, conv_round;
};

// One thread per problem: F from the fresh objective partials; a problem converges when its
// relative gap is <= tol_gap (known optimum) or, without one, when a round lowered F by no
// more than stall_tol * |F|.  Converged (or non-finite) problems are deactivated.
__global__ void batch_converge_kernel(ConvState* cs, BatchInst* inst, int count, double tol_gap, double stall_tol,
                                      int* round, int* n_active) {
    __shared__ int r0;
    if (threadIdx.x == 0) r0 = *round;
    __syncthreads();
    for (int k = threadIdx.x; k < count; k += blockDim.x) {
        if (!inst[k].active) continue;
        ConvState& s = cs[k];
        const double* v = s.norms;
        const double F = (s.loss == ASYFLEXA_LOSS_LASSO ? 0.5 * v[0] : v[0] - s.c * v[2]) + v[4] + s.lam * v[1];
        bool conv;
        if (isfinite(s.f_star))
            conv = (F - s.f_star) / fabs(s.f_star) <= tol_gap;
        else
            conv = isfinite(s.F_prev) && (s.F_prev - F) <= stall_tol * fabs(F);
        s.F_prev = F;
        s.F = F;
        if (!isfinite(F)) {
            inst[k].active = 0;
            s.conv_round = -1;  // diverged
        } else if (conv) {
            inst[k].active = 0;
            s.conv_round = r0;
        } else {
            atomicAdd(n_active, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *round = r0 + 1;
}

constexpr int kCandidates[] = {16, 32, 64};

// Two CUDA events destroyed with the scope (error returns included).
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Saves (to_save = 1) or restores the iterates of the problems order[0 .. cnt) to / from save,
// problem k at the offset of its (d_j, 1/d_j) table: the autotuner's sweeps leave x as it was.
__global__ void gs_copy_x_kernel(const asyflexa::GsInst* inst, const int* order, int cnt, const float2* dd_base,
                                 float* save, int to_save) {
    for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
        const asyflexa::GsInst& g = inst[order[q]];
        float* sv = save + (g.dd - dd_base);
        for (int64_t j = threadIdx.x; j < g.n; j += blockDim.x) {
            if (to_save)
                sv[j] = g.x[j];
            else
                g.x[j] = sv[j];
        }
    }
}

// (d_j, 1/d_j) in FP32 for the Gauss-Seidel form ((0, 0) where d_j <= 0).
__global__ void gs_coef_kernel(const double* dw, int64_t n, float2* dd) {
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double d = dw[j];
        dd[j] = d > 0.0 ? make_float2(static_cast<float>(d), static_cast<float>(1.0 / d)) : make_float2(0.f, 0.f);
    }
}

// Launch shape of the Gauss-Seidel form.
struct GsChoice {
    int nw = 0, upt = 0, stages = 0, ctas_per_sm = 0, grid = 0, w = 1;
    int64_t slot_cap = 0, slot_bytes = 0;
    size_t smem = 0;
    const void* kernel = nullptr;
    bool operator==(const GsChoice& o) const {
        return nw == o.nw && upt == o.upt && stages == o.stages && grid == o.grid && w == o.w &&
               slot_bytes == o.slot_bytes;
    }
};

// Instantiated (consumer warps, units per thread) pairs: columns of up to NW * 32 * UPT * 4 rows.
const void* gs_kernel(int nw, int upt) {
    using namespace asyflexa;
    if (nw == 7) {
        switch (upt) {
            case 2: return reinterpret_cast<const void*>(batch_gs_kernel<7, 2>);
            case 3: return reinterpret_cast<const void*>(batch_gs_kernel<7, 3>);
            case 5: return reinterpret_cast<const void*>(batch_gs_kernel<7, 5>);
            case 6: return reinterpret_cast<const void*>(batch_gs_kernel<7, 6>);
            default: return nullptr;
        }
    }
    if (nw == 15) {
        switch (upt) {
            case 1: return reinterpret_cast<const void*>(batch_gs_kernel<15, 1>);
            case 2: return reinterpret_cast<const void*>(batch_gs_kernel<15, 2>);
            case 3: return reinterpret_cast<const void*>(batch_gs_kernel<15, 3>);
            case 5: return reinterpret_cast<const void*>(batch_gs_kernel<15, 5>);
            default: return nullptr;
        }
    }
    return nullptr;
}

int gs_upt_for(int nw, int64_t units) {
    const int64_t t = static_cast<int64_t>(nw) * 32;
    const int64_t need = (units + t - 1) / t;
    static const int k7[] = {2, 3, 5, 6};
    static const int k15[] = {1, 2, 3, 5};
    const int* c = nw == 7 ? k7 : k15;
    for (int i = 0; i < 4; ++i)
        if (c[i] >= need) return c[i];
    return 0;
}

constexpr int64_t kGsMaxRows = 8192;   // the Gauss-Seidel form's column limit

// Autotuned launch shapes, per batch shape, for the life of the process.
std::mutex g_tune_mu;
struct GsTuned {
    GsChoice shape;
    std::vector<int> wpick;  // block width of each problem tuned (in the order of the members)
};
std::map<std::string, GsTuned> g_gs_tuned;
std::map<std::string, int> g_w_tuned;

}  // namespace

struct asyflexa_batch_s {
    std::vector<asyflexa_t> h;
    int count = 0;
    asyflexa_opts opts{};
    cudaStream_t user_stream = nullptr;  // the caller's stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;       // own non-blocking stream: all batch work and the graph capture
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int flags = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    int64_t max_mcopy = 0;
    int cpc = 0, stages = 0, w = 0;
    size_t smem = 0;
    const void* kernel = nullptr;
    std::vector<BatchInst> h_inst;
    BatchInst* d_inst = nullptr;
    int* d_blk_inst = nullptr;
    int* d_blk_local = nullptr;
    int total_blocks = 0;
    ConvState* d_conv = nullptr;
    std::vector<ConvState> h_conv;
    int* d_round = nullptr;
    int* d_nactive = nullptr;
    unsigned long long* counters = nullptr;
    unsigned long long* hist = nullptr;
    int* err = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<void*> graph_x;
    std::vector<cudaStream_t> fin_streams;  // streams of the async finishes (created on first use)
    int graph_w = 0;
    std::vector<int> cap;  // per problem: blocks it may have in flight, max(1, m / (4 w))
    int grid = 0;          // CTAs of the next sweep launch
    int graph_grid = 0;    // CTAs of the captured round
    long long launches = 0;
    // Gauss-Seidel form
    int form = 0;                       // ASYFLEXA_BATCH_FORM_ASYNC or ASYFLEXA_BATCH_FORM_GS
    int64_t max_units = 0;              // 16-byte units of the longest column
    int64_t max_colbytes = 0;           // bytes of the longest column (its 16-byte units)
    int64_t max_multi = 0;              // bytes of kGsWMax columns of the problem with the largest lda
    float2* d_dd = nullptr;             // (d_j, 1/d_j) in FP32 of every problem, concatenated
    float* d_xsave = nullptr;           // the iterates, saved across the autotuner's sweeps
    std::vector<asyflexa::GsInst> h_gs;
    asyflexa::GsInst* d_gs = nullptr;
    int* d_order = nullptr;             // problems, largest m * n first
    int* d_order2 = nullptr;            // the problems of the second Gauss-Seidel launch
    std::vector<int> h_order;
    int* d_queue = nullptr;
    GsChoice gs{};                      // launch shape (nw == 0: not chosen yet)
    cudaGraph_t gs_graph = nullptr;
    cudaGraphExec_t gs_exec = nullptr;
    GsChoice gs_graph_cfg{};
    int smem_per_sm = 0;
    std::string shape_key;
    // multi-lane form: one problem per lane of a multi-lane handle (shared A)
    asyflexa_multi_t multi = nullptr;
    float* d_bmat = nullptr;  // count x m: the problems' b, one lane per row
    float* d_xmat = nullptr;  // count x n: the iterates, gathered for a solve
};

namespace {

int bfail(const std::string& m, int code = ASYFLEXA_EINVAL) {
    asyflexa_internal::set_thread_error(m);
    return code;
}

#define BCK(call, where)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            (void)cudaGetLastError(); /* consume a non-sticky error so later launches do not report it */ \
            return bfail(std::string(where) + ": " + cudaGetErrorString(e_), ASYFLEXA_ECUDA);          \
        }                                                                                             \
    } while (0)

const void* batched_kernel(int cpc) {
    switch (cpc) {
        case 1: return reinterpret_cast<const void*>(asyflexa::sweep_async_reg_kernel<float, 1, true>);
        case 2: return reinterpret_cast<const void*>(asyflexa::sweep_async_reg_kernel<float, 2, true>);
        case 3: return reinterpret_cast<const void*>(asyflexa::sweep_async_reg_kernel<float, 3, true>);
        case 4: return reinterpret_cast<const void*>(asyflexa::sweep_async_reg_kernel<float, 4, true>);
        case 5: return reinterpret_cast<const void*>(asyflexa::sweep_async_reg_kernel<float, 5, true>);
        case 6: return reinterpret_cast<const void*>(asyflexa::sweep_async_reg_kernel<float, 6, true>);
        default: return nullptr;
    }
}

// Global block list for width w.  Shared A: interleaved by block index, so that the
// problems' reads of the same panel are close in time.  Otherwise every problem's blocks are
// spread evenly over the list (ordered by their fractional position (b + 1/2) / nb within
// their problem), so that any window of consecutive entries -- roughly what the CTAs work on
// at the same time -- holds blocks of a problem in proportion to its size.
int build_blocks(asyflexa_batch_s& B, int w) {
    std::vector<int> bi, bl;
    std::vector<int> nb(B.count);
    int maxnb = 0;
    B.cap.assign(B.count, 1);
    for (int k = 0; k < B.count; ++k) {
        nb[k] = static_cast<int>((B.h[k]->prob.n + w - 1) / w);
        maxnb = nb[k] > maxnb ? nb[k] : maxnb;
        const int64_t c = B.h[k]->prob.m / (4 * static_cast<int64_t>(w));
        B.cap[k] = c < 1 ? 1 : static_cast<int>(c);
    }
    if (B.flags & ASYFLEXA_BATCH_SHARED_A) {
        for (int b = 0; b < maxnb; ++b)
            for (int k = 0; k < B.count; ++k)
                if (b < nb[k]) {
                    bi.push_back(k);
                    bl.push_back(b);
                }
    } else {
        struct Entry {
            double key;
            int k, b;
        };
        std::vector<Entry> all;
        for (int k = 0; k < B.count; ++k)
            for (int b = 0; b < nb[k]; ++b) all.push_back({(b + 0.5) / nb[k], k, b});
        std::stable_sort(all.begin(), all.end(), [](const Entry& a, const Entry& c) { return a.key < c.key; });
        for (const Entry& e : all) {
            bi.push_back(e.k);
            bl.push_back(e.b);
        }
    }
    if (B.d_blk_inst) cudaFree(B.d_blk_inst);
    if (B.d_blk_local) cudaFree(B.d_blk_local);
    B.d_blk_inst = B.d_blk_local = nullptr;
    B.total_blocks = static_cast<int>(bi.size());
    BCK(cudaMalloc(&B.d_blk_inst, bi.size() * sizeof(int)), "alloc block list");
    BCK(cudaMalloc(&B.d_blk_local, bl.size() * sizeof(int)), "alloc block list");
    BCK(cudaMemcpy(B.d_blk_inst, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice), "copy block list");
    BCK(cudaMemcpy(B.d_blk_local, bl.data(), bl.size() * sizeof(int), cudaMemcpyHostToDevice), "copy block list");
    for (int k = 0; k < B.count; ++k) {
        B.h_inst[k].w = w;
        B.h_inst[k].nblocks = nb[k];
    }
    B.w = w;
    return ASYFLEXA_OK;
}

int launch_batched(asyflexa_batch_s& B, int sweeps) {
    asyflexa::SweepParams p{};
    std::memset(&p, 0, sizeof p);
    p.gamma = B.opts.gamma;
    p.sweeps = sweeps;
    p.stages = B.stages;
    p.tile_rows = static_cast<int>(B.max_mcopy);
    p.counters = B.counters;
    p.hist = B.hist;
    p.err = B.err;
    p.batch = B.d_inst;
    p.blk_inst = B.d_blk_inst;
    p.blk_local = B.d_blk_local;
    p.total_blocks = B.total_blocks;
    p.keep_a_in_l2 = (B.flags & ASYFLEXA_BATCH_SHARED_A) ? 1 : 0;
    void* args[] = {&p};
    const int full = B.opts.num_ctas > 0 ? B.opts.num_ctas : B.sm_count;
    const int grid = B.grid > 0 && B.grid < full ? B.grid : full;
    const cudaError_t e =
        cudaLaunchKernel(B.kernel, dim3(grid), dim3(asyflexa::kRegThreads), args, B.smem, B.stream);
    ++B.launches;
    BCK(e, "batched sweep launch");
    return ASYFLEXA_OK;
}

// CTAs for the next rounds: at most the sum over the active problems of their in-flight
// caps, so that a few problems left running are not spread over every SM (their updates in
// flight would then be many columns for few rows; Assumption D1).
int active_grid(asyflexa_batch_s& B) {
    const int full = B.opts.num_ctas > 0 ? B.opts.num_ctas : B.sm_count;
    long long g = 0;
    for (int k = 0; k < B.count; ++k)
        if (B.h_inst[k].active) g += B.cap[k];
    return static_cast<int>(std::max<long long>(1, std::min<long long>(full, g)));
}

int upload_table(asyflexa_batch_s& B) {
    BCK(cudaMemcpyAsync(B.d_inst, B.h_inst.data(), B.count * sizeof(BatchInst), cudaMemcpyHostToDevice, B.stream),
        "upload problem table");
    return ASYFLEXA_OK;
}

// One round: the batched sweep launch, then for every problem an exact refresh and its
// objective partials, then the convergence kernel.
int enqueue_round(asyflexa_batch_s& B, void* const* xs) {
    BCK(cudaMemsetAsync(B.d_nactive, 0, sizeof(int), B.stream), "clear active count");
    int rc = launch_batched(B, B.opts.refresh_every);
    if (rc) return rc;
    for (int k = 0; k < B.count; ++k) {
        asyflexa_s& hk = *B.h[k];
        BCK(Launcher<float>::refresh(hk, xs[k]), "refresh");
        BCK(Launcher<float>::norms(hk, xs[k]), "objective");
        hk.r_valid = true;
        hk.r_x = xs[k];
        B.launches += 6;
    }
    asyflexa_batch_s* bp = &B;
    batch_converge_kernel<<<1, 256, 0, B.stream>>>(bp->d_conv, bp->d_inst, B.count, B.opts.tol_gap, B.opts.switch_tol,
                                                     B.d_round, B.d_nactive);
    ++B.launches;
    BCK(cudaGetLastError(), "convergence kernel");
    return ASYFLEXA_OK;
}


// ------------------------------------------------------------------ Gauss-Seidel form

// A problem the Gauss-Seidel launch has not finished after this many sweeps leaves it and is
// finished, from its current iterate, by a second Gauss-Seidel launch over such problems only:
// they then run side by side, under a launch shape tuned for them.
constexpr int kGsHandoffSweeps = 300;
// At most this many problems left after a launch are finished by the async solver (all of them
// side by side); with kAsyncFinishEarly false, only when the next launch would run to the budget.
constexpr int kAsyncFinishMax = 16;
constexpr bool kAsyncFinishEarly = true;

// The launch shape for nw consumer warps and ring slots of at least the longest column, with room
// for up to kGsWMax columns within slot_cap bytes: units per thread for the longest column, the
// ring depth that fits the shared memory of the CTAs an SM holds, and the grid.
int64_t gs_slot(const asyflexa_batch_s& B, int64_t slot_cap) {
    const int64_t s = std::max(B.max_colbytes, std::min(B.max_multi, slot_cap));
    return (s + 127) / 128 * 128;
}

int gs_shape(asyflexa_batch_s& B, int nw, int64_t slot_cap, GsChoice* out) {
    GsChoice c;
    c.nw = nw;
    c.upt = gs_upt_for(nw, B.max_units);
    c.kernel = c.upt ? gs_kernel(nw, c.upt) : nullptr;
    if (!c.kernel) return ASYFLEXA_EUNSUPPORTED;
    const int want_per_sm = nw < 8 ? 2 : 1;
    const size_t slot_bytes = static_cast<size_t>(gs_slot(B, slot_cap));
    const asyflexa::GsLayout L0 = asyflexa::make_gs_layout(nw, slot_bytes, 0);
    const size_t budget = std::min<size_t>(B.smem_optin, static_cast<size_t>(B.smem_per_sm) / want_per_sm - 1024);
    if (L0.total + 2 * (L0.slot_bytes + 16) > budget) return ASYFLEXA_EUNSUPPORTED;
    int stages = static_cast<int>((budget - L0.total - 256) / (L0.slot_bytes + 16));
    stages = std::max(2, std::min(16, stages));
    while (stages > 2 && asyflexa::make_gs_layout(nw, slot_bytes, stages).total > budget) --stages;
    c.stages = stages;
    c.slot_cap = slot_cap;
    c.slot_bytes = static_cast<int64_t>(slot_bytes);
    c.smem = asyflexa::make_gs_layout(nw, slot_bytes, stages).total;
    // the opt-in maximum: launch shapes of one kernel differ in their shared memory
    BCK(cudaFuncSetAttribute(c.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(B.smem_optin)),
        "GS kernel shared-memory attribute");
    int per_sm = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c.kernel, (nw + 1) * 32, c.smem), "GS occupancy");
    if (per_sm < 1) return ASYFLEXA_EUNSUPPORTED;
    c.ctas_per_sm = per_sm;
    long long g = static_cast<long long>(per_sm) * B.sm_count;
    if (B.opts.num_ctas > 0) g = std::min<long long>(g, B.opts.num_ctas);
    c.grid = static_cast<int>(std::max<long long>(1, std::min<long long>(g, B.count)));
    *out = c;
    return ASYFLEXA_OK;
}

// One launch of the Gauss-Seidel kernel over the problems order[0 .. cnt) (device array; the
// queue is reset first).
int gs_enqueue(asyflexa_batch_s& B, const GsChoice& c, int sweeps_only, int max_sweeps, int handoff,
               const int* order, int cnt) {
    asyflexa::GsParams p{};
    p.inst = B.d_gs;
    p.order = order;
    p.count = cnt;
    p.queue = B.d_queue;
    p.gamma = B.opts.gamma;
    p.tol_gap = B.opts.tol_gap;
    p.tol_stat = B.opts.tol_stat;
    p.check_every = B.opts.check_every;
    p.max_sweeps = max_sweeps;
    p.stages = c.stages;
    p.w = c.w;
    p.slot_bytes = c.slot_bytes;
    p.sweeps_only = sweeps_only;
    p.handoff_sweeps = handoff;
    p.keep_a_in_l2 = (B.flags & ASYFLEXA_BATCH_SHARED_A) ? 1 : 0;
    p.err = B.err;
    BCK(cudaMemsetAsync(B.d_queue, 0, sizeof(int), B.stream), "reset queue");
    void* args[] = {&p};
    const int grid = std::max(1, std::min(c.grid, cnt));
    const cudaError_t e = cudaLaunchKernel(c.kernel, dim3(grid), dim3((c.nw + 1) * 32), args, c.smem, B.stream);
    ++B.launches;
    BCK(e, "GS batch launch");
    return ASYFLEXA_OK;
}

// Block width of the Gauss-Seidel form: opts.block_w in 1 .. kGsWMax fixes it, any other value
// lets the autotuner pick it from {1, 2, 4, 8}.  Ring slots hold up to kGsWMax columns within
// 16 KB, or (wider blocks of the longer columns, fewer stages) within 32 KB.
bool gs_fixed_w(const asyflexa_batch_s& B) { return B.opts.block_w >= 1 && B.opts.block_w <= asyflexa::kGsWMax; }

// The launch shape of the Gauss-Seidel form for the problems order[0 .. cnt) (members: their
// indices), and each member's block width (B.h_gs[k].wpick; the caller uploads the table):
// cached under `key`, else tuned.  Launch shapes: 7 or 15 consumer warps per CTA with 16 KB ring
// slots (widths 1, 2, 4) or 32 KB slots (widths 4, 8); opts.block_w in 1 .. kGsWMax fixes the
// width.  Every (shape, width) pair is timed over one sweep of the members, from their iterates,
// which are restored after each; every CTA times its problem.  Each member takes its fastest
// width under a shape, and the shape chosen minimises the summed times of the members (use_max
// = false: the GPU time the sweeps take, for a whole batch) or the largest one (use_max = true:
// for a few problems left over, which run side by side).  The device table must hold wpick = 0
// for the members.
int gs_choose(asyflexa_batch_s& B, const int* order, int cnt, const std::vector<int>& members, const std::string& key,
              bool use_max, GsChoice* out) {
    const size_t nm = members.size();
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto itc = g_gs_tuned.find(key);
        if (itc != g_gs_tuned.end() && itc->second.wpick.size() == nm) {
            const int rc = gs_shape(B, itc->second.shape.nw, itc->second.shape.slot_cap, out);
            if (rc == ASYFLEXA_OK) {
                out->w = itc->second.shape.w;
                for (size_t i = 0; i < nm; ++i) B.h_gs[members[i]].wpick = itc->second.wpick[i];
                return ASYFLEXA_OK;
            }
        }
    }
    struct Shape {
        GsChoice c;
        std::vector<int> widths;
    };
    std::vector<Shape> shapes;
    size_t ncand = 0;
    for (int nw : {7, 15})
        for (int64_t cap : {int64_t{16384}, int64_t{32768}}) {
            Shape sh;
            if (cap > 16384 && gs_slot(B, cap) == gs_slot(B, 16384)) continue;  // the same slots
            if (gs_shape(B, nw, cap, &sh.c) != ASYFLEXA_OK) continue;
            if (gs_fixed_w(B))
                sh.widths = {B.opts.block_w};
            else if (cap > 16384)
                sh.widths = {4, 8};
            else
                sh.widths = {1, 2, 4};
            ncand += sh.widths.size();
            shapes.push_back(sh);
        }
    if (shapes.empty()) return bfail("batched problems: no Gauss-Seidel launch shape fits", ASYFLEXA_EUNSUPPORTED);
    std::vector<int> pick(nm, shapes[0].widths[0]);
    *out = shapes[0].c;
    out->w = shapes[0].widths[0];
    if (ncand > 1) {
        double best = 0.0;
        std::vector<asyflexa::GsInst> tmp(B.count);
        const int cgrid = std::max(1, std::min(cnt, 4 * B.sm_count));
        gs_copy_x_kernel<<<cgrid, 256, 0, B.stream>>>(B.d_gs, order, cnt, B.d_dd, B.d_xsave, 1);
        ++B.launches;
        BCK(cudaGetLastError(), "save iterates");
        for (Shape& sh : shapes) {
            std::vector<double> fastest(nm, 0.0);
            std::vector<int> wbest(nm, sh.widths[0]);
            for (int w : sh.widths) {
                GsChoice c = sh.c;
                c.w = w;
                int rc = gs_enqueue(B, c, 1, 1, 0, order, cnt);
                if (rc) return rc;
                gs_copy_x_kernel<<<cgrid, 256, 0, B.stream>>>(B.d_gs, order, cnt, B.d_dd, B.d_xsave, 0);
                ++B.launches;
                BCK(cudaGetLastError(), "restore iterates");
                BCK(cudaMemcpyAsync(tmp.data(), B.d_gs, B.count * sizeof(asyflexa::GsInst), cudaMemcpyDeviceToHost,
                                    B.stream),
                    "read problem table");
                BCK(cudaStreamSynchronize(B.stream), "synchronize");
                for (size_t i = 0; i < nm; ++i) {
                    const double t = static_cast<double>(tmp[members[i]].ns);
                    if (fastest[i] == 0.0 || t < fastest[i]) {
                        fastest[i] = t;
                        wbest[i] = w;
                    }
                }
            }
            double obj = 0.0;
            for (size_t i = 0; i < nm; ++i) obj = use_max ? std::max(obj, fastest[i]) : obj + fastest[i];
            if (best == 0.0 || obj < best) {
                best = obj;
                *out = sh.c;
                pick = wbest;
            }
        }
        // the launch's own width: the one most members take
        int most = 0, nmost = -1;
        for (int w = 1; w <= asyflexa::kGsWMax; ++w) {
            const int c = static_cast<int>(std::count(pick.begin(), pick.end(), w));
            if (c > nmost) {
                nmost = c;
                most = w;
            }
        }
        out->w = most;
    }
    for (size_t i = 0; i < nm; ++i) B.h_gs[members[i]].wpick = pick[i];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_gs_tuned[key] = GsTuned{*out, pick};
    return ASYFLEXA_OK;
}

int gs_solve(asyflexa_batch_s& B, void* const* xs, const double* f_star, asyflexa_stats* per, asyflexa_stats* total) {
    const int count = B.count;
    for (int k = 0; k < count; ++k) {
        asyflexa::GsInst& g = B.h_gs[k];
        g.x = static_cast<float*>(xs[k]);
        g.f_star = f_star ? f_star[k] : NAN;
        g.F = g.stat = g.xmax = NAN;
        g.sweeps = g.nnz = 0;
        g.status = ASYFLEXA_ENOTCONV;
        g.checks = 0;
        g.wpick = 0;
    }
    auto upload = [&]() -> int {
        BCK(cudaMemcpyAsync(B.d_gs, B.h_gs.data(), count * sizeof(asyflexa::GsInst), cudaMemcpyHostToDevice,
                            B.stream),
            "upload problem table");
        return ASYFLEXA_OK;
    };
    int rc = upload();
    if (rc) return rc;
    EventPair ev_e0;
    BCK(cudaEventCreate(&ev_e0.a), "event");
    BCK(cudaEventCreate(&ev_e0.b), "event");
    cudaEvent_t e0 = ev_e0.a, e1 = ev_e0.b;
    BCK(cudaEventRecord(e0, B.stream), "event record");
    std::vector<int> all(count);
    for (int k = 0; k < count; ++k) all[k] = k;
    rc = gs_choose(B, B.d_order, count, all, B.shape_key, false, &B.gs);
    if (!rc) rc = upload();  // the widths picked
    if (rc) return rc;
    const int budget = B.opts.max_sweeps;
    const int handoff = budget > 2 * kGsHandoffSweeps ? kGsHandoffSweeps : 0;
    // the first launch as a CUDA graph (re-captured when the launch shape or budget changes)
    GsChoice key = B.gs;
    key.stages = B.gs.stages * 100000 + budget;  // the budget is a kernel argument
    key.grid = B.gs.grid * 1000 + handoff;
    if (!B.gs_exec || !(B.gs_graph_cfg == key)) {
        if (B.gs_exec) cudaGraphExecDestroy(B.gs_exec);
        if (B.gs_graph) cudaGraphDestroy(B.gs_graph);
        B.gs_exec = nullptr;
        B.gs_graph = nullptr;
        BCK(cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int erc = gs_enqueue(B, B.gs, 0, budget, handoff, B.d_order, count);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(B.stream, &g);
        if (erc) return erc;
        BCK(ce, "end capture");
        B.gs_graph = g;
        BCK(cudaGraphInstantiate(&B.gs_exec, g, 0), "instantiate graph");
        B.gs_graph_cfg = key;
    }
    BCK(cudaGraphLaunch(B.gs_exec, B.stream), "graph launch");
    BCK(cudaMemcpyAsync(B.h_gs.data(), B.d_gs, count * sizeof(asyflexa::GsInst), cudaMemcpyDeviceToHost, B.stream),
        "read problem table");
    BCK(cudaStreamSynchronize(B.stream), "synchronize");
    int errw = 0;
    BCK(cudaMemcpy(&errw, B.err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (errw) return bfail("a bounded device-side wait expired", ASYFLEXA_ETIMEOUT);
    // Problems still short of their tolerances after a launch's handoff sweeps continue from their
    // iterates in a further launch over them alone, under a launch shape tuned for them, with
    // twice the handoff sweeps (so that the last few problems end up with a shape of their own).
    std::vector<long long> done_sw(count), done_ns(count);
    std::vector<int> extra(count, 0);               // further launches each problem ran in
    std::vector<GsChoice> shape_of(count, B.gs);   // the launch that finished it
    std::vector<char> async_fin(count, 0);         // finished by the single-problem async solver
    for (int k = 0; k < count; ++k) {
        done_sw[k] = B.h_gs[k].sweeps;
        done_ns[k] = B.h_gs[k].ns;
    }
    int hand = handoff;
    for (int round = 1;; ++round) {
        std::vector<int> rest;
        long long done_max = 0;
        for (int k : B.h_order)
            if (B.h_gs[k].status == asyflexa::kGsHandoff) {
                rest.push_back(k);
                done_max = std::max(done_max, done_sw[k]);
            }
        if (rest.empty()) break;
        const int nrest = static_cast<int>(rest.size());
        const int budget2 = static_cast<int>(std::max<long long>(0, budget - done_max));
        hand *= 2;
        const int handoff2 = budget2 > 2 * hand ? hand : 0;
        if (nrest <= kAsyncFinishMax && (handoff2 == 0 || kAsyncFinishEarly)) {
            // The few problems left would each hold one SM while the others idle: they are
            // finished side by side, each by the single-problem async solver on a stream of its
            // own, with max(1, m / (2 w)) CTAs (about m / 2 columns in flight; each stops on the
            // solver's exact check).  The async kernels have no waits between CTAs, so the solves
            // need not be resident together.
            BCK(cudaStreamSynchronize(B.stream), "synchronize");
            while (static_cast<int>(B.fin_streams.size()) < nrest) {
                cudaStream_t fs = nullptr;
                BCK(cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking), "finish stream");
                B.fin_streams.push_back(fs);
            }
            std::vector<asyflexa_opts> saved(nrest);
            std::vector<int> saved_ctas(nrest), src(nrest, ASYFLEXA_OK);
            std::vector<cudaStream_t> saved_stream(nrest);
            std::vector<asyflexa_stats> sts(nrest);
            for (int i = 0; i < nrest; ++i) {
                const int k = rest[i];
                asyflexa_s& hk = *B.h[k];
                saved[i] = hk.opts;
                saved_ctas[i] = hk.sweep_ctas;
                saved_stream[i] = hk.stream;
                hk.opts.max_sweeps = static_cast<int>(std::max<long long>(1, budget - done_sw[k]));
                hk.opts.f_star = f_star ? f_star[k] : NAN;
                hk.sweep_ctas = static_cast<int>(std::max<int64_t>(
                    1, std::min<int64_t>({static_cast<int64_t>(hk.nblocks), static_cast<int64_t>(hk.sm_count),
                                          hk.prob.m / (2 * static_cast<int64_t>(hk.opts.block_w))})));
                hk.stream = B.fin_streams[i];
                hk.r_valid = false;
                std::memset(&sts[i], 0, sizeof sts[i]);
            }
            // (a new host thread starts on device 0: it is moved to the batch's device; the
            // calling thread's current device is left as it is)
            auto finish = [&](int i, bool worker) {
                const int k = rest[i];
                if (worker && cudaSetDevice(B.h[k]->device) != cudaSuccess) {
                    src[i] = ASYFLEXA_ECUDA;
                    return;
                }
                src[i] = asyflexa_solve(B.h[k], xs[k], &sts[i]);
            };
            {
                std::vector<std::thread> th;
                int next = 1;  // problem 0 runs on this thread; the others on threads of their own
                try {
                    for (; next < nrest; ++next) th.emplace_back(finish, next, true);
                } catch (...) {
                }
                finish(0, false);
                for (auto& t : th) t.join();
                for (int i = next; i < nrest; ++i) finish(i, false);  // threads that could not be started
            }
            for (int i = 0; i < nrest; ++i) {
                asyflexa_s& hk = *B.h[rest[i]];
                hk.opts = saved[i];
                hk.sweep_ctas = saved_ctas[i];
                hk.stream = saved_stream[i];
            }
            for (int i = 0; i < nrest; ++i) {
                const int k = rest[i];
                if (src[i] < 0 && src[i] != ASYFLEXA_ENONFINITE)
                    return bfail("problem " + std::to_string(k) + ", async finish: " + B.h[k]->msg, src[i]);
                const asyflexa_stats& st = sts[i];
                asyflexa::GsInst& g = B.h_gs[k];
                g.F = st.F;
                g.stat = st.stat_xhat;
                g.nnz = st.nnz;
                g.status = src[i] == ASYFLEXA_ENONFINITE ? ASYFLEXA_ENONFINITE : st.status;
                g.checks = 1;
                g.w_used = B.h[k]->opts.block_w;
                done_sw[k] += st.sweeps;
                done_ns[k] += static_cast<long long>(st.seconds * 1e9);
                ++extra[k];
                shape_of[k] = GsChoice{};  // not a Gauss-Seidel launch
                async_fin[k] = 1;
            }
            break;
        }
        BCK(cudaMemcpyAsync(B.d_order2, rest.data(), nrest * sizeof(int), cudaMemcpyHostToDevice, B.stream),
            "upload order");
        std::string key2 = B.shape_key + " round=" + std::to_string(round) + " of";
        for (int k : rest) key2 += " " + std::to_string(k);
        for (int k : rest) B.h_gs[k].wpick = 0;
        GsChoice c2;
        rc = upload();
        if (!rc) rc = gs_choose(B, B.d_order2, nrest, rest, key2, true, &c2);
        if (!rc) rc = upload();
        if (!rc) rc = gs_enqueue(B, c2, 0, budget2, handoff2, B.d_order2, nrest);
        if (rc) return rc;
        std::vector<asyflexa::GsInst> tmp(count);
        BCK(cudaMemcpyAsync(tmp.data(), B.d_gs, count * sizeof(asyflexa::GsInst), cudaMemcpyDeviceToHost, B.stream),
            "read problem table");
        BCK(cudaStreamSynchronize(B.stream), "synchronize");
        errw = 0;
        BCK(cudaMemcpy(&errw, B.err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
        if (errw) return bfail("a bounded device-side wait expired", ASYFLEXA_ETIMEOUT);
        for (int k : rest) {
            B.h_gs[k] = tmp[k];
            done_sw[k] += tmp[k].sweeps;
            done_ns[k] += tmp[k].ns;
            ++extra[k];
            shape_of[k] = c2;
        }
    }
    BCK(cudaEventRecord(e1, B.stream), "event record");
    BCK(cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long bu = 0, max_sweeps = 0;
    int nhanded = 0;
    int worst = ASYFLEXA_OK;
    for (int k = 0; k < count; ++k) {
        const asyflexa::GsInst& g = B.h_gs[k];
        const long long sw = done_sw[k];  // over every launch the problem ran in
        nhanded += extra[k] > 0 ? 1 : 0;
        bu += sw * g.n;
        max_sweeps = std::max(max_sweeps, sw);
        const int st = g.status;
        if (st != ASYFLEXA_OK && (worst == ASYFLEXA_OK || st < 0)) worst = st;
        if (per) {
            asyflexa_stats s;
            std::memset(&s, 0, sizeof s);
            s.F = g.F;
            s.rel_gap = std::isfinite(g.f_star) ? (g.F - g.f_star) / std::fabs(g.f_star) : NAN;
            s.stat_xhat = g.stat;
            s.stat_mf = NAN;
            s.kkt_viol = NAN;
            s.dual_gap = NAN;
            s.nnz = g.nnz;
            s.sweeps = sw;
            s.block_updates = sw * g.n;
            s.status = st;
            s.checked = g.checks > 0 ? 1 : 0;
            s.block_w = g.w_used;
            s.seconds = 1e-9 * static_cast<double>(done_ns[k]);
            s.batch_form = async_fin[k] ? ASYFLEXA_BATCH_FORM_ASYNC : ASYFLEXA_BATCH_FORM_GS;
            s.ctas_per_sm = shape_of[k].ctas_per_sm;
            s.kernel_variant = shape_of[k].nw;
            s.handed_over = extra[k];
            per[k] = s;
        }
    }
    if (total) {
        std::memset(total, 0, sizeof *total);
        total->sweeps = max_sweeps;
        total->block_updates = bu;
        total->seconds = ms * 1e-3;
        total->status = worst;
        total->kernel_launches = B.launches;
        total->block_w = B.gs.w;
        total->handed_over = nhanded;
        total->batch_form = ASYFLEXA_BATCH_FORM_GS;
        total->ctas_per_sm = B.gs.ctas_per_sm;
        total->kernel_variant = B.gs.nw;
    }
    return worst;
}


// The multi-lane form: the problems' iterates gathered into the lanes of the multi-lane handle,
// solved, and scattered back.
int multi_form_solve(asyflexa_batch_s& B, void* const* xs, const double* f_star, asyflexa_stats* per,
                     asyflexa_stats* total) {
    const int64_t n = B.h[0]->prob.n;
    for (int k = 0; k < B.count; ++k)
        BCK(cudaMemcpyAsync(B.d_xmat + k * n, xs[k], n * sizeof(float), cudaMemcpyDeviceToDevice, B.stream),
            "gather iterates");
    const int rc = asyflexa_multi_solve(B.multi, B.d_xmat, n, f_star, per, total);
    if (rc < 0) return rc;
    for (int k = 0; k < B.count; ++k)
        BCK(cudaMemcpyAsync(xs[k], B.d_xmat + k * n, n * sizeof(float), cudaMemcpyDeviceToDevice, B.stream),
            "scatter iterates");
    BCK(cudaStreamSynchronize(B.stream), "synchronize");
    if (per)
        for (int k = 0; k < B.count; ++k) per[k].batch_form = ASYFLEXA_BATCH_FORM_MULTI;
    if (total) total->batch_form = ASYFLEXA_BATCH_FORM_MULTI;
    return rc;
}

int rounds_solve(asyflexa_batch_s& Bref, void* const* xs, const double* f_star, asyflexa_stats* per,
                 asyflexa_stats* total) {
    asyflexa_batch_s* B = &Bref;
    const long long budget = B->opts.max_sweeps;
    const int count = B->count;
    EventPair ev_e0;
    BCK(cudaEventCreate(&ev_e0.a), "event");
    BCK(cudaEventCreate(&ev_e0.b), "event");
    cudaEvent_t e0 = ev_e0.a, e1 = ev_e0.b;
    BCK(cudaEventRecord(e0, B->stream), "event record");
    // reset problem states for these iterates
    for (int k = 0; k < count; ++k) {
        B->h_inst[k].x = xs[k];
        B->h_inst[k].active = 1;
        ConvState& c = B->h_conv[k];
        c.f_star = f_star ? f_star[k] : NAN;
        c.F = c.F_prev = NAN;
        c.conv_round = -2;
    }
    B->grid = 0;  // every problem active again: full grid until the first deactivation
    int rc = upload_table(*B);
    if (rc) return rc;
    BCK(cudaMemcpyAsync(B->d_conv, B->h_conv.data(), count * sizeof(ConvState), cudaMemcpyHostToDevice, B->stream),
        "upload convergence state");
    BCK(cudaMemsetAsync(B->d_round, 0, sizeof(int), B->stream), "clear round");
    for (int k = 0; k < count; ++k) {
        BCK(Launcher<float>::refresh(*B->h[k], xs[k]), "initial refresh");
        B->launches += 4;
    }
    long long sweeps = 0;
    // autotuner: time one sweep per candidate block width (these are real sweeps); the choice
    // is cached per batch shape
    if (B->opts.block_w == 0 && B->graph_w == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto itw = g_w_tuned.find(B->shape_key);
        if (itw != g_w_tuned.end()) {
            rc = build_blocks(*B, itw->second);
            if (!rc) rc = upload_table(*B);
            if (rc) return rc;
            B->graph_w = itw->second;
        }
    }
    if (B->opts.block_w == 0 && B->graph_w == 0) {
        float best = 0.f;
        int best_w = 32;
        EventPair ev_a0;
        BCK(cudaEventCreate(&ev_a0.a), "event");
        BCK(cudaEventCreate(&ev_a0.b), "event");
        cudaEvent_t a0 = ev_a0.a, a1 = ev_a0.b;
        for (int w : kCandidates) {
            rc = build_blocks(*B, w);
            if (!rc) rc = upload_table(*B);
            if (rc) return rc;
            BCK(cudaEventRecord(a0, B->stream), "event record");
            rc = launch_batched(*B, 1);
            if (rc) return rc;
            BCK(cudaEventRecord(a1, B->stream), "event record");
            BCK(cudaEventSynchronize(a1), "event sync");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a0, a1);
            if (best == 0.f || ms < best) {
                best = ms;
                best_w = w;
            }
            ++sweeps;
        }
        rc = build_blocks(*B, best_w);
        if (!rc) rc = upload_table(*B);
        if (rc) return rc;
        for (int k = 0; k < count; ++k) {
                BCK(Launcher<float>::refresh(*B->h[k], xs[k]), "refresh after autotune");
            B->launches += 4;
        }
        B->graph_w = best_w;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_w_tuned[B->shape_key] = best_w;
    }
    // one round as a CUDA graph, re-captured when the iterates, the width or the grid change
    std::vector<void*> xv(xs, xs + count);
    auto capture = [&]() -> int {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        B->exec = nullptr;
        B->graph = nullptr;
        BCK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const int erc = enqueue_round(*B, xs);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(B->stream, &g);
        if (erc) return erc;
        BCK(ce, "end capture");
        B->graph = g;
        BCK(cudaGraphInstantiate(&B->exec, g, 0), "instantiate graph");
        B->graph_x = xv;
        B->graph_w = B->w;
        B->graph_grid = B->grid;
        return ASYFLEXA_OK;
    };
    B->grid = active_grid(*B);
    if (!B->exec || B->graph_x != xv || B->graph_w != B->w || B->graph_grid != B->grid) {
        rc = capture();
        if (rc) return rc;
    }
    const int per_round = B->opts.refresh_every;
    int n_active = 0;
    n_active = count;
    int last_active = n_active;
    // exact check of each problem at its returned x: computed when it leaves the rounds
    std::vector<asyflexa_stats> checked(count);
    std::vector<char> have(count, 0);
    for (;;) {
        while (sweeps < budget && n_active > 0) {
            BCK(cudaGraphLaunch(B->exec, B->stream), "graph launch");
            sweeps += per_round;
            BCK(cudaMemcpyAsync(&n_active, B->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, B->stream),
                "read count");
            BCK(cudaStreamSynchronize(B->stream), "synchronize");
            int errw = 0;
            BCK(cudaMemcpy(&errw, B->err, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
            if (errw) return bfail("a bounded device-side wait expired", ASYFLEXA_ETIMEOUT);
            if (n_active > 0 && n_active < last_active) {
                // problems were deactivated on the device: shrink the grid to the active ones
                last_active = n_active;
                BCK(cudaMemcpy(B->h_inst.data(), B->d_inst, count * sizeof(BatchInst), cudaMemcpyDeviceToHost),
                    "read problem table");
                const int g = active_grid(*B);
                if (g < B->graph_grid) {
                    B->grid = g;
                    rc = capture();
                    if (rc) return rc;
                }
            }
        }
        // the problems that left the rounds: exact stationarity check; those above tol_stat
        // rejoin the rounds
        BCK(cudaMemcpy(B->h_conv.data(), B->d_conv, count * sizeof(ConvState), cudaMemcpyDeviceToHost),
            "read state");
        BCK(cudaMemcpy(B->h_inst.data(), B->d_inst, count * sizeof(BatchInst), cudaMemcpyDeviceToHost),
            "read problem table");
        int back = 0;
        for (int k = 0; k < count; ++k) {
            ConvState& c = B->h_conv[k];
            if (c.conv_round < 0 || have[k]) continue;
            asyflexa_stats st;
            std::memset(&st, 0, sizeof st);
            B->h[k]->opts.f_star = c.f_star;
            const int crc = asyflexa_check(B->h[k], xs[k], &st);
            B->launches += 8;
            st.status = crc;
            if (!crc && !(st.stat_xhat <= B->opts.tol_stat) && sweeps < budget) {
                c.conv_round = -2;
                c.F_prev = NAN;
                B->h_inst[k].active = 1;
                ++back;
            } else {
                checked[k] = st;
                have[k] = 1;
            }
        }
        if (back == 0) break;
        BCK(cudaMemcpyAsync(B->d_conv, B->h_conv.data(), count * sizeof(ConvState), cudaMemcpyHostToDevice,
                            B->stream),
            "upload convergence state");
        rc = upload_table(*B);
        if (rc) return rc;
        n_active = back;
        last_active = back;
        B->grid = active_grid(*B);
        rc = capture();
        if (rc) return rc;
    }
    BCK(cudaEventRecord(e1, B->stream), "event record");
    BCK(cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long bu = 0, max_k = 0;
    int worst = ASYFLEXA_OK;
    for (int k = 0; k < count; ++k) {
        const ConvState& c = B->h_conv[k];
        const long long nb = (B->h[k]->prob.n + B->w - 1) / B->w;
        const long long ksweeps = c.conv_round >= 0 ? static_cast<long long>(c.conv_round + 1) * per_round : sweeps;
        bu += nb * ksweeps;
        max_k = std::max(max_k, ksweeps);
        int st = c.conv_round >= 0 ? ASYFLEXA_OK : (c.conv_round == -1 ? ASYFLEXA_ENONFINITE : ASYFLEXA_ENOTCONV);
        if (have[k] && checked[k].status) st = checked[k].status;
        if (have[k] && !checked[k].status && !(checked[k].stat_xhat <= B->opts.tol_stat)) st = ASYFLEXA_ENOTCONV;
        if (per) {
            asyflexa_stats s;
            std::memset(&s, 0, sizeof s);
            if (have[k]) {
                s = checked[k];
            } else {
                B->h[k]->opts.f_star = c.f_star;
                const int crc = asyflexa_check(B->h[k], xs[k], &s);
                if (crc) st = crc;
            }
            s.sweeps = ksweeps;
            s.block_updates = nb * ksweeps;
            s.status = st;
            s.block_w = B->w;
            s.batch_form = ASYFLEXA_BATCH_FORM_ASYNC;
            per[k] = s;
        }
        if (st != ASYFLEXA_OK && (worst == ASYFLEXA_OK || st < 0)) worst = st;
    }
    if (total) {
        std::memset(total, 0, sizeof *total);
        total->sweeps = sweeps;
        total->block_updates = bu;
        total->seconds = ms * 1e-3;
        total->status = worst;
        total->kernel_launches = B->launches;
        total->block_w = B->w;
        total->batch_form = ASYFLEXA_BATCH_FORM_ASYNC;
    }
    return worst;
}



}  // namespace

extern "C" {

int asyflexa_batch_create(asyflexa_batch_t* out, const asyflexa_problem* probs, int32_t count,
                          const asyflexa_opts* opts, int32_t flags, void* stream) {
    if (!out) return bfail("out is NULL");
    *out = nullptr;
    if (!probs || !opts || count < 1) return bfail("probs/opts NULL or count < 1");
    if (opts->block_w < 0 || opts->block_w > asyflexa::kWMax) return bfail("block_w must be 0 (autotune) or 1..128");
    auto* B = new (std::nothrow) asyflexa_batch_s();
    if (!B) return bfail("host allocation failed", ASYFLEXA_ENOMEM);
    B->count = count;
    B->opts = *opts;
    B->flags = flags;
    B->user_stream = static_cast<cudaStream_t>(stream);
    auto fail = [&](int rc) {
        asyflexa_batch_destroy(B);
        return rc;
    };
    {
        // Graph capture is not possible on the legacy default stream, so the batch runs on a
        // stream of its own, ordered after the caller's stream by an event.
        cudaError_t e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(B->ev_in, B->user_stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, B->ev_in, 0);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(bfail(std::string("batch stream: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
        }
    }
    asyflexa_opts io = *opts;
    io.mode = ASYFLEXA_ASYNC;
    io.block_w = opts->block_w > 0 ? opts->block_w : 32;
    io.profile = 0;
    io.exact_grad = 0;  // the batched kernel accumulates in FP32
    for (int k = 0; k < count; ++k) {
        if (probs[k].a_dtype != ASYFLEXA_F32 || probs[k].A_master)
            return fail(bfail("batched problems use FP32 storage (problem " + std::to_string(k) + ")"));
        if (probs[k].loss != ASYFLEXA_LOSS_LASSO && probs[k].loss != ASYFLEXA_LOSS_NCQUAD)
            return fail(bfail("batched problems use the LASSO or NCQUAD loss (problem " + std::to_string(k) + ")",
                              ASYFLEXA_EUNSUPPORTED));
        asyflexa_t hk = nullptr;
        const int rc = asyflexa_create(&hk, &probs[k], &io, B->stream);
        if (rc) return fail(bfail("problem " + std::to_string(k) + ": " + asyflexa_last_error(nullptr), rc));
        B->h.push_back(hk);
        if (hk->mcopy > B->max_mcopy) B->max_mcopy = hk->mcopy;
    }
    B->sm_count = B->h[0]->sm_count;
    B->smem_optin = B->h[0]->smem_optin;
    {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, B->h[0]->device);
        B->smem_per_sm = v > 0 ? v : static_cast<int>(B->smem_optin);
    }
    const int64_t units = B->max_mcopy / 4;
    B->max_units = units;
    // the form: forced by the flags, else the Gauss-Seidel form when every problem fits it and
    // there are enough problems to occupy a good part of the GPU one CTA each
    {
        const bool gs_fits = B->max_mcopy <= kGsMaxRows;  // (15 warps x 5 units x 4 rows = 9600)
        const int forms = ((flags & ASYFLEXA_BATCH_FORM_GS) ? 1 : 0) + ((flags & ASYFLEXA_BATCH_FORM_ASYNC) ? 1 : 0) +
                          ((flags & ASYFLEXA_BATCH_FORM_MULTI) ? 1 : 0);
        if (forms > 1) return fail(bfail("at most one ASYFLEXA_BATCH_FORM_* flag"));
        // the multi-lane form fits a lambda path or several data vectors: shared A, LASSO, no
        // box or linear term, at most 64 problems
        bool multi_fits = count <= 64;
        for (int k = 0; k < count && multi_fits; ++k) {
            const asyflexa_problem& q = probs[k];
            multi_fits = q.A == probs[0].A && q.lda == probs[0].lda && q.m == probs[0].m && q.n == probs[0].n &&
                         q.loss == ASYFLEXA_LOSS_LASSO && q.x_dtype == ASYFLEXA_F32 && !q.lo && !q.hi && !q.lin;
        }
        if (flags & ASYFLEXA_BATCH_FORM_MULTI) {
            if (!multi_fits)
                return fail(bfail("the multi-lane form needs at most 64 LASSO problems sharing A, without box or "
                                  "linear term", ASYFLEXA_EUNSUPPORTED));
            B->form = ASYFLEXA_BATCH_FORM_MULTI;
        } else if (flags & ASYFLEXA_BATCH_FORM_GS) {
            if (!gs_fits)
                return fail(bfail("the Gauss-Seidel form needs m <= 8192 for every problem", ASYFLEXA_EUNSUPPORTED));
            B->form = ASYFLEXA_BATCH_FORM_GS;
        } else if (flags & ASYFLEXA_BATCH_FORM_ASYNC) {
            B->form = ASYFLEXA_BATCH_FORM_ASYNC;
        } else if (multi_fits && (flags & ASYFLEXA_BATCH_SHARED_A) && count > 1) {
            B->form = ASYFLEXA_BATCH_FORM_MULTI;
        } else {
            B->form = (gs_fits && count >= B->sm_count) ? ASYFLEXA_BATCH_FORM_GS : ASYFLEXA_BATCH_FORM_ASYNC;
        }
    }
    if (B->form == ASYFLEXA_BATCH_FORM_MULTI) {
        const int64_t m = probs[0].m, n = probs[0].n;
        cudaError_t e = cudaMalloc(&B->d_bmat, static_cast<size_t>(count) * m * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&B->d_xmat, static_cast<size_t>(count) * n * sizeof(float));
        for (int k = 0; k < count && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(B->d_bmat + k * m, probs[k].b, m * sizeof(float), cudaMemcpyDeviceToDevice, B->stream);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(bfail(std::string("batch allocation: ") + cudaGetErrorString(e), ASYFLEXA_ENOMEM));
        }
        std::vector<double> lams(count);
        for (int k = 0; k < count; ++k) lams[k] = probs[k].lambda;
        asyflexa_problem p0 = probs[0];
        p0.b = B->d_bmat;
        const int rc = asyflexa_multi_create(&B->multi, &p0, count, B->d_bmat, m, lams.data(), opts, B->stream);
        if (rc) return fail(rc);
        e = cudaEventRecord(B->ev_out, B->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->user_stream, B->ev_out, 0);
        if (e != cudaSuccess) return fail(bfail(std::string("batch set-up: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
        *out = B;
        return ASYFLEXA_OK;
    }
    B->cpc = static_cast<int>((units + asyflexa::kRegStageUnits - 1) / asyflexa::kRegStageUnits);
    B->kernel = batched_kernel(B->cpc);
    if (!B->kernel) return fail(bfail("batched problems need m <= 24576", ASYFLEXA_EUNSUPPORTED));
    const asyflexa::RegLayout L0 = asyflexa::make_reg_layout(static_cast<int>(B->max_mcopy), 0);
    if (L0.total + 512 + static_cast<size_t>(B->cpc + 1) * L0.stage_bytes > B->smem_optin)
        return fail(bfail("batched problems: m too large for shared memory", ASYFLEXA_EUNSUPPORTED));
    int stages = static_cast<int>((B->smem_optin - L0.total - 512) / L0.stage_bytes);
    B->stages = stages > 16 ? 16 : stages;
    B->smem = asyflexa::make_reg_layout(static_cast<int>(B->max_mcopy), B->stages).total;
    {
        cudaError_t e = cudaFuncSetAttribute(B->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(B->smem_optin));
        if (e != cudaSuccess) return fail(bfail(std::string("smem attribute: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
    }
    B->h_inst.resize(count);
    B->h_conv.resize(count);
    for (int k = 0; k < count; ++k) {
        const asyflexa_s& hk = *B->h[k];
        BatchInst& I = B->h_inst[k];
        std::memset(&I, 0, sizeof I);
        I.A = hk.prob.A;
        I.lda = hk.prob.lda;
        I.m = hk.prob.m;
        I.mcopy = hk.mcopy;
        I.n = hk.prob.n;
        I.r = hk.r;
        I.lo = hk.prob.lo;
        I.hi = hk.prob.hi;
        I.lin = hk.prob.lin;
        I.dw = hk.dw;
        I.scale = nullptr;
        I.lam = hk.prob.lambda;
        const bool lasso = hk.prob.loss == ASYFLEXA_LOSS_LASSO;
        I.s_loss = lasso ? 1.0 : 2.0;
        I.c2 = lasso ? 0.0 : 2.0 * hk.prob.c;
        I.active = 1;
        ConvState& c = B->h_conv[k];
        c.norms = hk.norms_out;
        c.lam = hk.prob.lambda;
        c.c = hk.prob.c;
        c.f_star = NAN;
        c.F = c.F_prev = NAN;
        c.loss = hk.prob.loss;
        c.conv_round = -2;  // not converged
    }
    cudaError_t e = cudaMalloc(&B->d_inst, count * sizeof(BatchInst));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_conv, count * sizeof(ConvState));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_round, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_nactive, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&B->counters, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&B->hist, 32 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&B->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(B->counters, 0, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(B->hist, 0, 32 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(B->err, 0, sizeof(int));
    if (e != cudaSuccess) return fail(bfail(std::string("batch allocation: ") + cudaGetErrorString(e), ASYFLEXA_ENOMEM));
    // the async rounds' block width (for a Gauss-Seidel batch, whose block_w 1..4 is the
    // Gauss-Seidel width, 32 for the problems it hands over)
    const bool gs_w = B->form == ASYFLEXA_BATCH_FORM_GS && opts->block_w <= asyflexa::kGsWMax;
    const int rc = build_blocks(*B, opts->block_w > 0 && !gs_w ? opts->block_w : 32);
    if (rc) return fail(rc);
    {
        // Gauss-Seidel form: the problem table and the queue order (largest m * n first)
        B->h_gs.resize(count);
        std::vector<int> order(count);
        double total_mn = 0.0;
        int64_t max_n = 0;
        for (int k = 0; k < count; ++k) {
            const asyflexa_s& hk = *B->h[k];
            asyflexa::GsInst& g = B->h_gs[k];
            std::memset(&g, 0, sizeof g);
            g.A = static_cast<const float*>(hk.prob.A);
            g.lda = hk.prob.lda;
            g.m = hk.prob.m;
            g.n = hk.prob.n;
            g.b = static_cast<const float*>(hk.prob.b);
            g.lo = static_cast<const float*>(hk.prob.lo);
            g.hi = static_cast<const float*>(hk.prob.hi);
            g.lin = static_cast<const float*>(hk.prob.lin);
            g.lam = hk.prob.lambda;
            const bool lasso = hk.prob.loss == ASYFLEXA_LOSS_LASSO;
            g.s_loss = lasso ? 1.0 : 2.0;
            g.c2 = lasso ? 0.0 : 2.0 * hk.prob.c;
            g.c = lasso ? 0.0 : hk.prob.c;
            g.loss = hk.prob.loss;
            g.f_star = NAN;
            order[k] = k;
            total_mn += static_cast<double>(hk.prob.m) * static_cast<double>(hk.prob.n);
            max_n = std::max<int64_t>(max_n, hk.prob.n);
        }
        // the (d_j, 1/d_j) table, and the sizes the ring slot is chosen from
        int64_t total_n = 0;
        for (int k = 0; k < count; ++k) {
            const asyflexa_s& hk = *B->h[k];
            total_n += hk.prob.n;
            B->max_colbytes = std::max<int64_t>(B->max_colbytes, hk.mcopy * 4);
            B->max_multi = std::max<int64_t>(B->max_multi, asyflexa::kGsWMax * hk.prob.lda * 4);
        }
        e = cudaMalloc(&B->d_dd, total_n * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&B->d_xsave, total_n * sizeof(float));
        if (e != cudaSuccess) return fail(bfail(std::string("batch allocation: ") + cudaGetErrorString(e), ASYFLEXA_ENOMEM));
        {
            int64_t off = 0;
            for (int k = 0; k < count; ++k) {
                const asyflexa_s& hk = *B->h[k];
                gs_coef_kernel<<<static_cast<int>(std::min<int64_t>(1024, (hk.prob.n + 255) / 256)), 256, 0, B->stream>>>(
                    hk.dw, hk.prob.n, B->d_dd + off);
                B->h_gs[k].dd = B->d_dd + off;
                off += hk.prob.n;
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return fail(bfail(std::string("coefficient kernel: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
        }
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return static_cast<double>(B->h_gs[a].m) * B->h_gs[a].n > static_cast<double>(B->h_gs[b].m) * B->h_gs[b].n;
        });
        e = cudaMalloc(&B->d_gs, count * sizeof(asyflexa::GsInst));
        if (e == cudaSuccess) e = cudaMalloc(&B->d_order, count * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&B->d_order2, count * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&B->d_queue, sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(B->d_order, order.data(), count * sizeof(int), cudaMemcpyHostToDevice);
        B->h_order = order;
        if (e != cudaSuccess) return fail(bfail(std::string("batch allocation: ") + cudaGetErrorString(e), ASYFLEXA_ENOMEM));
        char key[160];
        std::snprintf(key, sizeof key, "count=%d mn=%.0f max_m=%lld max_n=%lld flags=%d nctas=%d w=%d sms=%d", count,
                      total_mn, static_cast<long long>(B->max_mcopy), static_cast<long long>(max_n), flags,
                      opts->num_ctas, opts->block_w, B->sm_count);
        B->shape_key = key;
    }
    // the caller's stream continues after the set-up work
    e = cudaEventRecord(B->ev_out, B->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->user_stream, B->ev_out, 0);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(bfail(std::string("batch stream: ") + cudaGetErrorString(e), ASYFLEXA_ECUDA));
    }
    *out = B;
    return ASYFLEXA_OK;
}

int asyflexa_batch_destroy(asyflexa_batch_t B) {
    if (!B) return ASYFLEXA_OK;
    if (B->stream) cudaStreamSynchronize(B->stream);
    // the multi-lane handle (and its lane-0 handle) work on the batch's stream: destroyed first
    if (B->multi) asyflexa_multi_destroy(B->multi);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->gs_exec) cudaGraphExecDestroy(B->gs_exec);
    if (B->gs_graph) cudaGraphDestroy(B->gs_graph);
    for (auto hk : B->h) asyflexa_destroy(hk);
    for (cudaStream_t fs : B->fin_streams) cudaStreamDestroy(fs);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->stream) cudaStreamDestroy(B->stream);
    void* ptrs[] = {B->d_bmat, B->d_xmat, B->d_inst, B->d_blk_inst, B->d_blk_local, B->d_conv, B->d_round, B->d_nactive,
                    B->counters, B->hist, B->err, B->d_gs, B->d_order, B->d_order2, B->d_queue, B->d_dd, B->d_xsave};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete B;
    return ASYFLEXA_OK;
}

int asyflexa_batch_solve(asyflexa_batch_t B, void* const* xs, const double* f_star, asyflexa_stats* per,
                         asyflexa_stats* total) {
    if (!B || !xs) return bfail("batch or xs is NULL");
    // the batch's stream starts after the caller's prior work (the iterates may come from it)
    BCK(cudaEventRecord(B->ev_in, B->user_stream), "event record");
    BCK(cudaStreamWaitEvent(B->stream, B->ev_in, 0), "stream wait");
    const int rc = B->form == ASYFLEXA_BATCH_FORM_GS      ? gs_solve(*B, xs, f_star, per, total)
                   : B->form == ASYFLEXA_BATCH_FORM_MULTI ? multi_form_solve(*B, xs, f_star, per, total)
                                                          : rounds_solve(*B, xs, f_star, per, total);
    // the caller's stream continues after the batch's work
    cudaEventRecord(B->ev_out, B->stream);
    cudaStreamWaitEvent(B->user_stream, B->ev_out, 0);
    return rc;
}

int asyflexa_batch_check(asyflexa_batch_t B, void* const* xs, const double* f_star, asyflexa_stats* per) {
    if (!B || !xs || !per) return bfail("batch, xs or per is NULL");
    BCK(cudaEventRecord(B->ev_in, B->user_stream), "event record");
    BCK(cudaStreamWaitEvent(B->stream, B->ev_in, 0), "stream wait");
    int first = ASYFLEXA_OK;
    for (int k = 0; k < B->count; ++k) {
        asyflexa_stats s;
        std::memset(&s, 0, sizeof s);
        B->h[k]->opts.f_star = f_star ? f_star[k] : NAN;
        const int crc = asyflexa_check(B->h[k], xs[k], &s);
        if (crc && first == ASYFLEXA_OK) {
            first = crc;
            asyflexa_internal::set_thread_error("problem " + std::to_string(k) + ": " + asyflexa_last_error(B->h[k]));
        }
        s.status = crc;
        per[k] = s;
    }
    cudaEventRecord(B->ev_out, B->stream);
    cudaStreamWaitEvent(B->user_stream, B->ev_out, 0);
    return first;
}

}  // extern "C"
