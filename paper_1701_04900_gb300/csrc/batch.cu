// Batched form: many independent problems (uneven sizes, or one matrix with many lambda
// values) solved by one persistent asynchronous sweep launch per round, each round (sweeps,
// exact residual refreshes, objectives, device-side convergence test) replayed as a
// captured CUDA graph.
//
// Every problem keeps its own internal handle for the surrogate weights, the FP64 residual
// and the refresh / objective / check kernels.  The sweep kernel is the register-increment
// async kernel of sweep_async.cuh in its BATCHED form: the blocks of all problems form one
// global list, CTA c owns the global blocks c, c + G, ..., and a converged problem's blocks
// are skipped from the next round on.  The block width is fixed by the options or, with
// block_w = 0, picked by a small autotuner that times one sweep per candidate width.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "sweep_async.cuh"

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
    int graph_w = 0;
    std::vector<int> cap;  // per problem: blocks it may have in flight, max(1, m / (4 w))
    int grid = 0;          // CTAs of the next sweep launch
    int graph_grid = 0;    // CTAs of the captured round
    long long launches = 0;
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
    const int64_t units = B->max_mcopy / 4;
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
                                             static_cast<int>(B->smem));
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
    const int rc = build_blocks(*B, opts->block_w > 0 ? opts->block_w : 32);
    if (rc) return fail(rc);
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
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto hk : B->h) asyflexa_destroy(hk);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->stream) cudaStreamDestroy(B->stream);
    void* ptrs[] = {B->d_inst, B->d_blk_inst, B->d_blk_local, B->d_conv, B->d_round, B->d_nactive,
                    B->counters, B->hist, B->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete B;
    return ASYFLEXA_OK;
}

int asyflexa_batch_solve(asyflexa_batch_t B, void* const* xs, const double* f_star, asyflexa_stats* per,
                         asyflexa_stats* total) {
    if (!B || !xs) return bfail("batch or xs is NULL");
    const int count = B->count;
    // the batch's stream starts after the caller's prior work (the iterates may come from it)
    BCK(cudaEventRecord(B->ev_in, B->user_stream), "event record");
    BCK(cudaStreamWaitEvent(B->stream, B->ev_in, 0), "stream wait");
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
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
    // autotuner: time one sweep per candidate block width (these are real sweeps)
    if (B->opts.block_w == 0 && B->graph_w == 0) {
        float best = 0.f;
        int best_w = 32;
        cudaEvent_t a0, a1;
        BCK(cudaEventCreate(&a0), "event");
        BCK(cudaEventCreate(&a1), "event");
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
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
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
    int n_active = count, last_active = count;
    while (sweeps < B->opts.max_sweeps && n_active > 0) {
        BCK(cudaGraphLaunch(B->exec, B->stream), "graph launch");
        sweeps += per_round;
        BCK(cudaMemcpyAsync(&n_active, B->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, B->stream), "read count");
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
    BCK(cudaEventRecord(e1, B->stream), "event record");
    BCK(cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(cudaMemcpy(B->h_conv.data(), B->d_conv, count * sizeof(ConvState), cudaMemcpyDeviceToHost), "read state");
    long long bu = 0;
    int worst = ASYFLEXA_OK;
    for (int k = 0; k < count; ++k) {
        const ConvState& c = B->h_conv[k];
        const long long nb = (B->h[k]->prob.n + B->w - 1) / B->w;
        const long long ksweeps = c.conv_round >= 0 ? static_cast<long long>(c.conv_round + 1) * per_round : sweeps;
        bu += nb * ksweeps;
        int st = c.conv_round >= 0 ? ASYFLEXA_OK : (c.conv_round == -1 ? ASYFLEXA_ENONFINITE : ASYFLEXA_ENOTCONV);
        if (per) {
            asyflexa_stats s;
            std::memset(&s, 0, sizeof s);
            B->h[k]->opts.f_star = c.f_star;
            const int crc = asyflexa_check(B->h[k], xs[k], &s);
            if (crc) st = crc;
            s.sweeps = ksweeps;
            s.block_updates = nb * ksweeps;
            s.status = st;
            per[k] = s;
        }
        if (st != ASYFLEXA_OK && (worst == ASYFLEXA_OK || st < 0)) worst = st;
    }
    BCK(cudaEventRecord(B->ev_out, B->stream), "event record");
    BCK(cudaStreamWaitEvent(B->user_stream, B->ev_out, 0), "stream wait");
    if (total) {
        std::memset(total, 0, sizeof *total);
        total->sweeps = sweeps;
        total->block_updates = bu;
        total->seconds = ms * 1e-3;
        total->status = worst;
        total->kernel_launches = B->launches;
        total->block_w = B->w;
    }
    return worst;
}

}  // extern "C"
