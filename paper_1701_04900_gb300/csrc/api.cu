// C-ABI of the AsyFLEXA library: validation, handle lifetime, and the host-side control
// of sweeps, residual refreshes and checks.  All device work is in the kernels of
// sweep.cuh / aux.cuh, launched through Launcher<TA>.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "sweep.cuh"  // kernel geometry constants and the shared-memory layout

using asyflexa::Launcher;

extern template struct asyflexa::Launcher<double>;
extern template struct asyflexa::Launcher<float>;
extern template struct asyflexa::Launcher<__nv_bfloat16>;
extern template struct asyflexa::Launcher<__nv_fp8_e4m3>;

namespace {

thread_local std::string g_thread_msg = "no error";

constexpr int kNormsGridHost = 256;      // must match asyflexa::kNormsGrid
constexpr int kGemvUnitsHost = 2;        // must match asyflexa::kGemvUnits
constexpr int kCompactTileHost = 4096;   // must match asyflexa::kCompactTile

int set_error(asyflexa_s* h, int code, const std::string& msg) {
    if (h) {
        h->msg = msg;
        h->last_status = code;
    } else {
        g_thread_msg = msg;
    }
    return code;
}

int cuda_error(asyflexa_s* h, cudaError_t e, const char* where) {
    (void)cudaGetLastError();  // consume a non-sticky error so that later launches do not report it
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return set_error(h, e == cudaErrorMemoryAllocation ? ASYFLEXA_ENOMEM : ASYFLEXA_ECUDA, m);
}

// The async sweep kernel a handle launches: 2 register increment, 1 staged residual tile.
int async_variant(const asyflexa_s& h) {
    if (h.reg_upt <= 0) return 1;
    const bool exact = h.reg_exact_ok && h.opts.exact_grad == 1;
    return (h.reg_rc_ok && !h.reg_rc_off && !exact) ? 2 : 3;
}

#define CK(h, call, where)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_error(h, e_, where); \
    } while (0)

int elt_bytes(int dtype) {
    switch (dtype) {
        case ASYFLEXA_F64: return 8;
        case ASYFLEXA_F32: return 4;
        case ASYFLEXA_BF16: return 2;
        case ASYFLEXA_FP8E4M3: return 1;
        default: return 0;
    }
}

template <typename F>
auto dispatch(asyflexa_s& h, F&& f) {
    switch (h.prob.a_dtype) {
        case ASYFLEXA_F64: return f(Launcher<double>{});
        case ASYFLEXA_F32: return f(Launcher<float>{});
        case ASYFLEXA_BF16: return f(Launcher<__nv_bfloat16>{});
        default: return f(Launcher<__nv_fp8_e4m3>{});
    }
}

void free_buffers(asyflexa_s* h) {
    void* ptrs[] = {h->r, h->dw, h->delta, h->list_idx, h->list_val, h->tilecnt, h->count, h->partial,
                    h->norms_part, h->norms_out, h->counters, h->hist, h->meas, h->err, h->flag, h->gtab};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

int do_refresh(asyflexa_s& h, const void* x) {
    if (h.master) {
        // exact residual of the FP32 problem, shared with the low-precision sweeps
        int rc = do_refresh(*h.master, x);
        if (rc) return set_error(&h, rc, std::string("master refresh: ") + h.master->msg);
        CK(&h, cudaMemcpyAsync(h.r, h.master->r, h.prob.m * sizeof(double), cudaMemcpyDeviceToDevice, h.stream),
           "copy master residual");
    } else {
        cudaError_t e = dispatch(h, [&](auto L) { return decltype(L)::refresh(h, x); });
        if (e != cudaSuccess) return cuda_error(&h, e, "residual refresh");
    }
    h.r_valid = true;
    h.r_x = x;
    return ASYFLEXA_OK;
}

int device_error(asyflexa_s& h) {
    int e = 0;
    CK(&h, cudaMemcpyAsync(&e, h.err, sizeof(int), cudaMemcpyDeviceToHost, h.stream), "read error word");
    CK(&h, cudaStreamSynchronize(h.stream), "synchronize");
    if (e != 0) {
        h.r_valid = false;
        return set_error(&h, ASYFLEXA_ETIMEOUT, "a bounded device-side wait expired; results are invalid");
    }
    return ASYFLEXA_OK;
}

// F(x) from the handle's residual (must describe x): LASSO 0.5||r||^2 + lam||x||_1,
// NCQUAD ||r||^2 - c||x||^2 + lam||x||_1, DC ||r||^2 + lam sum_j h(x_j); plus lin^T x.
// Optionally also ||r||^2 and b^T r (for the LASSO duality gap).  Synchronises.
int objective(asyflexa_s& h, const void* x, double* F, double* nnz, double* rr = nullptr, double* br = nullptr) {
    cudaError_t e = dispatch(h, [&](auto L) { return decltype(L)::norms(h, x); });
    if (e != cudaSuccess) return cuda_error(&h, e, "norms");
    double v[7];
    CK(&h, cudaMemcpyAsync(v, h.norms_out, sizeof(v), cudaMemcpyDeviceToHost, h.stream), "read norms");
    CK(&h, cudaStreamSynchronize(h.stream), "synchronize");
    const auto& P = h.prob;
    if (loss_is_dc(P))
        *F = v[0] + P.lambda * v[5] + v[4];
    else
        *F = (P.loss == ASYFLEXA_LOSS_LASSO ? 0.5 * v[0] : v[0] - P.c * v[2]) + v[4] + P.lambda * v[1];
    if (nnz) *nnz = v[3];
    if (rr) *rr = v[0];
    if (br) *br = v[6];
    if (!std::isfinite(*F)) return set_error(&h, ASYFLEXA_ENONFINITE, "objective is not finite");
    return ASYFLEXA_OK;
}

// The plain LASSO (no box, no linear term) has the dual max -0.5||nu||^2 - b^T nu subject to
// ||A^T nu||_inf <= lam; nu = theta r, theta = min(1, lam / ||A^T r||_inf), is feasible, and
// P(x) - D(nu) >= P(x) - F* (weak duality): a certificate of the gap without F*.  Relative to
// max(1, |P|); NaN for the other problems.
bool plain_lasso(const asyflexa_s& h) {
    return h.prob.loss == ASYFLEXA_LOSS_LASSO && !h.prob.lo && !h.prob.hi && !h.prob.lin;
}
double lasso_dual_gap(const asyflexa_s& h, double P, double rr, double br, double atr) {
    if (!plain_lasso(h)) return std::nan("");
    const double lam = h.prob.lambda;
    const double theta = atr <= lam ? 1.0 : lam / atr;
    const double D = -0.5 * theta * theta * rr - theta * br;
    return (P - D) / std::max(1.0, std::fabs(P));
}

struct Measures {
    double mf, xh, kkt, xmax, atr;
    long long nnz;
    bool nonfinite;
};

int measure(asyflexa_s& h, const void* x, Measures* M) {
    CK(&h, cudaMemsetAsync(h.meas, 0, 8 * sizeof(unsigned long long), h.stream), "clear measures");
    cudaError_t e = dispatch(h, [&](auto L) { return decltype(L)::check(h, x); });
    if (e != cudaSuccess) return cuda_error(&h, e, "check");
    unsigned long long v[8];
    CK(&h, cudaMemcpyAsync(v, h.meas, sizeof(v), cudaMemcpyDeviceToHost, h.stream), "read measures");
    CK(&h, cudaStreamSynchronize(h.stream), "synchronize");
    auto asd = [](unsigned long long u) {
        double d;
        std::memcpy(&d, &u, sizeof d);
        return d;
    };
    M->mf = asd(v[0]);
    M->xh = asd(v[1]);
    M->kkt = asd(v[2]);
    M->xmax = asd(v[3]);
    M->nnz = static_cast<long long>(v[4]);
    M->nonfinite = v[5] != 0;
    M->atr = asd(v[6]);
    if (M->nonfinite) return set_error(&h, ASYFLEXA_ENONFINITE, "non-finite value in the optimality check");
    return ASYFLEXA_OK;
}

// Sum the elapsed times of recorded sweep-launch event pairs (synchronises the stream).
int drain_profile(asyflexa_s& h) {
    if (h.prof_events.empty()) return ASYFLEXA_OK;
    CK(&h, cudaStreamSynchronize(h.stream), "synchronize");
    for (size_t k = 0; k < h.prof_events.size(); ++k) {
        float ms = 0.f;
        CK(&h, cudaEventElapsedTime(&ms, h.prof_events[k].first, h.prof_events[k].second), "event time");
        h.prof_seconds += 1e-3 * ms;
        h.prof_sweep_total += h.prof_sweeps[k];
        ++h.prof_launches;
        cudaEventDestroy(h.prof_events[k].first);
        cudaEventDestroy(h.prof_events[k].second);
    }
    h.prof_events.clear();
    h.prof_sweeps.clear();
    return ASYFLEXA_OK;
}

// Launch one sweep kernel (k sweeps), bracketed by events when profiling.
// Steps of the next launch (k sweeps) from the diminishing rule, into the device table.
int fill_steps(asyflexa_s& h, int k) {
    const size_t cnt = static_cast<size_t>(k) * static_cast<size_t>(h.nblocks);
    if (cnt > h.gtab_cap) {
        CK(&h, cudaStreamSynchronize(h.stream), "synchronize");
        if (h.gtab) cudaFree(h.gtab);
        h.gtab = nullptr;
        h.gtab_cap = 0;
        CK(&h, cudaMalloc(&h.gtab, cnt * sizeof(double)), "alloc step table");
        h.gtab_cap = cnt;
    }
    // the previous launch's copy must have left the host buffer before it is rewritten
    CK(&h, cudaStreamSynchronize(h.stream), "synchronize");
    h.gtab_host.resize(cnt);
    double g = h.sched_gamma;
    const double mu = h.opts.gamma_mu;
    for (size_t i = 0; i < cnt; ++i) {
        h.gtab_host[i] = g;
        const double t = mu * g;  // two roundings, the order of the oracle's recurrence
        g = g * (1.0 - t);
    }
    CK(&h, cudaMemcpyAsync(h.gtab, h.gtab_host.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, h.stream),
       "upload steps");
    return ASYFLEXA_OK;
}

// Move the adaptive proximal weight to t (every d_j changes by t - tau_extra).
int set_tau_extra(asyflexa_s& h, double t) {
    if (t == h.tau_extra) return ASYFLEXA_OK;
    cudaError_t e = dispatch(h, [&](auto L) { return decltype(L)::shift_weights(h, t - h.tau_extra); });
    if (e != cudaSuccess) return cuda_error(&h, e, "shift weights");
    h.tau_extra = t;
    return ASYFLEXA_OK;
}

// Restart the diminishing-step sequence (k = 0, gamma^0 = opts.gamma) and the update counter.
int restart_steps(asyflexa_s& h) {
    h.sched_k = 0;
    h.sched_gamma = h.opts.gamma;
    CK(&h, cudaMemsetAsync(h.counters, 0, sizeof(unsigned long long), h.stream), "clear update counter");
    return ASYFLEXA_OK;
}

int launch_sweep(asyflexa_s& h, void* x, int mode, int k) {
    if (h.opts.gamma_mu > 0.0) {
        int rc = fill_steps(h, k);
        if (rc) return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h.opts.profile) {
        if (h.prof_events.size() >= 4096) {
            int rc = drain_profile(h);
            if (rc) return rc;
        }
        CK(&h, cudaEventCreate(&e0), "event");
        CK(&h, cudaEventCreate(&e1), "event");
        CK(&h, cudaEventRecord(e0, h.stream), "event record");
    }
    cudaError_t e = dispatch(h, [&](auto L) { return decltype(L)::sweep(h, x, mode, k); });
    if (e != cudaSuccess) return cuda_error(&h, e, mode == ASYFLEXA_ASYNC ? "async sweep" : "jacobi sweep");
    if (h.opts.profile) {
        CK(&h, cudaEventRecord(e1, h.stream), "event record");
        h.prof_events.emplace_back(e0, e1);
        h.prof_sweeps.push_back(k);
    }
    if (h.opts.gamma_mu > 0.0) {
        const long long cnt = static_cast<long long>(k) * h.nblocks;
        h.sched_k += cnt;
        h.sched_gamma = h.gtab_host[cnt - 1] * (1.0 - h.opts.gamma_mu * h.gtab_host[cnt - 1]);
    }
    return ASYFLEXA_OK;
}

int run_sweeps(asyflexa_s& h, void* x, int n_sweeps) {
    if (!h.r_valid || h.r_x != x) {
        int rc = do_refresh(h, x);
        if (rc) return rc;
    }
    const int mode = h.opts.mode;
    int since = 0;
    int remaining = n_sweeps;
    while (remaining > 0) {
        if (mode == ASYFLEXA_ASYNC) {
            const int k = std::min(remaining, h.opts.refresh_every - since);
            int rc = launch_sweep(h, x, ASYFLEXA_ASYNC, k);
            if (rc) return rc;
            since += k;
            remaining -= k;
        } else {
            int rc = launch_sweep(h, x, ASYFLEXA_SYNC, 1);
            if (rc) return rc;
            cudaError_t e;
            e = dispatch(h, [&](auto L) { return decltype(L)::jacobi_apply(h); });
            if (e != cudaSuccess) return cuda_error(&h, e, "jacobi scatter");
            since += 1;
            remaining -= 1;
        }
        if (since == h.opts.refresh_every || remaining == 0) {
            int rc = do_refresh(h, x);
            if (rc) return rc;
            since = 0;
        }
    }
    h.total_sweeps += n_sweeps;
    return ASYFLEXA_OK;
}

int validate_opts(const asyflexa_opts* o, std::string* why) {
    if (o->block_w < 1 || o->block_w > asyflexa::kWMax) return *why = "block_w must be in [1, 128]", 1;
    if (o->mode != ASYFLEXA_SYNC && o->mode != ASYFLEXA_ASYNC) return *why = "unknown mode", 1;
    if (!(o->gamma > 0.0) || !std::isfinite(o->gamma)) return *why = "gamma must be finite and > 0", 1;
    if (!(o->tau >= 0.0) || !std::isfinite(o->tau)) return *why = "tau must be finite and >= 0", 1;
    if (!(o->tau_rel >= 0.0) || !std::isfinite(o->tau_rel)) return *why = "tau_rel must be finite and >= 0", 1;
    if (o->refresh_every < 1 || o->check_every < 1 || o->max_sweeps < 1)
        return *why = "refresh_every, check_every and max_sweeps must be >= 1", 1;
    if (o->num_ctas < 0) return *why = "num_ctas must be >= 0", 1;
    if (o->variant < 0 || o->variant > 3) return *why = "variant must be 0, 1, 2 or 3", 1;
    if (o->delay_ns < 0 || o->delay_ns > 1000000) return *why = "delay_ns must be in [0, 1000000]", 1;
    if (!(o->tol_gap >= 0.0) || !(o->tol_stat >= 0.0)) return *why = "tolerances must be >= 0", 1;
    if (!(o->switch_tol >= 0.0)) return *why = "switch_tol must be >= 0", 1;
    if (!(o->gamma_mu >= 0.0) || !std::isfinite(o->gamma_mu)) return *why = "gamma_mu must be finite and >= 0", 1;
    if (o->tau_adapt != 0 && o->tau_adapt != 1) return *why = "tau_adapt must be 0 or 1", 1;
    if (o->exact_grad != 0 && o->exact_grad != 1) return *why = "exact_grad must be 0 or 1", 1;
    if (o->gamma_mu > 0.0 && o->gamma_mu * o->gamma >= 1.0)
        return *why = "gamma_mu * gamma must be < 1 (the steps must stay positive)", 1;
    return 0;
}

}  // namespace

namespace asyflexa_internal {
// Used by the handle-free entry point in noalloc.cu to report errors through
// asyflexa_last_error(NULL).  Not exported.
__attribute__((visibility("hidden"))) void set_thread_error(const std::string& msg) { g_thread_msg = msg; }
}  // namespace asyflexa_internal

extern "C" {

int asyflexa_version(void) { return ASYFLEXA_ABI_VERSION; }

const char* asyflexa_status_string(int s) {
    switch (s) {
        case ASYFLEXA_OK: return "ASYFLEXA_OK";
        case ASYFLEXA_ENOTCONV: return "ASYFLEXA_ENOTCONV";
        case ASYFLEXA_EINVAL: return "ASYFLEXA_EINVAL";
        case ASYFLEXA_ECUDA: return "ASYFLEXA_ECUDA";
        case ASYFLEXA_ENOMEM: return "ASYFLEXA_ENOMEM";
        case ASYFLEXA_ETIMEOUT: return "ASYFLEXA_ETIMEOUT";
        case ASYFLEXA_ENONFINITE: return "ASYFLEXA_ENONFINITE";
        case ASYFLEXA_EUNSUPPORTED: return "ASYFLEXA_EUNSUPPORTED";
        default: return "ASYFLEXA_UNKNOWN";
    }
}

void asyflexa_opts_default(asyflexa_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->block_w = 32;
    o->mode = ASYFLEXA_SYNC;
    o->gamma = 0.9;
    o->tau = 0.0;
    o->tau_rel = 0.0;
    o->refresh_every = 10;
    o->check_every = 10;
    o->max_sweeps = 1000;
    o->num_ctas = 0;
    o->tol_gap = 1e-6;
    o->tol_stat = 1e-6;
    o->f_star = std::nan("");
    o->seed = 0;
    o->switch_tol = 1e-7;
    o->gamma_mu = 0.0;
    o->tau_adapt = 0;
    o->exact_grad = 0;
    o->delay_ns = 0;
    o->reserved2 = 0;
}

const char* asyflexa_last_error(asyflexa_t h) { return h ? h->msg.c_str() : g_thread_msg.c_str(); }

int asyflexa_create(asyflexa_t* out, const asyflexa_problem* P, const asyflexa_opts* O, void* stream) {
    if (!out) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    *out = nullptr;
    if (!P || !O) return set_error(nullptr, ASYFLEXA_EINVAL, "problem or options is NULL");
    std::string why;
    if (validate_opts(O, &why)) return set_error(nullptr, ASYFLEXA_EINVAL, why);
    const int ea = elt_bytes(P->a_dtype);
    if (ea == 0) return set_error(nullptr, ASYFLEXA_EINVAL, "unknown a_dtype");
    const bool f64 = P->a_dtype == ASYFLEXA_F64;
    if (P->x_dtype != (f64 ? ASYFLEXA_F64 : ASYFLEXA_F32))
        return set_error(nullptr, ASYFLEXA_EINVAL, "x_dtype must be F64 for F64 A and F32 otherwise");
    if (P->m < 1 || P->n < 1) return set_error(nullptr, ASYFLEXA_EINVAL, "m and n must be >= 1");
    if (P->n > (int64_t(1) << 31) - 1 - 4096) return set_error(nullptr, ASYFLEXA_EINVAL, "n too large");
    if (P->lda < P->m) return set_error(nullptr, ASYFLEXA_EINVAL, "lda < m");
    if ((P->lda * ea) % 16 != 0) return set_error(nullptr, ASYFLEXA_EINVAL, "lda * element size must be a multiple of 16 bytes");
    if (!P->A || (reinterpret_cast<uintptr_t>(P->A) & 15u))
        return set_error(nullptr, ASYFLEXA_EINVAL, "A must be a non-NULL 16-byte aligned device pointer");
    if (!P->b) return set_error(nullptr, ASYFLEXA_EINVAL, "b is NULL");
    const bool quant = P->a_dtype == ASYFLEXA_BF16 || P->a_dtype == ASYFLEXA_FP8E4M3;
    if (quant && !P->col_scale) return set_error(nullptr, ASYFLEXA_EINVAL, "BF16/FP8 storage needs col_scale");
    if (!quant && P->col_scale) return set_error(nullptr, ASYFLEXA_EINVAL, "col_scale is only for BF16/FP8 storage");
    if (!(P->lambda >= 0.0) || !std::isfinite(P->lambda)) return set_error(nullptr, ASYFLEXA_EINVAL, "lambda must be finite and >= 0");
    if (P->loss < ASYFLEXA_LOSS_LASSO || P->loss > ASYFLEXA_LOSS_DC_EXP)
        return set_error(nullptr, ASYFLEXA_EINVAL, "unknown loss");
    if (loss_is_dc(*P) && !(P->c > 0.0 && std::isfinite(P->c)))
        return set_error(nullptr, ASYFLEXA_EINVAL, "the DC losses need theta (passed in c) > 0");
    if (!std::isfinite(P->c)) return set_error(nullptr, ASYFLEXA_EINVAL, "c must be finite");
    if (P->A_master) {
        if (!quant) return set_error(nullptr, ASYFLEXA_EINVAL, "A_master is only for BF16/FP8 storage");
        if (P->lda_master < P->m || (P->lda_master * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(P->A_master) & 15u))
            return set_error(nullptr, ASYFLEXA_EINVAL,
                             "A_master must be 16-byte aligned with lda_master >= m and lda_master a multiple of 4");
    }

    auto* h = new (std::nothrow) asyflexa_s();
    if (!h) return set_error(nullptr, ASYFLEXA_ENOMEM, "host allocation failed");
    h->prob = *P;
    h->opts = *O;
    h->stream = static_cast<cudaStream_t>(stream);
    h->elt_a = ea;
    h->vec = 16 / ea;
    h->elt_c = f64 ? 8 : 4;

    auto fail = [&](int rc) {
        std::string m = h->msg;
        free_buffers(h);
        delete h;
        set_error(nullptr, rc, m);
        return rc;
    };
#define CKC(call, where)                               \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return fail(cuda_error(h, e_, where)); \
    } while (0)

    CKC(cudaGetDevice(&h->device), "cudaGetDevice");
    CKC(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device), "SM count");
    int optin = 0;
    CKC(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device), "smem attribute");
    h->smem_optin = static_cast<size_t>(optin);

    const int64_t m = P->m, n = P->n;
    h->mcopy = (m + h->vec - 1) / h->vec * h->vec;
    h->nblocks = static_cast<int>((n + O->block_w - 1) / O->block_w);
    h->sweep_ctas = O->num_ctas > 0 ? O->num_ctas : h->sm_count;
    if (h->sweep_ctas > h->nblocks) h->sweep_ctas = h->nblocks;

    // sweep kernel geometry: ring of bulk-copy stages + residual tile in shared memory
    {
        const int chunk_bytes = 32 * 1024;
        int chunk_rows = chunk_bytes / ea;
        const int64_t tile_need = (h->mcopy + 15) / 16 * 16;
        if (tile_need < chunk_rows) chunk_rows = static_cast<int>(tile_need);
        const size_t stage_b = static_cast<size_t>((static_cast<size_t>(chunk_rows) * ea + 127) / 128 * 128);
        int stages = static_cast<int>((128 * 1024) / stage_b);
        stages = stages < 4 ? 4 : (stages > 16 ? 16 : stages);
        const auto L0 = asyflexa::make_sweep_layout(ea, h->elt_c, stages, chunk_rows, 0);
        if (L0.total + 1024 > h->smem_optin) {
            free_buffers(h);
            delete h;
            return set_error(nullptr, ASYFLEXA_EUNSUPPORTED, "device shared memory too small");
        }
        const size_t avail = h->smem_optin - L0.total - 256;
        int64_t cap_rows = static_cast<int64_t>(avail / h->elt_c) / 16 * 16;
        if (cap_rows < chunk_rows) cap_rows = chunk_rows / 16 * 16;
        if (tile_need <= cap_rows) {
            h->tile_rows = static_cast<int>(tile_need);
            h->ntiles = 1;
        } else {
            h->tile_rows = static_cast<int>(cap_rows);
            h->ntiles = static_cast<int>((h->mcopy + cap_rows - 1) / cap_rows);
        }
        h->chunk_rows = chunk_rows;
        h->stages = stages;
        h->sweep_smem = asyflexa::make_sweep_layout(ea, h->elt_c, stages, chunk_rows, h->tile_rows).total;
    }
    // gather-GEMV / compaction / check geometry
    {
        const int64_t units = h->mcopy / h->vec;
        const int64_t per_cta = 256 * kGemvUnitsHost;
        h->gemv_rowtiles = static_cast<int>((units + per_cta - 1) / per_cta);
        int nseg = static_cast<int>((4 * h->sm_count + h->gemv_rowtiles - 1) / h->gemv_rowtiles);
        h->nseg = nseg < 1 ? 1 : (nseg > 64 ? 64 : nseg);
        h->compact_tiles = static_cast<int>((n + kCompactTileHost - 1) / kCompactTileHost);
        h->check_ctas = h->sm_count;
        h->check_smem = static_cast<size_t>(2 * h->mcopy * h->elt_c);
        h->check_use_smem = h->check_smem + 1024 <= h->smem_optin;
        const int rc = dispatch(*h, [&](auto L) { return decltype(L)::setup_pipe(*h); });
        if (rc) CKC(static_cast<cudaError_t>(rc), "pipelined gather set-up");
    }

    CKC(cudaMalloc(&h->r, h->mcopy * sizeof(double)), "alloc r");
    CKC(cudaMalloc(&h->dw, n * sizeof(double)), "alloc weights");
    CKC(cudaMalloc(&h->delta, n * h->elt_c), "alloc delta");
    CKC(cudaMalloc(&h->list_idx, n * sizeof(int)), "alloc list");
    CKC(cudaMalloc(&h->list_val, n * h->elt_c), "alloc list");
    CKC(cudaMalloc(&h->tilecnt, h->compact_tiles * sizeof(int)), "alloc tiles");
    CKC(cudaMalloc(&h->count, sizeof(int)), "alloc count");
    CKC(cudaMalloc(&h->partial, static_cast<size_t>(std::max(h->nseg, h->pipe_nseg)) * h->mcopy * sizeof(double)),
        "alloc partials");
    CKC(cudaMalloc(&h->norms_part, kNormsGridHost * 8 * sizeof(double)), "alloc norms");
    CKC(cudaMalloc(&h->norms_out, 8 * sizeof(double)), "alloc norms");
    CKC(cudaMalloc(&h->counters, 4 * sizeof(unsigned long long)), "alloc counters");
    CKC(cudaMalloc(&h->hist, 32 * sizeof(unsigned long long)), "alloc hist");
    CKC(cudaMalloc(&h->meas, 8 * sizeof(unsigned long long)), "alloc measures");
    CKC(cudaMalloc(&h->err, sizeof(int)), "alloc err");
    CKC(cudaMalloc(&h->flag, sizeof(int)), "alloc flag");
    CKC(cudaMemsetAsync(h->r, 0, h->mcopy * sizeof(double), h->stream), "clear r");
    CKC(cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), h->stream), "clear counters");
    h->sched_k = 0;
    h->sched_gamma = O->gamma;
    CKC(cudaMemsetAsync(h->hist, 0, 32 * sizeof(unsigned long long), h->stream), "clear hist");
    CKC(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "clear err");
    CKC(cudaMemsetAsync(h->flag, 0, sizeof(int), h->stream), "clear flag");

    {
        int rc = dispatch(*h, [&](auto L) { return decltype(L)::set_smem_attrs(*h); });
        if (rc) CKC(static_cast<cudaError_t>(rc), "set shared-memory attribute");
        rc = dispatch(*h, [&](auto L) { return decltype(L)::choose_reg(*h); });
        if (rc < 0) CKC(static_cast<cudaError_t>(-rc), "set shared-memory attribute (register kernel)");
        if (O->variant == 1) {
            h->reg_upt = 0;
        } else if ((O->variant == 2 || O->variant == 3) && rc != 1) {
            set_error(h, ASYFLEXA_EUNSUPPORTED,
                      "variants 2 and 3 (register increment) need FP32/BF16/FP8 storage and m <= 24576");
            return fail(ASYFLEXA_EUNSUPPORTED);
        }
        // automatic choice between the two register-kernel forms: the column-in-registers form
        // issues the ring's refills from the consumer warps after each column barrier, which
        // pays only when a column carries enough work (measured on GB300: FP32 from 4 stages
        // per column, m > 12288; BF16 from 3 and FP8 from 2 stages, m > 16384)
        h->reg_rc_off = O->variant == 3 || (O->variant == 0 && h->prob.m <= (h->vec == 4 ? 12288 : 16384));
        if (O->exact_grad == 1 && !(h->reg_upt > 0 && h->reg_exact_ok && O->mode == ASYFLEXA_ASYNC)) {
            set_error(h, ASYFLEXA_EUNSUPPORTED,
                      "exact_grad 1 needs the asynchronous register kernel on FP32 storage (m <= 24576)");
            return fail(ASYFLEXA_EUNSUPPORTED);
        }
    }
    {
        cudaError_t e = dispatch(*h, [&](auto L) { return decltype(L)::colnorm(*h); });
        CKC(e, "surrogate weights");
        int neg = 0;
        CKC(cudaMemcpyAsync(&neg, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read flag");
        CKC(cudaStreamSynchronize(h->stream), "synchronize");
        if (neg) {
            set_error(h, ASYFLEXA_EINVAL,
                      "a surrogate weight d_j = (1+tau_rel)*kappa_j + tau is negative or not finite "
                      "(increase tau, or A holds non-finite values)");
            return fail(ASYFLEXA_EINVAL);
        }
    }
    if (O->tau_adapt) {
        // the adaptive proximal weight starts from 5% of the mean surrogate weight
        std::vector<double> dv(static_cast<size_t>(n));
        CKC(cudaMemcpy(dv.data(), h->dw, n * sizeof(double), cudaMemcpyDeviceToHost), "read weights");
        double sum = 0.0;
        for (double v : dv) sum += v > 0.0 ? v : 0.0;
        h->tau_unit = 0.05 * (sum > 0.0 ? sum / static_cast<double>(n) : 1.0);
    }
    if (P->lo || P->hi) {
        std::vector<double> lo(n, -INFINITY), hi(n, INFINITY);
        if (f64) {
            if (P->lo) CKC(cudaMemcpy(lo.data(), P->lo, n * 8, cudaMemcpyDeviceToHost), "read lo");
            if (P->hi) CKC(cudaMemcpy(hi.data(), P->hi, n * 8, cudaMemcpyDeviceToHost), "read hi");
        } else {
            std::vector<float> t(n);
            if (P->lo) {
                CKC(cudaMemcpy(t.data(), P->lo, n * 4, cudaMemcpyDeviceToHost), "read lo");
                for (int64_t j = 0; j < n; ++j) lo[j] = t[j];
            }
            if (P->hi) {
                CKC(cudaMemcpy(t.data(), P->hi, n * 4, cudaMemcpyDeviceToHost), "read hi");
                for (int64_t j = 0; j < n; ++j) hi[j] = t[j];
            }
        }
        for (int64_t j = 0; j < n; ++j) {
            if (!(lo[j] <= hi[j])) {
                set_error(h, ASYFLEXA_EINVAL, "lo[j] > hi[j] or a NaN bound at j = " + std::to_string(j));
                return fail(ASYFLEXA_EINVAL);
            }
        }
    }
    if (P->A_master) {
        asyflexa_problem mp = *P;
        mp.A = P->A_master;
        mp.lda = P->lda_master;
        mp.a_dtype = ASYFLEXA_F32;
        mp.x_dtype = ASYFLEXA_F32;
        mp.col_scale = nullptr;
        mp.A_master = nullptr;
        mp.lda_master = 0;
        asyflexa_opts mo = *O;
        mo.variant = 0;
        asyflexa_t mh = nullptr;
        const int rc = asyflexa_create(&mh, &mp, &mo, stream);
        if (rc) {
            set_error(h, rc, std::string("FP32 master copy: ") + asyflexa_last_error(nullptr));
            return fail(rc);
        }
        h->master = mh;
    }
#undef CKC
    h->msg = "no error";
    *out = h;
    return ASYFLEXA_OK;
}

int asyflexa_destroy(asyflexa_t h) {
    if (!h) return ASYFLEXA_OK;
    cudaStreamSynchronize(h->stream);
    for (auto& pr : h->prof_events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (h->master) asyflexa_destroy(h->master);
    free_buffers(h);
    delete h;
    return ASYFLEXA_OK;
}

int asyflexa_residual_refresh(asyflexa_t h, const void* x) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!x) return set_error(h, ASYFLEXA_EINVAL, "x is NULL");
    return do_refresh(*h, x);
}

int asyflexa_step(asyflexa_t h, void* x, int32_t n_sweeps) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!x) return set_error(h, ASYFLEXA_EINVAL, "x is NULL");
    if (n_sweeps < 0) return set_error(h, ASYFLEXA_EINVAL, "n_sweeps < 0");
    if (n_sweeps == 0) return ASYFLEXA_OK;
    return run_sweeps(*h, x, n_sweeps);
}

// The optimality part of asyflexa_stats from an exact residual's objective pieces and the
// check kernel's measures.
void fill_check_stats(asyflexa_s& h, double F, double rr, double br, const Measures& M, asyflexa_stats* out) {
    const double fs = h.opts.f_star;
    out->F = F;
    out->rel_gap = std::isfinite(fs) ? (F - fs) / std::fabs(fs) : std::nan("");
    const double xs = std::max(1.0, M.xmax);
    out->stat_xhat = M.xh / xs;
    out->stat_mf = M.mf / xs;
    const bool lasso_nobox = h.prob.loss == ASYFLEXA_LOSS_LASSO && !h.prob.lo && !h.prob.hi;
    out->kkt_viol = lasso_nobox ? M.kkt : std::nan("");
    out->nnz = M.nnz;
    out->dual_gap = lasso_dual_gap(h, F, rr, br, M.atr);
    out->checked = 1;
    out->kernel_variant = async_variant(h);
}

int asyflexa_check(asyflexa_t h, const void* x, asyflexa_stats* out) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!x || !out) return set_error(h, ASYFLEXA_EINVAL, "x or out is NULL");
    if (h->master) {
        // optimality of the FP32 problem, evaluated on the master copy
        int rc = asyflexa_check(h->master, x, out);
        if (rc) return set_error(h, rc, std::string("master check: ") + h->master->msg);
        CK(h, cudaMemcpyAsync(h->r, h->master->r, h->prob.m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream),
           "copy master residual");
        h->r_valid = true;
        h->r_x = x;
        out->kernel_launches = h->launches + h->master->launches;
        return ASYFLEXA_OK;
    }
    int rc = do_refresh(*h, x);
    if (rc) return rc;
    double F = 0.0, nnz = 0.0, rr = 0.0, br = 0.0;
    rc = objective(*h, x, &F, &nnz, &rr, &br);
    Measures M{};
    if (!rc) rc = measure(*h, x, &M);
    if (!rc) rc = device_error(*h);
    fill_check_stats(*h, F, rr, br, M, out);
    out->status = rc;
    out->kernel_launches = h->launches;
    return rc;
}

int asyflexa_solve(asyflexa_t h, void* x, asyflexa_stats* out) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!x) return set_error(h, ASYFLEXA_EINVAL, "x is NULL");
    asyflexa_stats st;
    std::memset(&st, 0, sizeof st);
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0), "event");
    CK(h, cudaEventCreate(&e1), "event");
    CK(h, cudaEventRecord(e0, h->stream), "event record");
    int rc = ASYFLEXA_OK;
    if (h->opts.gamma_mu > 0.0) rc = restart_steps(*h);  // each solve runs the step sequence from gamma^0
    if (!rc && h->opts.tau_adapt) {
        rc = set_tau_extra(*h, 0.0);  // and the adaptive proximal weight from 0
        h->tau_down = 0;
    }
    if (!rc && (!h->r_valid || h->r_x != x)) rc = do_refresh(*h, x);
    const double fs = h->opts.f_star;
    const bool known = std::isfinite(fs);
    long long sweeps = 0;
    int status = ASYFLEXA_ENOTCONV;
    double F = NAN, F_prev = NAN, rr = 0.0, br = 0.0;
    bool polish = false;
    // With a low-precision A (unit roundoff u: 2^-8 for BF16, 2^-4 for FP8 e4m3) the objective
    // of the stored problem's minimiser differs from the FP32 problem's by about u^2 relative:
    // the low-precision phase ends at that gap (or tol_gap, if larger)
    double switch_gap = h->opts.tol_gap;
    if (h->master) {
        const double u = h->prob.a_dtype == ASYFLEXA_BF16 ? 0x1p-8 : 0x1p-4;
        switch_gap = std::max(switch_gap, u * u);
    }
    // F is evaluated on an exact residual every check_every sweeps, and the exact stationarity
    // check follows once the gap test passes.  A stationarity check that fails within a factor
    // kNear of tol_stat is repeated after kNearSweeps sweeps (at most check_every times): near
    // tol_stat the stationarity of the FP32 iterates fluctuates from sweep to sweep around the
    // level that the FP32 residual snapshot allows.
    constexpr double kNear = 2.0;
    constexpr int kNearSweeps = 2;
    int next_k = h->opts.check_every, near_checks = 0;
    bool final_ok = false;  // the last exact check describes the returned x
    Measures Mf{};
    // With an FP32 master copy the loop below is the low-precision phase: F and the
    // stationarity are those of the FP32 problem (the refreshes use the master copy), and the
    // phase ends early when a check interval no longer lowers F by switch_tol * |F|.
    while (!rc && sweeps < h->opts.max_sweeps) {
        const int k = static_cast<int>(std::min<long long>(next_k, h->opts.max_sweeps - sweeps));
        rc = run_sweeps(*h, x, k);
        if (rc) break;
        sweeps += k;
        next_k = h->opts.check_every;
        rc = objective(*h, x, &F, nullptr, &rr, &br);
        if (rc) break;
        rc = device_error(*h);
        if (rc) break;
        const double gap = known ? (F - fs) / std::fabs(fs) : NAN;
        const bool stalled = h->master && std::isfinite(F_prev) && (F_prev - F) <= h->opts.switch_tol * std::fabs(F);
        if (h->opts.tau_adapt && std::isfinite(F_prev)) {
            if (F > F_prev + 1e-12 * std::fabs(F_prev)) {
                // the interval raised F: stronger proximal term
                rc = set_tau_extra(*h, h->tau_extra > 0.0 ? 2.0 * h->tau_extra : h->tau_unit);
                h->tau_down = 0;
            } else if (++h->tau_down >= 5 && h->tau_extra > 0.0) {
                // five intervals in a row lowered F: relax it again
                const double t = 0.5 * h->tau_extra;
                rc = set_tau_extra(*h, t < 0.01 * h->tau_unit ? 0.0 : t);
                h->tau_down = 0;
            }
            if (rc) break;
        }
        F_prev = F;
        if (known && !(gap <= switch_gap) && !stalled) continue;
        Measures M{};
        rc = h->master ? measure(*h->master, x, &M) : measure(*h, x, &M);
        if (rc) break;
        const double stat = M.xh / std::max(1.0, M.xmax);
        if (stat <= h->opts.tol_stat && (!known || gap <= h->opts.tol_gap)) {
            status = ASYFLEXA_OK;
            final_ok = !h->master;
            Mf = M;
            break;
        }
        // low-precision phase: once F is within switch_gap of f_star, further low-precision
        // sweeps only approach their own fixed point, so the FP32 polish takes over
        if (stalled || (h->master && known && gap <= switch_gap)) {
            polish = true;
            break;
        }
        if (!h->master && !h->opts.tau_adapt && stat <= kNear * h->opts.tol_stat &&
            ++near_checks <= h->opts.check_every)
            next_k = std::min(kNearSweeps, h->opts.check_every);
    }
    CK(h, cudaEventRecord(e1, h->stream), "event record");
    CK(h, cudaEventSynchronize(e1), "event sync");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    long long polish_sweeps = 0;
    double polish_seconds = 0.0;
    if (!rc && polish && sweeps < h->opts.max_sweeps) {
        // FP32 polish on the master copy, from the current x (its residual is current)
        asyflexa_s& mh = *h->master;
        const int saved = mh.opts.max_sweeps;
        mh.opts.max_sweeps = static_cast<int>(h->opts.max_sweeps - sweeps);
        asyflexa_stats ms_st;
        std::memset(&ms_st, 0, sizeof ms_st);
        const int prc = asyflexa_solve(&mh, x, &ms_st);
        mh.opts.max_sweeps = saved;
        if (prc < 0) return set_error(h, prc, std::string("FP32 polish: ") + mh.msg);
        polish_sweeps = ms_st.sweeps;
        polish_seconds = ms_st.seconds;
        sweeps += polish_sweeps;
        status = prc;
    }
    if (rc) {
        if (out) {
            out->status = rc;
        }
        return rc;
    }
    // final evaluation at the returned x
    if (final_ok) {
        // the loop ended on an exact refresh, objective and check of this x: report them
        fill_check_stats(*h, F, rr, br, Mf, &st);
        rc = device_error(*h);
    } else {
        rc = asyflexa_check(h, x, &st);
    }
    st.sweeps = sweeps;
    st.seconds = ms * 1e-3 + polish_seconds;
    st.polish_sweeps = polish_sweeps;
    st.polish_seconds = polish_seconds;
    st.hbm_bytes = (static_cast<double>(sweeps - polish_sweeps) * h->elt_a + static_cast<double>(polish_sweeps) * 4.0) *
                   static_cast<double>(h->prob.n) * static_cast<double>(h->prob.m);
    {
        unsigned long long hist[32];
        CK(h, cudaMemcpyAsync(hist, h->hist, sizeof hist, cudaMemcpyDeviceToHost, h->stream), "read hist");
        CK(h, cudaStreamSynchronize(h->stream), "synchronize");
        // every sweep updates every block exactly once
        st.block_updates = static_cast<int64_t>(sweeps) * h->nblocks;
        for (int k = 0; k < 32; ++k) st.staleness_hist[k] = hist[k];
    }
    st.kernel_launches = h->launches + (h->master ? h->master->launches : 0);
    st.kernel_variant = async_variant(*h);
    st.tau_extra = h->tau_extra;
    if (!rc) rc = status;
    st.status = rc;
    if (out) *out = st;
    h->last_status = rc;
    return rc;
}

int asyflexa_read_counters(asyflexa_t h, asyflexa_stats* out) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!out) return set_error(h, ASYFLEXA_EINVAL, "out is NULL");
    unsigned long long c[4], hist[32];
    CK(h, cudaMemcpyAsync(c, h->counters, sizeof c, cudaMemcpyDeviceToHost, h->stream), "read counters");
    CK(h, cudaMemcpyAsync(hist, h->hist, sizeof hist, cudaMemcpyDeviceToHost, h->stream), "read hist");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    out->sweeps = h->total_sweeps;
    out->block_updates = static_cast<int64_t>(c[1]);
    for (int k = 0; k < 32; ++k) out->staleness_hist[k] = hist[k];
    out->kernel_launches = h->launches;
    int rc = drain_profile(*h);
    if (rc) return rc;
    out->sweep_kernel_seconds = h->prof_seconds;
    out->sweep_kernel_launches = h->prof_launches;
    out->sweep_kernel_sweeps = h->prof_sweep_total;
    out->kernel_variant = async_variant(*h);
    return device_error(*h);
}

int asyflexa_reset_counters(asyflexa_t h) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    int rc = drain_profile(*h);
    if (rc) return rc;
    CK(h, cudaMemsetAsync(h->counters, 0, 4 * sizeof(unsigned long long), h->stream), "clear counters");
    h->sched_k = 0;
    h->sched_gamma = h->opts.gamma;
    CK(h, cudaMemsetAsync(h->hist, 0, 32 * sizeof(unsigned long long), h->stream), "clear hist");
    h->total_sweeps = 0;
    h->prof_seconds = 0.0;
    h->prof_launches = 0;
    h->prof_sweep_total = 0;
    return ASYFLEXA_OK;
}

int asyflexa_get_residual(asyflexa_t h, double* r_out) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!r_out) return set_error(h, ASYFLEXA_EINVAL, "r_out is NULL");
    CK(h, cudaMemcpyAsync(r_out, h->r, h->prob.m * sizeof(double), cudaMemcpyDeviceToDevice, h->stream), "copy r");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    return ASYFLEXA_OK;
}

int asyflexa_get_weights(asyflexa_t h, double* d_out) {
    if (!h) return set_error(nullptr, ASYFLEXA_EINVAL, "h is NULL");
    if (!d_out) return set_error(h, ASYFLEXA_EINVAL, "d_out is NULL");
    CK(h, cudaMemcpyAsync(d_out, h->dw, h->prob.n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream), "copy d");
    CK(h, cudaStreamSynchronize(h->stream), "synchronize");
    return ASYFLEXA_OK;
}

}  // extern "C"
