// Internal state of an asyflexa handle (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/asyflexa.h"
#include "types.cuh"

// Loss-dependent constants of the method (host side).
inline bool loss_is_dc(const asyflexa_problem& P) {
    return P.loss == ASYFLEXA_LOSS_DC_LOG || P.loss == ASYFLEXA_LOSS_DC_EXP;
}
// factor of A^T r in grad f: 1 for 0.5||Ax-b||^2, 2 for ||Ax-b||^2
inline double loss_s(const asyflexa_problem& P) { return P.loss == ASYFLEXA_LOSS_LASSO ? 1.0 : 2.0; }
// 2c of the nonconvex quadratic's -c||x||^2 (0 for the other losses)
inline double loss_c2(const asyflexa_problem& P) { return P.loss == ASYFLEXA_LOSS_NCQUAD ? 2.0 * P.c : 0.0; }
// the DC regulariser term (kind 0 for the other losses); theta is passed in P.c
inline asyflexa::DcTerm loss_dc(const asyflexa_problem& P) {
    asyflexa::DcTerm d{0, 0.0, 0.0, 0.0};
    if (loss_is_dc(P)) {
        d.kind = P.loss == ASYFLEXA_LOSS_DC_LOG ? 1 : 2;
        d.lam = P.lambda;
        d.theta = P.c;
        d.eta = d.kind == 2 ? P.c : P.c / std::log1p(P.c);
    }
    return d;
}
// weight of ||x||_1 in G: lambda, or lambda * eta for the DC losses
inline double loss_l1(const asyflexa_problem& P) { return loss_is_dc(P) ? P.lambda * loss_dc(P).eta : P.lambda; }

struct asyflexa_s {
    asyflexa_problem prob{};
    asyflexa_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;

    int elt_a = 0;          // bytes per stored element of A
    int vec = 0;            // rows per 16-byte unit of A
    int elt_c = 0;          // bytes of the compute type (double or float)
    int64_t mcopy = 0;      // m rounded up to whole 16-byte units
    int nblocks = 0;

    // sweep kernel geometry
    int sweep_ctas = 0;
    int stages = 0, chunk_rows = 0, tile_rows = 0, ntiles = 0;
    size_t sweep_smem = 0;

    // gather-GEMV / compaction geometry
    int nseg = 0, gemv_rowtiles = 0, compact_tiles = 0;
    int pipe_nseg = 0, pipe_rowtiles = 0;  // pipelined gather (refresh, Jacobi scatter)
    size_t pipe_smem = 0;
    // register-resident async kernel (0 = not used)
    // diminishing stepsize (opts.gamma_mu > 0): update index and step at the next launch, and
    // the device table of the steps of one launch
    long long sched_k = 0;
    double sched_gamma = 0.0;
    // adaptive proximal weight (opts.tau_adapt): tau added on top of opts.tau, its starting
    // increment, and the number of consecutive check intervals that lowered F
    double tau_extra = 0.0, tau_unit = 0.0;
    int tau_down = 0;
    double* gtab = nullptr;
    size_t gtab_cap = 0;
    std::vector<double> gtab_host;

    int reg_upt = 0, reg_cpc = 0, reg_stages = 0;
    size_t reg_smem = 0;
    // the column-in-registers form of the register kernel exists for this problem, and whether
    // the form with a producer warp was asked for instead (asyflexa_opts.variant 3)
    bool reg_rc_ok = false, reg_rc_off = false;
    int reg_g = 1;           // column-in-registers form: columns per barrier
    size_t rc_smem = 0;      // its shared memory


    int check_ctas = 0;
    size_t check_smem = 0;
    bool check_use_smem = false;

    // device buffers (owned)
    double* r = nullptr;                    // mcopy
    double* dw = nullptr;                   // n
    void* delta = nullptr;                  // n of the compute type
    int* list_idx = nullptr;                // n
    void* list_val = nullptr;               // n of the x type
    int* tilecnt = nullptr;                 // compact_tiles
    int* count = nullptr;                   // 1
    void* partial = nullptr;                // nseg * mcopy doubles
    double* norms_part = nullptr;           // kNormsGrid * 4
    double* norms_out = nullptr;            // 4
    unsigned long long* counters = nullptr; // 4
    unsigned long long* hist = nullptr;     // 32
    unsigned long long* meas = nullptr;     // 8
    int* err = nullptr;                     // 1
    int* flag = nullptr;                    // 1
    // the compensated-gradient form of the register kernel exists (FP32 storage)
    bool reg_exact_ok = false;

    // profile=1: event pairs around sweep launches (start, stop, sweeps), drained on read
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
    std::vector<int> prof_sweeps;
    double prof_seconds = 0.0;
    long long prof_launches = 0, prof_sweep_total = 0;

    // FP32 master copy of a BF16/FP8 problem (an internal handle), or null
    asyflexa_s* master = nullptr;

    // host-side bookkeeping
    bool r_valid = false;
    const void* r_x = nullptr;
    long long launches = 0;
    long long total_sweeps = 0;
    int last_status = 0;
    std::string msg;
};

namespace asyflexa {

// Per-storage-type launchers (instantiated in one translation unit per type).
template <typename TA>
struct Launcher {
    static cudaError_t colnorm(asyflexa_s& h);
    static cudaError_t sweep(asyflexa_s& h, void* x, int mode, int sweeps);
    static cudaError_t jacobi_apply(asyflexa_s& h);
    static cudaError_t refresh(asyflexa_s& h, const void* x);
    static cudaError_t norms(asyflexa_s& h, const void* x);
    static cudaError_t check(asyflexa_s& h, const void* x);
    static cudaError_t shift_weights(asyflexa_s& h, double delta);
    static int set_smem_attrs(asyflexa_s& h);
    static int setup_pipe(asyflexa_s& h);
    static int choose_reg(asyflexa_s& h);
};

}  // namespace asyflexa
