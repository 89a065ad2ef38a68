"""Benchmark: AsyFLEXA on the 20000 x 100000 FP32 planted LASSO (blocks of 32 columns).

One step = one solve from x = 0 with the asynchronous persistent-CTA mode until the
relative objective gap is <= 1e-6 and the stationarity merit ||xhat(x) - x||_inf /
max(1, ||x||_inf) is <= 1e-6 (every row of the hot path: block pick, stale residual read,
panel gradient, best response, fixed step, atomic scatter, counters, exact refresh and
checks).  Inputs are resident in HBM before the timed region (A is 8 GB, larger than L2,
so no L2 flush is needed).

Printed JSON line (rank 0): value = block-updates/s of the whole job, ms_per_step = time
to the 1e-6 gap, plus roofline (the async sweep kernel, timed live with CUDA events on its
stream), e2e (host buffers through the public API), the synchronous Jacobi mode on the
same instance, the oracle CPU baseline on a bounded sample, clocks sampled during the
timed region and the kernel-launch count.

--impl reference times the FP64 CPU oracle (the reference arm of this tier) on a bounded
sample of the same workload and prints the same kind of line with "impl": "reference".
Under torchrun with N > 1 each rank solves its own instance (independent replicas: the
path is not sharded), reported as weak scaling.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-6 rel. gap & block-updates/s, async vs sync vs oracle, % HBM peak"
M, N, K_PLANT, LAM, W_BLOCK, GAMMA = 20000, 100000, 1000, 1.0, 32, 0.9
WORKLOAD = "lasso_nesterov_20000x100000_fp32_w32"
SWEEP_SOURCES = ["sweep_async.cuh", "sweep.cuh", "ptx.cuh", "types.cuh", "convert.cuh"]
# the async sweep kernel behind each value of asyflexa_opts.variant / stats.kernel_variant
ASYNC_KERNELS = {
    1: "sweep_kernel<float, async> (staged residual tile)",
    2: "sweep_async_rc_kernel<float, 5> (register increment, column held in registers, residual snapshot "
       "in shared memory)",
    3: "sweep_async_reg_kernel<float, 5> (register increment with a producer warp)",
}


def aggregate_over_ranks(elapsed_s: float, units: float, device="cpu"):
    """Whole-job numbers for independent replicas: the slowest rank's time and the units
    all ranks processed (max / sum all-reduce; a no-op without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), float(units)
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def sweep_kernel_digest() -> str:
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1701_04900_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(kernel: str):
    """DRAM bytes per sweep of the async sweep kernel from a committed ncu summary, if it
    was taken on the current kernel source and on the kernel in use (else None)."""
    p = os.path.join(ROOT, "profiles", "sweep_async_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_digest") != sweep_kernel_digest() or not kernel.startswith(d.get("kernel", "?")):
        return None
    return d


class ClockSampler:
    """nvidia-smi samples of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sms.append(float(parts[0]))
                maxs.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        sms.sort()
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": max(maxs), "samples": len(sms),
                "reasons": sorted(reasons)}


def cpu_oracle_sample(At_sample, b_sample, lam, seconds: float, cores: int):
    """Time the FP64 oracle's cyclic Gauss-Seidel sweeps (w = 32) on a column sample, in a
    fresh interpreter with the BLAS thread count set to ``cores``."""
    import numpy as np
    with tempfile.TemporaryDirectory() as d:
        np.save(os.path.join(d, "At.npy"), At_sample)
        np.save(os.path.join(d, "b.npy"), b_sample)
        code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
import oracle as O
At = np.load({os.path.join(d, 'At.npy')!r}); b = np.load({os.path.join(d, 'b.npy')!r})
m = b.shape[0]
p = O.Problem(A=At[:, :m].astype(np.float64).T, b=b.astype(np.float64), lam={lam})
dw = O.surrogate_weights(p)
x = np.zeros(p.n); r = O.residual(p, x)
nb = len(O.block_ranges(p.n, {W_BLOCK}))
t0 = time.perf_counter(); sweeps = 0
while True:
    x, r = O.gauss_seidel_sweep(p, x, r, dw, {GAMMA}, w={W_BLOCK})
    sweeps += 1
    el = time.perf_counter() - t0
    if el >= {seconds}:
        break
print(json.dumps({{"block_updates": sweeps * nb, "seconds": el, "sweeps": sweeps, "blocks": nb}}))
"""
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(cores)
        res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
        if res.returncode != 0:
            raise RuntimeError(res.stderr)
        return json.loads(res.stdout.strip().splitlines()[-1])


def planted_f_ref(gen):
    """F(x*) on the stored (FP32) data, in FP64 on the host from the support columns."""
    import numpy as np
    sup = gen["support"].cpu().numpy()
    As = gen["At"][gen["support"], :M].double().cpu().numpy()
    xs = gen["x_star"].cpu().numpy()[sup]
    r = As.T @ xs - gen["b"].double().cpu().numpy()
    return 0.5 * float(r @ r) + LAM * float(np.abs(xs).sum())


def run_cpu_core_study(args, m=20000, n=40000, k=400):
    """Section 4.2's core-count study: time to a relative error of F below 1e-4 on the
    Nesterov LASSO the paper uses for it (20000 x 40000, lambda = 1, 1 % nonzero; a smaller
    instance of the same recipe by default), for the multi-core CPU oracle on c = 1, 2, 4, ...
    host threads (variables partitioned among the threads, lock-free) in both of its forms,
    next to the GPU's async solve to the same error.  The Gram form precomputes A^T A and A^T b
    (as the paper's experiments do; the precompute is timed apart); the residual form shares
    r = Ax - b as the GPU does.  The CPU times leave the per-sweep check out; the GPU time is the
    whole solve, checks included."""
    import numpy as np
    import torch
    from paper_1701_04900_gb300 import Solver
    from inputs import nesterov_lasso_torch
    from oracle import cores as oc
    tol = 1e-4
    gen = nesterov_lasso_torch(m, n, k, lam=LAM, seed=0, device="cuda")
    sup = gen["support"]
    r = gen["At"][sup, :m].double().T @ gen["x_star"][sup] - gen["b"].double()
    f_star = 0.5 * float(r @ r) + LAM * float(gen["x_star"].abs().sum())
    out = {"workload": f"lasso_nesterov_{m}x{n}", "nonzeros": k, "lambda": LAM, "tol_rel_err": tol,
           "f_star": "closed form of the generator, on the stored FP32 data"}
    t, st = _time_solves(lambda: Solver(gen["At"], gen["b"], LAM, m=m, block_w=W_BLOCK, mode="async", gamma=GAMMA,
                                        f_star=f_star, tol_gap=tol, tol_stat=1.0, check_every=1, refresh_every=10,
                                        max_sweeps=2000), n)
    out["gpu"] = {"seconds": t, "sweeps": st["sweeps"], "rel_gap": st["rel_gap"], "status": st["status"],
                  "block_w": W_BLOCK, "note": "async solve from x = 0, check every sweep, checks included"}
    At = gen["At"].cpu().numpy()
    b = gen["b"].double().cpu().numpy()
    del gen, r
    torch.cuda.empty_cache()
    avail = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    counts = [c for c in (1, 2, 4, 8, 16, 32, 64) if c <= avail]
    if counts[-1] != avail:
        counts.append(avail)
    out["host_cores"] = avail
    t0 = time.perf_counter()
    Q, q = oc.gram(At, b, m)
    out["gram_precompute_seconds"] = time.perf_counter() - t0
    for form, extra in (("gram", {"Q": Q, "q": q}), ("residual", {})):
        runs = []
        for c in counts:
            _, cs = oc.partitioned_lasso(At, b, m, LAM, gamma=GAMMA, w=1, threads=c, max_sweeps=500, f_star=f_star,
                                         tol=tol, **extra)
            runs.append({"cores": c, "seconds": cs["seconds"], "sweeps": cs["sweeps"],
                         "rel_err": (cs["F"] - f_star) / abs(f_star), "check_seconds": cs["check_seconds"]})
        for rr in runs:
            rr["speedup"] = runs[0]["seconds"] / rr["seconds"]
            rr["gpu_speedup_vs_this"] = rr["seconds"] / t
        out[form] = runs
    return out


# ---------------------------------------------------------------------- cpu_baseline leg
# Besides --impl reference, the one place where bench.py runs the oracle: it times the oracle on
# a bounded sample of the headline instance, runs the core-count study, and evaluates the system
# forms' returned iterates with the oracle (on sampled columns where an instance is large).  No
# value computed here feeds a GPU run.

def _host_residual(At, b64, x, m, chunk=8192):
    """r = A x - b in FP64 on the host from the nonzero columns of x, in column chunks."""
    import numpy as np
    import torch
    nz = np.nonzero(x)[0]
    r = -b64.copy()
    for c0 in range(0, nz.size, chunk):
        cols = nz[c0:c0 + chunk]
        Ac = At[torch.as_tensor(cols, device=At.device, dtype=torch.long), :m].double().cpu().numpy()
        r += Ac.T @ x[cols].astype(np.float64)
    return r


def oracle_check_iterate(At, b, m, x, lam, loss="lasso", c=0.0, lo=None, hi=None, sample=4096, seed=0):
    """The oracle's view of an iterate x of a large instance: F(x) from the exact FP64 residual of
    the nonzero columns, and the merit ||xhat(x) - x||_inf / max(1, ||x||_inf) (Section 4.3) on the
    support (|x_j| > 1e-5 max(1, ||x||_inf)) and `sample` random other columns, evaluated by the
    oracle on the sub-problem of those columns whose residual is r."""
    import numpy as np
    import torch
    import oracle as O
    x64 = x.astype(np.float64)
    r = _host_residual(At, b.double().cpu().numpy(), x, m)
    xabs = np.abs(x64)
    if loss == "lasso":
        F = 0.5 * float(r @ r) + lam * float(xabs.sum())
    else:
        F = float(r @ r) - c * float(x64 @ x64) + lam * float(xabs.sum())
    rng = np.random.default_rng(seed)
    cols = np.union1d(O.lasso_support(x64), rng.choice(x.size, size=min(sample, x.size), replace=False))
    Ac = At[torch.as_tensor(cols, device=At.device, dtype=torch.long), :m].double().cpu().numpy().T
    xs = x64[cols]
    p = O.Problem(A=Ac, b=Ac @ xs - r, lam=lam, loss=loss, c=c,
                  lo=None if lo is None else lo.double().cpu().numpy()[cols],
                  hi=None if hi is None else hi.double().cpu().numpy()[cols])
    merit = float(np.abs(O.xhat_merit(p, xs, O.surrogate_weights(p))).max()) / max(1.0, float(xabs.max()))
    return {"F": F, "merit": merit, "merit_columns": int(cols.size)}


def cpu_form_checks(ctx):
    """The oracle on the forms' outputs (each part reported on its own, errors included)."""
    import numpy as np
    import oracle as O
    out = {}
    fr = ctx.get("form_results", {})
    mp = fr.get("mixed_precision", {})
    try:
        res = {}
        if "lasso" in mp and ctx.get("gen") is not None:
            g = ctx["gen"]
            for name, x in mp["lasso"]["x"].items():
                q = oracle_check_iterate(g["At"], g["b"], M, x, LAM)
                q["rel_gap_vs_planted"] = (q["F"] - ctx["f_ref"]) / abs(ctx["f_ref"])
                res[name] = q
            for name in ("bf16", "fp8"):
                if name in res:
                    res[name]["rel_F_diff_vs_fp32"] = (res[name]["F"] - res["fp32"]["F"]) / abs(res["fp32"]["F"])
            out["mixed_precision_lasso"] = res
        if "ncquad" in mp:
            q = mp["ncquad"]
            res = {}
            for name, x in q["x"].items():
                res[name] = oracle_check_iterate(q["At"], q["b"], q["m"], x, q["lam"], loss="ncquad", c=q["c"],
                                                 lo=q["lo"], hi=q["hi"])
            for name in ("bf16", "fp8"):
                if name in res:
                    res[name]["rel_F_diff_vs_fp32"] = (res[name]["F"] - res["fp32"]["F"]) / abs(res["fp32"]["F"])
            out["mixed_precision_ncquad"] = res
    except Exception as exc:
        out["mixed_precision_error"] = f"{type(exc).__name__}: {exc}"[:300]
    try:
        gr = fr.get("gradient")
        if gr:
            AS, xs, AvS, bv = gr["AS"], gr["x_star_S"], gr["AvS"], gr["bv"]
            v = 2.0 * AvS.T @ (AvS @ xs - bv)          # dL/dx_S of L = ||A_val x - b_val||^2 at x*
            dlam_o, _, _, S = O.lasso_adjoint_gradient(AS, xs, v)
            out["gradient"] = {"oracle_dL_dlam_at_planted_optimum": dlam_o, "library_dL_dlam": gr["dL_dlam"],
                               "rel_diff_vs_oracle": abs(gr["dL_dlam"] - dlam_o) / abs(dlam_o),
                               "support": int(len(S)), "oracle": "FP64 Cholesky on the planted support"}
    except Exception as exc:
        out["gradient_error"] = f"{type(exc).__name__}: {exc}"[:300]
    try:
        bt = fr.get("batched_256")
        if bt:
            rows = []
            for (A, b), x, f in zip(bt["probs"], bt["x"], bt["f_ref"]):
                p = O.Problem(A=A.astype(np.float64), b=b.astype(np.float64), lam=1.0)
                x64 = x.astype(np.float64)
                rows.append({"rel_gap": (O.objective(p, x64) - f) / abs(f),
                             "merit": O.stationarity(O.xhat_merit(p, x64, O.surrogate_weights(p)), x64)})
            out["batched_first_8_instances"] = {"max_rel_gap": max(r["rel_gap"] for r in rows),
                                                "max_merit": max(r["merit"] for r in rows)}
    except Exception as exc:
        out["batched_error"] = f"{type(exc).__name__}: {exc}"[:300]
    try:
        ml = fr.get("multi_lane")
        if ml:
            A = ml["A"].astype(np.float64).T
            merits = []
            for x, lam in zip(ml["X"], ml["lams"]):
                p = O.Problem(A=A, b=ml["b"].astype(np.float64), lam=lam)
                x64 = x.astype(np.float64)
                merits.append(O.stationarity(O.xhat_merit(p, x64, O.surrogate_weights(p)), x64))
            out["multi_lane_lanes_0_31_63"] = {"merits": merits, "max_merit": max(merits)}
    except Exception as exc:
        out["multi_lane_error"] = f"{type(exc).__name__}: {exc}"[:300]
    return out


def cpu_baseline_leg(args, sample, ctx):
    """The oracle timed on the host cores on a bounded sample of the headline instance, the
    core-count study (a 4000 x 8000 instance of the paper's recipe; the paper's 20000 x 40000
    with --cpu-speedup), and the oracle checks of the forms."""
    cores = os.cpu_count() or 1
    At_s, b_s, ncols = sample
    r = cpu_oracle_sample(At_s, b_s, LAM, args.cpu_seconds, cores)
    out = {"value": r["block_updates"] / r["seconds"], "unit": "block-updates/s", "cores": cores, "kind": "oracle",
           "sample": f"FP64 numpy cyclic Gauss-Seidel sweeps (w={W_BLOCK}) over the first {ncols} columns "
                     f"({ncols // W_BLOCK} blocks) of this {M}x{N} instance for {r['seconds']:.1f} s "
                     f"({r['sweeps']} sweeps)"}
    try:
        out["core_study"] = run_cpu_core_study(args) if args.cpu_speedup else \
            run_cpu_core_study(args, m=4000, n=8000, k=80)
    except Exception as exc:  # reported, the headline line still prints
        out["core_study"] = {"error": f"{type(exc).__name__}: {exc}"[:400]}
    if ctx:
        out["form_checks"] = cpu_form_checks(ctx)
    return out


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import torch
    cores = os.cpu_count() or 1
    ncols = 3200
    gen = nesterov_lasso_cpu_sample(ncols)
    At = gen["At"].numpy()
    b = gen["b"].numpy()
    per_step = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(At, b, LAM, min(per_step, 2.0), cores)
    tot_bu, tot_s = 0, 0.0
    for _ in range(args.steps):
        r = cpu_oracle_sample(At, b, LAM, per_step, cores)
        tot_bu += r["block_updates"]
        tot_s += r["seconds"]
    val = tot_bu / tot_s
    sample = (f"cyclic Gauss-Seidel sweeps (w={W_BLOCK}, FP64 numpy) over the first {ncols} of {N} columns "
              f"({ncols // W_BLOCK} blocks) of the {M}x{N} instance, ~{per_step:.0f} s per step")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "block-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(world),
            "cpu_baseline": {"value": val, "unit": "block-updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "block-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    del torch
    print(json.dumps(line), flush=True)


def nesterov_lasso_cpu_sample(ncols):
    from inputs import nesterov_lasso_torch
    return nesterov_lasso_torch(M, N, K_PLANT, lam=LAM, seed=0, device="cpu", n_generate=ncols)


def bench_config(world):
    return {"workload": WORKLOAD, "m": M, "n": N, "planted_nonzeros": K_PLANT, "lambda": LAM,
            "block_w": W_BLOCK, "blocks": math.ceil(N / W_BLOCK), "gamma": GAMMA, "mode": "async",
            "tol_gap": 1e-6, "tol_stat": 1e-6, "x0": "zeros", "generator": "Nesterov-style planted LASSO, seed=rank",
            "l2": "no flush: A (8 GB) is larger than L2 and streamed every sweep",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1701_04900_gb300.build import build_library
    build_library()
    from paper_1701_04900_gb300 import Solver
    from inputs import nesterov_lasso_torch

    gen = nesterov_lasso_torch(M, N, K_PLANT, lam=LAM, seed=rank, device="cuda")
    f_ref = planted_f_ref(gen)
    At, b = gen["At"], gen["b"]
    refresh_every, check_every = args.refresh_every, args.check_every
    s = Solver(At, b, LAM, m=M, block_w=W_BLOCK, mode="async", gamma=GAMMA, refresh_every=refresh_every,
               check_every=check_every, max_sweeps=args.max_sweeps, f_star=f_ref, profile=True,
               variant=args.variant)
    x = torch.zeros(N, dtype=torch.float32, device="cuda")

    def one_step():
        x.zero_()
        return s.solve(x)

    for _ in range(args.warmup):
        one_step()
    s.reset_counters()
    launches0 = s.read_counters()["kernel_launches"]
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    stats, step_ev = [], []
    for _ in range(args.steps):
        stats.append(one_step())
        step_ev.append(torch.cuda.Event(enable_timing=True))
        step_ev[-1].record()
    ev1.record()
    torch.cuda.synchronize()
    step_ms = [ev0.elapsed_time(step_ev[0])] + [a.elapsed_time(b) for a, b in zip(step_ev, step_ev[1:])]
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    ctr = s.read_counters()
    launches = ctr["kernel_launches"] - launches0
    bu = sum(st["block_updates"] for st in stats)
    elapsed_all, bu_all = aggregate_over_ranks(elapsed, float(bu), device="cuda")

    # roofline of the dominant kernel: the async sweep kernel, timed live with CUDA events
    # recorded on its own stream by the library (profile=True)
    peak, peak_kind = measured_peaks()
    alg_bytes_per_sweep = N * M * 4 + N * (4 + 4 + 8)
    sk_launches = max(1, ctr["sweep_kernel_launches"])
    avg_launch_s = ctr["sweep_kernel_seconds"] / sk_launches
    sweeps_per_launch = ctr["sweep_kernel_sweeps"] / sk_launches
    achieved = alg_bytes_per_sweep * sweeps_per_launch / avg_launch_s / 1e9
    kernel = ASYNC_KERNELS[ctr["kernel_variant"]]
    tr = profile_traffic(kernel)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tr["dram_bytes_per_sweep"] * sweeps_per_launch if tr else None),
                "kernel": kernel,
                "peak_kind": peak_kind,
                "avg_launch_ms": avg_launch_s * 1e3, "sweeps_per_launch": sweeps_per_launch,
                "algorithmic_bytes_per_sweep": alg_bytes_per_sweep,
                "share_of_step_time": ctr["sweep_kernel_seconds"] / elapsed}

    last = stats[-1]
    result = {"metric": METRIC, "value": bu_all / elapsed_all, "unit": "block-updates/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_all / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic (Nesterov-style planted LASSO generated on the device)",
              "config": bench_config(world),
              "time_to_gap_s": elapsed / args.steps, "step_ms": [round(t, 3) for t in step_ms],
              "sweeps_to_gap": last["sweeps"],
              "rel_gap": last["rel_gap"], "stat_xhat": last["stat_xhat"], "stat_mf": last["stat_mf"],
              "kkt_viol": last["kkt_viol"], "nnz": last["nnz"], "status": last["status"],
              "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks,
              "staleness_hist": ctr["staleness_hist"]}

    # support recovery of the returned x: entries above 1e-5 max(1, ||x||_inf) (the fixed step
    # leaves geometric tails on coordinates that are zero at the optimum) against the planted
    # support
    sel = x.abs() > 1e-5 * max(1.0, float(x.abs().max()))
    planted = torch.zeros(N, dtype=torch.bool, device="cuda")
    planted[gen["support"]] = True
    hits = int((sel & planted).sum())
    result["support_recovery"] = {"nnz": int((x != 0).sum()), "nnz_rel_1e-5": int(sel.sum()),
                                  "planted": int(planted.sum()), "precision": hits / max(1, int(sel.sum())),
                                  "recall": hits / max(1, int(planted.sum()))}
    if rank == 0 and not args.no_sync:
        result["sync"] = run_sync(gen, f_ref, args)
    if rank == 0 and not args.no_e2e:
        result["e2e"] = run_e2e(gen, f_ref, args, refresh_every, check_every)
    cpu_sample = None
    if rank == 0 and not args.no_cpu:
        ncols = 3200
        cpu_sample = (At[:ncols].cpu().numpy(), b.cpu().numpy(), ncols)
    s.close()
    ctx = {"gen": gen, "f_ref": f_ref}
    del At, b
    if rank == 0 and not args.no_forms:
        result["forms"] = {}
        for name, fn in (("stepsize", run_form_stepsize), ("mixed_precision", run_form_mixed_precision),
                         ("gradient", run_form_gradient), ("batched", run_form_batched),
                         ("liu_wright", run_form_liu_wright), ("dc_regularisers", run_form_dc)):
            try:
                result["forms"][name] = fn(args, ctx)
            except Exception as exc:  # a failing form is reported, the headline line still prints
                result["forms"][name] = {"error": f"{type(exc).__name__}: {exc}"[:400]}
            torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline_leg(args, cpu_sample, ctx if not args.no_forms else None)
    ctx.clear()
    del gen
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)
    del np


def jacobi_safe_tau_rel(At, m: int, n: int, gamma: float = GAMMA):
    """Descent-safe relative proximal weight of the Jacobi mode: 1 + tau_rel = (gamma/2) *
    lambda_max(K^-1/2 A^T A K^-1/2) * 1.01, K = diag(||a_j||^2) (40 power iterations)."""
    import torch
    kap = torch.empty(n, dtype=torch.float64, device="cuda")
    for j0 in range(0, n, 8192):
        kap[j0:j0 + 8192] = (At[j0:j0 + 8192, :m].double() ** 2).sum(dim=1)
    sc = (1.0 / kap.sqrt()).float()
    v = torch.randn(n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    v /= v.norm()
    lmax = 0.0
    for _ in range(40):
        u = At[:, :m].T @ (sc * v)
        wv = sc * (At[:, :m] @ u)
        lmax = float(wv.norm())
        v = wv / lmax
    return max(0.0, 0.5 * gamma * lmax * 1.01 - 1.0), lmax


def run_sync(gen, f_ref, args):
    """Deterministic Jacobi mode on the same instance, with the descent-safe relative
    proximal weight 1 + tau_rel = (gamma/2) * lambda_max(K^-1/2 A^T A K^-1/2) * 1.01."""
    import torch
    from paper_1701_04900_gb300 import Solver
    At = gen["At"]
    tau_rel, lmax = jacobi_safe_tau_rel(At, M, N)
    s = Solver(At, gen["b"], LAM, m=M, block_w=W_BLOCK, mode="sync", gamma=GAMMA, tau_rel=tau_rel,
               refresh_every=args.refresh_every, check_every=args.check_every, max_sweeps=args.sync_sweeps,
               f_star=f_ref, profile=True)
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    s.step(x, 2)  # warm-up
    x.zero_()
    s.refresh(x)
    s.reset_counters()
    st = s.solve(x)
    ctr = s.read_counters()
    s.close()
    return {"mode": "sync (Jacobi)", "tau_rel": tau_rel, "lambda_max_normalized_gram": lmax,
            "seconds": st["seconds"], "sweeps": st["sweeps"], "rel_gap": st["rel_gap"],
            "stat_xhat": st["stat_xhat"], "status": st["status"],
            "block_updates_per_s": st["block_updates"] / st["seconds"] if st["seconds"] else None,
            "sweep_kernel_ms": 1e3 * ctr["sweep_kernel_seconds"] / max(1, ctr["sweep_kernel_launches"]),
            "reached_1e-6": bool(st["status"] == 0)}


def run_e2e(gen, f_ref, args, refresh_every, check_every):
    """Same metric through the public API from pinned host buffers: every step copies A, b
    and x0 host->device, creates the solver (weights), solves, and copies x back."""
    import torch
    from paper_1701_04900_gb300 import Solver
    At_h = gen["At"].cpu().pin_memory()
    b_h = gen["b"].cpu().pin_memory()
    x0_h = torch.zeros(N, dtype=torch.float32).pin_memory()
    x_h = torch.empty(N, dtype=torch.float32).pin_memory()
    At_d = gen["At"]          # same contents: the copy overwrites with identical data
    b_d = torch.empty_like(gen["b"])
    x_d = torch.empty(N, dtype=torch.float32, device="cuda")
    h2d = At_h.numel() * 4 + b_h.numel() * 4 + x0_h.numel() * 4
    d2h = x_h.numel() * 4
    steps = max(1, min(args.steps, 3))

    def step():
        At_d.copy_(At_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        x_d.copy_(x0_h, non_blocking=True)
        s = Solver(At_d, b_d, LAM, m=M, block_w=W_BLOCK, mode="async", gamma=GAMMA, refresh_every=refresh_every,
                   check_every=check_every, max_sweeps=args.max_sweeps, f_star=f_ref)
        st = s.solve(x_d)
        x_h.copy_(x_d, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        s.close()
        return st

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bu = 0
    for _ in range(steps):
        bu += step()["block_updates"]
    el = time.perf_counter() - t0
    return {"value": bu / el, "unit": "block-updates/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "steps": steps, "seconds_per_step": el / steps}


def _time_solves(make_solver, n, repeats=2, return_x=False):
    """Warm-up solve, then the best of `repeats` timed solves from x = 0 (same work each)."""
    import torch
    s = make_solver()
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    s.solve(x)
    times = []
    st = None
    for _ in range(repeats):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.solve(x)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    s.close()
    return (min(times), st, x) if return_x else (min(times), st)


def run_form_stepsize(args, ctx):
    """NEXT row: the diminishing stepsize rule of the paper's experiments (Section 4),
    gamma^0 = 1, gamma^{k+1} = gamma^k (1 - 1e-6 gamma^k) per block update, against the fixed
    step gamma = 0.9 of the headline, on the same 20000 x 100000 LASSO to a 1e-6 gap."""
    from paper_1701_04900_gb300 import Solver
    gen = ctx["gen"]
    out = {"workload": f"lasso_nesterov_{M}x{N}"}
    for name, kw in (("fixed_0.9", dict(gamma=GAMMA)), ("diminishing_1_1e-6", dict(gamma=1.0, gamma_mu=1e-6))):
        t, st = _time_solves(lambda: Solver(gen["At"], gen["b"], LAM, m=M, block_w=W_BLOCK, mode="async",
                                            refresh_every=10, check_every=10, max_sweeps=2000, tol_stat=1e-6,
                                            f_star=ctx["f_ref"], **kw), N)
        out[name] = {"seconds": t, "sweeps": st["sweeps"], "rel_gap": st["rel_gap"], "stat_xhat": st["stat_xhat"],
                     "status": st["status"]}
    out["diminishing_speedup_vs_fixed"] = out["fixed_0.9"]["seconds"] / out["diminishing_1_1e-6"]["seconds"]
    return out


def run_form_mixed_precision(args, ctx):
    """System form (1): A stored as FP32, BF16 or FP8-e4m3 codes with per-column scales (library
    quantiser).  The BF16/FP8 runs refresh and check on the FP32 master copy and finish with
    FP32 polish sweeps; each result is stated against the FP32 problem.
    (a) The 20000 x 100000 LASSO of the headline, to a 1e-6 relative gap against the planted
        optimum's objective (FP64) and ||xhat(x) - x||_inf / max(1, ||x||_inf) <= 1e-6.
    (b) The nonconvex quadratic 10000 x 50000 with box |x| <= 1, to the same stationarity.
    Reports time, sweeps and speedup over the plain FP32 form at that accuracy."""
    import torch
    from paper_1701_04900_gb300 import Solver
    from paper_1701_04900_gb300.native import quantize
    from inputs import ncquad_problem_torch
    out = {}
    kinds = {"fp32": None, "bf16": "bf16", "fp8": "fp8"}
    elt = {"fp32": 4, "bf16": 2, "fp8": 1}

    def run_all(At, b, lam, m, n, common, keep):
        res = {}
        for name, kind in kinds.items():
            if kind is None:
                t, st, x = _time_solves(lambda: Solver(At, b, lam, m=m, **common), n, return_x=True)
            else:
                Q, sc = quantize(At, m, kind)
                t, st, x = _time_solves(lambda: Solver(Q, b, lam, m=m, col_scale=sc, A_master=At, **common), n,
                                        return_x=True)
                del Q, sc
            res[name] = {"seconds": t, "sweeps": st["sweeps"], "polish_sweeps": st["polish_sweeps"],
                         "rel_gap": st["rel_gap"], "stat_xhat": st["stat_xhat"], "F": st["F"], "nnz": st["nnz"],
                         "status": st["status"], "A_bytes_per_sweep": n * m * elt[name]}
            keep[name] = x.cpu().numpy()
        for name in ("bf16", "fp8"):
            res[name]["speedup_vs_fp32"] = res["fp32"]["seconds"] / res[name]["seconds"]
        return res

    keep = ctx.setdefault("form_results", {}).setdefault("mixed_precision", {})
    gen = ctx.get("gen")
    if gen is not None:
        common = dict(block_w=W_BLOCK, mode="async", gamma=GAMMA, max_sweeps=2000, check_every=10,
                      refresh_every=10, tol_stat=1e-6, f_star=ctx["f_ref"])
        kl = keep.setdefault("lasso", {"x": {}})
        out["lasso"] = dict(workload=f"lasso_nesterov_{M}x{N}",
                            **run_all(gen["At"], gen["b"], LAM, M, N, common, kl["x"]))
        del gen
    m, n = 10000, 50000
    g = ncquad_problem_torch(m, n, seed=0, device="cuda")
    common = dict(loss="ncquad", c=g["c"], lo=g["lo"], hi=g["hi"], block_w=W_BLOCK, mode="async", gamma=GAMMA,
                  max_sweeps=4000, check_every=10, refresh_every=10, tol_stat=1e-6)
    kq = keep.setdefault("ncquad", {"x": {}})
    out["ncquad"] = dict(workload=f"ncquad_{m}x{n}_box1", c=g["c"], lam=g["lam"],
                         **run_all(g["At"], g["b"], g["lam"], m, n, common, kq["x"]))
    kq.update(At=g["At"], b=g["b"], lam=g["lam"], c=g["c"], lo=g["lo"], hi=g["hi"], m=m, n=n)
    return out


def run_form_gradient(args, ctx=None):
    """System form (3): L(lam, b) = ||A_val x*(lam, b) - b_val||^2 on the LASSO train split
    5000 x 20000 (Nesterov planted at lam = 1) with a 2000-row validation split from the same
    generator.  Times the forward solve, the backward (adjoint block update on the support,
    through torch.autograd), and central differences (2 solves); then tunes lam by 20 steps of
    gradient descent on log(lam) (first step normalised to 0.1 in log(lam))."""
    import torch
    from inputs import nesterov_lasso_torch, validation_rows_torch
    from paper_1701_04900_gb300.autograd import lasso_solution
    m, n, k = 5000, 20000, 200
    gen = nesterov_lasso_torch(m, n, k, lam=1.0, seed=0, device="cuda")
    val = validation_rows_torch(gen, 2000, seed=1)
    At, b = gen["At"], gen["b"]
    Av = val["At"][:, :2000].T.contiguous()
    bv = val["b"]
    solve_kw = dict(mode="async", block_w=W_BLOCK, gamma=GAMMA, max_sweeps=4000, check_every=10, tol_stat=1e-6,
                    num_ctas=32)

    def fwd_bwd(lam_v):
        lam = torch.tensor(lam_v, dtype=torch.float64, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = lasso_solution(lam, b, At, m, solve_kw)
        loss = ((Av @ x - bv) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return float(loss.detach()), float(lam.grad), t1 - t0, t2 - t1, int((x != 0).sum())

    def loss_only(lam_v):
        with torch.no_grad():
            x = lasso_solution(torch.tensor(lam_v, dtype=torch.float64, device="cuda"), b, At, m, solve_kw)
            return float(((Av @ x - bv) ** 2).sum())

    fwd_bwd(1.0)                                       # warm-up
    L0, g0, t_fwd, t_bwd, nnz = fwd_bwd(1.0)
    h = 1e-4
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fd = (loss_only(1.0 + h) - loss_only(1.0 - h)) / (2 * h)
    t_fd = time.perf_counter() - t0
    # 20 gradient steps on log(lam) with step control: move against the sign of
    # dL/dlog(lam) = lam dL/dlam; a step that lowers L is kept and the step grows by 1.5,
    # otherwise it is undone and the step halves (L(lam) has a sharp minimum near the planted
    # lam = 1, so plain fixed steps overshoot)
    log_best, L_best, dlog = 0.0, L0, g0
    step = 0.05
    traj = []
    t0 = time.perf_counter()
    for _ in range(20):
        cand = log_best - step * (1.0 if dlog > 0 else -1.0)
        L, g, _, _, _ = fwd_bwd(math.exp(cand))
        traj.append((math.exp(cand), L))
        if L < L_best:
            log_best, L_best, dlog = cand, L, math.exp(cand) * g
            step *= 1.5
        else:
            step *= 0.5
    t_tune = time.perf_counter() - t0
    if ctx is not None:
        sup = gen["support"]
        ctx.setdefault("form_results", {})["gradient"] = {
            "AS": At[sup, :m].double().T.cpu().numpy(), "x_star_S": gen["x_star"][sup].cpu().numpy(),
            "AvS": val["At"][sup, :2000].double().T.cpu().numpy(), "bv": bv.double().cpu().numpy(), "dL_dlam": g0}
    return {"workload": f"lasso_train_{m}x{n}_val_2000", "loss_at_lam1": L0, "dL_dlam": g0, "fd_dL_dlam": fd,
            "rel_diff_vs_fd": abs(g0 - fd) / max(abs(fd), 1e-30), "forward_s": t_fwd, "backward_s": t_bwd,
            "fd_two_solves_s": t_fd, "backward_speedup_vs_fd": t_fd / max(t_bwd, 1e-12), "nnz": nnz,
            "tune_20_steps_s": t_tune, "lambda_final": math.exp(log_best), "loss_at_start": L0, "loss_final": L_best}


def _batch_solve_timed(make, xs, f_star=None):
    """Warm-up solve (the autotuner runs on the first solve of a batch shape), then one timed
    solve from x = 0 (wall clock around the call; synchronised on both sides), then the
    library's exact check of every problem (outside the timed region)."""
    import torch
    bs = make()
    bs.solve(xs, f_star=f_star)
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per, tot = bs.solve(xs, f_star=f_star)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    exact = bs.check(xs, f_star=f_star)
    bs.close()
    return t, per, tot, exact


def _status_counts(stats):
    out = {}
    for st in stats:
        k = {0: "ok", 1: "not_converged", -5: "nonfinite"}.get(st["status"], str(st["status"]))
        out[k] = out.get(k, 0) + 1
    return out


def run_form_batched(args, ctx=None):
    """System form (2).
    (a) 256 LASSO instances of uneven sizes (m ~ U[500, 4000], n ~ U[2000, 20000], 2% planted,
        FP32) solved together in ONE persistent launch (the Gauss-Seidel form: one CTA per
        instance at a time from a largest-first queue, in-kernel stopping tests, launch
        captured in a CUDA graph, launch shape autotuned and cached), until every instance
        has a 1e-6 relative gap and ||xhat(x) - x||_inf / max(1, ||x||_inf) <= 1e-6; against
        measured sequential solves of all 256 instances with the plain async form to the same
        gap and stationarity.
    (b) A 64-point geometric lambda path on one 5000 x 20000 instance (lambda_max =
        ||A^T b||_inf down to the planted lambda = 1), every lane to stationarity <= 1e-6:
        the batch API's automatic choice (shared A: the multi-lane form), the Gauss-Seidel
        form, the async rounds form, the multi-lane tensor-core form called directly, and 64
        sequential warm-started (and cold) plain solves."""
    import numpy as np
    import torch
    from paper_1701_04900_gb300 import Solver
    from paper_1701_04900_gb300.batch import BatchSolver, MultiLaneSolver
    from inputs import nesterov_lasso_torch
    rng = np.random.default_rng(0)
    probs, f_ref, gens = [], [], []
    for i in range(256):
        m = int(rng.integers(500, 4001))
        n = int(rng.integers(2000, 20001))
        g = nesterov_lasso_torch(m, n, max(1, int(0.02 * n)), lam=1.0, seed=1000 + i, device="cuda")
        sup = g["support"]
        r = g["At"][sup, :m].double().T @ g["x_star"][sup] - g["b"].double()
        f_ref.append(0.5 * float(r @ r) + float(g["x_star"].abs().sum()))
        probs.append(dict(At=g["At"], b=g["b"], lam=1.0, m=m))
        gens.append((m, n))
    total_bytes = sum(m * n * 4 for m, n in gens)
    xs = [torch.zeros(p["At"].shape[0], dtype=torch.float32, device="cuda") for p in probs]
    t_batch, per, tot, exact = _batch_solve_timed(
        lambda: BatchSolver(probs, max_sweeps=3000, check_every=10, tol_stat=1e-6), xs, f_ref)
    swept = sum(st["sweeps"] * m * n * 4 for st, (m, n) in zip(per, gens))
    # sequential: the plain asynchronous form, one instance after another, with at most
    # about m/4 columns in flight (max(1, m / (4 w)) CTAs of w = 32 columns)
    t_seq, seq_stats, seq_times = 0.0, [], []
    for i, p in enumerate(probs):
        s = Solver(p["At"], p["b"], 1.0, m=p["m"], block_w=W_BLOCK, mode="async", refresh_every=10,
                   check_every=10, max_sweeps=3000, f_star=f_ref[i], tol_stat=1e-6,
                   num_ctas=max(1, min(152, p["m"] // (4 * W_BLOCK))))
        x = torch.zeros(p["At"].shape[0], dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        seq_stats.append(s.solve(x))
        torch.cuda.synchronize()
        seq_times.append(time.perf_counter() - t1)
        t_seq += seq_times[-1]
        s.close()
    # the Gauss-Seidel form's per-problem CTA times: their sum over the SMs bounds what a perfect
    # packing would take; the longest is the problem that holds the batch
    cta = [st["seconds"] for st in per]
    budget_bound = [i for i, st in enumerate(per) if st["status"] == 1]
    batched = {"instances": 256, "A_bytes": total_bytes, "form": "gs" if tot["batch_form"] == 4 else "async",
               "ctas_per_sm": tot["ctas_per_sm"], "consumer_warps": tot["kernel_variant"],
               "seconds_to_all_converged": t_batch, "status": tot["status"], "per_instance_status": _status_counts(per),
               "max_sweeps": tot["sweeps"], "mean_sweeps": sum(st["sweeps"] for st in per) / len(per),
               "block_w": tot["block_w"], "block_updates_per_s": tot["block_updates"] / t_batch,
               "sweep_A_bytes_per_s": swept / t_batch,
               "problems_in_later_launches": tot["handed_over"],
               "cta_seconds_sum": sum(cta), "cta_seconds_max": max(cta),
               "cta_seconds_sum_over_sms": sum(cta) / torch.cuda.get_device_properties(0).multi_processor_count,
               "not_converged_instances": [{"index": i, "m": gens[i][0], "n": gens[i][1], "sweeps": per[i]["sweeps"],
                                            "rel_gap": per[i]["rel_gap"], "cta_seconds": per[i]["seconds"],
                                            "sequential_seconds": seq_times[i],
                                            "sequential_status": seq_stats[i]["status"]} for i in budget_bound],
               "max_rel_gap": max(st["rel_gap"] for st in per),
               "max_stat_xhat": max(st["stat_xhat"] for st in per),
               "max_stat_xhat_exact_check": max(st["stat_xhat"] for st in exact),
               "max_rel_gap_exact_check": max(st["rel_gap"] for st in exact),
               "sequential_seconds_all_256": t_seq, "sequential_status": _status_counts(seq_stats),
               "sequential_max_stat_xhat": max(st["stat_xhat"] for st in seq_stats),
               "sequential_block_w": W_BLOCK,
               "speedup_vs_sequential": t_seq / t_batch}
    if ctx is not None:
        ctx.setdefault("form_results", {})["batched_256"] = {
            "x": [x.cpu().numpy() for x in xs[:8]], "probs": [(p["At"][:, :p["m"]].cpu().numpy().T,
                                                               p["b"].cpu().numpy()) for p in probs[:8]],
            "f_ref": f_ref[:8]}
    del probs, xs, gens
    torch.cuda.empty_cache()

    m, n = 5000, 20000
    g = nesterov_lasso_torch(m, n, 200, lam=1.0, seed=7, device="cuda")
    At, b = g["At"], g["b"]
    lam_max = float((At[:, :m].double() @ b.double()).abs().max())
    lams = [lam_max * (1.0 / lam_max) ** (k / 63) for k in range(64)]
    sup = g["support"]
    r = At[sup, :m].double().T @ g["x_star"][sup] - b.double()
    f1 = 0.5 * float(r @ r) + float(g["x_star"].abs().sum())
    base = dict(At=At, b=b, m=m)
    path = {"lambdas": 64, "lambda_max": lam_max, "tol_stat": 1e-6}
    for name, kw in (("batched_auto", dict(shared_a=True, check_every=10, refresh_every=10)),
                     ("gs", dict(form="gs", shared_a=True, check_every=10)),
                     ("async_rounds", dict(form="async", shared_a=True, block_w=32, refresh_every=10,
                                           switch_tol=1e-9))):
        xs = [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in lams]
        t, per, tot, exact = _batch_solve_timed(
            lambda: BatchSolver([dict(base, lam=l) for l in lams], max_sweeps=3000, tol_stat=1e-6, **kw), xs)
        path[name] = {"seconds": t, "status": tot["status"], "per_lane_status": _status_counts(per),
                      "form": {2: "async", 4: "gs", 8: "multi"}.get(tot["batch_form"], "?"),
                      "max_sweeps": tot["sweeps"], "max_stat_xhat_exact_check": max(q["stat_xhat"] for q in exact),
                      "last_lane_rel_gap_vs_planted": (exact[-1]["F"] - f1) / f1}
        del xs
    # sequential warm-started path (each solve to the same stationarity)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_sweeps, seq_stat = 0, 0.0
    for l in lams:
        s = Solver(At, b, l, m=m, block_w=32, mode="async", refresh_every=10, check_every=10, max_sweeps=3000,
                   tol_stat=1e-6)
        st = s.solve(x)
        seq_sweeps += st["sweeps"]
        seq_stat = max(seq_stat, st["stat_xhat"])
        s.close()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    # sequential cold starts (every lambda from x = 0, as the batched lanes start)
    t0 = time.perf_counter()
    cold_sweeps = 0
    for l in lams:
        x = torch.zeros(n, dtype=torch.float32, device="cuda")
        s = Solver(At, b, l, m=m, block_w=32, mode="async", refresh_every=10, check_every=10, max_sweeps=3000,
                   tol_stat=1e-6)
        cold_sweeps += s.solve(x)["sweeps"]
        s.close()
    torch.cuda.synchronize()
    t_cold = time.perf_counter() - t0
    # the multi-lane form: every block update for all 64 lanes at once on the tensor cores
    Bm = b.reshape(1, -1).expand(64, -1).contiguous()
    ml = MultiLaneSolver(At, Bm, lams, m, refresh_every=10, check_every=10, max_sweeps=3000, tol_stat=1e-6)
    Xm = torch.zeros((64, n), dtype=torch.float32, device="cuda")
    ml.solve(Xm)                                   # warm-up (same work)
    Xm.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mper, mtot = ml.solve(Xm)
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    ml.close()
    path["multi_lane"] = {"seconds": t_multi, "sweeps": mtot["sweeps"], "status": mtot["status"],
                          "max_stat_xhat": max(q["stat_xhat"] for q in mper),
                          "last_lane_rel_gap_vs_planted": (mper[-1]["F"] - f1) / f1}
    path["sequential_warm"] = {"seconds": t_seq, "sweeps": seq_sweeps, "max_stat_xhat": seq_stat}
    path["sequential_cold"] = {"seconds": t_cold, "sweeps": cold_sweeps}
    for name in ("batched_auto", "gs", "async_rounds", "multi_lane"):
        path[name]["speedup_vs_sequential_warm"] = t_seq / path[name]["seconds"]
        path[name]["speedup_vs_sequential_cold"] = t_cold / path[name]["seconds"]
    if ctx is not None:
        ctx.setdefault("form_results", {})["multi_lane"] = {
            "X": Xm[[0, 31, 63]].cpu().numpy(), "lams": [lams[0], lams[31], lams[63]],
            "A": At[:, :m].cpu().numpy(), "b": b.cpu().numpy()}
    return {"batched": batched, "lambda_path": path}


def run_form_liu_wright(args, ctx=None):
    """NEXT row: the Gaussian LASSO set of Section 4.2 (m = 20000, n = 40000, s = 40, sigma =
    0.01, lam = 20 sqrt(m log n) sigma), whose optimum is not known: async and sync solves to
    stationarity <= 1e-6, with the duality-gap certificate reported and the relative difference
    of the two final objectives (the paper estimates F* by a long synchronous run)."""
    import torch
    from paper_1701_04900_gb300 import Solver
    from inputs import liu_wright_lasso_torch
    m, n = 20000, 40000
    g = liu_wright_lasso_torch(m, n, 40, sigma=0.01, seed=0, device="cuda")
    out = {"workload": f"lasso_gaussian_{m}x{n}_s40", "lambda": g["lam"]}
    tau_rel, _ = jacobi_safe_tau_rel(g["At"], m, n)
    for mode, extra in (("async", {}), ("sync", {"tau_rel": tau_rel})):
        t, st = _time_solves(lambda: Solver(g["At"], g["b"], g["lam"], m=m, block_w=W_BLOCK, mode=mode, gamma=GAMMA,
                                            max_sweeps=3000, check_every=10, refresh_every=10, tol_stat=1e-6,
                                            **extra), n)
        out[mode] = {"seconds": t, "sweeps": st["sweeps"], "dual_gap": st["dual_gap"], "stat_xhat": st["stat_xhat"],
                     "F": st["F"], "nnz": st["nnz"], "status": st["status"]}
    out["async_speedup_vs_sync"] = out["sync"]["seconds"] / out["async"]["seconds"]
    out["rel_objective_difference_async_sync"] = abs(out["async"]["F"] - out["sync"]["F"]) / abs(out["sync"]["F"])
    del g
    torch.cuda.empty_cache()
    return out


def run_form_dc(args, ctx=None):
    """NEXT row: the nonconvex sparse-learning problem of Section 4.3, F = ||Ax-b||^2 + lam H(x)
    with the log regulariser (theta = 20) on the 20000 x 40000 instance shape the paper uses
    (unit-norm Gaussian columns, 5% nonzero xbar, noise sigma = 0.1).  Async and sync (Jacobi)
    solves from x = 0 to ||xhat(x) - x||_inf / max(1, ||x||_inf) <= 1e-6, plus the exp
    regulariser in async mode."""
    import torch
    from paper_1701_04900_gb300 import Solver
    from inputs import dc_problem_torch
    m, n = 20000, 40000
    out = {}
    for reg in ("log", "exp"):
        g = dc_problem_torch(m, n, reg=reg, theta=20.0, seed=0, device="cuda")
        modes = [("async", {})]
        if reg == "log":
            tau_rel, _ = jacobi_safe_tau_rel(g["At"], m, n)
            modes.append(("sync", {"tau_rel": tau_rel}))
        res = {"lambda": g["lam"], "theta": g["theta"]}
        for mode, extra in modes:
            t, st = _time_solves(lambda: Solver(g["At"], g["b"], g["lam"], m=m, loss="dc_" + reg, theta=g["theta"],
                                                block_w=W_BLOCK, mode=mode, gamma=GAMMA, max_sweeps=3000,
                                                check_every=10, refresh_every=10, tol_stat=1e-6, **extra), n)
            res[mode] = {"seconds": t, "sweeps": st["sweeps"], "stat_xhat": st["stat_xhat"], "F": st["F"],
                         "nnz": st["nnz"], "status": st["status"],
                         "block_updates_per_s": st["block_updates"] / t if t else None}
        if "sync" in res:
            res["async_speedup_vs_sync"] = res["sync"]["seconds"] / res["async"]["seconds"]
        out[f"dc_{reg}_{m}x{n}"] = res
        del g
        torch.cuda.empty_cache()
    return out


def run_ncu_case_multi():
    """ncu case of the multi-lane kernel: the 64-lane lambda path on the 5000 x 20000 instance
    (A = 400 MB, larger than L2), one solve capped at 10 sweeps: a refresh launch, then one
    launch of 10 sweeps of every lane (mode 0), then the objective and gradient launches."""
    import torch
    from paper_1701_04900_gb300.batch import MultiLaneSolver
    from inputs import nesterov_lasso_torch
    m, n, k = 5000, 20000, 64
    g = nesterov_lasso_torch(m, n, 200, lam=1.0, seed=7, device="cuda")
    lam_max = float((g["At"][:, :m].double() @ g["b"].double()).abs().max())
    lams = [lam_max * (1.0 / lam_max) ** (i / (k - 1)) for i in range(k)]
    B = g["b"].reshape(1, -1).expand(k, -1).contiguous()
    ml = MultiLaneSolver(g["At"], B, lams, m, refresh_every=10, check_every=10, max_sweeps=10)
    X = torch.zeros((k, n), dtype=torch.float32, device="cuda")
    per, tot = ml.solve(X)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": True, "mode": "multi", "lanes": k, "sweeps": tot["sweeps"],
                      "F_last_lane": per[-1]["F"]}))
    ml.close()


def run_ncu_case_batch():
    """ncu case of the batched Gauss-Seidel kernel: 152 planted Nesterov instances, m ~ U[500,
    2000], n ~ U[2000, 6000] (about 3 GB in all, larger than L2), 20 sweeps.  The first solve
    runs the autotuner (one-sweep launches) and its launch; the second reuses the cached shape:
    its single launch is the one summarised."""
    import numpy as np
    import torch
    from paper_1701_04900_gb300.batch import BatchSolver
    from inputs import nesterov_lasso_torch
    rng = np.random.default_rng(3)
    probs = []
    for i in range(152):
        m = int(rng.integers(500, 2001))
        n = int(rng.integers(2000, 6001))
        g = nesterov_lasso_torch(m, n, max(1, int(0.02 * n)), lam=1.0, seed=5000 + i, device="cuda")
        probs.append(dict(At=g["At"], b=g["b"], lam=1.0, m=m))
    bs = BatchSolver(probs, form="gs", max_sweeps=20, check_every=10, tol_stat=1e-6)
    xs = [torch.zeros(p["At"].shape[0], dtype=torch.float32, device="cuda") for p in probs]
    bs.solve(xs)
    for x in xs:
        x.zero_()
    per, tot = bs.solve(xs)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": True, "mode": "batch", "problems": len(probs), "sweeps": tot["sweeps"],
                      "block_w": tot["block_w"], "consumer_warps": tot["kernel_variant"],
                      "A_bytes": sum(p["m"] * p["At"].shape[0] * 4 for p in probs)}))
    bs.close()


def run_ncu_case(args):
    """Small case for ncu captures: the same generator with n = 12800 (A = 1 GB, larger
    than L2), one refresh, then `--ncu-launches` async sweep launches of 10 sweeps each
    (or Jacobi sweeps with --ncu-mode sync; --ncu-mode multi: the multi-lane case; --ncu-mode
    batch: the batched Gauss-Seidel case).  Used by
    the commands in profiles/."""
    import torch
    from paper_1701_04900_gb300.build import build_library
    build_library()
    from paper_1701_04900_gb300 import Solver
    from inputs import nesterov_lasso_torch
    torch.cuda.set_device(0)
    if args.ncu_mode == "multi":
        run_ncu_case_multi()
        return
    if args.ncu_mode == "batch":
        run_ncu_case_batch()
        return
    n = 12800
    gen = nesterov_lasso_torch(M, n, K_PLANT * n // N, lam=LAM, seed=0, device="cuda")
    s = Solver(gen["At"], gen["b"], LAM, m=M, block_w=W_BLOCK, mode=args.ncu_mode, gamma=GAMMA,
               refresh_every=10, tau_rel=4.0 if args.ncu_mode == "sync" else 0.0, variant=args.variant)
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    s.refresh(x)
    for _ in range(args.ncu_launches):
        s.step(x, 10 if args.ncu_mode == "async" else 1)
    torch.cuda.synchronize()
    st = s.check(x)
    print(json.dumps({"ncu_case": True, "n": n, "mode": args.ncu_mode, "F": st["F"], "nnz": st["nnz"]}))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncu-case", action="store_true", help="small profiling case (see run_ncu_case)")
    ap.add_argument("--ncu-mode", default="async", choices=["async", "sync", "multi", "batch"])
    ap.add_argument("--ncu-launches", type=int, default=3)
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1, 2],
                    help="async sweep kernel (asyflexa_opts.variant; 0 = automatic)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refresh-every", type=int, default=10)
    ap.add_argument("--check-every", type=int, default=10)
    ap.add_argument("--max-sweeps", type=int, default=2000)
    ap.add_argument("--sync-sweeps", type=int, default=400)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-sync", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--cpu-speedup", action="store_true",
                    help="run the core-count study on the paper's 20000 x 40000 instance (a few minutes of host "
                         "time) instead of the default 4000 x 8000 one")
    ap.add_argument("--cpu-speedup-only", action="store_true",
                    help="run only the core-count study and print it as one JSON line")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.cpu_speedup_only:
        from paper_1701_04900_gb300.build import build_library
        build_library()
        print(json.dumps({"cpu_core_study": run_cpu_core_study(args)}), flush=True)
    elif args.ncu_case:
        run_ncu_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
