"""Benchmark: time-to-1e-12 of the nested FP64/FP32 BiCGStab (Algs. 1-2) on
the 24^3 x 48 clover-Wilson workload on one GB300, beside the plain FP64
BiCGStab, with the clover Dslash (MULT) bandwidth against the HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete qcd_solve (b^_e preparation, the nested iteration,
x_o reconstruction and the FP64 true-residual check) from a device-resident
source; every step must reach ||b - D x|| / ||b|| <= 1e-12.  The solve runs
the library's default outer level: the solution x_e, the source b^_e and the
reconstruction x_o in FP64 arithmetic, the outer D^ applications and
recursion vectors in DF64, the inner iteration in FP32; the all-FP64 and
all-DF64 outer levels are timed beside it.  Under torchrun (N > 1) every rank
solves its own replica (no collective on the data path); the time is the
maximum over ranks.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1709_08785_gb300 import inputs  # noqa: E402

METRIC = "time-to-1e-12 mixed vs FP64 BiCGStab on 1 GB300; clover Dslash GB/s, % HBM"
WORKLOAD = dict(dims=(24, 24, 24, 48), eps=0.25, link_seed=3, kappa=0.124, csw=1.6, t_bc=-1, src_seed=30,
                tol=1e-12, inner_tol=1e-5)
WORKLOAD_NAME = ("24^3x48 clover-Wilson, even-odd preconditioned nested BiCGStab, FP64 outer / FP32 inner "
                 "(inner tol 1e-5), links exp(i 0.25 H) seed 3, kappa 0.124, csw 1.6, antiperiodic t, "
                 "Gaussian source seed 30, tol 1e-12")
DTYPE = ("f64 (solution x_e, source b^_e, reconstruction x_o, outer dots and norms, true residual) + "
         "df64 (outer D^ and recursion vectors) + f32 (inner iteration)")
# algorithmic bytes per output site of the FP32 stencil kernels of one D^:
# MULT (in 96 + links 8x48 + clover 288 + out 96) and the fused second half
STENCIL_SOURCES = ["paper_1709_08785_gb300/csrc/stencil_impl.cuh", "paper_1709_08785_gb300/csrc/stencil.cuh",
                   "paper_1709_08785_gb300/csrc/stencil_f32.cu", "paper_1709_08785_gb300/csrc/qcd_internal.cuh",
                   "paper_1709_08785_gb300/csrc/reduce.cuh"]
TUNE_CACHE = os.path.join(ROOT, "paper_1709_08785_gb300", "_build", "tune_cache.json")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stencil_hash():
    h = hashlib.sha256()
    for f in STENCIL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """Per-launch DRAM bytes of the FP32 stencil from the committed ncu
    summary, or None when it is absent or the kernel changed since."""
    p = os.path.join(ROOT, "profiles", "stencil_f32_24x24x24x48.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha") != stencil_hash():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for row in csv.reader(open(self.path)):
            if len(row) >= 9:
                rows.append([c.strip() for c in row])
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, dist, device) -> float:
    """The maximum of a per-rank time over all ranks (the replicas' timed
    region ends when the slowest rank ends); the value itself with one rank."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- oracle
def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.processor() or platform.machine()


def oracle_dhat_times(dims, U, b, W, reps, openmp):
    """Wall times of `reps` oracle D^ applications on the full lattice, with
    the single-threaded build or the OpenMP build on every host core (the
    clover term and its inverse are built first, outside the timing)."""
    import oracle

    threads = oracle.use_openmp(True)  # the set-up on all cores
    F = oracle.clover_field(dims, U, W["kappa"], W["csw"])
    Fi = oracle.invert_sites(F)
    del F
    if not openmp:
        threads = oracle.use_openmp(False)
    p = np.ascontiguousarray(b[: inputs.volume(dims) // 2])
    times = []
    try:
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.dhat(dims, W["t_bc"], U, Fi, W["kappa"], p)
            times.append(time.perf_counter() - t0)
    finally:
        oracle.use_openmp(False)
    return times, threads


def oracle_dirac_times(dims, U, b, W, reps, openmp):
    """Wall times of `reps` oracle D applications (Eq. 3, the full lattice)
    with the single-threaded build or the OpenMP build on every host core."""
    import oracle

    threads = oracle.use_openmp(True)
    F = oracle.clover_field(dims, U, W["kappa"], W["csw"])
    if not openmp:
        threads = oracle.use_openmp(False)
    times = []
    try:
        for _ in range(reps):
            t0 = time.perf_counter()
            oracle.dirac(dims, W["t_bc"], U, F, W["kappa"], b)
            times.append(time.perf_counter() - t0)
    finally:
        oracle.use_openmp(False)
    return times, threads


def oracle_c1_solve():
    """The oracle's plain FP64 BiCGStab on the 4^4 workload (links exp(i 0.3 H)
    seed 1, kappa 0.12, csw 1.0, source seed 2, tol 1e-12), single-threaded:
    wall time of the whole solve and its true residual."""
    import oracle

    dims, kappa, csw, t_bc = (4, 4, 4, 4), 0.12, 1.0, -1
    U = inputs.random_gauge(dims, 0.3, 1)
    b = inputs.gaussian_source(dims, 2)
    t0 = time.perf_counter()
    F = oracle.clover_field(dims, U, kappa, csw)
    x, st, it = oracle.bicgstab_full(dims, t_bc, U, F, kappa, b, 1e-12)
    secs = time.perf_counter() - t0
    return {"seconds": round(secs, 4), "iterations": it, "status": st,
            "true_resid": oracle.true_residual(dims, t_bc, U, F, kappa, b, x)}


def oracle_iterations():
    p = os.path.join(ROOT, "oracle", "iteration_counts.json")
    if os.path.exists(p):
        d = json.load(open(p))
        hosts = {h: e["fp64_eo_bicgstab_iterations"] for h, e in d.get("by_host", {}).items()}
        return d["fp64_eo_24x24x24x48"]["fp64_eo_bicgstab_iterations"], hosts
    return None, {}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_it, hosts = oracle_iterations()
    if n_it is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle/iteration_counts.json missing: the FP64 "
                          "iteration count of the workload has not been recorded"}))
        return 0
    W = WORKLOAD
    dims = W["dims"]
    U = inputs.random_gauge(dims, W["eps"], W["link_seed"])
    b = inputs.gaussian_source(dims, W["src_seed"])
    times, threads = oracle_dhat_times(dims, U, b, W, args.warmup + args.steps, openmp=True)
    times = times[args.warmup:]
    n_app = 2 * n_it + 2  # two D^ per iteration, plus b^_e and x_o
    per_dhat = statistics.mean(times)
    per_solve = per_dhat * n_app
    sample = ("one oracle D^ application on the full 24^3x48 lattice per step (%.3f s, OpenMP build on %d threads "
              "of %d host cores), extrapolated to a solve by the %d D^ applications of the oracle's own FP64 "
              "even-odd BiCGStab to 1e-12 (%d iterations, oracle/iteration_counts.json)"
              % (per_dhat, threads, os.cpu_count() or 0, n_app, n_it))
    out = {"impl": "reference", "metric": METRIC, "value": per_solve, "unit": "s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per_dhat * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "lattice": list(dims), "solver": "oracle FP64 even-odd BiCGStab"},
           "extrapolated": {"measured_per_step_s": per_dhat, "dhat_applications_per_solve": n_app,
                            "note": "value = measured D^ time x the D^ count of a full solve; ms_per_step is the "
                                    "time of the step actually run (one D^)"},
           "cpu_baseline": {"value": per_solve, "unit": "s", "cores": threads, "kind": "oracle", "sample": sample,
                            "host": {"nproc": os.cpu_count(), "cpu_model": cpu_model()},
                            "iterations_by_host": hosts},
           "e2e": {"value": per_solve, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def cpu_baseline_block(dims, U, b, W, n_app):
    """The oracle timed on this host: one D^ single-threaded and on all cores
    (OpenMP build), each extrapolated to the FP64 solve's n_app D^
    applications, and the whole 4^4 plain-BiCGStab solve."""
    t1, _ = oracle_dhat_times(dims, U, b, W, 2, openmp=False)
    tn, threads = oracle_dhat_times(dims, U, b, W, 3, openmp=True)
    d1, dn = min(t1), min(tn)
    D1, _ = oracle_dirac_times(dims, U, b, W, 1, openmp=False)
    Dn, _ = oracle_dirac_times(dims, U, b, W, 3, openmp=True)
    n_it, hosts = oracle_iterations()
    return {"value": round(dn * n_app, 3), "unit": "s", "cores": threads, "kind": "oracle",
            "sample": "oracle D^ on the full 24^3x48 lattice, OpenMP build on %d threads (best of 3: %.3f s), "
                      "extrapolated by the %d D^ applications (plus b^_e and x_o) of the FP64 BiCGStab to 1e-12"
                      % (threads, dn, n_app - 2),
            "single_core": {"dhat_s": round(d1, 3), "dirac_s": round(min(D1), 3),
                            "solve_s_extrapolated": round(d1 * n_app, 2)},
            "all_cores": {"threads": threads, "dhat_s": round(dn, 4), "dirac_s": round(min(Dn), 4),
                          "solve_s_extrapolated": round(dn * n_app, 3)},
            "c1_4x4x4x4_full_solve_single_core": oracle_c1_solve(),
            "host": {"nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "oracle_fp64_iterations": n_it, "iterations_by_host": hosts}


# --------------------------------------------------------------------- ours
def timed_solves(torch, ctx, bd, x, tol, opts, reps):
    """Best device time (s) of `reps` solves after one untimed one, and the
    last solve's info."""
    stream = torch.cuda.current_stream()
    ctx.solve(bd, x, tol=tol, opts=opts)
    best, info = None, None
    for _ in range(reps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        info = ctx.solve(bd, x, tol=tol, opts=opts)
        s1.record(stream)
        torch.cuda.synchronize()
        t = s0.elapsed_time(s1) * 1e-3
        best = t if best is None else min(best, t)
        if info["true_resid"] > tol:
            raise RuntimeError("solve missed the tolerance: %r" % info)
    return best, info


def solve_summary(t, info):
    return {"seconds": round(t, 6), "outer_iters": info["outer_iters"], "inner_iters": info["inner_iters"],
            "dhat_applies": info["dhat_applies"], "true_resid": info["true_resid"], "restarts": info["restarts"]}


# Algorithmic bytes per even site of one FP32 inner iteration (Alg. 2) as
# the kernels run it: two D^ (MULT 864 each; second halves 864 + y 96 + r~ 96
# for alpha and 864 + y 96 for omega), s = r - alpha q (3 x 96), the x, r
# update with its dots (7 x 96), and p (4 x 96)
INNER_ITER_BYTES = 864 + 1056 + 288 + 864 + 960 + 672 + 384  # 5088


def extra_workloads(torch, qcd, hbm):
    """The other workloads on this GPU: the 48^3x96 three-level solve, the
    48-problem batch (with its bytes-based roofline), the 16^3x32 adjoint."""
    out = {}
    # ---- 48^3x96, three levels FP64/FP32/FP16 (links generated on the GPU)
    dims = (48, 48, 48, 96)
    U = inputs.random_gauge_torch(dims, 0.25, 4, device="cuda")
    b = torch.from_numpy(inputs.gaussian_source(dims, 40)).cuda()
    c = qcd.Context(dims, -1)
    c.gauge_load(U)
    c.clover_build(0.124, 1.6)
    del U
    c.autotune(TUNE_CACHE)
    x = torch.zeros_like(b)
    # inner tolerances tuned at this size: FP32 middle level 1e-3, FP16 level 3e-2
    t, info = timed_solves(torch, c, b, x, 1e-12, qcd.default_opts(precision_levels=3, inner_tol=[1e-3, 3e-2]), 2)
    out["three_level_48x48x48x96"] = solve_summary(t, info)
    out["three_level_48x48x48x96"]["inner_tol"] = [1e-3, 3e-2]
    r = c.mult_benchmark(qcd.F16, 1, 10)
    out["three_level_48x48x48x96"]["dslash_f16_frac_hbm"] = round(r["gbs"] / hbm, 3)
    c.close()
    del b, x
    torch.cuda.empty_cache()
    # ---- 48 independent problems in one batched run
    probs = inputs.batch_problems(48, 99)
    ctxs, bs, xs = [], [], []
    for p in probs:
        U = inputs.random_gauge_torch(p["dims"], p["eps"], p["link_seed"], device="cuda")
        c = qcd.Context(p["dims"], -1)
        c.gauge_load(U)
        c.clover_build(p["kappa"], p["csw"])
        ctxs.append(c)
        bs.append(torch.from_numpy(inputs.gaussian_source(p["dims"], p["src_seed"])).cuda())
        xs.append(torch.zeros_like(bs[-1]))
    del U
    tol = [1e-10] * len(probs)
    qcd.solve_batched(ctxs, bs, xs, tol, precision_levels=2)
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        infos = qcd.solve_batched(ctxs, bs, xs, tol, precision_levels=2)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
    tb = min(times)
    # algorithmic bytes: the inner FP32 iterations and the outer D^ (two
    # DF64 MULT-class passes of 2112 B per output site plus the epilogue's
    # v, r~ or r: 2 x 2112 + 2 x 192) of every problem
    by = sum(i["inner_iters"][0] * INNER_ITER_BYTES * inputs.volume(p["dims"]) // 2 +
             i["dhat_applies"][0] * (2 * 2112 + 2 * 192) * inputs.volume(p["dims"]) // 2 for p, i in zip(probs, infos))
    out["batched_48"] = {"seconds": round(tb, 4), "max_true_resid": max(i["true_resid"] for i in infos),
                         "restarts": sum(i["restarts"] for i in infos),
                         "inner_iters": sum(i["inner_iters"][0] for i in infos),
                         "roofline": {"algorithmic_bytes": by, "achieved_gbs": round(by / tb / 1e9, 1),
                                      "frac": round(by / tb / 1e9 / hbm, 3),
                                      "counted": "inner FP32 iterations (5088 B per even site) and outer DF64 D^ "
                                                 "(4608 B per even site) of every problem, over the whole batch "
                                                 "time (set-up of b^ and the x_o / true-residual finish included)"}}
    for c in ctxs:
        c.close()
    del ctxs, bs, xs
    torch.cuda.empty_cache()
    # ---- 32^3x64, the 12 spin-colour point sources: one after another and
    # in lockstep (qcd_solve_multi, the FP32 iterations through the 12-RHS MULT)
    dims = (32, 32, 32, 64)
    U = inputs.random_gauge_torch(dims, 0.25, 5, device="cuda")
    c = qcd.Context(dims, -1)
    c.gauge_load(U)
    c.clover_build(0.1235, 1.6)
    del U
    c.autotune(TUNE_CACHE)
    B = torch.from_numpy(inputs.point_sources(dims)).cuda()
    X1, Xm = torch.zeros_like(B), torch.zeros_like(B)
    o2 = qcd.default_opts(precision_levels=2)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3, r

    c.solve(B[0], X1[0], tol=1e-12, opts=o2)  # warm-up
    ts, seq_infos = timed(lambda: [c.solve(B[k], X1[k], tol=1e-12, opts=o2) for k in range(12)])
    c.solve_multi(B, Xm, tol=1e-12, opts=o2)  # warm-up
    runs = [timed(lambda: c.solve_multi(B, Xm, tol=1e-12, opts=o2)) for _ in range(2)]
    tm, infos = min(r[0] for r in runs), runs[-1][1]
    out["point_sources_32x32x32x64"] = {
        "sequential_s": round(ts, 4), "lockstep_s": round(tm, 4), "lockstep_speedup": round(ts / tm, 3),
        "max_true_resid": max(i["true_resid"] for i in infos + seq_infos),
        "lockstep_equals_sequential": bool(torch.equal(Xm, X1)),
        "what": "12 point-source solves to 1e-12 (kappa 0.1235, csw 1.6, links exp(i 0.25 H) seed 5): qcd_solve "
                "one after another against qcd_solve_multi, whose FP32 iterations apply D^ to all 12 at once"}
    c.close()
    del B, X1, Xm
    torch.cuda.empty_cache()
    # ---- the paper's fixed-work protocol (Sec. IV, Tables I-II): 2000 D^ as
    # 4 x (500 inner FP32 D^ + 1 outer D^) at 24^3x48, the SOLVE rate by Table I
    import argparse

    import bench_suite

    fw = bench_suite.w_fixed_work(argparse.Namespace(lattice=24, kappa=0.155, dhat=2000))
    out["fixed_work_2000_dhat_24x24x24x48"] = {k: fw[k] for k in ("seconds", "inner_iterations", "dhat_applies",
                                                                  "ms_per_inner_dhat", "solve_tflops_table1")}
    out["fixed_work_2000_dhat_24x24x24x48"]["what"] = fw["workload"]
    torch.cuda.empty_cache()
    # ---- the 4^4 workload: plain FP64 BiCGStab on the full D, no preconditioning
    dims = (4, 4, 4, 4)
    U = torch.from_numpy(inputs.random_gauge(dims, 0.3, 1)).cuda()
    b = torch.from_numpy(inputs.gaussian_source(dims, 2)).cuda()
    c = qcd.Context(dims, -1)
    c.gauge_load(U)
    c.clover_build(0.12, 1.0)
    x = torch.zeros_like(b)
    t, info = timed_solves(torch, c, b, x, 1e-12, qcd.default_opts(precision_levels=1, even_odd=0, max_outer=5000), 3)
    out["unpreconditioned_fp64_4x4x4x4"] = {"seconds": round(t, 6), "iterations": info["outer_iters"],
                                            "true_resid": info["true_resid"],
                                            "what": "plain FP64 BiCGStab on D (no even-odd), links exp(i 0.3 H) seed 1, "
                                                    "kappa 0.12, csw 1.0, source seed 2, tol 1e-12"}
    c.close()
    del U, b, x
    # ---- adjoint gradient on 16^3x32
    from paper_1709_08785_gb300.autograd import clover_solve

    dims = (16, 16, 16, 32)
    U = torch.from_numpy(inputs.random_gauge(dims, 0.3, 6)).cuda().requires_grad_(True)
    b = torch.from_numpy(inputs.gaussian_source(dims, 61)).cuda().requires_grad_(True)
    eta = torch.from_numpy(inputs.gaussian_source(dims, 60)).cuda()
    c = qcd.Context(dims, -1)
    ts = []
    for _ in range(4):
        U.grad = None
        b.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xx = clover_solve(U, b, c, 0.12, 1.0, tol=1e-12, levels=2)
        L = torch.sum(torch.conj(eta) * xx).real
        L.backward()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    out["adjoint_16x16x16x32"] = {"forward_backward_s": round(min(ts[1:]), 4),
                                  "what": "gradient of Re<eta, D^-1 b> with respect to the links and b: forward "
                                          "and adjoint solves to 1e-12 plus the force kernels"}
    c.close()
    return out


def run_ours(args):
    import torch

    from paper_1709_08785_gb300 import qcd

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    W = WORKLOAD
    dims = W["dims"]
    V = inputs.volume(dims)
    U = inputs.random_gauge(dims, W["eps"], W["link_seed"])
    b = inputs.gaussian_source(dims, W["src_seed"])
    stream = torch.cuda.current_stream()
    ctx = qcd.Context(dims, W["t_bc"], stream)
    Ud = torch.from_numpy(U).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.gauge_load(Ud)
    ctx.clover_build(W["kappa"], W["csw"])
    e1.record(stream)
    torch.cuda.synchronize()
    setup_ms = e0.elapsed_time(e1)
    del Ud
    ctx.autotune(TUNE_CACHE)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    # the library's default outer level (outer_df64 = 1): FP64 solution
    opts = qcd.default_opts(precision_levels=2, inner_tol=[W["inner_tol"], 1e-2])
    assert opts.outer_df64 == 1
    infos = []

    def step():
        info = ctx.solve(bd, x, tol=W["tol"], opts=opts)
        if info["true_resid"] > W["tol"]:
            raise RuntimeError("solve missed the tolerance: %r" % info)
        infos.append(info)

    for _ in range(args.warmup):
        step()
    infos.clear()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    vis_list = vis if vis != [""] else []
    gpu_index = int(vis_list[local]) if local < len(vis_list) and vis_list[local].isdigit() else local
    sampler = ClockSampler(gpu_index)
    n0 = ctx.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    ms_total = t0.elapsed_time(t1)
    launches = ctx.launch_count() - n0
    mixed = infos[-1]
    # the same K solves again with CUDA events around every launch on the
    # library stream: per-kernel durations for the roofline.  The events and
    # their periodic collection add about 1.5 ms to a 20 ms solve, so they
    # stay out of the timed region above.
    ctx.reset_kernel_stats()
    ctx.set_profiling(True)
    infos.clear()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    ms_profiled = p0.elapsed_time(p1)
    inner_iters_profiled = sum(i["inner_iters"][0] for i in infos)
    stm = ctx.kernel_stats(qcd.K_MULT_F32)
    std = ctx.kernel_stats(qcd.K_DHAT_F32)
    st32 = {k: stm[k] + std[k] for k in ("launches", "ms", "bytes")}
    st64 = ctx.kernel_stats(qcd.K_MULT_F64)
    stdf = ctx.kernel_stats(qcd.K_MULT_DF64)
    stbl = ctx.kernel_stats(qcd.K_BLAS)
    stb32 = ctx.kernel_stats(qcd.K_BLAS_F32)
    # and K more with chunk timing: whole FP32 iterations, launched back to
    # back as in the timed solves, one event pair per queued chunk
    ctx.reset_kernel_stats()
    ctx.set_profiling(2)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    ctx.set_profiling(0)
    stit = ctx.kernel_stats(qcd.K_INNER_ITER)
    clocks = sampler.stop()
    ms_total = max_over_ranks(ms_total, dist, "cuda")
    ms_step = ms_total / args.steps

    # the other arithmetics of the outer level, beside the default
    outer_modes = {}
    for mode, name in ((0, "fp64_outer"), (2, "df64_outer")):
        o = qcd.default_opts(precision_levels=2, inner_tol=[W["inner_tol"], 1e-2], outer_df64=mode)
        t, info = timed_solves(torch, ctx, bd, x, W["tol"], o, 3)
        outer_modes[name] = solve_summary(t, info)
    o = qcd.default_opts(precision_levels=2, inner_tol=[W["inner_tol"], 1e-2], eo_hermitian=1)
    t, info = timed_solves(torch, ctx, bd, x, W["tol"], o, 3)
    eo_forms = {"dhat_eq8": dict(solve_summary(ms_step * 1e-3, mixed), what="D^_ee = 1 - k^2 F_ee^-1 H_eo F_oo^-1 H_oe "
                                 "(Eq. 8), the headline solve"),
                "schur_ee": dict(solve_summary(t, info), what="gamma5-hermitian S_ee = F_ee D^_ee on every level, "
                                 "same outer/inner precisions")}
    outer_modes["fp64_outer"]["what"] = "outer level all FP64 (Alg. 1 as printed), FP32 inner"
    outer_modes["df64_outer"]["what"] = ("outer level all DF64, x_e, b^_e and x_o included (FP64 dots, norms and "
                                         "true residual), FP32 inner")

    # plain FP64 BiCGStab on the same D^ (the comparison of the metric)
    opts64 = qcd.default_opts(precision_levels=1, max_outer=5000)
    fp64_s, info64 = timed_solves(torch, ctx, bd, x, W["tol"], opts64, 2)

    # the clover Dslash alone (L2 evicted before each launch)
    hbm, hbm_kind = peaks()
    dslash = {}
    for name, p, nrhs in (("f32", qcd.F32, 1), ("f16", qcd.F16, 1), ("df64", qcd.DF64, 1), ("f64", qcd.F64, 1),
                          ("f32_12rhs", qcd.F32, 12)):
        r = ctx.mult_benchmark(p, nrhs, 20 if nrhs == 1 else 10)
        q = ctx.mult_throughput(p, nrhs, 50 if p in (qcd.F32, qcd.F16) else 10)
        dslash[name] = {"gbs": round(r["gbs"], 1), "frac_hbm": round(r["gbs"] / hbm, 3), "us": round(r["ms"] * 1e3, 2),
                        "bytes": r["bytes"], "back_to_back_us": round(q["ms"] * 1e3, 2),
                        "back_to_back_frac_hbm": round(q["gbs"] / hbm, 3)}
    dslash["method"] = ("us/gbs: each launch alone, L2 evicted by reading 256 MB before it; back_to_back: "
                        "launches in a stream, launch gaps included, the input vector warm in L2")

    # end to end through the public API from pinned host buffers
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    ctx.solve(bh, xh, tol=W["tol"], opts=opts)
    e2e = []
    for _ in range(args.steps):
        t = time.perf_counter()
        info = ctx.solve(bh, xh, tol=W["tol"], opts=opts)
        e2e.append(time.perf_counter() - t)
        if info["true_resid"] > W["tol"]:
            raise RuntimeError("host-buffer solve missed the tolerance")
    vec_bytes = V * 12 * 16

    extras = None
    if not args.no_extras and ws == 1:
        ctx_keep = ctx
        extras = extra_workloads(torch, qcd, hbm)
        ctx = ctx_keep

    if rank != 0:
        return 0

    def frac_of(st):
        return round(st["bytes"] / (st["ms"] * 1e-3) / 1e9 / hbm, 3) if st["ms"] else None

    achieved = st32["bytes"] / (st32["ms"] * 1e-3) / 1e9 if st32["ms"] > 0 else None
    it_ms = st32["ms"] + stb32["ms"]
    it_bytes = st32["bytes"] + stb32["bytes"]
    Vh = V // 2
    it_gbs = stit["bytes"] / (stit["ms"] * 1e-3) / 1e9 if stit["ms"] > 0 else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1) if achieved else None, "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 3) if achieved else None,
                "traffic": ncu_traffic(), "kernel": "stencil_kernel<F32> (MULT and the fused D^ second half)",
                "launches": st32["launches"], "avg_launch_us": round(st32["ms"] * 1e3 / max(1, st32["launches"]), 2),
                "algorithmic_bytes_per_launch": round(st32["bytes"] / max(1, st32["launches"])),
                "by_kernel": {name: {"launches": st["launches"],
                                     "avg_launch_us": round(st["ms"] * 1e3 / max(1, st["launches"]), 2),
                                     "frac": frac_of(st)}
                              for name, st in (("mult", stm), ("dhat_second_half", std), ("blas_f32_level", stb32))},
                "inner_iteration": {
                    "iterations": stit["launches"],
                    "us_per_iteration": round(stit["ms"] * 1e3 / max(1, stit["launches"]), 2),
                    "algorithmic_bytes_per_even_site": round(stit["bytes"] / max(1, stit["launches"]) / Vh, 1),
                    "nominal_bytes_per_even_site": INNER_ITER_BYTES,
                    "achieved_gbs": round(it_gbs, 1) if it_gbs else None,
                    "frac": round(it_gbs / hbm, 3) if it_gbs else None,
                    "what": "whole FP32 BiCGStab iterations (two D^ with their fused dots, three fused BLAS-1 "
                            "updates): one CUDA event pair around each chunk of iterations the solver queues, "
                            "the launches inside back to back as in the timed solves (%d further solves)"
                            % args.steps,
                    "per_launch_events": {
                        "us_per_iteration": round(it_ms * 1e3 / max(1, inner_iters_profiled), 2),
                        "frac": round(it_bytes / (it_ms * 1e-3) / 1e9 / hbm, 3) if it_ms else None,
                        "what": "the same from events around every launch: each bracketed launch waits for its "
                                "predecessor and shows its own launch latency"}},
                "peak_kind": hbm_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)",
                "measured": "CUDA events around every launch on the library stream over %d further solves "
                            "(%.3f ms per solve with the events)" % (args.steps, ms_profiled / args.steps)}
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_block(dims, U, b, W, info64["dhat_applies"][0] + 2)
    out = {
        "metric": METRIC, "value": round(ms_step * 1e-3, 6), "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "lattice": list(dims), "sites": V, "tol": W["tol"],
                   "outer_level": "outer_df64 = 1: FP64 solution accumulation, DF64 outer D^",
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2: one FP32 MULT touches 287 MB, one solve several GB"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        # the median over the K host-timed steps (a host-side hiccup in one
        # step does not move it), the mean and the slowest step beside it
        "e2e": {"value": round(statistics.median(e2e), 6), "unit": "s", "h2d_bytes_per_step": vec_bytes,
                "d2h_bytes_per_step": vec_bytes, "statistic": "median of %d steps" % len(e2e),
                "mean": round(statistics.mean(e2e), 6), "max": round(max(e2e), 6)},
        "gpu_launches": launches,
        "clocks": clocks,
        "mixed": {"outer_iters": mixed["outer_iters"], "inner_iters": mixed["inner_iters"][0],
                  "dhat_applies": mixed["dhat_applies"], "true_resid": mixed["true_resid"],
                  "restarts": mixed["restarts"]},
        "outer_modes": outer_modes,
        "eo_operator": eo_forms,
        "fp64_only": {"seconds": round(fp64_s, 6), "iterations": info64["outer_iters"],
                      "dhat_applies": info64["dhat_applies"][0], "true_resid": info64["true_resid"]},
        "speedup_vs_fp64": round(fp64_s / (ms_step * 1e-3), 3),
        "dslash": dslash,
        "kernel_time_ms_per_step": {"stencil_f32": round(st32["ms"] / args.steps, 3),
                                    "blas_f32": round(stb32["ms"] / args.steps, 3),
                                    "stencil_df64": round(stdf["ms"] / args.steps, 3),
                                    "stencil_f64": round(st64["ms"] / args.steps, 3),
                                    "blas_other": round(stbl["ms"] / args.steps, 3)},
        "setup_ms": round(setup_ms, 2),
        "workloads": extras,
    }
    print(json.dumps(out))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (48^3x96 three-level, 48-problem batch, 16^3x32 adjoint)")
    ap.add_argument("--only-dslash", action="store_true",
                    help="time only the MULT kernel (L2 evicted between launches) on the workload's fields")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.only_dslash:
        return run_dslash_only(args)
    return run_ours(args)


def run_dslash_only(args):
    """The clover Dslash alone on the workload's fields: one JSON line with
    the per-launch time and bandwidth of each precision."""
    import torch

    from paper_1709_08785_gb300 import qcd

    W = WORKLOAD
    dims = W["dims"]
    U = inputs.random_gauge(dims, W["eps"], W["link_seed"])
    ctx = qcd.Context(dims, W["t_bc"], torch.cuda.current_stream())
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(W["kappa"], W["csw"])
    ctx.autotune(TUNE_CACHE)
    hbm, kind = peaks()
    out = {"mode": "dslash-only", "lattice": list(dims), "peak_gbs": hbm, "peak_kind": kind}
    for name, p, nrhs in (("f32", qcd.F32, 1), ("f16", qcd.F16, 1), ("f64", qcd.F64, 1), ("df64", qcd.DF64, 1),
                          ("f32_12rhs", qcd.F32, 12)):
        # one NVTX range per precision, so that a profiler can select it
        torch.cuda.nvtx.range_push("dslash_" + name)
        r = ctx.mult_benchmark(p, nrhs, max(3, args.steps))
        torch.cuda.nvtx.range_pop()
        out[name] = {"gbs": round(r["gbs"], 1), "frac_hbm": round(r["gbs"] / hbm, 3), "us": round(r["ms"] * 1e3, 2),
                     "bytes": r["bytes"]}
    out["tuned"] = [t for t in ctx.tune_info() if t["mode"] in (1, 2, 4) and t["nrhs"] in (1, 12)]
    print(json.dumps(out))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
