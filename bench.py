"""Benchmark: time-to-1e-12 of the nested FP64/FP32 BiCGStab (Algs. 1-2) on
the 24^3 x 48 clover-Wilson workload on one GB300, beside the plain FP64
BiCGStab, with the clover Dslash (MULT) bandwidth against the HBM roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete qcd_solve (b^_e preparation, the nested iteration,
x_o reconstruction and the FP64 true-residual check) from a device-resident
source; every step must reach ||b - D x|| / ||b|| <= 1e-12.  Under torchrun
(N > 1) every rank solves its own replica (no collective on the data path);
the time is the maximum over ranks.  Prints one JSON line on rank 0.
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
def oracle_sample(dims, U, b, W, reps):
    """Time `reps` oracle D^ applications (one core) on the full lattice."""
    import oracle

    F = oracle.clover_field(dims, U, W["kappa"], W["csw"])
    Fi = oracle.invert_sites(F)
    p = np.ascontiguousarray(b[: inputs.volume(dims) // 2])
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.dhat(dims, W["t_bc"], U, Fi, W["kappa"], p)
        times.append(time.perf_counter() - t0)
    return times


def oracle_iterations():
    p = os.path.join(ROOT, "oracle", "iteration_counts.json")
    if os.path.exists(p):
        return json.load(open(p))["fp64_eo_24x24x24x48"]["fp64_eo_bicgstab_iterations"]
    return None


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_it = oracle_iterations()
    if n_it is None:
        print(json.dumps({"impl": "reference", "unavailable": "oracle/iteration_counts.json missing: the FP64 "
                          "iteration count of the workload has not been recorded"}))
        return 0
    W = WORKLOAD
    dims = W["dims"]
    U = inputs.random_gauge(dims, W["eps"], W["link_seed"])
    b = inputs.gaussian_source(dims, W["src_seed"])
    times = oracle_sample(dims, U, b, W, args.warmup + args.steps)[args.warmup:]
    n_app = 2 * n_it + 2  # two D^ per iteration, plus b^_e and x_o
    per_step = statistics.mean(times) * n_app
    sample = ("one oracle D^ application on the full 24^3x48 lattice per step (%.2f s on 1 core), scaled by "
              "the %d D^ applications of the oracle's own FP64 even-odd BiCGStab to 1e-12 (%d iterations, "
              "oracle/iteration_counts.json)" % (statistics.mean(times), n_app, n_it))
    out = {"impl": "reference", "metric": METRIC, "value": per_step, "unit": "s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD_NAME, "lattice": list(dims), "solver": "oracle FP64 even-odd BiCGStab"},
           "cpu_baseline": {"value": per_step, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": per_step, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------- ours
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
    opts = qcd.default_opts(precision_levels=2, inner_tol=[W["inner_tol"], 1e-2])
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
    # the same K solves again with CUDA events around every launch on the
    # library stream: per-kernel durations for the roofline.  The events and
    # their periodic collection add about 1.5 ms to a 21 ms solve, so they
    # stay out of the timed region above.
    ctx.reset_kernel_stats()
    ctx.set_profiling(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step()
    p1.record(stream)
    torch.cuda.synchronize()
    ctx.set_profiling(False)
    ms_profiled = p0.elapsed_time(p1)
    clocks = sampler.stop()
    stm = ctx.kernel_stats(qcd.K_MULT_F32)
    std = ctx.kernel_stats(qcd.K_DHAT_F32)
    st32 = {k: stm[k] + std[k] for k in ("launches", "ms", "bytes")}
    st64 = ctx.kernel_stats(qcd.K_MULT_F64)
    stdf = ctx.kernel_stats(qcd.K_MULT_DF64)
    stbl = ctx.kernel_stats(qcd.K_BLAS)
    ms_total = max_over_ranks(ms_total, dist, "cuda")
    ms_step = ms_total / args.steps
    mixed = infos[-1]

    # plain FP64 BiCGStab on the same D^ (the comparison of the metric)
    opts64 = qcd.default_opts(precision_levels=1, max_outer=5000)
    ctx.solve(bd, x, tol=W["tol"], opts=opts64)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f64_times = []
    for _ in range(2):
        s0.record(stream)
        info64 = ctx.solve(bd, x, tol=W["tol"], opts=opts64)
        s1.record(stream)
        torch.cuda.synchronize()
        f64_times.append(s0.elapsed_time(s1))
    fp64_ms = min(f64_times)

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

    if rank != 0:
        return 0
    achieved = st32["bytes"] / (st32["ms"] * 1e-3) / 1e9 if st32["ms"] > 0 else None
    roofline = {"bound": "hbm", "achieved": round(achieved, 1) if achieved else None, "peak": hbm,
                "unit": "GB/s", "frac": round(achieved / hbm, 3) if achieved else None,
                "traffic": ncu_traffic(), "kernel": "stencil_kernel<F32> (MULT and the fused D^ second half)",
                "launches": st32["launches"], "avg_launch_us": round(st32["ms"] * 1e3 / max(1, st32["launches"]), 2),
                "algorithmic_bytes_per_launch": round(st32["bytes"] / max(1, st32["launches"])),
                "by_kernel": {name: {"launches": st["launches"],
                                     "avg_launch_us": round(st["ms"] * 1e3 / max(1, st["launches"]), 2),
                                     "frac": round(st["bytes"] / (st["ms"] * 1e-3) / 1e9 / hbm, 3) if st["ms"] else None}
                              for name, st in (("mult", stm), ("dhat_second_half", std))},
                "peak_kind": hbm_kind + " (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)",
                "measured": "CUDA events around every launch on the library stream over %d further solves "
                            "(%.3f ms per solve with the events)" % (args.steps, ms_profiled / args.steps)}
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        reps = 2
        times = oracle_sample(dims, U, b, W, reps)
        n_app = info64["dhat_applies"][0] + 2
        cpu = {"value": statistics.mean(times) * n_app, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": "%d oracle D^ applications on the full 24^3x48 lattice (%.2f s each, 1 core), scaled by "
                         "the %d D^ applications (plus b^_e and x_o) of the FP64 BiCGStab to 1e-12"
                         % (reps, statistics.mean(times), info64["dhat_applies"][0])}
        oi = oracle_iterations()
        if oi is not None:
            cpu["oracle_fp64_iterations"] = oi
    out = {
        "metric": METRIC, "value": round(ms_step * 1e-3, 6), "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "lattice": list(dims), "sites": V, "tol": W["tol"],
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "inputs larger than L2: one FP32 MULT touches 287 MB, one solve several GB"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(statistics.mean(e2e), 6), "unit": "s", "h2d_bytes_per_step": vec_bytes,
                "d2h_bytes_per_step": vec_bytes},
        "gpu_launches": launches,
        "clocks": clocks,
        "mixed": {"outer_iters": mixed["outer_iters"], "inner_iters": mixed["inner_iters"][0],
                  "dhat_applies": mixed["dhat_applies"], "true_resid": mixed["true_resid"],
                  "restarts": mixed["restarts"]},
        "fp64_only": {"seconds": round(fp64_ms * 1e-3, 6), "iterations": info64["outer_iters"],
                      "dhat_applies": info64["dhat_applies"][0], "true_resid": info64["true_resid"]},
        "speedup_vs_fp64": round(fp64_ms / ms_step, 3),
        "dslash": dslash,
        "kernel_time_ms_per_step": {"stencil_f32": round(st32["ms"] / args.steps, 3),
                                    "stencil_df64": round(stdf["ms"] / args.steps, 3),
                                    "stencil_f64": round(st64["ms"] / args.steps, 3),
                                    "blas": round(stbl["ms"] / args.steps, 3)},
        "setup_ms": round(setup_ms, 2),
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
        r = ctx.mult_benchmark(p, nrhs, max(3, args.steps))
        out[name] = {"gbs": round(r["gbs"], 1), "frac_hbm": round(r["gbs"] / hbm, 3), "us": round(r["ms"] * 1e3, 2),
                     "bytes": r["bytes"]}
    print(json.dumps(out))
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
