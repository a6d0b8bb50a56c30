"""Measurements of the workloads beside the headline (bench.py covers the
24^3x48 mixed solve).  One JSON line per workload:

  python bench_suite.py --workload c3    48^3x96: FP64/FP32/FP16 three-level solve
                                          beside the two-level and FP64-only solves,
                                          and the stencil bandwidths at that size
  python bench_suite.py --workload c4a   32^3x64: the 12-RHS Dslash against 12 single
                                          launches, and the 12 point-source solves
                                          as one batch
  python bench_suite.py --workload c4b   48 independent solves on lattices from
                                          {8^4, 12^3x24, 16^3x32, 20^3x40}, tol 1e-10:
                                          one batched persistent-kernel run against
                                          the same problems solved one by one
  python bench_suite.py --workload c5    16^3x32: adjoint gradient (forward and
                                          backward solves plus the force kernels)

Inputs are the seeded synthetic fields of paper_1709_08785_gb300.inputs; every
solve's true residual is computed in FP64 by the library and checked here.
"""
import argparse
import json
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1709_08785_gb300 import inputs  # noqa: E402

TUNE_CACHE = os.path.join(ROOT, "paper_1709_08785_gb300", "_build", "tune_cache.json")


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return float(json.load(open(p))["hbm_gbs"]) if os.path.exists(p) else 6800.0


def timed_solve(torch, ctx, bd, x, tol, reps=2, **kw):
    ctx.solve(bd, x, tol=tol, **kw)  # warm-up
    best, info = None, None
    for _ in range(reps):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        info = ctx.solve(bd, x, tol=tol, **kw)
        s1.record()
        torch.cuda.synchronize()
        t = s0.elapsed_time(s1) * 1e-3
        best = t if best is None else min(best, t)
        assert info["true_resid"] <= tol, info
    return best, info


def w_c3(args):
    import torch

    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, tol = (48, 48, 48, 96), 0.124, 1.6, 1e-12
    t0 = time.time()
    U = inputs.random_gauge_torch(dims, 0.25, 4, device="cuda")
    b = torch.from_numpy(inputs.gaussian_source(dims, 40)).cuda()
    gen_s = time.time() - t0
    ctx = qcd.Context(dims, -1)
    ctx.gauge_load(U)
    ctx.clover_build(kappa, csw)
    del U
    ctx.autotune(TUNE_CACHE)
    x = torch.zeros_like(b)
    out = {"workload": "48^3x96 clover-Wilson, eps 0.25 seed 4, kappa 0.124, csw 1.6, source seed 40, tol 1e-12",
           "sites": inputs.volume(dims), "input_generation_s": round(gen_s, 1)}
    for name, kw in (("three_level", dict(precision_levels=3, inner_tol=[1e-5, 1e-2])),
                     ("two_level", dict(precision_levels=2)),
                     ("fp64_only", dict(precision_levels=1, max_outer=5000))):
        t, info = timed_solve(torch, ctx, b, x, tol, reps=1 if name == "fp64_only" else 2, **kw)
        out[name] = {"seconds": round(t, 4), "outer_iters": info["outer_iters"], "inner_iters": info["inner_iters"],
                     "dhat_applies": info["dhat_applies"], "true_resid": info["true_resid"]}
    hbm = hbm_peak()
    for name, p, nrhs in (("f32", qcd.F32, 1), ("f16", qcd.F16, 1), ("f64", qcd.F64, 1)):
        r = ctx.mult_benchmark(p, nrhs, 10)
        out["dslash_" + name] = {"gbs": round(r["gbs"], 1), "frac_hbm": round(r["gbs"] / hbm, 3),
                                 "us": round(r["ms"] * 1e3, 1)}
    out["speedup_three_level_vs_fp64"] = round(out["fp64_only"]["seconds"] / out["three_level"]["seconds"], 2)
    out["speedup_two_level_vs_fp64"] = round(out["fp64_only"]["seconds"] / out["two_level"]["seconds"], 2)
    return out


def w_c4a(args):
    import torch

    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, tol = (32, 32, 32, 64), 0.1235, 1.6, 1e-12
    U = inputs.random_gauge_torch(dims, 0.25, 5, device="cuda")
    hbm = hbm_peak()
    ctx = qcd.Context(dims, -1)
    ctx.gauge_load(U)
    ctx.clover_build(kappa, csw)
    ctx.autotune(TUNE_CACHE)
    out = {"workload": "32^3x64, eps 0.25 seed 5, kappa 0.1235, csw 1.6: 12 spin-colour point sources at the origin"}
    for name, p in (("f32", qcd.F32), ("f16", qcd.F16)):
        r12 = ctx.mult_benchmark(p, 12, 10)
        r1 = ctx.mult_benchmark(p, 1, 10)
        out["mult_" + name] = {"12rhs_us": round(r12["ms"] * 1e3, 1), "12rhs_gbs": round(r12["gbs"], 1),
                               "12rhs_frac_hbm": round(r12["gbs"] / hbm, 3),
                               "12_single_us": round(12 * r1["ms"] * 1e3, 1),
                               "speedup_vs_12_single": round(12 * r1["ms"] / r12["ms"], 2),
                               "bytes_per_site_per_rhs": round(r12["bytes"] / (inputs.volume(dims) // 2) / 12, 1)}
    # the 12 point-source solves, one after another on this context (a
    # batch would need one context, i.e. one copy of the fields, per source)
    del U
    P = inputs.point_sources(dims)
    seq, res, outer = 0.0, [], []
    for k in range(12):
        bk = torch.from_numpy(np.ascontiguousarray(P[k])).cuda()
        xk = torch.zeros_like(bk)
        t1, info = timed_solve(torch, ctx, bk, xk, tol, reps=1, precision_levels=2)
        seq += t1
        res.append(info["true_resid"])
        outer.append(info["outer_iters"])
    out["solves"] = {"sequential_s": round(seq, 4), "max_true_resid": max(res), "outer_iters": outer}
    return out


def w_c4b(args):
    import torch

    from paper_1709_08785_gb300 import qcd

    probs = inputs.batch_problems(48, 99)
    tol = 1e-10
    ctxs, bs, xs = [], [], []
    t0 = time.time()
    for p in probs:
        U = inputs.random_gauge_torch(p["dims"], p["eps"], p["link_seed"], device="cuda")
        c = qcd.Context(p["dims"], -1)
        c.gauge_load(U)
        c.clover_build(p["kappa"], p["csw"])
        c.autotune(TUNE_CACHE)
        ctxs.append(c)
        b = torch.from_numpy(inputs.gaussian_source(p["dims"], p["src_seed"])).cuda()
        bs.append(b)
        xs.append(torch.zeros_like(b))
    setup_s = time.time() - t0
    qcd.solve_batched(ctxs, bs, xs, [tol] * 48, precision_levels=2)  # warm-up
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        infos = qcd.solve_batched(ctxs, bs, xs, [tol] * 48, precision_levels=2)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    assert all(i["true_resid"] <= tol for i in infos)
    seq_mixed = seq_fp64 = 0.0
    for c, b, x in zip(ctxs, bs, xs):
        t1, _ = timed_solve(torch, c, b, x, tol, reps=1, precision_levels=2)
        t2, _ = timed_solve(torch, c, b, x, tol, reps=1, precision_levels=1, max_outer=5000)
        seq_mixed += t1
        seq_fp64 += t2
    sizes = {}
    for p in probs:
        sizes["x".join(map(str, p["dims"]))] = sizes.get("x".join(map(str, p["dims"])), 0) + 1
    return {"workload": "48 independent FP64/FP32 solves, lattices from {8^4,12^3x24,16^3x32,20^3x40}, "
                        "eps U[0.15,0.35], kappa U[0.115,0.124], csw 1.0, tol 1e-10 (seeds 99, 100+i, 200+i)",
            "lattice_counts": sizes, "setup_s": round(setup_s, 1),
            "batched_s": round(min(times), 4), "sequential_mixed_s": round(seq_mixed, 4),
            "sequential_fp64_s": round(seq_fp64, 4),
            "speedup_vs_sequential_mixed": round(seq_mixed / min(times), 2),
            "speedup_vs_sequential_fp64": round(seq_fp64 / min(times), 2),
            "max_true_resid": max(i["true_resid"] for i in infos),
            "outer_iters": sorted({i["outer_iters"] for i in infos}), "restarts": sum(i["restarts"] for i in infos)}


def w_c5(args):
    import torch

    from paper_1709_08785_gb300 import qcd
    from paper_1709_08785_gb300.autograd import clover_solve

    dims, kappa, csw = (16, 16, 16, 32), 0.12, 1.0
    U = torch.from_numpy(inputs.random_gauge(dims, 0.3, 6)).cuda().requires_grad_(True)
    b = torch.from_numpy(inputs.gaussian_source(dims, 61)).cuda().requires_grad_(True)
    eta = torch.from_numpy(inputs.gaussian_source(dims, 60)).cuda()
    ctx = qcd.Context(dims, -1)
    ts = []
    for _ in range(4):
        U.grad = None
        b.grad = None
        torch.cuda.synchronize()
        t = time.perf_counter()
        x = clover_solve(U, b, ctx, kappa, csw, tol=1e-12, levels=2)
        L = torch.sum(torch.conj(eta) * x).real
        L.backward()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t)
    return {"workload": "adjoint gradient of Re<eta, D^-1 b> on 16^3x32 (eps 0.3 seed 6, kappa 0.12, csw 1.0)",
            "forward_backward_s": round(min(ts[1:]), 4), "grad_U_norm": float(U.grad.norm()),
            "grad_b_norm": float(b.grad.norm())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True, choices=["c3", "c4a", "c4b", "c5"])
    args = ap.parse_args()
    fn = {"c3": w_c3, "c4a": w_c4a, "c4b": w_c4b, "c5": w_c5}[args.workload]
    print(json.dumps(fn(args)))


if __name__ == "__main__":
    main()
