"""Run the oracle's FP64 even-odd BiCGStab to a true residual of 1e-12 on
the 24^3 x 48 workload and record how many iterations it took.

TEST INFRASTRUCTURE: the CPU reference arm of the benchmark scales its
bounded per-application timing by this count (it never runs the CUDA path).
Calls only the oracle and the seeded input generators.  Writes
oracle/iteration_counts.json.  Takes a few minutes on one core (--openmp: the site loops on all cores).

Workload: links reunitarised exp(i 0.25 H) seed 3, kappa 0.124, csw 1.6,
antiperiodic in time, Gaussian source seed 30.  The even-odd iteration stops
when |r^_e| < 0.5e-12 |b| (the criterion the GPU solver uses for its
recursive residual); the true residual is then recomputed.
"""
import argparse
import json
import os
import platform
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_1709_08785_gb300 import inputs  # noqa: E402

WORKLOAD = dict(name="24^3x48 clover-Wilson, eps 0.25 seed 3, kappa 0.124, csw 1.6, t_bc -1, source seed 30",
                dims=(24, 24, 24, 48), eps=0.25, link_seed=3, kappa=0.124, csw=1.6, t_bc=-1, src_seed=30, tol=1e-12)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--openmp", action="store_true", help="use the OpenMP build of the oracle (all host cores)")
    ap.add_argument("--out", default=os.path.join(HERE, "iteration_counts.json"),
                    help="JSON file to update (the entry of this host's architecture is replaced)")
    args = ap.parse_args()
    threads = oracle.use_openmp(args.openmp)
    W = WORKLOAD
    dims = W["dims"]
    U = inputs.random_gauge(dims, W["eps"], W["link_seed"])
    b = inputs.gaussian_source(dims, W["src_seed"])
    F = oracle.clover_field(dims, U, W["kappa"], W["csw"])
    Fi = oracle.invert_sites(F)
    bh = oracle.eo_source(dims, W["t_bc"], U, Fi, W["kappa"], b)
    tol_eo = 0.5 * W["tol"] * np.linalg.norm(b) / np.linalg.norm(bh)
    t0 = time.time()
    x, st, iters = oracle.bicgstab_eo(dims, W["t_bc"], U, Fi, W["kappa"], b, tol_eo, maxit=20000)
    secs = time.time() - t0
    res = oracle.true_residual(dims, W["t_bc"], U, F, W["kappa"], b, x)
    out = dict(workload=W["name"], fp64_eo_bicgstab_iterations=iters, status=st, true_residual=res,
               seconds=secs, threads=threads, host=platform.machine(), cpu=cpu_model())
    data = json.load(open(args.out)) if os.path.exists(args.out) else {}
    by_host = data.get("by_host", {})
    by_host[platform.machine()] = out
    data["by_host"] = by_host
    # the count the benchmark scales by.  Each host's entry is kept: the
    # links come from the host's LAPACK eigendecomposition and differ across
    # hosts at the rounding level, so the residuals differ in their last
    # digits; the iteration counts are what the by_host entries compare
    data["fp64_eo_24x24x24x48"] = out
    with open(args.out, "w") as f:
        json.dump(data, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
