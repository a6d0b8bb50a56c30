"""Run the oracle's FP64 even-odd BiCGStab to a true residual of 1e-12 on
the 24^3 x 48 workload and record how many iterations it took.

TEST INFRASTRUCTURE: the CPU reference arm of the benchmark scales its
bounded per-application timing by this count (it never runs the CUDA path).
Calls only the oracle and the seeded input generators.  Writes
oracle/iteration_counts.json.  Takes of the order of an hour on one core.

Workload: links reunitarised exp(i 0.25 H) seed 3, kappa 0.124, csw 1.6,
antiperiodic in time, Gaussian source seed 30.  The even-odd iteration stops
when |r^_e| < 0.5e-12 |b| (the criterion the GPU solver uses for its
recursive residual); the true residual is then recomputed.
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_1709_08785_gb300 import inputs  # noqa: E402

WORKLOAD = dict(name="24^3x48 clover-Wilson, eps 0.25 seed 3, kappa 0.124, csw 1.6, t_bc -1, source seed 30",
                dims=(24, 24, 24, 48), eps=0.25, link_seed=3, kappa=0.124, csw=1.6, t_bc=-1, src_seed=30, tol=1e-12)


def main():
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
               seconds_single_core=secs, host=platform.machine(), cpu=platform.processor())
    path = os.path.join(HERE, "iteration_counts.json")
    with open(path, "w") as f:
        json.dump({"fp64_eo_24x24x24x48": out}, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
