"""The OpenMP build of the oracle (used for the multi-core CPU baseline)
splits only the loops over sites; every site's arithmetic and every
reduction is the serial build's, so the two must agree bit for bit."""
import numpy as np

import oracle
from paper_1709_08785_gb300 import inputs


def test_openmp_build_matches_serial_bitwise():
    dims, kappa, csw, t_bc = (6, 4, 4, 8), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 3)
    b = inputs.gaussian_source(dims, 4)
    Vh = inputs.volume(dims) // 2
    out = {}
    try:
        for omp in (False, True):
            threads = oracle.use_openmp(omp, 4 if omp else None)
            assert threads >= 1
            F = oracle.clover_field(dims, U, kappa, csw)
            Fi = oracle.invert_sites(F)
            out[omp] = (F, oracle.dirac(dims, t_bc, U, F, kappa, b), oracle.dhat(dims, t_bc, U, Fi, kappa, b[:Vh]),
                        oracle.true_residual(dims, t_bc, U, F, kappa, b, b))
    finally:
        oracle.use_openmp(False)
    for a, c in zip(out[False], out[True]):
        assert np.array_equal(a, c)
