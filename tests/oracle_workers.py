"""Oracle work for the tests that check many GPU solutions at once, run in a
process pool (started with the spawn method: the parent holds a CUDA
context).  Each function regenerates its problem's links and source from the
seeds, so nothing larger than a solution crosses the process boundary."""
import numpy as np

import oracle
from paper_1709_08785_gb300 import inputs


def links_and_source(p):
    """The problem's links and source (numpy generators, canonical layouts)."""
    return inputs.random_gauge(p["dims"], p["eps"], p["link_seed"]), inputs.gaussian_source(p["dims"], p["src_seed"])


def true_residual(args):
    """||b - D x|| / ||b|| of a solution x of problem p, by the oracle."""
    p, x = args
    U, b = links_and_source(p)
    F = oracle.clover_field(p["dims"], U, p["kappa"], p["csw"])
    return float(oracle.true_residual(p["dims"], -1, U, F, p["kappa"], b, np.asarray(x)))
