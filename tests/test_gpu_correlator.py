"""qcd_pion_correlator against the oracle: random propagator columns on
lattices with ragged tails (device and host memory), and the whole chain on
8^3x16 -- twelve point-source solves whose oracle true residuals are checked,
then the pion correlator of those columns."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 2, 4, 10)])
@pytest.mark.parametrize("ncol", [3, 12])
@pytest.mark.parametrize("on_device", [True, False])
def test_correlator_matches_oracle(dims, ncol, on_device):
    from paper_1709_08785_gb300 import qcd

    V = inputs.volume(dims)
    rng = np.random.default_rng(80 + ncol)
    S = rng.standard_normal((ncol, V, 4, 3)) + 1j * rng.standard_normal((ncol, V, 4, 3))
    ctx = qcd.Context(dims)
    buf = torch.from_numpy(S).cuda() if on_device else S
    C = ctx.pion_correlator(buf, ncol)
    assert rel(C, oracle.pion_correlator(dims, S)) < 1e-14
    assert np.array_equal(C, ctx.pion_correlator(buf, ncol))  # fixed summation order
    with pytest.raises(qcd.QCDError):
        ctx.pion_correlator(buf, 0)
    ctx.close()


def test_point_source_propagator_chain():
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (8, 8, 8, 16), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 5)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    B = torch.from_numpy(inputs.point_sources(dims)).cuda()
    X = torch.zeros_like(B)
    for k in range(12):
        info = ctx.solve(B[k], X[k], tol=1e-12, precision_levels=2)
        assert info["true_resid"] <= 1e-12
    Xh = X.cpu().numpy()
    F = oracle.clover_field(dims, U, kappa, csw)
    Bh = inputs.point_sources(dims)
    for k in range(12):
        assert oracle.true_residual(dims, t_bc, U, F, kappa, Bh[k], Xh[k]) <= 1e-12
    C = ctx.pion_correlator(X, 12)
    assert rel(C, oracle.pion_correlator(dims, Xh)) < 1e-13
    assert np.all(C > 0) and C[0] > C[dims[3] // 2]  # decays away from the source
    ctx.close()
