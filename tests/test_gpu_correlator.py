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


@pytest.mark.slow
def test_point_source_propagator_32c64():
    """The point-source workload at its own size: twelve spin-colour point
    sources at the origin of a 32^3x64 field (links exp(i 0.25 H) seed 5,
    kappa 0.1235, csw 1.6), solved to 1e-12.  The oracle recomputes each
    column's residual b - D x at 256 sampled sites (the origin, where the
    source sits, among them), and the pion correlator of the twelve GPU
    columns against the oracle's definition."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (32, 32, 32, 64), 0.1235, 1.6, -1
    V = inputs.volume(dims)
    Ud = inputs.random_gauge_torch(dims, 0.25, 5, device="cuda")
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(Ud)
    ctx.clover_build(kappa, csw)
    U = Ud.cpu().numpy()
    del Ud
    X = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device="cuda")
    for k in range(12):
        b = torch.zeros((V, 4, 3), dtype=torch.complex128, device="cuda")
        b[0, k // 3, k % 3] = 1.0
        info = ctx.solve(b, X[k], tol=1e-12, precision_levels=2)
        assert info["status"] == 0 and info["true_resid"] <= 1e-12, (k, info)
        del b
    torch.cuda.synchronize()
    sites = np.concatenate([[0], np.random.default_rng(77).choice(np.arange(1, V), 255, replace=False)])
    Xh = X.cpu().numpy()
    for k in range(12):
        bk = np.zeros((len(sites), 4, 3), dtype=np.complex128)
        bk[0, k // 3, k % 3] = 1.0  # sites[0] is the origin; |b| = 1
        Dx = oracle.dirac_sites(dims, t_bc, U, kappa, csw, Xh[k], sites)
        assert np.linalg.norm((bk - Dx).ravel()) <= 1e-12, k
    C = ctx.pion_correlator(X, 12)
    assert rel(C, oracle.pion_correlator(dims, Xh)) < 1e-13
    ctx.close()
