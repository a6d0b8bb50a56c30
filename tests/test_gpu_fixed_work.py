"""The paper's fixed-work protocol (Sec. IV: 2000 or 4000 D^ multiplications,
500 inner per outer) as bench_suite.py runs it, on a small lattice: the D^
applications the solver reports must be exactly the protocol's counts."""
import pytest

torch = pytest.importorskip("torch")

from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_dhat", [2000, 4000])
def test_fixed_work_dhat_counts(n_dhat):
    import bench_suite
    from paper_1709_08785_gb300 import qcd

    # the protocol's near-critical kappa (0.155) on the synthetic fields of
    # its workload (links exp(i 0.25 H) seed 3, source seed 30), 8^3 x 16
    dims, kappa, csw = (8, 8, 8, 16), 0.155, 1.6
    ctx = qcd.Context(dims, -1)
    ctx.gauge_load(torch.from_numpy(inputs.random_gauge(dims, 0.25, 3)).cuda())
    ctx.clover_build(kappa, csw)
    b = torch.from_numpy(inputs.gaussian_source(dims, 30)).cuda()
    x = torch.zeros_like(b)
    info = bench_suite.fixed_work_solve(ctx, b, x, n_dhat)
    sets = n_dhat // 500
    assert info["rc"] == -4, info  # QCD_ENOTCONV: the 1e-30 target is never met
    assert info["outer_iters"] == sets // 2, info
    assert info["inner_iters"][0] == 250 * sets, info           # 250 FP32 iterations per set
    assert info["dhat_applies"][1] == n_dhat, info              # 500 inner D^ per set
    assert info["dhat_applies"][0] == sets, info                # one outer D^ per set
    assert info["restarts"] == 0
    ctx.close()
