"""Batched solves in one persistent cooperative kernel per outer half-step,
replayed from a CUDA graph: every problem's solution is checked by the
oracle's true residual, against the single-problem solver, with graphs on
and off; a grid-barrier wait limit of one spin must end the batch with
QCD_ETIMEOUT (no fault, no hang) and leave the contexts usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu

LATTICES = [(4, 4, 4, 4), (6, 2, 4, 10), (8, 8, 8, 8), (4, 4, 4, 8), (8, 4, 4, 8), (2, 2, 2, 2), (8, 8, 8, 16)]


@pytest.fixture(scope="module")
def batch():
    from paper_1709_08785_gb300 import qcd

    rng = np.random.default_rng(97)
    probs = []
    for i, dims in enumerate(LATTICES):
        eps = float(rng.uniform(0.15, 0.35))
        kappa = float(rng.uniform(0.115, 0.124))
        U = inputs.random_gauge(dims, eps, 300 + i)
        b = inputs.gaussian_source(dims, 400 + i)
        ctx = qcd.Context(dims, -1)
        ctx.gauge_load(torch.from_numpy(U).cuda())
        ctx.clover_build(kappa, 1.0)
        probs.append(dict(dims=dims, kappa=kappa, U=U, b=b, ctx=ctx, bd=torch.from_numpy(b).cuda()))
    yield probs
    for p in probs:
        p["ctx"].close()


def run_batch(probs, tol=1e-10, check=True, **kw):
    from paper_1709_08785_gb300 import qcd

    xs = [torch.zeros_like(p["bd"]) for p in probs]
    infos = qcd.solve_batched([p["ctx"] for p in probs], [p["bd"] for p in probs], xs, [tol] * len(probs),
                              check=check, precision_levels=2, **kw)
    torch.cuda.synchronize()
    return xs, infos


@pytest.mark.parametrize("graphs", [True, False])
def test_batched_solves_reach_tolerance(batch, graphs):
    from paper_1709_08785_gb300 import qcd

    qcd.set_graphs(graphs)
    try:
        xs, infos = run_batch(batch)
    finally:
        qcd.set_graphs(True)
    for p, x, info in zip(batch, xs, infos):
        assert info["status"] == 0, info
        F = oracle.clover_field(p["dims"], p["U"], p["kappa"], 1.0)
        r = oracle.true_residual(p["dims"], -1, p["U"], F, p["kappa"], p["b"], x.cpu().numpy())
        assert r <= 1e-10, (p["dims"], r, info)
        assert abs(r - info["true_resid"]) <= 1e-12 + 0.1 * r
        # the persistent kernels converged every problem themselves: no
        # problem was handed to the single-solve driver afterwards
        assert info["restarts"] == 0, info
        if p["dims"] != (2, 2, 2, 2):
            assert info["inner_iters"][0] > 0 and info["dhat_applies"][1] > 0


def test_batched_matches_single_solves(batch):
    xs, infos = run_batch(batch, tol=1e-12)
    for p, x in zip(batch, xs):
        xs1 = torch.zeros_like(p["bd"])
        p["ctx"].solve(p["bd"], xs1, tol=1e-12, precision_levels=2)
        a, b = x.cpu().numpy(), xs1.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-9


def test_batched_repeatable_bitwise(batch):
    x1, i1 = run_batch(batch)
    x2, i2 = run_batch(batch)
    for a, b in zip(x1, x2):
        assert torch.equal(a, b)
    assert [i["inner_iters"] for i in i1] == [i["inner_iters"] for i in i2]


def test_barrier_wait_limit_reports_timeout(batch):
    from paper_1709_08785_gb300 import qcd

    qcd.set_wait_limit(1)
    try:
        xs, infos = run_batch(batch, check=False)
        assert infos[0]["rc"] == -8  # QCD_ETIMEOUT: the wait gave up, the kernel returned
    finally:
        qcd.set_wait_limit(10_000_000)
    # the contexts stay usable
    xs, infos = run_batch(batch)
    assert all(i["status"] == 0 for i in infos)


def test_batched_rejects_bad_arguments(batch):
    from paper_1709_08785_gb300 import qcd

    p = batch[0]
    x = torch.zeros_like(p["bd"])
    with pytest.raises(qcd.QCDError):  # three precision levels are not batched
        qcd.solve_batched([p["ctx"]], [p["bd"]], [x], [1e-10], precision_levels=3)
    with pytest.raises(qcd.QCDError):  # one context twice
        qcd.solve_batched([p["ctx"], p["ctx"]], [p["bd"], p["bd"]], [x, torch.zeros_like(x)], [1e-10, 1e-10])


@pytest.mark.parametrize("mode", [0, 2])
def test_batched_outer_level_modes(batch, mode):
    """The batch with its outer level in FP64 (outer_df64 = 0) or all in
    DF64 (2) instead of the default (FP64 solution around DF64 operator
    applications)."""
    xs, infos = run_batch(batch, outer_df64=mode)
    for p, x, inf in zip(batch, xs, infos):
        assert inf["status"] == 0 and inf["restarts"] == 0, inf
        F = oracle.clover_field(p["dims"], p["U"], p["kappa"], 1.0)
        assert oracle.true_residual(p["dims"], -1, p["U"], F, p["kappa"], p["b"], x.cpu().numpy()) <= 1e-10


def test_batched_48_problem_workload():
    """The batched workload at its own sizes: 48 problems drawn from
    {8^4, 12^3x24, 16^3x32, 20^3x40} (inputs.batch_problems(48, 99)), tol
    1e-10, one batched run.  Every solution's true residual is recomputed by
    the oracle (in a spawned process pool) and must meet the tolerance, and
    no problem may have needed the single-solve fallback."""
    import multiprocessing as mp
    import os

    import oracle_workers
    from paper_1709_08785_gb300 import qcd

    probs = inputs.batch_problems(48, 99)
    tol = 1e-10
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        fields = pool.map(oracle_workers.links_and_source, probs, chunksize=1)
        ctxs, bs, xs = [], [], []
        for p, (U, b) in zip(probs, fields):
            c = qcd.Context(p["dims"], -1)
            c.gauge_load(torch.from_numpy(U).cuda())
            c.clover_build(p["kappa"], p["csw"])
            ctxs.append(c)
            bs.append(torch.from_numpy(b).cuda())
            xs.append(torch.zeros_like(bs[-1]))
        del fields
        infos = qcd.solve_batched(ctxs, bs, xs, [tol] * len(probs), precision_levels=2)
        torch.cuda.synchronize()
        res = pool.map(oracle_workers.true_residual, [(p, x.cpu().numpy()) for p, x in zip(probs, xs)], chunksize=1)
    for p, info, r in zip(probs, infos, res):
        assert info["status"] == 0 and info["restarts"] == 0, (p, info)
        assert r <= tol, (p, r, info)
        assert abs(r - info["true_resid"]) <= 1e-14 + 1e-3 * r, (p, r, info["true_resid"])
    assert {p["dims"] for p in probs} == set(inputs.BATCH_LATTICES)
    for c in ctxs:
        c.close()
