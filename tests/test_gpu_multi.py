"""qcd_solve_multi: the nested solve of several right-hand sides in lockstep
(the FP32 iterations through the multi-RHS MULT and a per-RHS reducing
second half of D^).  Each right-hand side repeats qcd_solve's arithmetic in
qcd_solve's order, so every column must equal the single solve's solution
bit for bit, with the same iteration counts; the oracle recomputes the true
residuals."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu

KAPPA, CSW, TBC = 0.124, 1.6, -1


def make_ctx(dims, seed, tune=None):
    from paper_1709_08785_gb300 import qcd

    U = inputs.random_gauge(dims, 0.25, seed)
    ctx = qcd.Context(dims, TBC)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(KAPPA, CSW)
    if tune:
        ctx.autotune(tune)
    return ctx, U


def sources(dims, kind, n, seed):
    if kind == "point":
        return inputs.point_sources(dims)[:n]
    return np.stack([inputs.gaussian_source(dims, seed + k) for k in range(n)])


def check_against_single(ctx, U, dims, B, outer_df64, tol=1e-12, converge=True, **kw):
    from paper_1709_08785_gb300 import qcd

    opts = qcd.default_opts(precision_levels=2, outer_df64=outer_df64, **kw)
    Bd = torch.from_numpy(B).cuda()
    X = torch.zeros_like(Bd)
    infos = ctx.solve_multi(Bd, X, tol=tol, opts=opts, check=converge)
    torch.cuda.synchronize()
    Xm = X.cpu().numpy()
    F = oracle.clover_field(dims, U, KAPPA, CSW)
    for k in range(B.shape[0]):
        x1 = torch.zeros_like(Bd[k])
        one = ctx.solve(Bd[k], x1, tol=tol, opts=opts, check=converge)
        torch.cuda.synchronize()
        assert np.array_equal(Xm[k], x1.cpu().numpy()), k
        for key in ("outer_iters", "inner_iters", "dhat_applies", "restarts", "status"):
            assert infos[k][key] == one[key], (k, key, infos[k][key], one[key])
        assert infos[k]["true_resid"] == one["true_resid"], k
        if converge and np.any(B[k]):  # (a zero right-hand side has no relative residual: x = 0 is checked by the caller)
            assert oracle.true_residual(dims, TBC, U, F, KAPPA, B[k], Xm[k]) <= tol, k
    return infos


@pytest.mark.parametrize("dims", [(6, 2, 4, 10), (8, 8, 8, 16)])
@pytest.mark.parametrize("kind,n", [("point", 12), ("gauss", 3), ("gauss", 1), ("gauss", 16)])
@pytest.mark.parametrize("outer_df64", [1, 0])
def test_multi_equals_single_solves(dims, kind, n, outer_df64):
    """Lockstep columns against one qcd_solve per column (untuned launch
    shapes), on a lattice with ragged blocks and on 8^3x16, point and
    Gaussian sources, both outer arithmetics."""
    ctx, U = make_ctx(dims, 130)
    check_against_single(ctx, U, dims, sources(dims, kind, n, 131), outer_df64)
    ctx.close()


def test_multi_equals_single_tuned(tmp_path):
    """The same with the autotuner's launch shapes (the capped-register and
    pipelined variants, its sites per block and right-hand-side tile)."""
    dims = (8, 8, 8, 16)
    ctx, U = make_ctx(dims, 132, str(tmp_path / "tune.json"))
    check_against_single(ctx, U, dims, sources(dims, "point", 12, 0), 1)
    ctx.close()


def test_multi_forced_shapes(tmp_path):
    """Every tuned entry forced to another shape through the cache (64 sites
    per block, the 80-register and pipelined kernels, a tile of 4 right-hand
    sides): the lockstep columns still equal the single solves."""
    from paper_1709_08785_gb300 import qcd

    dims = (6, 2, 4, 10)
    cache = str(tmp_path / "tune.json")
    ctx, U = make_ctx(dims, 133, cache)
    ctx.close()
    data = json.load(open(cache))
    for k, (variant, bx, us) in list(data.items()):
        key = int(k.rsplit("|", 1)[1])
        prec, mode, red, nrhs = key & 3, (key >> 2) & 7, (key >> 5) & 3, key >> 8
        if prec == 1 and nrhs > 1 and red == 0 and mode in (0, 1):
            data[k] = [1, 4, us]
        elif prec == 1 and nrhs == 1 and mode == 2:
            data[k] = [2 if red == 1 else 1, 64, us]  # the second halves: pipelined / capped, 64 sites
        elif nrhs == 1:
            data[k] = [variant, 64, us]
    with open(cache, "w") as f:
        f.write("{\n" + ",\n".join('  "%s": [%d, %d, %.3f]' % (k, *e) for k, e in data.items()) + "\n}\n")
    ctx, U = make_ctx(dims, 133, cache)
    assert any(e["threads"] == 4 and e["nrhs"] == 12 for e in ctx.tune_info())
    check_against_single(ctx, U, dims, sources(dims, "point", 12, 0), 1)
    ctx.close()


def test_multi_caps_and_restarts():
    """The exits that are not convergence, column by column as qcd_solve
    takes them: the outer iteration cap (QCD_ENOTCONV with no restart left)
    and a tolerance below what FP64 reaches (5e-16), where a recursive
    residual below the threshold meets a true residual above it and the
    solve restarts from the true residual until it runs out of restarts."""
    dims = (6, 2, 4, 10)
    ctx, U = make_ctx(dims, 137)
    B = sources(dims, "gauss", 5, 138)
    infos = check_against_single(ctx, U, dims, B, 1, converge=False, max_outer=1, max_restarts=0)
    assert all(i["status"] == -4 and i["restarts"] == 0 for i in infos)  # QCD_ENOTCONV
    infos = check_against_single(ctx, U, dims, B, 1, tol=5e-16, converge=False, max_restarts=2)
    assert any(i["restarts"] > 0 for i in infos), [i["restarts"] for i in infos]
    ctx.close()


def test_multi_zero_and_repeated_columns():
    """A zero right-hand side (converged before any iteration: x = 0) and a
    repeated one beside ordinary columns: the others are unaffected, the
    zero column stays zero, the repeated columns are equal."""
    from paper_1709_08785_gb300 import qcd

    dims = (8, 8, 8, 16)
    ctx, U = make_ctx(dims, 134)
    B = sources(dims, "gauss", 4, 135)
    B[1] = 0.0
    B[3] = B[2]
    infos = check_against_single(ctx, U, dims, B, 1)
    assert infos[1]["outer_iters"] == 0 and infos[1]["inner_iters"][0] == 0
    Bd = torch.from_numpy(B).cuda()
    X = torch.full_like(Bd, 7.0)
    ctx.solve_multi(Bd, X, tol=1e-12, opts=qcd.default_opts())
    Xh = X.cpu().numpy()
    assert not np.any(Xh[1])
    assert np.array_equal(Xh[2], Xh[3])
    ctx.close()


def test_multi_rejects_bad_arguments():
    from paper_1709_08785_gb300 import qcd

    dims = (4, 4, 4, 4)
    ctx, U = make_ctx(dims, 136)
    V = inputs.volume(dims)
    B = torch.zeros((2, V, 4, 3), dtype=torch.complex128, device="cuda")
    X = torch.zeros_like(B)
    for kw in (dict(precision_levels=3), dict(precision_levels=1), dict(eo_hermitian=1), dict(outer_df64=2),
               dict(use_x0=1)):
        with pytest.raises(qcd.QCDError):
            ctx.solve_multi(B, X, opts=qcd.default_opts(**kw))
    with pytest.raises(qcd.QCDError):  # host memory
        ctx.solve_multi(B.cpu().numpy(), X.cpu().numpy())
    Z = torch.zeros((17, V, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(qcd.QCDError):  # more than 16 right-hand sides
        ctx.solve_multi(Z, torch.zeros_like(Z))
    ctx.close()


@pytest.mark.slow
def test_multi_point_sources_32c64():
    """The point-source workload at its own size (32^3x64, links
    exp(i 0.25 H) seed 5, kappa 0.1235, csw 1.6): the twelve spin-colour
    point sources at the origin solved in lockstep equal the twelve single
    solves bit for bit; the oracle recomputes b - D x at 256 sampled sites of
    each column (the origin among them)."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw = (32, 32, 32, 64), 0.1235, 1.6
    V = inputs.volume(dims)
    Ud = inputs.random_gauge_torch(dims, 0.25, 5, device="cuda")
    ctx = qcd.Context(dims, TBC)
    ctx.gauge_load(Ud)
    ctx.clover_build(kappa, csw)
    U = Ud.cpu().numpy()
    del Ud
    B = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device="cuda")
    for k in range(12):
        B[k, 0, k // 3, k % 3] = 1.0
    X = torch.zeros_like(B)
    infos = ctx.solve_multi(B, X, tol=1e-12)
    for k in range(12):
        assert infos[k]["status"] == 0 and infos[k]["true_resid"] <= 1e-12, (k, infos[k])
    x1 = torch.zeros_like(B[0])
    for k in (0, 5, 11):  # single solves of three columns, bit for bit
        info = ctx.solve(B[k], x1, tol=1e-12)
        assert torch.equal(x1, X[k]), k
        assert info["inner_iters"] == infos[k]["inner_iters"], k
    Xh = X.cpu().numpy()
    sites = np.concatenate([[0], np.random.default_rng(78).choice(np.arange(1, V), 255, replace=False)])
    for k in range(12):
        bk = np.zeros((len(sites), 4, 3), dtype=np.complex128)
        bk[0, k // 3, k % 3] = 1.0  # sites[0] is the origin; |b| = 1
        Dx = oracle.dirac_sites(dims, TBC, U, kappa, csw, Xh[k], sites)
        assert np.linalg.norm((bk - Dx).ravel()) <= 1e-12, k
    ctx.close()
