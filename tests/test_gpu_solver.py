"""GPU solves checked by the CPU oracle: every solution's true residual
||b - D x|| / ||b|| is recomputed by the oracle in FP64 and must be <= 1e-12,
and the solution must agree with the oracle's own solve.  Covers the
unpreconditioned FP64 BiCGStab (4^4 workload), the even-odd FP64 BiCGStab,
the nested FP64/FP32 scheme of Algs. 1-2, the three-level FP64/FP32/FP16
scheme, host buffers, warm starts, and the failure paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lat4():
    """4^4, links exp(i 0.3 H) seed 1, kappa 0.12, csw 1.0, antiperiodic in
    time, Gaussian source seed 2."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (4, 4, 4, 4), 0.12, 1.0, -1
    U = inputs.random_gauge(dims, 0.3, 1)
    b = inputs.gaussian_source(dims, 2)
    F = oracle.clover_field(dims, U, kappa, csw)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    xo, st, _ = oracle.bicgstab_full(dims, t_bc, U, F, kappa, b, 1e-13)
    assert st == 0
    yield dict(dims=dims, kappa=kappa, csw=csw, t_bc=t_bc, U=U, b=b, F=F, ctx=ctx, xo=xo, qcd=qcd)
    ctx.close()


@pytest.fixture(scope="module")
def lat8():
    """A reduced copy of the 24^3x48 workload's parameters (eps 0.25,
    kappa 0.124, csw 1.6) on 8^3x16, for the nested and three-level solves."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (8, 8, 8, 16), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 3)
    b = inputs.gaussian_source(dims, 4)
    F = oracle.clover_field(dims, U, kappa, csw)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    yield dict(dims=dims, kappa=kappa, csw=csw, t_bc=t_bc, U=U, b=b, F=F, ctx=ctx, qcd=qcd)
    ctx.close()


def solve(P, **kw):
    bd = torch.from_numpy(P["b"]).cuda()
    x = torch.zeros_like(bd)
    info = P["ctx"].solve(bd, x, tol=kw.pop("tol", 1e-12), **kw)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


def true_res(P, x):
    return oracle.true_residual(P["dims"], P["t_bc"], P["U"], P["F"], P["kappa"], P["b"], x)


def test_unpreconditioned_fp64(lat4):
    x, info = solve(lat4, precision_levels=1, even_odd=0)
    assert info["status"] == 0
    assert true_res(lat4, x) <= 1e-12
    assert abs(info["true_resid"] - true_res(lat4, x)) <= 1e-13
    assert np.linalg.norm(x - lat4["xo"]) / np.linalg.norm(lat4["xo"]) < 1e-10


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_even_odd_solves_4c4(lat4, levels):
    x, info = solve(lat4, precision_levels=levels)
    assert info["status"] == 0, info
    assert true_res(lat4, x) <= 1e-12
    assert np.linalg.norm(x - lat4["xo"]) / np.linalg.norm(lat4["xo"]) < 1e-10


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_even_odd_solves_8c16(lat8, levels):
    x, info = solve(lat8, precision_levels=levels)
    assert info["status"] == 0, info
    r = true_res(lat8, x)
    assert r <= 1e-12, (r, info)
    # the solver's own FP64 true residual against the oracle's
    assert abs(info["true_resid"] - r) <= 5e-15, (info["true_resid"], r)
    if levels >= 2:
        assert info["dhat_applies"][1] > 0 and info["outer_iters"] >= 1
    if levels == 3:
        assert info["dhat_applies"][2] > 0


@pytest.mark.parametrize("levels", [2, 3])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_outer_level_modes(lat8, levels, mode):
    """The nested schemes with each arithmetic of the outer level: FP64
    throughout (0), FP64 solution around DF64 operator applications (1, the
    default) and DF64 throughout (2)."""
    x, info = solve(lat8, precision_levels=levels, outer_df64=mode)
    assert info["status"] == 0, info
    r = true_res(lat8, x)
    assert r <= 1e-12
    assert abs(info["true_resid"] - r) <= 5e-15, (info["true_resid"], r)


def test_default_outer_mode_agrees_with_fp64_outer(lat8):
    """The default (FP64 solution, DF64 operator) against the all-FP64 outer
    level: both solves meet 1e-12, so the solutions agree to the operator's
    conditioning times that."""
    x1, i1 = solve(lat8, precision_levels=2)
    x0, i0 = solve(lat8, precision_levels=2, outer_df64=0)
    assert i1["status"] == 0 and i0["status"] == 0
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < 1e-10


def even_mask(dims):
    Lx, Ly, Lz, Lt = dims
    t, z, y, xx = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((xx + y + z + t) % 2 == 0).ravel()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_solution_storage_is_fp64(lat8, mode):
    """Where the solution x_e lives.  The source b = D x0 is built by the
    oracle for a random FP64 x0 and x0 is given as the initial guess: its
    residual already meets the tolerance, so the solver updates nothing and
    returns x_e as it stored it.  With the solution kept in FP64 (modes 0 and
    1) the even sites come back bit for bit; the all-DF64 outer level
    (mode 2) rounds them to a float pair (~48 bits), which this check sees."""
    P = lat8
    x0 = inputs.gaussian_source(P["dims"], 77)
    b = oracle.dirac(P["dims"], P["t_bc"], P["U"], P["F"], P["kappa"], x0)
    bd = torch.from_numpy(b).cuda()
    x = torch.from_numpy(x0.copy()).cuda()
    info = P["ctx"].solve(bd, x, tol=1e-10, precision_levels=2, use_x0=1, outer_df64=mode)
    torch.cuda.synchronize()
    assert info["status"] == 0 and info["outer_iters"] == 0, info
    xs = x.cpu().numpy()
    ev = even_mask(P["dims"])
    same = np.array_equal(xs[ev], x0[ev])
    if mode in (0, 1):
        assert same
    else:
        assert not same
        assert np.linalg.norm(xs[ev] - x0[ev]) / np.linalg.norm(x0[ev]) < 1e-14
    # the odd sites are x_o = F_oo^-1 (b_o + kappa H_oe x_e), recomputed
    assert np.linalg.norm(xs[~ev] - x0[~ev]) / np.linalg.norm(x0[~ev]) < 1e-13


@pytest.mark.parametrize("levels", [1, 2, 3])
@pytest.mark.parametrize("lat", ["lat4", "lat8"])
def test_gamma5_hermitian_form_solves(request, lat, levels):
    """Every level iterating on the gamma5-hermitian S_ee = F_ee D^_ee
    (eo_hermitian = 1): the oracle's true residual meets 1e-12 and the
    solution agrees with the oracle's own BiCGStab on S_ee."""
    P = request.getfixturevalue(lat)
    x, info = solve(P, precision_levels=levels, eo_hermitian=1)
    assert info["status"] == 0, info
    r = true_res(P, x)
    assert r <= 1e-12, (r, info)
    assert abs(info["true_resid"] - r) <= 5e-15, (info["true_resid"], r)
    Fi = oracle.invert_sites(P["F"])
    xo, st, _ = oracle.bicgstab_schur(P["dims"], P["t_bc"], P["U"], P["F"], Fi, P["kappa"], P["b"], 1e-13)
    assert st == 0
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-10


def test_gamma5_hermitian_form_rejected_by_batched(lat4):
    qcd = lat4["qcd"]
    bd = torch.from_numpy(lat4["b"]).cuda()
    with pytest.raises(qcd.QCDError):
        qcd.solve_batched([lat4["ctx"]], [bd], [torch.zeros_like(bd)], [1e-10], precision_levels=2, eo_hermitian=1)


def test_host_buffers(lat4):
    x = np.zeros_like(lat4["b"])
    info = lat4["ctx"].solve(lat4["b"], x, tol=1e-12, precision_levels=2)
    assert info["status"] == 0
    assert true_res(lat4, x) <= 1e-12


def test_warm_start_from_solution(lat4):
    bd = torch.from_numpy(lat4["b"]).cuda()
    x = torch.from_numpy(lat4["xo"]).cuda()
    info = lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, use_x0=1)
    assert info["status"] == 0 and info["outer_iters"] <= 1
    assert true_res(lat4, x.cpu().numpy()) <= 1e-12


def test_zero_source(lat4):
    bd = torch.zeros_like(torch.from_numpy(lat4["b"])).cuda()
    x = torch.ones_like(bd)
    info = lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, check=False)
    assert info["rc"] == 0
    assert torch.count_nonzero(x).item() == 0


def test_nonfinite_source(lat4):
    b = lat4["b"].copy()
    b[3, 1, 2] = np.nan
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, check=False)
    assert info["rc"] == -6  # QCD_ENONFINITE


def test_singular_clover_block_reported(lat4):
    """A clover block whose LDL^H pivots are not finite (one NaN link) is
    reported as QCD_ECLOVER_SINGULAR; a good field afterwards builds again."""
    qcd = lat4["qcd"]
    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0.3, 1)
    bad = U.copy()
    bad[17, 2, 0, 1] = np.nan
    ctx = qcd.Context(dims)
    ctx.gauge_load(torch.from_numpy(bad).cuda())
    with pytest.raises(qcd.QCDError) as e:
        ctx.clover_build(0.12, 1.0)
    assert e.value.status == -7
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(0.12, 1.0)
    ctx.close()


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_pinned_host_buffers_match_device(lat8, levels):
    """Pinned host b and x: the solution is copied out while the true
    residual is checked, and equals the device-buffer solve bit for bit (the
    reductions are deterministic)."""
    bd = torch.from_numpy(lat8["b"]).cuda()
    xd = torch.zeros_like(bd)
    info_d = lat8["ctx"].solve(bd, xd, tol=1e-12, precision_levels=levels)
    bh = torch.from_numpy(lat8["b"]).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    info_h = lat8["ctx"].solve(bh, xh, tol=1e-12, precision_levels=levels)
    assert info_d["status"] == 0 and info_h["status"] == 0
    assert torch.equal(xh, xd.cpu())
    assert info_h["true_resid"] == info_d["true_resid"]
    assert true_res(lat8, xh.numpy()) <= 1e-12


def test_iteration_cap(lat4):
    bd = torch.from_numpy(lat4["b"]).cuda()
    x = torch.zeros_like(bd)
    info = lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=1, max_outer=1, max_restarts=0, check=False)
    assert info["rc"] == -4  # QCD_ENOTCONV
    assert info["true_resid"] > 1e-12


def test_invalid_arguments(lat4):
    qcd = lat4["qcd"]
    bd = torch.from_numpy(lat4["b"]).cuda()
    x = torch.zeros_like(bd)
    with pytest.raises(qcd.QCDError):
        lat4["ctx"].solve(bd, x, tol=-1.0)
    with pytest.raises(qcd.QCDError):
        lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, even_odd=0)
    with pytest.raises(qcd.QCDError):  # outer_df64 outside 0..2
        lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, outer_df64=3)
    with pytest.raises(qcd.QCDError):
        lat4["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, eo_hermitian=2)
    with pytest.raises(qcd.QCDError):
        qcd.Context((4, 4, 3, 4))
    ctx = qcd.Context((4, 4, 4, 4))
    with pytest.raises(qcd.QCDError):  # no gauge field yet
        ctx.clover_build(0.12, 1.0)
    with pytest.raises(qcd.QCDError):
        ctx.solve(bd, x)
    ctx.close()


def test_solve_repeatable_bitwise(lat8):
    x1, i1 = solve(lat8, precision_levels=2)
    x2, i2 = solve(lat8, precision_levels=2)
    assert np.array_equal(x1, x2)
    assert i1["inner_iters"] == i2["inner_iters"]


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_periodic_time_boundary(levels):
    """Periodic time (t_bc = +1) on a lattice with ragged 32-site blocks."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (6, 2, 4, 10), 0.12, 1.3, 1
    U = inputs.random_gauge(dims, 0.3, 21)
    b = inputs.gaussian_source(dims, 22)
    F = oracle.clover_field(dims, U, kappa, csw)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = ctx.solve(bd, x, tol=1e-12, precision_levels=levels)
    assert info["status"] == 0
    assert oracle.true_residual(dims, t_bc, U, F, kappa, b, x.cpu().numpy()) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("levels", [1, 2])
def test_degenerate_kappa_zero(levels):
    """kappa = 0: no hopping and no clover term, D = 1, so x = b exactly."""
    from paper_1709_08785_gb300 import qcd

    dims = (4, 4, 4, 4)
    U = inputs.random_gauge(dims, 0.3, 23)
    b = inputs.gaussian_source(dims, 24)
    ctx = qcd.Context(dims, -1)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(0.0, 1.0)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = ctx.solve(bd, x, tol=1e-12, precision_levels=levels)
    assert info["status"] == 0 and info["true_resid"] <= 1e-12
    assert np.max(np.abs(x.cpu().numpy() - b)) <= 1e-13 * np.max(np.abs(b))
    ctx.close()


def test_wilson_without_clover():
    """csw = 0: the plain Wilson operator (F = 1)."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, t_bc = (4, 4, 4, 8), 0.12, -1
    U = inputs.random_gauge(dims, 0.3, 25)
    b = inputs.gaussian_source(dims, 26)
    F = oracle.clover_field(dims, U, kappa, 0.0)
    assert np.max(np.abs(F - np.eye(12)[None])) == 0.0
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, 0.0)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = ctx.solve(bd, x, tol=1e-12, precision_levels=2)
    assert info["status"] == 0
    assert oracle.true_residual(dims, t_bc, U, F, kappa, b, x.cpu().numpy()) <= 1e-12
    ctx.close()


def test_chunk_timing_counts_whole_iterations(lat8):
    """qcd_set_profiling(ctx, 2): one event pair per queued chunk of FP32
    iterations; the class QCD_K_INNER_ITER must count exactly the solve's
    inner iterations, with their algorithmic bytes (two D^ with the fused
    dots and three BLAS-1 updates: about 5088 bytes per even site), and the
    solve must be unchanged by it."""
    qcd = lat8["qcd"]
    ctx = lat8["ctx"]
    x0, i0 = solve(lat8, precision_levels=2)
    ctx.reset_kernel_stats()
    ctx.set_profiling(2)
    x1, i1 = solve(lat8, precision_levels=2)
    ctx.set_profiling(0)
    assert np.array_equal(x0, x1)
    st = ctx.kernel_stats(qcd.K_INNER_ITER)
    assert st["launches"] == i1["inner_iters"][0] > 0
    assert st["ms"] > 0
    vh = inputs.volume(lat8["dims"]) // 2
    per_site = st["bytes"] / st["launches"] / vh
    assert 4800 < per_site < 5300, per_site
    with pytest.raises(qcd.QCDError):
        ctx.set_profiling(3)
