"""Parity at the full workload sizes, in the launch configurations the
benchmarks time (autotuned kernels):

* 24^3x48 (bench.py's workload): every operator precision at 96 sampled
  output sites against the oracle, computed one site at a time; the mixed
  FP64/FP32 solve against the oracle's true residual over the whole lattice;
* 48^3x96 (three precision levels): FP32 / FP16 MULT at sampled sites, and
  the three-level solve's residual b - D x recomputed by the oracle at 512
  sampled sites.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TUNE_CACHE = os.path.join(ROOT, "paper_1709_08785_gb300", "_build", "tune_cache.json")
TOL = {0: 1e-13, 1: 2e-6, 2: 2e-3, 3: 1e-13}


def mult_sampled(dims, t_bc, U, kappa, csw, v_half, out_parity, cbs):
    """Oracle F_pp^-1 (H v)(n) at sampled output sites n (cb indices)."""
    v_full = oracle.half_to_full(dims, 1 - out_parity, v_half)
    sites = oracle.site_of_cb(dims, out_parity, cbs)
    h = oracle.hop_sites(dims, t_bc, U, v_full, sites)
    F = oracle.clover_sites(dims, U, kappa, csw, sites)
    return np.linalg.solve(F, h.reshape(len(cbs), 12, 1)).reshape(len(cbs), 4, 3)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def lat24():
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (24, 24, 24, 48), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 3)
    b = inputs.gaussian_source(dims, 30)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(TUNE_CACHE)
    yield dict(dims=dims, kappa=kappa, csw=csw, t_bc=t_bc, U=U, b=b, ctx=ctx)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 3, 1, 2])
def test_24c48_mult_sampled(lat24, prec):
    dims = lat24["dims"]
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 70)[:Vh]
    dt = torch.complex128 if prec in (0, 3) else torch.complex64
    inp = torch.from_numpy(v).to(dt).cuda()
    out = torch.zeros_like(inp)
    lat24["ctx"].mult_eo(out, inp, 0, False, prec)
    torch.cuda.synchronize()
    cbs = np.random.default_rng(71).choice(Vh, 96, replace=False)
    want = mult_sampled(dims, lat24["t_bc"], lat24["U"], lat24["kappa"], lat24["csw"], v, 0, cbs)
    got = out.cpu().numpy().astype(np.complex128)[cbs]
    assert rel(got, want) < TOL[prec]


def test_24c48_dirac_sampled(lat24):
    dims = lat24["dims"]
    v = inputs.gaussian_source(dims, 72)
    inp = torch.from_numpy(v).cuda()
    out = torch.zeros_like(inp)
    lat24["ctx"].dirac(out, inp)
    torch.cuda.synchronize()
    sites = np.random.default_rng(73).choice(inputs.volume(dims), 96, replace=False)
    want = oracle.dirac_sites(dims, lat24["t_bc"], lat24["U"], lat24["kappa"], lat24["csw"], v, sites)
    assert rel(out.cpu().numpy()[sites], want) < 1e-13


@pytest.mark.parametrize("eo_hermitian", [0, 1])
def test_24c48_mixed_solve_true_residual(lat24, eo_hermitian):
    bd = torch.from_numpy(lat24["b"]).cuda()
    x = torch.zeros_like(bd)
    info = lat24["ctx"].solve(bd, x, tol=1e-12, precision_levels=2, eo_hermitian=eo_hermitian)
    assert info["status"] == 0 and info["true_resid"] <= 1e-12
    if "F" not in lat24:  # the oracle's clover field, built once for both forms
        lat24["F"] = oracle.clover_field(lat24["dims"], lat24["U"], lat24["kappa"], lat24["csw"])
    F = lat24["F"]
    r = oracle.true_residual(lat24["dims"], lat24["t_bc"], lat24["U"], F, lat24["kappa"], lat24["b"], x.cpu().numpy())
    assert r <= 1e-12, r
    # the solver's FP64 true residual against the oracle's
    assert abs(info["true_resid"] - r) <= 5e-15, (info["true_resid"], r)


@pytest.fixture(scope="module")
def lat48():
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (48, 48, 48, 96), 0.124, 1.6, -1
    Ud = inputs.random_gauge_torch(dims, 0.25, 4, device="cuda")
    b = inputs.gaussian_source(dims, 40)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(Ud)
    ctx.clover_build(kappa, csw)
    ctx.autotune(TUNE_CACHE)
    U = Ud.cpu().numpy()
    del Ud
    yield dict(dims=dims, kappa=kappa, csw=csw, t_bc=t_bc, U=U, b=b, ctx=ctx)
    ctx.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_48c96_mult_sampled(lat48, prec):
    dims = lat48["dims"]
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 74)[:Vh]
    inp = torch.from_numpy(v).to(torch.complex64).cuda()
    out = torch.zeros_like(inp)
    lat48["ctx"].mult_eo(out, inp, 1, False, prec)
    torch.cuda.synchronize()
    cbs = np.random.default_rng(75).choice(Vh, 96, replace=False)
    want = mult_sampled(dims, lat48["t_bc"], lat48["U"], lat48["kappa"], lat48["csw"], v, 1, cbs)
    got = out.cpu().numpy().astype(np.complex128)[cbs]
    assert rel(got, want) < TOL[prec]


def test_48c96_three_level_solve_sampled_residual(lat48):
    bd = torch.from_numpy(lat48["b"]).cuda()
    x = torch.zeros_like(bd)
    info = lat48["ctx"].solve(bd, x, tol=1e-12, precision_levels=3, inner_tol=[1e-5, 1e-2])
    assert info["status"] == 0 and info["true_resid"] <= 1e-12, info
    assert info["dhat_applies"][2] > 0
    sites = np.random.default_rng(76).choice(inputs.volume(lat48["dims"]), 512, replace=False)
    xs = x.cpu().numpy()
    Dx = oracle.dirac_sites(lat48["dims"], lat48["t_bc"], lat48["U"], lat48["kappa"], lat48["csw"], xs, sites)
    r = np.linalg.norm((lat48["b"][sites] - Dx).ravel()) / np.linalg.norm(lat48["b"][sites].ravel())
    assert r <= 1e-12, r
