"""Adjoint gradient of L = Re<eta, D^-1 b> through the C ABI and the
torch.autograd.Function, against the oracle and central finite differences.

* qcd_force against the oracle's product-rule gradient (random x, lambda);
* qcd_solve_adjoint: D^dag lambda = g to 1e-12, checked by the oracle;
* autograd on a 4^4 copy of the 16^3x32 workload against the oracle gradient;
* the 16^3x32 workload (links exp(i 0.3 H) seed 6, kappa 0.12, csw 1.0, eta and
  b seeds 60/61): directional derivatives along random su(3) directions on 32
  sampled links (seed 62) against central differences with h = 1e-6, taken as
  L(+h) - L(-h) = -Re<eta, D_+^-1 (D_+ - D_-) x_->, so that the solver
  tolerance is relative to the O(h) difference and not to L itself.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu

G5 = np.array([[0, 0, -1, 0], [0, 0, 0, -1], [-1, 0, 0, 0], [0, -1, 0, 0]], dtype=complex)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def g5(v):
    return np.einsum("ab,sbi->sai", G5, v)


def make_ctx(dims, U, kappa, csw, t_bc=-1):
    from paper_1709_08785_gb300 import qcd

    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    return ctx


@pytest.mark.parametrize("dims,t_bc,csw", [((4, 4, 4, 4), -1, 1.0), ((6, 2, 4, 10), 1, 1.6), ((2, 2, 2, 2), -1, 1.3)])
def test_force_matches_oracle(dims, t_bc, csw):
    kappa = 0.12
    U = inputs.random_gauge(dims, 0.3, 80)
    x = inputs.gaussian_source(dims, 81)
    lam = inputs.gaussian_source(dims, 82)
    want = oracle.link_grad(dims, t_bc, U, kappa, csw, x, lam)
    ctx = make_ctx(dims, U, kappa, csw, t_bc)
    G = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    ctx.force(torch.from_numpy(U).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(lam).cuda(), G)
    torch.cuda.synchronize()
    assert rel(G.cpu().numpy(), want) < 1e-12
    ctx.close()


def test_force_hopping_only_when_csw_zero():
    dims, kappa, t_bc = (4, 4, 2, 4), 0.12, -1
    U = inputs.random_gauge(dims, 0.3, 83)
    x, lam = inputs.gaussian_source(dims, 84), inputs.gaussian_source(dims, 85)
    want = oracle.link_grad(dims, t_bc, U, kappa, 0.0, x, lam)
    ctx = make_ctx(dims, U, kappa, 0.0, t_bc)
    G = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    ctx.force(torch.from_numpy(U).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(lam).cuda(), G)
    torch.cuda.synchronize()
    assert rel(G.cpu().numpy(), want) < 1e-12
    ctx.close()


def test_solve_adjoint():
    dims, kappa, csw, t_bc = (4, 4, 4, 8), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 86)
    g = inputs.gaussian_source(dims, 87)
    ctx = make_ctx(dims, U, kappa, csw, t_bc)
    lam = torch.zeros(g.shape, dtype=torch.complex128, device="cuda")
    info = ctx.solve_adjoint(torch.from_numpy(g).cuda(), lam, tol=1e-12, precision_levels=2)
    assert info["rc"] == 0
    lam = lam.cpu().numpy()
    F = oracle.clover_field(dims, U, kappa, csw)
    Ddag_lam = g5(oracle.dirac(dims, t_bc, U, F, kappa, g5(lam)))
    assert np.linalg.norm(g - Ddag_lam) / np.linalg.norm(g) <= 1e-12
    ctx.close()


def test_autograd_matches_oracle_gradient_4x4():
    """The 16^3x32 workload's parameters on a 4^4 copy: torch's gradients of
    L = Re<eta, D^-1 b> against the oracle's (dense solves)."""
    from paper_1709_08785_gb300 import qcd
    from paper_1709_08785_gb300.autograd import clover_solve

    dims, kappa, csw, t_bc = (4, 4, 4, 4), 0.12, 1.0, -1
    U = inputs.random_gauge(dims, 0.3, 6)
    b = inputs.gaussian_source(dims, 61)
    eta = inputs.gaussian_source(dims, 60)
    ctx = qcd.Context(dims, t_bc)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = clover_solve(Ut, bt, ctx, kappa, csw, tol=1e-12, levels=2)
    L = torch.sum(torch.conj(torch.from_numpy(eta).cuda()) * x).real
    L.backward()
    # oracle: x and lambda = D^-dag eta from dense solves
    F = oracle.clover_field(dims, U, kappa, csw)
    n = inputs.volume(dims) * 12
    D = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        D[:, k] = oracle.dirac(dims, t_bc, U, F, kappa, e.reshape(-1, 4, 3)).reshape(-1)
    xo = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    lo = np.linalg.solve(D.conj().T, eta.reshape(-1)).reshape(b.shape)
    Go = oracle.link_grad(dims, t_bc, U, kappa, csw, xo, lo)
    assert rel(x.detach().cpu().numpy(), xo) < 1e-10
    assert rel(bt.grad.cpu().numpy(), lo) < 1e-10
    assert rel(Ut.grad.cpu().numpy(), Go) < 1e-10
    ctx.close()


@pytest.mark.slow
def test_autograd_finite_differences_16c32():
    from paper_1709_08785_gb300 import qcd
    from paper_1709_08785_gb300.autograd import clover_solve

    dims, kappa, csw, t_bc = (16, 16, 16, 32), 0.12, 1.0, -1
    U = inputs.random_gauge(dims, 0.3, 6)
    eta = inputs.gaussian_source(dims, 60)
    b = inputs.gaussian_source(dims, 61)
    ctx = qcd.Context(dims, t_bc)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    etat = torch.from_numpy(eta).cuda()
    x = clover_solve(Ut, bt, ctx, kappa, csw, tol=1e-12, levels=2)
    L = torch.sum(torch.conj(etat) * x).real
    L.backward()
    G = Ut.grad.cpu().numpy()
    rng = np.random.default_rng(62)
    V = inputs.volume(dims)
    sites = rng.integers(0, V, size=32)
    mus = rng.integers(0, 4, size=32)
    T = inputs.random_su3_directions(32, 62)
    h = 1e-6
    cm, cp = qcd.Context(dims, t_bc), qcd.Context(dims, t_bc)
    U0 = torch.from_numpy(U).cuda()
    worst = 0.0
    for k in range(32):
        s, mu = int(sites[k]), int(mus[k])
        w, W = np.linalg.eigh(T[k])
        Up, Um = U0.clone(), U0.clone()
        Up[s, mu] = torch.from_numpy((W * np.exp(1j * h * w)) @ W.conj().T @ U[s, mu]).cuda()
        Um[s, mu] = torch.from_numpy((W * np.exp(-1j * h * w)) @ W.conj().T @ U[s, mu]).cuda()
        cm.gauge_load(Um)
        cm.clover_build(kappa, csw)
        cp.gauge_load(Up)
        cp.clover_build(kappa, csw)
        xm = torch.zeros_like(bt)
        cm.solve(bt.detach(), xm, tol=1e-12, precision_levels=2)
        Dp, Dm = torch.zeros_like(xm), torch.zeros_like(xm)
        cp.dirac(Dp, xm)
        cm.dirac(Dm, xm)
        r = (Dp - Dm).contiguous()
        d = torch.zeros_like(xm)
        cp.solve(r, d, tol=1e-12, precision_levels=2)
        fd = -torch.sum(torch.conj(etat) * d).real.item() / (2 * h)
        an = float(np.real(np.sum(np.conj(G[s, mu]) * (1j * T[k] @ U[s, mu]))))
        err = abs(fd - an) / max(abs(an), 1e-300)
        worst = max(worst, err)
        assert err < 1e-6, (k, fd, an)
    ctx.close()
    cm.close()
    cp.close()
