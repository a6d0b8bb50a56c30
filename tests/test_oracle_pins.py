"""Pins of the CPU oracle to things other than itself.

Each test checks the oracle against a closed form, an invariant, a special
case or brute force, chosen so that a plausible slip in it (a dropped term, a
wrong sign or index, a transposed operand, a wrong boundary phase) fails one
of them:

* free field (unit links): plane waves are eigenvectors with the closed-form
  spectrum, periodic and antiperiodic in time (Sec. II-A, Eqs. 3-4);
* unit links give F = 1 exactly; a constant abelian field in each of the six
  planes gives F = 1 - csw*kappa*sigma_munu (x) diag(sin theta) with
  sigma_munu typed out by hand (clover term, Sec. II-A);
* gamma5-hermiticity of H, D and the even-odd operator, gauge covariance;
* the gamma5-hermitian even-odd operator S_ee: exact gamma5-hermiticity,
  S_ee = F_ee D^_ee, its source, and a dense solve on 4^4;
* a dense brute-force matrix on a 2^4 lattice (every hop lands twice);
* the even-odd pieces: the half / full embedding by coordinate parity, the
  half-lattice hopping term as the full one restricted, MULT from D;
* the clover inverse, the even-odd identities (Eqs. 5-9), dense LU solves
  against BiCGStab (Algs. 1-2), and finite differences for the gradient.
"""
import numpy as np
import pytest

import oracle
from paper_1709_08785_gb300 import inputs

# ---- the Dirac basis typed out by hand (gamma_t diagonal, Sec. II-A)
I2 = np.eye(2)
Z2 = np.zeros((2, 2))
S1 = np.array([[0, 1], [1, 0]], dtype=complex)
S2 = np.array([[0, -1j], [1j, 0]], dtype=complex)
S3 = np.array([[1, 0], [0, -1]], dtype=complex)
G = [
    np.array([[0, 0, 0, -1j], [0, 0, -1j, 0], [0, 1j, 0, 0], [1j, 0, 0, 0]]),  # g_x
    np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex),  # g_y
    np.array([[0, 0, -1j, 0], [0, 0, 0, 1j], [1j, 0, 0, 0], [0, -1j, 0, 0]]),  # g_z
    np.diag([1, 1, -1, -1]).astype(complex),  # g_t
]
G5 = np.array([[0, 0, -1, 0], [0, 0, 0, -1], [-1, 0, 0, 0], [0, -1, 0, 0]], dtype=complex)


def blk(a, b, c, d):
    return np.block([[a, b], [c, d]])


# sigma_munu = (i/2)[g_mu, g_nu] worked out by hand in this basis:
#   sigma_jk = -eps_jkl diag(s_l, s_l),  sigma_k4 = [[0, -s_k], [-s_k, 0]]
SIGMA = {
    (0, 1): -blk(S3, Z2, Z2, S3),
    (0, 2): blk(S2, Z2, Z2, S2),
    (1, 2): -blk(S1, Z2, Z2, S1),
    (0, 3): blk(Z2, -S1, -S1, Z2),
    (1, 3): blk(Z2, -S2, -S2, Z2),
    (2, 3): blk(Z2, -S3, -S3, Z2),
}


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def coords(dims):
    V = inputs.volume(dims)
    s = np.arange(V)
    c = []
    for L in dims:
        c.append(s % L)
        s = s // L
    return np.stack(c, axis=1)  # [V, 4]


def parity(dims):
    return coords(dims).sum(axis=1) % 2


def vdot(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


def test_gamma_basis_matches_hand_typed():
    for mu in range(4):
        assert np.array_equal(oracle.gamma(mu), G[mu])
    assert np.allclose(oracle.gamma(4), G5, atol=0)
    for mu in range(4):
        for nu in range(4):
            ac = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.allclose(ac, 2 * np.eye(4) * (mu == nu))


# ------------------------------------------------------------- P1 free field
@pytest.mark.parametrize("t_bc", [1, -1])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8)])
def test_free_field_plane_waves(dims, t_bc):
    """D(p) = (1 - 2k sum cos p) + 2ik sum g_mu sin p on e^{ipn} u."""
    kappa, csw = 0.13, 1.7
    U = inputs.unit_gauge(dims)
    F = oracle.clover_field(dims, U, kappa, csw)
    rng = np.random.default_rng(7)
    c = coords(dims)
    for trial in range(4):
        m = rng.integers(0, np.array(dims))
        p = 2 * np.pi * m / np.array(dims, dtype=float)
        if t_bc == -1:
            p[3] = np.pi * (2 * m[3] + 1) / dims[3]
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (c @ p))
        psi = phase[:, None, None] * u[None]
        Dp = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(G[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (Dp @ u)[None]
        got = oracle.dirac(dims, t_bc, U, F, kappa, psi)
        assert rel(got, expect) < 1e-14
        # spectrum of D(p): 1 - 2k sum cos p +- 2ik |sin p|, each six-fold
        ev = np.linalg.eigvals(Dp)
        ev = ev[np.argsort(ev.imag)]
        s = np.sqrt((np.sin(p) ** 2).sum())
        cc = 1 - 2 * kappa * np.cos(p).sum()
        assert np.allclose(ev, [cc - 2j * kappa * s] * 2 + [cc + 2j * kappa * s] * 2, atol=1e-14)
        # even-odd operator: D^ psi_e = [(1 - k^2 H(p)^2) psi]_e
        Hp = 2 * np.cos(p).sum() * np.eye(4) - 2j * sum(G[mu] * np.sin(p[mu]) for mu in range(4))
        Finv = oracle.invert_sites(F)
        pe = oracle.full_to_half(dims, 0, psi)
        got_e = oracle.dhat(dims, t_bc, U, Finv, kappa, pe)
        want = oracle.full_to_half(dims, 0, phase[:, None, None] * ((np.eye(4) - kappa**2 * Hp @ Hp) @ u)[None])
        assert rel(got_e, want) < 1e-14
        # with F = 1 the gamma5-hermitian S_ee is the same operator
        assert rel(oracle.schur_ee(dims, t_bc, U, F, Finv, kappa, pe), want) < 1e-14


# ------------------------------------------------------------- P2, P3 clover
def test_clover_vanishes_on_unit_links():
    dims = (4, 2, 2, 4)
    F = oracle.clover_field(dims, inputs.unit_gauge(dims), 0.12, 1.9)
    assert np.max(np.abs(F - np.eye(12)[None])) < 1e-15


@pytest.mark.parametrize("plane", sorted(SIGMA))
def test_clover_constant_abelian_field(plane):
    """U_mu(n) = diag(exp(-i theta_a n_nu)), all else 1: every leaf in the
    (mu,nu) plane is diag(exp(i theta_a)), so F_munu = diag(sin theta_a), all
    other planes vanish and F = 1 - csw kappa sigma_munu (x) diag(sin theta)."""
    mu, nu = plane
    dims = (4, 4, 4, 4)
    kappa, csw = 0.124, 1.6
    k = np.array([1, 0, -1]) if nu != 1 else np.array([1, 1, -2])
    theta = 2 * np.pi * k / dims[nu]
    U = inputs.unit_gauge(dims)
    c = coords(dims)
    for a in range(3):
        U[:, mu, a, a] = np.exp(-1j * theta[a] * c[:, nu])
    F = oracle.clover_field(dims, U, kappa, csw)
    expect = np.eye(12) - csw * kappa * np.kron(SIGMA[plane], np.diag(np.sin(theta)))
    assert np.max(np.abs(F - expect[None])) < 1e-14
    # field strength itself, and its antisymmetry in (mu, nu)
    Fmn = oracle.field_strength(dims, U, 5, mu, nu)
    assert np.max(np.abs(Fmn - np.diag(np.sin(theta)))) < 1e-15
    assert np.max(np.abs(oracle.field_strength(dims, U, 5, nu, mu) + Fmn)) < 1e-15
    # the eigenvalue on spin-up (sigma_3 = +1) colour a fixes the overall sign
    if plane == (0, 1):
        e = np.zeros(12, dtype=complex)
        e[0 * 3 + 0] = 1
        assert np.allclose(F[0] @ e, (1 + csw * kappa * np.sin(theta[0])) * e)


def test_clover_is_hermitian_and_commutes_with_gamma5():
    dims = (4, 4, 2, 4)
    U = inputs.random_gauge(dims, 0.3, 11)
    F = oracle.clover_field(dims, U, 0.12, 1.3)
    assert np.max(np.abs(F - np.conj(np.swapaxes(F, 1, 2)))) < 1e-15
    g5 = np.kron(G5, np.eye(3))
    assert np.max(np.abs(g5 @ F - F @ g5)) < 1e-15
    # F - 1 is traceless over spin (sigma_munu is), so tr F = 12
    assert np.max(np.abs(np.trace(F, axis1=1, axis2=2) - 12)) < 1e-13


# ------------------------------------------------------------- P7 inverse
def test_clover_inverse():
    dims = (4, 4, 4, 2)
    U = inputs.random_gauge(dims, 0.3, 12)
    F = oracle.clover_field(dims, U, 0.124, 1.6)
    Fi = oracle.invert_sites(F)
    assert np.max(np.abs(F @ Fi - np.eye(12)[None])) < 1e-13
    assert np.max(np.abs(Fi - np.conj(np.swapaxes(Fi, 1, 2)))) < 1e-13


# ------------------------------------------------------------- P4 gamma5
@pytest.mark.parametrize("t_bc", [1, -1])
def test_gamma5_hermiticity(t_bc):
    dims = (4, 2, 4, 6)
    kappa, csw = 0.12, 1.0
    U = inputs.random_gauge(dims, 0.3, 13)
    F = oracle.clover_field(dims, U, kappa, csw)
    x = inputs.gaussian_source(dims, 14)
    y = inputs.gaussian_source(dims, 15)
    g5 = lambda v: np.einsum("ab,sbi->sai", G5, v)
    Dy = oracle.dirac(dims, t_bc, U, F, kappa, y)
    g5Dg5x = g5(oracle.dirac(dims, t_bc, U, F, kappa, g5(x)))
    assert abs(vdot(x, Dy) - vdot(g5Dg5x, y)) / abs(vdot(x, Dy)) < 1e-14
    # H^dag = gamma5 H gamma5 is what the dagger flag applies
    Hy = oracle.hopping(dims, t_bc, U, y)
    Hdx = oracle.hopping(dims, t_bc, U, x, dagger=True)
    assert abs(vdot(x, Hy) - vdot(Hdx, y)) / abs(vdot(x, Hy)) < 1e-14
    assert rel(Hdx, g5(oracle.hopping(dims, t_bc, U, g5(x)))) < 1e-15
    # even-odd: D^dag = F_ee g5 D^ g5 F_ee^-1
    Fi = oracle.invert_sites(F)
    Fe = oracle.field_to_half(dims, 0, F)
    Fie = oracle.field_to_half(dims, 0, Fi)
    xe = oracle.full_to_half(dims, 0, x)
    ye = oracle.full_to_half(dims, 0, y)
    lhs = vdot(xe, oracle.dhat(dims, t_bc, U, Fi, kappa, ye))
    w = oracle.site_apply(Fe, g5(oracle.dhat(dims, t_bc, U, Fi, kappa, g5(oracle.site_apply(Fie, xe)))))
    assert abs(lhs - vdot(w, ye)) / abs(lhs) < 1e-13


@pytest.mark.parametrize("t_bc", [1, -1])
def test_schur_operator_gamma5_hermitian_and_F_times_dhat(t_bc):
    """S_ee = F_ee - k^2 H_eo F_oo^-1 H_oe: <x, S y> = <g5 S g5 x, y>
    exactly (F commutes with g5, H^dag = g5 H g5), and S_ee = F_ee D^_ee,
    D^_ee the operator of Eq. 8 pinned above (free field, dense solves).
    The second identity fails if S applied F^-1 instead of F to p."""
    dims = (4, 2, 4, 6)
    kappa, csw = 0.124, 1.6
    U = inputs.random_gauge(dims, 0.3, 16)
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    Vh = inputs.volume(dims) // 2
    xe = inputs.gaussian_source(dims, 17)[:Vh]
    ye = inputs.gaussian_source(dims, 18)[:Vh]
    g5 = lambda v: np.einsum("ab,sbi->sai", G5, v)
    S = lambda v: oracle.schur_ee(dims, t_bc, U, F, Fi, kappa, v)
    lhs = vdot(xe, S(ye))
    assert abs(lhs - vdot(g5(S(g5(xe))), ye)) / abs(lhs) < 1e-14
    assert abs(lhs - vdot(S(xe), ye)) / abs(lhs) > 1e-3  # not Hermitian itself: the check above has teeth
    Fe = oracle.field_to_half(dims, 0, F)
    assert rel(S(ye), oracle.site_apply(Fe, oracle.dhat(dims, t_bc, U, Fi, kappa, ye))) < 1e-14
    # its source: with b = D x, S_ee x_e = b_e + k H_eo F_oo^-1 b_o
    x = inputs.gaussian_source(dims, 19)
    b = oracle.dirac(dims, t_bc, U, F, kappa, x)
    assert rel(S(oracle.full_to_half(dims, 0, x)), oracle.schur_source(dims, t_bc, U, Fi, kappa, b)) < 1e-14


# ------------------------------------------------------------- P5 covariance
def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    kappa, csw, t_bc = 0.12, 1.6, -1
    U = inputs.random_gauge(dims, 0.3, 16)
    g = inputs.random_su3(inputs.volume(dims), 17)
    V = inputs.volume(dims)
    c = coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        cc = c.copy()
        cc[:, mu] = (cc[:, mu] + 1) % dims[mu]
        nb = cc[:, 0] + dims[0] * (cc[:, 1] + dims[1] * (cc[:, 2] + dims[2] * cc[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[nb], 1, 2))
    psi = inputs.gaussian_source(dims, 18)
    Gpsi = np.einsum("sij,saj->sai", g, psi)
    F = oracle.clover_field(dims, U, kappa, csw)
    Fg = oracle.clover_field(dims, Ug, kappa, csw)
    lhs = oracle.dirac(dims, t_bc, Ug, Fg, kappa, Gpsi)
    rhs = np.einsum("sij,saj->sai", g, oracle.dirac(dims, t_bc, U, F, kappa, psi))
    assert rel(lhs, rhs) < 1e-13
    assert V == len(g)


# ------------------------------------------------------------- P6 brute force
def test_dense_brute_force_2x2x2x2():
    """Every matrix element of H from the Kronecker deltas of Eq. 4, on a
    lattice where n+mu = n-mu so both hops of a direction land together."""
    dims = (2, 2, 2, 2)
    t_bc = -1
    U = inputs.random_gauge(dims, 0.4, 19)
    V = 16
    c = coords(dims)
    Hd = np.zeros((V * 12, V * 12), dtype=complex)
    for n in range(V):
        for m in range(V):
            for mu in range(4):
                fw = c[n].copy()
                fw[mu] = (fw[mu] + 1) % dims[mu]
                bw = c[n].copy()
                bw[mu] = (bw[mu] - 1) % dims[mu]
                sign_f = t_bc if (mu == 3 and c[n][3] == dims[3] - 1) else 1
                sign_b = t_bc if (mu == 3 and c[n][3] == 0) else 1
                if np.array_equal(fw, c[m]):
                    Hd[n * 12:(n + 1) * 12, m * 12:(m + 1) * 12] += sign_f * np.kron(np.eye(4) - G[mu], U[n, mu])
                if np.array_equal(bw, c[m]):
                    Hd[n * 12:(n + 1) * 12, m * 12:(m + 1) * 12] += sign_b * np.kron(np.eye(4) + G[mu], np.conj(U[m, mu].T))
    cols = np.zeros((V * 12, V * 12), dtype=complex)
    for k in range(V * 12):
        e = np.zeros((V, 4, 3), dtype=complex)
        e.reshape(-1)[k] = 1
        cols[:, k] = oracle.hopping(dims, t_bc, U, e).reshape(-1)
    assert np.max(np.abs(cols - Hd)) < 1e-14
    # even-odd blocks: H connects only opposite parities
    par = np.repeat(parity(dims), 12)
    assert np.max(np.abs(Hd[np.ix_(par == 0, par == 0)])) == 0


# ------------------------------------------------------------- P9 Schur
@pytest.mark.parametrize("t_bc", [1, -1])
def test_even_odd_identities(t_bc):
    """With b = D x: D^ x_e = b^_e (Eqs. 5-6) and x_o = F_oo^-1 b_o + k H~_oe x_e (Eq. 7)."""
    dims = (4, 4, 2, 6)
    kappa, csw = 0.124, 1.6
    U = inputs.random_gauge(dims, 0.25, 20)
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    x = inputs.gaussian_source(dims, 21)
    b = oracle.dirac(dims, t_bc, U, F, kappa, x)
    xe = oracle.full_to_half(dims, 0, x)
    bh = oracle.eo_source(dims, t_bc, U, Fi, kappa, b)
    assert rel(oracle.dhat(dims, t_bc, U, Fi, kappa, xe), bh) < 1e-14
    assert rel(oracle.eo_reconstruct(dims, t_bc, U, Fi, kappa, b, xe), x) < 1e-14
    # the full residual restricted to the even sites is F_ee (b^_e - D^ x_e)
    ye = inputs.gaussian_source(dims, 22)[: inputs.volume(dims) // 2]
    xf = oracle.eo_reconstruct(dims, t_bc, U, Fi, kappa, b, ye)
    r = b - oracle.dirac(dims, t_bc, U, F, kappa, xf)
    assert np.max(np.abs(oracle.full_to_half(dims, 1, r))) < 1e-12
    re = oracle.site_apply(oracle.field_to_half(dims, 0, F), bh - oracle.dhat(dims, t_bc, U, Fi, kappa, ye))
    assert rel(oracle.full_to_half(dims, 0, r), re) < 1e-13


# ------------------------------------------------------------- even-odd pieces
def _parity_of_lex(dims, lex):
    """(x + y + z + t) mod 2 of lexicographic sites, x fastest (Sec. II-B)."""
    lex = np.asarray(lex)
    c, r = [], lex
    for L in dims:
        c.append(r % L)
        r = r // L
    return (c[0] + c[1] + c[2] + c[3]) % 2


@pytest.mark.parametrize("parity", [0, 1])
def test_half_full_embedding(parity):
    """A half-lattice vector lands on the sites of its parity (coordinate sum
    mod 2), in cb order, zero elsewhere, and comes back unchanged."""
    dims = (4, 2, 6, 4)
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 40 + parity)[:Vh]
    full = oracle.half_to_full(dims, parity, v)
    lex = oracle.site_of_cb(dims, parity, np.arange(Vh))
    assert np.all(_parity_of_lex(dims, lex) == parity)
    assert np.all(np.diff(lex) > 0)  # cb order is lexicographic order within the parity
    assert np.array_equal(full[lex], v)
    other = np.setdiff1d(np.arange(inputs.volume(dims)), lex)
    assert np.all(_parity_of_lex(dims, other) == 1 - parity)
    assert not np.any(full[other])
    assert np.array_equal(oracle.full_to_half(dims, parity, full), v)


@pytest.mark.parametrize("t_bc", [1, -1])
@pytest.mark.parametrize("dagger", [False, True])
def test_hop_eo_is_the_full_hopping_restricted(t_bc, dagger):
    """H_{p,1-p} on half vectors equals the full-lattice H (pinned above by the
    free field, the dense 2^4 matrix and gamma5-hermiticity) applied to the
    embedded vector and read on parity p."""
    dims = (4, 4, 2, 6)
    U = inputs.random_gauge(dims, 0.25, 42)
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 43)[:Vh]
    for p in (0, 1):
        want = oracle.full_to_half(dims, p, oracle.hopping(dims, t_bc, U, oracle.half_to_full(dims, 1 - p, v), dagger))
        assert rel(oracle.hop_eo(dims, t_bc, U, p, v, dagger), want) < 1e-15


@pytest.mark.parametrize("t_bc", [1, -1])
def test_mult_from_the_dirac_operator(t_bc):
    """MULT = F_pp^-1 H_{p,1-p} (Sec. II-B): for v on parity 1-p only, the
    Dirac operator gives (D v)_p = -kappa (H v)_p (F is site-diagonal), so
    MULT v = -F_pp^-1 (D v)_p / kappa, with D and F^-1 pinned above."""
    dims = (4, 2, 4, 6)
    kappa, csw = 0.124, 1.6
    U = inputs.random_gauge(dims, 0.25, 44)
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 45)[:Vh]
    for p in (0, 1):
        dv = oracle.dirac(dims, t_bc, U, F, kappa, oracle.half_to_full(dims, 1 - p, v))
        want = -oracle.site_apply(oracle.field_to_half(dims, p, Fi), oracle.full_to_half(dims, p, dv)) / kappa
        assert rel(oracle.mult(dims, t_bc, U, Fi, p, v), want) < 1e-14


# ------------------------------------------------------------- P8 solvers
@pytest.fixture(scope="module")
def c1_problem():
    """The 4^4 workload: links exp(i 0.3 H) seed 1, kappa 0.12, csw 1.0,
    antiperiodic in time, Gaussian source seed 2, and its dense LU solution."""
    dims = (4, 4, 4, 4)
    kappa, csw, t_bc = 0.12, 1.0, -1
    U = inputs.random_gauge(dims, 0.3, 1)
    b = inputs.gaussian_source(dims, 2)
    F = oracle.clover_field(dims, U, kappa, csw)
    n = inputs.volume(dims) * 12
    D = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        D[:, k] = oracle.dirac(dims, t_bc, U, F, kappa, e.reshape(-1, 4, 3)).reshape(-1)
    xd = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    return dict(dims=dims, kappa=kappa, csw=csw, t_bc=t_bc, U=U, b=b, F=F, Fi=oracle.invert_sites(F), xd=xd)


def test_bicgstab_full_matches_dense_solve(c1_problem):
    P = c1_problem
    x, st, it = oracle.bicgstab_full(P["dims"], P["t_bc"], P["U"], P["F"], P["kappa"], P["b"], 1e-12)
    assert st == 0 and it > 5
    assert oracle.true_residual(P["dims"], P["t_bc"], P["U"], P["F"], P["kappa"], P["b"], x) <= 1e-12
    assert rel(x, P["xd"]) < 1e-10


def test_bicgstab_eo_matches_dense_solve(c1_problem):
    P = c1_problem
    x, st, it = oracle.bicgstab_eo(P["dims"], P["t_bc"], P["U"], P["Fi"], P["kappa"], P["b"], 1e-13)
    assert st == 0
    assert oracle.true_residual(P["dims"], P["t_bc"], P["U"], P["F"], P["kappa"], P["b"], x) <= 1e-12
    assert rel(x, P["xd"]) < 1e-10


def test_nested_bicgstab_matches_dense_solve(c1_problem):
    P = c1_problem
    x, st, outer, inner = oracle.nested_bicgstab(P["dims"], P["t_bc"], P["U"], P["Fi"], P["kappa"], P["b"], 1e-13, 1e-5)
    assert st == 0 and 1 <= outer <= 6 and inner > 0
    assert oracle.true_residual(P["dims"], P["t_bc"], P["U"], P["F"], P["kappa"], P["b"], x) <= 1e-12
    assert rel(x, P["xd"]) < 1e-10


def test_schur_solve_matches_dense_solve(c1_problem):
    """BiCGStab on S_ee against the dense LU solve of D, and the dense S_ee
    (built column by column) against gamma5-hermiticity and its own solve."""
    P = c1_problem
    dims, t_bc, kappa = P["dims"], P["t_bc"], P["kappa"]
    x, st, it = oracle.bicgstab_schur(dims, t_bc, P["U"], P["F"], P["Fi"], kappa, P["b"], 1e-13)
    assert st == 0 and it > 5
    assert oracle.true_residual(dims, t_bc, P["U"], P["F"], kappa, P["b"], x) <= 1e-12
    assert rel(x, P["xd"]) < 1e-10
    n = inputs.volume(dims) // 2 * 12
    Sd = np.zeros((n, n), dtype=complex)
    for k in range(n):
        e = np.zeros(n, dtype=complex)
        e[k] = 1
        Sd[:, k] = oracle.schur_ee(dims, t_bc, P["U"], P["F"], P["Fi"], kappa, e.reshape(-1, 4, 3)).reshape(-1)
    G5h = np.kron(np.eye(n // 12), np.kron(G5, np.eye(3)))
    assert rel(Sd.conj().T, G5h @ Sd @ G5h) < 1e-14
    src = oracle.schur_source(dims, t_bc, P["U"], P["Fi"], kappa, P["b"]).reshape(-1)
    xe = np.linalg.solve(Sd, src).reshape(-1, 4, 3)
    assert rel(xe, oracle.full_to_half(dims, 0, P["xd"])) < 1e-10


# ------------------------------------------------------------- sampled sites
def test_sampled_site_helpers_match_the_full_lattice():
    """The per-site entry points used for the full-size checks agree with the
    full-lattice functions (same definitions, evaluated at chosen sites)."""
    dims, t_bc, kappa, csw = (4, 2, 4, 6), -1, 0.12, 1.3
    U = inputs.random_gauge(dims, 0.3, 40)
    psi = inputs.gaussian_source(dims, 41)
    sites = np.array([0, 5, 17, 63, 95, 191])
    assert np.array_equal(oracle.hop_sites(dims, t_bc, U, psi, sites), oracle.hopping(dims, t_bc, U, psi)[sites])
    F = oracle.clover_field(dims, U, kappa, csw)
    assert np.array_equal(oracle.clover_sites(dims, U, kappa, csw, sites), F[sites])
    Dx = oracle.dirac(dims, t_bc, U, F, kappa, psi)
    assert np.max(np.abs(oracle.dirac_sites(dims, t_bc, U, kappa, csw, psi, sites) - Dx[sites])) < 1e-13
    for par in (0, 1):
        half = oracle.full_to_half(dims, par, psi)
        cbs = np.arange(inputs.volume(dims) // 2)
        assert np.array_equal(psi[oracle.site_of_cb(dims, par, cbs)], half)


# ------------------------------------------------------------- pion correlator
def test_pion_correlator_brute_force():
    dims = (2, 2, 2, 4)
    V = inputs.volume(dims)
    rng = np.random.default_rng(31)
    S = rng.standard_normal((3, V, 4, 3)) + 1j * rng.standard_normal((3, V, 4, 3))
    want = np.zeros(dims[3])
    for col in range(3):
        for site in range(V):
            t = site // (dims[0] * dims[1] * dims[2])
            for sp in range(4):
                for c in range(3):
                    want[t] += abs(S[col, site, sp, c]) ** 2
    assert rel(oracle.pion_correlator(dims, S), want) < 1e-14


def test_pion_correlator_free_field_closed_form():
    """Unit links, antiperiodic time: the oracle's 12 point-source solutions
    give the pion correlator of the free propagator, which follows from the
    closed-form D(p) = (1 - 2k sum cos p) + 2ik sum g_mu sin p_mu: S(x) is
    the inverse Fourier transform of D(p)^-1 (x) 1_colour, so
    C(t) = 3 sum_xvec ||S_spin(xvec, t)||^2 with S_spin from an FFT over the
    momentum grid (p_t = pi (2n + 1) / Lt; the half-step shift is a phase)."""
    dims, kappa, t_bc = (2, 4, 4, 6), 0.12, -1
    U = inputs.unit_gauge(dims)
    F = oracle.clover_field(dims, U, kappa, 1.3)
    # dense D from the oracle's operator (BiCGStab from r~ = r0 = a point
    # source breaks down exactly on the free field: rho vanishes by symmetry)
    N = inputs.volume(dims) * 12
    Dm = np.empty((N, N), dtype=complex)
    e = np.zeros(N, dtype=complex)
    for k in range(N):
        e[k] = 1.0
        Dm[:, k] = oracle.dirac(dims, t_bc, U, F, kappa, e.reshape(-1, 4, 3)).ravel()
        e[k] = 0.0
    B = inputs.point_sources(dims).reshape(12, N).T
    cols = np.linalg.solve(Dm, B).T.reshape(12, -1, 4, 3)
    got = oracle.pion_correlator(dims, cols)
    n = [np.arange(L) for L in dims]
    px, py, pz, pt = np.meshgrid(*[2 * np.pi * k / L for k, L in zip(n, dims)], indexing="ij")
    pt = pt + np.pi / dims[3]
    p = [px, py, pz, pt]
    Dp = (1 - 2 * kappa * sum(np.cos(q) for q in p))[..., None, None] * np.eye(4)
    Dp = Dp + 2j * kappa * sum(np.sin(p[mu])[..., None, None] * G[mu] for mu in range(4))
    Ssp = np.fft.ifftn(np.linalg.inv(Dp), axes=(0, 1, 2, 3))  # [x, y, z, t, 4, 4]
    want = 3 * (np.abs(Ssp) ** 2).sum(axis=(0, 1, 2, 4, 5))
    assert rel(got, want) < 1e-12
    assert np.allclose(want[1:], want[1:][::-1], rtol=1e-12)  # time reflection of the free correlator


# ------------------------------------------------------------- P12 gradient
def test_link_gradient_finite_differences():
    """dF/dh along U_l -> exp(i h T) U_l, by central differences of the
    oracle's own D, against Re sum conj(G) (i T U_l)."""
    dims = (4, 4, 4, 4)
    kappa, csw, t_bc = 0.12, 1.3, -1
    U = inputs.random_gauge(dims, 0.4, 30)
    x = inputs.gaussian_source(dims, 31)
    lam = inputs.gaussian_source(dims, 32)
    G_or = oracle.link_grad(dims, t_bc, U, kappa, csw, x, lam)

    def f(Uv):
        F = oracle.clover_field(dims, Uv, kappa, csw)
        return -np.real(vdot(lam, oracle.dirac(dims, t_bc, Uv, F, kappa, x)))

    rng = np.random.default_rng(33)
    T = inputs.random_su3_directions(16, 34)
    h = 1e-5
    for k in range(16):
        s = int(rng.integers(0, inputs.volume(dims)))
        mu = int(rng.integers(0, 4))
        w, W = np.linalg.eigh(T[k])
        Up, Um = U.copy(), U.copy()
        Up[s, mu] = (W * np.exp(1j * h * w)) @ W.conj().T @ U[s, mu]
        Um[s, mu] = (W * np.exp(-1j * h * w)) @ W.conj().T @ U[s, mu]
        fd = (f(Up) - f(Um)) / (2 * h)
        an = np.real(np.sum(np.conj(G_or[s, mu]) * (1j * T[k] @ U[s, mu])))
        assert abs(fd - an) <= 1e-8 * max(1.0, abs(an)), (k, fd, an)
