"""GPU parity of the operator kernels against the CPU oracle, through the C ABI.

Tolerances (relative L2 against the oracle applied to the FP64 inputs):
FP64 1e-13, FP32 2e-6, FP16 storage 2e-3.  Lattices span several thread
blocks and a ragged tail (Vh not a multiple of the 32-site layout block nor
of the 128-thread block), both time boundary conditions, and L = 2
directions where both hops of a direction land on one neighbour.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 2e-3, 3: 1e-13}  # 3: DF64 (float pairs, complex128 buffers)
LATTICES = [
    # dims, t_bc, eps, kappa, csw
    ((4, 4, 4, 4), -1, 0.3, 0.12, 1.0),
    ((6, 2, 4, 10), 1, 0.25, 0.124, 1.6),   # Vh = 240: ragged 32-site and 128-thread tails
    ((8, 8, 8, 16), -1, 0.25, 0.124, 1.6),  # 32 thread blocks
    ((2, 2, 2, 2), -1, 0.4, 0.11, 1.3),     # every hop lands twice
]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module", params=LATTICES, ids=lambda p: "x".join(map(str, p[0])) + ("ap" if p[1] < 0 else "p"))
def lat(request):
    from paper_1709_08785_gb300 import qcd

    dims, t_bc, eps, kappa, csw = request.param
    U = inputs.random_gauge(dims, eps, 41)
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    yield dict(dims=dims, t_bc=t_bc, kappa=kappa, csw=csw, U=U, F=F, Fi=Fi, ctx=ctx, qcd=qcd)
    ctx.close()


def dev(a, prec):
    dt = np.complex128 if prec in (0, 3) else np.complex64
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def run(fn, a, prec, nrhs=1):
    inp = dev(a, prec)
    out = torch.zeros_like(inp)
    fn(out, inp, prec, nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("out_parity", [0, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_eo(lat, prec, out_parity, dagger):
    Vh = inputs.volume(lat["dims"]) // 2
    v = inputs.gaussian_source(lat["dims"], 50)[:Vh]
    want = oracle.hop_eo(lat["dims"], lat["t_bc"], lat["U"], out_parity, v, dagger)
    got = run(lambda o, i, p, n: lat["ctx"].dslash_eo(o, i, out_parity, dagger, p, n), v, prec)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("inverse", [False, True])
def test_clover_apply(lat, prec, parity, inverse):
    dims = lat["dims"]
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 51)[:Vh]
    M = oracle.field_to_half(dims, parity, lat["Fi"] if inverse else lat["F"])
    want = oracle.site_apply(M, v)
    got = run(lambda o, i, p, n: lat["ctx"].clover_apply(o, i, parity, inverse, p, n), v, prec)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_mult(lat, prec, out_parity):
    dims = lat["dims"]
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 52)[:Vh]
    want = oracle.mult(dims, lat["t_bc"], lat["U"], lat["Fi"], out_parity, v)
    got = run(lambda o, i, p, n: lat["ctx"].mult_eo(o, i, out_parity, False, p, n), v, prec)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_dhat(lat, prec):
    dims = lat["dims"]
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 53)[:Vh]
    want = oracle.dhat(dims, lat["t_bc"], lat["U"], lat["Fi"], lat["kappa"], v)
    got = run(lambda o, i, p, n: lat["ctx"].dhat(o, i, p, n), v, prec)
    assert rel(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_schur_ee(lat, prec, nrhs):
    """The gamma5-hermitian even-odd operator S_ee = F_ee - k^2 H_eo F_oo^-1 H_oe
    (second half with the clover term F, not its inverse)."""
    dims = lat["dims"]
    Vh = inputs.volume(dims) // 2
    vs = np.stack([inputs.gaussian_source(dims, 56 + k)[:Vh] for k in range(nrhs)])
    got = run(lambda o, i, p, n: lat["ctx"].schur_ee(o, i, p, n), vs if nrhs > 1 else vs[0], prec, nrhs)
    got = got.reshape(nrhs, Vh, 4, 3)
    for k in range(nrhs):
        want = oracle.schur_ee(dims, lat["t_bc"], lat["U"], lat["F"], lat["Fi"], lat["kappa"], vs[k])
        assert rel(got[k], want) < TOL[prec]


def test_dirac_full(lat):
    dims = lat["dims"]
    v = inputs.gaussian_source(dims, 54)
    want = oracle.dirac(dims, lat["t_bc"], lat["U"], lat["F"], lat["kappa"], v)
    inp = dev(v, 0)
    out = torch.zeros_like(inp)
    lat["ctx"].dirac(out, inp)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), want) < TOL[0]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("nrhs", [3, 12, 16])
def test_multi_rhs_matches_single(lat, prec, nrhs):
    """Each column of a multi-RHS launch equals the single-RHS result (bit
    for bit: same kernel arithmetic) and the oracle."""
    dims = lat["dims"]
    Vh = inputs.volume(dims) // 2
    vs = np.stack([inputs.gaussian_source(dims, 60 + k)[:Vh] for k in range(nrhs)])
    got = run(lambda o, i, p, n: lat["ctx"].mult_eo(o, i, 1, False, p, n), vs, prec, nrhs)
    for k in range(nrhs):
        single = run(lambda o, i, p, n: lat["ctx"].mult_eo(o, i, 1, False, p, n), vs[k], prec)
        assert np.array_equal(got[k], single)
        want = oracle.mult(dims, lat["t_bc"], lat["U"], lat["Fi"], 1, vs[k])
        assert rel(got[k], want) < TOL[prec]


def test_repeatable_bitwise(lat):
    dims = lat["dims"]
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 55)[:Vh]
    a = run(lambda o, i, p, n: lat["ctx"].dhat(o, i, p, n), v, 1)
    b = run(lambda o, i, p, n: lat["ctx"].dhat(o, i, p, n), v, 1)
    assert np.array_equal(a, b)
