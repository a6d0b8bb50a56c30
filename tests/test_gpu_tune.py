"""Autotuner: tunes every solver launch configuration, writes a JSON cache
that a second context reads back without re-timing, and leaves the operator
results within the parity tolerances."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_autotune_cache_and_parity(tmp_path):
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (8, 8, 8, 16), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 91)
    cache = str(tmp_path / "tune.json")
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    entries = ctx.tune_info()
    assert len(entries) >= 15
    assert all(e["threads"] in (32, 64, 128, 256) and e["variant"] in (0, 1) for e in entries)
    assert all(e["variant"] == 0 for e in entries if e["prec"] == 0)  # no capped FP64 variant
    data = json.load(open(cache))
    assert len(data) == len(entries)
    # a second context on the same lattice reads the cache: identical choices
    ctx2 = qcd.Context(dims, t_bc)
    ctx2.gauge_load(torch.from_numpy(U).cuda())
    ctx2.clover_build(kappa, csw)
    ctx2.autotune(cache)
    got = sorted((e["key"], e["variant"], e["threads"], round(e["us"], 3)) for e in ctx2.tune_info())
    assert got == sorted((e["key"], e["variant"], e["threads"], round(e["us"], 3)) for e in entries)
    # tuned kernels still match the oracle
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 92)[:Vh]
    want = oracle.dhat(dims, t_bc, U, Fi, kappa, v)
    for prec, tol, dt in ((0, 1e-13, torch.complex128), (1, 2e-6, torch.complex64), (2, 2e-3, torch.complex64)):
        inp = torch.from_numpy(v).to(dt).cuda()
        out = torch.zeros_like(inp)
        ctx.dhat(out, inp, prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol
    b = inputs.gaussian_source(dims, 93)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    info = ctx.solve(bd, x, tol=1e-12, precision_levels=2)
    assert info["status"] == 0
    assert oracle.true_residual(dims, t_bc, U, F, kappa, b, x.cpu().numpy()) <= 1e-12
    ctx.close()
    ctx2.close()
