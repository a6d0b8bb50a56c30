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
    def mrhs(e):  # the staged multi-RHS kernel: FP32 hopping / MULT, several RHS
        return e["prec"] == 1 and e["nrhs"] > 1 and e["red"] == 0 and e["mode"] in (0, 1)

    def piped(e):  # FP32 / FP16 single-RHS MULT and D^ halves: also the pipelined-hop kernel
        return e["prec"] in (1, 2) and e["nrhs"] == 1 and e["mode"] in (1, 2, 4)

    for e in entries:
        assert e["variant"] in ((0, 1, 2) if piped(e) else (0, 1))
        if mrhs(e):  # threads = right-hand sides per block, a divisor of nrhs
            assert e["nrhs"] % e["threads"] == 0
        else:
            assert e["threads"] in (32, 64, 128, 256)
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


@pytest.mark.parametrize("cap", [1, 2])
def test_forced_launch_shapes_keep_parity(tmp_path, cap):
    """Every tuned entry rewritten to 64 (32 with several right-hand sides)
    sites per block and, where it exists, the capped register budget (cap 1)
    or, for the FP32 / FP16 MULT and D^ halves, the pipelined-hop kernel
    (cap 2; the 80 / 128 cap elsewhere), and the multi-RHS kernel to a tile
    of 4 right-hand sides;
    a context that reads that cache runs those shapes, and the operators and
    a solve still match the oracle."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (6, 2, 4, 10), 0.124, 1.6, -1  # Vh = 240: ragged blocks
    U = inputs.random_gauge(dims, 0.25, 94)
    cache = str(tmp_path / "tune.json")
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    data = json.load(open(cache))
    for k, (variant, bx, us) in list(data.items()):
        key = int(k.rsplit("|", 1)[1])
        prec, mode, red, nrhs = key & 3, (key >> 2) & 7, (key >> 5) & 3, key >> 8
        if prec == 1 and nrhs > 1 and red == 0 and mode in (0, 1):  # multi-RHS kernel, tile 4
            data[k] = [{1: 1, 2: 0}[cap], 4, us]
        elif prec in (1, 2) and nrhs == 1 and mode in (1, 2, 4):
            data[k] = [cap, 64, us]
        else:
            data[k] = [0 if prec == 0 else 1, 64 if nrhs == 1 else 32, us]
    # the cache's own layout: one entry per line
    with open(cache, "w") as f:
        f.write("{\n" + ",\n".join('  "%s": [%d, %d, %.3f]' % (k, *e) for k, e in data.items()) + "\n}\n")
    ctx.close()
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    assert all(e["threads"] in (4, 32, 64) for e in ctx.tune_info())
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    Vh = inputs.volume(dims) // 2
    v = inputs.gaussian_source(dims, 95)[:Vh]
    want = oracle.dhat(dims, t_bc, U, Fi, kappa, v)
    for prec, tol, dt in ((0, 1e-13, torch.complex128), (1, 2e-6, torch.complex64), (2, 2e-3, torch.complex64),
                          (3, 1e-13, torch.complex128)):
        inp = torch.from_numpy(v).to(dt).cuda()
        out = torch.zeros_like(inp)
        ctx.dhat(out, inp, prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol, prec
    want = oracle.schur_ee(dims, t_bc, U, F, Fi, kappa, v)
    for prec, tol, dt in ((1, 2e-6, torch.complex64), (2, 2e-3, torch.complex64)):
        inp = torch.from_numpy(v).to(dt).cuda()
        out = torch.zeros_like(inp)
        ctx.schur_ee(out, inp, prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < tol, prec
    # 12 right-hand sides through the tiled kernel, against single-RHS oracle MULTs
    vs = np.stack([inputs.gaussian_source(dims, 96 + k)[:Vh] for k in range(12)])
    inp = torch.from_numpy(vs).to(torch.complex64).cuda()
    out = torch.zeros_like(inp)
    ctx.mult_eo(out, inp, 1, False, 1, 12)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.complex128)
    for k in range(12):
        wk = oracle.mult(dims, t_bc, U, Fi, 1, vs[k])
        assert np.linalg.norm(got[k] - wk) / np.linalg.norm(wk) < 2e-6, k
    b = inputs.gaussian_source(dims, 97)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    for levels, herm in ((2, 0), (3, 0), (2, 1)):
        info = ctx.solve(bd, x, tol=1e-12, precision_levels=levels, eo_hermitian=herm)
        assert info["status"] == 0
        assert oracle.true_residual(dims, t_bc, U, F, kappa, b, x.cpu().numpy()) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("tile", [12, 4])
def test_multi_rhs_variants_bit_exact(tmp_path, variant, tile):
    """The multi-RHS kernel with and without the register cap (variants 0, 1),
    at a tile of 12 and of 4 right-hand sides: every right-hand
    side of the FP32 MULT and hopping term, plain and daggered, equals the
    single-RHS kernel's result to the bit, on a lattice with a ragged last
    site block, and the MULT matches the oracle."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (6, 2, 4, 10), 0.124, 1.6, -1  # Vh = 240: ragged blocks
    U = inputs.random_gauge(dims, 0.25, 98)
    cache = str(tmp_path / "tune.json")
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    data = json.load(open(cache))
    forced = 0
    for k, (v, bx, us) in list(data.items()):
        key = int(k.rsplit("|", 1)[1])
        prec, mode, red, nrhs = key & 3, (key >> 2) & 7, (key >> 5) & 3, key >> 8
        if prec == 1 and nrhs == 12 and red == 0 and mode in (0, 1):
            data[k] = [variant, tile, us]
            forced += 1
    assert forced == 2  # the hopping term and the MULT
    with open(cache, "w") as f:  # the cache's own layout: one entry per line
        f.write("{\n" + ",\n".join('  "%s": [%d, %d, %.3f]' % (k, *e) for k, e in data.items()) + "\n}\n")
    ctx.close()
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    got_v = {(e["mode"], e["variant"], e["threads"]) for e in ctx.tune_info() if e["nrhs"] == 12 and e["prec"] == 1}
    assert got_v == {(0, variant, tile), (1, variant, tile)}
    F = oracle.clover_field(dims, U, kappa, csw)
    Fi = oracle.invert_sites(F)
    Vh = inputs.volume(dims) // 2
    vs = np.stack([inputs.gaussian_source(dims, 100 + k)[:Vh] for k in range(12)])
    inp = torch.from_numpy(vs).to(torch.complex64).cuda()

    def launch(fn, x, n):
        out = torch.zeros_like(x)
        fn(out, x, n)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    for dag in (False, True):
        for op in ("mult_eo", "dslash_eo"):
            f = getattr(ctx, op)
            many = launch(lambda o, x, n: f(o, x, 1, dag, 1, n), inp, 12)
            for k in range(12):
                one = launch(lambda o, x, n: f(o, x, 1, dag, 1, n), inp[k].contiguous(), 1)
                assert np.array_equal(many[k], one), (op, dag, k)
                if op == "mult_eo" and not dag:
                    wk = oracle.mult(dims, t_bc, U, Fi, 1, vs[k])
                    gk = many[k].astype(np.complex128)
                    assert np.linalg.norm(gk - wk) / np.linalg.norm(wk) < 2e-6, k
    ctx.close()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("tile", [12, 4])
def test_multi_rhs_resident_loop_bit_exact(tmp_path, variant, tile):
    """The multi-RHS kernel's resident blocks walk several site blocks each
    (16^3x32: 2048 site blocks, two blocks per SM), copying the next one in
    while they compute: every right-hand side of the FP32 MULT and hopping
    term, plain and daggered, equals the single-RHS kernel's result to the
    bit, and the MULT of the first matches the oracle at sampled sites."""
    from paper_1709_08785_gb300 import qcd

    dims, kappa, csw, t_bc = (16, 16, 16, 32), 0.124, 1.6, -1
    U = inputs.random_gauge(dims, 0.25, 99)
    cache = str(tmp_path / "tune.json")
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    data = json.load(open(cache))
    for k, (v, bx, us) in list(data.items()):
        key = int(k.rsplit("|", 1)[1])
        prec, mode, red, nrhs = key & 3, (key >> 2) & 7, (key >> 5) & 3, key >> 8
        if prec == 1 and nrhs == 12 and red == 0 and mode in (0, 1):
            data[k] = [variant, tile, us]
    with open(cache, "w") as f:  # the cache's own layout: one entry per line
        f.write("{\n" + ",\n".join('  "%s": [%d, %d, %.3f]' % (k, *e) for k, e in data.items()) + "\n}\n")
    ctx.close()
    ctx = qcd.Context(dims, t_bc)
    ctx.gauge_load(torch.from_numpy(U).cuda())
    ctx.clover_build(kappa, csw)
    ctx.autotune(cache)
    got_v = {(e["mode"], e["variant"], e["threads"]) for e in ctx.tune_info() if e["nrhs"] == 12 and e["prec"] == 1}
    assert got_v == {(0, variant, tile), (1, variant, tile)}
    Vh = inputs.volume(dims) // 2
    assert Vh // 32 > 2 * 152 * 2  # several site blocks per resident block
    vs = np.stack([inputs.gaussian_source(dims, 110 + k)[:Vh] for k in range(12)])
    inp = torch.from_numpy(vs).to(torch.complex64).cuda()

    def launch(fn, x, n):
        out = torch.zeros_like(x)
        fn(out, x, n)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    for dag in (False, True):
        for op in ("mult_eo", "dslash_eo"):
            f = getattr(ctx, op)
            many = launch(lambda o, x, n: f(o, x, 1, dag, 1, n), inp, 12)
            for k in range(12):
                one = launch(lambda o, x, n: f(o, x, 1, dag, 1, n), inp[k].contiguous(), 1)
                assert np.array_equal(many[k], one), (op, dag, k)
            if op == "mult_eo" and not dag:
                rng = np.random.default_rng(7)
                cbs = np.concatenate([rng.choice(Vh - 64, 56, replace=False), np.arange(Vh - 8, Vh)])
                v_full = oracle.half_to_full(dims, 0, vs[0])
                sites = oracle.site_of_cb(dims, 1, cbs)
                h = oracle.hop_sites(dims, t_bc, U, v_full, sites)
                F = oracle.clover_sites(dims, U, kappa, csw, sites)
                want = np.linalg.solve(F, h.reshape(len(cbs), 12, 1)).reshape(len(cbs), 4, 3)
                got = many[0].reshape(Vh, 4, 3)[cbs].astype(np.complex128)
                assert np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel()) < 2e-6
    ctx.close()
