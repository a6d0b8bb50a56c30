"""qcd_dslash_eo_noalloc: the hopping term for callers that must not allocate
device memory during the call (for instance a serving loop whose allocator
is frozen after start-up).  It runs the same kernels as qcd_dslash_eo on the
same inputs, so its result must equal qcd_dslash_eo's bit for bit, call after
call, while leaving the device's free memory untouched.

Named to be collected last: if it fails, a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1709_08785_gb300 import inputs

pytestmark = pytest.mark.gpu

F64, F32, F16, DF64 = 0, 1, 2, 3


def dtype_of(prec):
    return torch.complex64 if prec in (F32, F16) else torch.complex128


def make_ctx(dims, seed):
    from paper_1709_08785_gb300 import qcd

    ctx = qcd.Context(dims, -1)
    ctx.gauge_load(torch.from_numpy(inputs.random_gauge(dims, 0.25, seed)).cuda())
    return ctx


@pytest.mark.parametrize("prec", [F64, F32, F16, DF64])
def test_noalloc_matches_dslash_eo_twice(prec):
    dims = (8, 8, 8, 16)
    Vh = inputs.volume(dims) // 2
    ctx = make_ctx(dims, 71)
    dt = dtype_of(prec)
    srcs = [torch.from_numpy(inputs.gaussian_source(dims, 72 + k)[:Vh]).to(dt).cuda() for k in range(2)]
    # the first calls are the documented set-up: they look up the scratch
    # array and let the driver load the kernels used (one per dagger value)
    warm = torch.zeros_like(srcs[0])
    for dag in (False, True):
        ctx.dslash_eo_noalloc(warm, srcs[0], 0, dag, prec)
    # two further calls in a row on a context that never staged anything:
    # no device memory is taken (outputs are allocated before the baseline)
    got = [torch.zeros_like(s) for s in srcs]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k, (par, dag) in enumerate([(0, False), (1, True)]):
        ctx.dslash_eo_noalloc(got[k], srcs[k], par, dag, prec)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # the allocating entry point on the same inputs: the same kernels, so
    # the same bits
    for k, (par, dag) in enumerate([(0, False), (1, True)]):
        want = torch.zeros_like(srcs[k])
        ctx.dslash_eo(want, srcs[k], par, dag, prec)
        torch.cuda.synchronize()
        assert np.array_equal(got[k].cpu().numpy(), want.cpu().numpy())
    ctx.close()


def test_two_contexts_share_the_array_in_stream_order():
    """Two contexts of different lattices call the entry point alternately on
    one stream: each call overwrites the shared array, and each result must
    still equal the allocating entry point's."""
    shapes = [((8, 8, 8, 16), 81), ((6, 4, 4, 10), 82)]  # the second has a ragged last 32-site block
    ctxs = [make_ctx(d, s) for d, s in shapes]
    outs, ins = [], []
    for (d, _), ctx in zip(shapes, ctxs):
        Vh = inputs.volume(d) // 2
        ins.append(torch.from_numpy(inputs.gaussian_source(d, 90 + Vh)[:Vh]).cuda())
        outs.append([torch.zeros_like(ins[-1]) for _ in range(2)])
        ctx.dslash_eo_noalloc(outs[-1][0], ins[-1], 0, False, F64)  # set-up call
    for rep in range(2):
        for k, ctx in enumerate(ctxs):
            ctx.dslash_eo_noalloc(outs[k][rep], ins[k], 1, rep == 1, F64)
    torch.cuda.synchronize()
    for k, ctx in enumerate(ctxs):
        for rep in range(2):
            want = torch.zeros_like(ins[k])
            ctx.dslash_eo(want, ins[k], 1, rep == 1, F64)
            torch.cuda.synchronize()
            assert np.array_equal(outs[k][rep].cpu().numpy(), want.cpu().numpy()), (k, rep)
    for ctx in ctxs:
        ctx.close()


@pytest.mark.parametrize("prec", [F64, DF64])
def test_noalloc_rejects_lattices_beyond_its_scratch(prec):
    from paper_1709_08785_gb300 import qcd

    dims = (16, 16, 16, 64)  # 131072 sites per parity: twice the FP64 limit
    Vh = inputs.volume(dims) // 2
    ctx = qcd.Context(dims, -1)
    ctx.gauge_load(torch.from_numpy(inputs.unit_gauge(dims)).cuda())
    v = torch.zeros((Vh, 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(v)
    with pytest.raises(qcd.QCDError) as e:
        ctx.dslash_eo_noalloc(out, v, 0, False, prec)
    assert e.value.status == -1  # QCD_EINVAL
    ctx.close()
