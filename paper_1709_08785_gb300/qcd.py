"""Thin Python binding of the C ABI in include/qcd.h.

Argument marshalling only: every operation runs in the CUDA library
(_build/libqcd_gb300.so, built from csrc/ by build.py).  Device buffers are
torch CUDA tensors (their data_ptr is passed); host buffers may be numpy
arrays or CPU tensors where the C call accepts host memory.  There is no
CPU fallback: without the library or a GPU every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

F64, F32, F16, DF64 = 0, 1, 2, 3
K_MULT_F64, K_MULT_F32, K_MULT_F16, K_BLAS, K_OTHER, K_DHAT_F32, K_MULT_DF64, K_BLAS_F32, K_INNER_ITER = range(9)

STATUS = {
    0: "QCD_OK", -1: "QCD_EINVAL", -2: "QCD_ECUDA", -3: "QCD_ENOMEM", -4: "QCD_ENOTCONV",
    -5: "QCD_EBREAKDOWN", -6: "QCD_ENONFINITE", -7: "QCD_ECLOVER_SINGULAR", -8: "QCD_ETIMEOUT",
    -9: "QCD_ESTATE",
}


class QCDError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("precision_levels", ctypes.c_int),
        ("even_odd", ctypes.c_int),
        ("inner_tol", ctypes.c_double * 2),
        ("max_outer", ctypes.c_int),
        ("max_inner", ctypes.c_int * 2),
        ("max_restarts", ctypes.c_int),
        ("use_x0", ctypes.c_int),
        ("outer_df64", ctypes.c_int),
        ("eo_hermitian", ctypes.c_int),
    ]


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("outer_iters", ctypes.c_int),
        ("inner_iters", ctypes.c_int * 2),
        ("restarts", ctypes.c_int),
        ("dhat_applies", ctypes.c_long * 3),
        ("true_resid", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]

    def as_dict(self):
        return dict(status=self.status, outer_iters=self.outer_iters, inner_iters=list(self.inner_iters),
                    restarts=self.restarts, dhat_applies=list(self.dhat_applies), true_resid=self.true_resid,
                    seconds=self.seconds)


class KernelStat(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_long), ("ms", ctypes.c_double), ("bytes", ctypes.c_double)]


EXPORTS = [
    "qcd_create", "qcd_destroy", "qcd_set_stream", "qcd_gauge_load", "qcd_clover_build", "qcd_dslash_eo",
    "qcd_clover_apply", "qcd_mult_eo", "qcd_dhat", "qcd_dirac", "qcd_solve_opts_default", "qcd_solve",
    "qcd_set_profiling", "qcd_kernel_stats", "qcd_reset_kernel_stats", "qcd_strerror", "qcd_last_error",
    "qcd_volume", "qcd_launch_count", "qcd_mult_benchmark", "qcd_mult_throughput", "qcd_dslash_eo_noalloc",
    "qcd_solve_adjoint", "qcd_force", "qcd_autotune", "qcd_tune_info", "qcd_solve_batched", "qcd_set_wait_limit",
    "qcd_set_graphs", "qcd_pion_correlator", "qcd_schur_ee", "qcd_solve_multi",
]

_lib = None


def library_path() -> str:
    from . import build as _b
    return _b.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the CUDA library, building it first if it is missing or stale
    and nvcc is available.  Raises if it cannot be had."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _b
    path = _b.LIB
    if build_if_missing and not _b.up_to_date():
        path = _b.build()
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s is missing; run paper_1709_08785_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.qcd_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int), ip, vp]
    lib.qcd_destroy.argtypes = [vp]
    lib.qcd_set_stream.argtypes = [vp, vp]
    lib.qcd_gauge_load.argtypes = [vp, vp, ip]
    lib.qcd_clover_build.argtypes = [vp, dp, dp]
    lib.qcd_dslash_eo.argtypes = [vp, vp, vp, ip, ip, ip, ip]
    lib.qcd_clover_apply.argtypes = [vp, vp, vp, ip, ip, ip, ip]
    lib.qcd_mult_eo.argtypes = [vp, vp, vp, ip, ip, ip, ip]
    lib.qcd_dhat.argtypes = [vp, vp, vp, ip, ip]
    lib.qcd_schur_ee.argtypes = [vp, vp, vp, ip, ip]
    lib.qcd_dirac.argtypes = [vp, vp, vp]
    lib.qcd_solve_opts_default.argtypes = [ctypes.POINTER(SolveOpts)]
    lib.qcd_solve_opts_default.restype = None
    lib.qcd_solve.argtypes = [vp, vp, vp, dp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]
    lib.qcd_solve_multi.argtypes = [vp, vp, vp, ip, dp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]
    lib.qcd_set_profiling.argtypes = [vp, ip]
    lib.qcd_kernel_stats.argtypes = [vp, ip, ctypes.POINTER(KernelStat)]
    lib.qcd_reset_kernel_stats.argtypes = [vp]
    lib.qcd_strerror.argtypes = [ip]
    lib.qcd_strerror.restype = ctypes.c_char_p
    lib.qcd_last_error.restype = ctypes.c_char_p
    lib.qcd_volume.argtypes = [vp]
    lib.qcd_volume.restype = ctypes.c_long
    lib.qcd_launch_count.argtypes = [vp]
    lib.qcd_launch_count.restype = ctypes.c_long
    lib.qcd_dslash_eo_noalloc.argtypes = [vp, vp, vp, ip, ip, ip]
    lib.qcd_mult_benchmark.argtypes = [vp, ip, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp)]
    lib.qcd_mult_throughput.argtypes = [vp, ip, ip, ip, ctypes.POINTER(dp), ctypes.POINTER(dp)]
    lib.qcd_solve_adjoint.argtypes = [vp, vp, vp, dp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]
    lib.qcd_force.argtypes = [vp, vp, vp, vp, vp]
    lib.qcd_solve_batched.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.POINTER(dp), ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]
    lib.qcd_set_wait_limit.argtypes = [ctypes.c_longlong]
    lib.qcd_set_graphs.argtypes = [ip]
    lib.qcd_pion_correlator.argtypes = [vp, vp, ip, ip, ctypes.POINTER(dp)]
    lib.qcd_autotune.argtypes = [vp, ctypes.c_char_p]
    lib.qcd_tune_info.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ip), ctypes.POINTER(ip),
                                  ctypes.POINTER(dp)]
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise QCDError(rc, _lib.qcd_last_error().decode())


def _ptr(t) -> int:
    """Device or host address of a torch tensor or numpy array (contiguous)."""
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return t.data_ptr()
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("buffer must be C-contiguous")
    return t.ctypes.data


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def default_opts(**kw) -> SolveOpts:
    lib = load_library()
    o = SolveOpts()
    lib.qcd_solve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k in ("inner_tol", "max_inner"):
            seq = list(v) if hasattr(v, "__len__") else [v, getattr(o, k)[1]]
            for i, vi in enumerate(seq[:2]):
                getattr(o, k)[i] = vi
        else:
            setattr(o, k, int(v) if isinstance(getattr(o, k), int) else v)
    return o


def solve_batched(ctxs, bs, xs, tols, opts: SolveOpts | None = None, check: bool = True, **kw) -> list:
    """Solve problem i on ctxs[i] (b = bs[i], x = xs[i], device tensors) for all
    i in one batched persistent-kernel run; returns one info dict per problem."""
    lib = load_library()
    n = len(ctxs)
    if opts is None:
        opts = default_opts(**kw)
    H = (ctypes.c_void_p * n)(*[c._h.value for c in ctxs])
    B = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    T = (ctypes.c_double * n)(*[float(t) for t in tols])
    infos = (SolveInfo * n)()
    rc = lib.qcd_solve_batched(H, n, B, X, T, ctypes.byref(opts), infos)
    if check:
        _check(rc)
    out = [infos[i].as_dict() for i in range(n)]
    for d in out:
        d["rc"] = rc
    return out


def set_wait_limit(spins: int):
    _check(load_library().qcd_set_wait_limit(int(spins)))


def set_graphs(on: bool):
    _check(load_library().qcd_set_graphs(int(on)))


class Context:
    """One lattice, its gauge field and clover term on the current device."""

    def __init__(self, dims, t_bc: int = -1, stream=None):
        self.lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        self.V = 1
        for d in self.dims:
            self.V *= d
        self.Vh = self.V // 2
        self._h = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        _check(self.lib.qcd_create(ctypes.byref(self._h), arr, int(t_bc), _stream_handle(stream)))

    def close(self):
        if self._h:
            self.lib.qcd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(self.lib.qcd_set_stream(self._h, _stream_handle(stream)))

    # ---- fields
    def gauge_load(self, U):
        on_dev = int(hasattr(U, "is_cuda") and U.is_cuda)
        _check(self.lib.qcd_gauge_load(self._h, _ptr(U), on_dev))

    def clover_build(self, kappa: float, csw: float):
        _check(self.lib.qcd_clover_build(self._h, float(kappa), float(csw)))

    # ---- operators (device buffers)
    def dslash_eo(self, out, inp, out_parity: int, dagger: bool = False, prec: int = F64, nrhs: int = 1):
        _check(self.lib.qcd_dslash_eo(self._h, _ptr(out), _ptr(inp), int(out_parity), int(dagger), int(prec), int(nrhs)))

    def dslash_eo_noalloc(self, out, inp, out_parity: int, dagger: bool = False, prec: int = F64):
        """dslash_eo that allocates no device memory during the call (staging
        in a fixed 24 MiB array inside the library; small lattices only)."""
        _check(self.lib.qcd_dslash_eo_noalloc(self._h, _ptr(out), _ptr(inp), int(out_parity), int(dagger), int(prec)))

    def mult_eo(self, out, inp, out_parity: int, dagger: bool = False, prec: int = F64, nrhs: int = 1):
        _check(self.lib.qcd_mult_eo(self._h, _ptr(out), _ptr(inp), int(out_parity), int(dagger), int(prec), int(nrhs)))

    def clover_apply(self, out, inp, parity: int, inverse: bool = False, prec: int = F64, nrhs: int = 1):
        _check(self.lib.qcd_clover_apply(self._h, _ptr(out), _ptr(inp), int(parity), int(inverse), int(prec), int(nrhs)))

    def dhat(self, out, inp, prec: int = F64, nrhs: int = 1):
        _check(self.lib.qcd_dhat(self._h, _ptr(out), _ptr(inp), int(prec), int(nrhs)))

    def schur_ee(self, out, inp, prec: int = F64, nrhs: int = 1):
        """out = S_ee inp = F_ee inp - kappa^2 H_eo F_oo^-1 H_oe inp (even half vectors)."""
        _check(self.lib.qcd_schur_ee(self._h, _ptr(out), _ptr(inp), int(prec), int(nrhs)))

    def dirac(self, out, inp):
        _check(self.lib.qcd_dirac(self._h, _ptr(out), _ptr(inp)))

    # ---- solver (device or host buffers)
    def solve(self, b, x, tol: float = 1e-12, opts: SolveOpts | None = None, check: bool = True, **kw) -> dict:
        if opts is None:
            opts = default_opts(**kw)
        info = SolveInfo()
        rc = self.lib.qcd_solve(self._h, _ptr(b), _ptr(x), float(tol), ctypes.byref(opts), ctypes.byref(info))
        if check:
            _check(rc)
        d = info.as_dict()
        d["rc"] = rc
        return d

    def solve_multi(self, b, x, tol: float = 1e-12, opts: SolveOpts | None = None, check: bool = True,
                    **kw) -> list:
        """Lockstep solves of the right-hand sides b[r] (device, [nrhs, V, 4, 3]
        complex128) into x[r]; one info dict per right-hand side."""
        if opts is None:
            opts = default_opts(**kw)
        n = int(b.shape[0])
        infos = (SolveInfo * n)()
        rc = self.lib.qcd_solve_multi(self._h, _ptr(b), _ptr(x), n, float(tol), ctypes.byref(opts), infos)
        if check:
            _check(rc)
        out = []
        for i in range(n):
            d = infos[i].as_dict()
            d["rc"] = rc
            out.append(d)
        return out

    def solve_adjoint(self, g, lam, tol: float = 1e-12, opts: SolveOpts | None = None, check: bool = True,
                      **kw) -> dict:
        """lam = D^-dag g (device buffers)."""
        if opts is None:
            opts = default_opts(**kw)
        info = SolveInfo()
        rc = self.lib.qcd_solve_adjoint(self._h, _ptr(g), _ptr(lam), float(tol), ctypes.byref(opts),
                                        ctypes.byref(info))
        if check:
            _check(rc)
        d = info.as_dict()
        d["rc"] = rc
        return d

    def force(self, U, x, lam, G):
        """G = gradient of -Re<lam, D[U] x> with respect to the links (device buffers)."""
        _check(self.lib.qcd_force(self._h, _ptr(U), _ptr(x), _ptr(lam), _ptr(G)))

    # ---- kernel timing
    def set_profiling(self, on):
        """0 off, 1 (True) events around every launch, 2 chunk timing of the
        FP32-level iterations (qcd_set_profiling)."""
        _check(self.lib.qcd_set_profiling(self._h, int(on)))

    def kernel_stats(self, cls: int) -> dict:
        s = KernelStat()
        _check(self.lib.qcd_kernel_stats(self._h, int(cls), ctypes.byref(s)))
        return dict(launches=s.launches, ms=s.ms, bytes=s.bytes)

    def reset_kernel_stats(self):
        _check(self.lib.qcd_reset_kernel_stats(self._h))

    def launch_count(self) -> int:
        return int(self.lib.qcd_launch_count(self._h))

    def autotune(self, cache_path: str | None = None):
        """Tune the operator kernels' launch configurations (cached in JSON)."""
        _check(self.lib.qcd_autotune(self._h, cache_path.encode() if cache_path else None))

    def tune_info(self) -> list:
        n = self.lib.qcd_tune_info(self._h, 0, None, None, None, None)
        keys = (ctypes.c_uint * max(n, 1))()
        var, thr = (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))()
        us = (ctypes.c_double * max(n, 1))()
        self.lib.qcd_tune_info(self._h, n, keys, var, thr, us)
        out = []
        for i in range(n):
            k = keys[i]
            out.append(dict(key=k, prec=k & 3, mode=(k >> 2) & 7, red=(k >> 5) & 3, dagger=(k >> 7) & 1,
                            nrhs=k >> 8, variant=var[i], threads=thr[i], us=us[i]))
        return out

    def mult_benchmark(self, prec: int = F32, nrhs: int = 1, iters: int = 20) -> dict:
        ms, by = ctypes.c_double(0), ctypes.c_double(0)
        _check(self.lib.qcd_mult_benchmark(self._h, int(prec), int(nrhs), int(iters), ctypes.byref(ms),
                                           ctypes.byref(by)))
        return dict(ms=ms.value, bytes=by.value, gbs=by.value / (ms.value * 1e-3) / 1e9)

    def pion_correlator(self, S, ncol: int = 12):
        """C(t) of qcd_pion_correlator from ncol propagator columns stored one
        after another in S (a torch CUDA tensor, or host memory)."""
        import numpy as np

        Lt = self.dims[3]
        C = np.zeros(Lt, dtype=np.float64)
        on_device = bool(getattr(S, "is_cuda", False))
        _check(self.lib.qcd_pion_correlator(self._h, _ptr(S), int(ncol), int(on_device),
                                            C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return C

    def mult_throughput(self, prec: int = F32, nrhs: int = 1, iters: int = 100) -> dict:
        """Back-to-back MULT launches without cache eviction (qcd.h)."""
        ms, by = ctypes.c_double(0), ctypes.c_double(0)
        _check(self.lib.qcd_mult_throughput(self._h, int(prec), int(nrhs), int(iters), ctypes.byref(ms),
                                            ctypes.byref(by)))
        return dict(ms=ms.value, bytes=by.value, gbs=by.value / (ms.value * 1e-3) / 1e9)
