"""CPU oracle for the clover Wilson operator and its BiCGStab solvers.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product package.  The
arithmetic lives in plain C (qcd_oracle.c, FP64, written from the paper's
definitions); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  See qcd_oracle.c for the definitions followed and the
passages of the paper they come from.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_libs = {}
_openmp = False


def _compile(so: str, extra, force: bool):
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + ".tmp%d" % os.getpid()
        # no FMA contraction (the ISO C mode's default, stated): every host
        # rounds each operation the same way
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared"] + list(extra) +
                              ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so, and the
    same source with OpenMP (site loops split across threads, nothing else
    changed) into liboracle_omp.so for multi-core timings."""
    os.makedirs(_BUILD, exist_ok=True)
    _compile(_SO, [], force)
    _compile(_SO_OMP, ["-fopenmp"], force)
    return _SO


def use_openmp(on: bool, threads: int | None = None) -> int:
    """Route every later oracle call to the OpenMP build (on) or the
    single-threaded one; returns the threads the site loops then use."""
    global _openmp
    _openmp = bool(on)
    L = lib()
    if on and threads:
        L.oracle_set_threads(int(threads))
    return int(L.oracle_threads())


def lib():
    if _openmp not in _libs:
        build()
        L = ctypes.CDLL(_SO_OMP if _openmp else _SO)
        L.oracle_true_residual.restype = ctypes.c_double
        L.oracle_threads.restype = ctypes.c_int
        _libs[_openmp] = L
    return _libs[_openmp]


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


# ---------------------------------------------------------------- algebra
def gamma(which: int) -> np.ndarray:
    """gamma_mu for which = 0..3 (x, y, z, t) and gamma5 for which = 4."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().oracle_gamma(ctypes.c_int(which), _p(out))
    return out


# ---------------------------------------------------------------- operator
def hopping(dims, t_bc, U, psi, dagger=False):
    """H psi on the full lattice (Eq. 4); dagger gives gamma5 H gamma5."""
    U, psi = _c(U), _c(psi)
    out = np.empty_like(psi)
    lib().oracle_hopping(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(psi), _p(out), ctypes.c_int(int(dagger)))
    return out


def clover_field(dims, U, kappa, csw):
    """F(n) as [V, 12, 12], index 3*spin + colour."""
    U = _c(U)
    F = np.empty((volume(dims), 12, 12), dtype=np.complex128)
    lib().oracle_clover_field(_dims(dims), _p(U), ctypes.c_double(kappa), ctypes.c_double(csw), _p(F))
    return F


def field_strength(dims, U, site, mu, nu):
    """F_munu(n) = (Q - Q^dag)/(8i) at one site, [3, 3]."""
    U = _c(U)
    out = np.empty((3, 3), dtype=np.complex128)
    lib().oracle_field_strength(_dims(dims), _p(U), ctypes.c_long(site), ctypes.c_int(mu), ctypes.c_int(nu), _p(out))
    return out


def invert_sites(F):
    F = _c(F)
    Fi = np.empty_like(F)
    rc = lib().oracle_invert_sites(ctypes.c_long(F.shape[0]), _p(F), _p(Fi))
    if rc != 0:
        raise ArithmeticError("singular clover block")
    return Fi


def site_apply(M, psi):
    M, psi = _c(M), _c(psi)
    out = np.empty_like(psi)
    lib().oracle_site_apply(ctypes.c_long(M.shape[0]), _p(M), _p(psi), _p(out))
    return out


def dirac(dims, t_bc, U, F, kappa, psi):
    """D psi = F psi - kappa H psi (Eq. 3)."""
    U, F, psi = _c(U), _c(F), _c(psi)
    out = np.empty_like(psi)
    lib().oracle_dirac(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(F), ctypes.c_double(kappa), _p(psi), _p(out))
    return out


def dirac_sites(dims, t_bc, U, kappa, csw, psi, sites):
    """(D psi)(n) at the listed sites only, [len(sites), 4, 3]."""
    U, psi = _c(U), _c(psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    lib().oracle_dirac_sites(_dims(dims), ctypes.c_int(t_bc), _p(U), ctypes.c_double(kappa), ctypes.c_double(csw),
                             _p(psi), ctypes.c_long(len(sites)), _p(sites), _p(out))
    return out


def hop_sites(dims, t_bc, U, psi, sites, dagger=False):
    """(H psi)(n) at the listed lexicographic sites, [len(sites), 4, 3]."""
    U, psi = _c(U), _c(psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    lib().oracle_hop_sites(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(psi), ctypes.c_long(len(sites)), _p(sites),
                           _p(out), ctypes.c_int(int(dagger)))
    return out


def clover_sites(dims, U, kappa, csw, sites):
    """F(n) at the listed lexicographic sites, [len(sites), 12, 12]."""
    U = _c(U)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    F = np.empty((len(sites), 12, 12), dtype=np.complex128)
    lib().oracle_clover_sites(_dims(dims), _p(U), ctypes.c_double(kappa), ctypes.c_double(csw),
                              ctypes.c_long(len(sites)), _p(sites), _p(F))
    return F


def site_of_cb(dims, parity, cb):
    """Lexicographic index of the cb-th site of a parity (cb = lex/2)."""
    cb = np.asarray(cb, dtype=np.int64)
    s = 2 * cb
    Lx, Ly, Lz = int(dims[0]), int(dims[1]), int(dims[2])
    x, r = s % Lx, s // Lx
    y, r = r % Ly, r // Ly
    z, t = r % Lz, r // Lz
    return np.where((x + y + z + t) % 2 == parity, s, s + 1)


# ---------------------------------------------------------------- observables
def pion_correlator(dims, S):
    """C(t) = sum over columns, over the sites x of timeslice t and over spin
    and colour of |S(x)|^2, for propagator columns S [ncol, V, 4, 3] (sites
    lexicographic, t slowest).  With S the 12 spin-colour columns from a point
    source this is the pion two-point function sum_x Tr[S(x) S(x)^dag]
    (gamma5-hermiticity, Eq. 3 with g5 D g5 = D^dag), an observable the
    solutions of Eq. 1 serve (Sec. II-A)."""
    S = np.asarray(S)
    Lt = int(dims[3])
    V3 = volume(dims) // Lt
    a = np.abs(S.reshape(S.shape[0], Lt, V3, 12)) ** 2
    return a.sum(axis=(0, 2, 3))


# ---------------------------------------------------------------- even-odd
def half_to_full(dims, parity, half):
    half = _c(half)
    full = np.empty((volume(dims), 4, 3), dtype=np.complex128)
    lib().oracle_half_to_full(_dims(dims), ctypes.c_int(parity), _p(half), _p(full))
    return full


def full_to_half(dims, parity, full):
    full = _c(full)
    half = np.empty((volume(dims) // 2, 4, 3), dtype=np.complex128)
    lib().oracle_full_to_half(_dims(dims), ctypes.c_int(parity), _p(full), _p(half))
    return half


def field_to_half(dims, parity, F):
    F = _c(F)
    out = np.empty((volume(dims) // 2, 12, 12), dtype=np.complex128)
    lib().oracle_field_to_half(_dims(dims), ctypes.c_int(parity), _p(F), _p(out))
    return out


def hop_eo(dims, t_bc, U, out_parity, in_half, dagger=False):
    """H_{p,1-p} on half-lattice vectors."""
    U, in_half = _c(U), _c(in_half)
    out = np.empty_like(in_half)
    lib().oracle_hop_eo(_dims(dims), ctypes.c_int(t_bc), _p(U), ctypes.c_int(out_parity), _p(in_half), _p(out),
                        ctypes.c_int(int(dagger)))
    return out


def mult(dims, t_bc, U, Finv, out_parity, in_half):
    """MULT = F_pp^-1 H_{p,1-p} (Sec. II-B); Finv is the full [V,12,12] field."""
    U, Finv, in_half = _c(U), _c(Finv), _c(in_half)
    out = np.empty_like(in_half)
    lib().oracle_mult(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_int(out_parity), _p(in_half), _p(out))
    return out


def dhat(dims, t_bc, U, Finv, kappa, p):
    """D^_ee p = p - kappa^2 H~_eo H~_oe p (Eq. 8)."""
    U, Finv, p = _c(U), _c(Finv), _c(p)
    q = np.empty_like(p)
    lib().oracle_dhat(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_double(kappa), _p(p), _p(q))
    return q


def schur_ee(dims, t_bc, U, F, Finv, kappa, p):
    """S_ee p = F_ee p - kappa^2 H_eo F_oo^-1 H_oe p: the gamma5-hermitian
    even-odd operator, F_ee times D^_ee of Eq. 8."""
    U, F, Finv, p = _c(U), _c(F), _c(Finv), _c(p)
    q = np.empty_like(p)
    lib().oracle_schur_ee(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(F), _p(Finv), ctypes.c_double(kappa), _p(p),
                          _p(q))
    return q


def schur_source(dims, t_bc, U, Finv, kappa, b):
    """The right-hand side of S_ee x_e: b_e + kappa H_eo F_oo^-1 b_o."""
    U, Finv, b = _c(U), _c(Finv), _c(b)
    out = np.empty((volume(dims) // 2, 4, 3), dtype=np.complex128)
    lib().oracle_schur_source(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_double(kappa), _p(b),
                              _p(out))
    return out


def eo_source(dims, t_bc, U, Finv, kappa, b):
    """b^_e = F_ee^-1 b_e + kappa H~_eo F_oo^-1 b_o (Eq. 6)."""
    U, Finv, b = _c(U), _c(Finv), _c(b)
    out = np.empty((volume(dims) // 2, 4, 3), dtype=np.complex128)
    lib().oracle_eo_source(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_double(kappa), _p(b), _p(out))
    return out


def eo_reconstruct(dims, t_bc, U, Finv, kappa, b, x_e):
    """Full solution from x_e with x_o = F_oo^-1 b_o + kappa H~_oe x_e (Eq. 7)."""
    U, Finv, b, x_e = _c(U), _c(Finv), _c(b), _c(x_e)
    x = np.empty((volume(dims), 4, 3), dtype=np.complex128)
    lib().oracle_eo_reconstruct(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_double(kappa), _p(b),
                                _p(x_e), _p(x))
    return x


def true_residual(dims, t_bc, U, F, kappa, b, x) -> float:
    """||b - D x|| / ||b|| on the full lattice."""
    U, F, b, x = _c(U), _c(F), _c(b), _c(x)
    return float(lib().oracle_true_residual(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(F), ctypes.c_double(kappa),
                                            _p(b), _p(x)))


# ---------------------------------------------------------------- solvers
def bicgstab_full(dims, t_bc, U, F, kappa, b, tol, maxit=10000):
    """Unpreconditioned BiCGStab on D from x = 0; returns (x, status, iters)."""
    U, F, b = _c(U), _c(F), _c(b)
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    st = lib().oracle_bicgstab_full(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(F), ctypes.c_double(kappa), _p(b),
                                    _p(x), ctypes.c_double(tol), ctypes.c_int(maxit), ctypes.byref(it))
    return x, st, it.value


def bicgstab_eo(dims, t_bc, U, Finv, kappa, b, tol_eo, maxit=10000):
    """Even-odd preconditioned BiCGStab on D^_ee; returns (x_full, status, iters)."""
    U, Finv, b = _c(U), _c(Finv), _c(b)
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    st = lib().oracle_bicgstab_eo(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_double(kappa), _p(b),
                                  _p(x), ctypes.c_double(tol_eo), ctypes.c_int(maxit), ctypes.byref(it))
    return x, st, it.value


def bicgstab_schur(dims, t_bc, U, F, Finv, kappa, b, tol_eo, maxit=10000):
    """FP64 BiCGStab on the gamma5-hermitian S_ee, then x_o (Eq. 7); returns
    (x_full, status, iters)."""
    U, F, Finv, b = _c(U), _c(F), _c(Finv), _c(b)
    x = np.empty_like(b)
    it = ctypes.c_int(0)
    st = lib().oracle_bicgstab_schur(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(F), _p(Finv), ctypes.c_double(kappa),
                                     _p(b), _p(x), ctypes.c_double(tol_eo), ctypes.c_int(maxit), ctypes.byref(it))
    return x, st, it.value


def nested_bicgstab(dims, t_bc, U, Finv, kappa, b, tol_eo, inner_tol, inner_maxit=250, maxit=100):
    """Alg. 1 with Alg. 2 as the inner solve, all in FP64; returns
    (x_full, status, outer_iterations, inner_applications)."""
    U, Finv, b = _c(U), _c(Finv), _c(b)
    x = np.empty_like(b)
    outer = ctypes.c_int(0)
    inner = ctypes.c_int(0)
    st = lib().oracle_nested_bicgstab(_dims(dims), ctypes.c_int(t_bc), _p(U), _p(Finv), ctypes.c_double(kappa), _p(b),
                                      _p(x), ctypes.c_double(tol_eo), ctypes.c_double(inner_tol),
                                      ctypes.c_int(inner_maxit), ctypes.c_int(maxit), ctypes.byref(outer),
                                      ctypes.byref(inner))
    return x, st, outer.value, inner.value


# ---------------------------------------------------------------- gradient
def link_grad(dims, t_bc, U, kappa, csw, x, lam):
    """Gradient of f(U) = -Re<lam, D[U] x> with x, lam fixed, in the
    convention G = df/dRe U + i df/dIm U; [V, 4, 3, 3]."""
    U, x, lam = _c(U), _c(x), _c(lam)
    G = np.empty_like(U)
    lib().oracle_link_grad(_dims(dims), ctypes.c_int(t_bc), _p(U), ctypes.c_double(kappa), ctypes.c_double(csw),
                           _p(x), _p(lam), _p(G))
    return G
