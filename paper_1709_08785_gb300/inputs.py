"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on quenched gauge configurations (Sec. IV-C: beta = 7.90,
a 400^3 x 800 lattice) that are not available here.  These generators stand
in for them with reproducible fields of the same shape and structure:

* gauge links U_mu(n) = reunitarised exp(i * eps * H), H a traceless
  Hermitian 3x3 matrix with N(0,1) entries, drawn per link;
* Gaussian complex sources, N(0,1) in the real and the imaginary part of
  every spin-colour component;
* point sources (one spin-colour component at one site);
* random SU(3) gauge transformations.

This module holds none of the method's arithmetic: it only draws numbers.
Both the CUDA path and the CPU oracle take their inputs from it.

Layouts (canonical, complex128):
  links   [V, 4, 3, 3]  site s = x + Lx*(y + Ly*(z + Lz*t)), mu = x, y, z, t
  spinors [V, 4, 3]     spin, colour
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 20  # sites generated per numpy batch (bounds peak host memory)


def volume(dims) -> int:
    """Number of sites of a lattice with extents (Lx, Ly, Lz, Lt)."""
    v = 1
    for d in dims:
        v *= int(d)
    return v


def _reunitarise(M: np.ndarray) -> np.ndarray:
    """Gram-Schmidt on the first two columns; the third is conj(a x b), so
    that det = 1 exactly (up to rounding).  M has shape [..., 3, 3]."""
    a = M[..., :, 0]
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = M[..., :, 1]
    b = b - np.sum(np.conj(a) * b, axis=-1, keepdims=True) * a
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    c = np.conj(np.cross(a, b))
    out = np.empty_like(M)
    out[..., :, 0] = a
    out[..., :, 1] = b
    out[..., :, 2] = c
    return out


def _traceless_hermitian(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    A = X + 1j * Y
    H = np.triu(A, 1)
    H = H + np.conj(np.swapaxes(H, -1, -2))
    idx = np.arange(3)
    H[..., idx, idx] = X[..., idx, idx]
    tr = np.trace(H, axis1=-2, axis2=-1)
    H[..., idx, idx] -= (tr / 3.0)[..., None]
    return H


def random_gauge(dims, eps: float, seed: int) -> np.ndarray:
    """Links U = reunitarised exp(i eps H), [V, 4, 3, 3] complex128.

    X then Y are drawn with numpy's default_rng(seed) as standard normals of
    shape [V, 4, 3, 3]; H = strict-upper(X + iY) + h.c. + diag(X), made
    traceless; exp(i eps H) = W diag(exp(i eps lambda)) W^dag from eigh.
    """
    V = volume(dims)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((V, 4, 3, 3))
    Y = rng.standard_normal((V, 4, 3, 3))
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for s0 in range(0, V, _CHUNK):
        s1 = min(V, s0 + _CHUNK)
        H = _traceless_hermitian(X[s0:s1], Y[s0:s1])
        w, W = np.linalg.eigh(H)
        E = (W * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(W, -1, -2))
        U[s0:s1] = _reunitarise(E)
    return U


def random_gauge_torch(dims, eps: float, seed: int, device="cuda"):
    """The same draws as random_gauge (X then Y from default_rng(seed)), with
    exp(i eps H) taken by scaling and squaring of its Taylor series in torch
    on `device` and then reunitarised the same way; equal to random_gauge up
    to rounding.  For the large lattices, where numpy's eigh takes minutes.
    Returns a complex128 torch tensor [V, 4, 3, 3] on `device`."""
    import torch

    V = volume(dims)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((V, 4, 3, 3))
    Y = rng.standard_normal((V, 4, 3, 3))
    out = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device=device)
    eye = torch.eye(3, dtype=torch.complex128, device=device)
    chunk = 1 << 19
    for s0 in range(0, V, chunk):
        s1 = min(V, s0 + chunk)
        H = torch.from_numpy(_traceless_hermitian(X[s0:s1], Y[s0:s1])).to(device)
        A = (1j * eps) * H
        # scale so that the Frobenius norm is at most 1/2, Taylor to order 18
        nrm = torch.linalg.matrix_norm(A).max().item()
        k = max(0, int(np.ceil(np.log2(max(nrm, 1e-300) / 0.5))))
        A = A / (2.0 ** k)
        E = eye.expand_as(A).clone()
        T = eye.expand_as(A).clone()
        for n in range(1, 19):
            T = (T @ A) / n
            E = E + T
        for _ in range(k):
            E = E @ E
        a = E[..., :, 0]
        a = a / torch.linalg.vector_norm(a, dim=-1, keepdim=True)
        b = E[..., :, 1]
        b = b - torch.sum(torch.conj(a) * b, dim=-1, keepdim=True) * a
        b = b / torch.linalg.vector_norm(b, dim=-1, keepdim=True)
        c = torch.conj(torch.linalg.cross(a, b, dim=-1))
        out[s0:s1] = torch.stack([a, b, c], dim=-1)
    return out


def unit_gauge(dims) -> np.ndarray:
    """The free field: every link is the identity."""
    V = volume(dims)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def gaussian_source(dims, seed: int) -> np.ndarray:
    """b = N(0,1) + i N(0,1) per spin-colour component, [V, 4, 3]."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((V, 4, 3))
    im = rng.standard_normal((V, 4, 3))
    return re + 1j * im


def point_source(dims, spin: int, colour: int, site: int = 0) -> np.ndarray:
    """delta at one site, one spin and one colour component, [V, 4, 3]."""
    b = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def point_sources(dims, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at one site, [12, V, 4, 3], ordered
    spin-major (k = 3*spin + colour)."""
    out = np.zeros((12, volume(dims), 4, 3), dtype=np.complex128)
    for k in range(12):
        out[k, site, k // 3, k % 3] = 1.0
    return out


def random_su3(n: int, seed: int) -> np.ndarray:
    """n reunitarised complex Gaussian 3x3 matrices (det = 1), [n, 3, 3]."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    return _reunitarise(M)


def random_su3_directions(n: int, seed: int) -> np.ndarray:
    """n traceless Hermitian 3x3 matrices with unit Frobenius norm drawn from
    N(0,1) coefficients on the Gell-Mann basis, [n, 3, 3]."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((n, 8))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    s3 = 1.0 / np.sqrt(3.0)
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0], lam[2, 1, 1] = 1, -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    lam[7, 0, 0], lam[7, 1, 1], lam[7, 2, 2] = s3, s3, -2 * s3
    T = np.einsum("na,aij->nij", c, lam) / np.sqrt(2.0)  # ||lambda_a||_F = sqrt(2)
    return T


BATCH_LATTICES = ((8, 8, 8, 8), (12, 12, 12, 24), (16, 16, 16, 32), (20, 20, 20, 40))


def batch_problems(n: int = 48, seed: int = 99):
    """The batched-solve workload: n independent problems, each a dict with
    dims (drawn uniformly from BATCH_LATTICES), eps ~ U[0.15, 0.35],
    kappa ~ U[0.115, 0.124], csw = 1.0, links seed 100+i, source seed 200+i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dims = BATCH_LATTICES[int(rng.integers(0, len(BATCH_LATTICES)))]
        eps = float(rng.uniform(0.15, 0.35))
        kappa = float(rng.uniform(0.115, 0.124))
        out.append(dict(dims=dims, eps=eps, kappa=kappa, csw=1.0, link_seed=100 + i, src_seed=200 + i))
    return out
