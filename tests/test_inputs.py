"""The seeded input generators: unitarity, det U = 1 (which the 12-real link
storage relies on), the spread the recipe asks, and agreement of the torch
path with the numpy path."""
import numpy as np
import pytest

from paper_1709_08785_gb300 import inputs


def test_links_are_special_unitary():
    U = inputs.random_gauge((4, 4, 2, 4), 0.3, 5)
    UU = np.einsum("smij,smkj->smik", U, U.conj())
    assert np.max(np.abs(UU - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(U) - 1.0)) < 1e-14
    # third column is conj(a x b): what the reconstruction rebuilds
    c = np.conj(np.cross(U[..., :, 0], U[..., :, 1]))
    assert np.max(np.abs(c - U[..., :, 2])) < 1e-14


def test_link_spread_follows_eps():
    # |Tr U|/3 = 1 - O(eps^2): a smaller eps gives smoother links
    t1 = np.mean(np.abs(np.trace(inputs.random_gauge((4, 4, 4, 4), 0.15, 7), axis1=-2, axis2=-1))) / 3
    t2 = np.mean(np.abs(np.trace(inputs.random_gauge((4, 4, 4, 4), 0.35, 7), axis1=-2, axis2=-1))) / 3
    assert 1.0 > t1 > t2 > 0.5


def test_torch_generator_matches_numpy():
    torch = pytest.importorskip("torch")
    dims = (4, 2, 4, 4)
    a = inputs.random_gauge(dims, 0.3, 9)
    b = inputs.random_gauge_torch(dims, 0.3, 9, device="cpu").numpy()
    assert np.max(np.abs(a - b)) < 1e-13


def test_sources_and_batch_recipe():
    b = inputs.gaussian_source((4, 4, 4, 4), 2)
    assert b.shape == (256, 4, 3)
    assert abs(np.mean(np.abs(b) ** 2) - 2.0) < 0.2  # Re and Im each N(0,1)
    P = inputs.point_sources((2, 2, 2, 2))
    assert P.shape == (12, 16, 4, 3) and np.sum(np.abs(P)) == 12
    probs = inputs.batch_problems()
    assert len(probs) == 48
    assert all(p["dims"] in inputs.BATCH_LATTICES for p in probs)
    assert all(0.15 <= p["eps"] <= 0.35 and 0.115 <= p["kappa"] <= 0.124 for p in probs)
