"""Pins of the oracle's box solver (Sections 5.2-5.3): the sine-transform solve
must equal a dense LU solve of the explicitly assembled 5/7-point matrix."""
import numpy as np
import pytest

from kfbi_workloads.configs import Grid
from oracle import boxsolve


@pytest.mark.parametrize("dim,N,lam", [(2, 16, 0.0), (2, 16, 60.0), (3, 8, 40.0), (2, 12, 5.0)])
def test_dst_solve_equals_dense_lu(dim, N, lam):
    grid = Grid(dim, N)
    rng = np.random.default_rng(1)
    r = rng.standard_normal(grid.shape)
    A = boxsolve.dense_L(grid, lam)
    v_ref = np.linalg.solve(A, r.ravel()).reshape(grid.shape)
    v = boxsolve.solve(r, lam, grid)
    assert np.abs(v - v_ref).max() <= 1e-12 * np.abs(v_ref).max()


def test_apply_L_matches_dense():
    grid = Grid(3, 8)
    v = np.random.default_rng(2).standard_normal(grid.shape)
    A = boxsolve.dense_L(grid, 7.0)
    assert np.allclose(boxsolve.apply_L(v, 7.0, grid).ravel(), A @ v.ravel(), rtol=0, atol=1e-9)


def test_solve_inverts_operator_3d():
    grid = Grid(3, 24)
    v = np.random.default_rng(3).standard_normal(grid.shape)
    w = boxsolve.solve(boxsolve.apply_L(v, 40.0, grid), 40.0, grid)
    assert np.abs(w - v).max() < 1e-11


def test_eigenvector_closed_form():
    """sin(pi p x_k / ...) modes are eigenvectors with eigenvalue mu_p."""
    grid = Grid(2, 16)
    k = np.arange(1, 16)
    p, q = 3, 5
    mode = np.sin(np.pi * q * k / 16)[:, None] * np.sin(np.pi * p * k / 16)[None, :]
    mu = -(4 / grid.h ** 2) * (np.sin(np.pi * p / 32) ** 2 + np.sin(np.pi * q / 32) ** 2) - 2.0
    assert np.allclose(boxsolve.apply_L(mode, 2.0, grid), mu * mode, atol=1e-10)
    assert np.allclose(boxsolve.solve(mode, 2.0, grid), mode / mu, atol=1e-14)
