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


# ------------------------------------------------------------ Neumann box
# The box Green's function of Section 4 carries a zero normal derivative on
# the box boundary; its 5/7-point discretisation keeps all (N+1)^d nodes and
# mirrors the ghost value (v_{-1} = v_1).

@pytest.mark.parametrize("dim,N,lam", [(2, 8, 60.0), (2, 12, 5.0), (3, 6, 40.0), (2, 16, 0.5)])
def test_neumann_dct_solve_equals_dense_lu(dim, N, lam):
    grid = Grid(dim, N, bc="neumann")
    assert grid.shape == (N + 1,) * dim
    r = np.random.default_rng(4).standard_normal(grid.shape)
    A = boxsolve.dense_L(grid, lam)
    v_ref = np.linalg.solve(A, r.ravel()).reshape(grid.shape)
    v = boxsolve.solve(r, lam, grid)
    assert np.abs(v - v_ref).max() <= 1e-12 * np.abs(v_ref).max()


def test_neumann_dense_operator_by_hand():
    """The assembled 1-D-per-axis rows written out on a 2-D N = 4 box: a
    corner row couples to its two inner neighbours with weight 2/h^2, an edge
    row to its inner neighbour with 2/h^2, an interior row has the plain
    5-point weights."""
    grid = Grid(2, 4, bc="neumann")
    A = boxsolve.dense_L(grid, 3.0)
    ih2 = 1.0 / grid.h ** 2
    idx = lambda y, x: y * 5 + x  # noqa: E731
    row = A[idx(0, 0)]
    assert row[idx(0, 0)] == -4 * ih2 - 3.0 and row[idx(0, 1)] == 2 * ih2 and row[idx(1, 0)] == 2 * ih2
    assert np.count_nonzero(row) == 3
    row = A[idx(0, 2)]
    assert row[idx(0, 1)] == ih2 and row[idx(0, 3)] == ih2 and row[idx(1, 2)] == 2 * ih2
    row = A[idx(2, 2)]
    assert all(row[idx(y, x)] == ih2 for y, x in ((1, 2), (3, 2), (2, 1), (2, 3)))
    # every row sums to -lambda (constants are mapped to -lambda constants)
    assert np.allclose(A.sum(axis=1), -3.0)


def test_neumann_cosine_modes_are_eigenvectors():
    grid = Grid(3, 8, bc="neumann")
    k = np.arange(9)
    p, q, s = 0, 3, 8
    mode = (np.cos(np.pi * s * k / 8)[:, None, None] * np.cos(np.pi * q * k / 8)[None, :, None]
            * np.cos(np.pi * p * k / 8)[None, None, :])
    mu = -(4 / grid.h ** 2) * sum(np.sin(np.pi * m / 16) ** 2 for m in (p, q, s)) - 7.0
    assert np.allclose(boxsolve.apply_L(mode, 7.0, grid), mu * mode, atol=1e-9)
    assert np.allclose(boxsolve.solve(mode, 7.0, grid), mode / mu, atol=1e-14)


def test_neumann_planted_dirichlet_boundary_is_detected():
    """Solving with the sine transform on the Neumann layout (boundary values
    forced to the Dirichlet reading) misses the dense Neumann solution."""
    grid = Grid(2, 8, bc="neumann")
    r = np.random.default_rng(5).standard_normal(grid.shape)
    v_ref = np.linalg.solve(boxsolve.dense_L(grid, 60.0), r.ravel()).reshape(grid.shape)
    inner = boxsolve.solve(r[1:-1, 1:-1], 60.0, Grid(2, 8))
    assert np.abs(inner - v_ref[1:-1, 1:-1]).max() > 1e-3 * np.abs(v_ref).max()


def test_neumann_box_requires_positive_lambda():
    with pytest.raises(ValueError):
        boxsolve.solve(np.ones((9, 9)), 0.0, Grid(2, 8, bc="neumann"))
