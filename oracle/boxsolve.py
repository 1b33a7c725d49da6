"""Box solver for the corrected finite-difference system (oracle).

The equivalent interface problems of Section 5.1 are discretised with the
standard 5-point (2-D) / 7-point (3-D) stencil on the box grid (Eq. FDE with
unit isotropic conductivity),

    (L_h v)_k = sum_a (v_{k+e_a} - 2 v_k + v_{k-e_a}) / h^2 - lambda v_k,

with v = 0 on the box boundary (the interface problems carry v = 0 on the
boundary of the box).  Because the irregular-node correction only changes the
right-hand side, the matrix stays the symmetric definite L_h and is solved
exactly by sine transforms (Section 5.3, the FFT-based fast Poisson solver):

    v = (2/N)^d  S( mu^{-1} o S r ),   S_{kp} = sin(pi k p / N),
    mu_p = - sum_a (4/h^2) sin^2(pi p_a / (2N)) - lambda.

scipy's DST-I is 2 S along each axis, hence the factor (1/(2N))^d below.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft

from kfbi_workloads.configs import Grid

WORKERS = os.cpu_count() or 1


def eigenvalues(grid: Grid, lam: float) -> np.ndarray:
    """mu_p on the (N-1)^d mode grid, same layout as the field."""
    p = np.arange(1, grid.N, dtype=np.float64)
    m1 = -(4.0 / grid.h ** 2) * np.sin(np.pi * p / (2.0 * grid.N)) ** 2
    if grid.dim == 2:
        return m1[None, :] + m1[:, None] - lam
    return m1[None, None, :] + m1[None, :, None] + m1[:, None, None] - lam


def solve(r: np.ndarray, lam: float, grid: Grid) -> np.ndarray:
    """v = L_h^{-1} r with homogeneous Dirichlet data on the box."""
    mu = eigenvalues(grid, lam)
    rh = scipy.fft.dstn(r, type=1, workers=WORKERS)
    v = scipy.fft.dstn(rh / mu, type=1, workers=WORKERS)
    return v / (2.0 * grid.N) ** grid.dim


def apply_L(v: np.ndarray, lam: float, grid: Grid) -> np.ndarray:
    """L_h v with zero Dirichlet data (used for pins and residuals)."""
    d = v.ndim
    P = np.pad(v, 1)
    out = -(2.0 * d / grid.h ** 2 + lam) * v
    for ax in range(d):
        sl_m = [slice(1, -1)] * d
        sl_p = [slice(1, -1)] * d
        sl_m[ax] = slice(0, -2)
        sl_p[ax] = slice(2, None)
        out = out + (P[tuple(sl_m)] + P[tuple(sl_p)]) / grid.h ** 2
    return out


def dense_L(grid: Grid, lam: float) -> np.ndarray:
    """Assembled L_h as a dense matrix, written entry by entry from the stencil
    (tiny grids only)."""
    n1 = grid.N - 1
    d = grid.dim
    n = n1 ** d
    A = np.zeros((n, n))
    ih2 = 1.0 / grid.h ** 2
    for row in range(n):
        k = np.unravel_index(row, (n1,) * d)
        A[row, row] = -2.0 * d * ih2 - lam
        for ax in range(d):
            for step in (-1, 1):
                kk = list(k)
                kk[ax] += step
                if 0 <= kk[ax] < n1:
                    A[row, np.ravel_multi_index(kk, (n1,) * d)] += ih2
    return A
