"""Box solver for the corrected finite-difference system (oracle).

The equivalent interface problems of Section 5.1 are discretised with the
standard 5-point (2-D) / 7-point (3-D) stencil on the box grid (Eq. FDE with
unit isotropic conductivity),

    (L_h v)_k = sum_a (v_{k+e_a} - 2 v_k + v_{k-e_a}) / h^2 - lambda v_k,

with one of two box conditions:

* Dirichlet box, v = 0 on the box boundary (the reading of Section 5.1): the
  unknowns are the interior nodes k = 1..N-1 and the matrix is the symmetric
  definite L_h, solved exactly by sine transforms (Section 5.3, the FFT-based
  fast Poisson solver):
      v = (2/N)^d  S( mu^{-1} o S r ),   S_{kp} = sin(pi k p / N),
      mu_p = - sum_a (4/h^2) sin^2(pi p_a / (2N)) - lambda;
* Neumann box, zero normal derivative on the box boundary (the box Green's
  function of Section 4): the unknowns are all nodes k = 0..N, and the
  boundary rows use the mirrored ghost value v_{-1} = v_1 (v_{N+1} = v_{N-1}),
  the second-order discretisation of the zero flux.  The cosines
  cos(pi k p / N), p = 0..N, are its eigenvectors with the same mu_p, so
      v = (2/N)^d  C( mu^{-1} o C r ),
      C_{kp} = c_k cos(pi k p / N),  c_0 = c_N = 1/2, c_k = 1 otherwise.
  With lambda = 0 the mode p = 0 is singular (no Green's function exists),
  and the Neumann box requires lambda > 0.

Because the irregular-node correction only changes the right-hand side, the
matrix is the same for every evaluation.  scipy's DST-I / DCT-I are 2 S / 2 C
along each axis, hence the factor (1/(2N))^d below.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft

from kfbi_workloads.configs import Grid

WORKERS = os.cpu_count() or 1


def eigenvalues(grid: Grid, lam: float) -> np.ndarray:
    """mu_p on the mode grid (p = 1..N-1 Dirichlet, 0..N Neumann), same layout
    as the field."""
    p = np.arange(grid.first, grid.first + grid.n, dtype=np.float64)
    m1 = -(4.0 / grid.h ** 2) * np.sin(np.pi * p / (2.0 * grid.N)) ** 2
    if grid.dim == 2:
        return m1[None, :] + m1[:, None] - lam
    return m1[None, None, :] + m1[None, :, None] + m1[:, None, None] - lam


def solve(r: np.ndarray, lam: float, grid: Grid) -> np.ndarray:
    """v = L_h^{-1} r with the grid's box condition."""
    mu = eigenvalues(grid, lam)
    if grid.bc == "neumann":
        if lam <= 0.0:
            raise ValueError("the Neumann box needs lambda > 0")
        rh = scipy.fft.dctn(r, type=1, workers=WORKERS)
        v = scipy.fft.dctn(rh / mu, type=1, workers=WORKERS)
    else:
        rh = scipy.fft.dstn(r, type=1, workers=WORKERS)
        v = scipy.fft.dstn(rh / mu, type=1, workers=WORKERS)
    return v / (2.0 * grid.N) ** grid.dim


def apply_L(v: np.ndarray, lam: float, grid: Grid) -> np.ndarray:
    """L_h v with the grid's box condition (used for pins and residuals):
    zero values beyond the Dirichlet box, mirrored values beyond the Neumann
    box."""
    d = v.ndim
    P = np.pad(v, 1, mode="reflect") if grid.bc == "neumann" else np.pad(v, 1)
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
    (tiny grids only): a neighbour beyond the Dirichlet box drops out (value
    0), one beyond the Neumann box is its mirror image across the boundary."""
    n1 = grid.n
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
                if grid.bc == "neumann":
                    if kk[ax] < 0:
                        kk[ax] = 1
                    elif kk[ax] >= n1:
                        kk[ax] = n1 - 2
                if 0 <= kk[ax] < n1:
                    A[row, np.ravel_multi_index(kk, (n1,) * d)] += ih2
    return A
