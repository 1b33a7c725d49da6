"""Initial densities of the diffusion solves (oracle of the warm starts).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Neither warm start is
in the paper, which starts every solve from the previous density; both only
change GMRES's initial guess, so the converged density is still fixed by the
solver tolerance (Section 4: the residual of A psi = g decides).

History projection.  The densities psi_s of earlier solves and their images
b_s = A psi_s are kept.  For the new right-hand side g the coefficients c
minimise ||g - sum_s c_s b_s||_2 (plain least squares over the k <= 8 stored
solves); the projected density and its residual are
    psi_F = sum_s c_s psi_s,     r_F = g - sum_s c_s b_s,
and r_F is psi_F's exact residual g - A psi_F because A is linear.  The
start of the projection form is psi_F + 2 gamma r_F: one step of the paper's
simple iteration (Eq. simple iteration) from psi_F.

Learned correction of the projection.  A point-wise network (oracle.mlp)
reads, per interface node,
    (psi_F / rms(psi_F), r_F / rms(r_F), g / rms(g), x, y, z, n_x, n_y, n_z)
in float32 (rms = root mean square over the nodes), normalised by fixed
means and standard deviations, and returns o; the learned start is
    psi_L = psi_F + 2 gamma r_F + rms(r_F) (s_out o + m_out).
Its training target is therefore (psi - psi_F - 2 gamma r_F) / rms(r_F) for
the converged density psi of the same solve.
"""
from __future__ import annotations

import numpy as np

from . import mlp


def projection(hist_psi: np.ndarray, hist_img: np.ndarray, g: np.ndarray):
    """psi_F, r_F and the coefficients c of the least-squares fit of g by the
    stored images.  hist_psi, hist_img: [k, M] (k >= 0); g: [M]."""
    k = hist_img.shape[0]
    if k == 0:
        return np.zeros_like(g), g.copy(), np.zeros(0)
    c, *_ = np.linalg.lstsq(hist_img.T, g, rcond=None)
    psi_F = c @ hist_psi
    r_F = g - c @ hist_img
    return psi_F, r_F, c


def rms(v: np.ndarray) -> float:
    return float(np.sqrt(np.mean(np.asarray(v, dtype=np.float64) ** 2)))


def features(psi_F, r_F, g, nodes, normals) -> np.ndarray:
    """Raw float32 input rows [M, 9] of the learned correction."""
    cols = [psi_F / rms(psi_F), r_F / rms(r_F), g / rms(g)]
    F = np.concatenate([np.stack(cols, axis=1), np.asarray(nodes, dtype=np.float64),
                        np.asarray(normals, dtype=np.float64)], axis=1)
    return F.astype(np.float32)


def target(psi, psi_F, r_F, gamma=0.8) -> np.ndarray:
    """Training target of one solve (float32): the correction the network
    should add to psi_F + 2 gamma r_F, in units of rms(r_F)."""
    return ((psi - psi_F - 2.0 * gamma * r_F) / rms(r_F)).astype(np.float32)


def fit_norm(F: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Normalisation vector [mean_0..8, std_0..8, target mean, target std]
    (sample standard deviations, a zero one replaced by 1)."""
    F = np.asarray(F, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    mean = F.mean(axis=0)
    std = F.std(axis=0, ddof=1)
    std = np.where(std > 1e-12, std, 1.0)
    ts = T.std(ddof=1)
    return np.concatenate([mean, std, [T.mean(), ts if ts > 1e-30 else 1.0]]).astype(np.float32)


def prediction(psi_F, r_F, o, norm, gamma=0.8):
    """psi_L = psi_F + 2 gamma r_F + rms(r_F) (s_out o + m_out), the network
    output o denormalised in float32."""
    s_out, m_out = np.float32(norm[2 * mlp.N_IN + 1]), np.float32(norm[2 * mlp.N_IN])
    corr = (s_out * np.asarray(o, dtype=np.float32) + m_out).astype(np.float32).astype(np.float64)
    return psi_F + 2.0 * gamma * r_F + rms(r_F) * corr


def predict(flat, norm, psi_F, r_F, g, nodes, normals, gamma=0.8):
    """psi_L from the network with packed parameters `flat`; returns
    (psi_L, o)."""
    X = mlp.normalise(features(psi_F, r_F, g, nodes, normals), norm)
    o = mlp.forward(flat, X)
    return prediction(psi_F, r_F, o, norm, gamma), o
