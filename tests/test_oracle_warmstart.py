"""Pins of the oracle's warm starts (history projection, learned correction).

* projection: a right-hand side inside the span of the stored images is
  recovered exactly (psi_F is the density that produced it, r_F = 0); for any
  other one the residual r_F is orthogonal to every stored image (the normal
  equations of least squares), equals g - A psi_F for the linear map A that
  made the images, and no other combination of the history does better;
* features: unit root mean square of the three solver columns, node and
  normal copied, float32;
* prediction and target are inverse to each other (a network that returns
  the normalised target reproduces the converged density), and the untrained
  network (zero output layer) leaves the projection form's start
  psi_F + 2 gamma r_F;
* normalisation moments against closed forms.
"""
import numpy as np

from kfbi_workloads import configs as C
from oracle import mlp, warmstart as WS


def _history(M=40, k=6, seed=0):
    rng = np.random.default_rng(seed)
    A = np.eye(M) * 0.5 + 0.1 * rng.standard_normal((M, M))     # second-kind-like operator
    P = rng.standard_normal((k, M))
    return A, P, P @ A.T


def test_projection_recovers_a_combination_exactly():
    A, P, B = _history()
    c = np.array([0.3, -1.2, 0.0, 2.0, 0.7, -0.1])
    psi = c @ P
    psi_F, r_F, cc = WS.projection(P, B, A @ psi)
    assert np.abs(psi_F - psi).max() < 1e-12 * np.abs(psi).max()
    assert np.abs(r_F).max() < 1e-12 * np.abs(A @ psi).max()
    assert np.abs(cc - c).max() < 1e-11


def test_projection_residual_is_orthogonal_and_exact():
    A, P, B = _history(seed=1)
    g = np.random.default_rng(9).standard_normal(A.shape[0])
    psi_F, r_F, c = WS.projection(P, B, g)
    assert np.abs(B @ r_F).max() < 1e-12 * np.linalg.norm(g) * np.abs(B).max()
    assert np.abs(r_F - (g - A @ psi_F)).max() < 1e-12
    rng = np.random.default_rng(2)
    for _ in range(20):
        c2 = c + 0.05 * rng.standard_normal(c.size)
        assert np.linalg.norm(g - c2 @ B) > np.linalg.norm(r_F)


def test_projection_without_history():
    g = np.arange(5.0)
    psi_F, r_F, c = WS.projection(np.zeros((0, 5)), np.zeros((0, 5)), g)
    assert np.all(psi_F == 0) and np.all(r_F == g) and c.size == 0


def test_features_scaling_and_columns():
    rng = np.random.default_rng(3)
    M = 50
    psi_F, r_F, g = 3.0 * rng.standard_normal((3, M))
    X, n = rng.standard_normal((M, 3)), rng.standard_normal((M, 3))
    F = WS.features(psi_F, r_F, g, X, n)
    assert F.dtype == np.float32 and F.shape == (M, 9)
    for j in range(3):
        assert abs(np.sqrt(np.mean(F[:, j].astype(np.float64) ** 2)) - 1.0) < 1e-6
    assert np.array_equal(F[:, 3:6], X.astype(np.float32)) and np.array_equal(F[:, 6:], n.astype(np.float32))
    assert np.allclose(F[:, 1] * np.sqrt(np.mean(r_F ** 2)), r_F, rtol=1e-6)


def test_target_and_prediction_are_inverse():
    rng = np.random.default_rng(4)
    M = 64
    psi, psi_F, r_F = rng.standard_normal((3, M))
    t = WS.target(psi, psi_F, r_F)
    norm = np.concatenate([np.zeros(9), np.ones(9), [0.25, 1.5]]).astype(np.float32)
    o = ((t - norm[18]) / norm[19]).astype(np.float32)
    back = WS.prediction(psi_F, r_F, o, norm)
    assert np.abs(back - psi).max() < 1e-5 * np.abs(psi).max()


def test_untrained_network_gives_the_projection_start():
    rng = np.random.default_rng(5)
    M = 30
    psi_F, r_F, g = rng.standard_normal((3, M))
    X, n = rng.standard_normal((M, 3)), rng.standard_normal((M, 3))
    norm = np.concatenate([np.zeros(9), np.ones(9), [0.0, 1.0]]).astype(np.float32)
    psi_L, o = WS.predict(mlp.init(0), norm, psi_F, r_F, g, X, n)
    assert np.all(o == 0.0)
    assert np.array_equal(psi_L, psi_F + 2.0 * 0.8 * r_F)


def test_fit_norm_closed_form():
    n = 101
    F = np.zeros((n, 9), np.float32)
    F[:, 0] = np.arange(n)                    # mean 50, sample variance n (n + 1) / 12
    F[:, 1] = 2.0
    T = np.linspace(-1.0, 1.0, n).astype(np.float32)
    norm = WS.fit_norm(F, T)
    assert abs(norm[0] - 50.0) < 1e-5
    assert abs(norm[9] - np.sqrt(n * (n + 1) / 12.0)) < 1e-4
    assert norm[1] == 2.0 and norm[10] == 1.0                 # zero spread -> 1
    assert abs(norm[18]) < 1e-7
    assert abs(norm[19] - np.sqrt((n * (n + 1) / 12.0) * (2.0 / (n - 1)) ** 2)) < 1e-6


def test_initial_parameters_are_he_uniform():
    p = C.mlp_init_params(0)
    ps = mlp.unpack(p)
    assert p.size == mlp.n_params()
    assert np.abs(ps[0]).max() <= np.sqrt(6.0 / 9) and np.abs(ps[2]).max() <= np.sqrt(6.0 / 128)
    assert np.all(ps[8] == 0) and all(np.all(ps[2 * l + 1] == 0) for l in range(5))
