"""Pins of the FitzHugh-Nagumo half steps and the Strang step (Sections 3, 7)."""
import numpy as np
import scipy.optimize

from kfbi_workloads import configs as C, geometry as G
from kfbi_workloads.configs import FHN_CONFIG as P, Grid
from oracle.bidomain import lam_of  # noqa: E402
from oracle import reaction
from oracle.bidomain import Bidomain, extracellular


def test_rest_state_is_fixed_point():
    z = np.zeros(5)
    V, q = reaction.forward_euler(z, z, 0.025, P)
    assert np.all(V == 0) and np.all(q == 0)
    V, q, ok = reaction.backward_euler(z, z, 0.025, P)
    assert np.all(V == 0) and np.all(q == 0) and ok.all()


def test_forward_euler_hand_values():
    V0, q0, k = np.array([0.5]), np.array([0.2]), 0.025
    # I_ion = 1 * (0.2 - 0.5 * 0.4 * 0.5) = 0.1 ; dV = -0.1 ; dq = 0.01*0.5 - 0.005*0.2 = 0.004
    V, q = reaction.forward_euler(V0, q0, k, P)
    assert abs(V[0] - (0.5 - 0.025 * 0.1)) < 1e-16
    assert abs(q[0] - (0.2 + 0.025 * 0.004)) < 1e-16


def test_backward_euler_against_brentq():
    rng = np.random.default_rng(0)
    V0 = rng.uniform(-0.3, 1.2, 40)
    q0 = rng.uniform(-0.1, 0.3, 40)
    for fhn in (P, C.FHN_PAPER):
        k = 0.025 if fhn is P else 0.0025
        V1, q1, ok = reaction.backward_euler(V0, q0, k, fhn)
        assert ok.all()
        den = 1 + k * fhn.zeta
        for i in range(V0.size):
            def F(v):
                qq = (q0[i] + k * fhn.alpha * v) / den
                return v - V0[i] + k * fhn.H / fhn.Cm * (qq - v * (v - fhn.theta) * (1 - v))
            # unique root near V0 for these step sizes
            root = scipy.optimize.brentq(F, V0[i] - 2.0, V0[i] + 2.0, xtol=1e-15)
            assert abs(V1[i] - root) < 1e-10
            assert abs(F(V1[i])) < 1e-12
        assert np.allclose(q1, (q0 + k * fhn.alpha * V1) / den, rtol=0, atol=1e-15)


def test_strang_zero_state_stays_zero_and_mean_zero_ue():
    geom, grid = G.ellipse_config0(64), Grid(2, 32)
    cfg = C.StrangConfig(steps=2)
    lam = lam_of(cfg, C.FHN_CONFIG)
    assert lam == 60.0
    bd = Bidomain(geom, grid, cfg, P)
    V = np.zeros(grid.shape)
    q = np.zeros(grid.shape)
    V1, q1, info = bd.step(V, q)
    assert np.abs(V1).max() == 0.0 and np.abs(q1).max() == 0.0
    V0 = C.ball_stimulus(grid, (-0.4, 0.0), 0.15)
    V1, q1, info = bd.step(V0, q)
    assert info["converged"] and info["newton_ok"]
    ue = extracellular(V1, bd.k.inside, 1.0, 2.0)
    assert abs(ue[bd.k.inside].mean()) < 1e-14
    # the implicit midpoint rule damps nothing at high frequency (amplification
    # -> -1), so a step stimulus overshoots; the values stay bounded by 1
    assert np.abs(V1).max() < 1.0


def test_strang_constant_state_diffusion_is_identity():
    """A constant V (with matching q) is unchanged by the diffusion solve:
    the Neumann problem Lap u - lam u = -lam c has u = c."""
    geom, grid = G.ellipse_config0(64), Grid(2, 32)
    cfg = C.StrangConfig(steps=1)
    bd = Bidomain(geom, grid, cfg, P)
    c = 0.3
    w, psi, info = bd.k.solve_neumann(-60.0 * c * np.ones(grid.shape), np.zeros(geom.M), 60.0, tol=1e-12)
    assert np.abs(w[bd.k.inside] - c).max() < 2e-3        # O(h^2) discretisation error only
