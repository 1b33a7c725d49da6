"""Pins of the oracle's Strang step (Section 3) by what the mathematics fixes.

* Sub-step order: with the diffusion solve replaced by its exact result for a
  state that diffusion leaves unchanged (w = V), one step is forward Euler
  over dt/2 followed by backward Euler over dt/2 (Eqs. ode1, ode2), i.e. the
  trapezoidal rule y1 - y0 = (dt/2)(f(y0) + f(y1)) of the reaction ODE, to
  the Newton tolerance.  Swapping the two half steps breaks it.
* Implicit midpoint and lambda: on a disk with the reaction switched off,
  V^n = J0(k r) with J1(k R) = 0 is a Neumann eigenfunction of the Laplacian
  (Lap V = -k^2 V, dV/dn = 0).  The backward-Euler half step
  Lap w - lambda w = -lambda V^n then gives w = lambda/(lambda + k^2) V^n and
  the midpoint V^{n+1} = 2 w - V^n = (lambda - k^2)/(lambda + k^2) V^n, with
  lambda = (Cm beta/(dt/2))(1/sigma_i + 1/sigma_e) from Eq. pde1.  The
  oracle's step must reproduce that factor at second order in h; taking V =
  w, or kappa = Cm beta / dt, misses it by O(1).
* Extracellular potential: the sum of the two rows of Eq. pde1 without a
  stimulus is Lap(sigma_i Phi_i + sigma_e Phi_e) = 0, with Phi_i = u_e + V and
  Phi_e = u_e; the reported u_e also has zero mean over Omega.  Putting
  sigma_e in the numerator breaks the first relation.
"""
import math

import numpy as np
import pytest
import scipy.special

from kfbi_workloads import configs as C, geometry as G
from kfbi_workloads.configs import Grid
from oracle import bidomain as BD, reaction
from oracle.bidomain import Bidomain, extracellular


def _f(V, q, fhn):
    """Right-hand side of the FitzHugh-Nagumo ODE (Section 7)."""
    return (fhn.H / fhn.Cm) * (V * (V - fhn.theta) * (1.0 - V) - q), fhn.alpha * V - fhn.zeta * q


def _stub_diffusion(bd):
    bd.diffuse = lambda V, psi0=None: (V.copy(), {"converged": True, "iters": 0})


def _trapezoid_defect(bd, fhn, dt):
    rng = np.random.default_rng(3)
    V0 = rng.uniform(-0.2, 1.1, bd.k.inside.shape)
    q0 = rng.uniform(-0.05, 0.2, V0.shape)
    V1, q1, info = bd.step(V0, q0)
    fV0, fq0 = _f(V0, q0, fhn)
    fV1, fq1 = _f(V1, q1, fhn)
    k = dt / 2.0
    return max(np.abs(V1 - V0 - k * (fV0 + fV1)).max(), np.abs(q1 - q0 - k * (fq0 + fq1)).max())


@pytest.mark.parametrize("fhn", [C.FHN_CONFIG, C.FHN_PAPER], ids=["config", "paper"])
def test_strang_sub_steps_are_trapezoidal(fhn):
    geom, grid = G.ellipse_config0(64), Grid(2, 32)
    cfg = C.StrangConfig(dt=0.05 if fhn is C.FHN_CONFIG else 0.004, steps=1)
    bd = Bidomain(geom, grid, cfg, fhn)
    _stub_diffusion(bd)
    # Newton stops at |dV| < 1e-10; the trapezoid holds to that times (1 + k|f'|)
    assert _trapezoid_defect(bd, fhn, cfg.dt) < 1e-9


def test_strang_sub_step_swap_is_detected(monkeypatch):
    fe, be = reaction.forward_euler, reaction.backward_euler
    monkeypatch.setattr(BD.reaction, "forward_euler", lambda V, q, k, p: be(V, q, k, p)[:2])
    monkeypatch.setattr(BD.reaction, "backward_euler", lambda V, q, k, p: (*fe(V, q, k, p), np.ones(V.shape, bool)))
    geom, grid = G.ellipse_config0(64), Grid(2, 32)
    cfg = C.StrangConfig(dt=0.05, steps=1)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    _stub_diffusion(bd)
    assert _trapezoid_defect(bd, C.FHN_CONFIG, cfg.dt) > 1e-6


NO_REACTION = C.FHN(H=0.0, theta=0.1, alpha=0.0, zeta=0.0, Cm=1.0, beta=1.0)
R_DISK = 0.6


def _bessel_errors(plant=None):
    """Max error of one Strang step from V^n = J0(k r) against the closed-form
    factor, inside the disk, at N = 32 and 64."""
    k = scipy.special.jn_zeros(1, 1)[0] / R_DISK      # J0'(k R) = -J1(k R) = 0
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=1, tol=1e-12)
    # lambda from its definition, written out here: kappa = Cm beta / (dt/2)
    lam = (1.0 * 1.0 / (cfg.dt / 2.0)) * (1.0 / cfg.sigma_i + 1.0 / cfg.sigma_e)
    factor = (lam - k * k) / (lam + k * k)
    errs = []
    for N in (32, 64):
        geom, grid = G.disk2(R_DISK, 2 * N), Grid(2, N)
        x, y = grid.coords()
        Vn = scipy.special.j0(k * np.hypot(x, y)) * np.ones(grid.shape)
        bd = Bidomain(geom, grid, cfg, NO_REACTION)
        if plant == "V=w":
            solve = bd.diffuse
            # a returned w' = (w + V)/2 turns V = 2 w' - V^n into V = w
            bd.diffuse = lambda V, psi0=None: ((solve(V, psi0)[0] + V) / 2.0, {"converged": True})
        V1, q1, info = bd.step(Vn, np.zeros(grid.shape))
        ins = bd.k.inside
        errs.append(np.abs(V1 - factor * Vn)[ins].max())
    return errs, factor


def test_midpoint_and_lambda_against_bessel_eigenfunction():
    errs, factor = _bessel_errors()
    assert 0.1 < factor < 0.3                       # a non-trivial factor
    assert errs[1] < 2e-3 and errs[0] / errs[1] > 3.0, errs


def test_midpoint_planted_backward_euler_is_detected():
    errs, factor = _bessel_errors(plant="V=w")
    assert errs[1] > 0.3


def test_lambda_planted_full_step_kappa_is_detected(monkeypatch):
    monkeypatch.setattr(BD, "helmholtz_lambda",
                        lambda si, se, dt, Cm, beta: (Cm * beta / dt) * (1.0 / si + 1.0 / se))
    errs, factor = _bessel_errors()
    assert errs[1] > 0.05


def _ue_defects(ue_fn):
    geom, grid = G.ellipse_config0(128), Grid(2, 64)
    cfg = C.StrangConfig(steps=1, tol=1e-12)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V1, q1, info = bd.step(C.ball_stimulus(grid, (-0.4, 0.0), 0.15), np.zeros(grid.shape))
    ue = ue_fn(V1, bd.k.inside, cfg.sigma_i, cfg.sigma_e)
    T = cfg.sigma_i * (ue + V1) + cfg.sigma_e * ue
    lap = (T[1:-1, 2:] + T[1:-1, :-2] + T[2:, 1:-1] + T[:-2, 1:-1] - 4.0 * T[1:-1, 1:-1]) / grid.h ** 2
    reg = bd.k.inside.copy()
    reg.ravel()[bd.k.irregular] = False
    scale = np.abs(V1).max() / grid.h ** 2
    return np.abs(lap[reg[1:-1, 1:-1]]).max() / scale, abs(ue[bd.k.inside].mean())


def test_extracellular_satisfies_summed_rows():
    lap, mean = _ue_defects(extracellular)
    assert lap < 1e-13 and mean < 1e-14


def test_extracellular_planted_sigma_e_is_detected():
    def planted(V, inside, si, se):
        return se * (V[inside].mean() - V) / (si + se)
    lap, mean = _ue_defects(planted)
    assert lap > 1e-4


def test_helmholtz_lambda_reads_eq_pde1():
    # kappa = Cm beta / (dt/2) of the midpoint's backward-Euler half step, and
    # the isotropic elimination divides Eq. pde1's rows by sigma_i and sigma_e
    assert math.isclose(BD.helmholtz_lambda(1.0, 2.0, 0.05, 1.0, 1.0), 60.0, rel_tol=1e-15)
    assert math.isclose(BD.helmholtz_lambda(2.0, 2.0, 0.1, 3.0, 0.5), 30.0, rel_tol=1e-15)
