"""Pointwise FitzHugh-Nagumo reaction half steps (oracle).

Model (Section 7): I_ion(V, q) = H (q - V (V - theta)(1 - V)),
M(V, q) = alpha V - zeta q, with Cm dV/dt = -I_ion, dq/dt = M.

* Step 1 of the Strang splitting (Eq. ode1): forward Euler over dt/2.
* Step 3 (Eq. ode2): backward Euler over dt/2.  q enters linearly, so
  q1 = (q0 + k alpha V1) / (1 + k zeta) and V1 solves the scalar cubic
      F(V) = V - V0 - (k H / Cm) (V (V - theta)(1 - V) - q1(V)) = 0
  by Newton's method from V0 with absolute tolerance 1e-10 on the update
  (Section 7) and at most 50 iterations.
"""
from __future__ import annotations

import numpy as np

NEWTON_TOL = 1e-10
NEWTON_MAX = 50


def forward_euler(V, q, k, fhn):
    cubic = V * (V - fhn.theta) * (1.0 - V)
    Iion = fhn.H * (q - cubic)
    Vn = V + k * (-Iion / fhn.Cm)
    qn = q + k * (fhn.alpha * V - fhn.zeta * q)
    return Vn, qn


def backward_euler(V0, q0, k, fhn):
    """Returns (V1, q1, ok) where ok flags Newton convergence per node."""
    c = k * fhn.H / fhn.Cm
    den = 1.0 + k * fhn.zeta
    r = k * fhn.alpha / den
    V = V0.copy()
    ok = np.zeros(V.shape, dtype=bool)
    for _ in range(NEWTON_MAX):
        q1 = (q0 + k * fhn.alpha * V) / den
        cubic = V * (V - fhn.theta) * (1.0 - V)
        F = V - V0 - c * (cubic - q1)
        dcubic = -3.0 * V * V + 2.0 * (1.0 + fhn.theta) * V - fhn.theta
        dF = 1.0 - c * (dcubic - r)
        dV = F / dF
        V = np.where(ok, V, V - dV)
        ok |= np.abs(dV) < NEWTON_TOL
        if ok.all():
            break
    q1 = (q0 + k * fhn.alpha * V) / den
    return V, q1, ok
