"""Strang-split FitzHugh-Nagumo bidomain step (oracle).

Section 3: reaction over dt/2 by forward Euler, diffusion over dt by the
implicit midpoint rule, reaction over dt/2 by backward Euler.  The midpoint
rule is computed as a backward-Euler step of dt/2 for w = (u^{n+1} + u^n)/2,
then u^{n+1} = 2 w - u^n.

With isotropic conductivities D_i = sigma_i I, D_e = sigma_e I and no
extracellular stimulus, the coupled system (Eq. pde1) with kappa = Cm beta/(dt/2)
decouples exactly: dividing by the conductivities and subtracting gives
    Lap V - lambda V = -lambda V^n,   lambda = kappa (1/sigma_i + 1/sigma_e),
with homogeneous Neumann data (both potentials are insulated), and adding
gives Lap(sigma_i Phi_i + sigma_e Phi_e) = 0, so sigma_i Phi_i + sigma_e Phi_e
is constant and the extracellular potential with zero mean over Omega is
    u_e = sigma_i (mean_Omega V - V) / (sigma_i + sigma_e).

The state (V, q) lives on every box node: the right-hand side -lambda V^n is
the continuous extension of the source to the box (Section 5.1) and the
diffusion result u = v_V + v_B is kept on all nodes.
"""
from __future__ import annotations

import numpy as np

from . import reaction
from .kfbi import KFBI


def extracellular(V, inside, sigma_i, sigma_e):
    mean = V[inside].mean()
    return sigma_i * (mean - V) / (sigma_i + sigma_e)


class Bidomain:
    def __init__(self, geom, grid, cfg, fhn, lam):
        self.k = KFBI(geom, grid)
        self.cfg, self.fhn, self.lam = cfg, fhn, lam
        self.psi_prev = np.zeros(geom.M)
        self.gN = np.zeros(geom.M)

    def step(self, V, q, psi0=None):
        """One Strang step; returns (V, q, stats).  psi0 is the GMRES initial
        guess (default: the previous step's density)."""
        cfg, fhn = self.cfg, self.fhn
        kk = cfg.dt / 2.0
        V, q = reaction.forward_euler(V, q, kk, fhn)
        x0 = self.psi_prev if psi0 is None else psi0
        w, psi, info = self.k.solve_neumann(-self.lam * V, self.gN, self.lam, tol=cfg.tol, psi0=x0)
        self.psi_prev = psi
        V = 2.0 * w - V
        V, q, ok = reaction.backward_euler(V, q, kk, fhn)
        info["newton_ok"] = bool(ok.all())
        return V, q, info
