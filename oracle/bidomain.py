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

With the extracellular stimulus I_stim of the virtual electrode (Section 7),
the same elimination of Eq. pde1 gives
    Lap V - lambda V = -lambda V^n + beta I_stim / sigma_e,
    Lap S = -beta I_stim,   S = sigma_i Phi_i + sigma_e Phi_e,
both with homogeneous Neumann data; the S problem is a Poisson problem
(lambda = 0, solved with the rank-one modification of the boundary operator)
whose right-hand side does not change with time, so it is solved once.  Then
Phi_e = (S - sigma_i V) / (sigma_i + sigma_e), reported with zero mean over
Omega.
"""
from __future__ import annotations

import numpy as np

from . import reaction
from .kfbi import KFBI


def helmholtz_lambda(sigma_i, sigma_e, dt, Cm, beta):
    """lambda of the decoupled transmembrane problem of the implicit-midpoint
    half step (Section 3): the backward-Euler step over dt/2 gives
    kappa = Cm beta / (dt/2) in Eq. pde1, and dividing its rows by the
    conductivities and subtracting gives Lap V - lambda V = -lambda V^n with
    lambda = kappa (1/sigma_i + 1/sigma_e)."""
    kappa = Cm * beta / (dt / 2.0)
    return kappa * (1.0 / sigma_i + 1.0 / sigma_e)


def lam_of(cfg, fhn):
    """helmholtz_lambda of a workload (conductivities and dt) and membrane."""
    return helmholtz_lambda(cfg.sigma_i, cfg.sigma_e, cfg.dt, fhn.Cm, fhn.beta)


def extracellular(V, inside, sigma_i, sigma_e):
    mean = V[inside].mean()
    return sigma_i * (mean - V) / (sigma_i + sigma_e)


def extracellular_S(V, S, inside, sigma_i, sigma_e):
    """Phi_e = (S - sigma_i V) / (sigma_i + sigma_e) with zero mean over Omega."""
    phi = (S - sigma_i * V) / (sigma_i + sigma_e)
    return phi - phi[inside].mean()


class Bidomain:
    def __init__(self, geom, grid, cfg, fhn, istim=None):
        self.k = KFBI(geom, grid)
        self.cfg, self.fhn = cfg, fhn
        self.lam = helmholtz_lambda(cfg.sigma_i, cfg.sigma_e, cfg.dt, fhn.Cm, fhn.beta)
        self.psi_prev = np.zeros(geom.M)
        self.gN = np.zeros(geom.M)
        self.istim = istim
        self.S = None
        self.S_info = None

    def solve_S(self):
        """The Poisson problem Lap S = -beta I_stim with homogeneous Neumann data."""
        if self.S is None:
            self.S, _, self.S_info = self.k.solve_neumann(-self.fhn.beta * self.istim, self.gN, 0.0,
                                                          tol=self.cfg.tol)
        return self.S

    def diffuse(self, V, psi0=None):
        """Backward-Euler half step of the diffusion (the midpoint's w)."""
        cfg, fhn = self.cfg, self.fhn
        x0 = self.psi_prev if psi0 is None else psi0
        f = -self.lam * V
        if self.istim is not None:
            f = f + (fhn.beta / cfg.sigma_e) * self.istim
        w, psi, info = self.k.solve_neumann(f, self.gN, self.lam, tol=cfg.tol, psi0=x0)
        self.psi_prev = psi
        return w, info

    def step(self, V, q, psi0=None):
        """One Strang step; returns (V, q, stats).  psi0 is the GMRES initial
        guess (default: the previous step's density)."""
        cfg, fhn = self.cfg, self.fhn
        kk = cfg.dt / 2.0
        V, q = reaction.forward_euler(V, q, kk, fhn)
        w, info = self.diffuse(V, psi0)
        V = 2.0 * w - V
        V, q, ok = reaction.backward_euler(V, q, kk, fhn)
        info["newton_ok"] = bool(ok.all())
        return V, q, info
