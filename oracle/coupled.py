"""Anisotropic coupled bidomain system (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The backward-Euler half step of the diffusion with diagonal conductivity
tensors D_i = diag(d_i), D_e = diag(d_e) (fibres along the axes, Section 5.2)
is the vector Neumann problem of Eqs. pde1 / bvp,

    div(D_i grad Phi_i) - kappa (Phi_i - Phi_e) = f_i,
    div(D_e grad Phi_e) + kappa (Phi_i - Phi_e) = f_e,   n.D_c grad Phi_c = g_c,

with kappa = Cm beta / (dt/2), f = (-kappa V*, kappa V* - beta I_stim).  The
KFBI method of Sections 4-5 applies component by component with the vector
density psi = (psi_i, psi_e):

* box solve (Section 5.2, Eq. FDE with sigma, eta per axis): each second
  difference along axis a, scaled by d_a, is diagonalised by the sine
  transform, leaving per mode p the 2 x 2 system
      [A_i(p) - kappa, kappa; kappa, A_e(p) - kappa] (v_i, v_e) = (r_i, r_e),
      A_c(p) = sum_a d_c,a mu1(p_a),  mu1(p) = -(4/h^2) sin^2(pi p / (2N));
* jumps of the single layer of one component with conductivity D (its
  interface conditions: [v] = 0, n.D[grad v] = psi, and the PDE jump
  [div(D grad v)] - kappa-terms = 0, the kappa-terms vanishing with [v]):
      [grad v] = alpha n,           alpha = psi / q,  q = n.D n,
      grad_G alpha = grad_G psi / q - 2 psi S D n / q^2,
      [D^2 v] = alpha S + n (grad_G alpha)^T + (grad_G alpha) n^T + c n n^T,
      c = -(alpha tr(D S) + 2 n.D grad_G alpha) / q,
  with S the shape operator (d n / d t = S t for tangent t).  These follow
  from differentiating [v] = 0 twice along the surface and from
  tr(D [D^2 v]) = 0; the paper defers them to its references.  With D = I
  they reduce to the isotropic relations of oracle.kfbi;
* correction (Section 5.3, Eq. correct): the corrections of the component
  carry the conductivity of the crossing's axis, RHS(p) -+= d_a J(p') / h^2;
* limits (Section 5.4): A psi = n.D grad v_B^+ (the conormal derivative) per
  component, from the same Taylor systems, points outside Omega shifted by
  the component's jump polynomial.

The coupled Neumann problem determines (Phi_i, Phi_e) only up to a common
constant: constants solve the homogeneous system, and the range of A is
orthogonal to (ds, ds) (the sum of the two rows integrates to zero).  As for
the Poisson problem of oracle.kfbi, every application of A adds the
rank-one term (1, 1) <(ds, ds), psi> / (2 |Gamma|), which has the same
solutions for compatible data; V = Phi_i - Phi_e is unaffected.

Reading for the Strang step (the paper is silent on the level at which
Phi_e is reported): the extracellular potential of a step is the coupled
solve's Phi_e (at the midpoint level t^n + dt/2), with zero mean over Omega.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

from . import boxsolve, krylov, reaction
from .kfbi import KFBI

WORKERS = boxsolve.WORKERS


def jump_grad_hess(psi, gpsi, n, S, D):
    """[grad v] [P, d] and [D^2 v] [P, d, d] of one component with diagonal
    conductivity D [d] from psi [P], grad_Gamma psi [P, d], normals n [P, d]
    and shape operators S [P, d, d]."""
    D = np.asarray(D, dtype=np.float64)
    Dn = n * D[None, :]
    q = (n * Dn).sum(axis=1)
    alpha = psi / q
    SDn = np.einsum("pij,pj->pi", S, Dn)
    galpha = gpsi / q[:, None] - (2.0 * psi / (q * q))[:, None] * SDn
    trDS = np.einsum("i,pii->p", D, S)
    c = -(alpha * trDS + 2.0 * (Dn * galpha).sum(axis=1)) / q
    jg = alpha[:, None] * n
    ng = n[:, :, None] * galpha[:, None, :]
    jH = (alpha[:, None, None] * S + ng + ng.transpose(0, 2, 1)
          + c[:, None, None] * n[:, :, None] * n[:, None, :])
    return jg, jH


class CoupledKFBI:
    """Setup and integral evaluations of the coupled system for one geometry,
    grid and pair of diagonal conductivities."""

    def __init__(self, geom, grid, Di, De):
        self.k = KFBI(geom, grid)
        self.geom, self.grid = geom, grid
        self.d = grid.dim
        self.D = [np.asarray(Di, dtype=np.float64)[:self.d], np.asarray(De, dtype=np.float64)[:self.d]]
        self.M = geom.M

    # --------------------------------------------------------- box solve
    def mode_sums(self):
        """A_i(p), A_e(p) on the mode grid ([z][y][x] layout)."""
        g = self.grid
        p = np.arange(1, g.N, dtype=np.float64)
        m1 = -(4.0 / g.h ** 2) * np.sin(np.pi * p / (2.0 * g.N)) ** 2
        out = []
        for D in self.D:
            if self.d == 2:
                out.append(D[0] * m1[None, :] + D[1] * m1[:, None])
            else:
                out.append(D[0] * m1[None, None, :] + D[1] * m1[None, :, None] + D[2] * m1[:, None, None])
        return out

    def box_solve(self, ri, re, kappa):
        """(v_i, v_e) = L_h^{-1} (r_i, r_e), zero Dirichlet data on the box."""
        Ai, Ae = self.mode_sums()
        a, c, b = Ai - kappa, Ae - kappa, kappa
        det = a * c - b * b
        hi = scipy.fft.dstn(ri, type=1, workers=WORKERS)
        he = scipy.fft.dstn(re, type=1, workers=WORKERS)
        vi = (c * hi - b * he) / det
        ve = (a * he - b * hi) / det
        s = (2.0 * self.grid.N) ** self.d
        return (scipy.fft.dstn(vi, type=1, workers=WORKERS) / s, scipy.fft.dstn(ve, type=1, workers=WORKERS) / s)

    def apply_L(self, vi, ve, kappa):
        """The coupled 5/7-point operator with zero Dirichlet data (pins)."""
        out = []
        for c, (v, D) in enumerate(zip((vi, ve), self.D)):
            P = np.pad(v, 1)
            acc = np.zeros_like(v)
            for a in range(self.d):
                ax = self.d - 1 - a
                sm, sp = [slice(1, -1)] * self.d, [slice(1, -1)] * self.d
                sm[ax], sp[ax] = slice(0, -2), slice(2, None)
                acc = acc + D[a] * (P[tuple(sm)] + P[tuple(sp)] - 2.0 * v) / self.grid.h ** 2
            out.append(acc)
        w = kappa * (vi - ve)
        return out[0] - w, out[1] + w

    # ------------------------------------------------------ jumps, rows
    def jumps(self, psi, D):
        """Crossing jumps ([d_a v], [d_aa v]) and node jumps ([grad v],
        [D^2 v]) of one component."""
        k = self.k
        p_int, g_int, g_node = k.density(psi)
        jg_i, jH_i = jump_grad_hess(p_int, g_int, k.n_int, k.S_int, D)
        a = k.ints["axis"]
        r = np.arange(a.size)
        jg_n, jH_n = jump_grad_hess(psi, g_node, k.n_node, k.S_node, D)
        return (jg_i[r, a], jH_i[r, a, a]), (jg_n, jH_n)

    def correction(self, dv, ddv, D):
        """Corrections of one component: those of oracle.kfbi with the
        conductivity of each crossing's axis."""
        scale = D[self.k.ints["axis"]]
        return self.k.correction(np.zeros_like(dv), scale * dv, scale * ddv)

    def interp(self, v, D, node_jumps=None):
        """Conormal limit n.D grad v^+ at the interface nodes."""
        k = self.k
        vals = v.ravel()[k.st_flat].copy()
        if node_jumps is not None:
            jg, jH = node_jumps
            xi = k.st_xi
            J = np.einsum("mpd,md->mp", xi, jg) + 0.5 * np.einsum("mpd,mde,mpe->mp", xi, jH, xi)
            vals = vals + np.where(k.st_out, J, 0.0)
        coef = np.linalg.solve(k.st_A, vals[:, :, None])[:, :, 0]
        grad = coef[:, 1:1 + self.d] / self.grid.h
        return (grad * D[None, :] * k.n_node).sum(axis=1)

    # --------------------------------------------------------- operators
    def rank_one(self, psi2):
        ds = self.k.ds
        M = self.M
        return (ds @ psi2[:M] + ds @ psi2[M:]) / (2.0 * self.k.area)

    def single_layer(self, psi2, kappa):
        """v_B of the density pair and the node jumps of both components."""
        M = self.M
        rhs, nj = [], []
        for c in range(2):
            (dv, ddv), jn = self.jumps(psi2[c * M:(c + 1) * M], self.D[c])
            rhs.append(self.correction(dv, ddv, self.D[c]))
            nj.append(jn)
        return self.box_solve(rhs[0], rhs[1], kappa), nj

    def apply_A(self, psi2, kappa):
        """A psi (conormal limits of the single layer of both components)
        plus the rank-one term."""
        (vi, ve), nj = self.single_layer(psi2, kappa)
        out = np.concatenate([self.interp(vi, self.D[0], nj[0]), self.interp(ve, self.D[1], nj[1])])
        return out + self.rank_one(psi2)

    def rhs_g(self, fi, fe, gNi, gNe, kappa):
        vi, ve = self.box_solve(fi, fe, kappa)
        g = np.concatenate([gNi - self.interp(vi, self.D[0]), gNe - self.interp(ve, self.D[1])])
        return g, (vi, ve)

    def solve_neumann(self, fi, fe, gNi, gNe, kappa, tol=1e-10, psi0=None, restart=50, max_iter=500):
        """(Phi_i, Phi_e, psi, stats) of the coupled Neumann problem."""
        g, (vVi, vVe) = self.rhs_g(fi, fe, gNi, gNe, kappa)
        x0 = np.zeros(2 * self.M) if psi0 is None else np.asarray(psi0, dtype=np.float64)
        psi, info = krylov.gmres(lambda x: self.apply_A(x, kappa), g, x0, tol, restart=restart, max_iter=max_iter)
        (vBi, vBe), nj = self.single_layer(psi, kappa)
        ui, ue = vVi + vBi, vVe + vBe
        r = np.concatenate([gNi - self.interp(ui, self.D[0], nj[0]), gNe - self.interp(ue, self.D[1], nj[1])])
        r = r - self.rank_one(psi)
        gn = np.linalg.norm(g)
        info["true_rel_res"] = float(np.linalg.norm(r) / gn) if gn > 0 else float(np.linalg.norm(r))
        return ui, ue, psi, info


def kappa_of(dt, fhn):
    """kappa of Eq. pde1 for the midpoint's backward-Euler half step."""
    return fhn.Cm * fhn.beta / (dt / 2.0)


class CoupledBidomain:
    """Strang steps (Section 3) with the coupled anisotropic diffusion step."""

    def __init__(self, geom, grid, Di, De, dt, fhn, tol=1e-10, istim=None):
        self.c = CoupledKFBI(geom, grid, Di, De)
        self.dt, self.fhn, self.tol, self.istim = dt, fhn, tol, istim
        self.kappa = kappa_of(dt, fhn)
        self.psi = np.zeros(2 * geom.M)
        self.zero = np.zeros(geom.M)

    def step(self, V, q):
        """One Strang step; returns (V, q, u_e, stats)."""
        k = self.dt / 2.0
        fhn, kap = self.fhn, self.kappa
        V, q = reaction.forward_euler(V, q, k, fhn)
        fi, fe = -kap * V, kap * V
        if self.istim is not None:
            fe = fe - fhn.beta * self.istim
        Pi, Pe, self.psi, info = self.c.solve_neumann(fi, fe, self.zero, self.zero, kap, tol=self.tol,
                                                      psi0=self.psi)
        w = Pi - Pe
        V = 2.0 * w - V
        V, q, ok = reaction.backward_euler(V, q, k, fhn)
        ins = self.c.k.inside
        ue = Pe - Pe[ins].mean()
        info["newton_ok"] = bool(ok.all())
        info["w"] = w
        return V, q, ue, info
