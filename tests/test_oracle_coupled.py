"""Pins of the anisotropic coupled oracle (Eqs. pde1, FDE, correct; Section 5).

* box solve: inverts the coupled 5/7-point operator of Eq. FDE (diagonal
  conductivities per axis, coupling kappa) assembled as a dense matrix and
  LU-solved, 2-D and 3-D;
* jump relations of one component, by the properties that define them, on
  an ellipse and an ellipsoid with anisotropic D: symmetric, conormal jump
  n.D[grad v] = psi, PDE jump tr(D [D^2 v]) = 0, and the tangential
  derivative of [grad v] along the surface (finite differences of alpha n
  along an analytic parametrisation) equal to [D^2 v] t; dropping the
  n n^T term breaks the PDE jump; with D = sigma I they are those of the
  isotropic oracle divided by sigma;
* GMRES on the coupled A against a dense LU solve of A assembled column by
  column;
* second-order convergence on manufactured anisotropic solutions (the
  unique parts: Phi_i - Phi_e and Phi_e up to its mean);
* with isotropic conductivities the coupled Strang step reproduces the
  decoupled oracle's V (Section 3 elimination) and its Phi_e is the
  decoupled u_e of the midpoint state, to solver tolerance.
"""
import math

import numpy as np
import pytest

from kfbi_workloads import configs as C, geometry as G
from kfbi_workloads.configs import Grid
from oracle import coupled as CP, levelset as LS, krylov
from oracle.bidomain import Bidomain
from oracle.kfbi import KFBI

DI = (3.0, 0.5, 0.5)   # the paper's diag(30, 5[, 5]) and diag(20, 10[, 10]), scaled by 1/10
DE = (2.0, 1.0, 1.0)


@pytest.mark.parametrize("dim,N", [(2, 12), (3, 6)])
def test_box_solve_inverts_dense_operator(dim, N):
    geom = G.ellipse_config0(32) if dim == 2 else G.sphere3(0.4, 2)
    grid = Grid(dim, N)
    c = CP.CoupledKFBI.__new__(CP.CoupledKFBI)
    c.grid, c.d = grid, dim
    c.D = [np.asarray(DI[:dim]), np.asarray(DE[:dim])]
    kappa = 7.0
    n = (N - 1) ** dim
    Lm = np.zeros((2 * n, 2 * n))
    for j in range(2 * n):
        e = np.zeros(2 * n)
        e[j] = 1.0
        vi, ve = c.apply_L(e[:n].reshape(grid.shape), e[n:].reshape(grid.shape), kappa)
        Lm[:, j] = np.concatenate([vi.ravel(), ve.ravel()])
    rng = np.random.default_rng(dim)
    r = rng.standard_normal(2 * n)
    x = np.linalg.solve(Lm, r)
    vi, ve = c.box_solve(r[:n].reshape(grid.shape), r[n:].reshape(grid.shape), kappa)
    assert np.abs(np.concatenate([vi.ravel(), ve.ravel()]) - x).max() < 1e-12 * np.abs(x).max()
    # one row of Eq. FDE written out at an interior node (2-D: s, t sums)
    if dim == 2:
        Pi = rng.standard_normal(grid.shape)
        Pe = rng.standard_normal(grid.shape)
        li, le = c.apply_L(Pi, Pe, kappa)
        k, l, h = 4, 5, grid.h
        s = DI[0] * (Pi[l, k + 1] + Pi[l, k - 1]) + DI[1] * (Pi[l + 1, k] + Pi[l - 1, k])
        t = DE[0] * (Pe[l, k + 1] + Pe[l, k - 1]) + DE[1] * (Pe[l + 1, k] + Pe[l - 1, k])
        ri = (s - 2 * DI[0] * Pi[l, k] - 2 * DI[1] * Pi[l, k]) / h ** 2 - kappa * Pi[l, k] + kappa * Pe[l, k]
        re = (t - 2 * DE[0] * Pe[l, k] - 2 * DE[1] * Pe[l, k]) / h ** 2 + kappa * Pi[l, k] - kappa * Pe[l, k]
        assert abs(li[l, k] - ri) < 1e-10 and abs(le[l, k] - re) < 1e-10


def _ellipse_point(t, a=0.7, b=0.45):
    cs, sn = math.sqrt(3) / 2, 0.5
    x, y = a * np.cos(t), b * np.sin(t)
    P = np.stack([cs * x - sn * y, sn * x + cs * y], axis=-1)
    dx, dy = -a * np.sin(t), b * np.cos(t)
    T = np.stack([cs * dx - sn * dy, sn * dx + cs * dy], axis=-1)
    return P, T


def _psi_fn(P):
    return 1.0 + 0.4 * P[..., 0] - 0.7 * P[..., 1] ** 2 + (0.3 * P[..., 2] if P.shape[-1] == 3 else 0.0)


def _psi_grad(P):
    g = np.zeros_like(P)
    g[..., 0] = 0.4
    g[..., 1] = -1.4 * P[..., 1]
    if P.shape[-1] == 3:
        g[..., 2] = 0.3
    return g


def _jump_properties(geom, P, tangents, D, jump_fn=CP.jump_grad_hess):
    """Max defects of the defining properties at surface points P with unit
    tangent fields tangents(P) -> list of (T [P, d], dP/ds function)."""
    D = np.asarray(D)
    n, S = LS.normal_shape(geom, 0, P)
    gfull = _psi_grad(P)
    gpsi = gfull - (gfull * n).sum(1)[:, None] * n
    psi = _psi_fn(P)
    jg, jH = jump_fn(psi, gpsi, n, S, D)
    sym = np.abs(jH - jH.transpose(0, 2, 1)).max()
    conormal = np.abs((n * D[None, :] * jg).sum(1) - psi).max()
    pde = np.abs(np.einsum("i,pii->p", D, jH)).max() / np.abs(jH).max()
    tang = 0.0
    for T, move in tangents:
        eps = 1e-5
        vals = []
        for sgn in (1.0, -1.0):
            Q = move(sgn * eps)
            nq, Sq = LS.normal_shape(geom, 0, Q)
            gq = _psi_grad(Q)
            gq = gq - (gq * nq).sum(1)[:, None] * nq
            vals.append(jump_fn(_psi_fn(Q), gq, nq, Sq, D)[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        tang = max(tang, np.abs(fd - np.einsum("pij,pj->pi", jH, T)).max() / np.abs(jH).max())
    return sym, conormal, pde, tang


def _ellipse_case():
    geom = G.ellipse_config0(64)
    t0 = np.linspace(0.1, 2 * np.pi, 23)
    P, T = _ellipse_point(t0)
    sp = np.linalg.norm(T, axis=1)

    def move(ds):
        # arc-length step ds along the curve: dt = ds / |X_t|
        return _ellipse_point(t0 + ds / sp)[0]
    return geom, P, [(T / sp[:, None], move)]


def _ellipsoid_case():
    ax = np.array([0.7, 0.5, 0.45])
    geom = G.ellipsoid3(*ax, 4)
    th, ph = np.meshgrid(np.linspace(0.3, 2.8, 5), np.linspace(0.2, 6.0, 6))
    th, ph = th.ravel(), ph.ravel()

    def X(a, b):
        return np.stack([ax[0] * np.sin(a) * np.cos(b), ax[1] * np.sin(a) * np.sin(b), ax[2] * np.cos(a)], 1)
    P = X(th, ph)
    Xt = np.stack([ax[0] * np.cos(th) * np.cos(ph), ax[1] * np.cos(th) * np.sin(ph), -ax[2] * np.sin(th)], 1)
    Xp = np.stack([-ax[0] * np.sin(th) * np.sin(ph), ax[1] * np.sin(th) * np.cos(ph), 0 * th], 1)
    lt, lp = np.linalg.norm(Xt, axis=1), np.linalg.norm(Xp, axis=1)
    return geom, P, [(Xt / lt[:, None], lambda ds: X(th + ds / lt, ph)), (Xp / lp[:, None], lambda ds: X(th, ph + ds / lp))]


@pytest.mark.parametrize("case", ["ellipse", "ellipsoid"])
def test_jump_relations_defining_properties(case):
    geom, P, tans = _ellipse_case() if case == "ellipse" else _ellipsoid_case()
    D = DI[:P.shape[1]]
    sym, conormal, pde, tang = _jump_properties(geom, P, tans, D)
    assert sym < 1e-13 and conormal < 1e-13 and pde < 1e-13, (sym, conormal, pde)
    assert tang < 1e-6, tang


def test_jump_relations_planted_isotropic_normal_term_is_detected():
    """Taking the isotropic n n^T coefficient (-alpha tr S) with an
    anisotropic D breaks the PDE jump."""
    def planted(psi, gpsi, n, S, D):
        jg, jH = CP.jump_grad_hess(psi, gpsi, n, S, D)
        alpha = psi / (n * np.asarray(D)[None, :] * n).sum(1)
        c_full = np.einsum("pij,pi,pj->p", jH, n, n)
        c_iso = -alpha * np.trace(S, axis1=1, axis2=2)
        return jg, jH + (c_iso - c_full)[:, None, None] * n[:, :, None] * n[:, None, :]
    geom, P, tans = _ellipse_case()
    sym, conormal, pde, tang = _jump_properties(geom, P, tans, DI[:2], jump_fn=planted)
    assert pde > 1e-3


def test_jump_relations_reduce_to_isotropic():
    geom, P, _ = _ellipsoid_case()
    n, S = LS.normal_shape(geom, 0, P)
    g = _psi_grad(P)
    g = g - (g * n).sum(1)[:, None] * n
    psi = _psi_fn(P)
    jg, jH = CP.jump_grad_hess(psi, g, n, S, (2.5, 2.5, 2.5))
    jg0, jH0 = KFBI.jump_grad_hess(psi, g, n, S)
    assert np.abs(jg - jg0 / 2.5).max() < 1e-14 and np.abs(jH - jH0 / 2.5).max() < 1e-12


def test_gmres_matches_dense_lu():
    geom, grid = G.ellipse_config0(20), Grid(2, 16)
    c = CP.CoupledKFBI(geom, grid, DI[:2], DE[:2])
    kappa = 40.0
    M2 = 2 * geom.M
    A = np.stack([c.apply_A(e, kappa) for e in np.eye(M2)], axis=1)
    g = np.random.default_rng(4).standard_normal(M2)
    x_ref = np.linalg.solve(A, g)
    x, info = krylov.gmres(lambda v: c.apply_A(v, kappa), g, np.zeros(M2), 1e-13, restart=50, max_iter=200)
    assert info["converged"]
    assert np.abs(x - x_ref).max() < 1e-9 * np.abs(x_ref).max()


def _manufactured(geom, grid, kappa, D_i, D_e):
    """Phi_i = cos(pi x) cos(pi y) [cos(pi z)], Phi_e = sin(2 x) cos(y) [cos(z/2)]."""
    X = grid.coords()
    d = grid.dim
    Pi = np.cos(np.pi * X[0]) * np.cos(np.pi * X[1]) * (np.cos(np.pi * X[2]) if d == 3 else 1.0)
    Pe = np.sin(2 * X[0]) * np.cos(X[1]) * (np.cos(0.5 * X[2]) if d == 3 else 1.0)
    li = -np.pi ** 2 * sum(D_i[:d]) * Pi
    le = -(4.0 * D_e[0] + D_e[1] + (0.25 * D_e[2] if d == 3 else 0.0)) * Pe
    fi = li - kappa * (Pi - Pe)
    fe = le + kappa * (Pi - Pe)
    Q = geom.nodes
    n = C.analytic_normals(geom)
    gi = np.stack([-np.pi * np.sin(np.pi * Q[:, 0]) * np.cos(np.pi * Q[:, 1]),
                   -np.pi * np.cos(np.pi * Q[:, 0]) * np.sin(np.pi * Q[:, 1])], 1)
    ge = np.stack([2 * np.cos(2 * Q[:, 0]) * np.cos(Q[:, 1]), -np.sin(2 * Q[:, 0]) * np.sin(Q[:, 1])], 1)
    if d == 3:
        cz, sz = np.cos(np.pi * Q[:, 2]), np.sin(np.pi * Q[:, 2])
        gi = np.concatenate([gi * cz[:, None], (-np.pi * np.cos(np.pi * Q[:, 0]) * np.cos(np.pi * Q[:, 1]) * sz)[:, None]], 1)
        c2, s2 = np.cos(0.5 * Q[:, 2]), np.sin(0.5 * Q[:, 2])
        ge = np.concatenate([ge * c2[:, None], (-0.5 * np.sin(2 * Q[:, 0]) * np.cos(Q[:, 1]) * s2)[:, None]], 1)
    gNi = (n * np.asarray(D_i[:d])[None, :] * gi).sum(1)
    gNe = (n * np.asarray(D_e[:d])[None, :] * ge).sum(1)
    return fi, fe, gNi, gNe, Pi, Pe


def _rate(e):
    return [math.log2(a / b) for a, b in zip(e, e[1:])]


def test_second_order_convergence_anisotropic_2d():
    kappa = 40.0
    ew, ee = [], []
    for N in (32, 64, 128):
        geom, grid = G.ellipse_config0(2 * N), Grid(2, N)
        fi, fe, gNi, gNe, Pi, Pe = _manufactured(geom, grid, kappa, DI, DE)
        c = CP.CoupledKFBI(geom, grid, DI[:2], DE[:2])
        ui, ue, psi, info = c.solve_neumann(fi, fe, gNi, gNe, kappa, tol=1e-11)
        assert info["converged"] and info["iters"] < 60
        ins = c.k.inside
        ew.append(np.abs((ui - ue) - (Pi - Pe))[ins].max())
        de = (ue - ue[ins].mean()) - (Pe - Pe[ins].mean())
        ee.append(np.abs(de[ins]).max())
    print("coupled 2-D errors", ew, ee)
    assert min(_rate(ew)) > 1.7 and min(_rate(ee)) > 1.7
    assert ew[-1] < 1e-3


@pytest.mark.slow
def test_second_order_convergence_anisotropic_3d():
    kappa = 40.0
    ew = []
    for N in (16, 32):
        geom, grid = G.sphere3(0.6, C.surface_res(N)), Grid(3, N)
        fi, fe, gNi, gNe, Pi, Pe = _manufactured(geom, grid, kappa, DI, DE)
        c = CP.CoupledKFBI(geom, grid, DI, DE)
        ui, ue, psi, info = c.solve_neumann(fi, fe, gNi, gNe, kappa, tol=1e-10)
        assert info["converged"]
        ins = c.k.inside
        ew.append(np.sqrt(np.mean(((ui - ue) - (Pi - Pe))[ins] ** 2)))
    print("coupled 3-D rms errors", ew)
    assert _rate(ew)[0] > 1.5


def test_isotropic_coupled_step_reproduces_decoupled():
    geom, grid = G.ellipse_config0(128), Grid(2, 64)
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=1, tol=1e-12)
    V0 = C.ball_stimulus(grid, (-0.4, 0.0), 0.15)
    q0 = np.zeros(grid.shape)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    cb = CP.CoupledBidomain(geom, grid, (1.0, 1.0), (2.0, 2.0), cfg.dt, C.FHN_CONFIG, tol=1e-12)
    V, q = V0.copy(), q0.copy()
    Vc, qc = V0.copy(), q0.copy()
    for _ in range(2):
        V, q, _ = bd.step(V, q)
        Vc, qc, ue, info = cb.step(Vc, qc)
    ins = bd.k.inside
    assert np.abs(Vc - V).max() < 1e-9 * np.abs(V).max()
    assert np.abs(qc - q).max() < 1e-9 * np.abs(q).max()
    w = info["w"]
    ue_dec = cfg.sigma_i * (w[ins].mean() - w) / (cfg.sigma_i + cfg.sigma_e)
    assert np.abs(ue - ue_dec)[ins].max() < 1e-9 * np.abs(ue_dec[ins]).max()
