"""Pins of the oracle's KFBI pieces (Sections 4-5, Algorithm 1).

* correction (Section 5.3): exact for piecewise quadratics whose jump vanishes
  on the interface (the corrected 5/7-point operator reproduces the
  continuous operator on each side);
* interpolation (Section 5.4): exact for quadratics, with and without jumps;
* jump relations: checked against harmonic jump functions on a circle and a
  sphere with constant and varying density;
* density interpolation: periodic spline against scipy's, local quadratic fit
  exact for quadratics on a plane and O(h^3)/O(h^2) on a sphere;
* GMRES against a dense LU solve of the assembled discrete operator;
* second-order convergence on manufactured solutions (Tables 1-11 report
  rho ~ 2).
"""
import math

import numpy as np
import pytest
import scipy.interpolate

from kfbi_workloads import configs as C, geometry as G
from kfbi_workloads.configs import Grid
from oracle import boxsolve, density, levelset as LS
from oracle.kfbi import KFBI
from oracle import krylov


def _phi_derivs(geom, comp, P):
    J = LS._phi_jet(geom, comp, P)
    return J.v, J.g, J.H


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("case", ["ellipse", "ellipsoid"])
def test_correction_exact_for_piecewise_quadratic(case, bc):
    """On both box layouts (interior nodes, or all nodes of the Neumann box)
    the corrected operator reproduces the continuous operator of each side."""
    if case == "ellipse":
        geom, grid = G.ellipse_config0(64), Grid(2, 32, bc=bc)
    else:
        geom, grid = G.ellipsoid3(0.7, 0.5, 0.45, 6), Grid(3, 20, bc=bc)
    k = KFBI(geom, grid)
    lam, K = 3.0, 0.7
    d = grid.dim
    Xg = np.stack(np.broadcast_arrays(*grid.coords()), axis=-1)
    Pq = lambda X: 0.3 + X[..., 0] ** 2 - 0.5 * X[..., 0] * X[..., 1] + 0.2 * X[..., -1] ** 2 + 0.1 * X[..., 1]  # noqa: E731
    lapP = 2.0 + 0.4 if d == 2 else 2.0 + 0.4
    phi = LS.component_phi(geom, 0, tuple(Xg[..., a] for a in range(d)))
    v = np.where(k.inside, Pq(Xg), Pq(Xg) - K * phi)
    # exact jumps [v] = K phi(z) = 0, [d_a v] = K phi_a, [d_aa v] = K phi_aa
    _, g, H = _phi_derivs(geom, 0, k.Pint)
    a = k.ints["axis"]
    r = np.arange(a.size)
    corr = k.correction(np.zeros(a.size), K * g[r, a], K * H[r, a, a])
    lhs = boxsolve.apply_L(v, lam, grid) - corr
    # continuous operator on each side (Laplacian of phi is constant)
    _, _, Hphi = _phi_derivs(geom, 0, Xg.reshape(-1, d))
    lap_phi = np.trace(Hphi, axis1=1, axis2=2).reshape(grid.shape)
    rhs = np.where(k.inside, lapP - lam * Pq(Xg), lapP - K * lap_phi - lam * (Pq(Xg) - K * phi))
    # away from the box boundary (zero Dirichlet data or the mirrored ghost
    # value breaks the quadratic there)
    interior = np.ones(grid.shape, dtype=bool)
    for ax in range(d):
        sl = [slice(None)] * d
        sl[ax] = 0
        interior[tuple(sl)] = False
        sl[ax] = -1
        interior[tuple(sl)] = False
    err = np.abs(lhs - rhs)[interior]
    assert err.max() < 1e-9 * grid.N ** 2


@pytest.mark.parametrize("bc", ["dirichlet", "neumann"])
@pytest.mark.parametrize("dim", [2, 3])
def test_interpolation_exact_for_quadratics(dim, bc):
    if dim == 2:
        geom, grid = G.ellipse_config0(48), Grid(2, 32, bc=bc)
    else:
        geom, grid = G.ellipsoid3(0.7, 0.5, 0.45, 6), Grid(3, 24, bc=bc)
    k = KFBI(geom, grid)
    Xg = np.stack(np.broadcast_arrays(*grid.coords()), axis=-1)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(10)

    def P(X):
        x, y = X[..., 0], X[..., 1]
        z = X[..., 2] if dim == 3 else 0 * x
        return c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * y * y + c[6] * z * z \
            + c[7] * x * y + c[8] * x * z + c[9] * y * z

    def gradP(X):
        x, y = X[..., 0], X[..., 1]
        z = X[..., 2] if dim == 3 else 0 * x
        g = [c[1] + 2 * c[4] * x + c[7] * y + c[8] * z, c[2] + 2 * c[5] * y + c[7] * x + c[9] * z]
        if dim == 3:
            g.append(c[3] + 2 * c[6] * z + c[8] * x + c[9] * y)
        return np.stack(g, -1)

    exact = (gradP(geom.nodes) * k.n_node).sum(1)
    # no jumps
    assert np.abs(k.interp(P(Xg)) - exact).max() < 1e-10
    # with the jump of v^- = P - K phi (a quadratic vanishing on the surface)
    K = 1.3
    phi = LS.component_phi(geom, 0, tuple(Xg[..., a] for a in range(dim)))
    v = np.where(k.inside, P(Xg), P(Xg) - K * phi)
    _, g, H = _phi_derivs(geom, 0, geom.nodes)
    out = k.interp(v, (np.zeros(geom.M), K * g, K * H))
    assert np.abs(out - exact).max() < 1e-10


def test_jump_relations_circle():
    """v^- = v^+ - J with J = R (p0 + p1 (r/R - R/r)/2 ... ) harmonic,
    J = 0 on r = R, dJ/dr = psi(theta) there: D^2 J must equal the formula."""
    R, p0, p1 = 0.55, 0.8, -0.35
    th = np.linspace(0, 2 * np.pi, 17)[:-1]
    Pt = R * np.stack([np.cos(th), np.sin(th)], 1)
    n = Pt / R
    S = (np.eye(2)[None] - n[:, :, None] * n[:, None, :]) / R
    psi = p0 + p1 * np.cos(th)
    tau = np.stack([-n[:, 1], n[:, 0]], 1)
    gpsi = (-p1 * np.sin(th) / R)[:, None] * tau
    jg, jH = KFBI.jump_grad_hess(psi, gpsi, n, S)

    def J(X):
        r = np.hypot(X[:, 0], X[:, 1])
        return p0 * R * np.log(r / R) + p1 * R * 0.5 * (r / R - R / r) * X[:, 0] / r

    eps = 1e-4
    for i in range(2):
        for j in range(2):
            ei = np.eye(2)[i] * eps
            ej = np.eye(2)[j] * eps
            fd = (J(Pt + ei + ej) - J(Pt + ei - ej) - J(Pt - ei + ej) + J(Pt - ei - ej)) / (4 * eps * eps)
            assert np.allclose(jH[:, i, j], fd, atol=2e-6)
        fd1 = (J(Pt + np.eye(2)[i] * eps) - J(Pt - np.eye(2)[i] * eps)) / (2 * eps)
        assert np.allclose(jg[:, i], fd1, atol=1e-7)


def test_jump_relations_sphere():
    R, p0, p1 = 0.6, 0.5, 0.3
    geom = G.sphere3(R, 4)
    Pt = geom.nodes
    n = Pt / R
    S = (np.eye(3)[None] - n[:, :, None] * n[:, None, :]) / R
    # J = R^2 p0 (1/R - 1/r) + x (a + b/r^3): both harmonic; zero at r = R when
    # a = -b/R^3, and dJ/dr = p0 + (a - 2b/R^3) x/R = p0 + p1 x/R when b = -p1 R^3/3
    b = -p1 * R ** 3 / 3.0
    a = -b / R ** 3

    def J(X):
        r = np.linalg.norm(X, axis=1)
        return R * R * p0 * (1 / R - 1 / r) + X[:, 0] * (a + b / r ** 3)

    psi = p0 + p1 * Pt[:, 0] / R
    gfull = np.zeros_like(Pt)
    gfull[:, 0] = p1 / R
    gpsi = gfull - (gfull * n).sum(1)[:, None] * n
    jg, jH = KFBI.jump_grad_hess(psi, gpsi, n, S)
    eps = 1e-4
    for i in range(3):
        for j in range(3):
            ei = np.eye(3)[i] * eps
            ej = np.eye(3)[j] * eps
            fd = (J(Pt + ei + ej) - J(Pt + ei - ej) - J(Pt - ei + ej) + J(Pt - ei - ej)) / (4 * eps * eps)
            assert np.allclose(jH[:, i, j], fd, atol=5e-6)
        fd1 = (J(Pt + np.eye(3)[i] * eps) - J(Pt - np.eye(3)[i] * eps)) / (2 * eps)
        assert np.allclose(jg[:, i], fd1, atol=1e-7)


def test_periodic_spline_matches_scipy():
    M = 40
    t = 2 * np.pi * np.arange(M) / M
    psi = np.sin(t) + 0.3 * np.cos(3 * t) + 0.1
    m = density.spline_moments(psi)
    cs = scipy.interpolate.CubicSpline(np.append(t, 2 * np.pi), np.append(psi, psi[0]), bc_type="periodic")
    tq = np.random.default_rng(0).uniform(0, 2 * np.pi, 200)
    val, der = density.spline_eval(psi, m, tq)
    assert np.allclose(val, cs(tq), atol=1e-13)
    assert np.allclose(der, cs(tq, 1), atol=1e-12)


def test_local_fit_exact_on_plane():
    rng = np.random.default_rng(3)
    X = np.zeros((4, 6, 3))
    X[:, :, :2] = rng.uniform(-1, 1, (4, 6, 2))
    X[:, :, 2] = 0.0
    z = np.zeros((4, 3))
    z[:, :2] = rng.uniform(-0.2, 0.2, (4, 2))
    n = np.tile([0.0, 0.0, 1.0], (4, 1))
    w0, wg, _ = density.fit_weights(X, z, n)
    f = lambda P: 1 + 2 * P[..., 0] - P[..., 1] + 0.5 * P[..., 0] ** 2 - 0.7 * P[..., 0] * P[..., 1] + 0.3 * P[..., 1] ** 2  # noqa: E731
    gx = 2 + z[:, 0] - 0.7 * z[:, 1]
    gy = -1 - 0.7 * z[:, 0] + 0.6 * z[:, 1]
    vals = f(X)
    assert np.allclose((w0 * vals).sum(1), f(z), atol=1e-12)
    grad = np.einsum("pdk,pk->pd", wg, vals)
    assert np.allclose(grad[:, 0], gx, atol=1e-11) and np.allclose(grad[:, 1], gy, atol=1e-11)
    assert np.allclose(grad[:, 2], 0, atol=1e-12)


def test_local_fit_converges_on_sphere():
    errs = []
    for nres in (8, 16, 32):
        geom = G.sphere3(0.6, nres)
        grid = Grid(3, 2 * nres)
        k = KFBI(geom, grid)
        psi = np.exp(geom.nodes[:, 0]) * (1 + geom.nodes[:, 2])
        p_int, g_int, g_node = k.density(psi)
        P = k.Pint
        ex = np.exp(P[:, 0]) * (1 + P[:, 2])
        gf = np.stack([ex, 0 * ex, np.exp(P[:, 0])], 1)
        n = k.n_int
        gt = gf - (gf * n).sum(1)[:, None] * n
        errs.append((np.abs(p_int - ex).max(), np.abs(g_int - gt).max()))
    for (e1, g1), (e2, g2) in zip(errs, errs[1:]):
        assert e1 / e2 > 5.0      # ~ 2^3
        assert g1 / g2 > 2.8      # ~ 2^2


def test_gmres_matches_dense_lu():
    geom, grid = G.ellipse_config0(24), Grid(2, 16)
    k = KFBI(geom, grid)
    lam = 60.0
    A = np.stack([k.apply_A(e, lam) for e in np.eye(geom.M)], axis=1)
    rng = np.random.default_rng(4)
    g = rng.standard_normal(geom.M)
    x_ref = np.linalg.solve(A, g)
    x, info = krylov.gmres(lambda v: k.apply_A(v, lam), g, np.zeros(geom.M), 1e-13, restart=50)
    assert info["converged"]
    assert np.abs(x - x_ref).max() < 1e-10 * np.abs(x_ref).max()
    # restarted GMRES converges to the same solution
    x2, info2 = krylov.gmres(lambda v: k.apply_A(v, lam), g, np.zeros(geom.M), 1e-13, restart=5)
    assert np.abs(x2 - x_ref).max() < 1e-9 * np.abs(x_ref).max()
    # the simple iteration converges too (gamma = 0.8 of Section 7)
    x3, info3 = krylov.richardson(lambda v: k.apply_A(v, lam), g, np.zeros(geom.M), 1e-10, max_iter=400)
    assert info3["converged"] and np.abs(x3 - x_ref).max() < 1e-8 * np.abs(x_ref).max()


def test_gmres_fixed_iterations_and_residual():
    geom, grid = G.ellipse_config0(32), Grid(2, 32)
    k = KFBI(geom, grid)
    g = np.random.default_rng(6).standard_normal(geom.M)
    A = lambda v: k.apply_A(v, 60.0)  # noqa: E731
    x, info = krylov.gmres(A, g, np.zeros(geom.M), 0.0, max_iter=4)
    assert info["iters"] == 4
    r = np.linalg.norm(g - A(x)) / np.linalg.norm(g)
    assert abs(r - info["rel_res"]) < 1e-12


def _rate(e):
    return [math.log2(a / b) for a, b in zip(e, e[1:])]


def test_second_order_convergence_2d():
    errs = []
    for N in (32, 64, 128):
        geom, grid = G.ellipse_config0(2 * N), Grid(2, N)
        f, u, gN = C.manufactured(geom, grid, 60.0)
        k = KFBI(geom, grid)
        uh, psi, info = k.solve_neumann(f, gN, 60.0, tol=1e-10)
        assert info["converged"] and info["iters"] < 20
        e = (uh - u)[k.inside]
        errs.append(math.sqrt((e ** 2).mean()))
    assert min(_rate(errs)) > 1.7


def test_neumann_box_second_order_and_box_independent():
    """The solution in Omega does not depend on the box condition of the
    Green's function (Section 4): with the Neumann box the KFBI solution
    converges at second order, and it differs from the Dirichlet-box solution
    by a second-order amount."""
    errs, diffs = [], []
    for N in (32, 64, 128):
        geom = G.ellipse_config0(2 * N)
        sol = {}
        for bc in ("dirichlet", "neumann"):
            grid = Grid(2, N, bc=bc)
            f, u, gN = C.manufactured(geom, grid, 60.0)
            k = KFBI(geom, grid)
            uh, psi, info = k.solve_neumann(f, gN, 60.0, tol=1e-11)
            assert info["converged"] and info["iters"] < 20
            ins = k.inside
            if bc == "neumann":
                assert uh.shape == (N + 1, N + 1) and not ins[0].any() and not ins[:, -1].any()
                e = (uh - u)[ins]
                errs.append(math.sqrt((e ** 2).mean()))
                sol[bc] = uh[1:-1, 1:-1][ins[1:-1, 1:-1]]
            else:
                sol[bc] = uh[ins]
        diffs.append(np.abs(sol["neumann"] - sol["dirichlet"]).max())
    # the max-norm difference is irregular from one grid to the next; its rate
    # over the two refinements is second order
    assert min(_rate(errs)) > 1.7 and math.log2(diffs[0] / diffs[-1]) / 2.0 > 1.6


def test_neumann_box_gmres_matches_dense_lu():
    geom, grid = G.ellipse_config0(24), Grid(2, 16, bc="neumann")
    k = KFBI(geom, grid)
    A = np.stack([k.apply_A(e, 60.0) for e in np.eye(geom.M)], axis=1)
    g = np.random.default_rng(9).standard_normal(geom.M)
    x_ref = np.linalg.solve(A, g)
    x, info = krylov.gmres(lambda v: k.apply_A(v, 60.0), g, np.zeros(geom.M), 1e-13, restart=50)
    assert info["converged"] and np.abs(x - x_ref).max() < 1e-10 * np.abs(x_ref).max()


def test_second_order_convergence_disk_poisson_like():
    errs = []
    for N in (32, 64, 128):
        geom, grid = G.disk2(0.6, 2 * N), Grid(2, N)
        f, u, gN = C.manufactured(geom, grid, 1.0)
        k = KFBI(geom, grid)
        uh, psi, info = k.solve_neumann(f, gN, 1.0, tol=1e-10)
        e = (uh - u)[k.inside]
        errs.append(np.abs(e).max())
    assert min(_rate(errs)) > 1.6


@pytest.mark.slow
def test_second_order_convergence_sphere():
    errs = []
    for N in (16, 32, 64):
        geom, grid = G.sphere3(0.6, C.surface_res(N)), Grid(3, N)
        f, u, gN = C.manufactured(geom, grid, 40.0)
        k = KFBI(geom, grid)
        uh, psi, info = k.solve_neumann(f, gN, 40.0, tol=1e-10)
        assert info["converged"] and info["iters"] < 30
        e = (uh - u)[k.inside]
        errs.append(math.sqrt((e ** 2).mean()))
    assert min(_rate(errs)) > 1.5


def test_green_identity_discrete():
    """For Lap u - lam u = f with du/dn = g^N, the boundary flux equals the
    volume integral of f + lam u.  The node-sum quadrature of the volume
    integral is only first-order accurate on the staircase of inside nodes,
    so the flux balance of the numerical solution is compared with that of the
    exact solution under the same quadrature: the difference (lam h^2 times
    the summed error over the inside nodes) vanishes at second order."""
    d = []
    for N in (32, 64, 128):
        geom, grid = G.ellipse_config0(2 * N), Grid(2, N)
        f, u, gN = C.manufactured(geom, grid, 60.0)
        k = KFBI(geom, grid)
        uh, psi, info = k.solve_neumann(f, gN, 60.0, tol=1e-12)
        vol_h = ((f + 60.0 * uh) * k.inside).sum() * grid.h ** 2
        vol_x = ((f + 60.0 * u) * k.inside).sum() * grid.h ** 2
        d.append(abs(vol_h - vol_x))
    assert d[-1] < 5e-3 * abs(vol_x)
    assert min(_rate(d)) > 1.7


# ------------------------------------------------ Poisson case and stimulus

def test_surface_weights():
    from oracle.kfbi import surface_weights
    import scipy.integrate as si
    geom = G.ellipse_config0(256)
    per = si.quad(lambda t: math.hypot(0.7 * math.sin(t), 0.45 * math.cos(t)), 0.0, 2.0 * math.pi,
                  epsabs=1e-13)[0]
    assert abs(surface_weights(geom).sum() / per - 1.0) < 1e-4
    # inscribed triangles: the area converges to 4 pi r^2 from below at second order
    e = [4.0 * math.pi * 0.36 - surface_weights(G.sphere3(0.6, n)).sum() for n in (8, 16)]
    assert 0.0 < e[1] < e[0] and 3.0 < e[0] / e[1] < 5.0


def test_poisson_neumann_second_order_2d():
    """lambda = 0 with the rank-one modification: the solution (up to its
    constant) converges at second order, and <ds, psi> (the part of the
    density that absorbs the discrete incompatibility of the data) vanishes
    at second order."""
    errs, dpsi = [], []
    for N in (32, 64, 128):
        geom, grid = G.ellipse_config0(2 * N), Grid(2, N)
        f, u, gN = C.manufactured(geom, grid, 0.0)
        k = KFBI(geom, grid)
        uh, psi, info = k.solve_neumann(f, gN, 0.0, tol=1e-12)
        assert info["converged"]
        ins = k.inside
        e = (uh - uh[ins].mean()) - (u - u[ins].mean())
        errs.append(math.sqrt((e[ins] ** 2).mean()))
        dpsi.append(abs(k.ds @ psi))
    assert min(_rate(errs)) > 1.7
    assert min(_rate(dpsi)) > 1.7


def test_virtual_electrode_symmetry():
    """On a disk the electrode is odd in x, so S + S(-x) is constant."""
    from oracle.bidomain import Bidomain
    geom, grid = G.disk2(0.6, 128), Grid(2, 64)
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=grid.h, steps=1, tol=1e-12)
    bd = Bidomain(geom, grid, cfg, C.FHN_PAPER,
                  istim=C.virtual_electrode(grid))
    S = bd.solve_S()
    assert bd.S_info["converged"]
    T = S + S[:, ::-1]
    ins = bd.k.inside
    assert np.abs(T[ins] - T[ins].mean()).max() < 1e-10 * np.abs(S[ins]).max()


def test_virtual_electrode_coupled_equations():
    """The elimination behind the V and S problems, checked against Eq. pde1
    itself: with Phi_i = (S + sigma_e w)/(sigma_i + sigma_e) and
    Phi_e = (S - sigma_i w)/(sigma_i + sigma_e) from the oracle's w and S,
        sigma_i Lap_h Phi_i - kappa (w - V^n) = 0,
        sigma_e Lap_h Phi_e + kappa (w - V^n) = -beta I_stim
    hold at every regular node inside (where L_h u equals the right-hand side
    exactly)."""
    from oracle.bidomain import Bidomain
    from oracle import boxsolve
    geom, grid = G.ellipse_config0(256), Grid(2, 64)
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=grid.h, steps=1, tol=1e-12)
    fhn = C.FHN_PAPER
    I = C.virtual_electrode(grid)
    bd = Bidomain(geom, grid, cfg, fhn, istim=I)
    Vn = 0.3 * np.cos(3.0 * grid.coords()[0]) * np.ones(grid.shape)
    w, info = bd.diffuse(Vn)
    S = bd.solve_S()
    si_, se_ = cfg.sigma_i, cfg.sigma_e
    kappa = fhn.Cm * fhn.beta / (cfg.dt / 2.0)
    phi_i = (S + se_ * w) / (si_ + se_)
    phi_e = (S - si_ * w) / (si_ + se_)
    lap = lambda v: boxsolve.apply_L(v, 0.0, grid)  # noqa: E731
    reg = bd.k.inside.copy()
    reg.ravel()[bd.k.irregular] = False
    r1 = si_ * lap(phi_i) - kappa * (w - Vn)
    r2 = se_ * lap(phi_e) + kappa * (w - Vn) + fhn.beta * I
    scale = fhn.beta * np.abs(I).max()
    assert np.abs(r1[reg]).max() < 1e-9 * scale
    assert np.abs(r2[reg]).max() < 1e-9 * scale


def test_extracellular_from_constant_S():
    """Without a stimulus S is constant and the S-based potential reduces to
    sigma_i (mean V - V)/(sigma_i + sigma_e)."""
    from oracle.bidomain import extracellular, extracellular_S
    rng = np.random.default_rng(2)
    V = rng.standard_normal((20, 20))
    inside = rng.random((20, 20)) < 0.6
    a = extracellular(V, inside, 1.0, 2.0)
    b = extracellular_S(V, np.full_like(V, 3.7), inside, 1.0, 2.0)
    assert np.abs(a - b).max() < 1e-14
