"""Pins of the oracle's geometry preprocessing (Sections 5.3, 6): level-set
derivatives against closed forms and finite differences, classification
against independent trigonometric inside tests, crossings against closed-form
roots, cell indexing against its definition."""
import math

import numpy as np
import pytest

from kfbi_workloads import geometry as G
from kfbi_workloads.configs import Grid
from oracle import grid as GR, levelset as LS


def test_sphere_normal_and_shape_closed_form():
    R = 0.6
    geom = G.sphere3(R, 8)
    n, S = LS.normals_shapes_at_nodes(geom)
    X = geom.nodes
    assert np.abs(n - X / R).max() < 1e-14
    P = np.eye(3)[None] - n[:, :, None] * n[:, None, :]
    assert np.abs(S - P / R).max() < 1e-13


def test_ellipse_curvature_closed_form():
    geom = G.ellipse_config0(64)
    a, b = 0.7, 0.45
    n, S = LS.normals_shapes_at_nodes(geom)
    t = 2 * np.pi * np.arange(64) / 64
    kappa = a * b / (a * a * np.sin(t) ** 2 + b * b * np.cos(t) ** 2) ** 1.5
    tau = np.stack([-n[:, 1], n[:, 0]], 1)
    assert np.allclose(np.einsum("mi,mij,mj->m", tau, S, tau), kappa, atol=1e-12)
    assert np.abs(np.einsum("mi,mij->mj", n, S)).max() < 1e-12


def test_shell_inner_normal_points_into_hole():
    geom = G.shell_config2(8)
    n, S = LS.normals_shapes_at_nodes(geom)
    C = geom.components[1]
    sl = slice(C.vert_offset, C.vert_offset + C.n_vert)
    X = geom.nodes[sl]
    assert np.all((n[sl] * X).sum(1) < 0)             # points toward the centre
    assert np.all(np.trace(S[sl], axis1=1, axis2=2) < 0)  # concave from Omega's outside


def test_star_jet_against_finite_differences():
    geom = G.star_config1(8)
    rng = np.random.default_rng(0)
    P = rng.uniform(-0.8, 0.8, (50, 3))
    P = P[np.hypot(P[:, 0], P[:, 1]) > 0.05]
    J = LS._phi_jet(geom, 0, P)
    eps = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        fp = LS.phi_star(*(P + e).T, 0.6, 0.1)
        fm = LS.phi_star(*(P - e).T, 0.6, 0.1)
        assert np.allclose(J.g[:, k], (fp - fm) / (2 * eps), atol=1e-6)
        Jp = LS._phi_jet(geom, 0, P + e)
        Jm = LS._phi_jet(geom, 0, P - e)
        assert np.allclose(J.H[:, :, k], (Jp.g - Jm.g) / (2 * eps), atol=1e-5)
    assert np.allclose(J.v, LS.phi_star(*P.T, 0.6, 0.1), rtol=0, atol=1e-15)


def test_star_classification_against_trig_formula():
    grid = Grid(3, 32)
    geom = G.star_config1(8)
    ins = GR.classify(geom, grid)
    X, Y, Z = np.broadcast_arrays(*grid.coords())
    rho = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    with np.errstate(invalid="ignore"):
        th = np.arccos(np.clip(Z / rho, -1, 1))
    ph = np.arctan2(Y, X)
    r = 0.6 + 0.1 * np.sin(3 * th) * np.cos(2 * ph)
    far = np.abs(rho - r) > 1e-9
    assert np.array_equal(ins[far], (rho <= r)[far])


def test_ellipse_classification_against_parametric_test():
    grid = Grid(2, 64)
    geom = G.ellipse_config0(32)
    ins = GR.classify(geom, grid)
    X, Y = np.broadcast_arrays(*grid.coords())
    ang = math.radians(30.0)
    xr = math.cos(ang) * X + math.sin(ang) * Y
    yr = -math.sin(ang) * X + math.cos(ang) * Y
    r = np.hypot(xr / 0.7, yr / 0.45)
    far = np.abs(r - 1) > 1e-9
    assert np.array_equal(ins[far], (r <= 1)[far])
    # area check: count * h^2 approximates pi a b
    assert abs(ins.sum() * grid.h ** 2 - math.pi * 0.7 * 0.45) < 0.02


def test_crossings_match_closed_form_roots_ellipse():
    grid = Grid(2, 64)
    geom = G.ellipse_config0(32)
    ins = GR.classify(geom, grid)
    ints = GR.intersections(geom, grid, ins)
    P = GR.intersection_points(grid, ins.shape, ints)
    c, s, a, b = math.sqrt(3) / 2, 0.5, 0.7, 0.45
    A11 = c * c / a ** 2 + s * s / b ** 2
    A22 = s * s / a ** 2 + c * c / b ** 2
    A12 = c * s / a ** 2 - c * s / b ** 2
    for ax in (0, 1):
        m = ints["axis"] == ax
        other = P[m, 1 - ax]
        qa = A11 if ax == 0 else A22
        qb = 2 * A12 * other
        qc = (A22 if ax == 0 else A11) * other ** 2 - 1
        disc = np.sqrt(qb * qb - 4 * qa * qc)
        r1 = (-qb - disc) / (2 * qa)
        r2 = (-qb + disc) / (2 * qa)
        z = P[m, ax]
        err = np.minimum(np.abs(z - r1), np.abs(z - r2))
        assert err.max() < 1e-13
    # every crossing lies inside its edge, and both ends differ in status
    insf = ins.ravel()
    assert np.all(insf[ints["lo"]] != insf[ints["hi"]])


def test_crossings_on_surface_3d():
    for geom in (G.star_config1(8), G.shell_config2(8)):
        grid = Grid(3, 32)
        ins = GR.classify(geom, grid)
        ints = GR.intersections(geom, grid, ins)
        P = GR.intersection_points(grid, ins.shape, ints)
        for c in range(LS.n_components(geom)):
            m = ints["comp"] == c
            ph = LS.component_phi(geom, c, tuple(P[m].T))
            assert np.abs(ph).max() < 1e-14
        # edge count equals the number of status changes along every axis
        n_changes = sum(int((np.diff(ins.astype(np.int8), axis=ax) != 0).sum()) for ax in range(3))
        assert n_changes == ints["z"].size


def test_irregular_definition_bruteforce():
    grid = Grid(2, 24)
    geom = G.ellipse_config0(32)
    ins = GR.classify(geom, grid)
    irr = set(GR.irregular_list(ins).tolist())
    n1 = grid.N - 1
    for j in range(n1):
        for i in range(n1):
            nb = []
            for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jj, ii = j + dj, i + di
                nb.append(bool(ins[jj, ii]) if 0 <= jj < n1 and 0 <= ii < n1 else False)
            expect = any(v != bool(ins[j, i]) for v in nb)
            assert (j * n1 + i in irr) == expect


def test_cell_index_definition():
    grid = Grid(3, 32)
    P = np.array([[0.0, 0.03125, -0.5], [0.1, -0.2, 0.3], [0.0625 * 3, 0.5 - 1e-17, -0.03125]])
    c, s = GR.cell_index(grid, P)
    for m in range(P.shape[0]):
        for a in range(3):
            t = (P[m, a] + 1.0) / grid.h
            assert c[m, a] == math.floor(t + 0.5)
            xc = -1.0 + c[m, a] * grid.h
            assert s[m, a] == (1 if P[m, a] >= xc else -1)


def test_box_contact_is_an_error():
    grid = Grid(2, 8)
    geom = G.ellipse2(0.95, 0.95, 1.0, 0.0, 16)
    with pytest.raises(GR.GeometryError):
        GR.irregular_list(GR.classify(geom, grid))
