"""Pins of the oracle's mesh-only domains (Section 5.3, Fig. 1, Example 4):
classification by ray parity, crossings on the local quadratic surfaces of
the triangles, normals and shape operators from those surfaces, and the whole
KFBI solve on meshes."""
import math

import numpy as np
import pytest

from kfbi_workloads import configs as C, geometry as G
from kfbi_workloads.configs import Grid
from oracle import density, mesh as MESH
from oracle.kfbi import KFBI


def _rate(e):
    return [math.log2(a / b) for a, b in zip(e, e[1:])]


def _nodes(grid):
    return np.stack(np.broadcast_arrays(*grid.coords()), axis=-1)


def test_classification_equals_convex_polyhedron_test():
    """A convex mesh (the convex hull of points on an ellipsoid) encloses
    exactly the points on the inner side of every face plane: brute force
    over all faces."""
    from scipy.spatial import ConvexHull
    V = G.sphere3(1.0, 6).nodes * np.array([0.62, 0.5, 0.45])[None, :]
    hull = ConvexHull(V)
    T = hull.simplices.copy()
    A, B, Cc = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    inward = (np.cross(B - A, Cc - A) * (A - V.mean(axis=0))).sum(axis=1) < 0
    T[inward] = T[inward][:, ::-1]
    geom, grid = G.mesh3(V, T), Grid(3, 32)
    ins = MESH.classify(geom, grid)
    X = geom.nodes
    A, B, Cc = X[T[:, 0]], X[T[:, 1]], X[T[:, 2]]
    nf = np.cross(B - A, Cc - A)
    P = _nodes(grid).reshape(-1, 3)
    side = np.einsum("pfd,fd->pf", P[:, None, :] - A[None], nf)
    clear = np.abs(side).min(axis=1) > 1e-12
    brute = (side < 0).all(axis=1)
    assert clear.mean() > 0.99
    assert np.array_equal(ins.reshape(-1)[clear], brute[clear])
    assert ins.sum() > 1000


def _octahedron(r):
    V = np.array([[r, 0, 0], [-r, 0, 0], [0, r, 0], [0, -r, 0], [0, 0, r], [0, 0, -r]], dtype=np.float64)
    F = []
    for sx, ix in ((1, 0), (-1, 1)):
        for sy, iy in ((1, 2), (-1, 3)):
            for sz, iz in ((1, 4), (-1, 5)):
                tri = [ix, iy, iz]
                if sx * sy * sz < 0:
                    tri = [ix, iz, iy]
                F.append(tri)
    return G.mesh3(V, np.array(F))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rays_through_vertices_and_edges(axis):
    """An octahedron whose vertices and edges lie on grid lines: rays through
    vertices and along edge lines still cross the closed surface an even
    number of times, and nodes off the faces are classified exactly."""
    geom, grid = _octahedron(0.5), Grid(3, 32)   # 0.5 = 8 h: vertices on grid nodes
    T = np.asarray(geom.tri)
    fn = np.cross(geom.nodes[T[:, 1]] - geom.nodes[T[:, 0]], geom.nodes[T[:, 2]] - geom.nodes[T[:, 0]])
    assert ((fn * geom.nodes[T].mean(axis=1)).sum(axis=1) > 0).all()   # outward winding
    lu, lv, x, _ = MESH.ray_hits(geom, grid, axis)
    _, counts = np.unique(lv * grid.n + lu, return_counts=True)
    assert (counts % 2 == 0).all() and counts.size > 100
    ins = MESH.classify(geom, grid)
    P = _nodes(grid)
    l1 = np.abs(P).sum(axis=-1)
    off = np.abs(l1 - 0.5) > 1e-12
    assert np.array_equal(ins[off], (l1 < 0.5)[off])


def test_status_changes_match_crossings_on_every_axis():
    """Parity along y and z lines agrees with the x-line classification: every
    edge whose nodes differ holds an odd number of its line's crossings."""
    geom, grid = G.bean_mesh(8), Grid(3, 32)
    ins = MESH.classify(geom, grid)
    for a in (1, 2):
        lu, lv, x, _ = MESH.ray_hits(geom, grid, a)
        arr_ax = 2 - a
        n = grid.n
        k = np.arange(n - 1)
        for line in np.unique(lv * n + lu):
            ku, kv = line % n, line // n
            idx = [None, None, None]
            u, v = (a + 1) % 3, (a + 2) % 3
            idx[2 - u], idx[2 - v], idx[arr_ax] = ku - grid.first, kv - grid.first, slice(None)
            st = ins[tuple(idx)]
            hx = x[(lv * n + lu) == line]
            xs = MESH.node_coord(grid, np.arange(grid.first, grid.first + n))
            cnt = np.array([np.count_nonzero((hx > xs[i]) & (hx <= xs[i + 1])) for i in k])
            assert np.array_equal(st[:-1] != st[1:], cnt % 2 == 1)


def test_local_surface_normals_shapes_and_crossings_converge():
    """On meshed spheres the local quadratic surfaces give crossing points,
    normals and shape operators converging to the sphere's (R = 0.6): points
    at third order, normals at second, shape operators at first."""
    R = 0.6
    ep, en, eS = [], [], []
    for N in (16, 32, 64):
        geom, grid = G.as_mesh(G.sphere3(R, C.surface_res(N))), Grid(3, N)
        k = KFBI(geom, grid)
        P = k.Pint
        r = np.linalg.norm(P, axis=1)
        ep.append(np.abs(r - R).max())
        nx = P / r[:, None]
        en.append(np.abs(k.n_int - nx).max())
        S_ex = (np.eye(3)[None] - nx[:, :, None] * nx[:, None, :]) / R
        eS.append(np.abs(k.S_int - S_ex).max())
    assert min(_rate(ep)) > 2.5 and min(_rate(en)) > 1.6 and min(_rate(eS)) > 0.8


def test_flat_hit_is_on_the_triangle():
    """Each crossing's triangle contains the projected line point: the hit
    lies in the triangle's plane within rounding."""
    geom, grid = G.bean_mesh(6), Grid(3, 32)
    X, T = geom.nodes, np.asarray(geom.tri, dtype=np.int64)
    for a in range(3):
        lu, lv, x, tri = MESH.ray_hits(geom, grid, a)
        P = np.zeros((x.size, 3))
        P[:, a] = x
        P[:, (a + 1) % 3] = MESH.node_coord(grid, lu)
        P[:, (a + 2) % 3] = MESH.node_coord(grid, lv)
        A, B, Cc = X[T[tri, 0]], X[T[tri, 1]], X[T[tri, 2]]
        nf = np.cross(B - A, Cc - A)
        nf /= np.linalg.norm(nf, axis=1)[:, None]
        assert np.abs(((P - A) * nf).sum(axis=1)).max() < 1e-12


def test_mesh_solution_second_order_non_convex_valence5():
    """A non-convex mesh-only domain whose mesh has vertices of valence 5
    (ring fits there): the manufactured Neumann solve converges at second
    order with flat iteration counts."""
    errs, its = [], []
    for N, level in ((32, 8), (64, 16)):
        geom, grid = G.bean_mesh(level), Grid(3, N)
        k = KFBI(geom, grid)
        f, u, gN = C.manufactured(geom, grid, 40.0)
        uh, psi, info = k.solve_neumann(f, gN, 40.0, tol=1e-10)
        assert info["converged"]
        its.append(info["iters"])
        errs.append(math.sqrt(((uh - u)[k.inside] ** 2).mean()))
    assert min(_rate(errs)) > 1.7 and max(its) - min(its) <= 2


def test_mesh_matches_analytic_geometry():
    """The sphere handed over as a bare mesh gives the solution of the
    analytic sphere up to far less than the discretisation error."""
    N = 32
    ga = G.sphere3(0.6, C.surface_res(N))
    gm = G.as_mesh(ga)
    grid = Grid(3, N)
    f, u, gN = C.manufactured(ga, grid, 40.0)
    ka, km = KFBI(ga, grid), KFBI(gm, grid)
    ua, _, _ = ka.solve_neumann(f, gN, 40.0, tol=1e-11)
    um, _, _ = km.solve_neumann(f, gN, 40.0, tol=1e-11)
    both = ka.inside & km.inside
    err = np.abs(ua - u)[both].max()
    assert np.abs(um - ua)[both].max() < 0.2 * err


def test_open_mesh_rejected():
    geom = G.as_mesh(G.sphere3(0.6, 4))
    with pytest.raises(ValueError):
        density.patches(np.asarray(geom.tri)[1:], geom.M)
