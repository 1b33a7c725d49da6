"""Seeded, synthetic geometry inputs for the KFBI bidomain workloads.

This module only *generates input data*: the interface node sets that the
method is given (Section 6: "a set of quasi-uniformly spaced nodes"), the
surface triangulation used by the three-dimensional local coordinate systems
(Section 5.3, Fig. 1), and the shape parameters of each domain.  It holds none
of the method's arithmetic: no level-set classification, no normals or
curvatures, no jumps, corrections, interpolation or solves.  Both the CPU
oracle and the CUDA library consume the arrays produced here.

Geometry kinds (the domain Omega, always inside the box [-1, 1]^d):

* ``ELLIPSE2``   2-D ellipse with semi-axes (a, b) rotated by an angle whose
                 cosine/sine are given as data (c, s).
* ``ELLIPSOID3`` 3-D axis-aligned ellipsoid (a, b, c); a sphere when equal.
* ``STAR3``      3-D star body r = A + B sin(3 theta) cos(2 phi), theta polar,
                 phi azimuth.
* ``SHELL3``     3-D region between an outer and an inner axis-aligned
                 ellipsoid (a thick prolate shell).
* ``MESH3``      3-D domain given only by a closed triangle mesh of its
                 boundary (Section 5.3, Fig. 1 and Example 4: the method then
                 uses nothing but the vertices and triangles): the vertices
                 are the interface nodes, every triangle is wound
                 counter-clockwise seen from outside Omega (face normals
                 point out of Omega; on an inner wall they point into the
                 hole), and the mesh is a closed manifold.

Three-dimensional surfaces are meshed as equiangular cube-spheres of
resolution n: 6 n^2 + 2 vertices and 12 n^2 triangles per surface component,
with a canonical triangle order so that a point can be located on the mesh
from its cube-face coordinates (see ``Geometry.tri_index``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ELLIPSE2 = 1
ELLIPSOID3 = 2
STAR3 = 3
SHELL3 = 4
MESH3 = 5

# surface-component map types used for locating a point on a cube-sphere mesh
MAP_RADIAL = 0      # cube point = the position itself (star body, centred at 0)
MAP_ELLIPSOID = 1   # cube point = (x/a, y/b, z/c)


@dataclass
class Component:
    """One closed surface of a 3-D domain, meshed as a cube-sphere."""
    map_type: int
    axes: tuple            # (a, b, c) for MAP_ELLIPSOID, unused for MAP_RADIAL
    flip: bool             # True when Omega's outward normal points to -grad(level set)
    vert_offset: int
    n_vert: int
    tri_offset: int
    n_tri: int


@dataclass
class Geometry:
    dim: int
    kind: int
    params: np.ndarray                 # float64[16]
    nodes: np.ndarray                  # float64[M, dim], interface nodes
    # 3-D only
    tri: np.ndarray | None = None      # int32[n_tri, 3]
    cube_n: int = 0                    # cube-sphere resolution
    cube_t: np.ndarray | None = None   # float64[cube_n + 1], equiangular face coordinates
    components: list = field(default_factory=list)
    # MESH3 only, input data for manufactured Neumann data (never read by the
    # method): the analytic geometry the mesh was cut from, or the exact
    # outward normals at the nodes
    source: "Geometry | None" = None
    exact_normals: np.ndarray | None = None

    @property
    def M(self) -> int:
        return int(self.nodes.shape[0])

    def tri_index(self, comp: int, face: int, i: int, j: int, half: int) -> int:
        """Canonical index of triangle `half` (0 lower, 1 upper) of quad (i, j)
        on cube face `face` of surface component `comp`."""
        n = self.cube_n
        return self.components[comp].tri_offset + (((face * n + j) * n + i) * 2 + half)


def ellipse2(a: float, b: float, c: float, s: float, M: int) -> Geometry:
    """Ellipse with semi-axes (a, b) rotated so that its a-axis points along
    (c, s); M nodes equally spaced in the parameter t (t_i = 2 pi i / M),
    counter-clockwise."""
    t = 2.0 * np.pi * np.arange(M) / M
    xa = a * np.cos(t)
    yb = b * np.sin(t)
    nodes = np.stack([c * xa - s * yb, s * xa + c * yb], axis=1)
    params = np.zeros(16)
    params[:4] = [a, b, c, s]
    return Geometry(dim=2, kind=ELLIPSE2, params=params, nodes=nodes)


def cube_table(n: int) -> np.ndarray:
    """Equiangular gnomonic face coordinates tan(-pi/4 + m pi/(2n)), m = 0..n,
    made exactly antisymmetric with exact end points -1 and 1."""
    t = np.tan(-np.pi / 4 + np.arange(n + 1) * (np.pi / (2 * n)))
    t[0], t[n] = -1.0, 1.0
    for m in range(n // 2 + 1):
        t[n - m] = -t[m]
    if n % 2 == 0:
        t[n // 2] = 0.0
    return t


def _cube_sphere(n: int):
    """Unit-cube lattice of a cube-sphere: returns (cube points [V,3],
    triangles [12 n^2, 3]) in the canonical order (face, j, i, half)."""
    T = cube_table(n)
    key_to_id: dict = {}
    pts = []
    tris = np.empty((12 * n * n, 3), dtype=np.int64)

    def vid(face, i, j):
        k = face // 2
        sgn = 1 if face % 2 == 0 else -1
        k1, k2 = (k + 1) % 3, (k + 2) % 3
        key = [0, 0, 0]
        key[k] = n if sgn > 0 else 0
        key[k1] = i
        key[k2] = j
        key = tuple(key)
        v = key_to_id.get(key)
        if v is None:
            v = len(pts)
            key_to_id[key] = v
            p = [0.0, 0.0, 0.0]
            p[k] = float(sgn)
            p[k1] = T[i]
            p[k2] = T[j]
            pts.append(p)
        return v

    # vertices first in a fixed order so that ids do not depend on triangle order
    for face in range(6):
        for j in range(n + 1):
            for i in range(n + 1):
                vid(face, i, j)
    t = 0
    for face in range(6):
        for j in range(n):
            for i in range(n):
                v00, v10 = vid(face, i, j), vid(face, i + 1, j)
                v01, v11 = vid(face, i, j + 1), vid(face, i + 1, j + 1)
                tris[t] = (v00, v10, v01)
                tris[t + 1] = (v10, v11, v01)
                t += 2
    pts = np.asarray(pts, dtype=np.float64)
    assert pts.shape[0] == 6 * n * n + 2
    return pts, tris, T


def _directions(cube_pts: np.ndarray) -> np.ndarray:
    return cube_pts / np.sqrt((cube_pts ** 2).sum(axis=1))[:, None]


def _star_radius(d: np.ndarray, A: float, B: float) -> np.ndarray:
    """r(theta, phi) = A + B sin(3 theta) cos(2 phi) for unit directions d."""
    sxy2 = d[:, 0] ** 2 + d[:, 1] ** 2
    sin_t = np.sqrt(sxy2)
    sin3 = sin_t * (3.0 - 4.0 * sxy2)
    with np.errstate(invalid="ignore", divide="ignore"):
        cos2p = np.where(sxy2 > 0, (d[:, 0] ** 2 - d[:, 1] ** 2) / np.where(sxy2 > 0, sxy2, 1.0), 0.0)
    return A + B * sin3 * cos2p


def _mesh3(comps_spec, n, kind, params) -> Geometry:
    cube_pts, tris, T = _cube_sphere(n)
    dirs = _directions(cube_pts)
    nodes, tri_all, comps = [], [], []
    voff, toff = 0, 0
    for map_type, axes, flip, extra in comps_spec:
        if map_type == MAP_RADIAL:
            A, B = extra
            X = dirs * _star_radius(dirs, A, B)[:, None]
        else:
            X = dirs * np.asarray(axes)[None, :]
        nodes.append(X)
        tri_all.append(tris + voff)
        comps.append(Component(map_type, tuple(axes), flip, voff, X.shape[0], toff, tris.shape[0]))
        voff += X.shape[0]
        toff += tris.shape[0]
    return Geometry(dim=3, kind=kind, params=params, nodes=np.concatenate(nodes, axis=0),
                    tri=np.concatenate(tri_all, axis=0).astype(np.int32), cube_n=n, cube_t=T,
                    components=comps)


def ellipsoid3(a: float, b: float, c: float, n: int) -> Geometry:
    params = np.zeros(16)
    params[:3] = [a, b, c]
    return _mesh3([(MAP_ELLIPSOID, (a, b, c), False, None)], n, ELLIPSOID3, params)


def star3(A: float, B: float, n: int) -> Geometry:
    params = np.zeros(16)
    params[:2] = [A, B]
    return _mesh3([(MAP_RADIAL, (1.0, 1.0, 1.0), False, (A, B))], n, STAR3, params)


def shell3(outer, inner, n: int) -> Geometry:
    params = np.zeros(16)
    params[:3] = outer
    params[3:6] = inner
    return _mesh3([(MAP_ELLIPSOID, tuple(outer), False, None),
                   (MAP_ELLIPSOID, tuple(inner), True, None)], n, SHELL3, params)


def ellipse_config0(M: int = 256) -> Geometry:
    """Ellipse with semi-axes 0.7, 0.45 rotated by 30 degrees."""
    return ellipse2(0.7, 0.45, math.sqrt(3.0) / 2.0, 0.5, M)


def disk2(R: float, M: int) -> Geometry:
    return ellipse2(R, R, 1.0, 0.0, M)


def sphere3(R: float, n: int) -> Geometry:
    return ellipsoid3(R, R, R, n)


def star_config1(n: int) -> Geometry:
    return star3(0.6, 0.1, n)


SHELL_OUTER = (0.9, 0.6, 0.6)
SHELL_INNER = (0.7, 0.4, 0.4)


def shell_config2(n: int) -> Geometry:
    return shell3(SHELL_OUTER, SHELL_INNER, n)


# ------------------------------------------------------------ triangle meshes

def mesh3(nodes: np.ndarray, tri: np.ndarray) -> Geometry:
    """A MESH3 input: vertices (the interface nodes) and outward-wound
    triangles, nothing else."""
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    comp = Component(-1, (1.0, 1.0, 1.0), False, 0, nodes.shape[0], 0, tri.shape[0])
    return Geometry(dim=3, kind=MESH3, params=np.zeros(16), nodes=nodes, tri=tri, components=[comp])


def as_mesh(geom: Geometry) -> Geometry:
    """The cube-sphere triangulation of an analytic 3-D geometry handed over as
    a bare mesh (the level set, the cube maps and the component structure are
    dropped); triangles are rewound where needed so that every face normal
    points out of Omega (decided from the analytic shape, which is input
    preparation only)."""
    tri = np.array(geom.tri, dtype=np.int64)
    X = geom.nodes
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    fn = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    out_dir = np.empty_like(cen)
    for C in geom.components:
        sl = slice(C.tri_offset, C.tri_offset + C.n_tri)
        ax = np.asarray(C.axes, dtype=np.float64)
        g = cen[sl] / (ax * ax)[None, :] if C.map_type == MAP_ELLIPSOID else cen[sl]
        out_dir[sl] = -g if C.flip else g
    flip = (fn * out_dir).sum(axis=1) < 0.0
    tri[flip] = tri[flip][:, ::-1]
    m = mesh3(X, tri)
    m.source = geom
    return m


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
                  [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5],
                  [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1)[:, None], f


def geodesic_sphere(level: int):
    """Unit-sphere vertices and outward triangles of the icosahedron with every
    edge split into `level` parts (10 level^2 + 2 vertices; the 12 original
    vertices keep valence 5)."""
    v0, f0 = _icosahedron()
    verts = [tuple(p) for p in v0]
    index = {}

    def vid(p):
        key = tuple(np.round(p, 12))
        if key not in index:
            index[key] = len(verts)
            verts.append(tuple(p))
        return index[key]

    for i, p in enumerate(v0):
        index[tuple(np.round(p, 12))] = i
    faces = []
    n = level
    for a, b, c in f0:
        A, B, C = v0[a], v0[b], v0[c]
        grid = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                p = A + (B - A) * (i / n) + (C - A) * (j / n)
                grid[(i, j)] = vid(p / np.linalg.norm(p))
        for i in range(n):
            for j in range(n - i):
                faces.append((grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]))
                if i + j < n - 1:
                    faces.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    V = np.array(verts, dtype=np.float64)
    V = V / np.linalg.norm(V, axis=1)[:, None]
    F = np.array(faces, dtype=np.int64)
    fn = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    bad = (fn * (V[F[:, 0]] + V[F[:, 1]] + V[F[:, 2]])).sum(axis=1) < 0.0
    F[bad] = F[bad][:, ::-1]
    return V, F


def bean_mesh(level: int) -> Geometry:
    """A smooth, non-convex closed surface meshed as a geodesic sphere mapped
    radially (a stand-in for a measured organ surface such as the left
    ventricle of Example 4, which is not available): the unit direction d goes
    to r(d) d with r = 0.55 (1 + 0.25 d_x^2 - 0.2 d_z) and the x axis
    stretched by 1.2."""
    V, F = geodesic_sphere(level)
    m = mesh3(_bean_map(V), F)
    # exact normals of the mapped sphere from two tangents by central
    # differences (error ~1e-10, far below any discretisation error)
    t1 = np.cross(V, np.where(np.abs(V[:, :1]) < 0.9, [[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]]))
    t1 /= np.linalg.norm(t1, axis=1)[:, None]
    t2 = np.cross(V, t1)
    eps = 1e-5

    def on_sphere(d):
        return d / np.linalg.norm(d, axis=1)[:, None]

    T1 = _bean_map(on_sphere(V + eps * t1)) - _bean_map(on_sphere(V - eps * t1))
    T2 = _bean_map(on_sphere(V + eps * t2)) - _bean_map(on_sphere(V - eps * t2))
    n = np.cross(T1, T2)
    n /= np.linalg.norm(n, axis=1)[:, None]
    n *= np.sign((n * m.nodes).sum(axis=1))[:, None]
    m.exact_normals = n
    return m


def _bean_map(d: np.ndarray) -> np.ndarray:
    r = 0.55 * (1.0 + 0.25 * d[:, 0] ** 2 - 0.2 * d[:, 2])
    X = d * r[:, None]
    X[:, 0] *= 1.2
    return X
