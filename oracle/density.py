"""Density and its surface gradient away from the interface nodes (oracle).

The jumps of Section 5.3 need psi and its surface gradient at the crossing
points of the interface with grid lines, and the Taylor systems of Section 5.4
need the surface gradient at the nodes themselves.

* 2-D (Section 7: boundaries given by nodes "and the periodic cubic splines on
  these points"): psi is a periodic cubic spline in the node parameter t, with
  nodes at t_i = 2 pi i / M.  For an ellipse the parameter of a surface point
  comes from the inverse map t = atan2(y'/b, x'/a), and the arc-length
  derivative is psi_s = psi_t / |X_t|.  The surface gradient is psi_s tau with
  tau = (-n_y, n_x), the direction of increasing t.
* 3-D (Section 5.3, Fig. 1: a local coordinate system on six surface points
  around a triangle): psi is fitted by the quadratic in local tangent-plane
  coordinates through the three vertices of a triangle and the three vertices
  opposite its edges; psi(z) and grad_Gamma psi(z) are the fit's value and
  gradient at z.  A crossing point uses the triangle that contains it on the
  cube-sphere (located from its cube-face coordinates); a node uses its
  lowest-numbered incident triangle.
  Reading for the few triangles that touch a vertex of valence other than 6
  (the cube corners), where the six points repeat or lie on a conic: the
  quadratic is fitted by least squares through every vertex of the triangles
  that share a vertex with the base triangle (decided from the mesh topology
  alone, so both implementations choose identically).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from kfbi_workloads import geometry as G


# ----------------------------------------------------------------------- 2-D

def spline_moments(psi: np.ndarray) -> np.ndarray:
    """Second derivatives m_i of the periodic cubic spline through (t_i, psi_i),
    uniform spacing D = 2 pi / M:  m_{i-1} + 4 m_i + m_{i+1}
    = 6 (psi_{i+1} - 2 psi_i + psi_{i-1}) / D^2 (cyclic)."""
    M = psi.size
    D = 2.0 * np.pi / M
    rhs = 6.0 * (np.roll(psi, -1) - 2.0 * psi + np.roll(psi, 1)) / (D * D)
    col = np.zeros(M)
    col[0], col[1], col[-1] = 4.0, 1.0, 1.0
    return scipy.linalg.solve_circulant(col, rhs)


def spline_eval(psi, m, t):
    """Value and t-derivative of the periodic spline at parameters t."""
    M = psi.size
    D = 2.0 * np.pi / M
    tt = np.mod(t, 2.0 * np.pi)
    i = np.minimum(np.floor(tt / D).astype(np.int64), M - 1)
    u = (tt - i * D) / D
    ip = (i + 1) % M
    w = 1.0 - u
    val = w * psi[i] + u * psi[ip] + (D * D / 6.0) * ((w ** 3 - w) * m[i] + (u ** 3 - u) * m[ip])
    der = (psi[ip] - psi[i]) / D + (D / 6.0) * (-(3.0 * w * w - 1.0) * m[i] + (3.0 * u * u - 1.0) * m[ip])
    return val, der


def ellipse_param(geom: G.Geometry, P: np.ndarray):
    """Parameter t and speed |X_t| of points on the ellipse."""
    a, b, c, s = geom.params[:4]
    xr = c * P[:, 0] + s * P[:, 1]
    yr = c * P[:, 1] - s * P[:, 0]
    t = np.mod(np.arctan2(yr / b, xr / a), 2.0 * np.pi)
    speed = np.sqrt((a * yr / b) ** 2 + (b * xr / a) ** 2)
    return t, speed


def surface_2d(geom, psi, m, t, speed, n):
    """psi and grad_Gamma psi at surface points with parameters t."""
    val, der = spline_eval(psi, m, t)
    tau = np.stack([-n[:, 1], n[:, 0]], axis=1)
    return val, (der / speed)[:, None] * tau


# ----------------------------------------------------------------------- 3-D

def six_point_patches(tri: np.ndarray) -> np.ndarray:
    """For every triangle (v0, v1, v2): [v0, v1, v2, o01, o12, o20] where oAB is
    the vertex opposite edge AB in the neighbouring triangle."""
    edge_tris: dict = {}
    for t, (a, b, c) in enumerate(tri):
        for (u, v, w) in ((a, b, c), (b, c, a), (c, a, b)):
            edge_tris.setdefault((min(u, v), max(u, v)), []).append((t, w))
    six = np.empty((tri.shape[0], 6), dtype=np.int64)
    for t, (a, b, c) in enumerate(tri):
        six[t, :3] = (a, b, c)
        for slot, (u, v) in enumerate(((a, b), (b, c), (c, a))):
            lst = edge_tris[(min(u, v), max(u, v))]
            if len(lst) != 2:
                raise ValueError("surface mesh is not a closed manifold")
            other = lst[0] if lst[0][0] != t else lst[1]
            six[t, 3 + slot] = other[1]
    return six


PATCH_MAX = 16


def patches(tri: np.ndarray, n_vert: int):
    """Point lists of every triangle's local fit: the six-point patch
    [v0, v1, v2, o01, o12, o20] when all its points have valence 6, else the
    sorted vertex set of all triangles sharing a vertex with it.
    Returns (ids [n_tri, PATCH_MAX] padded with -1, counts [n_tri])."""
    six = six_point_patches(tri)
    val = np.bincount(tri.ravel(), minlength=n_vert)
    vtris: list = [[] for _ in range(n_vert)]
    for t, row in enumerate(tri):
        for v in row:
            vtris[v].append(t)
    ids = np.full((tri.shape[0], PATCH_MAX), -1, dtype=np.int64)
    cnt = np.empty(tri.shape[0], dtype=np.int64)
    for t in range(tri.shape[0]):
        if np.all(val[six[t]] == 6):
            ids[t, :6] = six[t]
            cnt[t] = 6
            continue
        ring = sorted({int(v) for c in tri[t] for tt in vtris[c] for v in tri[tt]})
        if len(ring) > PATCH_MAX or len(ring) < 6:
            raise ValueError("unsupported vertex ring size")
        ids[t, :len(ring)] = ring
        cnt[t] = len(ring)
    return ids, cnt


def vertex_triangle(tri: np.ndarray, n_vert: int) -> np.ndarray:
    """Lowest-numbered triangle incident to each vertex."""
    vt = np.full(n_vert, np.iinfo(np.int64).max, dtype=np.int64)
    for k in range(3):
        np.minimum.at(vt, tri[:, k], np.arange(tri.shape[0]))
    return vt


def locate(geom: G.Geometry, comp: int, P: np.ndarray) -> np.ndarray:
    """Triangle of the cube-sphere mesh of component `comp` containing the
    surface points P, from their cube-face coordinates."""
    C = geom.components[comp]
    if C.map_type == G.MAP_ELLIPSOID:
        q = P / np.asarray(C.axes)[None, :]
    else:
        q = P.copy()
    aq = np.abs(q)
    k = np.zeros(P.shape[0], dtype=np.int64)
    best = aq[:, 0].copy()
    for ax in (1, 2):
        m = aq[:, ax] > best
        k[m] = ax
        best[m] = aq[m, ax]
    rows = np.arange(P.shape[0])
    qk = q[rows, k]
    face = 2 * k + (qk < 0.0)
    u = q[rows, (k + 1) % 3] / best
    v = q[rows, (k + 2) % 3] / best
    T = geom.cube_t
    n = geom.cube_n
    inner = T[1:n]
    i = np.searchsorted(inner, u, side="right")
    j = np.searchsorted(inner, v, side="right")
    fu = (u - T[i]) / (T[i + 1] - T[i])
    fv = (v - T[j]) / (T[j + 1] - T[j])
    half = (fu + fv > 1.0).astype(np.int64)
    return C.tri_offset + (((face * n + j) * n + i) * 2 + half)


def tangent_basis(n: np.ndarray):
    """Orthonormal tangent vectors t1, t2 with (t1, t2, n) right-handed; t1 is
    built from the coordinate axis least aligned with n."""
    an = np.abs(n)
    k = np.zeros(n.shape[0], dtype=np.int64)
    best = an[:, 0].copy()
    for ax in (1, 2):
        m = an[:, ax] < best
        k[m] = ax
        best[m] = an[m, ax]
    e = np.zeros_like(n)
    e[np.arange(n.shape[0]), k] = 1.0
    t1 = np.cross(e, n)
    t1 /= np.linalg.norm(t1, axis=1)[:, None]
    t2 = np.cross(n, t1)
    return t1, t2


def fit_weights(X: np.ndarray, z: np.ndarray, n: np.ndarray):
    """Weights of the local quadratic fit through K points: psi(z) = w0 . psi_K
    and grad_Gamma psi(z) = wg @ psi_K (interpolation for K = 6, least squares
    for K > 6).  X [P, K, 3], z [P, 3], n [P, 3]; tangent-plane coordinates
    are scaled by the largest distance from z."""
    t1, t2 = tangent_basis(n)
    D = X - z[:, None, :]
    ell = np.sqrt((D ** 2).sum(axis=2)).max(axis=1)
    s = np.einsum("pkd,pd->pk", D, t1) / ell[:, None]
    t = np.einsum("pkd,pd->pk", D, t2) / ell[:, None]
    V = np.stack([np.ones_like(s), s, t, s * s, s * t, t * t], axis=2)
    Vinv = np.linalg.pinv(V)                                   # [P, 6, K]
    w0 = Vinv[:, 0, :]
    wg = (t1[:, :, None] * Vinv[:, 1, None, :] + t2[:, :, None] * Vinv[:, 2, None, :]) / ell[:, None, None]
    return w0, wg, np.linalg.cond(V)


def patch_weights(geom: G.Geometry, ids, cnt, tri_of_point, P, n):
    """Fit weights for points P lying on triangles tri_of_point.  Returns
    (point ids [P, PATCH_MAX], w0 [P, PATCH_MAX], wg [P, 3, PATCH_MAX], cond)
    with zero weights in unused slots."""
    npts = P.shape[0]
    pid = ids[tri_of_point]
    pc = cnt[tri_of_point]
    w0 = np.zeros((npts, PATCH_MAX))
    wg = np.zeros((npts, 3, PATCH_MAX))
    cond = np.zeros(npts)
    for K in np.unique(pc):
        m = pc == K
        a, b, c = fit_weights(geom.nodes[pid[m, :K]], P[m], n[m])
        w0[m, :K] = a
        wg[m, :, :K] = b
        cond[m] = c
    return np.where(pid >= 0, pid, 0), w0, wg, cond
