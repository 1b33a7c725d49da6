"""Domains given only by a closed triangle mesh of the boundary (oracle).

Section 5.3 (Fig. 1) and Example 4: in three dimensions the method needs
nothing but the triangulated boundary; normals, tangents and curvatures come
from local coordinate systems built on the six surface points around a
triangle.  This module supplies what the analytic level sets supply for the
other domain kinds:

* Classification of the grid nodes (parity of ray crossings).  For every
  axis a, every triangle is projected onto the plane of the other two axes
  (u, v) = (a+1, a+2 mod 3) and tested against the grid lines parallel to a.
  Each edge is evaluated once, in a canonical direction (lower vertex index
  first), as
      E(p) = (Q_u - P_u)(p_v - P_v) - (Q_v - P_v)(p_u - P_u),
  so the two triangles sharing an edge see the same number.  A point exactly
  on an edge line (E = 0) is moved by the symbolic perturbation
  p + (eps, eps^2): its sign is that of -(Q_v - P_v), or of (Q_u - P_u) when
  that is zero.  A line meets a triangle iff the three signs, each taken in
  the triangle's winding direction, agree; the crossing coordinate is the
  barycentric combination of the vertices' a-coordinates (the centroid's for
  a triangle that is degenerate in projection), clamped to the triangle's
  extent.  A node is inside Omega iff an odd number of crossings on its
  x-line lie beyond it (coordinate > the node's).  Every expression uses only
  correctly rounded +, -, * and / in the order written, so the CUDA setup
  reproduces classification and crossing triangles bit for bit.
* Crossings.  A grid edge whose two nodes differ in status takes the single
  ray crossing of its line in (x_lo, x_hi] (the counting rule above); with
  none, the nearest crossing of the line within 1e-6 h; with more than one,
  or none near, the geometry is rejected.  The crossing point is then moved
  onto the local quadratic surface of that triangle (below) by Newton steps
  along the edge.
* Local surface of a triangle: the frame (centroid o, unit face normal n_f,
  tangents t1, t2 from n_f as for the density fit), coordinates scaled by the
  largest distance ell of the patch points from o, and the quadratic height
  w = h(s, t) = c0 + c1 s + c2 t + c3 s^2 + c4 s t + c5 t^2 through the same
  patch points as the density fit (the six-point patch, or least squares over
  the vertex ring where a vertex has valence other than 6).  The surface is
  the zero set of phi = w - h(s, t), which grows out of Omega, so
  n = grad phi / |grad phi| and S = P Hess(phi) P / |grad phi| as for the
  level sets.
* Normals and shape operators at the interface nodes come from the local
  surface of the node's lowest-numbered incident triangle (the triangle its
  density fit uses).
"""
from __future__ import annotations

import numpy as np

from kfbi_workloads import geometry as G
from kfbi_workloads.configs import Grid
from . import density

NEWTON_STEPS = 30
NEAR_TOL = 1e-6       # fallback window for a crossing, in units of h


class GeometryError(RuntimeError):
    pass


def node_coord(grid: Grid, k):
    return grid.lo + np.asarray(k, dtype=np.float64) * grid.h


# ------------------------------------------------------------ ray crossings

def _canon_sign(Pu, Pv, Qu, Qv, pu, pv):
    """Canonical edge value E and its perturbed sign (+1 / -1)."""
    d1 = Qu - Pu
    d2 = pv - Pv
    d3 = Qv - Pv
    d4 = pu - Pu
    E = d1 * d2 - d3 * d4
    sp = np.where(d3 != 0.0, np.where(d3 < 0.0, 1, -1), np.where(d1 > 0.0, 1, -1))
    sg = np.where(E > 0.0, 1, np.where(E < 0.0, -1, sp))
    return E, sg


def ray_hits(geom: G.Geometry, grid: Grid, axis: int):
    """All crossings of the mesh with the grid's lines parallel to `axis`.

    Returns (lu, lv, x, tri): the node indices k_u, k_v of the line (u, v =
    the two other axes in cyclic order), the crossing coordinate along axis
    and the triangle, sorted by (line, x, tri) with line = k_v * (n) + k_u on
    the field layout."""
    X = geom.nodes
    T = np.asarray(geom.tri, dtype=np.int64)
    a = axis
    u, v = (a + 1) % 3, (a + 2) % 3
    k0, k1 = grid.first, grid.first + grid.n - 1
    out_u, out_v, out_x, out_t = [], [], [], []
    h, lo = grid.h, grid.lo
    for t in range(T.shape[0]):
        ids = T[t]
        P = X[ids]
        umin, umax = P[:, u].min(), P[:, u].max()
        vmin, vmax = P[:, v].min(), P[:, v].max()
        ju0 = max(k0, int(np.floor((umin - lo) / h)) - 1)
        ju1 = min(k1, int(np.ceil((umax - lo) / h)) + 1)
        jv0 = max(k0, int(np.floor((vmin - lo) / h)) - 1)
        jv1 = min(k1, int(np.ceil((vmax - lo) / h)) + 1)
        if ju0 > ju1 or jv0 > jv1:
            continue
        JU, JV = np.meshgrid(np.arange(ju0, ju1 + 1), np.arange(jv0, jv1 + 1), indexing="ij")
        JU, JV = JU.ravel(), JV.ravel()
        pu, pv = node_coord(grid, JU), node_coord(grid, JV)
        e, sg = [], []
        for (i0, i1) in ((0, 1), (1, 2), (2, 0)):
            A, B = ids[i0], ids[i1]
            if A < B:
                E, s = _canon_sign(X[A, u], X[A, v], X[B, u], X[B, v], pu, pv)
            else:
                E, s = _canon_sign(X[B, u], X[B, v], X[A, u], X[A, v], pu, pv)
                E, s = -E, -s
            e.append(E)
            sg.append(s)
        hit = (sg[0] == sg[1]) & (sg[1] == sg[2])
        if not np.any(hit):
            continue
        eAB, eBC, eCA = e[0][hit], e[1][hit], e[2][hit]
        den = (eBC + eCA) + eAB
        mag = (np.abs(eBC) + np.abs(eCA)) + np.abs(eAB)
        Aa, Ba, Ca = X[ids[0], a], X[ids[1], a], X[ids[2], a]
        cen = ((Aa + Ba) + Ca) / 3.0
        degenerate = np.abs(den) <= 1e-12 * mag
        safe = np.where(degenerate, 1.0, den)
        xb = ((eBC * Aa + eCA * Ba) + eAB * Ca) / safe
        xh = np.where(degenerate, cen, xb)
        xh = np.minimum(np.maximum(xh, min(Aa, Ba, Ca)), max(Aa, Ba, Ca))
        out_u.append(JU[hit])
        out_v.append(JV[hit])
        out_x.append(xh)
        out_t.append(np.full(xh.size, t, dtype=np.int64))
    if not out_x:
        z = np.zeros(0, dtype=np.int64)
        return z, z, np.zeros(0), z
    lu, lv = np.concatenate(out_u), np.concatenate(out_v)
    x, tt = np.concatenate(out_x), np.concatenate(out_t)
    line = lv * grid.n + lu
    order = np.lexsort((tt, x, line))
    return lu[order], lv[order], x[order], tt[order]


def classify(geom: G.Geometry, grid: Grid) -> np.ndarray:
    """Inside-Omega mask on the field layout: odd number of x-line crossings
    beyond the node."""
    if grid.dim != 3:
        raise ValueError("mesh domains are three-dimensional")
    lu, lv, x, _ = ray_hits(geom, grid, 0)   # x-lines: u = y, v = z
    n, k0 = grid.n, grid.first
    inside = np.zeros(grid.shape, dtype=bool)
    xs = node_coord(grid, np.arange(k0, k0 + n))
    line = (lv - k0) * n + (lu - k0)
    for ln in np.unique(line):
        hx = x[line == ln]
        beyond = hx.size - np.searchsorted(hx, xs, side="right")   # crossings > node
        iz, iy = divmod(int(ln), n)
        inside[iz, iy, :] = (beyond % 2) == 1
    return inside


# ------------------------------------------------------------ local surfaces

def tri_frames(geom: G.Geometry, ids: np.ndarray, cnt: np.ndarray):
    """Per triangle: centroid o, tangents t1, t2, unit face normal nf, scale
    ell and the height coefficients c [n_tri, 6]."""
    X = geom.nodes
    T = np.asarray(geom.tri, dtype=np.int64)
    A, B, C = X[T[:, 0]], X[T[:, 1]], X[T[:, 2]]
    o = ((A + B) + C) / 3.0
    nf = np.cross(B - A, C - A)
    nf /= np.linalg.norm(nf, axis=1)[:, None]
    t1, t2 = density.tangent_basis(nf)
    ell = np.empty(T.shape[0])
    coef = np.empty((T.shape[0], 6))
    for t in range(T.shape[0]):
        Pp = X[ids[t, :cnt[t]]] - o[t]
        ell[t] = np.sqrt((Pp ** 2).sum(axis=1)).max()
        s = Pp @ t1[t] / ell[t]
        q = Pp @ t2[t] / ell[t]
        w = Pp @ nf[t] / ell[t]
        V = np.stack([np.ones_like(s), s, q, s * s, s * q, q * q], axis=1)
        coef[t] = np.linalg.lstsq(V, w, rcond=None)[0]
    return o, t1, t2, nf, ell, coef


def _local(fr, tri, P):
    o, t1, t2, nf, ell, c = fr
    D = P - o[tri]
    e = ell[tri]
    return (D * t1[tri]).sum(1) / e, (D * t2[tri]).sum(1) / e, (D * nf[tri]).sum(1) / e


def _height(c, s, t):
    h = c[:, 0] + c[:, 1] * s + c[:, 2] * t + c[:, 3] * s * s + c[:, 4] * s * t + c[:, 5] * t * t
    hs = c[:, 1] + 2.0 * c[:, 3] * s + c[:, 4] * t
    ht = c[:, 2] + c[:, 4] * s + 2.0 * c[:, 5] * t
    return h, hs, ht


def normal_shape(fr, tri: np.ndarray, P: np.ndarray):
    """Outward unit normal and shape operator of triangle tri's local surface
    at points P (on or next to it)."""
    o, t1, t2, nf, ell, c = fr
    s, t, _ = _local(fr, tri, P)
    cc = c[tri]
    _, hs, ht = _height(cc, s, t)
    e = ell[tri]
    g = (nf[tri] - hs[:, None] * t1[tri] - ht[:, None] * t2[tri]) / e[:, None]
    T1, T2 = t1[tri], t2[tri]
    o11 = T1[:, :, None] * T1[:, None, :]
    o12 = T1[:, :, None] * T2[:, None, :] + T2[:, :, None] * T1[:, None, :]
    o22 = T2[:, :, None] * T2[:, None, :]
    H = -(2.0 * cc[:, 3, None, None] * o11 + cc[:, 4, None, None] * o12 + 2.0 * cc[:, 5, None, None] * o22)
    H = H / (e * e)[:, None, None]
    gn = np.sqrt((g ** 2).sum(1))
    n = g / gn[:, None]
    Pm = np.eye(3)[None] - n[:, :, None] * n[:, None, :]
    S = np.einsum("nij,njk,nkl->nil", Pm, H, Pm) / gn[:, None, None]
    return n, S


def refine(fr, tri, X0, a, h, tau0):
    """Point X0 + tau h e_a on triangle tri's local surface (Newton from tau0)."""
    o, t1, t2, nf, ell, c = fr
    P = X0.copy()
    P[np.arange(P.shape[0]), a] += tau0 * h
    s0, q0, w0 = _local(fr, tri, X0)
    e = ell[tri]
    ds = h * t1[tri, a] / e
    dq = h * t2[tri, a] / e
    dw = h * nf[tri, a] / e
    cc = c[tri]
    tau = tau0.copy()
    for _ in range(NEWTON_STEPS):
        s, q, w = s0 + tau * ds, q0 + tau * dq, w0 + tau * dw
        hh, hs, hq = _height(cc, s, q)
        f = w - hh
        fp = dw - (hs * ds + hq * dq)
        tau = tau - f / fp
    return tau


# ------------------------------------------------------------ crossings

def intersections(geom: G.Geometry, grid: Grid, inside: np.ndarray, fr):
    """Crossings of the mesh with grid edges whose nodes differ in status:
    dict of axis, lo, hi, z, comp (0) and tri, sorted by (axis, lower node)."""
    d = 3
    n, k0 = grid.n, grid.first
    flat = np.arange(inside.size).reshape(inside.shape)
    out = {k: [] for k in ("axis", "lo", "hi", "z", "comp", "tri")}
    for a in range(d):
        arr_ax = d - 1 - a
        sl0 = [slice(None)] * d
        sl1 = [slice(None)] * d
        sl0[arr_ax] = slice(0, n - 1)
        sl1[arr_ax] = slice(1, n)
        diff = inside[tuple(sl0)] != inside[tuple(sl1)]
        lo_idx = flat[tuple(sl0)][diff]
        hi_idx = flat[tuple(sl1)][diff]
        if lo_idx.size == 0:
            continue
        multi = np.unravel_index(lo_idx, inside.shape)
        kk = [multi[d - 1 - g] + k0 for g in range(d)]       # node indices k of the lower node
        lu, lv, hx, ht = ray_hits(geom, grid, a)
        line_h = lv * n + lu
        u, v = (a + 1) % 3, (a + 2) % 3
        line_c = kk[v] * n + kk[u]
        xl = node_coord(grid, kk[a])
        xh = node_coord(grid, kk[a] + 1)
        tri = np.empty(lo_idx.size, dtype=np.int64)
        xhit = np.empty(lo_idx.size)
        for i in range(lo_idx.size):
            m = line_h == line_c[i]
            hxi, hti = hx[m], ht[m]
            sel = (hxi > xl[i]) & (hxi <= xh[i])
            if np.count_nonzero(sel) == 1:
                j = np.flatnonzero(sel)[0]
            elif np.count_nonzero(sel) == 0 and hxi.size > 0:
                dist = np.maximum(xl[i] - hxi, hxi - xh[i])
                j = int(np.argmin(dist))
                if dist[j] > NEAR_TOL * grid.h:
                    raise GeometryError("status change without a crossing on the edge")
            else:
                raise GeometryError("grid edge crosses the surface more than once")
            tri[i], xhit[i] = hti[j], hxi[j]
        X0 = np.stack([node_coord(grid, kk[g]) for g in range(d)], axis=1)
        tau = refine(fr, tri, X0, a, grid.h, (xhit - xl) / grid.h)
        out["axis"].append(np.full(lo_idx.size, a, dtype=np.int64))
        out["lo"].append(lo_idx.astype(np.int64))
        out["hi"].append(hi_idx.astype(np.int64))
        out["z"].append(xl + tau * grid.h)
        out["comp"].append(np.zeros(lo_idx.size, dtype=np.int64))
        out["tri"].append(tri)
    res = {k: (np.concatenate(v) if v else np.zeros(0, dtype=np.float64 if k == "z" else np.int64))
           for k, v in out.items()}
    order = np.lexsort((res["lo"], res["axis"]))
    return {k: v[order] for k, v in res.items()}
