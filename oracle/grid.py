"""Cartesian-grid preprocessing (oracle): node classification, irregular
nodes, grid-line intersections and interface-to-cell indexing (Section 5.3,
Section 6).

Grid: box [lo, hi]^d with N intervals per axis, h = (hi - lo)/N; node k has
coordinate lo + k*h (one multiply, one add).  Arrays hold the grid's field
nodes, [z][y][x] with x fastest: the (N-1)^d interior nodes of the Dirichlet
box (box-boundary nodes carry the value 0 and count as outside Omega), or all
(N+1)^d nodes of the Neumann box (Omega never reaches the box boundary, so
those nodes are outside Omega and regular).

* A node is irregular iff one of its 2d axis neighbours has the other
  inside/outside status (its 5/7-point stencil crosses the interface).
* Every axis edge whose two end nodes differ in status holds one crossing
  point z, found by 64 bisection steps on the level set of the surface whose
  predicate changes along the edge (bit-reproducible: only the level set's
  correctly rounded operations and midpoints).
* Interface-to-cell indexing of a point q: centre index
  c_a = floor((q_a - lo)/h + 0.5) and diagonal sign s_a = +1 if
  q_a >= lo + c_a h, else -1.
"""
from __future__ import annotations

import numpy as np

from kfbi_workloads.configs import Grid
from kfbi_workloads import geometry as G
from . import levelset as LS

BISECT_ITERS = 64


class GeometryError(RuntimeError):
    pass


def node_coord(grid: Grid, k):
    return grid.lo + np.asarray(k, dtype=np.float64) * grid.h


def classify(geom: G.Geometry, grid: Grid) -> np.ndarray:
    """Boolean inside-Omega mask over the interior nodes, shape (N-1)^d."""
    return LS.inside(geom, grid.coords())


def irregular_mask(inside: np.ndarray) -> np.ndarray:
    """Irregular iff an axis neighbour differs; box-boundary neighbours are
    outside.  An inside node next to the box boundary is a geometry error."""
    d = inside.ndim
    irr = np.zeros_like(inside)
    for ax in range(d):
        pad = [(0, 0)] * d
        pad[ax] = (1, 1)
        P = np.pad(inside, pad, constant_values=False)
        sl_m = [slice(None)] * d
        sl_p = [slice(None)] * d
        sl_m[ax] = slice(0, -2)
        sl_p[ax] = slice(2, None)
        irr |= (P[tuple(sl_m)] != inside) | (P[tuple(sl_p)] != inside)
        # inside nodes touching the box boundary
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = 0
        last[ax] = -1
        if inside[tuple(first)].any() or inside[tuple(last)].any():
            raise GeometryError("domain touches the box boundary")
    return irr


def irregular_list(inside: np.ndarray) -> np.ndarray:
    """Compacted flat indices of the irregular nodes, increasing."""
    return np.flatnonzero(irregular_mask(inside)).astype(np.int64)


def _axis_of_flat(d: int, ax: int):
    """Array axis holding geometric axis `ax` (x is the last array axis)."""
    return d - 1 - ax


def intersections(geom: G.Geometry, grid: Grid, inside: np.ndarray):
    """All crossings of the interface with grid-line edges.

    Returns a dict of arrays sorted by (axis, lower node):
      axis  int   geometric axis a (0 = x)
      lo    int   flat index of the lower end node (index k along a)
      hi    int   flat index of the upper end node (k + 1)
      z     float coordinate of the crossing along axis a
      comp  int   surface component crossed
    """
    d = grid.dim
    n1 = grid.n
    out = {k: [] for k in ("axis", "lo", "hi", "z", "comp")}
    flat = np.arange(inside.size).reshape(inside.shape)
    ncomp = LS.n_components(geom)
    for a in range(d):
        arr_ax = _axis_of_flat(d, a)
        sl0 = [slice(None)] * d
        sl1 = [slice(None)] * d
        sl0[arr_ax] = slice(0, n1 - 1)
        sl1[arr_ax] = slice(1, n1)
        diff = inside[tuple(sl0)] != inside[tuple(sl1)]
        lo_idx = flat[tuple(sl0)][diff]
        hi_idx = flat[tuple(sl1)][diff]
        if lo_idx.size == 0:
            continue
        # node indices k of the lower node along each axis
        multi = np.unravel_index(lo_idx, inside.shape)
        kk = [None] * d
        for g_ax in range(d):
            kk[g_ax] = multi[_axis_of_flat(d, g_ax)] + grid.first
        Xlo = [node_coord(grid, kk[g]) for g in range(d)]
        Xhi = list(Xlo)
        Xhi[a] = node_coord(grid, kk[a] + 1)
        # which surface changes its predicate along the edge
        comp = np.full(lo_idx.size, -1, dtype=np.int64)
        for c in range(ncomp):
            ch = LS.component_pred(geom, c, Xlo) != LS.component_pred(geom, c, Xhi)
            if np.any(ch & (comp >= 0)):
                raise GeometryError("edge crosses two surfaces")
            comp[ch] = c
        if np.any(comp < 0):
            raise GeometryError("status change without a crossing surface")
        z = np.empty(lo_idx.size)
        for c in range(ncomp):
            m = comp == c
            if not np.any(m):
                continue
            lo_u = Xlo[a][m].copy()
            hi_u = Xhi[a][m].copy()
            fixed = [X[m] for X in Xlo]
            X = list(fixed)
            X[a] = lo_u
            p_lo = LS.component_pred(geom, c, X)
            for _ in range(BISECT_ITERS):
                mid = 0.5 * (lo_u + hi_u)
                X[a] = mid
                pm = LS.component_pred(geom, c, X)
                same = pm == p_lo
                lo_u = np.where(same, mid, lo_u)
                hi_u = np.where(same, hi_u, mid)
            z[m] = 0.5 * (lo_u + hi_u)
        out["axis"].append(np.full(lo_idx.size, a, dtype=np.int64))
        out["lo"].append(lo_idx.astype(np.int64))
        out["hi"].append(hi_idx.astype(np.int64))
        out["z"].append(z)
        out["comp"].append(comp)
    res = {k: (np.concatenate(v) if v else np.zeros(0, dtype=np.float64 if k == "z" else np.int64))
           for k, v in out.items()}
    order = np.lexsort((res["lo"], res["axis"]))
    return {k: v[order] for k, v in res.items()}


def intersection_points(grid: Grid, shape, ints) -> np.ndarray:
    """Cartesian coordinates [n_int, d] of the crossing points."""
    d = grid.dim
    multi = np.unravel_index(ints["lo"], shape)
    P = np.empty((ints["lo"].size, d))
    for g in range(d):
        P[:, g] = node_coord(grid, multi[_axis_of_flat(d, g)] + grid.first)
    for a in range(d):
        m = ints["axis"] == a
        P[m, a] = ints["z"][m]
    return P


def cell_index(grid: Grid, P: np.ndarray):
    """Stencil centre indices c [M, d] (1-based node indices) and diagonal
    signs s [M, d] of points P [M, d]."""
    t = (P - grid.lo) / grid.h
    c = np.floor(t + 0.5).astype(np.int64)
    xc = grid.lo + c.astype(np.float64) * grid.h
    s = np.where(P >= xc, 1, -1).astype(np.int64)
    if np.any(c < 2) or np.any(c > grid.N - 2):
        raise GeometryError("interpolation stencil leaves the interior grid")
    return c, s
