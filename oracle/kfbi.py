"""Kernel-free boundary integral evaluation of the Neumann problem (oracle).

Scalar problem (Section 2-4 after the decoupling of the isotropic system):
    Lap u - lambda u = f  in Omega,   du/dn = g^N  on the boundary,
with n the outward normal of Omega.  The solution is u = v_V + v_B where
(Section 5.1, Eqs. volume and single)

* v_V solves the box problem with the continuously extended right-hand side
  f on the whole box (no interface jumps, so no correction is needed);
* v_B solves the single-layer interface problem: [v] = 0, [dv/dn] = psi,
  [Lap v - lambda v] = 0 across the boundary, v = 0 on the box boundary.

The boundary integral equation A psi = g (Eq. bie) has
    A psi = dv_B^+/dn   (interior limit, Eq. single-use),
    g     = g^N - dv_V^+/dn.

Jumps used by the correction and the interpolation (derived from [v] = 0 on
the surface, [dv/dn] = psi and [Lap v] = lambda [v] = 0; the paper defers them
to its references):
    [grad v]  = psi n
    [D^2 v]   = psi S + n (grad_G psi)^T + (grad_G psi) n^T - psi tr(S) n n^T
with S the shape operator (positive on convex parts seen from outside).

Correction (Section 5.3, Eq. correct): for a node p whose neighbour p' along
axis a lies across the crossing z, with d = x_{p'} - z,
    J(p') = [v] + [d_a v] d + 1/2 [d_aa v] d^2,
    RHS(p) += -J(p')/h^2 if p is inside Omega, +J(p')/h^2 otherwise,
summed over every crossing arm of the node.

Poisson case (lambda = 0): A then has a one-dimensional null space and its
range is orthogonal to constants (Green's identity: the boundary integral of
dv_B^+/dn equals the volume integral of Lap v_B = 0).  The paper is silent;
reading: the operator is replaced by the rank-one modification
    A psi + <ds, psi> / |Gamma|,
with ds the boundary quadrature weights (2-D: half the lengths of the two
chords at a node; 3-D: a third of the areas of the incident triangles) and
|Gamma| their sum, which is nonsingular and has the same solutions for
compatible data.

Interpolation (Section 5.4, Eqs. taylor-*, ji, je): at an interface node q,
the quadratic Taylor polynomial of v^+ about q is fitted through a 6-point
(2-D) / 10-point (3-D) stencil: the grid node c nearest to q, its 2d axis
neighbours and the d(d-1)/2 diagonal nodes c + s_a e_a + s_b e_b on the side
of q.  Rows of nodes outside Omega use v_j + J_j, with J_j the second-order
Taylor polynomial of the jump about q.  Coordinates are scaled by h.  The
limit is dv^+/dn = n . grad v^+(q).
"""
from __future__ import annotations

import numpy as np

from kfbi_workloads import geometry as G
from kfbi_workloads.configs import Grid
from . import boxsolve, density, grid as GR, krylov
from . import levelset as LS
from . import mesh as MESH


def stencil_offsets(d: int, s: np.ndarray) -> np.ndarray:
    """Index offsets [M, P, d] of the interpolation stencil (geometric axis
    order x, y[, z]); s are the diagonal signs [M, d]."""
    M = s.shape[0]
    offs = [np.zeros((M, d), dtype=np.int64)]
    for a in range(d):
        for step in (-1, 1):
            o = np.zeros((M, d), dtype=np.int64)
            o[:, a] = step
            offs.append(o)
    for a in range(d):
        for b in range(a + 1, d):
            o = np.zeros((M, d), dtype=np.int64)
            o[:, a] = s[:, a]
            o[:, b] = s[:, b]
            offs.append(o)
    return np.stack(offs, axis=1)


def taylor_rows(xi: np.ndarray) -> np.ndarray:
    """Rows of the Taylor system for scaled offsets xi [..., d]: unknowns
    (v, h grad v, h^2 second derivatives)."""
    d = xi.shape[-1]
    cols = [np.ones(xi.shape[:-1])]
    cols += [xi[..., a] for a in range(d)]
    cols += [0.5 * xi[..., a] ** 2 for a in range(d)]
    for a in range(d):
        for b in range(a + 1, d):
            cols.append(xi[..., a] * xi[..., b])
    return np.stack(cols, axis=-1)


def surface_weights(geom: G.Geometry) -> np.ndarray:
    """Quadrature weights of the interface nodes: 2-D, half the lengths of the
    chords to the two neighbouring nodes; 3-D, a third of the areas of the
    triangles incident to the node."""
    X = geom.nodes
    if X.shape[1] == 2:
        seg = np.linalg.norm(np.roll(X, -1, axis=0) - X, axis=1)
        return 0.5 * (seg + np.roll(seg, 1))
    tri = np.asarray(geom.tri, dtype=np.int64)
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    ds = np.zeros(X.shape[0])
    for k in range(3):
        np.add.at(ds, tri[:, k], area / 3.0)
    return ds


class KFBI:
    """Setup (Section 6) and integral evaluations for one geometry and grid."""

    def __init__(self, geom: G.Geometry, grid: Grid):
        self.geom, self.grid = geom, grid
        d = grid.dim
        self.d = d
        self.mesh = geom.kind == G.MESH3
        if self.mesh:
            # the boundary is only a triangle mesh (Section 5.3, Example 4)
            self.patch_ids, self.patch_cnt = density.patches(geom.tri, geom.M)
            self.frames = MESH.tri_frames(geom, self.patch_ids, self.patch_cnt)
            self.inside = MESH.classify(geom, grid)
            self.irregular = GR.irregular_list(self.inside)
            self.ints = MESH.intersections(geom, grid, self.inside, self.frames)
        else:
            self.inside = GR.classify(geom, grid)
            self.irregular = GR.irregular_list(self.inside)
            self.ints = GR.intersections(geom, grid, self.inside)
        self.Pint = GR.intersection_points(grid, self.inside.shape, self.ints)
        nI = self.Pint.shape[0]
        self.n_int = np.empty((nI, d))
        self.S_int = np.empty((nI, d, d))
        if self.mesh:
            if nI:
                self.n_int, self.S_int = MESH.normal_shape(self.frames, self.ints["tri"], self.Pint)
            vt = density.vertex_triangle(geom.tri, geom.M)
            self.n_node, self.S_node = MESH.normal_shape(self.frames, vt, geom.nodes)
        else:
            for c in range(LS.n_components(geom)):
                m = self.ints["comp"] == c
                if np.any(m):
                    self.n_int[m], self.S_int[m] = LS.normal_shape(geom, c, self.Pint[m])
            self.n_node, self.S_node = LS.normals_shapes_at_nodes(geom)
        self.center, self.sign = GR.cell_index(grid, geom.nodes)
        self.ds = surface_weights(geom)
        self.area = float(self.ds.sum())
        self._setup_stencils()
        self._setup_density()

    # ------------------------------------------------------------- setup
    def _setup_stencils(self):
        g, d = self.grid, self.d
        offs = stencil_offsets(d, self.sign)                     # [M, P, d]
        pts = self.center[:, None, :] + offs                     # 1-based node indices
        self.st_idx = pts
        X = g.lo + pts.astype(np.float64) * g.h
        self.st_xi = X - self.geom.nodes[:, None, :]             # physical offsets
        A = taylor_rows(self.st_xi / g.h)
        self.st_A = A
        arr = tuple((pts[..., d - 1 - k] - g.first) for k in range(d))  # array index order
        self.st_flat = np.ravel_multi_index(arr, self.inside.shape)
        self.st_out = ~self.inside.ravel()[self.st_flat]

    def _setup_density(self):
        geom = self.geom
        if self.d == 2:
            self.t_int, self.speed_int = density.ellipse_param(geom, self.Pint)
            M = geom.M
            self.t_node = 2.0 * np.pi * np.arange(M) / M
            _, self.speed_node = density.ellipse_param(geom, geom.nodes)
            return
        ids, cnt = density.patches(geom.tri, geom.M)
        self.patch_ids, self.patch_cnt = ids, cnt
        vt = density.vertex_triangle(geom.tri, geom.M)
        if self.mesh:
            tri_int = self.ints["tri"].copy()       # the triangle the ray crossed
        else:
            tri_int = np.empty(self.Pint.shape[0], dtype=np.int64)
            for c in range(LS.n_components(geom)):
                m = self.ints["comp"] == c
                if np.any(m):
                    tri_int[m] = density.locate(geom, c, self.Pint[m])
        self.tri_int, self.tri_node = tri_int, vt
        self.pid_int, self.w0_int, self.wg_int, self.cond_int = density.patch_weights(
            geom, ids, cnt, tri_int, self.Pint, self.n_int)
        self.pid_node, _, self.wg_node, self.cond_node = density.patch_weights(
            geom, ids, cnt, vt, geom.nodes, self.n_node)

    # --------------------------------------------------------- density
    def density(self, psi: np.ndarray):
        """psi and grad_Gamma psi at the crossings, grad_Gamma psi at the nodes."""
        if self.d == 2:
            m = density.spline_moments(psi)
            p_int, g_int = density.surface_2d(self.geom, psi, m, self.t_int, self.speed_int, self.n_int)
            _, g_node = density.surface_2d(self.geom, psi, m, self.t_node, self.speed_node, self.n_node)
            return p_int, g_int, g_node
        p6 = psi[self.pid_int]
        p_int = (self.w0_int * p6).sum(axis=1)
        g_int = np.einsum("pdk,pk->pd", self.wg_int, p6)
        g_node = np.einsum("pdk,pk->pd", self.wg_node, psi[self.pid_node])
        return p_int, g_int, g_node

    # ----------------------------------------------------------- jumps
    @staticmethod
    def jump_grad_hess(psi, gpsi, n, S):
        """[grad v] and [D^2 v] from psi, grad_Gamma psi, n and S."""
        trS = np.trace(S, axis1=1, axis2=2)
        jg = psi[:, None] * n
        nn = n[:, :, None] * n[:, None, :]
        ng = n[:, :, None] * gpsi[:, None, :]
        jH = psi[:, None, None] * S + ng + ng.transpose(0, 2, 1) - (psi * trS)[:, None, None] * nn
        return jg, jH

    def jumps(self, psi: np.ndarray):
        """Jumps at the crossings ([d_a v], [d_aa v] along each crossing's axis)
        and at the nodes ([grad v], [D^2 v])."""
        p_int, g_int, g_node = self.density(psi)
        jg_i, jH_i = self.jump_grad_hess(p_int, g_int, self.n_int, self.S_int)
        a = self.ints["axis"]
        r = np.arange(a.size)
        dv = jg_i[r, a]
        ddv = jH_i[r, a, a]
        jg_n, jH_n = self.jump_grad_hess(psi, g_node, self.n_node, self.S_node)
        return (dv, ddv), (jg_n, jH_n)

    # ------------------------------------------------------ correction
    def correction(self, jv, dv, ddv) -> np.ndarray:
        """Right-hand side that is zero at regular nodes and carries the
        summed corrections at the irregular nodes.  jv = [v], dv = [d_a v],
        ddv = [d_aa v] at every crossing."""
        g = self.grid
        rhs = np.zeros(self.inside.size)
        ins = self.inside.ravel()
        lo, hi, a, z = self.ints["lo"], self.ints["hi"], self.ints["axis"], self.ints["z"]
        # coordinates of the two end nodes along the crossing axis
        kk = np.unravel_index(lo, self.inside.shape)
        k_a = np.empty(lo.size, dtype=np.int64)
        for ax in range(self.d):
            m = a == ax
            k_a[m] = kk[self.d - 1 - ax][m] + g.first
        xl = g.lo + k_a.astype(np.float64) * g.h
        xh = g.lo + (k_a + 1).astype(np.float64) * g.h
        for node, dist in ((lo, xh - z), (hi, xl - z)):
            J = jv + dv * dist + 0.5 * ddv * dist * dist
            sgn = np.where(ins[node], -1.0, 1.0)
            np.add.at(rhs, node, sgn * J / (g.h * g.h))
        return rhs.reshape(self.inside.shape)

    def correction_from_psi(self, psi):
        (dv, ddv), _ = self.jumps(psi)
        return self.correction(np.zeros_like(dv), dv, ddv)

    # ---------------------------------------------------- interpolation
    def interp(self, v: np.ndarray, node_jumps=None) -> np.ndarray:
        """dv^+/dn at every interface node from the Taylor system; node_jumps
        = ([v] [M], [grad v] [M, d], [D^2 v] [M, d, d]) or None (no jumps)."""
        vals = v.ravel()[self.st_flat].copy()                    # [M, P]
        if node_jumps is not None:
            jv, jg, jH = node_jumps
            xi = self.st_xi
            J = (jv[:, None] + np.einsum("mpd,md->mp", xi, jg)
                 + 0.5 * np.einsum("mpd,mde,mpe->mp", xi, jH, xi))
            vals = vals + np.where(self.st_out, J, 0.0)
        coef = np.linalg.solve(self.st_A, vals[:, :, None])[:, :, 0]
        grad = coef[:, 1:1 + self.d] / self.grid.h
        return (grad * self.n_node).sum(axis=1)

    # -------------------------------------------------------- operators
    def apply_A(self, psi: np.ndarray, lam: float) -> np.ndarray:
        """A psi, plus the rank-one term <ds, psi>/|Gamma| when lam = 0."""
        (dv, ddv), (jg, jH) = self.jumps(psi)
        rhs = self.correction(np.zeros_like(dv), dv, ddv)
        vB = boxsolve.solve(rhs, lam, self.grid)
        out = self.interp(vB, (np.zeros(psi.size), jg, jH))
        if lam == 0.0:
            out = out + (self.ds @ psi) / self.area
        return out

    def volume(self, f: np.ndarray, lam: float) -> np.ndarray:
        return boxsolve.solve(f, lam, self.grid)

    def rhs_g(self, vV: np.ndarray, gN: np.ndarray) -> np.ndarray:
        return gN - self.interp(vV)

    def solve_neumann(self, f, gN, lam, tol=1e-10, psi0=None, restart=50, max_iter=500,
                      method="gmres", gamma=0.8):
        """Full KFBI solve (Algorithm 1, with GMRES or the simple iteration).
        Returns (u on the grid, psi, stats)."""
        vV = self.volume(f, lam)
        g = self.rhs_g(vV, gN)
        x0 = np.zeros(self.geom.M) if psi0 is None else np.asarray(psi0, dtype=np.float64)
        A = lambda x: self.apply_A(x, lam)  # noqa: E731
        if method == "gmres":
            psi, info = krylov.gmres(A, g, x0, tol, restart=restart, max_iter=max_iter)
        else:
            psi, info = krylov.richardson(A, g, x0, tol, gamma=gamma, max_iter=max_iter)
        (dv, ddv), (jg, jH) = self.jumps(psi)
        vB = boxsolve.solve(self.correction(np.zeros_like(dv), dv, ddv), lam, self.grid)
        u = vV + vB
        r = gN - self.interp(u, (np.zeros(psi.size), jg, jH))
        gn = np.linalg.norm(g)
        info["true_rel_res"] = float(np.linalg.norm(r) / gn) if gn > 0 else float(np.linalg.norm(r))
        return u, psi, info
