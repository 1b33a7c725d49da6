"""Level sets of the domains, their normals and shape operators (oracle).

Classification (Section 5.3: regular/irregular nodes) needs the sign of a level
set Phi at every grid node, and the GPU must agree bit for bit.  Every level
set here therefore uses only correctly rounded +, -, *, / and sqrt, in the
fixed order written below (numpy applies no FMA contraction to elementwise
expressions).  Phi < 0 is inside a closed surface; Phi == 0 counts as inside
Omega.

Normals and shape operators at surface points (needed for the jumps of
Section 5.3 and the Taylor systems of Section 5.4) come from the gradient and
Hessian of the same level sets, evaluated with a small second-order
forward-mode jet: n = grad Phi / |grad Phi| and S = P (Hess Phi) P / |grad Phi|
with P = I - n n^T, negated on surfaces whose outward normal (of Omega) is
-grad Phi (the inner wall of the shell).

Reading for the star body at the two poles (x = y = 0), where
r = A + B sin(3 theta) cos(2 phi) is not differentiable: the B term and its
derivatives are taken as zero there.
"""
from __future__ import annotations

import numpy as np

from kfbi_workloads import geometry as G


# ----------------------------------------------------------------- plain values

def phi_ellipse2(x, y, a, b, c, s):
    xr = c * x + s * y
    yr = c * y - s * x
    u = xr / a
    v = yr / b
    return (u * u + v * v) - 1.0


def phi_ellipsoid(x, y, z, a, b, c):
    u = x / a
    v = y / b
    w = z / c
    return ((u * u + v * v) + w * w) - 1.0


def phi_star(x, y, z, A, B):
    x2 = x * x
    y2 = y * y
    z2 = z * z
    s2 = x2 + y2
    r2 = s2 + z2
    rho = np.sqrt(r2)
    pos = s2 > 0.0
    s2s = np.where(pos, s2, 1.0)
    r2s = np.where(pos, r2, 1.0)
    rhos = np.where(pos, rho, 1.0)
    s = np.sqrt(s2s)
    g = ((x2 - y2) / s2s) * ((s / rhos) * (3.0 - 4.0 * (s2s / r2s)))
    g = np.where(pos, g, 0.0)
    return (rho - A) - B * g


def component_phi(geom: G.Geometry, comp: int, X):
    """Level set of one closed surface; X = (x, y[, z]) broadcastable arrays."""
    p = geom.params
    if geom.kind == G.ELLIPSE2:
        return phi_ellipse2(X[0], X[1], p[0], p[1], p[2], p[3])
    if geom.kind == G.ELLIPSOID3:
        return phi_ellipsoid(X[0], X[1], X[2], p[0], p[1], p[2])
    if geom.kind == G.STAR3:
        return phi_star(X[0], X[1], X[2], p[0], p[1])
    if geom.kind == G.SHELL3:
        o = 0 if comp == 0 else 3
        return phi_ellipsoid(X[0], X[1], X[2], p[o], p[o + 1], p[o + 2])
    raise ValueError("unknown geometry kind")


def n_components(geom: G.Geometry) -> int:
    return 2 if geom.kind == G.SHELL3 else 1


def component_pred(geom: G.Geometry, comp: int, X):
    """Per-surface predicate used for crossings: True on the 'enclosed' side.
    Outer surfaces enclose Phi <= 0; the inner wall of the shell encloses the
    hole Phi < 0 (so that Phi == 0 on either wall counts as inside Omega)."""
    ph = component_phi(geom, comp, X)
    if geom.kind == G.SHELL3 and comp == 1:
        return ph < 0.0
    return ph <= 0.0


def inside(geom: G.Geometry, X):
    """True where the point lies in Omega (ties on the surface count inside)."""
    if geom.kind == G.SHELL3:
        return component_pred(geom, 0, X) & ~component_pred(geom, 1, X)
    return component_pred(geom, 0, X)


# ------------------------------------------------------------------ 2-jets

class Jet:
    """Value, gradient and Hessian of a scalar field at n points."""
    __slots__ = ("v", "g", "H")

    def __init__(self, v, g, H):
        self.v, self.g, self.H = v, g, H

    @staticmethod
    def var(X, k):
        n, d = X.shape
        g = np.zeros((n, d))
        g[:, k] = 1.0
        return Jet(X[:, k].copy(), g, np.zeros((n, d, d)))

    @staticmethod
    def const(c, n, d):
        return Jet(np.full(n, float(c)), np.zeros((n, d)), np.zeros((n, d, d)))

    def __add__(self, o):
        if isinstance(o, Jet):
            return Jet(self.v + o.v, self.g + o.g, self.H + o.H)
        return Jet(self.v + o, self.g, self.H)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, -self.H)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if isinstance(o, Jet):
            outer = self.g[:, :, None] * o.g[:, None, :]
            return Jet(self.v * o.v, self.g * o.v[:, None] + o.g * self.v[:, None],
                       self.H * o.v[:, None, None] + o.H * self.v[:, None, None] + outer
                       + outer.transpose(0, 2, 1))
        return Jet(self.v * o, self.g * o, self.H * o)

    __rmul__ = __mul__

    def recip(self):
        r = 1.0 / self.v
        gg = self.g[:, :, None] * self.g[:, None, :]
        return Jet(r, -self.g * (r * r)[:, None],
                   -self.H * (r * r)[:, None, None] + 2.0 * gg * (r * r * r)[:, None, None])

    def __truediv__(self, o):
        if isinstance(o, Jet):
            return self * o.recip()
        return self * (1.0 / o)

    def sqrt(self):
        s = np.sqrt(self.v)
        gg = self.g[:, :, None] * self.g[:, None, :]
        return Jet(s, self.g / (2.0 * s)[:, None],
                   self.H / (2.0 * s)[:, None, None] - gg / (4.0 * s ** 3)[:, None, None])


def _phi_jet(geom: G.Geometry, comp: int, P: np.ndarray) -> Jet:
    n, d = P.shape
    X = [Jet.var(P, k) for k in range(d)]
    p = geom.params
    if geom.kind == G.ELLIPSE2:
        a, b, c, s = p[:4]
        u = (X[0] * c + X[1] * s) * (1.0 / a)
        v = (X[1] * c - X[0] * s) * (1.0 / b)
        return u * u + v * v - 1.0
    if geom.kind in (G.ELLIPSOID3, G.SHELL3):
        o = 3 if (geom.kind == G.SHELL3 and comp == 1) else 0
        a, b, c = p[o:o + 3]
        u, v, w = X[0] * (1.0 / a), X[1] * (1.0 / b), X[2] * (1.0 / c)
        return u * u + v * v + w * w - 1.0
    if geom.kind == G.STAR3:
        A, B = p[:2]
        x2, y2, z2 = X[0] * X[0], X[1] * X[1], X[2] * X[2]
        s2 = x2 + y2
        r2 = s2 + z2
        rho = r2.sqrt()
        out = rho - A
        pos = s2.v > 0.0
        if np.any(pos):
            idx = np.nonzero(pos)[0]
            sub = lambda J: Jet(J.v[idx], J.g[idx], J.H[idx])  # noqa: E731
            S2, R2, X2, Y2 = sub(s2), sub(r2), sub(x2), sub(y2)
            gterm = ((X2 - Y2) / S2) * ((S2.sqrt() / R2.sqrt()) * (3.0 - 4.0 * (S2 / R2)))
            out.v[idx] -= B * gterm.v
            out.g[idx] -= B * gterm.g
            out.H[idx] -= B * gterm.H
        return out
    raise ValueError("unknown geometry kind")


def normal_shape(geom: G.Geometry, comp: int, P: np.ndarray):
    """Outward (of Omega) unit normal n [n, d] and shape operator S [n, d, d]
    (tangential, S = P Hess(Phi) P / |grad Phi|) at surface points P [n, d]."""
    J = _phi_jet(geom, comp, np.asarray(P, dtype=np.float64))
    gnorm = np.sqrt((J.g ** 2).sum(axis=1))
    n = J.g / gnorm[:, None]
    d = P.shape[1]
    Pm = np.eye(d)[None] - n[:, :, None] * n[:, None, :]
    S = np.einsum("nij,njk,nkl->nil", Pm, J.H, Pm) / gnorm[:, None, None]
    flip = geom.kind == G.SHELL3 and comp == 1
    if flip:
        n, S = -n, -S
    return n, S


def node_components(geom: G.Geometry) -> np.ndarray:
    """Surface component of every interface node."""
    comp = np.zeros(geom.M, dtype=np.int64)
    for c, C in enumerate(geom.components):
        comp[C.vert_offset:C.vert_offset + C.n_vert] = c
    return comp


def normals_shapes_at_nodes(geom: G.Geometry):
    d = geom.dim
    n = np.empty((geom.M, d))
    S = np.empty((geom.M, d, d))
    comp = node_components(geom)
    for c in range(n_components(geom)):
        m = comp == c
        n[m], S[m] = normal_shape(geom, c, geom.nodes[m])
    return n, S
