"""Seeded synthetic workloads: box grids, FitzHugh-Nagumo parameters, initial
states, manufactured exact solutions and random smooth right-hand sides.

Only input data is produced here.  The exact normals used for manufactured
Neumann data come from the analytic surface parametrisation, not from the
level-set machinery of either implementation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import geometry as G


@dataclass(frozen=True)
class Grid:
    """Uniform box grid on [lo, hi]^dim with N intervals per axis, nodes
    x_k = lo + k h (Section 5.2).  The box condition of the interface problems
    picks the unknowns: bc = "dirichlet" (v = 0 on the box boundary) keeps the
    (N-1)^dim interior nodes k = 1..N-1; bc = "neumann" (zero normal
    derivative on the box boundary, the box Green's function of Section 4)
    keeps all (N+1)^dim nodes k = 0..N."""
    dim: int
    N: int
    lo: float = -1.0
    hi: float = 1.0
    bc: str = "dirichlet"

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / self.N

    @property
    def first(self) -> int:
        """Node index k of array index 0 along every axis."""
        return 0 if self.bc == "neumann" else 1

    @property
    def n(self) -> int:
        """Nodes per axis held in a field."""
        return self.N + 1 if self.bc == "neumann" else self.N - 1

    @property
    def shape(self):
        return (self.n,) * self.dim     # [z][y][x] / [y][x], x fastest

    def axis(self) -> np.ndarray:
        k = np.arange(self.first, self.first + self.n, dtype=np.float64)
        return self.lo + k * self.h

    def coords(self):
        """Node coordinates as broadcastable arrays, ordered (x, y[, z])."""
        a = self.axis()
        if self.dim == 2:
            return a[None, :], a[:, None]
        return a[None, None, :], a[None, :, None], a[:, None, None]


@dataclass(frozen=True)
class FHN:
    """FitzHugh-Nagumo membrane model of Section 7:
    I_ion = H (q - V (V - theta)(1 - V)),  M(V, q) = alpha V - zeta q."""
    H: float = 1.0
    theta: float = 0.1
    alpha: float = 0.01
    zeta: float = 0.005
    Cm: float = 1.0
    beta: float = 1.0


FHN_CONFIG = FHN()
FHN_PAPER = FHN(H=100.0, theta=0.25, alpha=0.25, zeta=1.0, Cm=1.0, beta=1000.0)


@dataclass(frozen=True)
class StrangConfig:
    sigma_i: float = 1.0
    sigma_e: float = 2.0
    dt: float = 0.05
    steps: int = 20
    tol: float = 1e-10


def ball_stimulus(grid: Grid, center, radius: float) -> np.ndarray:
    """V = 1 strictly inside the ball |x - center| < radius, else 0."""
    X = grid.coords()
    r2 = sum((X[a] - center[a]) ** 2 for a in range(grid.dim))
    return np.where(r2 < radius * radius, 1.0, 0.0)


# --------------------------------------------------------------------- workloads

def config0(bc: str = "dirichlet"):
    """2-D ellipse, 128^2, 256 nodes, 20 Strang steps of FHN, tol 1e-10 (bc:
    the box condition of the interface problems)."""
    geom = G.ellipse_config0(256)
    grid = Grid(2, 128, bc=bc)
    cfg = StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=20, tol=1e-10)
    V0 = ball_stimulus(grid, (-0.4, 0.0), 0.1)
    return geom, grid, cfg, V0, np.zeros_like(V0)


def surface_res(N: int) -> int:
    """Cube-sphere resolution n for an N^3 grid: n = N/4 (6 n^2 + 2 nodes per
    surface), which keeps the node spacing between about h and 2h.  Nodes much
    finer than the grid leave density modes the grid cannot see, and the
    discrete integral equation then loses its second-kind conditioning
    (GMRES iterations 11, 16, 22, 36, >300 at spacing 2.5h ... 0.47h on a
    sphere of radius 0.6 at N = 32)."""
    return max(4, N // 4)


def config1(N: int):
    """3-D star body, N^3 box grid, cube-sphere nodes of resolution N/4,
    manufactured Neumann modified-Helmholtz solve with lambda = 2/dt = 40,
    tol 1e-10."""
    return G.star_config1(surface_res(N)), Grid(3, N), 40.0, 1e-10


def config2(N: int = 256, steps: int = 200, n_surf: int | None = None, bc: str = "dirichlet"):
    """3-D prolate shell, N^3, FHN bidomain, tol 1e-8; stimulus ball of radius
    0.1 centred on the mid-wall at (0.8, 0, 0) (bc: the box condition)."""
    geom = G.shell_config2(n_surf if n_surf is not None else surface_res(N))
    grid = Grid(3, N, bc=bc)
    cfg = StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=steps, tol=1e-8)
    V0 = ball_stimulus(grid, (0.8, 0.0, 0.0), 0.1)
    return geom, grid, cfg, V0, np.zeros_like(V0)


def virtual_electrode(grid: Grid, v_stim: float = 10.0, offset: float = 0.3, radius: float = 0.25) -> np.ndarray:
    """I_stim of the virtual electrode (Section 7): +v_stim within `radius` of
    the anode at (-offset, 0[, 0]), -v_stim within `radius` of the cathode at
    (+offset, 0[, 0]) (reading of the order of the two positions)."""
    X = grid.coords()
    ra = sum((X[a] - (-offset if a == 0 else 0.0)) ** 2 for a in range(grid.dim))
    rc = sum((X[a] - (offset if a == 0 else 0.0)) ** 2 for a in range(grid.dim))
    out = np.zeros(np.broadcast(*X).shape)
    out[ra < radius * radius] = v_stim
    out[rc < radius * radius] = -v_stim
    return out


def midwall_centers(seeds):
    """Stimulus centres uniform over the mid-wall ellipsoid (0.8, 0.5, 0.5):
    cos(theta) ~ U(-1, 1), phi ~ U(0, 2 pi) from default_rng(seed)."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(s)
        ct = rng.uniform(-1.0, 1.0)
        ph = rng.uniform(0.0, 2.0 * np.pi)
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        out.append((0.8 * st * math.cos(ph), 0.5 * st * math.sin(ph), 0.5 * ct))
    return out


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the warm-start network (9 inputs, 4 hidden
    layers of width 128, 1 output), packed W0[128][9], b0, W1[128][128], b1,
    ..., W4[1][128], b4 as float32: hidden weights uniform in
    +-sqrt(6 / fan_in), biases and the output layer zero."""
    rng = np.random.default_rng(seed)
    dims = [9, 128, 128, 128, 128, 1]
    out = []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        if fan_out > 1:
            lim = np.sqrt(6.0 / fan_in)
            out.append(rng.uniform(-lim, lim, fan_out * fan_in))
        else:
            out.append(np.zeros(fan_out * fan_in))
        out.append(np.zeros(fan_out))
    return np.concatenate(out).astype(np.float32)


TRAIN_SEEDS = tuple(range(8))
HELDOUT_SEEDS = (100, 101, 102, 103)


def gaussian_bumps(seed: int = 0, count: int = 32):
    """Parameters of the smooth random right-hand side: amplitudes U(-1, 1),
    widths U(0.05, 0.2), centres uniform in the outer box of the shell."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(-1.0, 1.0, count)
    width = rng.uniform(0.05, 0.2, count)
    lo = np.array([-0.9, -0.6, -0.6])
    cen = lo + rng.uniform(0.0, 1.0, (count, 3)) * (-2.0 * lo)
    return amp, width, cen


def gaussian_rhs(grid: Grid, seed: int = 0, count: int = 32) -> np.ndarray:
    """f = sum_k a_k exp(-|x - c_k|^2 / (2 s_k^2)) on the interior nodes,
    evaluated through its separable factors."""
    amp, width, cen = gaussian_bumps(seed, count)
    ax = grid.axis()
    e = [np.exp(-((ax[None, :] - cen[:, a:a + 1]) ** 2) / (2.0 * width[:, None] ** 2)) for a in range(3)]
    n = ax.size
    # [z*y, k] @ [k, x]: the bump sum as one matrix product
    zy = (amp[:, None, None] * e[2][:, :, None] * e[1][:, None, :]).reshape(count, n * n)
    return (zy.T @ e[0]).reshape(n, n, n)


# ------------------------------------------------------- manufactured solutions

def exact_u(X):
    """u = prod_a cos(pi x_a)."""
    u = np.ones(np.broadcast(*X).shape)
    for x in X:
        u = u * np.cos(np.pi * x)
    return u


def exact_grad(P: np.ndarray) -> np.ndarray:
    d = P.shape[1]
    c = np.cos(np.pi * P)
    s = np.sin(np.pi * P)
    g = np.empty_like(P)
    for a in range(d):
        t = -np.pi * s[:, a]
        for b in range(d):
            if b != a:
                t = t * c[:, b]
        g[:, a] = t
    return g


def analytic_normals(geom: G.Geometry) -> np.ndarray:
    """Outward unit normals of Omega at the interface nodes, from the analytic
    surface parametrisation (independent of any level-set code)."""
    if geom.kind == G.MESH3:
        if geom.exact_normals is not None:
            return geom.exact_normals
        return analytic_normals(geom.source)
    P = geom.nodes
    if geom.kind == G.ELLIPSE2:
        a, b, c, s = geom.params[:4]
        xr = c * P[:, 0] + s * P[:, 1]
        yr = -s * P[:, 0] + c * P[:, 1]
        t = np.arctan2(yr / b, xr / a)
        # tangent of (a cos t, b sin t) is (-a sin t, b cos t); outward normal (b cos t, a sin t)
        nr = np.stack([b * np.cos(t), a * np.sin(t)], axis=1)
        n = np.stack([c * nr[:, 0] - s * nr[:, 1], s * nr[:, 0] + c * nr[:, 1]], axis=1)
        return n / np.linalg.norm(n, axis=1)[:, None]
    out = np.empty_like(P)
    for comp in geom.components:
        sl = slice(comp.vert_offset, comp.vert_offset + comp.n_vert)
        X = P[sl]
        if comp.map_type == G.MAP_ELLIPSOID:
            ax = np.asarray(comp.axes)
            n = X / ax[None, :] ** 2
        else:
            A, B = geom.params[:2]
            rho = np.linalg.norm(X, axis=1)
            d = X / rho[:, None]
            th = np.arccos(np.clip(d[:, 2], -1.0, 1.0))
            ph = np.arctan2(d[:, 1], d[:, 0])
            st, ct = np.sin(th), np.cos(th)
            e_th = np.stack([ct * np.cos(ph), ct * np.sin(ph), -st], axis=1)
            e_ph = np.stack([-np.sin(ph), np.cos(ph), np.zeros_like(ph)], axis=1)
            r_th = 3.0 * B * np.cos(3 * th) * np.cos(2 * ph)
            # r_phi / sin(theta) = -2 B sin(3 theta)/sin(theta) sin(2 phi); limit 3 at the poles
            q = np.where(st > 1e-300, np.sin(3 * th) / np.where(st > 1e-300, st, 1.0), 3.0 * np.sign(ct))
            r_ph_s = -2.0 * B * q * np.sin(2 * ph)
            n = d - (r_th / rho)[:, None] * e_th - (r_ph_s / rho)[:, None] * e_ph
        n = n / np.linalg.norm(n, axis=1)[:, None]
        out[sl] = -n if comp.flip else n
    return out


def manufactured(geom: G.Geometry, grid: Grid, lam: float):
    """Exact u = prod cos(pi x_a): returns (f on the grid, u on the grid, g^N at
    the nodes) for  Lap u - lam u = f  in Omega,  du/dn = g^N  on the boundary.
    f is the smooth extension  -(d pi^2 + lam) u  evaluated on the whole box."""
    X = grid.coords()
    u = exact_u(X)
    f = -(grid.dim * np.pi ** 2 + lam) * u
    n = analytic_normals(geom)
    gN = (exact_grad(geom.nodes) * n).sum(axis=1)
    return f, u, gN
