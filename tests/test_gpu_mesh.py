"""GPU parity of mesh-only domains (Section 5.3, Example 4: the boundary is
given by its triangle mesh alone) through the C ABI against the oracle.

* classification (ray parity), irregular nodes, crossing edges, stencil
  centres and signs bit-exact; crossing coordinates (moved onto each
  triangle's local surface by Newton steps) within 1e-13;
* correction, interface limit, A psi and g: 1e-10;
* GMRES at fixed iteration counts and the manufactured Neumann solve:
  1e-10, iteration counts within one;
* Strang steps in float64 and with float32 transforms (GMRES-IR): 1e-10 and
  1e-8.
Meshes: a sphere's and the shell's cube-spheres handed over bare (the shell's
inner wall wound towards the hole), and a non-convex geodesic mesh with
valence-5 vertices.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from oracle import krylov  # noqa: E402
from oracle.bidomain import Bidomain  # noqa: E402
from oracle.kfbi import KFBI as OK  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL64 = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


CASES = {
    "sphere_mesh32": lambda: (G.as_mesh(G.sphere3(0.6, C.surface_res(32))), C.Grid(3, 32)),
    "bean32": lambda: (G.bean_mesh(8), C.Grid(3, 32)),
    "bean64": lambda: (G.bean_mesh(16), C.Grid(3, 64)),
    "shell_mesh64": lambda: (G.as_mesh(G.shell_config2(C.surface_res(64))), C.Grid(3, 64)),
    "bean128": lambda: (G.bean_mesh(32), C.Grid(3, 128)),
}
_cache = {}


def pair(name):
    if name not in _cache:
        geom, grid = CASES[name]()
        _cache[name] = (geom, grid, OK(geom, grid), K.KFBI(geom, grid, tol=1e-12))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_mesh_setup(name):
    geom, grid, o, g = pair(name)
    s = g.export_setup()
    assert np.array_equal(s["inside"], o.inside)
    assert np.array_equal(s["irregular"], o.irregular.astype(np.int32))
    assert np.array_equal(s["axis"], o.ints["axis"].astype(np.int32))
    assert np.array_equal(s["lo"], o.ints["lo"].astype(np.int32))
    assert np.abs(s["z"] - o.ints["z"]).max() < 1e-13
    assert np.array_equal(s["center"], o.center.astype(np.int32))
    assert np.array_equal(s["sign"], o.sign.astype(np.int8))
    assert g.info["n_inside"] == int(o.inside.sum())


def _density(geom):
    X = geom.nodes
    return np.cos(2.0 * X[:, 0]) + 0.3 * X[:, 1] * X[:, 2] + 0.5


@pytest.mark.parametrize("name", list(CASES))
def test_mesh_operators(name):
    geom, grid, o, g = pair(name)
    psi = _density(geom)
    out = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.correction(cuda(psi), out)
    assert rel(out.cpu().numpy(), o.correction_from_psi(psi)) < TOL64
    X = np.stack(np.broadcast_arrays(*grid.coords()), -1)
    v = np.cos(2 * X[..., 0]) * np.exp(0.5 * X[..., 1]) + X[..., 2] ** 2
    _, (jg, jH) = o.jumps(psi)
    lim = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.interface_limit(cuda(v), cuda(psi), lim)
    assert rel(lim.cpu().numpy(), o.interp(v, (np.zeros(geom.M), jg, jH))) < TOL64
    g.apply_A(cuda(psi), lim, 40.0)
    assert rel(lim.cpu().numpy(), o.apply_A(psi, 40.0)) < TOL64
    f, u, gN = C.manufactured(geom, grid, 40.0)
    gd = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.rhs_g(cuda(f), cuda(gN), gd, 40.0)
    assert rel(gd.cpu().numpy(), o.rhs_g(o.volume(f, 40.0), gN)) < TOL64


@pytest.mark.parametrize("name", ["bean32", "shell_mesh64"])
def test_mesh_gmres_fixed_iterations(name):
    geom, grid, o, g = pair(name)
    gv = np.random.default_rng(11).standard_normal(geom.M)
    for its in (1, 6):
        x, _ = krylov.gmres(lambda v: o.apply_A(v, 40.0), gv, np.zeros(geom.M), 0.0, max_iter=its)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
        st = g.solve_bie(cuda(gv), psi, 40.0, tol=0.0, max_iter=its)
        g.set_opts(tol=1e-12, max_iter=500)
        assert st["iters"] == its
        assert rel(psi.cpu().numpy(), x) < TOL64


@pytest.mark.parametrize("name", ["sphere_mesh32", "bean64", "shell_mesh64"])
def test_mesh_solve_neumann_manufactured(name):
    geom, grid, o, g = pair(name)
    f, u_ex, gN = C.manufactured(geom, grid, 40.0)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, 40.0, tol=1e-12)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(cuda(f), cuda(gN), u, psi, 40.0, tol=1e-12, max_iter=500)
    assert abs(st["iters"] - info["iters"]) <= 1
    assert st["true_rel_res"] < TOL64
    assert rel(u.cpu().numpy(), u_ref) < TOL64 and rel(psi.cpu().numpy(), psi_ref) < TOL64
    # and the solution is the manufactured one to discretisation accuracy
    assert np.abs(u.cpu().numpy() - u_ex)[o.inside].max() < 2e-2


@pytest.mark.parametrize("prec,bar", [(K.FP64, TOL64), (K.MIXED, 1e-8)])
def test_mesh_strang_steps(prec, bar):
    geom, grid = G.bean_mesh(16), C.Grid(3, 64)
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=3, tol=1e-12 if prec == K.FP64 else 1e-10)
    V0 = C.ball_stimulus(grid, (0.45, 0.0, 0.0), 0.15)
    w0 = np.zeros_like(V0)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, info = bd.step(V, w)
        assert info["converged"]
    h = K.KFBI(geom, grid, tol=cfg.tol, precision=prec, warm=K.WARM_PROJECTION)
    Vd, wd = cuda(V0), cuda(w0)
    st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=cfg.steps)
    h.close()
    assert all(s["rel_res"] <= cfg.tol for s in st)
    assert rel(Vd.cpu().numpy(), V) < bar and rel(wd.cpu().numpy(), w) < bar


def test_mesh_in_the_neumann_box():
    """The mesh-only setup and the Neumann box combine: operators and the
    manufactured solve on the field layout of all (N+1)^3 nodes."""
    geom, grid = G.bean_mesh(8), C.Grid(3, 32, bc="neumann")
    o, g = OK(geom, grid), K.KFBI(geom, grid, tol=1e-12)
    psi = _density(geom)
    lim = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.apply_A(cuda(psi), lim, 40.0)
    assert rel(lim.cpu().numpy(), o.apply_A(psi, 40.0)) < TOL64
    f, u_ex, gN = C.manufactured(geom, grid, 40.0)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, 40.0, tol=1e-12)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    p = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(cuda(f), cuda(gN), u, p, 40.0, tol=1e-12)
    g.close()
    assert abs(st["iters"] - info["iters"]) <= 1
    assert rel(u.cpu().numpy(), u_ref) < TOL64 and rel(p.cpu().numpy(), psi_ref) < TOL64


def test_mesh_coupled_system():
    """The anisotropic coupled system on a mesh-only domain: A psi of the
    density pair and the coupled solve against the coupled oracle."""
    from oracle import coupled as CP
    DI, DE = (3.0, 0.5, 0.5), (2.0, 1.0, 1.0)
    geom, grid = G.bean_mesh(8), C.Grid(3, 32)
    o = CP.CoupledKFBI(geom, grid, DI, DE)
    g = K.KFBI(geom, grid, D_i=DI, D_e=DE, tol=1e-12)
    X = geom.nodes
    psi = np.concatenate([1.0 + 0.5 * X[:, 0] - 0.3 * X[:, 1] ** 2, 0.4 - 0.2 * X[:, 1] + 0.3 * X[:, 2]])
    out = torch.empty(2 * geom.M, dtype=torch.float64, device=DEV)
    g.apply_A_coupled(cuda(psi), out, 40.0)
    assert rel(out.cpu().numpy(), o.apply_A(psi, 40.0)) < TOL64
    Xg = grid.coords()
    V = np.exp(-((Xg[0] - 0.45) ** 2 + Xg[1] ** 2 + Xg[2] ** 2) / 0.05) * np.ones(grid.shape)
    z = np.zeros(geom.M)
    ui_o, ue_o, psi_o, info = o.solve_neumann(-40.0 * V, 40.0 * V, z, z, 40.0, tol=1e-12)
    ui, ue = (torch.empty(grid.shape, dtype=torch.float64, device=DEV) for _ in range(2))
    pd = torch.zeros(2 * geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_coupled(cuda(-40.0 * V), cuda(40.0 * V), cuda(z), cuda(z), ui, ue, pd, 40.0, tol=1e-12)
    g.close()
    assert abs(st["iters"] - info["iters"]) <= 1
    assert rel(ui.cpu().numpy(), ui_o) < TOL64 and rel(ue.cpu().numpy(), ue_o) < TOL64
