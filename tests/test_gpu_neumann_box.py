"""GPU parity of the Neumann box (the box Green's function of Section 4 with
zero normal derivative on the box boundary: all (N+1)^d nodes, mirrored ghost
rows, cosine transforms) through the C ABI against the oracle.

* DCT-I box solve: 1e-12 relative at sizes whose tiles are ragged (N + 1
  lines never fill the last tile);
* correction scatter, interface limit, A psi and g on the Neumann layout:
  1e-10;
* GMRES at fixed iteration counts and the manufactured Neumann solve: 1e-10,
  iteration counts within one;
* Strang steps (config 0 for its 20 steps, the 3-D shell for 2): V, w and
  u_e within 1e-10;
* the solution inside Omega agrees with the Dirichlet box's to second order;
* float32 transforms: the plain float32 solve within 2e-5, refined solves,
  GMRES-IR and the float32 Strang forms within 1e-8 of the float64 oracle;
* what the Neumann box does not support is rejected with KFBI_ERR_ARG.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from oracle import boxsolve, krylov  # noqa: E402
from oracle.bidomain import Bidomain, extracellular, lam_of  # noqa: E402
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


def ngrid(dim, N):
    return C.Grid(dim, N, bc="neumann")


CASES = {
    "ellipse128": lambda: (G.ellipse_config0(256), ngrid(2, 128)),
    "ellipse64": lambda: (G.ellipse_config0(128), ngrid(2, 64)),
    "star32": lambda: (G.star_config1(C.surface_res(32)), ngrid(3, 32)),
    "shell64": lambda: (G.shell_config2(C.surface_res(64)), ngrid(3, 64)),
}
_cache = {}


def pair(name):
    if name not in _cache:
        geom, grid = CASES[name]()
        _cache[name] = (geom, grid, OK(geom, grid), K.KFBI(geom, grid, tol=1e-12))
    return _cache[name]


@pytest.mark.parametrize("dim,N,lam", [(2, 16, 60.0), (2, 64, 5.0), (2, 128, 60.0), (2, 512, 60.0), (3, 8, 40.0),
                                       (3, 16, 40.0), (3, 32, 60.0), (3, 64, 40.0), (3, 128, 40.0)])
def test_dct_box_solve(dim, N, lam):
    geom = G.ellipse_config0(64) if dim == 2 else G.sphere3(0.5, 4)
    grid = ngrid(dim, N)
    g = K.KFBI(geom, grid)
    r = np.random.default_rng(N + dim).standard_normal(grid.shape)
    ref = boxsolve.solve(r, lam, grid)
    v = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.box_solve(cuda(r), v, lam, precision=K.FP64)
    g.close()
    assert rel(v.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("name", ["ellipse128", "star32", "shell64"])
def test_correction_and_limit(name):
    geom, grid, o, g = pair(name)
    X = geom.nodes
    psi = 1.0 + 0.5 * X[:, 0] - 0.3 * X[:, 1] ** 2 + (0.2 * X[:, 2] if geom.dim == 3 else 0.0)
    out = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.correction(cuda(psi), out)
    assert rel(out.cpu().numpy(), o.correction_from_psi(psi)) < TOL64
    Xg = np.stack(np.broadcast_arrays(*grid.coords()), -1)
    v = np.cos(2 * Xg[..., 0]) * np.exp(0.5 * Xg[..., 1]) + (Xg[..., 2] ** 2 if grid.dim == 3 else 0)
    _, (jg, jH) = o.jumps(psi)
    lim = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.interface_limit(cuda(v), cuda(psi), lim)
    assert rel(lim.cpu().numpy(), o.interp(v, (np.zeros(geom.M), jg, jH))) < TOL64
    pa = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.apply_A(cuda(psi), pa, 60.0)
    assert rel(pa.cpu().numpy(), o.apply_A(psi, 60.0)) < TOL64
    f, u, gN = C.manufactured(geom, grid, 60.0)
    gd = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.rhs_g(cuda(f), cuda(gN), gd, 60.0)
    assert rel(gd.cpu().numpy(), o.rhs_g(o.volume(f, 60.0), gN)) < TOL64


@pytest.mark.parametrize("name,lam", [("ellipse64", 60.0), ("star32", 40.0)])
def test_gmres_fixed_iterations(name, lam):
    geom, grid, o, g = pair(name)
    gv = np.random.default_rng(3).standard_normal(geom.M)
    for its in (1, 4, 7):
        x, info = krylov.gmres(lambda v: o.apply_A(v, lam), gv, np.zeros(geom.M), 0.0, max_iter=its)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
        st = g.solve_bie(cuda(gv), psi, lam, tol=0.0, max_iter=its)
        assert st["iters"] == its
        assert rel(psi.cpu().numpy(), x) < TOL64


@pytest.mark.parametrize("name,lam", [("ellipse128", 60.0), ("star32", 40.0), ("shell64", 60.0)])
def test_solve_neumann_manufactured(name, lam):
    geom, grid, o, g = pair(name)
    f, u_ex, gN = C.manufactured(geom, grid, lam)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, lam, tol=1e-12)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(cuda(f), cuda(gN), u, psi, lam, tol=1e-12, max_iter=500)
    assert abs(st["iters"] - info["iters"]) <= 1
    # the recomputed residual bottoms out at the rounding of the float64
    # transforms seen through the 1/h of the limit (2.5e-11 at 128^2; the
    # oracle's library transform reaches 7e-13)
    assert st["true_rel_res"] < TOL64
    assert rel(u.cpu().numpy(), u_ref) < TOL64
    assert rel(psi.cpu().numpy(), psi_ref) < TOL64


def test_neumann_and_dirichlet_box_agree_inside():
    """Both boxes represent the same solution in Omega (Section 4): on the
    manufactured problem their GPU solutions differ by about the
    discretisation error, far less than either's distance to zero."""
    geom = G.ellipse_config0(256)
    out = {}
    for bc in ("dirichlet", "neumann"):
        grid = C.Grid(2, 128, bc=bc)
        f, u_ex, gN = C.manufactured(geom, grid, 60.0)
        g = K.KFBI(geom, grid, tol=1e-12)
        u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
        g.solve_neumann(cuda(f), cuda(gN), u, psi, 60.0)
        g.close()
        ins = OK(geom, grid).inside
        un = u.cpu().numpy()
        out[bc] = (un[1:-1, 1:-1][ins[1:-1, 1:-1]] if bc == "neumann" else un[ins],
                   np.abs(un - u_ex)[ins].max())
    d = np.abs(out["neumann"][0] - out["dirichlet"][0]).max()
    assert d < 2.0 * max(out["neumann"][1], out["dirichlet"][1]) and d < 1e-3


def test_strang_config0_neumann_box():
    geom, grid, cfg, V0, w0 = C.config0(bc="neumann")
    assert V0.shape == (129, 129)
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=20, tol=1e-12)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, _ = bd.step(V, w)
    ue_ref = extracellular(V, bd.k.inside, cfg.sigma_i, cfg.sigma_e)
    h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-12)
    Vd, wd, ued = cuda(V0), cuda(w0), torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, ued, nsteps=cfg.steps, tol=1e-12)
    h.close()
    assert all(s["rel_res"] <= 1e-12 and s["true_rel_res"] < 1e-10 for s in st)
    assert rel(Vd.cpu().numpy(), V) < TOL64
    assert rel(wd.cpu().numpy(), w) < TOL64
    assert rel(ued.cpu().numpy(), ue_ref) < TOL64


def test_strang_shell64_neumann_box_projection():
    """3-D shell with the projection warm start: 3 steps against the oracle's
    steps (any initial guess converges to the same density)."""
    geom, grid, cfg, V0, w0 = C.config2(N=64, steps=3, bc="neumann")
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=3, tol=1e-12)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, _ = bd.step(V, w)
    h = K.KFBI(geom, grid, tol=1e-12, warm=K.WARM_PROJECTION)
    Vd, wd = cuda(V0), cuda(w0)
    st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=cfg.steps, tol=1e-12)
    h.close()
    assert all(s["true_rel_res"] < 1e-10 for s in st)
    assert rel(Vd.cpu().numpy(), V) < TOL64
    assert rel(wd.cpu().numpy(), w) < TOL64


def test_unsupported_forms_rejected():
    geom, grid = G.ellipse_config0(128), ngrid(2, 64)
    with pytest.raises(K.KFBIError) as e:
        K.KFBI(geom, grid, D_i=(1.0, 1.0), D_e=(2.0, 2.0))
    assert e.value.code == K.ERR_ARG
    g = K.KFBI(geom, grid)
    r = torch.zeros(grid.shape, dtype=torch.float64, device=DEV)
    v = torch.empty_like(r)
    with pytest.raises(K.KFBIError) as e:        # no Poisson Green's function
        g.box_solve(r, v, 0.0, precision=K.FP64)
    assert e.value.code == K.ERR_ARG
    g.close()


# ----------------------------------------- float32 transforms, refinement, GMRES-IR

@pytest.mark.parametrize("dim,N", [(2, 128), (3, 64), (3, 128)])
def test_dct_box_solve_float32_and_refined(dim, N):
    geom = G.ellipse_config0(64) if dim == 2 else G.sphere3(0.5, 4)
    grid = ngrid(dim, N)
    g = K.KFBI(geom, grid, tol=1e-10)
    r = np.random.default_rng(N + 7).standard_normal(grid.shape)
    ref = boxsolve.solve(r, 60.0, grid)
    v = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.box_solve(cuda(r), v, 60.0, precision=K.FP32)
    assert rel(v.cpu().numpy(), ref) < 2e-5
    g.box_solve(cuda(r), v, 60.0, precision=K.MIXED)   # float32 transforms + float64 residual rounds
    g.close()
    assert rel(v.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("name,lam", [("ellipse128", 60.0), ("shell64", 60.0)])
def test_solve_neumann_mixed(name, lam):
    geom, grid, o, _ = pair(name)
    f, u_ex, gN = C.manufactured(geom, grid, lam)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, lam, tol=1e-12)
    g = K.KFBI(geom, grid, tol=1e-10, precision=K.MIXED)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(cuda(f), cuda(gN), u, psi, lam)
    g.close()
    assert st["rel_res"] <= 1e-10 and st["true_rel_res"] < 1e-9 and st["outer"] >= 1
    assert rel(u.cpu().numpy(), u_ref) < 1e-8


def test_strang_config0_neumann_box_mixed_learned_forms():
    """Config 0 in the Neumann box with float32 transforms, from the previous
    density and from the history projection: V, w within 1e-8 of the oracle."""
    geom, grid, cfg, V0, w0 = C.config0(bc="neumann")
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=10, tol=1e-12)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, _ = bd.step(V, w)
    for warm in (K.WARM_PREVIOUS, K.WARM_PROJECTION):
        h = K.KFBI(geom, grid, tol=1e-10, precision=K.MIXED, warm=warm)
        Vd, wd = cuda(V0), cuda(w0)
        st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=cfg.steps)
        h.close()
        assert all(s["rel_res"] <= 1e-10 and s["true_rel_res"] < 1e-9 for s in st)
        assert rel(Vd.cpu().numpy(), V) < 1e-8 and rel(wd.cpu().numpy(), w) < 1e-8
