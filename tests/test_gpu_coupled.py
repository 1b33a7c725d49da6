"""GPU parity of the anisotropic coupled system (Eq. pde1 with diagonal
conductivities, Section 5.2) through the C ABI against the coupled oracle.

* setup rows: correction and limit tables of both components, through the
  operator they build;
* coupled box solve (per-mode 2 x 2 solve): 1e-12;
* A psi of the density pair: 1e-10;
* the coupled Neumann solve on manufactured data and GMRES at fixed
  iteration counts: 1e-10, iteration counts within one;
* Strang steps with the paper's conductivity ratios (2-D ellipse, 3-D shell):
  V, w and Phi_e within 1e-10 of the oracle's steps;
* with isotropic conductivities the coupled GPU step reproduces the
  decoupled GPU step (Section 3 elimination) to the solver tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from oracle import coupled as CP, krylov  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL64 = 1e-10
DI = (3.0, 0.5, 0.5)   # the paper's diag(30, 5[, 5]), diag(20, 10[, 10]) scaled by 1/10
DE = (2.0, 1.0, 1.0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


CASES = {
    "ellipse128": lambda: (G.ellipse_config0(256), C.Grid(2, 128)),
    "star32": lambda: (G.star_config1(C.surface_res(32)), C.Grid(3, 32)),
    "shell64": lambda: (G.shell_config2(C.surface_res(64)), C.Grid(3, 64)),
    "sphere128": lambda: (G.sphere3(0.9, C.surface_res(128)), C.Grid(3, 128)),
}
_cache = {}


def pair(name):
    if name not in _cache:
        geom, grid = CASES[name]()
        d = grid.dim
        _cache[name] = (geom, grid, CP.CoupledKFBI(geom, grid, DI[:d], DE[:d]),
                        K.KFBI(geom, grid, D_i=DI[:d], D_e=DE[:d], tol=1e-12))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_coupled_box_solve(name):
    geom, grid, o, g = pair(name)
    rng = np.random.default_rng(3)
    ri, re = rng.standard_normal((2,) + grid.shape)
    vi_o, ve_o = o.box_solve(ri, re, 40.0)
    vi = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    ve = torch.empty_like(vi)
    g.box_solve_coupled(cuda(ri), cuda(re), vi, ve, 40.0)
    assert rel(vi.cpu().numpy(), vi_o) < 1e-12 and rel(ve.cpu().numpy(), ve_o) < 1e-12


def _density_pair(geom):
    X = geom.nodes
    a = 1.0 + 0.5 * X[:, 0] - 0.3 * X[:, 1] ** 2
    b = 0.4 - 0.2 * X[:, 1] + (0.3 * X[:, 2] if geom.dim == 3 else 0.1 * X[:, 0] ** 2)
    return np.concatenate([a, b])


@pytest.mark.parametrize("name", list(CASES))
def test_coupled_apply_A(name):
    geom, grid, o, g = pair(name)
    psi = _density_pair(geom)
    out = torch.empty(2 * geom.M, dtype=torch.float64, device=DEV)
    g.apply_A_coupled(cuda(psi), out, 40.0)
    assert rel(out.cpu().numpy(), o.apply_A(psi, 40.0)) < TOL64


@pytest.mark.parametrize("name", ["ellipse128", "star32"])
def test_coupled_gmres_fixed_iterations(name):
    geom, grid, o, g = pair(name)
    gv = np.random.default_rng(5).standard_normal(2 * geom.M)
    for its in (1, 5):
        x, info = krylov.gmres(lambda v: o.apply_A(v, 40.0), gv, np.zeros(2 * geom.M), 0.0, max_iter=its)
        psi = torch.zeros(2 * geom.M, dtype=torch.float64, device=DEV)
        st = g.solve_bie(cuda(gv), psi, 40.0, tol=0.0, max_iter=its)
        g.set_opts(tol=1e-12, max_iter=500)
        assert st["iters"] == its
        assert rel(psi.cpu().numpy(), x) < TOL64


@pytest.mark.parametrize("name", ["ellipse128", "shell64"])
def test_coupled_solve_manufactured(name):
    import test_oracle_coupled as T
    geom, grid, o, g = pair(name)
    kappa = 40.0
    if geom.dim == 2:
        fi, fe, gNi, gNe, _, _ = T._manufactured(geom, grid, kappa, DI, DE)
    else:
        fi, fe, gNi, gNe = _shell_data(geom, grid)
    ui_o, ue_o, psi_o, info = o.solve_neumann(fi, fe, gNi, gNe, kappa, tol=1e-12)
    ui = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    ue = torch.empty_like(ui)
    psi = torch.zeros(2 * geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_coupled(cuda(fi), cuda(fe), cuda(gNi), cuda(gNe), ui, ue, psi, kappa, tol=1e-12)
    print(f"{name}: GMRES iterations GPU {st['iters']} oracle {info['iters']}, true residual {st['true_rel_res']:.2e}")
    assert abs(st["iters"] - info["iters"]) <= 1
    assert st["rel_res"] <= 1e-12 and st["true_rel_res"] < 1e-10
    assert rel(ui.cpu().numpy(), ui_o) < TOL64 and rel(ue.cpu().numpy(), ue_o) < TOL64
    assert rel(psi.cpu().numpy(), psi_o) < TOL64


def _shell_data(geom, grid):
    """Smooth sources for the shell (no closed form needed: parity only):
    f_i = -kappa V, f_e = kappa V for a smooth V, zero Neumann data."""
    X = grid.coords()
    V = np.exp(-((X[0] - 0.8) ** 2 + X[1] ** 2 + X[2] ** 2) / 0.05) * np.ones(grid.shape)
    z = np.zeros(geom.M)
    return -40.0 * V, 40.0 * V, z, z


@pytest.mark.parametrize("name,steps", [("ellipse128", 4), ("shell64", 2)])
def test_coupled_strang_steps(name, steps):
    geom, grid, o, g = pair(name)
    d = grid.dim
    dt = 0.05
    if d == 2:
        V0 = C.ball_stimulus(grid, (-0.4, 0.0), 0.1)
    else:
        V0 = C.ball_stimulus(grid, (0.8, 0.0, 0.0), 0.1)
    w0 = np.zeros_like(V0)
    cb = CP.CoupledBidomain(geom, grid, DI[:d], DE[:d], dt, C.FHN_CONFIG, tol=1e-12)
    V, w = V0.copy(), w0.copy()
    for _ in range(steps):
        V, w, ue_o, info = cb.step(V, w)
        assert info["converged"] and info["newton_ok"]
    h = K.KFBI(geom, grid, D_i=DI[:d], D_e=DE[:d], dt=dt, tol=1e-12)
    Vd, wd = cuda(V0), cuda(w0)
    ued = torch.empty_like(Vd)
    st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, ued, nsteps=steps)
    h.close()
    print(f"coupled {name}: iterations per step {[s['iters'] for s in st]}, "
          f"V {rel(Vd.cpu().numpy(), V):.2e} w {rel(wd.cpu().numpy(), w):.2e} ue {rel(ued.cpu().numpy(), ue_o):.2e}")
    assert all(s["rel_res"] <= 1e-12 and s["true_rel_res"] < 1e-10 for s in st)
    assert rel(Vd.cpu().numpy(), V) < TOL64
    assert rel(wd.cpu().numpy(), w) < TOL64
    assert rel(ued.cpu().numpy(), ue_o) < TOL64


@pytest.mark.parametrize("prec", [K.FP64, K.MIXED])
def test_coupled_fused_reaction_pass_same_as_separate_calls(prec):
    """The coupled step runs the next step's forward half step in the
    backward pass as well: three steps in one call equal three one-step
    calls bit for bit."""
    geom, grid = CASES["ellipse128"]()
    V0 = C.ball_stimulus(grid, (-0.4, 0.0), 0.1)
    w0 = np.zeros_like(V0)
    out = []
    for calls in ((3,), (1, 1, 1)):
        h = K.KFBI(geom, grid, D_i=DI[:2], D_e=DE[:2], dt=0.05, tol=1e-10, precision=prec)
        Vd, wd = cuda(V0), cuda(w0)
        for n in calls:
            h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=n)
        h.close()
        out.append((Vd.cpu().numpy(), wd.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_isotropic_coupled_matches_decoupled_gpu():
    geom, grid, cfg, V0, w0 = C.config0()
    hs = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-12)
    hc = K.KFBI(geom, grid, D_i=(1.0, 1.0), D_e=(2.0, 2.0), dt=0.05, tol=1e-12)
    Vs, ws = cuda(V0), cuda(w0)
    Vc, wc = cuda(V0), cuda(w0)
    hs.bidomain_step(C.FHN_CONFIG, Vs, ws, None, nsteps=3)
    hc.bidomain_step(C.FHN_CONFIG, Vc, wc, None, nsteps=3)
    hs.close()
    hc.close()
    assert rel(Vc.cpu().numpy(), Vs.cpu().numpy()) < 1e-9
    assert rel(wc.cpu().numpy(), ws.cpu().numpy()) < 1e-9


# --------------------------------- float32 transforms with refinement (GMRES-IR)

@pytest.mark.parametrize("name", ["ellipse128", "shell64"])
def test_coupled_mixed_solve(name):
    """The coupled solve with float32 transforms inside GMRES and float64
    refinement: the float64-accurate residual reaches the tolerance and the
    potentials match the float64 oracle to 1e-8."""
    import test_oracle_coupled as T
    geom, grid, o, _ = pair(name)
    kappa = 40.0
    d = grid.dim
    if d == 2:
        fi, fe, gNi, gNe, _, _ = T._manufactured(geom, grid, kappa, DI, DE)
    else:
        fi, fe, gNi, gNe = _shell_data(geom, grid)
    ui_o, ue_o, psi_o, info = o.solve_neumann(fi, fe, gNi, gNe, kappa, tol=1e-12)
    g = K.KFBI(geom, grid, D_i=DI[:d], D_e=DE[:d], tol=1e-10, precision=K.MIXED)
    ui = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    ue = torch.empty_like(ui)
    psi = torch.zeros(2 * geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_coupled(cuda(fi), cuda(fe), cuda(gNi), cuda(gNe), ui, ue, psi, kappa)
    g.close()
    print(f"{name}: mixed iterations {st['iters']} outer {st['outer']}, float64 oracle {info['iters']}, "
          f"true residual {st['true_rel_res']:.2e}")
    assert st["rel_res"] <= 1e-10 and st["true_rel_res"] < 1e-9 and st["outer"] >= 1
    assert rel(ui.cpu().numpy(), ui_o) < 1e-8 and rel(ue.cpu().numpy(), ue_o) < 1e-8


@pytest.mark.parametrize("name,steps", [("ellipse128", 4), ("shell64", 2)])
def test_coupled_mixed_strang_steps(name, steps):
    geom, grid, o, _ = pair(name)
    d = grid.dim
    dt = 0.05
    V0 = C.ball_stimulus(grid, (-0.4, 0.0), 0.1) if d == 2 else C.ball_stimulus(grid, (0.8, 0.0, 0.0), 0.1)
    w0 = np.zeros_like(V0)
    cb = CP.CoupledBidomain(geom, grid, DI[:d], DE[:d], dt, C.FHN_CONFIG, tol=1e-12)
    V, w = V0.copy(), w0.copy()
    for _ in range(steps):
        V, w, ue_o, info = cb.step(V, w)
    h = K.KFBI(geom, grid, D_i=DI[:d], D_e=DE[:d], dt=dt, tol=1e-10, precision=K.MIXED)
    Vd, wd = cuda(V0), cuda(w0)
    ued = torch.empty_like(Vd)
    st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, ued, nsteps=steps)
    h.close()
    print(f"coupled mixed {name}: iterations {[s['iters'] for s in st]}, outer {[s['outer'] for s in st]}, "
          f"V {rel(Vd.cpu().numpy(), V):.2e} ue {rel(ued.cpu().numpy(), ue_o):.2e}")
    assert all(s["rel_res"] <= 1e-10 and s["true_rel_res"] < 1e-9 for s in st)
    assert rel(Vd.cpu().numpy(), V) < 1e-8 and rel(wd.cpu().numpy(), w) < 1e-8
    assert rel(ued.cpu().numpy(), ue_o) < 1e-8


@pytest.mark.parametrize("name,prec,bar", [("ellipse128", K.FP64, TOL64), ("shell64", K.MIXED, 1e-8)])
def test_coupled_projection_warm_start(name, prec, bar):
    """The density-history projection (least squares over the last density
    pairs by their images, plus one simple-iteration step) starts the coupled
    solves: the converged steps are the oracle's, in fewer iterations than
    from the previous density pair."""
    geom, grid, o, _ = pair(name)
    d = grid.dim
    steps = 6
    V0 = C.ball_stimulus(grid, (-0.4, 0.0), 0.1) if d == 2 else C.ball_stimulus(grid, (0.8, 0.0, 0.0), 0.1)
    w0 = np.zeros_like(V0)
    tol = 1e-12 if prec == K.FP64 else 1e-10
    cb = CP.CoupledBidomain(geom, grid, DI[:d], DE[:d], 0.05, C.FHN_CONFIG, tol=1e-12)
    V, w = V0.copy(), w0.copy()
    for _ in range(steps):
        V, w, ue_o, info = cb.step(V, w)
    its = {}
    for warm in (K.WARM_PREVIOUS, K.WARM_PROJECTION):
        h = K.KFBI(geom, grid, D_i=DI[:d], D_e=DE[:d], dt=0.05, tol=tol, precision=prec, warm=warm)
        Vd, wd = cuda(V0), cuda(w0)
        st = h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=steps)
        h.close()
        its[warm] = sum(s["iters"] for s in st[2:])
        assert all(s["rel_res"] <= tol for s in st)
        assert rel(Vd.cpu().numpy(), V) < bar and rel(wd.cpu().numpy(), w) < bar
    print(f"coupled {name}: iterations over steps 3..{steps}: previous {its[K.WARM_PREVIOUS]}, "
          f"projection {its[K.WARM_PROJECTION]}")
    assert its[K.WARM_PROJECTION] < its[K.WARM_PREVIOUS]
