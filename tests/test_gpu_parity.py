"""GPU parity: every step of the hot path, called through the C ABI, against
the CPU oracle on the same seeded inputs.

Bars: classification, irregular-node lists, crossings and interface-to-cell
indices bit-exact; float64 fields within 1e-10 relative L-infinity (the
float64 transforms reach ~1e-14); float32 box solves within 2e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from oracle.bidomain import lam_of  # noqa: E402
from oracle import boxsolve, krylov, reaction  # noqa: E402
from oracle.kfbi import KFBI as OK  # noqa: E402
from oracle.bidomain import Bidomain, extracellular  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL64 = 1e-10


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


CASES = {
    "ellipse128": lambda: (G.ellipse_config0(256), C.Grid(2, 128)),
    "ellipse64": lambda: (G.ellipse_config0(128), C.Grid(2, 64)),
    "star32": lambda: (G.star_config1(C.surface_res(32)), C.Grid(3, 32)),
    "star64": lambda: (G.star_config1(C.surface_res(64)), C.Grid(3, 64)),
    "shell64": lambda: (G.shell_config2(C.surface_res(64)), C.Grid(3, 64)),
    "sphere32": lambda: (G.sphere3(0.6, 8), C.Grid(3, 32)),
}

_cache = {}


def pair(name):
    if name not in _cache:
        geom, grid = CASES[name]()
        _cache[name] = (geom, grid, OK(geom, grid), K.KFBI(geom, grid, tol=1e-12))
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_setup_bit_exact(name):
    geom, grid, o, g = pair(name)
    s = g.export_setup()
    assert np.array_equal(s["inside"], o.inside)
    assert np.array_equal(s["irregular"], o.irregular.astype(np.int32))
    assert np.array_equal(s["axis"], o.ints["axis"].astype(np.int32))
    assert np.array_equal(s["lo"], o.ints["lo"].astype(np.int32))
    assert np.array_equal(s["z"].view(np.uint64), o.ints["z"].view(np.uint64))
    assert np.array_equal(s["center"], o.center.astype(np.int32))
    assert np.array_equal(s["sign"], o.sign.astype(np.int8))
    assert g.info["n_inside"] == int(o.inside.sum())


@pytest.mark.parametrize("name,lam", [("ellipse128", 60.0), ("star32", 40.0), ("shell64", 60.0), ("ellipse64", 0.0)])
def test_box_solve(name, lam):
    geom, grid, o, g = pair(name)
    r = np.random.default_rng(7).standard_normal(grid.shape)
    ref = boxsolve.solve(r, lam, grid)
    v = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.box_solve(cuda(r), v, lam, precision=K.FP64)
    assert rel(v.cpu().numpy(), ref) < 1e-12
    g.box_solve(cuda(r), v, lam, precision=K.FP32)
    assert rel(v.cpu().numpy(), ref) < 2e-5
    # float32 transforms refined by two rounds of float64 residuals reach the
    # float64 parity bar
    g.box_solve(cuda(r), v, lam, precision=K.MIXED)
    err = rel(v.cpu().numpy(), ref)
    print(f"refined float32 box solve {name}: rel err {err:.2e}")
    assert err < TOL64


@pytest.mark.parametrize("N", [8, 16, 128])
def test_box_solve_sizes(N):
    # geometry-free sizes: small tiles (one column tile) and the 128^3 pipeline
    geom = G.sphere3(0.3, 4) if N >= 16 else G.sphere3(0.45, 2)
    grid = C.Grid(3, N)
    if N == 8:
        pytest.skip("8^3 grid cannot hold an interface two cells from the box")
    g = K.KFBI(geom, grid)
    r = np.random.default_rng(N).standard_normal(grid.shape)
    v = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.box_solve(cuda(r), v, 40.0)
    assert rel(v.cpu().numpy(), boxsolve.solve(r, 40.0, grid)) < 1e-12


def _smooth_density(geom):
    X = geom.nodes
    return 1.0 + 0.5 * X[:, 0] - 0.3 * X[:, 1] ** 2 + (0.2 * X[:, 2] if geom.dim == 3 else 0.0)


@pytest.mark.parametrize("name", ["ellipse128", "star32", "shell64"])
def test_correction(name):
    geom, grid, o, g = pair(name)
    psi = _smooth_density(geom)
    ref = o.correction_from_psi(psi)
    out = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    g.correction(cuda(psi), out)
    assert rel(out.cpu().numpy(), ref) < TOL64


@pytest.mark.parametrize("name", ["ellipse128", "star32", "shell64"])
def test_interface_limit(name):
    geom, grid, o, g = pair(name)
    X = np.stack(np.broadcast_arrays(*grid.coords()), -1)
    v = np.cos(2 * X[..., 0]) * np.exp(0.5 * X[..., 1]) + (X[..., 2] ** 2 if grid.dim == 3 else 0)
    psi = _smooth_density(geom)
    _, (jg, jH) = o.jumps(psi)
    ref = o.interp(v, (np.zeros(geom.M), jg, jH))
    out = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.interface_limit(cuda(v), cuda(psi), out)
    assert rel(out.cpu().numpy(), ref) < TOL64
    g.interface_limit(cuda(v), None, out)
    assert rel(out.cpu().numpy(), o.interp(v)) < TOL64


@pytest.mark.parametrize("name,lam", [("ellipse128", 60.0), ("star32", 40.0), ("shell64", 60.0)])
def test_apply_A_and_rhs(name, lam):
    geom, grid, o, g = pair(name)
    psi = _smooth_density(geom)
    out = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.apply_A(cuda(psi), out, lam)
    ref = o.apply_A(psi, lam)
    assert rel(out.cpu().numpy(), ref) < TOL64
    g.apply_A(cuda(psi), out, lam, precision=K.MIXED)
    assert rel(out.cpu().numpy(), ref) < 1e-4
    f, u, gN = C.manufactured(geom, grid, lam)
    gd = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.rhs_g(cuda(f), cuda(gN), gd, lam)
    assert rel(gd.cpu().numpy(), o.rhs_g(o.volume(f, lam), gN)) < TOL64


@pytest.mark.parametrize("name,lam", [("ellipse64", 60.0), ("star32", 40.0)])
def test_gmres_fixed_iterations(name, lam):
    geom, grid, o, g = pair(name)
    rng = np.random.default_rng(3)
    gv = rng.standard_normal(geom.M)
    for its in (1, 4, 7):
        x, info = krylov.gmres(lambda v: o.apply_A(v, lam), gv, np.zeros(geom.M), 0.0, max_iter=its)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
        st = g.solve_bie(cuda(gv), psi, lam, tol=0.0, max_iter=its)
        assert st["iters"] == its
        assert rel(psi.cpu().numpy(), x) < TOL64
        assert abs(st["rel_res"] - info["rel_res"]) < 1e-9 * max(info["rel_res"], 1e-3)


@pytest.mark.parametrize("name,lam", [("ellipse64", 60.0), ("sphere32", 40.0)])
def test_gmres_restarted_and_early_stop(name, lam):
    """Restarted GMRES(3) at fixed counts and tolerances met inside a cycle,
    against the oracle's GMRES.  The library enqueues iteration j + 1 before
    the host reads iteration j's residual estimate; the device's stop flag
    must turn that iteration into no work without changing the result."""
    geom, grid, o, _ = pair(name)
    gv = np.random.default_rng(5).standard_normal(geom.M)
    for restart in (3, 50):
        g = K.KFBI(geom, grid, tol=1e-12, restart=restart, max_iter=300)
        try:
            if restart == 3:
                for its in (3, 7):
                    x, info = krylov.gmres(lambda v: o.apply_A(v, lam), gv, np.zeros(geom.M), 0.0, restart=3,
                                           max_iter=its)
                    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
                    st = g.solve_bie(cuda(gv), psi, lam, tol=0.0, max_iter=its)
                    assert st["iters"] == its
                    assert rel(psi.cpu().numpy(), x) < TOL64
            for tol in ((1e-6,) if restart == 3 else (1e-6, 1e-11)):
                x, info = krylov.gmres(lambda v: o.apply_A(v, lam), gv, np.zeros(geom.M), tol, restart=restart,
                                       max_iter=300)
                psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
                st = g.solve_bie(cuda(gv), psi, lam, tol=tol, max_iter=300)
                assert info["converged"] and st["rel_res"] <= tol
                assert st["iters"] == info["iters"], (restart, tol, st["iters"], info["iters"])
                assert rel(psi.cpu().numpy(), x) < max(TOL64, 1e-3 * tol)
        finally:
            g.close()


@pytest.mark.parametrize("name,lam", [("ellipse64", 60.0), ("star32", 40.0)])
def test_richardson_fixed_iterations(name, lam):
    """The simple iteration psi <- psi + 2 gamma (g - A psi), gamma = 0.8
    (Eq. simple iteration, Section 7), against the oracle's at fixed counts."""
    geom, grid, o, g = pair(name)
    gv = np.random.default_rng(4).standard_normal(geom.M)
    for its in (1, 5, 12):
        x, info = krylov.richardson(lambda v: o.apply_A(v, lam), gv, np.zeros(geom.M), 0.0, max_iter=its)
        psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
        st = g.solve_bie(cuda(gv), psi, lam, tol=0.0, max_iter=its, solver=K.RICHARDSON)
        g.set_opts(solver=K.GMRES, max_iter=500)
        assert st["iters"] == its
        assert rel(psi.cpu().numpy(), x) < TOL64
        assert abs(st["rel_res"] - info["rel_res"]) < 1e-9 * info["rel_res"]


def test_strang_stiff_richardson():
    """The paper's stiff FitzHugh-Nagumo parameters (H = 100, theta = 0.25,
    alpha = 0.25, zeta = 1, beta = 1000, Section 7) with dt = h and the simple
    iteration as the solver, on the config-0 ellipse: three Strang steps
    against the oracle (GMRES there; both converged to 1e-12)."""
    geom, grid, _, V0, w0 = C.config0()
    dt = grid.h
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=dt, steps=3, tol=1e-12)
    lam = lam_of(cfg, C.FHN_PAPER)
    bd = Bidomain(geom, grid, cfg, C.FHN_PAPER)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, info = bd.step(V, w)
        assert info["converged"] and info["newton_ok"]
    for prec, tol, bar in ((K.FP64, 1e-12, TOL64), (K.MIXED, 1e-10, 1e-8)):
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=dt, tol=tol, solver=K.RICHARDSON, max_iter=2000,
                   precision=prec)
        Vd, wd = cuda(V0), cuda(w0)
        st = h.bidomain_step(C.FHN_PAPER, Vd, wd, None, nsteps=cfg.steps)
        h.close()
        print(f"stiff FHN, simple iteration, precision {prec}: iterations per step {[s['iters'] for s in st]}")
        assert all(s["rel_res"] <= tol for s in st)
        assert rel(Vd.cpu().numpy(), V) < bar
        assert rel(wd.cpu().numpy(), w) < bar


@pytest.mark.parametrize("name,lam", [("ellipse128", 60.0), ("star64", 40.0), ("shell64", 60.0), ("sphere32", 40.0)])
def test_solve_neumann_manufactured(name, lam):
    geom, grid, o, g = pair(name)
    f, u_ex, gN = C.manufactured(geom, grid, lam)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, lam, tol=1e-12)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(cuda(f), cuda(gN), u, psi, lam, tol=1e-12, max_iter=500)
    assert abs(st["iters"] - info["iters"]) <= 1
    assert st["true_rel_res"] < 1e-11
    assert rel(u.cpu().numpy(), u_ref) < TOL64
    assert rel(psi.cpu().numpy(), psi_ref) < TOL64


@pytest.mark.parametrize("name,lam", [("ellipse128", 60.0), ("star64", 40.0), ("shell64", 60.0)])
def test_solve_neumann_mixed(name, lam):
    """GMRES-IR (float32 box solves inside GMRES, float64 Arnoldi, refined
    float64-accurate outer residuals) converges to the float64 solution: at a
    1e-10 GMRES tolerance the fields agree with the oracle's to 1e-8."""
    geom, grid, o, g = pair(name)
    f, u_ex, gN = C.manufactured(geom, grid, lam)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, lam, tol=1e-12)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(cuda(f), cuda(gN), u, psi, lam, tol=1e-10, max_iter=500, precision=K.MIXED)
    g.set_opts(precision=K.FP64)
    assert st["rel_res"] <= 1e-10 and st["true_rel_res"] < 1e-9 and st["outer"] >= 1
    assert rel(u.cpu().numpy(), u_ref) < 1e-8
    assert rel(psi.cpu().numpy(), psi_ref) < 1e-8


def test_strang_config0_mixed():
    geom, grid, cfg, V0, w0 = C.config0()
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=5, tol=1e-12)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, _ = bd.step(V, w)
    h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-10, precision=K.MIXED)
    Vd, wd = cuda(V0), cuda(w0)
    h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=cfg.steps, tol=1e-10, precision=K.MIXED)
    assert rel(Vd.cpu().numpy(), V) < 1e-8
    assert rel(wd.cpu().numpy(), w) < 1e-8


@pytest.mark.parametrize("prec,warm", [(K.FP64, K.WARM_PREVIOUS), (K.MIXED, K.WARM_PROJECTION)])
def test_fused_reaction_pass_same_as_separate_calls(prec, warm):
    """Within one call the forward half step of every step after the first
    runs in the previous step's backward pass (and, for the float32 forms,
    the midpoint too): the same float64 operations as the separate passes, so
    three steps in one call equal three one-step calls bit for bit."""
    geom, grid, cfg, V0, w0 = C.config0()
    out = []
    for calls in ((3,), (1, 1, 1)):
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-10, precision=prec, warm=warm)
        Vd, wd = cuda(V0), cuda(w0)
        for n in calls:
            h.bidomain_step(C.FHN_CONFIG, Vd, wd, None, nsteps=n)
        h.close()
        out.append((Vd.cpu().numpy(), wd.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_reaction_half_steps():
    rng = np.random.default_rng(11)
    V0 = rng.uniform(-0.3, 1.2, 100_003)
    q0 = rng.uniform(-0.1, 0.3, V0.size)
    for fhn, k in ((C.FHN_CONFIG, 0.025), (C.FHN_PAPER, 0.002)):
        V, q = cuda(V0), cuda(q0)
        K.react_fe(fhn, k, V, q)
        Vr, qr = reaction.forward_euler(V0, q0, k, fhn)
        assert rel(V.cpu().numpy(), Vr) < 1e-15 and rel(q.cpu().numpy(), qr) < 1e-15
        V, q = cuda(V0), cuda(q0)
        K.react_be(fhn, k, V, q)
        Vr, qr, ok = reaction.backward_euler(V0, q0, k, fhn)
        assert ok.all()
        assert rel(V.cpu().numpy(), Vr) < 1e-12 and rel(q.cpu().numpy(), qr) < 1e-12


def test_reaction_be_float_pair_paths():
    """Backward Euler on the float-pair path and its float64 fallback against
    the oracle: states at and below the pairs' range (zeros, |v| < 2^-60,
    1e-17), ordinary states, and stiff half steps (c = k H / Cm up to 3.5)
    whose float32 Newton phase may not settle, so that float64 steps finish
    them.  V and q within 1e-12 of the oracle (max-normalised) and, for the
    tiny states, within 1e-17 absolute."""
    rng = np.random.default_rng(23)
    tiny = np.array([0.0, -0.0, 1e-25, -3e-20, 5e-19, -1e-17, 2.0 ** -60, 1e-12])
    V0 = np.concatenate([tiny, rng.uniform(-0.3, 1.2, 20_000)])
    q0 = np.concatenate([tiny[::-1], rng.uniform(-0.1, 0.3, 20_000)])
    for fhn, k in ((C.FHN_CONFIG, 0.025), (C.FHN_PAPER, 0.002), (C.FHN_PAPER, 0.02), (C.FHN_PAPER, 0.035)):
        Vr, qr, ok = reaction.backward_euler(V0, q0, k, fhn)
        assert ok.all()
        V, q = cuda(V0), cuda(q0)
        K.react_be(fhn, k, V, q)
        Vg, qg = V.cpu().numpy(), q.cpu().numpy()
        assert rel(Vg, Vr) < 1e-12 and rel(qg, qr) < 1e-12, (fhn, k)
        n = tiny.size
        assert np.abs(Vg[:n] - Vr[:n]).max() < 1e-17 and np.abs(qg[:n] - qr[:n]).max() < 1e-17, (fhn, k)


def test_strang_config0():
    """Config 0 (2-D ellipse, 128^2) for its 20 Strang steps against the
    oracle, with a 1e-12 GMRES tolerance on both sides: V, w and u_e within
    1e-10."""
    geom, grid, cfg, V0, w0 = C.config0()
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=0.05, steps=20, tol=1e-12)
    lam = lam_of(cfg, C.FHN_CONFIG)
    bd = Bidomain(geom, grid, cfg, C.FHN_CONFIG)
    V, w = V0.copy(), w0.copy()
    for _ in range(cfg.steps):
        V, w, _ = bd.step(V, w)
    ue_ref = extracellular(V, bd.k.inside, cfg.sigma_i, cfg.sigma_e)
    h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-12)
    Vd, wd, ued = cuda(V0), cuda(w0), torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    stats = h.bidomain_step(C.FHN_CONFIG, Vd, wd, ued, nsteps=cfg.steps, tol=1e-12)
    assert all(s["rel_res"] <= 1e-12 for s in stats)
    assert rel(Vd.cpu().numpy(), V) < TOL64
    assert rel(wd.cpu().numpy(), w) < TOL64
    assert rel(ued.cpu().numpy(), ue_ref) < TOL64
