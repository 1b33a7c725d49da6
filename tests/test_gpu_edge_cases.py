"""Degenerate inputs and error paths through the C ABI: zero data gives the
zero solution without iterating, an exhausted iteration budget returns
KFBI_ERR_NOT_CONVERGED with finite outputs written, a domain whose stencils
reach the box boundary is rejected at setup with KFBI_ERR_GEOMETRY, and
out-of-range arguments are rejected before any work."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("prec", [K.FP64, K.MIXED])
def test_zero_data_zero_solution(prec):
    geom, grid = G.star_config1(C.surface_res(32)), C.Grid(3, 32)
    g = K.KFBI(geom, grid, tol=1e-10)
    u = torch.full(grid.shape, 7.0, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    f = torch.zeros(grid.shape, dtype=torch.float64, device=DEV)
    gN = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(f, gN, u, psi, 40.0, precision=prec)
    g.close()
    assert st["iters"] == 0 and st["rel_res"] == 0.0
    assert float(u.abs().max()) == 0.0 and float(psi.abs().max()) == 0.0


@pytest.mark.parametrize("prec", [K.FP64, K.MIXED])
def test_iteration_budget_exhausted(prec):
    geom, grid = G.ellipse_config0(256), C.Grid(2, 128)
    g = K.KFBI(geom, grid)
    f, u_ex, gN = C.manufactured(geom, grid, 60.0)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    st = g.solve_neumann(torch.tensor(f, device=DEV), torch.tensor(gN, device=DEV), u, psi, 60.0,
                         tol=1e-14, max_iter=2, precision=prec)
    g.close()
    assert st["iters"] == 2 and st["rel_res"] > 1e-14
    assert bool(torch.isfinite(u).all()) and bool(torch.isfinite(psi).all())


def test_domain_touching_the_box_is_rejected():
    with pytest.raises(K.KFBIError) as e:
        K.KFBI(G.sphere3(0.95, 8), C.Grid(3, 32))
    assert e.value.code == K.ERR_GEOMETRY


def test_bad_arguments_rejected():
    geom, grid = G.sphere3(0.5, 8), C.Grid(3, 32)
    with pytest.raises(K.KFBIError) as e:
        K.KFBI(geom, C.Grid(3, 48))            # no transform of that length
    assert e.value.code == K.ERR_ARG
    g = K.KFBI(geom, grid)
    with pytest.raises(K.KFBIError) as e:
        g.set_opts(restart=65)                 # above the Krylov basis capacity
    assert e.value.code == K.ERR_ARG
    g.close()
    with pytest.raises(K.KFBIError) as e:
        K.selftest_bounded_wait(0)
    assert e.value.code == K.ERR_ARG


# ------------------------------------------- failures injected on the host

@pytest.mark.parametrize("prec", [K.FP64, K.MIXED])
def test_nan_in_host_data_returns_err_nan(prec):
    """A NaN in the caller's source (or Neumann data) spreads through the box
    solve into g; the solver's first residual is then not finite and the
    call returns KFBI_ERR_NAN (every loop on the way is bounded)."""
    geom, grid = G.ellipse_config0(128), C.Grid(2, 64)
    g = K.KFBI(geom, grid, tol=1e-10)
    f, u_ex, gN = C.manufactured(geom, grid, 60.0)
    u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
    psi = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
    for bad in ("f", "gN"):
        fb, gb = f.copy(), gN.copy()
        if bad == "f":
            fb[10, 20] = np.nan
        else:
            gb[3] = np.nan
        with pytest.raises(K.KFBIError) as e:
            g.solve_neumann(torch.tensor(fb, device=DEV), torch.tensor(gb, device=DEV), u, psi.zero_(), 60.0,
                            precision=prec)
        assert e.value.code == K.ERR_NAN
    # the handle and the context stay usable
    st = g.solve_neumann(torch.tensor(f, device=DEV), torch.tensor(gN, device=DEV), u, psi.zero_(), 60.0,
                         precision=prec)
    assert st["rel_res"] <= 1e-10
    V = torch.tensor(C.ball_stimulus(grid, (-0.4, 0.0), 0.1), device=DEV)
    V[5, 5] = float("nan")
    with pytest.raises(K.KFBIError) as e:
        g.bidomain_step(C.FHN_CONFIG, V, torch.zeros_like(V), None, nsteps=1, precision=prec)
    assert e.value.code == K.ERR_NAN
    g.close()


def test_newton_cap_returns_err_newton():
    """The backward-Euler Newton iteration stops at its cap (|dV| never below
    1e-10 for a NaN state) and the call returns KFBI_ERR_NEWTON; the next call
    on clean data succeeds."""
    V = torch.linspace(-0.2, 1.1, 4096, dtype=torch.float64, device=DEV)
    w = torch.zeros_like(V)
    V[100] = float("nan")
    with pytest.raises(K.KFBIError) as e:
        K.react_be(C.FHN_CONFIG, 0.025, V, w)
    assert e.value.code == K.ERR_NEWTON
    V = torch.linspace(-0.2, 1.1, 4096, dtype=torch.float64, device=DEV)
    w = torch.zeros_like(V)                  # the failed call left a NaN in w too
    K.react_be(C.FHN_CONFIG, 0.025, V, w)
    assert bool(torch.isfinite(V).all())


@pytest.mark.parametrize("prec,tol", [(K.FP64, 1e-10), (K.MIXED, 1e-8)])
def test_step_record_true_residual_and_log(tmp_path, prec, tol):
    """Every Strang step reports the recomputed true residual of the final
    u = v_V + v_B(psi) (not only the solver's estimate) and the device time of
    its phases; the log gets one JSON line per step."""
    import json
    geom, grid, cfg, V0, w0 = C.config0()
    h = K.KFBI(geom, grid, tol=tol, precision=prec, warm=K.WARM_PROJECTION)
    V, w = torch.tensor(V0, device=DEV), torch.tensor(w0, device=DEV)
    log = tmp_path / "steps.jsonl"
    st = h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=3, log=str(log))
    st += h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=2, log=str(log))
    h.close()
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert [x["step"] for x in lines] == [1, 2, 3, 4, 5]
    for s, x in zip(st, lines):
        assert s["rel_res"] <= tol
        # the solver's estimate and the recomputed residual agree to the
        # accuracy of the box solves
        assert 0.0 <= s["true_rel_res"] < 10.0 * tol
        for k in ("react_ms", "rhs_ms", "warm_ms", "solve_ms", "assemble_ms"):
            assert s[k] >= 0.0 and x[k] == s[k]
        assert s["solve_ms"] > 0.0 and x["iters"] == s["iters"]
