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
