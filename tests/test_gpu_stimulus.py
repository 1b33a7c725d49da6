"""The Poisson case (lambda = 0, rank-one modification of the boundary
operator) and the virtual-electrode stimulus (Section 7) through the C ABI,
against the oracle:

* A psi at lambda = 0 (with the rank-one term) and the Neumann Poisson solve
  of a manufactured problem, float64 within 1e-10 and float32 transforms with
  refinement within 1e-8;
* Strang steps with the paper's stiff FitzHugh-Nagumo parameters, dt = h and
  the stimulus on the config-0 ellipse and a 3-D sphere: V, w and the
  extracellular potential from the S problem within 1e-10 (float64) / 1e-8
  (refined float32); and at the stimulus benchmark's size (sphere, 256^3).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from oracle.kfbi import KFBI as OK  # noqa: E402
from oracle.bidomain import Bidomain, extracellular_S  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

DEV = torch.device("cuda:0")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


CASES = {
    "ellipse128": lambda: (G.ellipse_config0(256), C.Grid(2, 128)),
    "sphere32": lambda: (G.sphere3(0.6, 8), C.Grid(3, 32)),
    "star32": lambda: (G.star_config1(C.surface_res(32)), C.Grid(3, 32)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_poisson_apply_and_solve(name):
    geom, grid = CASES[name]()
    o = OK(geom, grid)
    g = K.KFBI(geom, grid, tol=1e-12)
    X = geom.nodes
    psi = 1.0 + 0.5 * X[:, 0] - 0.3 * X[:, 1] ** 2
    out = torch.empty(geom.M, dtype=torch.float64, device=DEV)
    g.apply_A(cuda(psi), out, 0.0)
    assert rel(out.cpu().numpy(), o.apply_A(psi, 0.0)) < 1e-10
    f, u_ex, gN = C.manufactured(geom, grid, 0.0)
    u_ref, psi_ref, info = o.solve_neumann(f, gN, 0.0, tol=1e-12)
    for prec, tol, bar in ((K.FP64, 1e-12, 1e-10), (K.MIXED, 1e-10, 1e-8)):
        u = torch.empty(grid.shape, dtype=torch.float64, device=DEV)
        ps = torch.zeros(geom.M, dtype=torch.float64, device=DEV)
        st = g.solve_neumann(cuda(f), cuda(gN), u, ps, 0.0, tol=tol, max_iter=500, precision=prec)
        assert st["rel_res"] <= tol
        assert rel(u.cpu().numpy(), u_ref) < bar
        assert rel(ps.cpu().numpy(), psi_ref) < bar
    g.close()


STIM = {
    "ellipse128": lambda: (G.ellipse_config0(256), C.Grid(2, 128)),
    "sphere32": lambda: (G.sphere3(0.6, 8), C.Grid(3, 32)),
}


@pytest.mark.parametrize("name", list(STIM))
def test_virtual_electrode_strang(name):
    geom, grid = STIM[name]()
    fhn = C.FHN_PAPER
    steps = 3
    cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=grid.h, steps=steps, tol=1e-12)
    I = C.virtual_electrode(grid)
    bd = Bidomain(geom, grid, cfg, fhn, istim=I)
    V, w = np.zeros(grid.shape), np.zeros(grid.shape)
    for _ in range(steps):
        V, w, info = bd.step(V, w)
        assert info["converged"] and info["newton_ok"]
    ue_ref = extracellular_S(V, bd.solve_S(), bd.k.inside, cfg.sigma_i, cfg.sigma_e)
    for prec, tol, bar in ((K.FP64, 1e-12, 1e-10), (K.MIXED, 1e-10, 1e-8)):
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=grid.h, tol=tol, precision=prec)
        Vd = torch.zeros(grid.shape, dtype=torch.float64, device=DEV)
        wd = torch.zeros_like(Vd)
        ue = torch.empty_like(Vd)
        st = h.bidomain_step(fhn, Vd, wd, ue, nsteps=steps, istim=cuda(I))
        h.close()
        print(f"{name} precision {prec}: V {rel(Vd.cpu().numpy(), V):.2e} w {rel(wd.cpu().numpy(), w):.2e} "
              f"ue {rel(ue.cpu().numpy(), ue_ref):.2e}, iterations {[s['iters'] for s in st]}")
        assert all(s["rel_res"] <= tol for s in st)
        assert rel(Vd.cpu().numpy(), V) < bar
        assert rel(wd.cpu().numpy(), w) < bar
        assert rel(ue.cpu().numpy(), ue_ref) < bar


def test_virtual_electrode_sphere256():
    """The stimulus workload at its benchmark size (sphere r = 0.6, 256^3,
    n = 64): one float64 step (GMRES to 1e-12) within 1e-10 of the oracle, and
    two steps of the float32 form with the history projection at the
    benchmark's 1e-8 tolerance within 1e-7."""
    geom, grid = G.sphere3(0.6, C.surface_res(256)), C.Grid(3, 256)
    fhn = C.FHN_PAPER
    I = C.virtual_electrode(grid)
    for prec, warm, tol_gpu, tol_ref, steps, bar in ((K.FP64, K.WARM_PREVIOUS, 1e-12, 1e-12, 1, 1e-10),
                                                     (K.MIXED, K.WARM_PROJECTION, 1e-8, 1e-10, 2, 1e-7)):
        cfg = C.StrangConfig(sigma_i=1.0, sigma_e=2.0, dt=grid.h, steps=steps, tol=tol_ref)
        bd = Bidomain(geom, grid, cfg, fhn, istim=I)
        V, w = np.zeros(grid.shape), np.zeros(grid.shape)
        for _ in range(steps):
            V, w, info = bd.step(V, w)
            assert info["converged"] and info["newton_ok"]
        ue_ref = extracellular_S(V, bd.solve_S(), bd.k.inside, cfg.sigma_i, cfg.sigma_e)
        h = K.KFBI(geom, grid, sigma_i=1.0, sigma_e=2.0, dt=grid.h, tol=tol_gpu, precision=prec, warm=warm)
        Vd = torch.zeros(grid.shape, dtype=torch.float64, device=DEV)
        wd = torch.zeros_like(Vd)
        ue = torch.empty_like(Vd)
        st = h.bidomain_step(fhn, Vd, wd, ue, nsteps=steps, istim=cuda(I))
        h.close()
        print(f"sphere 256^3 precision {prec}: V {rel(Vd.cpu().numpy(), V):.2e} w {rel(wd.cpu().numpy(), w):.2e} "
              f"ue {rel(ue.cpu().numpy(), ue_ref):.2e}")
        assert all(s["rel_res"] <= tol_gpu for s in st)
        assert rel(Vd.cpu().numpy(), V) < bar
        assert rel(wd.cpu().numpy(), w) < bar
        assert rel(ue.cpu().numpy(), ue_ref) < bar
