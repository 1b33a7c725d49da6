"""GPU parity of the warm starts' steps against the oracle (oracle/warmstart).

After Strang steps of the learned form on the 64^3 shell (float32 transforms
with GMRES-IR, tol 1e-8) with a non-zero network:
* the history projection: psi_F and r_F of the next step against the
  oracle's least-squares projection of the same history and right-hand side,
  element by element (r_F is unique; psi_F too, the stored images being
  linearly independent here);
* the network's input rows and training targets (kfbi_training_rows) against
  the oracle's features and targets built from the GPU's psi_F, r_F, g and psi;
* the initial density the solve started from (kfbi_get_warm_guess) against
  the oracle's prediction psi_F + 2 gamma r_F + rms(r_F)(s_out o + m_out) for
  the network's output o on those rows;
* the projection form (no network): its start psi_F + 2 gamma r_F.
The network's own layers are checked element-wise in test_gpu_mlp.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C  # noqa: E402
from oracle import mlp as OM, warmstart as OW  # noqa: E402
from oracle.kfbi import KFBI as OK  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _vec(M):
    return torch.empty(M, dtype=torch.float64, device=DEV)


def _net(seed=3):
    rng = np.random.default_rng(seed)
    flat = OM.init(seed) + 0.05 * rng.standard_normal(OM.n_params()).astype(np.float32)
    norm = np.concatenate([np.zeros(9), np.ones(9), [0.05, 0.5]]).astype(np.float32)
    return flat, norm


@pytest.mark.parametrize("form", ["learned", "projection"])
def test_warm_start_steps_match_oracle(form):
    geom, grid, cfg, V0, w0 = C.config2(N=64)
    M = geom.M
    prec = K.MIXED_LEARNED if form == "learned" else K.MIXED
    h = K.KFBI(geom, grid, sigma_i=cfg.sigma_i, sigma_e=cfg.sigma_e, dt=cfg.dt, tol=cfg.tol, precision=prec,
               warm=K.WARM_PROJECTION)
    flat, norm = _net()
    m = None
    if form == "learned":
        m = K.MLP(flat, norm, M)
        h.set_warmstart(m)
    V, w = torch.tensor(V0, device=DEV), torch.tensor(w0, device=DEV)
    h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=4)
    ph = torch.empty((K.HISTORY, M), dtype=torch.float64, device=DEV)
    gh = torch.empty_like(ph)
    n = h.get_history(ph, gh)
    st = h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=1)[0]
    psiF, rF, psi0, psi, g = _vec(M), _vec(M), _vec(M), _vec(M), _vec(M)
    h.get_projection(psiF, rF)
    h.get_warm_guess(psi0)
    h.get_densities(psi, None, g)
    F = torch.empty((M, 9), dtype=torch.float32, device=DEV)
    T = torch.empty(M, dtype=torch.float32, device=DEV)
    h.training_rows(F, T)
    torch.cuda.synchronize()
    k = min(n, K.HISTORY)
    psiF_g, rF_g, g_g = psiF.cpu().numpy(), rF.cpu().numpy(), g.cpu().numpy()
    # projection
    psiF_o, rF_o, c = OW.projection(ph.cpu().numpy()[:k], gh.cpu().numpy()[:k], g_g)
    print(f"{form}: history {k}, coefficients {np.round(c, 4)}, |r_F|/|g| "
          f"{np.linalg.norm(rF_o) / np.linalg.norm(g_g):.2e}")
    assert np.abs(rF_g - rF_o).max() <= 1e-9 * np.abs(g_g).max()
    assert rel(psiF_g, psiF_o) < 1e-7
    # rows and targets from the GPU's own projection and converged density
    o_nodes = OK(geom, grid).n_node
    F_o = OW.features(psiF_g, rF_g, g_g, geom.nodes, o_nodes)
    T_o = OW.target(psi.cpu().numpy(), psiF_g, rF_g)
    Fg = F.cpu().numpy()
    assert np.abs(Fg - F_o).max() <= 4e-7 * np.maximum(np.abs(F_o).max(axis=0), 1.0).max()
    assert np.abs(T.cpu().numpy() - T_o).max() <= 1e-6 * np.abs(T_o).max()
    # the start of the solve
    if form == "learned":
        o = torch.empty(M, dtype=torch.float32, device=DEV)
        m.forward(F, o)
        ref = OW.prediction(psiF_g, rF_g, o.cpu().numpy(), norm)
        # the network saw these rows: its output is checked against the
        # oracle's in test_gpu_mlp; here only the denormalisation and sum
        # float64 sum; s_out o + m_out in float32 on both sides (possibly
        # fused into one rounding on the GPU)
        rF_rms = float(np.sqrt(np.mean(rF_g ** 2)))
        corr = np.abs(norm[19] * o.cpu().numpy()) + abs(norm[18])
        assert np.all(np.abs(psi0.cpu().numpy() - ref) <= 1e-13 * np.abs(ref).max() + 2.0 ** -22 * rF_rms * corr)
        assert float(o.abs().max()) > 1e-3                    # the network adds something
        o_ref = OM.forward(flat, OM.normalise(F_o, norm))
        assert np.linalg.norm(o.cpu().numpy() - o_ref) < 1e-2 * np.linalg.norm(o_ref)
        print(f"learned guess kept: {st['warmstart']}")
        m.close()
    else:
        assert rel(psi0.cpu().numpy(), psiF_g + 2.0 * 0.8 * rF_g) < 1e-14
    assert st["rel_res"] <= cfg.tol
    h.close()
