"""GPU parity of the learned warm start's network and its effect.

* forward outputs and every parameter's gradient against the CPU oracle MLP
  (same bfloat16 rounding of weights and activations, float32 accumulation;
  the remaining differences are summation order and activations that round to
  the other bfloat16 neighbour), relative L2 within 1e-2 (forward) and 3e-2
  (gradients);
* Adam training on the GPU lowers the loss;
* with a network trained on solves of shell runs from four stimulus
  locations, a run from a held-out location needs fewer GMRES iterations
  than with the previous-density start, and the converged states agree with
  that start's to the solver tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C  # noqa: E402
from oracle import mlp as OM  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K, warmstart as WS  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _case(seed=0, B=700):
    rng = np.random.default_rng(seed)
    flat = OM.init(seed) + 0.05 * rng.standard_normal(OM.n_params()).astype(np.float32)
    norm = np.concatenate([rng.uniform(-0.5, 0.5, 9), rng.uniform(0.5, 2.0, 9), [0.1, 2.0]]).astype(np.float32)
    F = rng.standard_normal((B, 9)).astype(np.float32)
    t = rng.standard_normal(B).astype(np.float32)
    return flat, norm, F, t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_forward_matches_oracle():
    flat, norm, F, _ = _case(1)
    m = K.MLP(flat, norm, 1024)
    o = torch.empty(F.shape[0], dtype=torch.float32, device=DEV)
    m.forward(torch.tensor(F, device=DEV), o)
    ref = OM.forward(flat, OM.normalise(F, norm))
    assert _rel(o.cpu().numpy(), ref) < 1e-2
    m.close()


def test_gradients_match_oracle():
    flat, norm, F, t = _case(2, B=512)
    m = K.MLP(flat, norm, 1024)
    loss, g = m.grad(torch.tensor(F, device=DEV), torch.tensor(t, device=DEV))
    loss_ref, g_ref = OM.loss_and_grad(flat, OM.normalise(F, norm), t)
    assert abs(loss - loss_ref) <= 1e-2 * loss_ref
    off = 0
    for s in OM.shapes():
        k = int(np.prod(s))
        assert _rel(g[off:off + k], g_ref[off:off + k]) < 3e-2, (s, _rel(g[off:off + k], g_ref[off:off + k]))
        off += k
    m.close()


def test_training_lowers_loss():
    rng = np.random.default_rng(5)
    F = rng.standard_normal((4096, 9)).astype(np.float32)
    t = (F[:, 0] - F[:, 1] + 0.3 * F[:, 2]).astype(np.float32)
    norm = np.concatenate([np.zeros(9), np.ones(9), [0.0, 1.0]]).astype(np.float32)
    m = K.MLP(OM.init(0), norm, 4096)
    Fd, td = torch.tensor(F, device=DEV), torch.tensor(t, device=DEV)
    l0 = m.grad(Fd, td)[0]
    for _ in range(150):
        loss = m.train_step(Fd, td, 2e-3)
    assert loss < 0.05 * l0
    m.close()


def _run(h, V0, w0, steps, precision):
    V, w = torch.tensor(V0, device=DEV), torch.tensor(w0, device=DEV)
    st = h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=steps, precision=precision)
    return V, w, st


def test_learned_warm_start_reduces_iterations():
    """Runs from a held-out stimulus: the previous-density start (the paper's),
    the history projection, and the projection corrected by a network trained
    on four other stimulus runs.  The learned start needs fewer GMRES
    iterations than the previous-density start; its gain over the projection
    alone is printed (the residual judge keeps the network's guess when its
    residual is smaller, which is not always fewer iterations)."""
    N, steps = 64, 24
    geom, grid, cfg, _, _ = C.config2(N=N, steps=steps)
    normals = C.analytic_normals(geom)
    Fs, Ts = [], []
    for c in C.midwall_centers(C.TRAIN_SEEDS[:4]):
        h = K.KFBI(geom, grid, tol=cfg.tol, precision=K.MIXED)
        V = torch.tensor(C.ball_stimulus(grid, c, 0.1), device=DEV)
        w = torch.zeros_like(V)
        F, T = WS.collect(h, C.FHN_CONFIG, V, w, steps, geom.nodes, normals)
        Fs.append(F)
        Ts.append(T)
        h.close()
    F, T = torch.cat(Fs), torch.cat(Ts)
    norm = WS.fit_norm(F, T)
    m = K.MLP(OM.init(0), norm, max(8192, geom.M))
    losses = WS.train(m, F, T, norm, epochs=20, batch=4096, lr=2e-3)
    assert losses[-1] < 0.5 * losses[0]
    c = C.midwall_centers(C.HELDOUT_SEEDS[:1])[0]
    V0 = C.ball_stimulus(grid, c, 0.1)
    w0 = np.zeros_like(V0)
    runs = {}
    for name, prec, warm in (("previous", K.MIXED, K.WARM_PREVIOUS), ("projection", K.MIXED, K.WARM_PROJECTION),
                             ("learned", K.MIXED_LEARNED, K.WARM_PREVIOUS)):
        hh = K.KFBI(geom, grid, tol=cfg.tol, precision=prec, warm=warm)
        if prec == K.MIXED_LEARNED:
            hh.set_warmstart(m)
        runs[name] = _run(hh, V0, w0, steps, prec)
        hh.close()
    its = {k: sum(s["iters"] for s in r[2][2:]) for k, r in runs.items()}
    used = sum(s["warmstart"] for s in runs["learned"][2])
    print(f"GMRES iterations, steps 3..{steps}: {its} (network guess kept {used}x)")
    assert its["learned"] < its["previous"] and its["projection"] < its["previous"]
    assert all(s["rel_res"] <= cfg.tol for r in runs.values() for s in r[2])
    Vp = runs["previous"][0]
    scale = float(Vp.abs().max())
    for k in ("projection", "learned"):
        assert float((runs[k][0] - Vp).abs().max()) < 1e-6 * scale
