"""GPU parity of the learned warm start's network and its effect.

* every layer of the forward pass (training path), the output, the deltas of
  the backward pass and every parameter's gradient, element by element
  against the CPU oracle MLP applied to the GPU's own inputs of each layer,
  within bounds derived from bfloat16 rounding and float32 summation order
  (tests/mlp_bounds.py); the fused inference kernel against the training
  path's output;
* Adam training on the GPU lowers the loss;
* with a network trained on solves of shell runs from four stimulus
  locations, runs from a held-out location: GMRES iterations of the
  previous-density start (the paper's), the history projection and the
  learned correction of the projection.  The learned start needs fewer
  iterations than the previous density; against the projection it does not
  gain: a point-wise network cannot represent the non-local correction the
  projection leaves (the measured ratio is printed and bounded).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import mlp_bounds as MB  # noqa: E402
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
    T = rng.standard_normal(B).astype(np.float32)
    return flat, norm, F, T


def test_forward_layers_elementwise():
    flat, norm, F, _ = _case(1)
    m = K.MLP(flat, norm, 1024)
    Fd = torch.tensor(F, device=DEV)
    z, o, _, _ = m.layers(Fd)
    report = {}
    MB.check_forward(flat, OM.normalise(F, norm), z.cpu().numpy(), o.cpu().numpy(), report)
    # the fused inference kernel: same fragments, order and epilogue per element
    o2 = torch.empty_like(o)
    m.forward(Fd, o2)
    d = float((o2 - o).abs().max())
    print(f"per-layer (max |diff|, max bound, violations): {report}; fused vs layered max |diff| {d:.2e}")
    assert d <= 1e-5 * (1.0 + float(o.abs().max()))
    # the whole network against the oracle's, for scale: flips of bfloat16
    # roundings compound over the layers, so this is a loose sanity check
    ref = OM.forward(flat, OM.normalise(F, norm))
    assert np.linalg.norm(o.cpu().numpy() - ref) < 1e-2 * np.linalg.norm(ref)
    m.close()


def test_backward_layers_and_gradients_elementwise():
    flat, norm, F, T = _case(2, B=512)
    m = K.MLP(flat, norm, 1024)
    Fd, Td = torch.tensor(F, device=DEV), torch.tensor(T, device=DEV)
    z, o, d, d4 = m.layers(Fd, Td)
    loss, g = m.grad(Fd, Td)
    X = OM.normalise(F, norm)
    t = ((T - norm[18]) / norm[19]).astype(np.float32)
    report = {}
    zn, on = z.cpu().numpy(), o.cpu().numpy()
    MB.check_forward(flat, X, zn, on, report)
    MB.check_backward(flat, X, t, zn, on, d.cpu().numpy(), d4.cpu().numpy(), g, loss, report)
    print(f"per-layer (max |diff|, max bound, violations): {report}")
    m.close()


def test_fit_norm_matches_oracle():
    from oracle import warmstart as OW
    rng = np.random.default_rng(7)
    F = (rng.standard_normal((5000, 9)) * rng.uniform(0.1, 3.0, 9) + rng.uniform(-2, 2, 9)).astype(np.float32)
    F[:, 4] = 0.25                                   # zero spread -> 1
    T = (0.3 * rng.standard_normal(5000) + 0.1).astype(np.float32)
    got = K.MLP.fit_norm(torch.tensor(F, device=DEV), torch.tensor(T, device=DEV))
    ref = OW.fit_norm(F, T)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


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


def test_learned_warm_start_against_previous_and_projection():
    """Runs from a held-out stimulus: the previous-density start (the paper's),
    the history projection, and the projection corrected by a network trained
    on four other stimulus runs.  The learned start needs fewer GMRES
    iterations than the previous density.  It does not beat the projection it
    corrects: the residual judge keeps the network's guess when its residual
    is smaller, but that guess's error is spread over more modes of A, which
    GMRES resolves more slowly.  The measured ratio is printed and bounded."""
    N, steps = 64, 24
    geom, grid, cfg, _, _ = C.config2(N=N, steps=steps)
    Fs, Ts = [], []
    for c in C.midwall_centers(C.TRAIN_SEEDS[:4]):
        h = K.KFBI(geom, grid, tol=cfg.tol, precision=K.MIXED)
        V = torch.tensor(C.ball_stimulus(grid, c, 0.1), device=DEV)
        w = torch.zeros_like(V)
        F, T = WS.collect(h, C.FHN_CONFIG, V, w, steps)
        Fs.append(F)
        Ts.append(T)
        h.close()
    F, T = torch.cat(Fs), torch.cat(Ts)
    norm = WS.fit_norm(F, T)
    m = K.MLP(WS.init_params(0), norm, max(8192, geom.M))
    losses = WS.train(m, F, T, epochs=20, batch=4096, lr=2e-3)
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
    ratio = its["learned"] / its["projection"]
    print(f"GMRES iterations, steps 3..{steps}: {its} (network guess kept {used}x); "
          f"learned / projection = {ratio:.3f}")
    assert its["learned"] < its["previous"] and its["projection"] < its["previous"]
    assert ratio < 1.25
    assert all(s["rel_res"] <= cfg.tol for r in runs.values() for s in r[2])
    Vp = runs["previous"][0]
    scale = float(Vp.abs().max())
    for k in ("projection", "learned"):
        assert float((runs[k][0] - Vp).abs().max()) < 1e-6 * scale
