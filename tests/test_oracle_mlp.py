"""Pins of the oracle MLP: bfloat16 rounding against its definition, the
written-out backward pass against central finite differences (checked with
bfloat16 rounding switched off so the loss is smooth), Adam against a
closed-form first step, and training on a linear target.  The untrained
network's effect on the warm start is pinned in test_oracle_warmstart."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_definition():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-39, np.inf], np.float32)
    r = mlp.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # exactly half an ulp: ties to even (down)
    assert r[2] == np.float32(1.0 + 2 ** -7)  # representable
    assert r[3] == np.float32(1.0 + 2 ** -6)  # half an ulp above an odd mantissa: up
    assert r[4] == -2.5 and np.isinf(r[6])
    bits = r.view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)


def test_backward_matches_finite_differences(monkeypatch):
    monkeypatch.setattr(mlp, "bf16", lambda a: np.asarray(a, dtype=np.float32))
    rng = np.random.default_rng(0)
    flat = mlp.init(1)
    flat += 0.05 * rng.standard_normal(flat.size).astype(np.float32)   # non-zero output layer
    X = rng.standard_normal((12, mlp.N_IN)).astype(np.float32)
    t = rng.standard_normal(12).astype(np.float32)
    loss, g = mlp.loss_and_grad(flat, X, t)
    f64 = flat.astype(np.float64)
    idx = rng.choice(flat.size, 40, replace=False)
    for i in idx:
        e = 1e-2 * max(1.0, abs(f64[i]))
        fp = f64.copy()
        fm = f64.copy()
        fp[i] += e
        fm[i] -= e
        lp = 0.5 * np.mean((mlp.forward(fp.astype(np.float32), X) - t) ** 2)
        lm = 0.5 * np.mean((mlp.forward(fm.astype(np.float32), X) - t) ** 2)
        fd = (lp - lm) / (2 * e)
        assert abs(fd - g[i]) <= 2e-3 * max(1.0, abs(fd)) + 2e-4, (i, fd, g[i])


def test_adam_first_step_closed_form():
    flat = np.zeros(5, np.float32)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0], np.float32)
    m = np.zeros(5, np.float32)
    v = np.zeros(5, np.float32)
    new, m, v = mlp.adam(flat, g, m, v, 1, lr=0.01)
    # the first bias-corrected step is lr * sign(g) (eps aside)
    assert np.allclose(new, -0.01 * np.sign(g), atol=1e-7)


def test_training_reduces_loss_on_a_linear_target():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((256, mlp.N_IN)).astype(np.float32)
    t = (X[:, 0] - X[:, 1]).astype(np.float32)          # extrapolation-like target
    flat = mlp.init(3)
    m = np.zeros_like(flat)
    v = np.zeros_like(flat)
    l0, _ = mlp.loss_and_grad(flat, X, t)
    for s in range(1, 201):
        loss, g = mlp.loss_and_grad(flat, X, t)
        flat, m, v = mlp.adam(flat, g, m, v, s, lr=3e-3)
    assert loss < 0.05 * l0
