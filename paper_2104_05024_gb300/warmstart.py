"""Training data and training loop of the learned density warm start.

Orchestration only: Strang steps, density exports, the forward/backward/Adam
step and inference all run in libkfbi.so kernels; this module only arranges
the rows (on the device, with torch as the memory allocator) and the loop.

A training row of step n is (psi^{n-1}, psi^{n-2}, g^n, x, n) -> psi^n - psi^{n-1}
for every interface node, from runs of the method itself.
"""
from __future__ import annotations

import numpy as np

from . import kfbi as K


def _torch():
    import torch
    return torch


N_IN, WIDTH, N_HIDDEN = 9, 128, 4


def init_params(seed: int = 0) -> np.ndarray:
    """Packed float32 parameters: uniform He initialisation of the hidden
    layers (bound sqrt(6 / fan_in)), zero biases and a zero output layer, so
    the untrained network returns the previous density."""
    rng = np.random.default_rng(seed)
    dims = [N_IN] + [WIDTH] * N_HIDDEN + [1]
    out = []
    for l in range(len(dims) - 1):
        fan_in, fan_out = dims[l], dims[l + 1]
        if fan_out > 1:
            out.append(rng.uniform(-np.sqrt(6.0 / fan_in), np.sqrt(6.0 / fan_in), fan_out * fan_in))
        else:
            out.append(np.zeros(fan_out * fan_in))
        out.append(np.zeros(fan_out))
    return np.concatenate(out).astype(np.float32)


def collect(h: K.KFBI, fhn, V, w, steps, nodes, normals, first=3):
    """Advance (V, w) by `steps` Strang steps on handle h and return the rows
    (F [rows, 9] float32, T [rows] float32 raw targets) of steps >= first."""
    torch = _torch()
    dev = V.device
    M = h.M
    psi = torch.empty(M, dtype=torch.float64, device=dev)
    psi1 = torch.empty_like(psi)
    g = torch.empty_like(psi)
    X = torch.tensor(np.asarray(nodes), dtype=torch.float32, device=dev)
    Nn = torch.tensor(np.asarray(normals), dtype=torch.float32, device=dev)
    prev1 = None
    Fs, Ts = [], []
    for n in range(1, steps + 1):
        h.bidomain_step(fhn, V, w, None, nsteps=1)
        h.get_densities(psi, psi1, g)
        if n >= first and prev1 is not None:
            F = torch.cat([psi1.float()[:, None], prev1.float()[:, None], g.float()[:, None], X, Nn], dim=1)
            Fs.append(F)
            Ts.append((psi - psi1).float())
        prev1 = psi1.clone()
    return torch.cat(Fs), torch.cat(Ts)


def fit_norm(F, T):
    """Per-feature means and standard deviations, then the target's."""
    torch = _torch()
    mean = F.double().mean(0)
    std = F.double().std(0)
    std = torch.where(std > 1e-12, std, torch.ones_like(std))
    tm = T.double().mean()
    ts = T.double().std()
    ts = ts if ts > 1e-30 else torch.tensor(1.0, dtype=torch.float64)
    return np.concatenate([mean.cpu().numpy(), std.cpu().numpy(), [tm.item(), ts.item()]]).astype(np.float32)


def train(mlp: K.MLP, F, T, norm, epochs=4, batch=4096, lr=2e-3, seed=0):
    """Adam on 0.5 mean (o - t)^2 with t the normalised target; returns the
    per-epoch mean losses."""
    torch = _torch()
    t = ((T.double() - float(norm[18])) / float(norm[19])).float()
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    n = F.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen).to(F.device)
        acc, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            acc += mlp.train_step(F[idx].contiguous(), t[idx].contiguous(), lr)
            cnt += 1
        losses.append(acc / max(cnt, 1))
    return losses
