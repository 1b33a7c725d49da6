"""Training data and training loop of the learned density warm start.

Orchestration only: Strang steps, the density-history projection, density
exports, the forward/backward/Adam step and inference all run in libkfbi.so
kernels; this module only arranges the rows (on the device, with torch as the
memory allocator) and the loop.

A training row of solve n is, for every interface node,
  (psi_F / rms(psi_F), r_F / rms(r_F), g^n / rms(g^n), x, n)
  -> (psi^n - psi_F - 2 gamma r_F) / rms(r_F),
with psi_F the projection of the density history and r_F = g^n - A psi_F its
residual, from runs of the method itself (the same features the library's
feature kernel builds at inference).
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


def _rms(v):
    return (v.double().norm() / v.numel() ** 0.5).clamp_min(1e-150)


def features(psiF, rF, g, X, Nn):
    """Input rows of the network (float32), as the library's feature kernel
    builds them."""
    torch = _torch()
    return torch.cat([(psiF / _rms(psiF)).float()[:, None], (rF / _rms(rF)).float()[:, None],
                      (g / _rms(g)).float()[:, None], X, Nn], dim=1).contiguous()


def collect(h: K.KFBI, fhn, V, w, steps, nodes, normals, first=2, gamma=0.8):
    """Advance (V, w) by `steps` Strang steps on handle h (projection warm
    start) and return the rows (F [rows, 9] float32, T [rows] float32 raw
    targets) of the solves >= first."""
    torch = _torch()
    dev = V.device
    M = h.M
    h.set_opts(warm=K.WARM_PROJECTION)
    psi = torch.empty(M, dtype=torch.float64, device=dev)
    g = torch.empty_like(psi)
    psiF = torch.empty_like(psi)
    rF = torch.empty_like(psi)
    X = torch.tensor(np.asarray(nodes), dtype=torch.float32, device=dev)
    Nn = torch.tensor(np.asarray(normals), dtype=torch.float32, device=dev)
    Fs, Ts = [], []
    for n in range(1, steps + 1):
        h.bidomain_step(fhn, V, w, None, nsteps=1)
        if n >= first:
            h.get_densities(psi, None, g)
            h.get_projection(psiF, rF)
            Fs.append(features(psiF, rF, g, X, Nn))
            Ts.append(((psi - psiF - 2.0 * gamma * rF) / _rms(rF)).float())
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
