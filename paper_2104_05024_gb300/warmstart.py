"""Training loop of the learned density warm start.

Orchestration only: the Strang steps, the density-history projection, the
training rows, their normalisation moments, the forward/backward/Adam step
and inference all run in libkfbi.so kernels; this module only allocates the
row buffers (torch as the device allocator), concatenates them, and draws
the order of the minibatches (indexing).

A training row of solve n is, for every interface node,
  (psi_F / rms(psi_F), r_F / rms(r_F), g^n / rms(g^n), x, n)
  -> (psi^n - psi_F - 2 gamma r_F) / rms(r_F),
with psi_F the projection of the density history and r_F = g^n - A psi_F its
residual, from runs of the method itself (kfbi_training_rows builds them
with the same feature code the library's inference uses).
"""
from __future__ import annotations

from kfbi_workloads.configs import mlp_init_params

from . import kfbi as K


def _torch():
    import torch
    return torch


def init_params(seed: int = 0):
    """The seeded initial parameters (untrained: the network adds nothing to
    the projection start)."""
    return mlp_init_params(seed)


def collect(h: K.KFBI, fhn, V, w, steps, first=2):
    """Advance (V, w) by `steps` Strang steps on handle h (projection warm
    start) and return the rows (F [rows, 9], T [rows] raw targets; float32,
    device) of the solves >= first."""
    torch = _torch()
    dev = V.device
    h.set_opts(warm=K.WARM_PROJECTION)
    Fs, Ts = [], []
    for n in range(1, steps + 1):
        h.bidomain_step(fhn, V, w, None, nsteps=1)
        if n >= first:
            F = torch.empty((h.M, 9), dtype=torch.float32, device=dev)
            T = torch.empty(h.M, dtype=torch.float32, device=dev)
            h.training_rows(F, T)
            Fs.append(F)
            Ts.append(T)
    return torch.cat(Fs), torch.cat(Ts)


def fit_norm(F, T):
    """Normalisation vector of the rows (library kernel)."""
    return K.MLP.fit_norm(F.contiguous(), T.contiguous())


def train(mlp: K.MLP, F, T, epochs=4, batch=4096, lr=2e-3, seed=0):
    """Adam on 0.5 mean (o - t)^2, t the targets normalised by the network's
    vector; returns the per-epoch mean losses."""
    torch = _torch()
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    n = F.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen).to(F.device)
        acc, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            acc += mlp.train_step(F[idx].contiguous(), T[idx].contiguous(), lr)
            cnt += 1
        losses.append(acc / max(cnt, 1))
    return losses
