"""Point-wise MLP of the learned density warm start (oracle).

Test infrastructure only.  Per interface node the network maps 9 input
features (normalised by fixed means and standard deviations) through 4
hidden layers of width 128 with SiLU to one output o; oracle.warmstart
builds the features from the history projection and turns o into the
initial density.  Weights are rounded to bfloat16, activations entering each
matrix product are rounded to bfloat16, products accumulate in float32 --
the arithmetic of the GPU kernels.  GMRES still decides the converged
density, so the network only changes the initial guess.

The backward pass is written out layer by layer; Adam follows Kingma & Ba.
"""
from __future__ import annotations

import numpy as np

from kfbi_workloads.configs import mlp_init_params

N_IN = 9
WIDTH = 128
N_HIDDEN = 4


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def shapes():
    """Parameter shapes in packing order: W0, b0, W1, b1, ..., W4, b4
    (W_l is [out, in])."""
    dims = [N_IN] + [WIDTH] * N_HIDDEN + [1]
    out = []
    for l in range(len(dims) - 1):
        out.append((dims[l + 1], dims[l]))
        out.append((dims[l + 1],))
    return out


def n_params() -> int:
    return sum(int(np.prod(s)) for s in shapes())


def unpack(flat: np.ndarray):
    ps, o = [], 0
    for s in shapes():
        k = int(np.prod(s))
        ps.append(np.asarray(flat[o:o + k], dtype=np.float32).reshape(s))
        o += k
    return ps


def pack(ps) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float32).ravel() for p in ps])


def init(seed: int = 0) -> np.ndarray:
    """The seeded initial parameters of the workloads (He-uniform hidden
    layers, zero biases, zero output layer: the untrained network adds
    nothing to the projection)."""
    return mlp_init_params(seed)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def normalise(F: np.ndarray, norm: np.ndarray) -> np.ndarray:
    """norm = [mean_0..8, std_0..8, out_mean, out_std] (float32)."""
    return ((F - norm[:N_IN]) / norm[N_IN:2 * N_IN]).astype(np.float32)


def forward(flat, X, keep=False):
    """X: normalised features [B, 9] (float32).  Returns o [B] (and the
    cached pre-activations / activations when keep=True)."""
    ps = unpack(flat)
    a = X.astype(np.float32)
    zs, acts = [], [a]
    L = len(ps) // 2
    for l in range(L):
        W, b = bf16(ps[2 * l]), ps[2 * l + 1]
        z = (bf16(a) @ W.T).astype(np.float32) + b
        if l < L - 1:
            zs.append(z)
            a = silu(z).astype(np.float32)
            acts.append(a)
        else:
            a = z
    o = a[:, 0]
    return (o, zs, acts) if keep else o


def loss_and_grad(flat, X, t, keep=False):
    """Mean-squared error 0.5 mean (o - t)^2 and its gradient (float32);
    keep=True also returns the forward cache (o, zs, acts) and the deltas
    dL/dz of every layer (output layer first)."""
    ps = unpack(flat)
    o, zs, acts = forward(flat, X, keep=True)
    B = X.shape[0]
    r = (o - t).astype(np.float32)
    loss = 0.5 * float(np.mean(r.astype(np.float64) ** 2))
    L = len(ps) // 2
    grads = [None] * len(ps)
    delta = (r / B)[:, None].astype(np.float32)              # dL/dz of the output layer
    deltas = [delta]
    for l in range(L - 1, -1, -1):
        a_in = bf16(acts[l])
        # weight gradients from bfloat16 operands with float32 accumulation
        grads[2 * l] = (bf16(delta).T @ a_in).astype(np.float32)
        grads[2 * l + 1] = delta.sum(axis=0).astype(np.float32)
        if l > 0:
            W = bf16(ps[2 * l])
            da = (bf16(delta) @ W).astype(np.float32)
            delta = (da * dsilu(zs[l - 1])).astype(np.float32)
            deltas.append(delta)
    if keep:
        return loss, pack(grads), (o, zs, acts), deltas
    return loss, pack(grads)


def adam(flat, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns (flat, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return (flat - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32), m.astype(np.float32), v.astype(np.float32)
