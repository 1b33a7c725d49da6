"""Element-wise checks of the GPU network, one layer at a time.

The GPU and the CPU oracle MLP round the same weights and activations to
bfloat16, multiply them exactly and sum in float32; they differ in the order
of the sums (tensor-core fragments, atomics), in the float32 exponential of
SiLU, and -- through those -- in activations that round to the other
bfloat16 neighbour.  A comparison of the whole network would let such flips
compound over four layers of width 128, so each layer's output is checked
against the oracle's arithmetic applied to the GPU's own input to that layer
(kfbi_mlp_layers returns them).  The bounds per element:

* a float32 sum of K terms: EPS_ACC (K + 1) sum |terms|, EPS_ACC = 2^-21 (four
  float32 units per term, room for tensor cores that do not round every
  partial sum to nearest);
* SiLU and its derivative through CUDA's expf against numpy's: 32 float32
  units of s (1 + |z|), s the logistic function;
* a bfloat16 rounding of a SiLU output: if s (1 -+ 32 u) round to different
  bfloat16 values the two sides may differ by that gap, else not at all.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

EPS_ACC = 2.0 ** -21
U32 = 2.0 ** -24


def _act(z):
    """The GPU's bfloat16 activation of pre-activations z, as the oracle
    computes it, and the bound on its difference from the GPU's value."""
    a = mlp.silu(np.asarray(z, dtype=np.float32)).astype(np.float32)
    d = 32.0 * U32 * (np.abs(a.astype(np.float64)) + 1e-30)
    lo = mlp.bf16((a - d).astype(np.float32)).astype(np.float64)
    hi = mlp.bf16((a + d).astype(np.float32)).astype(np.float64)
    return mlp.bf16(a).astype(np.float64), np.abs(hi - lo)


def _dsilu_err(z):
    z = np.asarray(z, dtype=np.float64)
    s = 1.0 / (1.0 + np.exp(-z))
    return 32.0 * U32 * s * (1.0 + np.abs(z))


def _check(name, got, ref, bound, report):
    got = np.asarray(got, dtype=np.float64)
    excess = np.abs(got - ref) - bound
    report[name] = (float(np.abs(got - ref).max()), float(bound.max()), int((excess > 0).sum()))
    assert np.all(excess <= 0.0), (name, report[name])


def check_forward(flat, X, z, o, report):
    """X [B, 9] normalised inputs (float32); z [4, B, 128] and o [B] from the
    GPU.  Checks every hidden layer and the output element-wise."""
    ps = mlp.unpack(flat)
    A, dA = mlp.bf16(X).astype(np.float64), np.zeros(X.shape)
    for l in range(5):
        W = mlp.bf16(ps[2 * l]).astype(np.float64)
        b = ps[2 * l + 1].astype(np.float64)
        ref = A @ W.T + b[None, :]
        bound = EPS_ACC * (A.shape[1] + 1) * (np.abs(A) @ np.abs(W).T + np.abs(b)[None, :]) + dA @ np.abs(W).T
        if l < 4:
            _check(f"z{l}", z[l], ref, bound, report)
            A, dA = _act(z[l])
        else:
            _check("o", o, ref[:, 0], bound[:, 0], report)


def check_backward(flat, X, t, z, o, d, d4, grad, loss, report):
    """t [B] normalised targets; d [4, B, 128] GPU deltas of hidden layers
    3..0, d4 [B]; grad and loss from kfbi_mlp_grad on the same rows."""
    ps = mlp.unpack(flat)
    B = X.shape[0]
    r = o.astype(np.float64) - t.astype(np.float64)
    _check("d4", d4, r / B, 4.0 * U32 * np.abs(r / B) + 1e-45, report)
    lref = 0.5 * float(np.mean(r * r))
    assert abs(loss - lref) <= EPS_ACC * (B + 1) * lref + 1e-30, (loss, lref)
    # inputs of every layer as the GPU sees them (bfloat16), with flip bounds
    ins = [(mlp.bf16(X).astype(np.float64), np.zeros(X.shape))] + [_act(z[l]) for l in range(4)]
    deltas = [d4[:, None].astype(np.float64)] + [d[k].astype(np.float64) for k in range(4)]   # layers 4, 3, 2, 1, 0
    gref = mlp.unpack(grad.astype(np.float32))
    for l in range(4, -1, -1):
        dl = deltas[4 - l]
        D = mlp.bf16(dl.astype(np.float32)).astype(np.float64)
        A, dA = ins[l]
        gW = D.T @ A
        bW = EPS_ACC * (B + 1) * (np.abs(D).T @ np.abs(A)) + np.abs(D).T @ dA
        _check(f"gW{l}", gref[2 * l], gW, bW, report)
        gb = dl.sum(axis=0)
        _check(f"gb{l}", gref[2 * l + 1], gb, EPS_ACC * (B + 1) * np.abs(dl).sum(axis=0) + 1e-45, report)
        if l > 0:
            W = mlp.bf16(ps[2 * l]).astype(np.float64)
            da = D @ W
            zz = z[l - 1].astype(np.float64)
            ds = mlp.dsilu(z[l - 1]).astype(np.float64)
            ref = da * ds
            bound = (EPS_ACC * (W.shape[0] + 1) * (np.abs(D) @ np.abs(W)) * np.abs(ds)
                     + np.abs(da) * _dsilu_err(zz) + 4.0 * U32 * np.abs(ref) + 1e-45)
            _check(f"d{l - 1}", deltas[5 - l], ref, bound, report)
