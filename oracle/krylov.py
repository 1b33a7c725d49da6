"""Iterative solvers for the boundary integral equation A psi = g (oracle).

* ``richardson``: the simple iteration psi <- psi + 2 gamma (g - A psi)
  (Eq. simple iteration, gamma = 0.8 in Section 7).
* ``gmres``: restarted GMRES (the Krylov improvement named after Eq. bie),
  modified Gram-Schmidt Arnoldi, Givens rotations.  Convergence is measured
  as ||g - A psi||_2 / ||g||_2 (unweighted over nodes, relative to g so that
  warm starts count).
"""
from __future__ import annotations

import numpy as np


def richardson(apply, b, x0, tol, gamma=0.8, max_iter=500):
    bn = np.linalg.norm(b)
    x = x0.copy()
    hist = []
    it = 0
    while True:
        r = b - apply(x)
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel <= tol or it >= max_iter:
            break
        x = x + 2.0 * gamma * r
        it += 1
    return x, {"iters": it, "rel_res": float(rel), "history": hist, "converged": bool(rel <= tol)}


def gmres(apply, b, x0, tol, restart=50, max_iter=500):
    """Restarted GMRES(m).  With tol = 0 it runs exactly max_iter Arnoldi
    steps (used to compare implementations at fixed iteration counts)."""
    bn = np.linalg.norm(b)
    x = np.array(x0, dtype=np.float64, copy=True)
    n = b.size
    it = 0
    hist = []
    rel = np.inf
    if bn == 0.0:
        return np.zeros_like(b), {"iters": 0, "rel_res": 0.0, "history": [0.0], "converged": True}
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        rel = beta / bn
        if not hist:
            hist.append(rel)
        if rel <= tol or it >= max_iter or beta == 0.0:
            break
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gv = np.zeros(m + 1)
        gv[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = apply(V[j])
            it += 1
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gv[j + 1] = -sn[j] * gv[j]
            gv[j] = cs[j] * gv[j]
            rel = abs(gv[j + 1]) / bn
            hist.append(rel)
            j_done = j + 1
            if rel <= tol or it >= max_iter:
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (gv[i] - np.dot(H[i, i + 1:j_done], y[i + 1:])) / H[i, i]
        x = x + V[:j_done].T @ y
        if rel <= tol or it >= max_iter:
            break
    return x, {"iters": it, "rel_res": float(rel), "history": hist, "converged": bool(rel <= tol)}
