"""Flexible GMRES(m), right-preconditioned (oracle, FP64).

The outer FP64 loop around the multigrid cycle has no counterpart in the paper
(which iterates the cycle as a stationary method); it is the standard flexible
GMRES of Saad (1993): Arnoldi with modified Gram-Schmidt on the preconditioned
directions z_j = B_j^{-1} v_j, Givens rotations on the Hessenberg matrix, and
x = x_0 + Z_m y_m.  Stops when the relative residual ||b - K x|| / ||b|| <= rtol;
the recurrence estimate is confirmed by an explicit residual at every restart.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_K, precond, b, rtol=1e-10, restart=30, maxit=300, x0=None):
    """Returns (x, iterations, history of relative residual estimates)."""
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while True:
        r = b - apply_K(x)
        beta = float(np.linalg.norm(r))
        hist.append(beta / bnorm)
        if beta <= rtol * bnorm or it >= maxit:
            return x, it, hist
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            Z[j] = precond(V[j])
            w = apply_K(Z[j])
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
