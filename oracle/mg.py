"""Monolithic geometric multigrid, Algorithm 1 (oracle, FP64).

MG(x_l, b_l): on l = 0 solve directly and return (the printed algorithm has no
explicit return there; returning is the reading taken); otherwise m pre-smoothing
steps, residual, restriction by P^T, gamma recursive calls on the coarse
correction from zero (gamma = 1: V-cycle, 2: W-cycle), prolongation, correction,
m post-smoothing steps.

Coarse solve (Sec. 4.1: assembled coarse matrix, direct method).  With Dirichlet
data on the whole boundary the constant pressure spans the kernel of K_0; the
solve then uses the bordered matrix [K_0 e; e^T 0] with e = (0, 1_p), which picks
the solution with sum(p) = 0 and absorbs any inconsistent part of b into the
multiplier.  Dense LU by scipy.

Stationary driver (Sec. 4.1): x^0 = 0, at most 15 iterations, stop at a residual
reduction of 1e-10, rate q = (r^j / r^{j-3})^{1/3}, T(eps) = T_iter log(eps)/log(q).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .assemble import assemble
from .smoother import LevelSmoother
from .transfer import prolongation


class CoarseSolver:
    def __init__(self, level, K, pker=None):
        Kd = K.toarray()
        self.bordered = level.has_pressure_kernel() if pker is None else pker
        self.n = Kd.shape[0]
        if self.bordered:
            e = np.concatenate([np.zeros(level.n_u), np.ones(level.n_p)])
            Kd = np.block([[Kd, e[:, None]], [e[None, :], np.zeros((1, 1))]])
        self.lu = sla.lu_factor(Kd)

    def solve(self, b):
        if self.bordered:
            return sla.lu_solve(self.lu, np.concatenate([b, [0.0]]))[: self.n]
        return sla.lu_solve(self.lu, b)


class Multigrid:
    def __init__(self, hier, mu=1.0, gamma_rho=0.0, kA=3, kS=3, m=2, cycle="V", schur_diag="loc",
                 mu_cells=None, eig_steps=40, eig_safety=1.1, seed=0x5EED, c_mass=0.0, c_grad=0.0, rho_cells=None,
                 sym=False):
        """mu_cells / rho_cells: optional lists (one array per level, coarse to fine) of per-cell
        viscosities / densities; sym: the symmetric-gradient form of a(u,v)."""
        self.hier = hier
        self.m = m
        self.gamma = {"V": 1, "W": 2}[cycle]
        self.ops, self.smoothers, self.P = [], [], []
        for l, lev in enumerate(hier.levels):
            mc = None if mu_cells is None else mu_cells[l]
            rc = None if rho_cells is None else rho_cells[l]
            ops = assemble(lev, mu, gamma_rho, mc, c_mass=c_mass, c_grad=c_grad, rho_cell=rc, sym=sym)
            self.ops.append(ops)
            if l == 0:
                self.coarse = CoarseSolver(lev, ops["K"], ops["pker"])
                self.smoothers.append(None)
                self.P.append(None)
            else:
                self.smoothers.append(LevelSmoother(lev, ops, kA, kS, schur_diag, mu, gamma_rho, mc,
                                                    eig_steps, eig_safety, seed, rho_cell=rc, sym=sym))
                self.P.append(prolongation(hier.levels[l - 1], lev))

    @property
    def K(self):
        return self.ops[-1]["K"]

    def cycle(self, l, x, b):
        if l == 0:
            return self.coarse.solve(b)
        S = self.smoothers[l]
        x = S.smooth(x, b, self.m)
        r = b - self.ops[l]["K"] @ x
        rc = self.P[l].T @ r
        w = np.zeros_like(rc)
        for _ in range(self.gamma):
            w = self.cycle(l - 1, w, rc)
        x = x + self.P[l] @ w
        return S.smooth(x, b, self.m)

    def precondition(self, b):
        """One cycle on the finest level from a zero start: the preconditioner B^{-1} b."""
        return self.cycle(len(self.hier.levels) - 1, np.zeros_like(b), b)

    def stationary(self, b, max_iter=15, reduction=1e-10):
        """Stationary MG iteration from x^0 = 0; returns (x, residual history, q)."""
        L = len(self.hier.levels) - 1
        x = np.zeros_like(b)
        res = [float(np.linalg.norm(b))]
        for _ in range(max_iter):
            x = self.cycle(L, x, b)
            res.append(float(np.linalg.norm(b - self.K @ x)))
            if res[-1] <= reduction * res[0]:
                break
        j = len(res) - 1
        q = (res[j] / res[j - 3]) ** (1.0 / 3.0) if j >= 3 else float("nan")
        return x, res, q


def time_to_reduce(T_iter, q, eps=0.1):
    """T(eps) = T_iter log(eps) / log(q)  (Sec. 4.1)."""
    return T_iter * np.log(eps) / np.log(q)
