"""Grid transfers (oracle).  Sec. 3.2: prolongation is the canonical injection
V_{l-1} x Q_{l-1} -> V_l x Q_l, written as a matrix by evaluating every coarse basis
function at every fine node; restriction is its transpose.

On the structured hierarchy the injection factors into 1D matrices per axis: a
fine node i lies in fine cell f = i // k at local node a; that cell is child
h = f mod 2 of coarse cell c = f // 2, so its reference coordinate inside the
coarse cell is (h + t_a)/2 with t_a the fine Gauss-Lobatto node.  Constrained
(Dirichlet) velocity DoFs are removed on both sides: P_eff = Z_fine P Z_coarse.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fe import gauss_lobatto, lagrange_values


def prolongation_1d(degree, n_coarse):
    """(degree*2*n_coarse+1) x (degree*n_coarse+1) dense 1D injection matrix."""
    t = gauss_lobatto(degree)
    nf = degree * 2 * n_coarse + 1
    nc = degree * n_coarse + 1
    P = np.zeros((nf, nc))
    for i in range(nf):
        f = min(i // degree, 2 * n_coarse - 1)
        a = i - degree * f
        c, h = divmod(f, 2)
        xi = 0.5 * (h + t[a])
        P[i, degree * c:degree * c + degree + 1] = lagrange_values(t, [xi])[:, 0]
    return P


def _kron_all(mats):
    """kron over axes with x fastest: mats = [P_x, P_y(, P_z)]."""
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(sp.csr_matrix(m), out, format="csr")
    return out


def prolongation(coarse, fine):
    """Full prolongation [u|p] coarse -> fine with Dirichlet DoFs removed on both sides."""
    d, k = fine.dim, fine.k
    Pv = _kron_all([prolongation_1d(k, coarse.n[a]) for a in range(d)])
    Pp = _kron_all([prolongation_1d(k - 1, coarse.n[a]) for a in range(d)])
    Pu = sp.block_diag([Pv] * d, format="csr")
    Zf = sp.diags((~np.tile(fine.velocity_constrained(), d)).astype(np.float64))
    Zc = sp.diags((~np.tile(coarse.velocity_constrained(), d)).astype(np.float64))
    Pu = (Zf @ Pu @ Zc).tocsr()
    return sp.block_diag([Pu, Pp], format="csr")
