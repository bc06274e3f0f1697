"""Adjoint gradients of a Stokes solve w.r.t. per-cell viscosity and forcing (oracle, FP64).

No counterpart in the paper (its mu is a constant); this is the plain discrete adjoint of
    K(mu) x = b,  b = Z M_v f,  J(x) = 1/2 ||u - u_obs||^2 (Euclidean over velocity DoFs):
    lambda = K^{-T} dJ/dx = K^{-1} dJ/dx          (K symmetric)
    dJ/dmu_c = -lambda^T (dK/dmu_c) x = -sum_comp lambda_comp,c^T K0_c x_comp,c
    dJ/df    = (Z M_v)^T lambda_u
with K0_c the element stiffness (grad.grad, no mu) of cell c restricted to free DoFs.  Solves
are sparse direct (bordered when the constant pressure is in the kernel).  Pinned against central
finite differences of J by tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import Tables, assemble, element_matrices, load_vector_nodal


def direct_solve(level, K, b):
    if not level.has_pressure_kernel():
        return spla.spsolve(K.tocsc(), b)
    e = np.concatenate([np.zeros(level.n_u), np.ones(level.n_p)])
    Kb = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    return spla.spsolve(Kb, np.concatenate([b, [0.0]]))[:-1]


def forward(level, mu_cell, f, gamma_rho=0.0):
    ops = assemble(level, 1.0, gamma_rho, mu_cell)
    b = load_vector_nodal(level, ops, f)
    return ops, b, direct_solve(level, ops["K"], b)


def objective(level, x, u_obs):
    d = x[: level.n_u] - u_obs[: level.n_u]
    return 0.5 * float(d @ d)


def cell_gradient(level, x, lam):
    """dJ/dmu_c = -sum_comp lam_c^T K0_c x_c on free DoFs, for every cell."""
    tab = Tables(level.dim, level.k)
    E = element_matrices(level, tab, 1.0, 0.0)
    vn = level.cell_velocity_nodes()
    free = ~level.velocity_constrained()
    g = np.zeros(level.n_cells)
    for c in range(level.dim):
        xc = x[c * level.nv:(c + 1) * level.nv] * free
        lc = lam[c * level.nv:(c + 1) * level.nv] * free
        g -= np.einsum("ci,cij,cj->c", lc[vn], E["K0"], xc[vn])
    return g


def gradients(level, mu_cell, f, u_obs, gamma_rho=0.0):
    """Returns (J, x, lam, dJ/dmu per cell, dJ/df nodal)."""
    ops, b, x = forward(level, mu_cell, f, gamma_rho)
    J = objective(level, x, u_obs)
    dJdx = np.zeros(level.size)
    dJdx[: level.n_u] = x[: level.n_u] - u_obs[: level.n_u]
    lam = direct_solve(level, ops["K"], dJdx)
    gmu = cell_gradient(level, x, lam)
    lam_u = lam[: level.n_u].reshape(level.dim, level.nv) * (~level.velocity_constrained())[None, :]
    gf = np.concatenate([ops["Mv_full"] @ lam_u[c] for c in range(level.dim)])
    return J, x, lam, gmu, gf
