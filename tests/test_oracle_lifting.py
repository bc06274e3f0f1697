"""Pins of inhomogeneous Dirichlet data by lifting against exact polynomial Stokes flows (CPU)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle.assemble import assemble, lift
from oracle.mesh import Level


def _node_coords(level, lo, hi):
    ax = [np.linspace(lo[a], hi[a], level.N[a]) for a in range(level.dim)]
    g = np.meshgrid(*ax[::-1], indexing="ij")[::-1]
    return [c.reshape(-1) for c in g]


def _pressure_coords(level, lo, hi):
    ax = [np.linspace(lo[a], hi[a], level.Pn[a]) for a in range(level.dim)]
    g = np.meshgrid(*ax[::-1], indexing="ij")[::-1]
    return [c.reshape(-1) for c in g]


@pytest.mark.parametrize("dim,faces", [(2, 0xF), (3, 0x3F), (3, 0x3F & ~0x2)])
def test_poiseuille_flow_is_reproduced_exactly(dim, faces):
    # u = (y (1 - y), 0[, 0]), p = 2 mu (L - x): -mu Lap u + grad p = 0, div u = 0; Q2 velocity and
    # Q1 pressure represent it exactly.  With the outflow face x = L left natural (do-nothing),
    # mu du/dn - p n = 0 holds there since p(L) = 0.
    mu, L = 1.0, 2.0
    n = (4, 2, 2)[:dim]
    lo, hi = (0.0, 0.0, 0.0), (L, 1.0, 1.0)
    lev = Level(dim, 2, n, W.lattice_vertices(dim, n, lo, hi), faces)
    ops = assemble(lev, mu, 0.0)
    X = _node_coords(lev, lo, hi)
    uex = np.zeros((dim, lev.nv))
    uex[0] = X[1] * (1 - X[1])
    P = _pressure_coords(lev, lo, hi)
    pex = 2 * mu * (L - P[0])
    uD = np.concatenate([(uex * lev.velocity_constrained()[None, :]).reshape(-1), np.zeros(lev.n_p)])
    b = -lift(lev, ops, uD)
    K = ops["K"]
    if lev.has_pressure_kernel():
        e = np.concatenate([np.zeros(lev.n_u), np.ones(lev.n_p)])
        Kb = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
        x0 = spla.spsolve(Kb, np.concatenate([b, [0.0]]))[:-1]
    else:
        x0 = spla.spsolve(K.tocsc(), b)
    x = x0 + uD
    np.testing.assert_allclose(x[: lev.n_u], uex.reshape(-1), atol=1e-12)
    p = x[lev.n_u:]
    if lev.has_pressure_kernel():
        p = p - p.mean() + pex.mean()
    np.testing.assert_allclose(p, pex, atol=1e-11)
