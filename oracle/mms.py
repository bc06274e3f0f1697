"""Manufactured-solution errors (oracle).  Sec. 2: with elliptic regularity the
Q_k-Q_{k-1} solution satisfies ||u-u_h||_L2 = O(h^{k+1}) and
||u-u_h||_H1 + ||p-p_h||_L2 = O(h^k).  Errors are integrated cell by cell with a
(k+3)-point Gauss rule per direction (not the assembly rule).
"""
from __future__ import annotations

import numpy as np

from .assemble import Tables, geometry
from .fe import Element1D, tensor_tables


def load_vector(level, f_func, quad_extra=2):
    """b = [int f . phi_i ; 0] with f = f_func(x, y) -> (f1, f2) (2D) evaluated at quadrature points."""
    k, d = level.k, level.dim
    nq = k + 1 + quad_extra
    tab = Tables(d, k, quad_points=nq)
    Xv = level.cell_vertices()
    _, detJ, _ = geometry(tab, Xv)
    xq = np.einsum("cva,vq->cqa", Xv, tab.gphi)
    fq = np.stack(f_func(*[xq[..., a] for a in range(d)]), axis=-1)  # (nc, nq, d)
    loc = np.einsum("cq,iq,cqa->cai", detJ * tab.w, tab.phi, fq)
    vn = level.cell_velocity_nodes()
    b = np.zeros(level.size)
    for a in range(d):
        np.add.at(b, a * level.nv + vn, loc[:, a, :])
    b[level.constrained()] = 0.0
    return b


def l2_errors(level, x, u_func, p_func, quad_extra=2):
    """(||u - u_h||_L2, ||p - p_h||_L2) with p_h shifted to the mean of p over the domain."""
    k, d = level.k, level.dim
    nq = k + 1 + quad_extra
    vel = Element1D(k, nq)
    pre = Element1D(k - 1, nq)
    geo = Element1D(1, nq)
    phi, _, w = tensor_tables(vel, d)
    psi, _, _ = tensor_tables(pre, d)
    gphi, gdphi, _ = tensor_tables(geo, d)
    Xv = level.cell_vertices()
    J = np.einsum("cva,vqb->cqab", Xv, gdphi)
    wdet = np.linalg.det(J) * w
    xq = np.einsum("cva,vq->cqa", Xv, gphi)
    vn = level.cell_velocity_nodes()
    pn = level.cell_pressure_nodes()
    uex = np.stack(u_func(*[xq[..., a] for a in range(d)]), axis=-1)
    pex = p_func(*[xq[..., a] for a in range(d)])
    uh = np.stack([np.einsum("ci,iq->cq", x[a * level.nv + vn], phi) for a in range(d)], axis=-1)
    ph = np.einsum("ci,iq->cq", x[level.n_u + pn], psi)
    vol = wdet.sum()
    ph = ph - (wdet * ph).sum() / vol + (wdet * pex).sum() / vol
    eu = np.sqrt(np.sum(wdet[..., None] * (uex - uh) ** 2))
    ep = np.sqrt(np.sum(wdet * (pex - ph) ** 2))
    return float(eu), float(ep)


def mms2d_exact():
    """The smooth solution of the 2D manufactured problem: u = curl(sin^2 sin^2), p = cos cos."""
    pi = np.pi

    def u(x, y):
        return pi * np.sin(pi * x) ** 2 * np.sin(2 * pi * y), -pi * np.sin(2 * pi * x) * np.sin(pi * y) ** 2

    def p(x, y):
        return np.cos(pi * x) * np.cos(pi * y)

    return u, p
