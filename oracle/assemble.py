"""Element matrices by plain quadrature and assembled CSR operators (oracle, FP64).

Bilinear forms (Sec. 2, Eqs. a(u,v), b(v,q)):
    a(u,v) = int mu grad u : grad v + gamma*rho u.v
  or, in the symmetric-gradient form of Sec. 2 (sym=True),
    a(u,v) = int mu eps(u) : eps(v) + gamma*rho u.v,   eps(u) = (grad u + grad u^T) / 2,
  with mu and rho constant per cell (mu_cell, rho_cell; rho defaults to 1)
    b(v,q) = -int q div v
The sign of b follows the reading that makes K x = b the discretisation of
-mu Lap u + grad p = f (the paper prints both signs; the velocity is unaffected,
only p flips).  The linear system is K = [A B^T; B -C] (Eq. Kx=f).  The paper leaves
the stabilisation C open (non-negative, usually 0, Sec. 1); read here as
    c(p,q) = c_mass int p q + c_grad sum_tau h_tau^2 int_tau grad p . grad q,
h_tau = |tau|^(1/d): a pressure-mass penalty plus a Brezzi-Pitkaranta pressure Laplacian.

Dirichlet treatment: a constrained velocity DoF keeps its slot in the vector;
its row and column of K are replaced by the identity (y_i = x_i).

Geometry: each cell is the image of (0,1)^d under the bi/trilinear map through
its 2^d vertices; gradients transform with J^{-T} and integrals pick up det J.
Quadrature: (k+1)-point Gauss-Legendre per direction for every term.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .fe import Element1D, tensor_tables


class Tables:
    """Reference-cell tables for Q_k / Q_{k-1} / Q_1 (geometry) at the (k+1)^d Gauss points."""

    def __init__(self, dim, k, quad_points=None):
        nq = k + 1 if quad_points is None else quad_points
        self.dim, self.k = dim, k
        self.vel = Element1D(k, nq)
        self.pre = Element1D(k - 1, nq)
        self.geo = Element1D(1, nq)
        self.phi, self.dphi, self.w = tensor_tables(self.vel, dim)
        self.psi, self.dpsi, _ = tensor_tables(self.pre, dim)
        self.gphi, self.gdphi, _ = tensor_tables(self.geo, dim)


def geometry(tab, Xv):
    """Jacobians at quadrature points for cells with vertex coordinates Xv (nc, 2^d, d).

    Returns J (nc, nq, d, d) with J[.., a, b] = d x_a / d xi_b, det J (nc, nq), J^{-T} (nc, nq, d, d).
    """
    J = np.einsum("cva,vqb->cqab", Xv, tab.gdphi)
    detJ = np.linalg.det(J)
    JinvT = np.linalg.inv(J).swapaxes(-1, -2)
    return J, detJ, JinvT


def element_matrices(level, tab, mu, gamma_rho, mu_cell=None, cells=None, rho_cell=None, sym=False):
    """Element matrices of a block of cells.

    Returns dict with
      As  (nc, nphi, nphi)        scalar velocity block: mu_c grad.grad + gamma*rho mass
      B   (nc, npsi, d, nphi)     B_tau[i, c, j] = -int psi_i d(phi_j)/dx_c
      Mv  (nc, nphi, nphi)        scalar velocity mass
      Mp  (nc, npsi, npsi)        pressure mass
      K0  (nc, nphi, nphi)        scalar stiffness grad.grad (no mu)
      Kp  (nc, npsi, npsi)        pressure stiffness grad.grad
      vol (nc,)                   cell volumes
      Af  (nc, d, nphi, d, nphi)  coupled velocity block of the symmetric form (sym=True):
                                  Af[c,i,e,j] = mu_c (1/2 delta_ce int grad phi_i . grad phi_j
                                  + 1/2 int d_e phi_i d_c phi_j) + delta_ce gamma rho_c int phi_i phi_j
    """
    Xv = level.cell_vertices()
    if cells is not None:
        Xv = Xv[cells]
    _, detJ, JinvT = geometry(tab, Xv)
    if np.any(detJ <= 0):
        raise ValueError("inverted or degenerate cell")
    wdet = detJ * tab.w[None, :]                                   # (nc, nq)
    grad = np.einsum("cqab,iqb->ciqa", JinvT, tab.dphi)             # physical gradients (nc, nphi, nq, d)
    K0 = np.einsum("cq,ciqa,cjqa->cij", wdet, grad, grad)
    Mv = np.einsum("cq,iq,jq->cij", wdet, tab.phi, tab.phi)
    Mp = np.einsum("cq,iq,jq->cij", wdet, tab.psi, tab.psi)
    B = -np.einsum("cq,iq,cjqa->ciaj", wdet, tab.psi, grad)
    gradp = np.einsum("cqab,iqb->ciqa", JinvT, tab.dpsi)
    Kp = np.einsum("cq,ciqa,cjqa->cij", wdet, gradp, gradp)
    if mu_cell is None:
        muv = np.full(len(Xv), float(mu))
    else:
        muv = np.asarray(mu_cell, dtype=np.float64)
        if cells is not None:
            muv = muv[cells]
    rhov = np.ones(len(Xv)) if rho_cell is None else np.asarray(rho_cell, dtype=np.float64)
    if rho_cell is not None and cells is not None:
        rhov = rhov[cells]
    grho = gamma_rho * rhov[:, None, None]
    As = muv[:, None, None] * K0 + grho * Mv
    out = {"As": As, "B": B, "Mv": Mv, "Mp": Mp, "K0": K0, "Kp": Kp, "vol": wdet.sum(axis=1)}
    if sym:
        d = level.dim
        X = np.einsum("cq,ciqa,cjqb->cijab", wdet, grad, grad)   # int d_a phi_i d_b phi_j
        eye = np.eye(d)
        Af = 0.5 * np.einsum("ce,kij->kciej", eye, K0) + 0.5 * np.einsum("kijec->kciej", X)
        Af = muv[:, None, None, None, None] * Af + np.einsum("ce,kij->kciej", eye, grho * Mv)
        out["Af"] = Af
    return out


def _scatter(rows_loc, cols_loc, vals, shape):
    nc, a, b = vals.shape
    r = np.broadcast_to(rows_loc[:, :, None], (nc, a, b)).reshape(-1)
    c = np.broadcast_to(cols_loc[:, None, :], (nc, a, b)).reshape(-1)
    return sp.coo_matrix((vals.reshape(-1), (r, c)), shape=shape).tocsr()


def assemble(level, mu=1.0, gamma_rho=0.0, mu_cell=None, chunk=4096, c_mass=0.0, c_grad=0.0, rho_cell=None,
             sym=False):
    """Assembled operators of one level.

    Returns dict of CSR matrices (all FP64):
      As_full  scalar velocity block without constraints (nv x nv)
      Mv_full  scalar velocity mass without constraints
      Mp       pressure mass
      B_full   n_p x n_u divergence block without constraints
      A        n_u x n_u velocity block, Dirichlet rows/columns -> identity
      B        n_p x n_u with constrained columns zeroed
      C        n_p x n_p stabilisation c_mass M_p + c_grad sum h^2 K_p (zero by default)
      K        [A B^T; B -C]
      free     boolean mask of unconstrained entries of the full vector
    """
    tab = Tables(level.dim, level.k)
    vn = level.cell_velocity_nodes()
    pn = level.cell_pressure_nodes()
    nv, d = level.nv, level.dim
    As = sp.csr_matrix((nv, nv))
    Mv = sp.csr_matrix((nv, nv))
    Mp = sp.csr_matrix((level.n_p, level.n_p))
    Bf = sp.csr_matrix((level.n_p, level.n_u))
    Cs = sp.csr_matrix((level.n_p, level.n_p))
    Afull = sp.csr_matrix((level.n_u, level.n_u)) if sym else None
    for s in range(0, level.n_cells, chunk):
        cells = np.arange(s, min(s + chunk, level.n_cells))
        E = element_matrices(level, tab, mu, gamma_rho, mu_cell, cells, rho_cell, sym)
        As = As + _scatter(vn[cells], vn[cells], E["As"], (nv, nv))
        Mv = Mv + _scatter(vn[cells], vn[cells], E["Mv"], (nv, nv))
        Mp = Mp + _scatter(pn[cells], pn[cells], E["Mp"], (level.n_p, level.n_p))
        if c_mass or c_grad:
            h2 = E["vol"] ** (2.0 / d)
            Ce = c_mass * E["Mp"] + c_grad * h2[:, None, None] * E["Kp"]
            Cs = Cs + _scatter(pn[cells], pn[cells], Ce, (level.n_p, level.n_p))
        nc = len(cells)
        cols = (vn[cells][:, None, :] + (np.arange(d) * nv)[None, :, None]).reshape(nc, -1)
        if sym:
            Afull = Afull + _scatter(cols, cols, E["Af"].reshape(nc, cols.shape[1], cols.shape[1]),
                                     (level.n_u, level.n_u))
        Bf = Bf + _scatter(pn[cells], cols, E["B"].reshape(nc, pn.shape[1], -1), (level.n_p, level.n_u))
    return finish(level, As, Mv, Mp, Bf, Cs, c_mass, Afull)


def finish(level, As, Mv, Mp, Bf, C=None, c_mass=0.0, A_full=None):
    d = level.dim
    vmask = level.velocity_constrained()
    umask = np.tile(vmask, d)
    Zu = sp.diags((~umask).astype(np.float64))
    if A_full is None:
        A_full = sp.block_diag([As] * d, format="csr")
    A_full = A_full.tocsr()
    A = (Zu @ A_full @ Zu + sp.diags(umask.astype(np.float64))).tocsr()
    B = (Bf @ Zu).tocsr()
    C = sp.csr_matrix((level.n_p, level.n_p)) if C is None else C.tocsr()
    K = sp.bmat([[A, B.T], [B, -C]], format="csr")
    free = ~level.constrained()
    # constant pressures stay in the kernel of K under full Dirichlet data unless C has a mass part
    pker = level.has_pressure_kernel() and c_mass == 0.0
    return {"As_full": As.tocsr(), "A_full": A_full, "Mv_full": Mv.tocsr(), "Mp": Mp.tocsr(), "B_full": Bf.tocsr(),
            "A": A, "B": B, "C": C, "K": K, "free": free, "umask": umask, "pker": pker}


def load_vector_nodal(level, ops, f_nodal):
    """Right-hand side b = [Z M_v f ; 0] for a velocity field given by its nodal values.

    f_nodal: (d, nv) or flat (n_u,).  Constrained rows of b are zero (homogeneous data).
    """
    f = np.asarray(f_nodal, dtype=np.float64).reshape(level.dim, level.nv)
    bu = np.concatenate([ops["Mv_full"] @ f[c] for c in range(level.dim)])
    bu[ops["umask"]] = 0.0
    return np.concatenate([bu, np.zeros(level.n_p)])


def lift(level, ops, uD):
    """Z K_full u_D: the operator applied to Dirichlet values without the constraint masking,
    with the rows of constrained DoFs zeroed (inhomogeneous data by lifting: solve
    K x0 = b - Z K_full u_D, then x = x0 + u_D)."""
    A_full = ops["A_full"]
    Bf = ops["B_full"]
    K_full = sp.bmat([[A_full, Bf.T], [Bf, None]], format="csr")
    y = K_full @ uD
    y[level.constrained()] = 0.0
    return y
