"""1D finite-element ingredients on the reference interval [0, 1] (oracle, FP64).

Sec. 2 (Fig. 1): Q_k / Q_{k-1} shape functions are tensor products of 1D
Lagrange polynomials on the reference cell (0,1)^d.  The paper leaves the node
placement to its library; this oracle (and the CUDA path) uses Gauss-Lobatto
nodes, which for k = 2 are the equispaced points {0, 1/2, 1}.  Every integral
uses the (k+1)-point Gauss-Legendre rule per direction.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(npts):
    """npts-point Gauss-Legendre rule on [0, 1]: (points, weights)."""
    x, w = npleg.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(degree):
    """degree+1 Gauss-Lobatto nodes on [0, 1]: endpoints plus the roots of P'_degree."""
    if degree < 1:
        return np.array([0.5])
    if degree == 1:
        return np.array([0.0, 1.0])
    coeffs = np.zeros(degree + 1)
    coeffs[-1] = 1.0
    inner = np.sort(np.real(npleg.legroots(npleg.legder(coeffs))))
    return np.concatenate([[0.0], 0.5 * (inner + 1.0), [1.0]])


def lagrange_values(nodes, x):
    """L[i, q] = l_i(x_q), the Lagrange polynomial through `nodes` that is 1 at node i."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((n, len(x)))
    for i in range(n):
        for j in range(n):
            if j != i:
                L[i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return L


def lagrange_derivatives(nodes, x):
    """D[i, q] = l_i'(x_q), by the product rule over the factors of l_i."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((n, len(x)))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term = term * (x - nodes[j]) / (nodes[i] - nodes[j])
            D[i] += term
    return D


class Element1D:
    """Tables of one 1D Lagrange space of a given degree at the Gauss points of a rule."""

    def __init__(self, degree, quad_points):
        self.degree = degree
        self.nodes = gauss_lobatto(degree)
        self.qx, self.qw = gauss_legendre(quad_points)
        self.val = lagrange_values(self.nodes, self.qx)      # (n_nodes, n_q)
        self.der = lagrange_derivatives(self.nodes, self.qx)  # (n_nodes, n_q)


def tensor_tables(el1d, dim):
    """Tensor-product basis tables on (0,1)^dim.

    Returns (phi, dphi, w):
      phi[i, q]      basis value, i and q lexicographic with x fastest
      dphi[i, q, a]  reference derivative d/dxi_a
      w[q]           tensor Gauss weight
    """
    n = len(el1d.nodes)
    nq = len(el1d.qx)
    V, Dv, W = el1d.val, el1d.der, el1d.qw
    if dim == 2:
        # index i = iy*n + ix, q = qy*nq + qx
        phi = np.einsum("xa,yb->yxba", V, V).reshape(n * n, nq * nq)
        dx = np.einsum("xa,yb->yxba", Dv, V).reshape(n * n, nq * nq)
        dy = np.einsum("xa,yb->yxba", V, Dv).reshape(n * n, nq * nq)
        dphi = np.stack([dx, dy], axis=-1)
        w = np.einsum("a,b->ba", W, W).reshape(-1)
    else:
        phi = np.einsum("xa,yb,zc->zyxcba", V, V, V).reshape(n**3, nq**3)
        dx = np.einsum("xa,yb,zc->zyxcba", Dv, V, V).reshape(n**3, nq**3)
        dy = np.einsum("xa,yb,zc->zyxcba", V, Dv, V).reshape(n**3, nq**3)
        dz = np.einsum("xa,yb,zc->zyxcba", V, V, Dv).reshape(n**3, nq**3)
        dphi = np.stack([dx, dy, dz], axis=-1)
        w = np.einsum("a,b,c->cba", W, W, W).reshape(-1)
    return phi, dphi, w
