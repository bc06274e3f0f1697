"""Structured box mesh hierarchy and DoF numbering (oracle).

Sec. 2: cells are images of (0,1)^d under bi/trilinear maps T_tau; Sec. 3.1: the
hierarchy T_0..T_L comes from L uniform refinements.  Here every level is an
n_x x n_y (x n_z) box of cells, n_l = n_L / 2^(L-l); the vertices of a coarse
level are every 2^(L-l)-th vertex of the finest level.

Global DoF vector layout: [u_1 | ... | u_d | p], each block lexicographic over
its node lattice with x fastest.  Velocity lattice: k*n+1 nodes per direction;
pressure lattice: (k-1)*n+1.  A velocity node on a Dirichlet face is constrained
in all components.  Dirichlet faces are a bit mask: bit 2a is the face x_a = lo,
bit 2a+1 the face x_a = hi.
"""
from __future__ import annotations

import itertools

import numpy as np

ALL_FACES = 0x3F


def dof_counts(dim, k, n):
    """(n_u, n_p): d*(k n+1)^d velocity and ((k-1) n+1)^d pressure DoFs (all boundary DoFs included)."""
    nu = dim * int(np.prod([k * n[a] + 1 for a in range(dim)]))
    npr = int(np.prod([(k - 1) * n[a] + 1 for a in range(dim)]))
    return nu, npr


class Level:
    def __init__(self, dim, k, n, vertices, dirichlet_faces=ALL_FACES):
        self.dim = dim
        self.k = k
        self.n = tuple(int(v) for v in n[:dim])
        self.vertices = np.asarray(vertices, dtype=np.float64)
        assert self.vertices.shape == tuple(c + 1 for c in self.n[::-1]) + (dim,)
        self.faces = dirichlet_faces
        self.N = tuple(k * c + 1 for c in self.n)          # velocity nodes per direction
        self.Pn = tuple((k - 1) * c + 1 for c in self.n)   # pressure nodes per direction
        self.nv = int(np.prod(self.N))                     # per velocity component
        self.n_u = dim * self.nv
        self.n_p = int(np.prod(self.Pn))
        self.size = self.n_u + self.n_p
        self.n_cells = int(np.prod(self.n))

    # --- numbering -------------------------------------------------------------
    def vnode(self, idx):
        """Flat velocity-lattice index of integer node coordinates idx = (i_x, i_y[, i_z])."""
        out = 0
        stride = 1
        for a in range(self.dim):
            out = out + idx[a] * stride
            stride *= self.N[a]
        return out

    def pnode(self, idx):
        out = 0
        stride = 1
        for a in range(self.dim):
            out = out + idx[a] * stride
            stride *= self.Pn[a]
        return out

    def cells(self):
        """Integer coordinates of every cell, shape (n_cells, dim), x fastest."""
        rng = [np.arange(c) for c in self.n[::-1]]
        g = np.meshgrid(*rng, indexing="ij")
        return np.stack([a.reshape(-1) for a in g[::-1]], axis=-1)

    def cell_velocity_nodes(self):
        """(n_cells, (k+1)^d) flat velocity-lattice node indices, local order x fastest."""
        C = self.cells()
        loc = list(itertools.product(range(self.k + 1), repeat=self.dim))
        loc = [t[::-1] for t in loc]  # x fastest
        out = np.empty((len(C), len(loc)), dtype=np.int64)
        for j, t in enumerate(loc):
            out[:, j] = self.vnode([self.k * C[:, a] + t[a] for a in range(self.dim)])
        return out

    def cell_pressure_nodes(self):
        C = self.cells()
        km = self.k - 1
        loc = list(itertools.product(range(km + 1), repeat=self.dim))
        loc = [t[::-1] for t in loc]
        out = np.empty((len(C), len(loc)), dtype=np.int64)
        for j, t in enumerate(loc):
            out[:, j] = self.pnode([km * C[:, a] + t[a] for a in range(self.dim)])
        return out

    def cell_vertices(self):
        """(n_cells, 2^d, dim) vertex coordinates, local vertex order x fastest."""
        C = self.cells()
        out = np.empty((len(C), 2**self.dim, self.dim))
        for j, t in enumerate(itertools.product(range(2), repeat=self.dim)):
            t = t[::-1]
            idx = tuple(C[:, a] + t[a] for a in range(self.dim))[::-1]
            out[:, j, :] = self.vertices[idx]
        return out

    def velocity_constrained(self):
        """Boolean mask over one velocity component's lattice: node lies on a Dirichlet face."""
        grids = np.meshgrid(*[np.arange(c) for c in self.N[::-1]], indexing="ij")[::-1]
        mask = np.zeros(grids[0].shape, dtype=bool)
        for a in range(self.dim):
            if self.faces & (1 << (2 * a)):
                mask |= grids[a] == 0
            if self.faces & (1 << (2 * a + 1)):
                mask |= grids[a] == self.N[a] - 1
        return mask.reshape(-1)

    def constrained(self):
        """Boolean mask over the full vector [u | p]."""
        vm = self.velocity_constrained()
        return np.concatenate([np.tile(vm, self.dim), np.zeros(self.n_p, dtype=bool)])

    def has_pressure_kernel(self):
        """Full Dirichlet data leaves the constant pressure in the kernel of K (Sec. 2, L^2_0)."""
        full = (1 << (2 * self.dim)) - 1
        return (self.faces & full) == full


class Hierarchy:
    """Levels 0..L of a uniformly refined box (Sec. 3.1)."""

    def __init__(self, dim, k, n_fine, n_levels, fine_vertices, dirichlet_faces=ALL_FACES):
        self.dim = dim
        self.k = k
        self.levels = []
        fine_vertices = np.asarray(fine_vertices, dtype=np.float64)
        for l in range(n_levels):
            s = 2 ** (n_levels - 1 - l)
            n = tuple(c // s for c in n_fine[:dim])
            assert all(c * s == f for c, f in zip(n, n_fine[:dim])), "n_fine must be divisible by 2^L"
            sl = tuple(slice(None, None, s) for _ in range(dim))
            self.levels.append(Level(dim, k, n, fine_vertices[sl], dirichlet_faces))

    @property
    def L(self):
        return len(self.levels) - 1
