"""Selected rows of K x without assembling the global matrix (oracle, FP64).

For meshes too large to assemble on the CPU in seconds, (K x)_i is computed for a
sample of rows i from the definition K x = sum_tau P_tau K_tau P_tau^T x (Sec. 3.1):
only the cells whose closure contains DoF i contribute, each through its element
matrix built by plain quadrature (assemble.element_matrices).  Dirichlet rows are
identity rows and constrained columns are dropped, exactly as in assemble.finish.
"""
from __future__ import annotations

import itertools

import numpy as np

from .assemble import Tables, element_matrices


def _cells_around(level, coords, deg):
    """Cells (flat indices) whose closure contains the lattice node `coords` of a degree-`deg` lattice."""
    ranges = []
    for a in range(level.dim):
        g = coords[a]
        cands = [c for c in (g // deg - 1, g // deg) if 0 <= c < level.n[a] and deg * c <= g <= deg * c + deg]
        ranges.append(cands)
    out = []
    for t in itertools.product(*ranges):
        idx = 0
        stride = 1
        for a in range(level.dim):
            idx += t[a] * stride
            stride *= level.n[a]
        out.append(idx)
    return out


def apply_rows(level, x, rows, mu=1.0, gamma_rho=0.0, mu_cell=None):
    """(K x)[rows] for the full vector x = [u | p]."""
    tab = Tables(level.dim, level.k)
    d, k = level.dim, level.k
    vmask = level.velocity_constrained()
    vn_all = level.cell_velocity_nodes()
    pn_all = level.cell_pressure_nodes()
    xu = np.asarray(x[: level.n_u]).reshape(d, level.nv).copy()
    xu[:, vmask] = 0.0
    xp = np.asarray(x[level.n_u:])
    out = np.empty(len(rows))
    for r, i in enumerate(rows):
        i = int(i)
        if i < level.n_u:
            comp, node = divmod(i, level.nv)
            if vmask[node]:
                out[r] = x[i]
                continue
            coords = np.unravel_index(node, level.N[::-1])[::-1]
            cells = _cells_around(level, coords, k)
            E = element_matrices(level, tab, mu, gamma_rho, mu_cell, np.array(cells))
            s = 0.0
            for j, c in enumerate(cells):
                loc = int(np.nonzero(vn_all[c] == node)[0][0])
                s += E["As"][j, loc, :] @ xu[comp, vn_all[c]]
                s += E["B"][j, :, comp, loc] @ xp[pn_all[c]]   # (B^T p)_i
            out[r] = s
        else:
            node = i - level.n_u
            coords = np.unravel_index(node, level.Pn[::-1])[::-1]
            cells = _cells_around(level, coords, k - 1)
            E = element_matrices(level, tab, mu, gamma_rho, mu_cell, np.array(cells))
            s = 0.0
            for j, c in enumerate(cells):
                loc = int(np.nonzero(pn_all[c] == node)[0][0])
                for a in range(d):
                    s += E["B"][j, loc, a, :] @ xu[a, vn_all[c]]
            out[r] = s
    return out
