"""Shared problem definitions for the GPU-vs-oracle parity tests (seeded, synthetic).

Each case fixes the mesh (structured box, optionally perturbed by the smooth seeded
field of workloads.perturbed_vertices), the degree k, the number of multigrid levels,
the Dirichlet faces and the coefficients.  The oracle side and the CUDA side are built
from the same vertex array; nothing flows from the CUDA side into the oracle.
"""
from __future__ import annotations

import numpy as np

import workloads as W

CASES = {
    # 2D Q2-Q1 on 16x16, 4 levels: the size of the paper's 2D studies (2467 DoFs)
    "2d_q2_cart": dict(dim=2, k=2, n=(16, 16), levels=4),
    "2d_q2_ragged": dict(dim=2, k=2, n=(6, 10), levels=2, perturb=True, gamma_rho=10.0),
    "2d_q3_pert": dict(dim=2, k=3, n=(8, 8), levels=3, perturb=True),
    "2d_q4_pert": dict(dim=2, k=4, n=(4, 4), levels=2, perturb=True, mu=0.5),
    "3d_q2_pert": dict(dim=3, k=2, n=(8, 8, 8), levels=3, perturb=True, gamma_rho=100.0),
    "3d_q2_single": dict(dim=3, k=2, n=(3, 5, 7), levels=1, perturb=True),
    "3d_q3_cart": dict(dim=3, k=3, n=(4, 4, 4), levels=2),
    # (a single-cell coarse mesh would violate inf-sup for Q4-Q3: use 2^3 coarse cells)
    "3d_q4_pert": dict(dim=3, k=4, n=(4, 4, 4), levels=2, perturb=True),
    # channel [0,4]x[0,1]^2, do-nothing outflow at x = 4 (no pressure kernel)
    "3d_q2_channel": dict(dim=3, k=2, n=(8, 4, 4), levels=2, hi=(4.0, 1.0, 1.0), faces=0x3F & ~0x2, mu=1e-3),
}


def vertices(case, seed=0):
    dim, n = case["dim"], case["n"]
    hi = case.get("hi", (1.0, 1.0, 1.0))
    if case.get("perturb"):
        return W.perturbed_vertices(dim, n, seed=seed, hi=hi)
    return W.lattice_vertices(dim, n, hi=hi)


def faces(case):
    return case.get("faces", 0x3F if case["dim"] == 3 else 0xF)


def oracle_hierarchy(case, seed=0):
    from oracle.mesh import Hierarchy
    return Hierarchy(case["dim"], case["k"], case["n"], case["levels"], vertices(case, seed), faces(case))


def gpu_solver(case, seed=0, **kw):
    from paper_2205_15770_gb300 import StokesMG
    V = vertices(case, seed) if case.get("perturb") else None
    return StokesMG(dim=case["dim"], n=case["n"], n_levels=case["levels"], k=case["k"], mu=case.get("mu", 1.0),
                    gamma_rho=case.get("gamma_rho", 0.0), vertices=V, hi=case.get("hi", (1.0, 1.0, 1.0)),
                    dirichlet_faces=faces(case), **kw)


def random_full(level, seed, constrained_zero=False):
    x = W.random_vector(level.size, seed)
    if constrained_zero:
        x[level.constrained()] = 0.0
    return x


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
