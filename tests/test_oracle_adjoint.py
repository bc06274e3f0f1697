"""Pins of the oracle's adjoint gradients against central finite differences (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle.adjoint import forward, gradients, objective
from oracle.mesh import Level


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 2)])
def test_adjoint_gradients_match_central_differences(dim, n):
    V = W.perturbed_vertices(dim, (n,) * dim, seed=1, amplitude=0.3)
    lev = Level(dim, 2, (n,) * dim, V)
    rng = np.random.default_rng(0)
    mu = np.exp(0.5 * rng.standard_normal(lev.n_cells))
    f = W.fourier_forcing(dim, 2, (n,) * dim, seed=2).reshape(-1) + 0.3  # nonzero on the boundary too
    _, _, u_obs = forward(lev, np.exp(0.5 * rng.standard_normal(lev.n_cells)), f)
    J, x, lam, gmu, gf = gradients(lev, mu, f, u_obs, gamma_rho=3.0)
    eps = 1e-6
    for c in rng.choice(lev.n_cells, min(6, lev.n_cells), replace=False):
        mp, mm = mu.copy(), mu.copy()
        mp[c] *= 1 + eps
        mm[c] *= 1 - eps
        Jp = objective(lev, forward(lev, mp, f, 3.0)[2], u_obs)
        Jm = objective(lev, forward(lev, mm, f, 3.0)[2], u_obs)
        fd = (Jp - Jm) / (2 * eps * mu[c])
        assert abs(fd - gmu[c]) <= 1e-6 * np.abs(gmu).max(), (c, fd, gmu[c])
    for j in rng.choice(lev.n_u, 6, replace=False):
        fp, fm = f.copy(), f.copy()
        fp[j] += eps
        fm[j] -= eps
        Jp = objective(lev, forward(lev, mu, fp, 3.0)[2], u_obs)
        Jm = objective(lev, forward(lev, mu, fm, 3.0)[2], u_obs)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - gf[j]) <= 1e-6 * np.abs(gf).max() + 1e-14, (j, fd, gf[j])
