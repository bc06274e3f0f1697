"""Adjoint layer on the GPU: per-cell viscosity gradient kernel, mass maps, set_viscosity, and the
differentiable solve (torch.autograd), against the CPU oracle and central finite differences."""
import numpy as np
import pytest

import workloads as W
from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("name", ["2d_q3_pert", "3d_q2_pert", "3d_q3_cart"])
def test_cell_grad_kernel_matches_oracle(name):
    from oracle.adjoint import cell_gradient
    case = CASES[name]
    lev = oracle_hierarchy(case).levels[-1]
    S = gpu_solver(case)
    x = random_full(lev, 1)
    lam = random_full(lev, 2)
    g = _n(S.cell_grad(_t(x), _t(lam)))
    assert rel_err(g, cell_gradient(lev, x, lam)) < 1e-12


@pytest.mark.parametrize("name", ["2d_q2_ragged", "3d_q2_pert", "3d_q2_channel"])
def test_mass_maps_with_boundary_data(name):
    from oracle.assemble import assemble, load_vector_nodal
    case = CASES[name]
    lev = oracle_hierarchy(case).levels[-1]
    ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))
    S = gpu_solver(case)
    f = W.random_vector(lev.n_u, 3)  # nonzero on Dirichlet nodes as well
    assert rel_err(_n(S.mass_rhs(_t(f))), load_vector_nodal(lev, ops, f)) < 1e-12
    free = np.tile(~lev.velocity_constrained(), lev.dim)
    ref = np.concatenate([ops["Mv_full"] @ (f * free)[c * lev.nv:(c + 1) * lev.nv] for c in range(lev.dim)])
    assert rel_err(_n(S.mass(_t(f), full_rows=True)), ref) < 1e-12


def _adjoint_problem(n=4, levels=2, seed=0):
    V = W.perturbed_vertices(3, (n,) * 3, seed=seed)
    g = W.gaussian_field_cells(n, seed=seed)
    mu = np.exp(g).reshape(-1)
    mu_obs = np.exp(W.gaussian_field_cells(n, seed=seed + 1)).reshape(-1)
    f = W.fourier_forcing(3, 2, (n,) * 3, seed=seed).reshape(-1)
    return V, mu, mu_obs, f


def test_set_viscosity_rebuilds_the_operator():
    from oracle.assemble import assemble
    from oracle.mesh import Hierarchy
    from paper_2205_15770_gb300 import StokesMG
    V, mu, _, _ = _adjoint_problem()
    S = StokesMG(dim=3, n=(4, 4, 4), n_levels=2, k=2, vertices=V)
    S.set_viscosity(mu)
    lev = Hierarchy(3, 2, (4, 4, 4), 2, V).levels[-1]
    x = random_full(lev, 5)
    assert rel_err(_n(S.vmult(_t(x))), assemble(lev, 1.0, 0.0, mu)["K"] @ x) < 1e-12
    # coarse level viscosity = mean of the 8 children
    lev0 = Hierarchy(3, 2, (4, 4, 4), 2, V).levels[0]
    mu0 = mu.reshape(4, 4, 4).reshape(2, 2, 2, 2, 2, 2).mean(axis=(1, 3, 5)).reshape(-1)
    x0 = random_full(lev0, 6)
    assert rel_err(_n(S.vmult(_t(x0), level=0)), assemble(lev0, 1.0, 0.0, mu0)["K"] @ x0) < 1e-12


def test_autograd_matches_oracle_adjoint_and_finite_differences():
    from oracle.adjoint import gradients
    from oracle.mesh import Hierarchy
    from paper_2205_15770_gb300 import StokesMG, stokes_solve_fn
    V, mu, mu_obs, f = _adjoint_problem()
    lev = Hierarchy(3, 2, (4, 4, 4), 2, V).levels[-1]
    S = StokesMG(dim=3, n=(4, 4, 4), n_levels=2, k=2, vertices=V, vcycle_fp32=False)
    u_obs = stokes_solve_fn(S, _t(mu_obs), _t(f), 1e-13).detach()
    mu_t = _t(mu).requires_grad_(True)
    f_t = _t(f).requires_grad_(True)
    x = stokes_solve_fn(S, mu_t, f_t, 1e-13)
    nu = lev.n_u
    J = 0.5 * ((x[:nu] - u_obs[:nu]) ** 2).sum()
    J.backward()
    gmu, gf = _n(mu_t.grad), _n(f_t.grad)
    Jo, _, _, gmu_o, gf_o = gradients(lev, mu, f, _n(u_obs))
    assert abs(J.item() - Jo) < 1e-9 * Jo
    assert rel_err(gmu, gmu_o) < 1e-7
    assert rel_err(gf, gf_o) < 1e-7

    def Jof(m):
        with torch.no_grad():
            xx = stokes_solve_fn(S, _t(m), _t(f), 1e-13)
            return 0.5 * float(((xx[:nu] - u_obs[:nu]) ** 2).sum())

    eps = 1e-6
    rng = np.random.default_rng(7)
    for c in rng.choice(lev.n_cells, 8, replace=False):
        mp, mm = mu.copy(), mu.copy()
        mp[c] *= 1 + eps
        mm[c] *= 1 - eps
        fd = (Jof(mp) - Jof(mm)) / (2 * eps * mu[c])
        assert abs(fd - gmu[c]) <= 1e-5 * np.abs(gmu).max(), (c, fd, gmu[c])


def test_adjoint_fd_full_size_32cubed():
    # 3D Q2-Q1 on 32^3 Cartesian hexes, mu_c = exp(g_c) with g a seeded Gaussian field
    # (correlation length 0.2, std 1), J = 0.5 ||u - u_obs||^2 with u_obs from seed + 1; FP64
    # multigrid, solves to 1e-13; central differences (eps = 1e-6) on 20 seeded cells.  The FD error
    # is dominated by the solve tolerance: 1e-13 ||b|| in each of the two J values, divided by
    # 2 eps mu_c, stays below 1e-6 of max |dJ/dmu|.
    from paper_2205_15770_gb300 import StokesMG, stokes_solve_fn
    n = 32
    mu = np.exp(W.gaussian_field_cells(n, seed=0)).reshape(-1)
    mu_obs = np.exp(W.gaussian_field_cells(n, seed=1)).reshape(-1)
    f = _t(W.fourier_forcing(3, 2, (n,) * 3, seed=0).reshape(-1))
    S = StokesMG(dim=3, n=(n,) * 3, n_levels=5, k=2, vcycle_fp32=False)
    u_obs = stokes_solve_fn(S, _t(mu_obs), f, 1e-13).detach()
    mu_t = _t(mu).requires_grad_(True)
    x = stokes_solve_fn(S, mu_t, f, 1e-13)
    nu = S.sizes()[0]
    (0.5 * ((x[:nu] - u_obs[:nu]) ** 2).sum()).backward()
    gmu = _n(mu_t.grad)

    def Jof(m):
        with torch.no_grad():
            xx = stokes_solve_fn(S, _t(m), f, 1e-13)
            return 0.5 * float(((xx[:nu] - u_obs[:nu]) ** 2).sum())

    rng = np.random.default_rng(0)
    eps = 1e-6
    for c in rng.choice(n ** 3, 20, replace=False):
        mp, mm = mu.copy(), mu.copy()
        mp[c] *= 1 + eps
        mm[c] *= 1 - eps
        fd = (Jof(mp) - Jof(mm)) / (2 * eps * mu[c])
        assert abs(fd - gmu[c]) <= 1e-6 * np.abs(gmu).max(), (c, fd, gmu[c])
