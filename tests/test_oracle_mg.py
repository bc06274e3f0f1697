"""Pins of the oracle's multigrid cycle, coarse solve and outer Krylov loop (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle.assemble import assemble, load_vector_nodal
from oracle.krylov import fgmres
from oracle.mesh import Hierarchy, Level
from oracle.mg import CoarseSolver, Multigrid


def _bordered_direct(lev, K, b):
    if not lev.has_pressure_kernel():
        return spla.spsolve(K.tocsc(), b)
    e = np.concatenate([np.zeros(lev.n_u), np.ones(lev.n_p)])
    Kb = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
    return spla.spsolve(Kb, np.concatenate([b, [0.0]]))[:-1]


def _problem(dim, n, levels, seed=0, perturb=False, gamma_rho=0.0, faces=0x3F, **kw):
    V = (W.perturbed_vertices(dim, (n,) * dim, seed=seed) if perturb else W.lattice_vertices(dim, (n,) * dim))
    H = Hierarchy(dim, 2, (n,) * dim, levels, V, faces)
    mg = Multigrid(H, gamma_rho=gamma_rho, **kw)
    lev = H.levels[-1]
    f = W.fourier_forcing(dim, 2, (n,) * dim, seed=seed)
    b = load_vector_nodal(lev, mg.ops[-1], f)
    return H, mg, lev, b


def test_coarse_bordered_solve_picks_mean_free_pressure():
    lev = Level(2, 2, (2, 2), W.lattice_vertices(2, (2, 2)))
    K = assemble(lev)["K"]
    cs = CoarseSolver(lev, K)
    rng = np.random.default_rng(0)
    x_true = rng.standard_normal(lev.size) * ~lev.constrained()
    x_true[lev.n_u:] -= x_true[lev.n_u:].mean()
    x = cs.solve(K @ x_true)
    np.testing.assert_allclose(x, x_true, atol=1e-11)


@pytest.mark.parametrize("dim,n,levels,perturb", [(2, 8, 3, False), (2, 8, 3, True), (3, 4, 2, True)])
def test_fgmres_vcycle_matches_direct_solve(dim, n, levels, perturb):
    H, mg, lev, b = _problem(dim, n, levels, perturb=perturb, kA=2, kS=2, m=2)
    x, its, hist = fgmres(lambda v: mg.K @ v, mg.precondition, b, rtol=1e-12)
    xd = _bordered_direct(lev, mg.K, b)
    x[lev.n_u:] -= x[lev.n_u:].mean()
    xd[lev.n_u:] -= xd[lev.n_u:].mean()
    assert np.linalg.norm(b - mg.K @ x) <= 1e-12 * np.linalg.norm(b) * 1.01
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
    assert its <= 15


def test_level_independent_iteration_counts():
    # q and FGMRES iteration counts stay flat under h-refinement (Sec. 4.3.3)
    counts, rates = [], []
    # (coarsest mesh 2x2; levels 4..6 are past the pre-asymptotic range)
    for levels in (4, 5, 6):
        n = 2 ** levels
        H, mg, lev, b = _problem(2, n, levels, kA=1, kS=1, m=2)
        _, its, _ = fgmres(lambda v: mg.K @ v, mg.precondition, b, rtol=1e-10)
        _, _, q = mg.stationary(b)
        counts.append(its)
        rates.append(q)
    assert max(counts) - min(counts) <= 1, counts
    assert max(rates) - min(rates) < 0.05 and max(rates) < 0.35, rates


def test_rate_improves_with_smoothing_steps_and_v_close_to_w():
    qs = {}
    for m in (1, 2, 4):
        for cyc in ("V", "W"):
            H, mg, lev, b = _problem(2, 16, 4, kA=1, kS=1, m=m, cycle=cyc)
            qs[(m, cyc)] = mg.stationary(b)[2]
    assert qs[(1, "V")] > qs[(2, "V")] > qs[(4, "V")]
    for m in (1, 2, 4):
        assert abs(qs[(m, "V")] - qs[(m, "W")]) < 0.5 * qs[(m, "W")] + 0.02


def test_generalized_stokes_rates_independent_of_gamma():
    # Sec. 4.6: the mass term gamma*rho does not deteriorate the rates
    qs = []
    for g in (0.0, 1.0, 100.0):
        H, mg, lev, b = _problem(2, 16, 4, gamma_rho=g, kA=2, kS=2, m=2)
        qs.append(mg.stationary(b)[2])
    assert max(qs) < 0.25, qs


def test_partial_dirichlet_has_no_pressure_kernel():
    # do-nothing outflow at x = 1: K is nonsingular and the coarse solve is not bordered
    H, mg, lev, b = _problem(2, 8, 3, faces=0x3F & ~0x2, kA=2, kS=2, m=2)
    assert not lev.has_pressure_kernel() and not mg.coarse.bordered
    x, its, _ = fgmres(lambda v: mg.K @ v, mg.precondition, b, rtol=1e-11)
    xd = spla.spsolve(mg.K.tocsc(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8


def test_schur_diagonal_choices_follow_the_papers_comparison():
    # Sec. 4.3 (2D driven cavity, 2,467 DoFs): diag d gives nearly the rates of the exact diagonal,
    # the local one falls behind, more smoothing steps help.  With k_A = 0, A^-1_hat = sigma
    # diag(A)^-1, so the exact diagonal is sigma times diag d and the Chebyshev iteration (whose
    # eigenvalue bound is rescaled by Lanczos) is the same: equal rates.
    q = {}
    for k in (0, 3):
        for m in (1, 2):
            for diag in ("loc", "p", "d", "exact"):
                _, mg, _, b = _problem(2, 16, 4, kA=k, kS=k, m=m, cycle="W", schur_diag=diag)
                q[(k, m, diag)] = mg.stationary(b)[2]
    for m in (1, 2):
        assert abs(q[(0, m, "d")] - q[(0, m, "exact")]) <= 1e-6 * q[(0, m, "exact")]
        assert abs(q[(3, m, "d")] - q[(3, m, "exact")]) <= 0.2 * q[(3, m, "exact")]
        assert q[(3, m, "loc")] > q[(3, m, "exact")]
    for diag in ("loc", "p", "d", "exact"):
        assert q[(3, 2, diag)] < q[(3, 1, diag)] < 1


# ---- exact pin of Algorithm 1: the cycle's error propagation operator ----------------------------
def _dense_smoother_propagation(sm, K):
    """S = I - M_s K for one compact-form Uzawa step (Sec. 3.3.1, K_hat), written from the dense
    A^-1_hat and S^-1_hat: for a residual (r_u, r_p),
        dp = S^-1_hat (B A^-1_hat r_u - r_p),  du = A^-1_hat (r_u - B^T dp)."""
    Ai, Si = sm.dense_Ainv_hat(), sm.dense_Sinv_hat()
    B = sm.B.toarray()
    Cm = sm.C.toarray()
    nu, npr = Ai.shape[0], Si.shape[0]
    # dp = Si (B Ai r_u - r_p - C p)  -- with C = 0 here the pressure residual is g - B u
    M = np.zeros((nu + npr, nu + npr))
    M[nu:, :nu] = Si @ B @ Ai
    M[nu:, nu:] = -Si
    M[:nu, :nu] = Ai - Ai @ B.T @ M[nu:, :nu]
    M[:nu, nu:] = -Ai @ B.T @ M[nu:, nu:]
    assert np.abs(Cm).max() == 0.0
    return np.eye(nu + npr) - M @ K.toarray()


def _bordered_pinv(lev, K):
    """The coarse direct solve as a matrix: top-left block of inv([K e; e^T 0]), e = (0, 1_p) when
    the constant pressure spans the kernel, else inv(K) (numpy, independent of the oracle's LU)."""
    Kd = K.toarray()
    if not lev.has_pressure_kernel():
        return np.linalg.inv(Kd)
    e = np.concatenate([np.zeros(lev.n_u), np.ones(lev.n_p)])
    Kb = np.block([[Kd, e[:, None]], [e[None, :], np.zeros((1, 1))]])
    return np.linalg.inv(Kb)[: lev.size, : lev.size]


def _cycle_propagation(mg, l, gamma):
    """E_l = S_l^m (I - P_l (I - E_{l-1}^gamma) K_{l-1}^+ P_l^T K_l) S_l^m, E_0 = 0 (exact coarse
    solve): the error propagation of Algorithm 1 (pre-smoothing, residual, restriction, gamma
    recursive calls from zero, prolongation and correction, post-smoothing)."""
    if l == 0:
        return np.zeros((mg.hier.levels[0].size,) * 2)
    K = mg.ops[l]["K"]
    S = np.linalg.matrix_power(_dense_smoother_propagation(mg.smoothers[l], K), mg.m)
    P = mg.P[l].toarray()
    Ec = _cycle_propagation(mg, l - 1, gamma)
    lc = mg.hier.levels[l - 1]
    inner = (np.eye(lc.size) - np.linalg.matrix_power(Ec, gamma)) @ _bordered_pinv(lc, mg.ops[l - 1]["K"])
    return S @ (np.eye(K.shape[0]) - P @ inner @ P.T @ K.toarray()) @ S


@pytest.mark.parametrize("dim,n,levels,cycle,diag", [(2, 4, 2, "V", "loc"), (3, 4, 2, "V", "d"),
                                                     (2, 8, 3, "V", "d"), (2, 8, 3, "W", "loc")])
def test_cycle_error_propagation_is_algorithm_1(dim, n, levels, cycle, diag):
    """One oracle cycle maps the error x - x* to E (x - x*), E formed densely from the smoother,
    transfer and coarse-solve matrices in the order of Algorithm 1, to 1e-12.  A dropped or
    reordered step (smoothing on one side only, a missing restriction or correction, the wrong
    number of recursive calls) changes E."""
    H, mg, lev, _ = _problem(dim, n, levels, perturb=True, gamma_rho=3.0, kA=2, kS=1, m=2, cycle=cycle,
                             schur_diag=diag)
    rng = np.random.default_rng(7)
    free = ~lev.constrained()
    x_true = rng.standard_normal(lev.size) * free
    b = mg.K @ x_true
    x0 = rng.standard_normal(lev.size) * free
    x1 = mg.cycle(levels - 1, x0, b)
    E = _cycle_propagation(mg, levels - 1, mg.gamma)
    pred = E @ (x0 - x_true)
    err = np.abs((x1 - x_true) - pred).max() / np.abs(pred).max()
    assert err < 1e-12, err
    # the pin is sharp: the cycle without its post-smoothing, or with the other number of recursive
    # calls, is far from E
    K = mg.ops[-1]["K"]
    S = np.linalg.matrix_power(_dense_smoother_propagation(mg.smoothers[-1], K), mg.m)
    E_nopost = np.linalg.solve(S, E)
    assert np.abs(E_nopost @ (x0 - x_true) - pred).max() / np.abs(pred).max() > 1e-3
    if levels == 3:
        E_other = _cycle_propagation(mg, levels - 1, 3 - mg.gamma)
        assert np.abs(E_other @ (x0 - x_true) - pred).max() / np.abs(pred).max() > 1e-3
