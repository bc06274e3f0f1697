"""Pins of the oracle's transfers, Chebyshev-Jacobi smoother and Algorithm 2 (CPU only)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle.assemble import assemble
from oracle.fe import gauss_lobatto
from oracle.mesh import Hierarchy, Level
from oracle.smoother import (LevelSmoother, cheb_C, cheb_scalar_error, chebyshev, lanczos_max,
                             lemma1_scaling, local_schur_diag, splitmix64_uniform)
from oracle.transfer import prolongation, prolongation_1d

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --- transfers (Sec. 3.2) ------------------------------------------------------------------
def test_q2_injection_worked_row():
    g = json.load(open(os.path.join(GOLD, "q2_1d.json")))
    P = prolongation_1d(2, 1)
    np.testing.assert_allclose(P[1], g["injection_row_quarter"], atol=1e-15)
    np.testing.assert_allclose(P[::2], np.eye(3), atol=1e-15)  # coarse nodes are fine nodes


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_injection_reproduces_coarse_polynomials(deg):
    nc = 3
    P = prolongation_1d(deg, nc)
    t = gauss_lobatto(deg)
    xc = np.concatenate([(c + t[:-1]) / nc for c in range(nc)] + [[1.0]])
    xf = np.concatenate([(c + t[:-1]) / (2 * nc) for c in range(2 * nc)] + [[1.0]])
    # every polynomial of degree <= deg lies in the coarse space and is reproduced exactly
    rng = np.random.default_rng(0)
    coef = rng.standard_normal(deg + 1)
    np.testing.assert_allclose(P @ np.polyval(coef, xc), np.polyval(coef, xf), atol=1e-12)
    # a continuous piecewise-linear hat (in every space with deg >= 1) is reproduced too
    hat = np.maximum(0.0, 1.0 - np.abs(3.0 * xc - 1.0))
    np.testing.assert_allclose(P @ hat, np.maximum(0.0, 1.0 - np.abs(3.0 * xf - 1.0)), atol=1e-12)


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 2)])
def test_galerkin_identity_on_affine_meshes(dim, n):
    # nested spaces + exact quadrature on affine cells: K_{l-1} = P^T K_l P on the free DoFs
    V = W.lattice_vertices(dim, (2 * n,) * dim, hi=(2.0, 1.0, 0.5))
    H = Hierarchy(dim, 2, (2 * n,) * dim, 2, V)
    c, f = H.levels
    Kc = assemble(c, mu=0.7, gamma_rho=3.0)["K"]
    Kf = assemble(f, mu=0.7, gamma_rho=3.0)["K"]
    P = prolongation(c, f)
    G = (P.T @ Kf @ P).toarray()
    free = ~c.constrained()
    np.testing.assert_allclose(G[np.ix_(free, free)], Kc.toarray()[np.ix_(free, free)], atol=1e-12)


# --- Chebyshev-Jacobi (Sec. 3.3.1, Lemma 1, Algorithm 2) -----------------------------------
def test_lemma1_scaling_closed_forms():
    g = json.load(open(os.path.join(GOLD, "lemma1_scaling.json")))
    for c in g["cases"]:
        assert abs(lemma1_scaling(c["k"]) - c["num"] / c["den"]) < 1e-15
        assert Fraction(int(round(cheb_C(c["k"] + 1, 3.0)))) == c["num"]
    assert abs(cheb_C(5, 0.3) - np.cos(5 * np.arccos(0.3))) < 1e-14


@pytest.mark.parametrize("k", [0, 1, 2, 3, 5])
def test_chebyshev_error_polynomial_on_diagonal_matrix(k):
    # For M = diag(lambda), D = I: (I - Cheb(M, I, k) M) e = T_{k+1}(lambda) e in closed form
    lam = np.linspace(0.01, 2.0, 50)
    beta = 2.0
    e = np.ones_like(lam)
    x = chebyshev(lambda v: lam * v, np.ones_like(lam), lam * e, k, beta)
    np.testing.assert_allclose(e - x, cheb_scalar_error(lam, k, beta), atol=1e-13)


def test_chebyshev_degree0_is_damped_jacobi():
    rng = np.random.default_rng(1)
    Dinv = rng.uniform(0.5, 2, 20)
    r = rng.standard_normal(20)
    beta = 1.7
    x = chebyshev(None, Dinv, r, 0, beta)
    np.testing.assert_allclose(x, 2.0 / (0.5 * beta + beta) * Dinv * r, atol=1e-15)


def test_lanczos_matches_dense_eigensolver():
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    ev = np.concatenate([rng.uniform(0, 1, 59), [1.7]])
    S = (Q * ev) @ Q.T
    est = lanczos_max(lambda v: S @ v, rng.standard_normal(60), 40)
    assert abs(est - 1.7) < 1e-8 and est <= 1.7 + 1e-12


def test_splitmix64_reference_values():
    # SplitMix64 with seed 0: first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4 (published test vector)
    u = splitmix64_uniform(0, 2)
    for val, ref in zip(u, (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4)):
        assert val == 2.0 * ((ref >> 11) * 2.0**-53) - 1.0


def _tiny_smoother(schur_diag="loc", gamma_rho=0.0, dim=2, n=4, kA=2, kS=2):
    V = W.perturbed_vertices(dim, (n,) * dim, seed=5, amplitude=0.3)
    lev = Level(dim, 2, (n,) * dim, V)
    ops = assemble(lev, mu=1.0, gamma_rho=gamma_rho)
    return lev, ops, LevelSmoother(lev, ops, kA, kS, schur_diag, 1.0, gamma_rho, eig_steps=60)


@pytest.mark.parametrize("diag", ["loc", "p", "d", "exact"])
def test_lemma1_spectral_inequalities(diag):
    # A_hat >= A and S_hat >= S_tilde: eigenvalues of A^-1_hat A and S^-1_hat S_tilde in (0, 1]
    lev, ops, S = _tiny_smoother(diag)
    free = ~ops["umask"]
    Ai = S.dense_Ainv_hat()[np.ix_(free, free)]
    A = ops["A"].toarray()[np.ix_(free, free)]
    ev = np.real(np.linalg.eigvals(Ai @ A))
    assert ev.min() > 0 and ev.max() <= 1.0 + 1e-12
    Si = S.dense_Sinv_hat()
    St = np.stack([S.S_tilde(e) for e in np.eye(lev.n_p)], axis=1)
    ev = np.sort(np.real(np.linalg.eigvals(Si @ St)))
    # one zero eigenvalue: the constant pressure under full Dirichlet data
    assert abs(ev[0]) < 1e-10 and ev[1] > 0 and ev[-1] <= 1.0 + 1e-12


def test_schur_diagonal_variants_brute_force():
    lev, ops, S = _tiny_smoother("d")
    B = ops["B"].toarray()
    DA = ops["A"].diagonal()
    np.testing.assert_allclose(S.DS, (B**2 / DA[None, :]).sum(1), rtol=1e-13)
    # local variant by an explicit per-cell loop
    from oracle.assemble import Tables, element_matrices
    tab = Tables(2, 2)
    E = element_matrices(lev, tab, 1.0, 0.0)
    vn, pn = lev.cell_velocity_nodes(), lev.cell_pressure_nodes()
    vm = lev.velocity_constrained()
    ref = np.zeros(lev.n_p)
    for c in range(lev.n_cells):
        for i in range(pn.shape[1]):
            s = 0.0
            for a in range(2):
                for j in range(vn.shape[1]):
                    if not vm[vn[c, j]]:
                        s += E["B"][c, i, a, j] ** 2 / E["As"][c, j, j]
            ref[pn[c, i]] += s
    np.testing.assert_allclose(local_schur_diag(lev, 1.0, 0.0), ref, rtol=1e-13)


def test_smoother_compact_form_identity():
    # the Uzawa step equals x + K_hat^{-1}(b - K x), K_hat = [A_hat B^T; B B A_hat^-1 B^T - S_hat]
    lev, ops, S = _tiny_smoother("loc", gamma_rho=10.0, kA=1, kS=2)
    free = ~lev.constrained()
    nu = lev.n_u
    rng = np.random.default_rng(4)
    x = rng.standard_normal(lev.size) * free
    b = rng.standard_normal(lev.size) * free
    x1 = S.step(x, b)
    fu = free[:nu]
    Ai = S.dense_Ainv_hat()[np.ix_(fu, fu)]
    Si = S.dense_Sinv_hat()
    Ah = np.linalg.inv(Ai)
    Sh = np.linalg.inv(Si)
    B = ops["B"].toarray()[:, fu]
    Kh = np.block([[Ah, B.T], [B, B @ Ai @ B.T - Sh]])
    K = ops["K"].toarray()[np.ix_(free, free)]
    ref = x[free] + np.linalg.solve(Kh, b[free] - K @ x[free])
    np.testing.assert_allclose(x1[free], ref, rtol=1e-9, atol=1e-11)
    assert np.all(x1[~free] == 0)
