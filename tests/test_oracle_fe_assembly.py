"""Pins of the oracle's finite-element layer against closed forms and invariants (CPU only)."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle.assemble import Tables, assemble, element_matrices
from oracle.fe import gauss_legendre, gauss_lobatto, lagrange_derivatives, lagrange_values
from oracle.mesh import Hierarchy, Level, dof_counts

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_gauss_lobatto_closed_forms():
    np.testing.assert_allclose(gauss_lobatto(2), [0, 0.5, 1], atol=1e-15)
    a = 0.5 * (1 - np.sqrt(1 / 5))
    np.testing.assert_allclose(gauss_lobatto(3), [0, a, 1 - a, 1], atol=1e-14)
    b = 0.5 * (1 - np.sqrt(3 / 7))
    np.testing.assert_allclose(gauss_lobatto(4), [0, b, 0.5, 1 - b, 1], atol=1e-14)


def test_gauss_legendre_closed_form_and_exactness():
    x, w = gauss_legendre(3)
    np.testing.assert_allclose(x, [0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)], atol=1e-15)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], atol=1e-15)
    for n in (2, 3, 4, 5):
        x, w = gauss_legendre(n)
        for p in range(2 * n):
            assert abs(w @ x**p - 1.0 / (p + 1)) < 1e-14


@pytest.mark.parametrize("deg", [1, 2, 3, 4])
def test_lagrange_interpolates_and_differentiates_polynomials(deg):
    nodes = gauss_lobatto(deg)
    x = np.linspace(-0.2, 1.3, 17)
    L = lagrange_values(nodes, x)
    D = lagrange_derivatives(nodes, x)
    np.testing.assert_allclose(lagrange_values(nodes, nodes), np.eye(deg + 1), atol=1e-14)
    for p in range(deg + 1):
        np.testing.assert_allclose((nodes**p) @ L, x**p, atol=1e-12)
        np.testing.assert_allclose((nodes**p) @ D, p * x ** max(p - 1, 0) if p else 0 * x, atol=1e-11)


def test_q2_1d_textbook_matrices():
    g = json.load(open(os.path.join(GOLD, "q2_1d.json")))
    from oracle.fe import Element1D
    e = Element1D(2, 3)
    K = np.einsum("iq,jq,q->ij", e.der, e.der, e.qw)
    M = np.einsum("iq,jq,q->ij", e.val, e.val, e.qw)
    np.testing.assert_allclose(3 * K, g["stiffness_times_3"], atol=1e-13)
    np.testing.assert_allclose(30 * M, g["mass_times_30"], atol=1e-13)


def test_dof_counts_match_paper():
    g = json.load(open(os.path.join(GOLD, "dof_counts.json")))
    for c in g["cases"]:
        nu, npr = dof_counts(c["dim"], c["k"], (c["n"],) * c["dim"])
        assert nu + npr == c["total"], c


def test_dof_counts_large_configs():
    # 3D Q2-Q1 on 32^3 and Q3-Q2 on a 64^3 channel: d(kn+1)^d + ((k-1)n+1)^d
    assert dof_counts(3, 2, (32, 32, 32)) == (823875, 35937)
    assert dof_counts(3, 3, (64, 64, 64)) == (21567171, 2146689)


def test_cartesian_element_is_kronecker_of_1d():
    # 2D unit-square cell: scalar stiffness = K1 (x) M1 + M1 (x) K1, mass = M1 (x) M1
    from oracle.fe import Element1D
    e = Element1D(2, 3)
    K1 = np.einsum("iq,jq,q->ij", e.der, e.der, e.qw)
    M1 = np.einsum("iq,jq,q->ij", e.val, e.val, e.qw)
    lev = Level(2, 2, (1, 1), W.lattice_vertices(2, (1, 1)))
    E = element_matrices(lev, Tables(2, 2), mu=1.0, gamma_rho=0.0)
    np.testing.assert_allclose(E["K0"][0], np.kron(M1, K1) + np.kron(K1, M1), atol=1e-13)
    np.testing.assert_allclose(E["Mv"][0], np.kron(M1, M1), atol=1e-14)


def _perturbed_level(dim, n, k=2, seed=3):
    V = W.perturbed_vertices(dim, (n,) * dim, seed=seed, amplitude=0.3)
    return Level(dim, k, (n,) * dim, V)


@pytest.mark.parametrize("dim,k", [(2, 2), (2, 3), (3, 2)])
def test_operator_invariants(dim, k):
    lev = _perturbed_level(dim, 3 if dim == 3 else 4, k)
    ops = assemble(lev, mu=1.3, gamma_rho=0.0)
    K = ops["K"]
    assert abs(K - K.T).max() < 1e-13
    # stiffness annihilates constants before Dirichlet elimination
    assert np.abs(ops["As_full"] @ np.ones(lev.nv)).max() < 1e-12
    # B^T 1_p = 0 under full Dirichlet data, also on trilinear cells (exact (k+1)-point Gauss)
    bt1 = ops["B"].T @ np.ones(lev.n_p)
    assert np.abs(bt1).max() < 1e-13
    # mass row sums give the (unchanged) domain volume
    assert abs(ops["Mv_full"].sum() - 1.0) < 1e-13
    assert abs(ops["Mp"].sum() - 1.0) < 1e-13
    # A is SPD on the free DoFs
    free = ~ops["umask"]
    Af = ops["A"].toarray()[np.ix_(free, free)]
    assert np.linalg.eigvalsh(Af).min() > 0


def test_b_sign_reading_gives_grad_p():
    # With b(v,q) = -int q div v, B^T p is the weak form of grad p: for p = x on (0,1)^2 and a
    # smooth bubble v, (B^T p) . v = int grad(p) . v = int v_1.
    lev = Level(2, 2, (4, 4), W.lattice_vertices(2, (4, 4)))
    ops = assemble(lev)
    xs = np.linspace(0, 1, lev.N[0])
    X, Y = np.meshgrid(xs, xs)  # y slow, x fast
    p = np.linspace(0, 1, lev.Pn[0])[None, :].repeat(lev.Pn[1], 0).reshape(-1)
    v1 = (X * (1 - X) * Y * (1 - Y)).reshape(-1)
    v = np.concatenate([v1, np.zeros(lev.nv)])
    lhs = (ops["B"].T @ p) @ v
    assert abs(lhs - 1.0 / 36.0) < 1e-13  # int x(1-x) y(1-y) = 1/36


def test_hierarchy_vertices_are_subsampled():
    V = W.perturbed_vertices(3, (8, 8, 8), seed=0)
    H = Hierarchy(3, 2, (8, 8, 8), 3, V)
    assert [lv.n for lv in H.levels] == [(2, 2, 2), (4, 4, 4), (8, 8, 8)]
    np.testing.assert_array_equal(H.levels[0].vertices, V[::4, ::4, ::4])


def test_mms_convergence_rates():
    from oracle import mms
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    uex, pex = mms.mms2d_exact()
    errs = []
    for n in (4, 8, 16, 32):
        lev = Level(2, 2, (n, n), W.lattice_vertices(2, (n, n)))
        ops = assemble(lev)
        b = mms.load_vector(lev, W.mms2d_forcing)
        e = np.concatenate([np.zeros(lev.n_u), np.ones(lev.n_p)])
        Kb = sp.bmat([[ops["K"], sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
        x = spla.spsolve(Kb, np.concatenate([b, [0.0]]))[:-1]
        errs.append(mms.l2_errors(lev, x, uex, pex))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    # ||u-u_h||_L2 = O(h^{k+1}) = O(h^3); ||p-p_h||_L2 = O(h^k) = O(h^2)  (Sec. 2 estimates)
    assert np.all(rates[1:, 0] > 2.9), rates
    assert np.all(rates[:, 1] > 1.9), rates


@pytest.mark.parametrize("k", [3, 4])
def test_sampled_oracle_rows_on_an_anisotropic_channel(k):
    """Sampled rows of K x (the oracle's full-size parity reference) against the assembled operator
    on a Cartesian channel box [0,4] x [0,1]^2 of anisotropic cells with the do-nothing face open
    (x = 4), for the higher degrees: the row-by-row gathering of the touching cells' element
    matrices must reproduce every kind of row (Dirichlet, outflow face, interior, pressure)."""
    import workloads as W
    from oracle.assemble import assemble
    from oracle.mesh import Level
    from oracle.sampled import apply_rows
    n = (4, 2, 2)
    lev = Level(3, k, n, W.lattice_vertices(3, n, hi=(4.0, 1.0, 1.0)), dirichlet_faces=0x3F & ~0x2)
    ops = assemble(lev, mu=1e-3, gamma_rho=0.0)
    x = W.random_vector(lev.size, 3)
    rows = np.random.default_rng(1).choice(lev.size, 80, replace=False)
    y = ops["K"] @ x
    np.testing.assert_allclose(apply_rows(lev, x, rows, 1e-3, 0.0), y[rows], rtol=1e-12,
                               atol=1e-12 * np.abs(y).max())
