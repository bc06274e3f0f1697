"""Oracle with a stabilisation block C != 0 in K = [A B^T; B -C] (Sec. 1: C non-negative, usually
zero, non-trivial under stabilisations).  Reading of the paper's open C:
    c(p, q) = c_mass int p q + c_grad sum_tau h_tau^2 int_tau grad p . grad q,  h_tau = |tau|^(1/d).
Pins: the textbook Q1 stiffness stencils on Cartesian cells, constants in the kernel of the
Laplacian part, the total of the mass part, the compact form of the smoother with C, and
FGMRES + multigrid against a sparse direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle.assemble import assemble, load_vector_nodal
from oracle.krylov import fgmres
from oracle.mesh import Hierarchy, Level
from oracle.mg import Multigrid
from oracle.smoother import LevelSmoother


def _cart(dim, n):
    return Level(dim, 2, (n,) * dim, W.lattice_vertices(dim, (n,) * dim))


def test_q1_pressure_laplacian_matches_the_textbook_stencils():
    # Q1 stiffness on a square of side h: 8/3 on the diagonal, -1/3 to each of the 8 neighbours;
    # on a cube of side h: 8h/3, 0 to face, -h/6 to edge and -h/12 to corner neighbours.  With
    # the factor h_tau^2 of the stabilisation, an interior row of C is h^2 times the assembled stencil.
    for dim, n in ((2, 4), (3, 4)):
        lev = _cart(dim, n)
        h = 1.0 / n
        C = assemble(lev, c_grad=1.0)["C"].toarray()
        Pn = lev.Pn[0]
        centre = (n // 2,) * dim
        idx = lambda g: sum(g[a] * Pn ** a for a in range(dim))
        i = idx(centre)
        if dim == 2:
            # interior Q1 9-point stencil of -Laplace (scale-invariant in 2D): 8/3, -1/3 (all 8)
            for off in np.ndindex(3, 3):
                g = tuple(c + o - 1 for c, o in zip(centre, off))
                ndiff = sum(o != 1 for o in off)
                ref = (8 / 3 if ndiff == 0 else -1 / 3) * h ** 2
                assert abs(C[i, idx(g)] - ref) < 1e-13
        else:
            for off in np.ndindex(3, 3, 3):
                g = tuple(c + o - 1 for c, o in zip(centre, off))
                ndiff = sum(o != 1 for o in off)
                ref = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[ndiff] * h ** 2
                assert abs(C[i, idx(g)] - ref) < 1e-14
        assert abs(C[i]).sum() > 0 and np.count_nonzero(np.abs(C[i]) > 1e-15) <= 3 ** dim


def test_laplacian_part_kills_constants_and_mass_part_integrates():
    V = W.perturbed_vertices(3, (4, 4, 4), seed=2)
    lev = Level(3, 2, (4, 4, 4), V)
    one = np.ones(lev.n_p)
    Cg = assemble(lev, c_grad=2.5)["C"]
    assert np.abs(Cg @ one).max() < 1e-14
    Cm = assemble(lev, c_mass=0.7)["C"]
    assert abs(one @ (Cm @ one) - 0.7) < 1e-12  # c_mass |Omega|, |Omega| = 1 (boundary fixed)
    Ca = assemble(lev, c_mass=0.7, c_grad=2.5)["C"]
    ev = np.linalg.eigvalsh(Ca.toarray())
    assert ev.min() > 0 and np.abs(Ca - Ca.T).max() < 1e-15


def test_smoother_compact_form_with_stabilisation():
    # with C the step is still x + K_hat^-1 (b - K x), K_hat = [A_hat B^T; B B A_hat^-1 B^T - S_hat]:
    # C enters through the residual b - K x and through S~ = B A_hat^-1 B^T + C, which S_hat
    # approximates
    lev = Level(2, 2, (3, 3), W.perturbed_vertices(2, (3, 3), seed=3))
    ops = assemble(lev, 1.0, 10.0, c_mass=0.3, c_grad=4.0)
    S = LevelSmoother(lev, ops, 1, 2, "loc", 1.0, 10.0)
    free = ~lev.constrained()
    nu = lev.n_u
    rng = np.random.default_rng(5)
    x = rng.standard_normal(lev.size) * free
    b = rng.standard_normal(lev.size) * free
    x1 = S.step(x, b)
    fu = free[:nu]
    Ai = S.dense_Ainv_hat()[np.ix_(fu, fu)]
    Sh = np.linalg.inv(S.dense_Sinv_hat())
    B = ops["B"].toarray()[:, fu]
    Kh = np.block([[np.linalg.inv(Ai), B.T], [B, B @ Ai @ B.T - Sh]])
    K = ops["K"].toarray()[np.ix_(free, free)]
    ref = x[free] + np.linalg.solve(Kh, b[free] - K @ x[free])
    np.testing.assert_allclose(x1[free], ref, rtol=1e-9, atol=1e-11)
    # S~ includes C, and D_S~ includes diag(C)
    q = rng.standard_normal(lev.n_p)
    Sq = ops["B"] @ S.Ainv_hat(ops["B"].T @ q) + ops["C"] @ q
    np.testing.assert_allclose(S.S_tilde(q), Sq, rtol=1e-12, atol=1e-14)


def test_fgmres_multigrid_with_stabilisation_matches_direct_solve():
    V = W.perturbed_vertices(2, (16, 16), seed=1)
    H = Hierarchy(2, 2, (16, 16), 3, V)
    for cm, cg in ((0.5, 0.0), (0.0, 2.0), (0.2, 1.0)):
        mg = Multigrid(H, kA=1, kS=2, m=2, c_mass=cm, c_grad=cg)
        lev = H.levels[-1]
        b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(2, 2, (16, 16), seed=4).reshape(-1))
        x, its, _ = fgmres(lambda v: mg.K @ v, mg.precondition, b, rtol=1e-12)
        assert its <= 20
        if mg.ops[-1]["pker"]:  # c_mass = 0: constants remain in the pressure kernel
            x[lev.n_u:] -= x[lev.n_u:].mean()
            r = lev.n_u  # pin the first pressure value for the reference solve
            xd = spla.spsolve(mg.K.tocsc()[:, np.r_[0:r, r + 1:lev.size]][np.r_[0:r, r + 1:lev.size]],
                              b[np.r_[0:r, r + 1:lev.size]])
            xd = np.insert(xd, r, 0.0)
            xd[lev.n_u:] -= xd[lev.n_u:].mean()
        else:
            xd = spla.spsolve(mg.K.tocsc(), b)
        assert np.abs(x - xd).max() < 1e-8 * np.abs(xd).max()


@pytest.mark.parametrize("diag", ["loc", "p", "d", "exact"])
def test_lemma1_inequalities_with_stabilisation(diag):
    # Lemma 1 with C: A_hat >= A and S_hat >= S~ = B A^-1_hat B^T + C, i.e. the eigenvalues of
    # A_hat^-1 A and S_hat^-1 S~ lie in (0, 1]
    lev = Level(2, 2, (4, 4), W.perturbed_vertices(2, (4, 4), seed=5, amplitude=0.3))
    ops = assemble(lev, c_mass=0.4, c_grad=3.0)
    S = LevelSmoother(lev, ops, 2, 2, diag, eig_steps=60)
    free = ~ops["umask"]
    Ai = S.dense_Ainv_hat()[np.ix_(free, free)]
    A = ops["A"].toarray()[np.ix_(free, free)]
    ea = np.linalg.eigvals(Ai @ A).real
    assert ea.min() > 0 and ea.max() <= 1 + 1e-10
    St = np.stack([S.S_tilde(e) for e in np.eye(lev.n_p)], axis=1)
    es = np.linalg.eigvals(S.dense_Sinv_hat() @ St).real
    assert es.min() > 0 and es.max() <= 1 + 1e-10
