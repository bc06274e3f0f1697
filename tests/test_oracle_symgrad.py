"""Oracle of the symmetric-gradient form (Sec. 2): a(u,v) = int mu eps(u):eps(v) + gamma rho u.v,
eps(u) = (grad u + grad u^T)/2, mu and rho constant per cell.  Pins (all on the assembled velocity
block without Dirichlet rows): a field with a symmetric gradient sees the same operator as in the
Laplacian form, an infinitesimal rotation is in the kernel, on H^1_0 and Cartesian cells the form is
half the Laplacian plus half grad-div (integration by parts, exact quadrature), rho scales the mass
part cell by cell; and FGMRES + multigrid agrees with a sparse direct solve."""
import numpy as np
import scipy.sparse.linalg as spla

import workloads as W
from oracle.assemble import assemble, load_vector_nodal
from oracle.krylov import fgmres
from oracle.mesh import Hierarchy, Level


def _nodes(lev):
    N = lev.N[: lev.dim]
    xs = [np.linspace(0.0, 1.0, N[a]) for a in range(lev.dim)]
    g = np.meshgrid(*xs[::-1], indexing="ij")[::-1]  # x fastest
    return [c.reshape(-1) for c in g]


def test_symmetric_gradient_field_and_rotation():
    for dim, n in ((2, 4), (3, 3)):
        # affine fields need the physical node coordinates: the Cartesian lattice
        lev = Level(dim, 2, (n,) * dim, W.lattice_vertices(dim, (n,) * dim))
        X = _nodes(lev)
        As = assemble(lev, mu=1.3, sym=True)["A_full"]
        Al = assemble(lev, mu=1.3)["A_full"]
        zero = np.zeros(lev.nv)
        # u = (x, -y[, 0]): grad u symmetric, so eps(u):eps(v) = grad u : grad v
        u = np.concatenate([X[0], -X[1]] + ([zero] if dim == 3 else []))
        np.testing.assert_allclose(As @ u, Al @ u, atol=1e-13)
        assert np.abs(Al @ u).max() > 1e-3
        # u = (-y, x[, 0]): eps(u) = 0
        u = np.concatenate([-X[1], X[0]] + ([zero] if dim == 3 else []))
        assert np.abs(As @ u).max() < 1e-13
        assert np.abs(Al @ u).max() > 1e-3


def test_half_laplacian_plus_half_grad_div_on_h10_cartesian():
    from oracle.assemble import Tables, _scatter, geometry
    for dim, n in ((2, 4), (3, 2)):
        lev = Level(dim, 2, (n,) * dim, W.lattice_vertices(dim, (n,) * dim))
        free = ~np.tile(lev.velocity_constrained(), dim)
        As = assemble(lev, mu=1.0, sym=True)["A_full"].toarray()[np.ix_(free, free)]
        Al = assemble(lev, mu=1.0)["A_full"].toarray()[np.ix_(free, free)]
        # grad-div, int (div phi)(div psi), by quadrature of the physical gradients
        tab = Tables(dim, 2)
        vn = lev.cell_velocity_nodes()
        nc = lev.n_cells
        cols = (vn[:, None, :] + (np.arange(dim) * lev.nv)[None, :, None]).reshape(nc, -1)
        _, detJ, JinvT = geometry(tab, lev.cell_vertices())
        grad = np.einsum("cqab,iqb->ciqa", JinvT, tab.dphi)
        wdet = detJ * tab.w[None, :]
        GD = np.einsum("cq,ciqa,cjqb->caibj", wdet, grad, grad).reshape(nc, dim * grad.shape[1], -1)
        Gd = _scatter(cols, cols, GD, (lev.n_u, lev.n_u)).toarray()[np.ix_(free, free)]
        np.testing.assert_allclose(As, 0.5 * Al + 0.5 * Gd, atol=1e-13)


def test_rho_scales_the_mass_part_per_cell():
    lev = Level(3, 2, (2, 2, 2), W.perturbed_vertices(3, (2, 2, 2), seed=1))
    rho = np.array([1.0, 2.0, 0.5, 3.0, 1.5, 0.25, 4.0, 1.0])
    g = 7.0
    A1 = assemble(lev, mu=1.0, gamma_rho=g, rho_cell=rho, sym=True)["A_full"]
    A0 = assemble(lev, mu=1.0, gamma_rho=0.0, rho_cell=rho, sym=True)["A_full"]
    ones = np.concatenate([np.ones(lev.nv), np.zeros(2 * lev.nv)])
    vol = assemble(lev)["Mv_full"].sum()  # |Omega|
    from oracle.assemble import Tables, element_matrices
    E = element_matrices(lev, Tables(3, 2), 1.0, 0.0)
    assert abs(ones @ ((A1 - A0) @ ones) - g * (rho * E["vol"]).sum()) < 1e-12
    assert abs(E["vol"].sum() - vol) < 1e-12


def test_symmetric_form_fgmres_matches_direct_solve():
    from oracle.mg import Multigrid
    n = (8, 8, 8)
    V = W.perturbed_vertices(3, n, seed=2)
    H = Hierarchy(3, 2, n, 3, V)
    rng = np.random.default_rng(0)
    mu = np.exp(rng.standard_normal(512) * 0.5)
    rho = np.exp(rng.standard_normal(512) * 0.5)
    mus, rhos = [mu], [rho]
    for _ in range(2):  # coarse values: mean of the 2^3 children
        m = mus[0].reshape(n[0] // 2 ** (len(mus) - 1), -1)
        k = n[0] // 2 ** (len(mus) - 1)
        coarsen = lambda a: a.reshape(k // 2, 2, k // 2, 2, k // 2, 2).mean(axis=(1, 3, 5)).reshape(-1)
        mus.insert(0, coarsen(mus[0]))
        rhos.insert(0, coarsen(rhos[0]))
    mg = Multigrid(H, gamma_rho=10.0, kA=1, kS=2, m=2, mu_cells=mus, rho_cells=rhos, sym=True)
    lev = H.levels[-1]
    b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(3, 2, n, seed=5).reshape(-1))
    x, its, _ = fgmres(lambda v: mg.K @ v, mg.precondition, b, rtol=1e-11)
    assert its <= 20
    x[lev.n_u:] -= x[lev.n_u:].mean()
    r = lev.n_u
    keep = np.r_[0:r, r + 1:lev.size]
    xd = np.insert(spla.spsolve(mg.K.tocsc()[keep][:, keep], b[keep]), r, 0.0)
    xd[lev.n_u:] -= xd[lev.n_u:].mean()
    assert np.abs(x - xd).max() < 1e-8 * np.abs(xd).max()
