"""Lifting of inhomogeneous Dirichlet data and the paper's stationary multigrid driver on the GPU,
against the CPU oracle and exact polynomial Stokes flows."""
import numpy as np
import pytest

import workloads as W
from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", ["3d_q2_pert", "3d_q2_channel", "2d_q3_pert"])
def test_lift_rhs_matches_oracle(name):
    from oracle.assemble import assemble, lift
    case = CASES[name]
    lev = oracle_hierarchy(case).levels[-1]
    ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))
    S = gpu_solver(case)
    uD = random_full(lev, 31) * lev.constrained()
    b = random_full(lev, 32, constrained_zero=True)
    bg = S.lift_rhs(_t(uD), _t(b)).cpu().numpy()
    assert rel_err(bg, b - lift(lev, ops, uD)) < 1e-12


@pytest.mark.parametrize("outflow", [False, True])
def test_poiseuille_channel_solve(outflow):
    # u = (y (1 - y), 0, 0), p = 2 mu (L - x) in [0, 2] x [0, 1]^2: exact in Q2-Q1
    from paper_2205_15770_gb300 import StokesMG
    from oracle.mesh import Level
    mu, L = 1.0, 2.0
    faces = 0x3F & ~0x2 if outflow else 0x3F
    n = (8, 4, 4)
    S = StokesMG(dim=3, n=n, n_levels=3, k=2, mu=mu, hi=(L, 1.0, 1.0), dirichlet_faces=faces, vcycle_fp32=False)
    lev = Level(3, 2, n, W.lattice_vertices(3, n, hi=(L, 1.0, 1.0)), faces)
    xs = [np.linspace(0, (L, 1.0, 1.0)[a], lev.N[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    uex = np.zeros((3, lev.nv))
    uex[0] = (Y * (1 - Y)).reshape(-1)
    ps = [np.linspace(0, (L, 1.0, 1.0)[a], lev.Pn[a]) for a in range(3)]
    PZ, PY, PX = np.meshgrid(ps[2], ps[1], ps[0], indexing="ij")
    pex = 2 * mu * (L - PX.reshape(-1))
    uD = np.concatenate([(uex * lev.velocity_constrained()[None, :]).reshape(-1), np.zeros(lev.n_p)])
    b = S.lift_rhs(_t(uD), torch.zeros(lev.size, dtype=torch.float64, device="cuda"))
    x0, its, rel = S.solve(b, rtol=1e-12)
    x = x0.cpu().numpy() + uD
    assert np.abs(x[: lev.n_u] - uex.reshape(-1)).max() < 1e-9
    p = x[lev.n_u:]
    if not outflow:
        p = p - p.mean() + pex.mean()
    assert np.abs(p - pex).max() < 1e-8


def test_stationary_driver_matches_oracle():
    from oracle.assemble import load_vector_nodal
    from oracle.mg import Multigrid
    case = CASES["2d_q2_cart"]
    H = oracle_hierarchy(case)
    mg = Multigrid(H, kA=1, kS=1, m=2)
    lev = H.levels[-1]
    f = W.fourier_forcing(2, 2, case["n"], seed=2).reshape(-1)
    b = load_vector_nodal(lev, mg.ops[-1], f)
    x_o, res_o, q_o = mg.stationary(b)
    S = gpu_solver(case, kA=1, kS=1, m=2)
    x, it, hist, q = S.mg_iterate(_t(b), max_iter=15, reduction=1e-10)
    assert it == len(res_o) - 1
    np.testing.assert_allclose(hist, res_o, rtol=1e-6)
    assert abs(q - q_o) < 1e-6
    assert rel_err(x.cpu().numpy(), x_o) < 1e-8


@pytest.mark.parametrize("diag", ["p", "d", "exact"])
def test_stationary_driver_with_each_schur_diagonal(diag):
    # the paper's diagonal comparison (2D, 16^2, Chebyshev degree 3, W-cycle): GPU residual
    # history of the stationary driver against the oracle's
    from oracle.assemble import load_vector_nodal
    from oracle.mesh import Hierarchy
    from oracle.mg import Multigrid
    H = Hierarchy(2, 2, (16, 16), 4, W.lattice_vertices(2, (16, 16)))
    mg = Multigrid(H, kA=3, kS=3, m=1, cycle="W", schur_diag=diag)
    lev = H.levels[-1]
    b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(2, 2, (16, 16), seed=0).reshape(-1))
    _, res_o, q_o = mg.stationary(b)
    from paper_2205_15770_gb300 import StokesMG
    S = StokesMG(dim=2, n=(16, 16), n_levels=4, k=2, kA=3, kS=3, m=1, cycle="W", schur_diag=diag,
                 vcycle_fp32=False)
    _, it, hist, q = S.mg_iterate(_t(b), max_iter=15, reduction=1e-10)
    assert it == len(res_o) - 1
    # residuals near 1e-11 ||r_0|| carry the FP64 rounding of b - K x (~1e-16 |K||x|) in absolute terms
    np.testing.assert_allclose(hist, res_o, rtol=1e-6, atol=1e-14 * res_o[0])
    assert abs(q - q_o) < 1e-6


def test_w_cycle_stationary_rates_close_to_v_cycle():
    """Sec. 4.3.4: the V-cycle gives almost the same rate as the W-cycle.  The rates themselves are
    pinned to the oracle's stationary iteration (same mesh, data and smoother): for (k_A, k_S, m) =
    (1, 1, 2) with the local Schur diagonal in 3D both are q = 0.598, in line with the paper's 3D
    finding that this setting converges at q ~ 0.6 (Sec. 4.5; the GPU sweep of the 3D cavity gives
    0.60 as well), so the bound is q < 0.65 rather than a bound taken from 2D settings."""
    from oracle.assemble import load_vector_nodal
    from oracle.mg import Multigrid
    case = CASES["3d_q2_pert"]
    H = oracle_hierarchy(case)
    lev = H.levels[-1]
    fn = W.fourier_forcing(3, 2, case["n"], seed=3).reshape(-1)
    qs = {}
    for cyc in ("V", "W"):
        S = gpu_solver(case, kA=1, kS=1, m=2, cycle=cyc)
        b = S.mass_rhs(torch.as_tensor(fn, device="cuda"))
        _, it, hist, q = S.mg_iterate(b, max_iter=15, reduction=1e-10)
        qs[cyc] = q
        assert hist[-1] <= 1e-7 * hist[0]  # at most 15 cycles, as in the paper's protocol
        mg = Multigrid(H, gamma_rho=case["gamma_rho"], kA=1, kS=1, m=2, cycle=cyc)
        _, res, q_or = mg.stationary(load_vector_nodal(lev, mg.ops[-1], fn))
        assert abs(q - q_or) < 1e-6, (cyc, q, q_or)
        S.close()
    assert qs["V"] < 0.65, qs
    assert abs(qs["W"] - qs["V"]) <= 0.05, qs


@pytest.mark.parametrize("name", ["3d_q3_cart", "3d_q2_pert", "2d_q4_pert", "3d_q2_channel"])
def test_velocity_node_coordinates(name):
    from oracle.fe import gauss_lobatto
    case = CASES[name]
    lev = oracle_hierarchy(case).levels[-1]
    S = gpu_solver(case)
    xyz = S.velocity_nodes().cpu().numpy()
    k, d = lev.k, lev.dim
    t = gauss_lobatto(k)
    # reference: every cell maps its Gauss-Lobatto nodes through the bi/trilinear vertex map
    ref = np.full((lev.nv, d), np.nan)
    Xv = lev.cell_vertices()
    vn = lev.cell_velocity_nodes()
    import itertools
    loc = [tt[::-1] for tt in itertools.product(range(k + 1), repeat=d)]
    for j, tt in enumerate(loc):
        xi = [t[tt[a]] for a in range(d)]
        w = np.array([np.prod([xi[a] if (v >> a) & 1 else 1 - xi[a] for a in range(d)]) for v in range(2 ** d)])
        ref[vn[:, j]] = np.einsum("v,cva->ca", w, Xv)
    assert np.abs(xyz - ref).max() < 1e-13


@pytest.mark.parametrize("fp32", [True, False])
def test_device_krylov_loop_matches_host_loop(monkeypatch, fp32):
    """FGMRES with the Arnoldi state and the stopping test on the device (one graph launch per
    restart cycle) against the host-driven loop: same iteration counts, solutions within 1e-10,
    both at the requested FP64 residual under the oracle's assembled K."""
    import workloads as W
    from oracle.assemble import load_vector_nodal
    from oracle.mg import Multigrid
    from parity_cases import CASES, gpu_solver, oracle_hierarchy
    case = CASES["3d_q2_pert"]
    H = oracle_hierarchy(case)
    mg = Multigrid(H, gamma_rho=case["gamma_rho"], kA=1, kS=1, m=2, schur_diag="d")
    lev = H.levels[-1]
    b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(3, 2, case["n"], seed=8).reshape(-1))
    out = {}
    for host in (False, True):
        if host:
            monkeypatch.setenv("STOKES_HOST_KRYLOV", "1")
        else:
            monkeypatch.delenv("STOKES_HOST_KRYLOV", raising=False)
        S = gpu_solver(case, kA=1, kS=1, m=2, schur_diag="d", vcycle_fp32=fp32, restart=4)
        x, its, rel = S.solve(torch.as_tensor(b, device="cuda"), rtol=1e-10)
        assert S.krylov_mode == (0 if host else 1)
        xs = x.cpu().numpy()
        assert np.linalg.norm(b - mg.K @ xs) <= 1.01e-10 * np.linalg.norm(b)
        out[host] = (xs, its)
        S.close()
    assert out[False][1] == out[True][1]
    assert np.abs(out[False][0] - out[True][0]).max() <= 1e-10 * np.abs(out[True][0]).max()


@pytest.mark.parametrize("diag,kdeg,m", [("loc", 0, 4), ("p", 3, 1), ("d", 3, 2), ("exact", 3, 1)])
def test_laser_beam_stationary_driver_matches_oracle(diag, kdeg, m):
    """The laser-beam problem of Sec. 4.2 (unit square, Q2-Q1 on 16^2 = 2467 DoFs, mu = 0.0022,
    u_D = 0, Gaussian force at (0.75, 0.75)): the GPU stationary FP64 W-cycle iteration against the
    oracle's for each Schur diagonal, residual histories within 1e-6 and the rate q within 1e-6."""
    from oracle.assemble import load_vector_nodal
    from oracle.mesh import Hierarchy
    from oracle.mg import Multigrid
    from paper_2205_15770_gb300 import StokesMG
    mu = 0.0022
    H = Hierarchy(2, 2, (16, 16), 4, W.lattice_vertices(2, (16, 16)))
    mg = Multigrid(H, mu=mu, kA=kdeg, kS=kdeg, m=m, cycle="W", schur_diag=diag)
    lev = H.levels[-1]
    assert lev.size == 2467
    fn = W.laser_beam_forcing((16, 16)).reshape(-1)
    b = load_vector_nodal(lev, mg.ops[-1], fn)
    _, res_o, q_o = mg.stationary(b)
    S = StokesMG(dim=2, n=(16, 16), n_levels=4, k=2, mu=mu, kA=kdeg, kS=kdeg, m=m, cycle="W", schur_diag=diag,
                 vcycle_fp32=False)
    bg = S.mass_rhs(_t(fn))
    assert rel_err(bg.cpu().numpy(), b) < 1e-12
    _, it, hist, q = S.mg_iterate(bg, max_iter=15, reduction=1e-10, allow_divergence=True)
    assert it == len(res_o) - 1
    np.testing.assert_allclose(hist, res_o, rtol=1e-6, atol=1e-14 * res_o[0])
    # q = (r_j / r_{j-3})^(1/3) takes the last residuals, near 1e-11 r_0, where the FP64 rounding of
    # b - K x (about 1e-16 |K| |x|, the atol above) is 1e-5 of r_j: q agrees to 1e-4 of itself
    assert abs(q - q_o) < 1e-4 * q_o
    S.close()
