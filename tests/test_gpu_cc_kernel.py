"""Cell-component kernel (launch shape 5: one thread per cell and velocity component) against the
CPU oracle and against the column kernel, through the C ABI.

Shape 5 is forced on every level of both precisions; levels it does not serve (FP64 trilinear,
k = 4, 2D) fall back to the column kernel, which the same checks then cover.  Cases: trilinear
Q2 (Sec. 2 cell map, the geometry shared through shared memory), Cartesian Q2 and Q3 (the
Kronecker form of Sec. 3.1's element action), a ragged single-level mesh whose cell count is not a
multiple of the 10 cells of a warp, the channel with a do-nothing outflow, and per-cell viscosity.
Tolerances as in test_gpu_parity: FP64 operator 1e-12, FP32 operator 2e-5 (max-norm relative).
"""
import numpy as np
import pytest

from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CC_CASES = ["3d_q2_pert", "3d_q2_single", "3d_q3_cart", "3d_q2_channel"]


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


_cache = {}


def _setup(name, mu_cell=None):
    key = (name, mu_cell is not None)
    if key not in _cache:
        from oracle.assemble import assemble
        case = CASES[name]
        H = oracle_hierarchy(case)
        lev = H.levels[-1]
        ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0), mu_cell=mu_cell)
        kw = {} if mu_cell is None else {"mu_cell": mu_cell}
        S = gpu_solver(case, **kw)
        for prec in (32, 64):
            for l in range(case["levels"]):
                S.set_launch_shape(l, 5, precision=prec)
        _cache[key] = (case, H, ops, S)
    return _cache[key]


@pytest.mark.parametrize("name", CC_CASES)
def test_shape5_vmult_fp64(name):
    case, H, ops, S = _setup(name)
    assert S.launch_shapes(64)[-1] == 5
    x = random_full(H.levels[-1], 31)
    y = _n(S.vmult(_t(x)))
    assert rel_err(y, ops["K"] @ x) < 1e-12


@pytest.mark.parametrize("name", CC_CASES)
def test_shape5_vmult_fp32(name):
    case, H, ops, S = _setup(name)
    x = random_full(H.levels[-1], 32)
    y = _n(S.vmult(_t(x, torch.float32)))
    assert rel_err(y, ops["K"] @ x.astype(np.float32).astype(np.float64)) < 2e-5


@pytest.mark.parametrize("name", CC_CASES)
@pytest.mark.parametrize("prec", [32, 64])
def test_shape5_blocks(name, prec):
    case, H, ops, S = _setup(name)
    lev = H.levels[-1]
    dt = torch.float32 if prec == 32 else torch.float64
    tol = 2e-5 if prec == 32 else 1e-12
    rng = np.random.default_rng(5)
    u = rng.standard_normal(lev.n_u)
    u[ops["umask"]] = 0.0
    p = rng.standard_normal(lev.n_p)
    if prec == 32:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    free = ~ops["umask"]
    A, B = ops["A"], ops["B"]
    yu, _ = S.apply_blocks(1, u=_t(u, dt))
    assert rel_err(_n(yu)[free], (A @ u)[free]) < tol
    assert np.all(_n(yu)[~free] == 0)
    yu, _ = S.apply_blocks(2, p=_t(p, dt))
    assert rel_err(_n(yu), B.T @ p) < tol
    _, yp = S.apply_blocks(4, u=_t(u, dt))
    assert rel_err(_n(yp), B @ u) < tol
    yu, _ = S.apply_blocks(3, u=_t(u, dt), p=_t(p, dt))
    ref = A @ u + B.T @ p
    assert rel_err(_n(yu)[free], ref[free]) < tol


def test_shape5_per_cell_viscosity():
    import workloads as W
    case = CASES["3d_q3_cart"]
    mu = np.exp(W.gaussian_field_cells(case["n"][0], seed=2)).reshape(-1)
    case_, H, ops, S = _setup("3d_q3_cart", mu_cell=mu)
    x = random_full(H.levels[-1], 33)
    assert rel_err(_n(S.vmult(_t(x))), ops["K"] @ x) < 1e-12
    assert rel_err(_n(S.vmult(_t(x, torch.float32))), ops["K"] @ x.astype(np.float32).astype(np.float64)) < 2e-5


@pytest.mark.parametrize("n,levels,pert", [((32, 32, 32), 4, True), ((24, 16, 8), 3, False)])
def test_shape5_matches_column_kernel_fp32(n, levels, pert):
    """Full-size check of the FP32 kernel against the column kernel (the workload's 32^3 perturbed
    mesh, and a Cartesian box), each output within FP32 rounding of the other."""
    import workloads as W
    from paper_2205_15770_gb300 import StokesMG
    V = W.perturbed_vertices(3, n, seed=0) if pert else None
    S = StokesMG(dim=3, n=n, n_levels=levels, k=2, vertices=V, gamma_rho=100.0)
    x = torch.as_tensor(W.random_vector(S.size(), 7), dtype=torch.float32, device="cuda")
    out = {}
    for shape in (4, 5):
        S.set_launch_shape(levels - 1, shape, precision=32)
        out[shape] = _n(S.vmult(x))
    assert rel_err(out[5], out[4]) < 2e-5
    S.close()


def test_shape5_solve_reaches_fp64_tolerance():
    """FGMRES with the FP32 V-cycle running the cell-component kernel on every level: the FP64
    residual under the oracle's assembled K reaches the requested 1e-10."""
    from oracle.assemble import load_vector_nodal
    import workloads as W
    case = CASES["3d_q2_pert"]
    H = oracle_hierarchy(case)
    from oracle.mg import Multigrid
    mg = Multigrid(H, gamma_rho=case["gamma_rho"], kA=1, kS=1, m=2, schur_diag="d")
    S = gpu_solver(case, kA=1, kS=1, m=2, schur_diag="d")
    for prec in (32, 64):
        for l in range(case["levels"]):
            S.set_launch_shape(l, 5, precision=prec)
    lev = H.levels[-1]
    b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(3, 2, case["n"], seed=3).reshape(-1))
    x, its, rel = S.solve(_t(b), rtol=1e-10)
    xs = _n(x)
    assert np.linalg.norm(b - mg.K @ xs) <= 1.01e-10 * np.linalg.norm(b)
    assert its <= 12
    S.close()
