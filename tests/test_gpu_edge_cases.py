"""Degenerate and boundary cases of the GPU path against the oracle: single-cell meshes (one warp
holds fewer cells than it has slots), meshes one cell thick, no Dirichlet face at all (generalized
Stokes keeps K nonsingular through gamma rho > 0), a ragged two-level hierarchy, and the
smallest right-hand sides.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

import workloads as W
from parity_cases import gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EDGE = {
    "3d_q2_one_cell_natural": dict(dim=3, k=2, n=(1, 1, 1), levels=1, faces=0, gamma_rho=1.0),
    "3d_q3_one_cell_natural": dict(dim=3, k=3, n=(1, 1, 1), levels=1, faces=0, gamma_rho=3.0, perturb=True),
    "3d_q4_one_cell_natural": dict(dim=3, k=4, n=(1, 1, 1), levels=1, faces=0, gamma_rho=1.0),
    "2d_q2_one_cell_natural": dict(dim=2, k=2, n=(1, 1), levels=1, faces=0, gamma_rho=2.0),
    "3d_q2_thin_slab": dict(dim=3, k=2, n=(1, 4, 2), levels=1, faces=0x3F & ~0x1, gamma_rho=1.0, perturb=True),
    "3d_q2_ragged_two_level": dict(dim=3, k=2, n=(4, 2, 6), levels=2, perturb=True, gamma_rho=10.0),
    "2d_q3_thin_strip": dict(dim=2, k=3, n=(1, 6), levels=1, faces=0xF & ~0x2, gamma_rho=1.0),
}


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


def _setup(name):
    from oracle.assemble import assemble
    case = EDGE[name]
    H = oracle_hierarchy(case)
    lev = H.levels[-1]
    ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))
    return case, lev, ops, gpu_solver(case, kA=1, kS=2, m=2)


@pytest.mark.parametrize("name", list(EDGE))
def test_operator_on_degenerate_meshes(name):
    case, lev, ops, S = _setup(name)
    x = random_full(lev, 5)
    assert rel_err(_n(S.vmult(_t(x))), ops["K"] @ x) < 1e-12
    assert rel_err(_n(S.vmult(_t(x, torch.float32))), ops["K"] @ x.astype(np.float32).astype(np.float64)) < 2e-5
    # blocks: constrained entries of u are ignored and constrained rows of yu are zero
    u, p = x[: lev.n_u].copy(), x[lev.n_u:]
    free = ~ops["umask"]
    u[~free] = 0.0
    yu, _ = S.apply_blocks(1, u=_t(x[: lev.n_u]))
    assert rel_err(_n(yu)[free], (ops["A"] @ u)[free]) < 1e-12
    assert np.all(_n(yu)[~free] == 0)
    _, yp = S.apply_blocks(4, u=_t(x[: lev.n_u]))
    assert rel_err(_n(yp), ops["B"] @ u) < 1e-12
    yu, _ = S.apply_blocks(2, p=_t(p))
    assert rel_err(_n(yu), ops["B"].T @ p) < 1e-12
    S.close()


@pytest.mark.parametrize("name", list(EDGE))
def test_solve_on_degenerate_meshes(name):
    import scipy.sparse.linalg as spla
    from oracle.assemble import load_vector_nodal
    case, lev, ops, S = _setup(name)
    f = W.fourier_forcing(case["dim"], case["k"], case["n"], seed=3).reshape(-1)
    b = load_vector_nodal(lev, ops, f)
    x, its, rel = S.solve(_t(b), rtol=1e-10)
    x = _n(x)
    assert np.linalg.norm(b - ops["K"] @ x) <= 1.01e-10 * np.linalg.norm(b)
    if not lev.has_pressure_kernel():
        assert rel_err(x, spla.spsolve(ops["K"].tocsc(), b)) < 1e-7
    S.close()


def test_rhs_with_a_single_nonzero_entry():
    """A unit right-hand side in one free velocity row (the smallest nonzero input) solves to the
    bound like any other."""
    case, lev, ops, S = _setup("3d_q2_ragged_two_level")
    free = np.flatnonzero(~lev.constrained())
    b = np.zeros(lev.size)
    b[free[len(free) // 3]] = 1.0
    x, its, rel = S.solve(_t(b), rtol=1e-10)
    assert np.linalg.norm(b - ops["K"] @ _n(x)) <= 1.01e-10
    S.close()
