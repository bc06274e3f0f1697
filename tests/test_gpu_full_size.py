"""Parity at the benchmark's full size: the 32^3 perturbed Q2-Q1 workload (859,812 DoFs, 5 levels,
smooth trilinear perturbation 0.1 h, seed 0, gamma rho in {0, 1e2, 1e4}) in the launch
configuration bench.py times (the shapes and smoother forms the setup's timing picks).  The oracle
computes sampled rows of K x one by one (oracle.sampled: cell element matrices by plain
quadrature); the solve is checked by properties that hold at any size."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_CELLS = (32, 32, 32)
K = 2


def _level():
    from oracle.mesh import Level
    return Level(3, K, N_CELLS, W.perturbed_vertices(3, N_CELLS, seed=0, amplitude=0.1), dirichlet_faces=0x3F)


def _solver(gamma):
    import bench
    from paper_2205_15770_gb300 import StokesMG
    wl = bench.WL
    return StokesMG(dim=3, n=N_CELLS, n_levels=wl["levels"], k=K,
                    vertices=W.perturbed_vertices(3, N_CELLS, seed=0, amplitude=0.1), gamma_rho=gamma, kA=wl["kA"],
                    kS=wl["kS"], m=wl["m"], schur_diag=wl["schur_diag"], restart=wl["restart"])


def _rows(lev, n_random=600, seed=0):
    """Random rows plus rows chosen by position: the first and last velocity nodes of each
    component, nodes on, next to and at the corners of the Dirichlet boundary, and pressure
    nodes at corners, on faces and inside."""
    Nv = [K * n + 1 for n in N_CELLS]
    Np = [(K - 1) * n + 1 for n in N_CELLS]
    nv = Nv[0] * Nv[1] * Nv[2]
    vel = lambda c, x, y, z: c * nv + x + Nv[0] * (y + Nv[1] * z)
    pre = lambda x, y, z: lev.n_u + x + Np[0] * (y + Np[1] * z)
    rows = set(np.random.default_rng(seed).choice(lev.size, n_random, replace=False).tolist())
    e = Nv[0] - 1
    for c in range(3):
        for (x, y, z) in [(0, 0, 0), (e, e, e), (1, 1, 1), (e - 1, 1, e - 1), (1, e // 2, e // 2), (0, 5, 7),
                          (e // 2, e // 2, e // 2), (2, 2, 2), (e - 2, 3, 1), (1, e - 1, e // 3)]:
            rows.add(vel(c, x, y, z))
    pe = Np[0] - 1
    for (x, y, z) in [(0, 0, 0), (pe, pe, pe), (0, pe // 2, pe // 2), (1, 1, 1), (pe // 2, pe // 2, pe // 2), (pe, 0, 3)]:
        rows.add(pre(x, y, z))
    return np.array(sorted(rows))


@pytest.mark.parametrize("gamma", [0.0, 1e4])
def test_vmult_sampled_rows(gamma):
    from oracle.sampled import apply_rows
    lev = _level()
    S = _solver(gamma)
    assert S.size() == lev.size == 859812
    x = W.random_vector(lev.size, 11)
    rows = _rows(lev)
    y_ref = apply_rows(lev, x, rows, 1.0, gamma)
    x64 = torch.as_tensor(x, device="cuda")
    y64 = S.vmult(x64).cpu().numpy()
    y32 = S.vmult(x64.float()).double().cpu().numpy()
    scale = np.max(np.abs(y64))
    assert np.max(np.abs(y64[rows] - y_ref)) / scale < 1e-12
    assert np.max(np.abs(y32[rows] - y_ref)) / scale < 2e-5
    S.close()


def test_solve_full_size_residual_and_sampled_rows():
    """FP32-MG FGMRES solve of b = M_v f (the bench's forcing) to 1e-8: the solver's residual
    estimate, the residual recomputed through the FP64 operator, and sampled rows of b - K x
    recomputed by the oracle all meet the bound."""
    from oracle.sampled import apply_rows
    lev = _level()
    S = _solver(1e2)
    f = torch.as_tensor(W.fourier_forcing(3, K, N_CELLS, seed=0).reshape(-1), device="cuda")
    b = S.mass_rhs(f)
    x = torch.zeros_like(b)
    _, its, rel = S.solve(b, x, rtol=1e-8)
    assert rel <= 1e-8 and its <= 10
    r = b - S.vmult(x)
    bn = float(torch.linalg.norm(b))
    assert float(torch.linalg.norm(r)) / bn <= 1.05e-8
    rows = _rows(lev, n_random=300, seed=1)
    xr = x.cpu().numpy()
    r_ref = b.cpu().numpy()[rows] - apply_rows(lev, xr, rows, 1.0, 1e2)
    # entries of the residual, from the oracle's operator, are bounded by its norm
    assert np.max(np.abs(r_ref)) <= 1.05e-8 * bn + 1e-12 * np.max(np.abs(b.cpu().numpy()))
    assert np.max(np.abs(r_ref - r.cpu().numpy()[rows])) <= 1e-12 * float(torch.max(torch.abs(S.vmult(x))))
    S.close()
