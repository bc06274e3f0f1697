"""Fused smoothing (k_A = 1, 3D): the Chebyshev-Jacobi and Uzawa vector updates folded into the
cell-kernel gathers, against the CPU oracle and against the unfused GPU path (STOKES_NO_FUSE=1).

Tolerances as in test_gpu_parity: FP64 smoothing steps and cycles 1e-10 of the oracle, FP32
cycles 1e-3; fused vs unfused FP64 1e-12 (same arithmetic, different summation order).
"""
import numpy as np
import pytest

import workloads as W
from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FUSED_CASES = ["3d_q2_pert", "3d_q3_cart", "3d_q4_pert", "3d_q2_channel"]


@pytest.fixture(autouse=True)
def _fused_everywhere(monkeypatch):
    # without the setup's timing every eligible level keeps the fused smoother, so these tests
    # exercise it on every level whatever the timing would pick
    monkeypatch.setenv("STOKES_NO_AUTOTUNE", "1")


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


def _oracle_mg(case, **kw):
    from oracle.mg import Multigrid
    H = oracle_hierarchy(case)
    return H, Multigrid(H, mu=case.get("mu", 1.0), gamma_rho=case.get("gamma_rho", 0.0), **kw)


def _solver(case, shape, **kw):
    """gpu_solver with the launch shape pinned on every level (0: the default column kernel; 5: the
    cell-component kernel, whose fused form then runs wherever it serves the level)."""
    S = gpu_solver(case, **kw)
    if shape:
        for prec in (32, 64):
            for l in range(case["levels"]):
                S.set_launch_shape(l, shape, precision=prec)
    return S


def _unfused(monkeypatch, case, **kw):
    monkeypatch.setenv("STOKES_NO_FUSE", "1")
    S = gpu_solver(case, **kw)
    monkeypatch.delenv("STOKES_NO_FUSE")
    return S


@pytest.mark.parametrize("shape", [0, 5])
@pytest.mark.parametrize("name", FUSED_CASES)
@pytest.mark.parametrize("kS", [1, 2, 3, 4])
def test_fused_smoothing_matches_oracle(name, kS, shape):
    case = CASES[name]
    H, mg = _oracle_mg(case, kA=1, kS=kS, m=2)
    l = len(H.levels) - 1
    lev = H.levels[l]
    S = _solver(case, shape, kA=1, kS=kS, m=2)
    assert S.fused_levels(64)[l] and S.fused_levels(32)[l]
    b = random_full(lev, 6, constrained_zero=True)
    x0 = random_full(lev, 7, constrained_zero=True)
    ref = mg.smoothers[l].smooth(x0.copy(), b, 3)
    xg = _t(x0)
    S.smooth(_t(b), xg, steps=3)
    assert rel_err(_n(xg), ref) < 1e-10
    x32 = _t(x0, torch.float32)
    S.smooth(_t(b, torch.float32), x32, steps=3)
    assert rel_err(_n(x32), ref) < 1e-4


@pytest.mark.parametrize("shape", [0, 5])
@pytest.mark.parametrize("name", FUSED_CASES)
@pytest.mark.parametrize("cycle", ["V", "W"])
def test_fused_cycle_matches_oracle(name, cycle, shape):
    case = CASES[name]
    H, mg = _oracle_mg(case, kA=1, kS=2, m=2, cycle=cycle)
    lev = H.levels[-1]
    S = _solver(case, shape, kA=1, kS=2, m=2, cycle=cycle)
    b = random_full(lev, 8, constrained_zero=True)
    x0 = random_full(lev, 9, constrained_zero=True)
    for start in (np.zeros(lev.size), x0):
        ref = mg.cycle(len(H.levels) - 1, start.copy(), b)
        for _ in range(2):  # capture, then graph replay
            xg = S.vcycle(_t(b), _t(start))
            assert rel_err(_n(xg), ref) < 1e-10
        x32 = S.vcycle(_t(b, torch.float32), _t(start, torch.float32))
        assert rel_err(_n(x32), ref) < 1e-3


@pytest.mark.parametrize("name", ["3d_q2_pert", "3d_q2_channel"])
def test_fused_cycle_with_the_benchmark_smoother(name):
    """(k_A, k_S, m) = (1, 1, 2) with the Schur-complement diagonal d, the benchmark's smoother."""
    case = CASES[name]
    kw = dict(kA=1, kS=1, m=2, schur_diag="d")
    H, mg = _oracle_mg(case, **kw)
    lev = H.levels[-1]
    S = gpu_solver(case, **kw)
    b = random_full(lev, 18, constrained_zero=True)
    x0 = random_full(lev, 19, constrained_zero=True)
    for start in (np.zeros(lev.size), x0):
        ref = mg.cycle(len(H.levels) - 1, start.copy(), b)
        xg = S.vcycle(_t(b), _t(start))
        assert rel_err(_n(xg), ref) < 1e-10
        x32 = S.vcycle(_t(b, torch.float32), _t(start, torch.float32))
        assert rel_err(_n(x32), ref) < 1e-3


@pytest.mark.parametrize("name", ["3d_q2_pert", "3d_q2_channel"])
def test_fused_and_unfused_paths_agree(monkeypatch, name):
    case = CASES[name]
    lev = oracle_hierarchy(case).levels[-1]
    Sf = gpu_solver(case, kA=1, kS=2, m=2)
    Su = _unfused(monkeypatch, case, kA=1, kS=2, m=2)
    # right-hand side and start with nonzero constrained entries: both paths treat them alike
    b = _t(random_full(lev, 12))
    x0 = random_full(lev, 13)
    xf, xu = _t(x0), _t(x0)
    Sf.smooth(b, xf, steps=2)
    Su.smooth(b, xu, steps=2)
    assert rel_err(_n(xf), _n(xu)) < 1e-12
    bz = _t(random_full(lev, 14, constrained_zero=True))
    c0f, c0u = Sf.launch_count, Su.launch_count
    yf = Sf.vcycle(bz)
    yu = Su.vcycle(bz)
    assert rel_err(_n(yf), _n(yu)) < 1e-12
    # one cycle: 5 + 3 k_S launches per fused step instead of 10 + 6 k_S
    assert (Sf.launch_count - c0f) < 0.6 * (Su.launch_count - c0u)


def test_fused_every_launch_shape(monkeypatch):
    case = CASES["3d_q2_pert"]
    lev = oracle_hierarchy(case).levels[-1]
    S = gpu_solver(case, kA=1, kS=2, m=2)
    b = _t(random_full(lev, 15, constrained_zero=True))
    ref = _n(S.vcycle(b))
    for shape in (1, 3, 4, -1, 5):  # -1: point kernel, unfused smoother on that level
        for l in range(1, case["levels"]):
            S.set_launch_shape(l, shape, precision=64)
        assert rel_err(_n(S.vcycle(b)), ref) < 1e-12, shape


def test_fused_solve_and_stationary_driver():
    import scipy.sparse.linalg as spla
    from oracle.assemble import assemble, load_vector_nodal
    case = CASES["3d_q2_channel"]
    H, mg = _oracle_mg(case, kA=1, kS=2, m=2)
    lev = H.levels[-1]
    ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))
    f = W.fourier_forcing(3, 2, case["n"], seed=1).reshape(-1)
    b = load_vector_nodal(lev, ops, f)
    for fp32 in (True, False):
        S = gpu_solver(case, kA=1, kS=2, m=2, vcycle_fp32=fp32)
        x, its, rel = S.solve(_t(b), rtol=1e-10)
        assert np.linalg.norm(b - ops["K"] @ _n(x)) <= 1.01e-10 * np.linalg.norm(b)
        assert rel_err(_n(x), spla.spsolve(ops["K"].tocsc(), b)) < 1e-7
    S = gpu_solver(case, kA=1, kS=2, m=2, vcycle_fp32=False)
    x_o, res_o, q_o = mg.stationary(b)
    x, it, hist, q = S.mg_iterate(_t(b), max_iter=15, reduction=1e-10)
    assert it == len(res_o) - 1
    np.testing.assert_allclose(hist, res_o, rtol=1e-6)
    assert rel_err(_n(x), x_o) < 1e-8


def test_autotuned_fusion_choice_keeps_parity(monkeypatch):
    # the setup's timing picks fused or unfused smoothing per level; the cycle is the same either way
    monkeypatch.delenv("STOKES_NO_AUTOTUNE", raising=False)
    case = CASES["3d_q2_pert"]
    H, mg = _oracle_mg(case, kA=1, kS=2, m=2)
    lev = H.levels[-1]
    S = gpu_solver(case, kA=1, kS=2, m=2)
    for prec in (32, 64):
        fl = S.fused_levels(prec)
        assert len(fl) == case["levels"] and fl[0] is False
    b = random_full(lev, 16, constrained_zero=True)
    ref = mg.cycle(len(H.levels) - 1, np.zeros(lev.size), b)
    assert rel_err(_n(S.vcycle(_t(b))), ref) < 1e-10
    Sk = gpu_solver(case, kA=3, kS=3, m=2)  # k_A != 1: never fused
    assert not any(Sk.fused_levels(32)) and not any(Sk.fused_levels(64))
