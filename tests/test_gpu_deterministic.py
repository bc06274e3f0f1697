"""Deterministic mode (opts.deterministic) through the C ABI, both forms of K x = sum_tau P_tau K_tau
P_tau^T x (Sec. 3.1) without atomic scatter: mode 1, owner-computes (each cell's local results
stored, then summed per DoF in a fixed order), and mode 2, one cooperative launch over the 8 parity
classes of cells with grid barriers between the classes and plain read-modify-write scatter.
Checked: parity with the oracle at the usual tolerances, bitwise repetition of operator
applications and of whole FP32-MG solves, and mode 2's bounded barrier wait (STOKES_ETIMEOUT when
the budget runs out, made to happen by a one-cycle budget; no GPU fault)."""
import numpy as np
import pytest

import workloads as W
from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STOKES_ETIMEOUT = 6
DET_CASES = ["3d_q2_pert", "3d_q2_single", "3d_q3_cart", "3d_q2_channel"]


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


_cache = {}


def _setup(name, mode=1):
    if (name, mode) not in _cache:
        from oracle.assemble import assemble
        case = CASES[name]
        H = oracle_hierarchy(case)
        ops = assemble(H.levels[-1], case.get("mu", 1.0), case.get("gamma_rho", 0.0))
        S = gpu_solver(case, deterministic=mode)
        assert S.launch_shapes(32) == [5] * case["levels"] and not any(S.fused_levels(32))
        _cache[(name, mode)] = (case, H, ops, S)
    return _cache[(name, mode)]


# mode 1: owner-computes (per-cell local results, per-DoF sums in a fixed order); mode 2: colour classes
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", DET_CASES)
def test_deterministic_vmult_matches_oracle(name, mode):
    case, H, ops, S = _setup(name, mode)
    x = random_full(H.levels[-1], 41)
    assert rel_err(_n(S.vmult(_t(x))), ops["K"] @ x) < 1e-12
    x32 = x.astype(np.float32).astype(np.float64)
    assert rel_err(_n(S.vmult(_t(x, torch.float32))), ops["K"] @ x32) < 2e-5


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", [32, 64])
def test_deterministic_blocks_match_oracle(prec, mode):
    case, H, ops, S = _setup("3d_q2_pert", mode)
    lev = H.levels[-1]
    dt = torch.float32 if prec == 32 else torch.float64
    tol = 2e-5 if prec == 32 else 1e-12
    rng = np.random.default_rng(6)
    u = rng.standard_normal(lev.n_u)
    u[ops["umask"]] = 0.0
    p = rng.standard_normal(lev.n_p)
    if prec == 32:
        u = u.astype(np.float32).astype(np.float64)
        p = p.astype(np.float32).astype(np.float64)
    free = ~ops["umask"]
    yu, _ = S.apply_blocks(1, u=_t(u, dt))
    assert rel_err(_n(yu)[free], (ops["A"] @ u)[free]) < tol
    yu, _ = S.apply_blocks(2, p=_t(p, dt))
    assert rel_err(_n(yu), ops["B"].T @ p) < tol
    _, yp = S.apply_blocks(4, u=_t(u, dt))
    assert rel_err(_n(yp), ops["B"] @ u) < tol


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", ["3d_q2_pert", "3d_q3_cart"])
def test_deterministic_vmults_repeat_bitwise(name, mode):
    case, H, ops, S = _setup(name, mode)
    for dt in (torch.float32, torch.float64):
        x = _t(random_full(H.levels[-1], 42), dt)
        y1 = S.vmult(x).clone()
        y2 = S.vmult(x).clone()
        assert torch.equal(y1, y2)


@pytest.mark.parametrize("mode", [1, 2])
def test_deterministic_solves_repeat_bitwise_and_reach_the_oracle_residual(mode):
    from oracle.assemble import load_vector_nodal
    from oracle.mg import Multigrid
    case = CASES["3d_q2_pert"]
    H = oracle_hierarchy(case)
    mg = Multigrid(H, gamma_rho=case["gamma_rho"], kA=1, kS=1, m=2, schur_diag="d")
    lev = H.levels[-1]
    b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(3, 2, case["n"], seed=5).reshape(-1))
    bt = _t(b)
    xs = []
    for _ in range(2):  # two contexts: setup (diagonals, Lanczos, coarse matrix) is reproducible too
        S = gpu_solver(case, kA=1, kS=1, m=2, schur_diag="d", deterministic=mode)
        for _ in range(2):
            x, its, rel = S.solve(bt, rtol=1e-10)
            xs.append((x.clone(), its))
        S.close()
    for x, its in xs[1:]:
        assert its == xs[0][1]
        assert torch.equal(x, xs[0][0])
    x0 = _n(xs[0][0])
    assert np.linalg.norm(b - mg.K @ x0) <= 1.01e-10 * np.linalg.norm(b)


def test_barrier_budget_expiry_returns_etimeout_and_the_context_recovers():
    from paper_2205_15770_gb300 import StokesError
    case, H, ops, _ = _setup("3d_q2_pert", 2)
    S = gpu_solver(case, deterministic=2, wait_cycles=1)
    x = _t(random_full(H.levels[-1], 43))
    with pytest.raises(StokesError) as e:
        S.vmult(x)
    assert e.value.status == STOKES_ETIMEOUT and "budget" in str(e.value)
    b = S.mass_rhs(_t(W.fourier_forcing(3, 2, case["n"], seed=5).reshape(-1)))
    with pytest.raises(StokesError) as e:
        S.solve(b, rtol=1e-8)
    assert e.value.status == STOKES_ETIMEOUT
    S.set_wait_cycles(0)  # the default budget: the same context works again
    assert rel_err(_n(S.vmult(x)), ops["K"] @ _n(x)) < 1e-12
    S.close()
