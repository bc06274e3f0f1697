"""Symmetric-gradient form a(u,v) = int mu eps(u):eps(v) + gamma rho u.v (Sec. 2) with per-cell mu and
rho on the GPU against the CPU oracle.  Tolerances as in test_gpu_parity: FP64 operator and setup
diagonals 1e-12, FP32 operator 2e-5, FP64 smoothing and cycles 1e-10, solves 1e-10 residual."""
import numpy as np
import pytest

import workloads as W
from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


def _coeffs(case, seed):
    """Per-cell coefficient on every level, coarse first (coarse = mean of the 2^d children)."""
    dim, n, L = case["dim"], case["n"], case["levels"]
    rng = np.random.default_rng(seed)
    fine = np.exp(0.5 * rng.standard_normal(int(np.prod(n[:dim]))))
    out = [fine]
    for l in range(1, L):
        m = out[0].reshape(tuple(c // 2 ** (l - 1) for c in n[:dim])[::-1])
        sh = []
        for c in m.shape:
            sh += [c // 2, 2]
        out.insert(0, m.reshape(sh).mean(axis=tuple(range(1, 2 * dim, 2))).reshape(-1))
    return out


def _pair(name, sym=True, rho=True, mu=True, **kw):
    from oracle.mg import Multigrid
    case = CASES[name]
    H = oracle_hierarchy(case)
    mus = _coeffs(case, 1) if mu else None
    rhos = _coeffs(case, 2) if rho else None
    g = case.get("gamma_rho", 0.0) or 5.0
    mg = Multigrid(H, mu=case.get("mu", 1.0), gamma_rho=g, mu_cells=mus, rho_cells=rhos, sym=sym, **kw) \
        if case["levels"] > 1 else None
    S = gpu_solver(dict(case, gamma_rho=g), sym_grad=sym, mu_cell=None if mus is None else mus[-1],
                   rho_cell=None if rhos is None else rhos[-1],
                   **{k2: v for k2, v in kw.items() if k2 in ("kA", "kS", "m", "cycle", "schur_diag")})
    return case, H, mg, S, g, mus, rhos


@pytest.mark.parametrize("name", ["2d_q2_ragged", "2d_q3_pert", "3d_q2_pert", "3d_q3_cart", "3d_q2_single"])
@pytest.mark.parametrize("sym,rho", [(True, True), (True, False), (False, True)])
def test_operator(name, sym, rho):
    from oracle.assemble import assemble
    case, H, mg, S, g, mus, rhos = _pair(name, sym=sym, rho=rho)
    lev = H.levels[-1]
    ops = assemble(lev, case.get("mu", 1.0), g, mus[-1], rho_cell=None if rhos is None else rhos[-1], sym=sym)
    x = random_full(lev, 3)
    assert rel_err(_n(S.vmult(_t(x))), ops["K"] @ x) < 1e-12
    assert rel_err(_n(S.vmult(_t(x, torch.float32))), ops["K"] @ x) < 2e-5
    yu, _ = S.apply_blocks(1, u=_t(x[: lev.n_u]))
    assert rel_err(_n(yu), (ops["A"] @ x[: lev.n_u]) * ~ops["umask"]) < 1e-12


@pytest.mark.parametrize("diag", ["loc", "p", "d"])
def test_setup_diagonals(diag):
    case, H, mg, S, g, _, _ = _pair("3d_q2_pert", kA=1, kS=2, schur_diag=diag)
    for l in range(1, len(H.levels)):
        sm = mg.smoothers[l]
        DA, DS = S.diagonals(l)
        assert rel_err(_n(DA), sm.DA) < 1e-12
        assert rel_err(_n(DS), sm.DS) < 1e-12
        assert abs(S.level_params(l)["beta_A"] - sm.beta_A) < 1e-9 * sm.beta_A


@pytest.mark.parametrize("name", ["2d_q3_pert", "3d_q2_pert", "3d_q2_channel"])
def test_smoothing_and_cycles(name):
    case, H, mg, S, g, _, _ = _pair(name, kA=1, kS=2, m=2)
    assert not any(S.fused_levels(32))
    l = len(H.levels) - 1
    lev = H.levels[l]
    b = random_full(lev, 6, constrained_zero=True)
    x0 = random_full(lev, 7, constrained_zero=True)
    xg = _t(x0)
    S.smooth(_t(b), xg, steps=2)
    assert rel_err(_n(xg), mg.smoothers[l].smooth(x0.copy(), b, 2)) < 1e-10
    ref = mg.cycle(l, x0.copy(), b)
    assert rel_err(_n(S.vcycle(_t(b), _t(x0))), ref) < 1e-10
    assert rel_err(_n(S.vcycle(_t(b, torch.float32), _t(x0, torch.float32))), ref) < 1e-3


@pytest.mark.parametrize("fp32", [True, False])
def test_solve_matches_direct_solution(fp32):
    import scipy.sparse.linalg as spla
    from oracle.assemble import load_vector_nodal
    case, H, mg, S, g, _, _ = _pair("3d_q2_pert", kA=1, kS=2, m=2)
    S = gpu_solver(dict(case, gamma_rho=g), sym_grad=True, mu_cell=_coeffs(case, 1)[-1],
                   rho_cell=_coeffs(case, 2)[-1], kA=1, kS=2, m=2, vcycle_fp32=fp32)
    lev = H.levels[-1]
    K = mg.K
    b = load_vector_nodal(lev, mg.ops[-1], W.fourier_forcing(3, 2, case["n"], seed=1).reshape(-1))
    x, its, rel = S.solve(_t(b), rtol=1e-10)
    x = _n(x)
    assert np.linalg.norm(b - K @ x) <= 1.01e-10 * np.linalg.norm(b)
    r = lev.n_u
    keep = np.r_[0:r, r + 1:lev.size]
    xd = np.insert(spla.spsolve(K.tocsc()[keep][:, keep], b[keep]), r, 0.0)
    xd[lev.n_u:] -= xd[lev.n_u:].mean()
    assert rel_err(x, xd) < 1e-7


def test_viscosity_gradient_is_for_the_laplacian_form():
    from paper_2205_15770_gb300 import StokesError
    case, H, mg, S, g, _, _ = _pair("3d_q2_single")
    x = torch.zeros(S.size(), dtype=torch.float64, device="cuda")
    with pytest.raises(StokesError):
        S.cell_grad(x, x)
