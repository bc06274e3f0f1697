"""Failure detection through the C ABI, made on the host (no GPU fault, trap or hang): the
iteration limit, non-finite right-hand sides, a smoother whose Chebyshev interval is cut below the
spectrum (eig_safety 0.3: Algorithm 2's lambda_max estimate times 0.3), and one failing member of
a batch.  Each case checks the status, the error text, and that the context solves afterwards.
The stopping protocol follows Sec. 4.1 (iteration limit, residual reduction)."""
import math

import pytest

import workloads as W
from parity_cases import CASES, gpu_solver

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STOKES_ENOTCONV, STOKES_EBREAKDOWN = 4, 5
CASE = CASES["3d_q2_pert"]
SM = dict(kA=1, kS=1, m=2, schur_diag="d")


def _rhs(S, seed=8):
    f = torch.as_tensor(W.fourier_forcing(3, 2, CASE["n"], seed=seed).reshape(-1), device="cuda")
    return S.mass_rhs(f)


def test_enotconv_on_iteration_limit_then_usable():
    from paper_2205_15770_gb300 import StokesError
    S = gpu_solver(CASE, **SM)
    b = _rhs(S)
    with pytest.raises(StokesError) as e:
        S.solve(b, rtol=1e-12, maxit=1)
    assert e.value.status == STOKES_ENOTCONV
    assert "maxit" in str(e.value)
    _, its, rel = S.solve(b, rtol=1e-10)
    assert rel <= 1e-10 and its > 1
    S.close()


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_ebreakdown_on_non_finite_rhs_then_usable(bad):
    from paper_2205_15770_gb300 import StokesError
    S = gpu_solver(CASE, **SM)
    b = _rhs(S)
    bh = b.cpu().numpy().copy()
    bh[7] = bad  # planted on the host before the call
    with pytest.raises(StokesError) as e:
        S.solve(torch.as_tensor(bh, device="cuda"), rtol=1e-10)
    assert e.value.status == STOKES_EBREAKDOWN
    assert "not finite" in str(e.value)
    _, its, rel = S.solve(b, rtol=1e-10)
    assert rel <= 1e-10
    S.close()


def test_diverging_smoother_is_reported():
    """lambda_max taken at 0.3 x its estimate: the Chebyshev smoother amplifies the upper part of
    the spectrum and the stationary multigrid iteration grows past 1e6 r0 (EBREAKDOWN).  FGMRES
    around the same cycle stays bounded (it minimises the residual over its Krylov space): it
    either converges or stops at the iteration limit."""
    from paper_2205_15770_gb300 import StokesError
    S = gpu_solver(CASE, eig_safety=0.3, **SM)
    b = _rhs(S)
    with pytest.raises(StokesError) as e:
        S.mg_iterate(b, max_iter=15, reduction=1e-10)
    assert e.value.status == STOKES_EBREAKDOWN
    assert "diverged" in str(e.value)
    try:
        _, its, rel = S.solve(b, rtol=1e-8, maxit=20)
        assert rel <= 1e-8
    except StokesError as err:
        assert err.status in (STOKES_ENOTCONV, STOKES_EBREAKDOWN), err
    S.close()
    ok = gpu_solver(CASE, **SM)
    _, its, rel = ok.solve(_rhs(ok), rtol=1e-10)
    assert rel <= 1e-10
    ok.close()


def test_batch_member_failure_leaves_the_others_converged():
    from paper_2205_15770_gb300 import StokesBatch
    members = [dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=0.0),
               dict(dim=3, n=(8, 8, 8), n_levels=3, gamma_rho=1e3),
               dict(dim=3, n=(6, 6, 6), n_levels=2, gamma_rho=10.0)]
    Bt = StokesBatch(members, **SM)
    bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=30 + i).reshape(-1), device="cuda"))
          for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    bad = bs[1].cpu().numpy().copy()
    bad[11] = float("nan")
    xs, its, rels, st = Bt.solve([bs[0], torch.as_tensor(bad, device="cuda"), bs[2]], rtol=1e-10, check=False)
    assert st == STOKES_EBREAKDOWN
    assert "breakdown" in Bt.last_error
    assert rels[0] <= 1e-10 and rels[2] <= 1e-10
    assert not math.isfinite(rels[1])
    xs, its, rels = Bt.solve(bs, rtol=1e-10)  # usable afterwards
    assert max(rels) <= 1e-10
    Bt.close()
