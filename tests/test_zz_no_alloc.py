"""The allocation-free smoothing entry point (stokes_smooth_noalloc) against stokes_smooth.

stokes_smooth_noalloc serves callers that cannot allocate device memory where they call it (under
stream capture, in real-time loops, or when their own allocator owns the device memory): the
smoother's work vectors live in a static device array of the library instead of the context.
This file is collected last on purpose; it runs the same way alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W
from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
@pytest.mark.parametrize("kA,kS", [(3, 3), (1, 2)])  # (1, 2): the fused smoother
def test_noalloc_smoothing_matches_stokes_smooth_on_two_calls(monkeypatch, dtype, tol, kA, kS):
    case = CASES["3d_q2_pert"]
    H = oracle_hierarchy(case)
    if kA == 1:
        # no setup timing: the fused form is kept wherever eligible, so the fused path is the one run
        monkeypatch.setenv("STOKES_NO_AUTOTUNE", "1")
    S = gpu_solver(case, kA=kA, kS=kS)
    level = len(H.levels) - 1
    prec = 64 if dtype == torch.float64 else 32
    assert S.fused_levels(prec)[level] == (kA == 1)
    lev = H.levels[level]
    b = _t(random_full(lev, 21, constrained_zero=True), dtype)
    x0 = _t(random_full(lev, 22, constrained_zero=True), dtype)
    x_ref = x0.clone()
    x_na = x0.clone()
    for call in range(2):
        S.smooth(b, x_ref, steps=1, level=level)
        S.smooth_noalloc(b, x_na, steps=1, level=level)
        torch.cuda.synchronize()
        err = rel_err(x_na.double().cpu().numpy(), x_ref.double().cpu().numpy())
        assert err < tol, (call, err)


def test_noalloc_rejects_levels_beyond_the_static_scratch():
    from paper_2205_15770_gb300 import StokesError, StokesMG
    S = StokesMG(dim=3, n=(32, 32, 32), n_levels=3, k=2)
    # finest level (823,875 velocity DoFs, FP64): 11 + 6 work vectors need ~72 MB > 16 MiB
    b = torch.zeros(S.size(2), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(StokesError) as e:
        S.smooth_noalloc(b, x, steps=1, level=2)
    assert "static scratch" in str(e.value)
    # the 16^3 level fits (~9.7 MB) and agrees with stokes_smooth
    bc = torch.as_tensor(W.random_vector(S.size(1), 3), device="cuda")
    x1 = torch.zeros_like(bc)
    x2 = torch.zeros_like(bc)
    S.smooth(bc, x1, steps=2, level=1)
    S.smooth_noalloc(bc, x2, steps=2, level=1)
    assert rel_err(x2.cpu().numpy(), x1.cpu().numpy()) < 1e-12
