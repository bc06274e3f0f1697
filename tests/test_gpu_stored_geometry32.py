"""FP32 column kernels reading the per-point geometry stored at setup (3D trilinear levels of at
most 32^3 cells; a plain setup keeps it on a level where its timing of the column kernel is faster
that way): the FP32 operator, its blocks, fused and unfused cycles against the CPU oracle with the
stored geometry pinned on every level through STOKES_TUNING's g32 list, for each column launch
shape, and the on-the-fly and stored forms against each other.

Tolerances as in test_gpu_parity: FP32 operator 2e-5, FP32 cycles 1e-3 of the FP64 oracle.
"""
import numpy as np
import pytest

from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TRILINEAR = ["3d_q2_pert", "3d_q4_pert", "3d_q2_single"]


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


def _tuning(nl, shape, fused, g32):
    """STOKES_TUNING value: the same column shape on every level, fused smoothing (or not) above the
    coarsest level, the stored FP32 geometry on every level (or none)."""
    j = lambda v: ",".join(str(v) for _ in range(nl))
    f32 = ",".join(["0"] + [str(int(fused))] * (nl - 1))
    return f"s32={j(shape)};s64={j(4)};f32={f32};f64={j(0)};g32={j(int(g32))}"


def _solver(monkeypatch, case, shape, g32, fused=False, **kw):
    monkeypatch.setenv("STOKES_TUNING", _tuning(case["levels"], shape, fused, g32))
    S = gpu_solver(case, **kw)
    monkeypatch.delenv("STOKES_TUNING")
    assert S.geometry_stored(32) == [bool(g32)] * case["levels"]
    assert S.launch_shapes(32) == [shape] * case["levels"]
    return S


def _ops(case):
    from oracle.assemble import assemble
    H = oracle_hierarchy(case)
    return H, [assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0)) for lev in H.levels]


@pytest.mark.parametrize("shape", [1, 3, 4])
@pytest.mark.parametrize("name", TRILINEAR)
def test_vmult_fp32_stored_geometry(monkeypatch, name, shape):
    case = CASES[name]
    H, ops = _ops(case)
    S = _solver(monkeypatch, case, shape, True)
    for l in range(len(H.levels)):
        x = random_full(H.levels[l], 30 + l)
        y = _n(S.vmult(_t(x, torch.float32), level=l))
        assert rel_err(y, ops[l]["K"] @ x.astype(np.float32).astype(np.float64)) < 2e-5, l


@pytest.mark.parametrize("shape", [1, 3, 4])
def test_blocks_fp32_stored_geometry(monkeypatch, shape):
    case = CASES["3d_q2_pert"]
    H, ops = _ops(case)
    lev, o = H.levels[-1], ops[-1]
    S = _solver(monkeypatch, case, shape, True)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(lev.n_u).astype(np.float32).astype(np.float64)
    u[o["umask"]] = 0.0
    p = rng.standard_normal(lev.n_p).astype(np.float32).astype(np.float64)
    free = ~o["umask"]
    yu, _ = S.apply_blocks(1, u=_t(u, torch.float32))
    assert rel_err(_n(yu)[free], (o["A"] @ u)[free]) < 2e-5
    yu, _ = S.apply_blocks(2, p=_t(p, torch.float32))
    assert rel_err(_n(yu), o["B"].T @ p) < 2e-5
    _, yp = S.apply_blocks(4, u=_t(u, torch.float32))
    assert rel_err(_n(yp), o["B"] @ u) < 2e-5


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("shape", [1, 3, 4])
def test_cycle_fp32_stored_geometry(monkeypatch, shape, fused):
    """The benchmark's smoother ((k_A, k_S, m) = (1, 1, 2), Schur diagonal d); fused: the smoother's
    vector updates folded into the column kernel's gathers, which then read the stored geometry."""
    from oracle.mg import Multigrid
    case = CASES["3d_q2_pert"]
    kw = dict(kA=1, kS=1, m=2, schur_diag="d")
    H = oracle_hierarchy(case)
    mg = Multigrid(H, mu=case.get("mu", 1.0), gamma_rho=case.get("gamma_rho", 0.0), **kw)
    S = _solver(monkeypatch, case, shape, True, fused=fused, **kw)
    assert S.fused_levels(32)[1:] == [fused] * (case["levels"] - 1)
    lev = H.levels[-1]
    b = random_full(lev, 18, constrained_zero=True)
    x0 = random_full(lev, 19, constrained_zero=True)
    for start in (np.zeros(lev.size), x0):
        ref = mg.cycle(len(H.levels) - 1, start.copy(), b)
        x32 = S.vcycle(_t(b, torch.float32), _t(start, torch.float32))
        assert rel_err(_n(x32), ref) < 1e-3


@pytest.mark.parametrize("name", ["3d_q2_pert", "3d_q4_pert"])
def test_stored_and_on_the_fly_geometry_agree(monkeypatch, name):
    """Same arithmetic per Gauss point (the stored factors come from the same geometry routine):
    the two FP32 results differ by FP32 rounding only."""
    case = CASES[name]
    H, _ = _ops(case)
    S1 = _solver(monkeypatch, case, 4, True)
    S0 = _solver(monkeypatch, case, 4, False)
    x = _t(random_full(H.levels[-1], 40), torch.float32)
    y1, y0 = _n(S1.vmult(x)), _n(S0.vmult(x))
    assert rel_err(y1, y0) < 2e-5


def test_g32_rejected_where_nothing_is_stored(monkeypatch):
    """Cartesian levels keep no per-point geometry: asking for it is an argument error at setup."""
    case = CASES["3d_q2_channel"]
    monkeypatch.setenv("STOKES_TUNING", _tuning(case["levels"], 4, False, True))
    with pytest.raises(RuntimeError, match="g32"):
        gpu_solver(case)
