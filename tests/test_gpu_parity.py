"""GPU (C ABI) vs CPU oracle parity, element by element, on seeded synthetic inputs.

Tolerances: FP64 operator applications 1e-12 (max-norm relative), FP64 setup
quantities 1e-12, Lanczos estimates 1e-9, one FP64 smoothing step / cycle 1e-10,
FP32 operator 2e-5 (random inputs; ~30 dependent FP32 roundings times a
|K||x|/|Kx| ratio of O(10)), FP32 cycle 1e-3 of the FP64 result.
"""
import numpy as np
import pytest

from parity_cases import CASES, gpu_solver, oracle_hierarchy, random_full, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _n(t):
    return t.detach().double().cpu().numpy()


_cache = {}


def _pair(name, **kw):
    key = (name, tuple(sorted(kw.items())))
    if key not in _cache:
        from oracle.mg import Multigrid
        case = CASES[name]
        H = oracle_hierarchy(case)
        mg = Multigrid(H, mu=case.get("mu", 1.0), gamma_rho=case.get("gamma_rho", 0.0), **kw) \
            if case["levels"] > 1 else None
        S = gpu_solver(case, **{k2: v for k2, v in kw.items() if k2 in ("kA", "kS", "m", "cycle", "schur_diag")})
        _cache[key] = (case, H, mg, S)
    return _cache[key]


def _ops(name):
    from oracle.assemble import assemble
    case, H, mg, S = _pair(name)
    if mg is not None:
        return case, H, mg.ops, S
    lev = H.levels[-1]
    return case, H, [assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))], S


@pytest.mark.parametrize("name", list(CASES))
def test_vmult_fp64(name):
    case, H, ops, S = _ops(name)
    lev = H.levels[-1]
    x = random_full(lev, 11)
    y = _n(S.vmult(_t(x)))
    assert rel_err(y, ops[-1]["K"] @ x) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_vmult_fp32(name):
    case, H, ops, S = _ops(name)
    lev = H.levels[-1]
    x = random_full(lev, 12)
    y = _n(S.vmult(_t(x, torch.float32)))
    assert rel_err(y, ops[-1]["K"] @ x.astype(np.float32).astype(np.float64)) < 2e-5


@pytest.mark.parametrize("name", ["2d_q3_pert", "3d_q2_pert", "3d_q4_pert", "3d_q2_channel"])
def test_vmult_coarser_levels(name):
    case, H, ops, S = _ops(name)
    for l in range(len(H.levels)):
        x = random_full(H.levels[l], 20 + l)
        y = _n(S.vmult(_t(x), level=l))
        assert rel_err(y, ops[l]["K"] @ x) < 1e-12, l


@pytest.mark.parametrize("name", ["2d_q2_ragged", "3d_q2_pert", "3d_q3_cart"])
def test_blocks(name):
    case, H, ops, S = _ops(name)
    lev = H.levels[-1]
    A, B = ops[-1]["A"], ops[-1]["B"]
    rng = np.random.default_rng(3)
    u = rng.standard_normal(lev.n_u)
    u[ops[-1]["umask"]] = 0.0
    p = rng.standard_normal(lev.n_p)
    free = ~ops[-1]["umask"]
    yu, _ = S.apply_blocks(1, u=_t(u))
    assert rel_err(_n(yu)[free], (A @ u)[free]) < 1e-12
    assert np.all(_n(yu)[~free] == 0)
    yu, _ = S.apply_blocks(2, p=_t(p))
    assert rel_err(_n(yu), B.T @ p) < 1e-12
    _, yp = S.apply_blocks(4, u=_t(u))
    assert rel_err(_n(yp), B @ u) < 1e-12


@pytest.mark.parametrize("name", ["2d_q2_cart", "3d_q2_pert", "3d_q4_pert"])
def test_mass_rhs(name):
    from oracle.assemble import load_vector_nodal
    import workloads as W
    case, H, ops, S = _ops(name)
    lev = H.levels[-1]
    f = W.fourier_forcing(case["dim"], case["k"], case["n"], seed=4).reshape(-1)
    b = _n(S.mass_rhs(_t(f)))
    assert rel_err(b, load_vector_nodal(lev, ops[-1], f)) < 1e-12


@pytest.mark.parametrize("name", ["2d_q3_pert", "3d_q2_pert", "3d_q4_pert", "3d_q2_channel"])
def test_setup_diagonals_and_eigen_estimates(name):
    case, H, mg, S = _pair(name)
    for l in range(1, len(H.levels)):
        sm = mg.smoothers[l]
        DA, DS = S.diagonals(l)
        assert rel_err(_n(DA), sm.DA) < 1e-12
        assert rel_err(_n(DS), sm.DS) < 1e-12
        prm = S.level_params(l)
        assert abs(prm["beta_A"] - sm.beta_A) < 1e-9 * sm.beta_A
        assert abs(prm["beta_S"] - sm.beta_S) < 1e-9 * sm.beta_S
        assert prm["sigma"] == pytest.approx(sm.sigma, rel=1e-15)
        assert prm["tau"] == pytest.approx(sm.tau, rel=1e-15)


def test_pressure_mass_schur_diagonal():
    case, H, mg, S = _pair("3d_q2_pert", schur_diag="p")
    DA, DS = S.diagonals(len(H.levels) - 1)
    assert rel_err(_n(DS), mg.ops[-1]["Mp"].diagonal()) < 1e-12


@pytest.mark.parametrize("name", ["2d_q3_pert", "3d_q2_pert", "3d_q3_cart", "3d_q2_channel"])
def test_schur_diagonal_d(name):
    # Eq. diag d: D = diag(B diag(A)^-1 B^T), probed through the matrix-free B on the GPU
    case, H, mg, S = _pair(name, schur_diag="d", kA=1, kS=2)
    for l in range(1, len(H.levels)):
        sm = mg.smoothers[l]
        DA, DS = S.diagonals(l)
        assert rel_err(_n(DS), sm.DS) < 1e-12
        assert abs(S.level_params(l)["beta_S"] - sm.beta_S) < 1e-9 * sm.beta_S
    lev = H.levels[-1]
    b = random_full(lev, 17, constrained_zero=True)
    ref = mg.cycle(len(H.levels) - 1, np.zeros(lev.size), b)
    assert rel_err(_n(S.vcycle(_t(b))), ref) < 1e-10


@pytest.mark.parametrize("name", ["2d_q3_pert", "3d_q2_pert", "3d_q2_channel"])
@pytest.mark.parametrize("kA", [1, 3])
def test_schur_diagonal_exact(name, kA):
    # the exact diagonal of S~ = B A^-1_hat B^T, probed through S~ on the GPU, against the oracle's
    # dense A^-1_hat on the coarser level (the oracle's beta_A set to the GPU's Lanczos value)
    from oracle.assemble import assemble
    from oracle.smoother import LevelSmoother
    case = CASES[name]
    H = oracle_hierarchy(case)
    S = gpu_solver(case, schur_diag="exact", kA=kA, kS=2)
    lev = H.levels[1]
    ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))
    prm = S.level_params(1)
    sm = LevelSmoother(lev, ops, kA, 2, schur_diag="exact", mu=case.get("mu", 1.0),
                       gamma_rho=case.get("gamma_rho", 0.0), beta_A=prm["beta_A"], beta_S=1.0)
    DA, DS = S.diagonals(1)
    assert rel_err(_n(DS), sm.DS) < 1e-12


def test_schur_diagonal_exact_rejects_large_meshes():
    from paper_2205_15770_gb300 import StokesError, StokesMG
    with pytest.raises(StokesError) as e:
        # k = 4, k_A = 3: probe period 19 pressure nodes, 37 nodes per axis on the 12^3 level
        StokesMG(dim=3, n=(12, 12, 12), n_levels=2, k=4, schur_diag="exact", kA=3, kS=1)
    assert "small meshes" in str(e.value)


@pytest.mark.parametrize("name", ["2d_q2_cart", "2d_q3_pert", "3d_q2_pert", "3d_q4_pert", "3d_q2_channel"])
def test_transfers(name):
    case, H, mg, S = _pair(name)
    for l in range(1, len(H.levels)):
        P = mg.P[l]
        xf = random_full(H.levels[l], 30 + l, constrained_zero=True)
        xc = random_full(H.levels[l - 1], 40 + l, constrained_zero=True)
        assert rel_err(_n(S.restrict(_t(xf), l)), P.T @ xf) < 1e-13
        assert rel_err(_n(S.prolongate(_t(xc), l)), P @ xc) < 1e-13


@pytest.mark.parametrize("name", ["2d_q2_cart", "3d_q2_pert", "3d_q4_pert", "3d_q2_channel"])
def test_coarse_solve(name):
    case, H, mg, S = _pair(name)
    lev0 = H.levels[0]
    b = random_full(lev0, 5, constrained_zero=True)
    x = _n(S.coarse_solve(_t(b)))
    assert rel_err(x, mg.coarse.solve(b)) < 1e-10


@pytest.mark.parametrize("name", ["2d_q2_ragged", "2d_q3_pert", "3d_q2_pert", "3d_q2_channel"])
def test_smoother_steps_fp64(name):
    case, H, mg, S = _pair(name)
    l = len(H.levels) - 1
    lev = H.levels[l]
    b = random_full(lev, 6, constrained_zero=True)
    x0 = random_full(lev, 7, constrained_zero=True)
    ref = mg.smoothers[l].smooth(x0.copy(), b, 2)
    xg = _t(x0)
    S.smooth(_t(b), xg, steps=2)
    assert rel_err(_n(xg), ref) < 1e-10


@pytest.mark.parametrize("name", ["2d_q2_cart", "2d_q4_pert", "3d_q2_pert", "3d_q3_cart", "3d_q2_channel"])
def test_vcycle_fp64_and_fp32(name):
    case, H, mg, S = _pair(name)
    lev = H.levels[-1]
    b = random_full(lev, 8, constrained_zero=True)
    x0 = random_full(lev, 9, constrained_zero=True)
    ref = mg.cycle(len(H.levels) - 1, x0.copy(), b)
    xg = S.vcycle(_t(b), _t(x0))
    assert rel_err(_n(xg), ref) < 1e-10
    xg32 = S.vcycle(_t(b, torch.float32), _t(x0, torch.float32))
    assert rel_err(_n(xg32), ref) < 1e-3
    # the captured graph is replayed: a second call gives the same result
    xg2 = S.vcycle(_t(b), _t(x0))
    assert rel_err(_n(xg2), ref) < 1e-10


def test_wcycle_fp64():
    case, H, mg, S = _pair("2d_q3_pert", cycle="W", kA=1, kS=2, m=1)
    lev = H.levels[-1]
    b = random_full(lev, 10, constrained_zero=True)
    ref = mg.cycle(len(H.levels) - 1, np.zeros(lev.size), b)
    assert rel_err(_n(S.vcycle(_t(b))), ref) < 1e-10


@pytest.mark.parametrize("name", ["2d_q2_cart", "3d_q2_pert", "3d_q2_channel", "3d_q2_single"])
@pytest.mark.parametrize("fp32", [True, False])
def test_solve_matches_direct_solution(name, fp32):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import workloads as W
    from oracle.assemble import assemble, load_vector_nodal
    case = CASES[name]
    H = oracle_hierarchy(case)
    lev = H.levels[-1]
    ops = assemble(lev, case.get("mu", 1.0), case.get("gamma_rho", 0.0))
    S = gpu_solver(case, vcycle_fp32=fp32)
    f = W.fourier_forcing(case["dim"], case["k"], case["n"], seed=1).reshape(-1)
    b = load_vector_nodal(lev, ops, f)
    x, its, rel = S.solve(_t(b), rtol=1e-10)
    x = _n(x)
    K = ops["K"]
    assert np.linalg.norm(b - K @ x) <= 1.01e-10 * np.linalg.norm(b)
    if lev.has_pressure_kernel():
        e = np.concatenate([np.zeros(lev.n_u), np.ones(lev.n_p)])
        Kb = sp.bmat([[K, sp.csr_matrix(e[:, None])], [sp.csr_matrix(e[None, :]), None]], format="csc")
        xd = spla.spsolve(Kb, np.concatenate([b, [0.0]]))[:-1]
        assert abs(x[lev.n_u:].mean()) < 1e-12 * np.abs(x).max()
    else:
        xd = spla.spsolve(K.tocsc(), b)
    # forward error <= cond(K) * backward error; the seeded cases stay below 1e-7
    assert rel_err(x, xd) < 1e-7
    assert its <= 30


def test_zero_rhs_returns_zero():
    case, H, mg, S = _pair("2d_q2_cart")
    b = torch.zeros(S.size(), dtype=torch.float64, device="cuda")
    x, its, rel = S.solve(b)
    assert its == 0 and rel == 0.0 and torch.count_nonzero(x).item() == 0


def test_point_and_column_kernels_agree(tmp_path):
    # The 3D operator runs in the column kernel by default; STOKES_GENERIC_KERNEL=1 selects the
    # point-per-thread kernel.  Both must give the same FP64 result to rounding.
    import subprocess
    import sys
    import os
    case = CASES["3d_q2_pert"]
    H = oracle_hierarchy(case)
    lev = H.levels[-1]
    x = random_full(lev, 99)
    np.save(tmp_path / "x.npy", x)
    code = (
        "import sys, numpy as np, torch; sys.path.insert(0, %r); sys.path.insert(0, %r)\n"
        "from parity_cases import CASES, gpu_solver\n"
        "S = gpu_solver(CASES['3d_q2_pert'])\n"
        "x = torch.as_tensor(np.load(%r), device='cuda')\n"
        "np.save(%r, S.vmult(x).cpu().numpy())\n"
        "np.save(%r, S.vmult(x.float()).double().cpu().numpy())\n"
    ) % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), os.path.dirname(os.path.abspath(__file__)),
         str(tmp_path / "x.npy"), str(tmp_path / "y64.npy"), str(tmp_path / "y32.npy"))
    env = dict(os.environ, STOKES_GENERIC_KERNEL="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    _, _, _, S = _pair("3d_q2_pert")
    y_col = _n(S.vmult(_t(x)))
    y_pt = np.load(tmp_path / "y64.npy")
    assert rel_err(y_col, y_pt) < 1e-13
    y_col32 = _n(S.vmult(_t(x, torch.float32)))
    assert rel_err(y_col32, np.load(tmp_path / "y32.npy")) < 2e-6
