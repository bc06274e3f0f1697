"""Batched solves of independent meshes (one graph launch per iteration for all members) and the
launch-shape autotuner, against single-mesh solves and the CPU oracle."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_batch_matches_single_solves_and_oracle_residuals():
    from oracle.assemble import assemble, load_vector_nodal
    from oracle.mesh import Hierarchy
    from paper_2205_15770_gb300 import StokesBatch, StokesMG
    members = [
        dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=0.0),
        dict(dim=3, n=(8, 8, 8), n_levels=3, gamma_rho=1e3),
        dict(dim=3, n=(6, 6, 6), n_levels=2, gamma_rho=0.0),
        dict(dim=2, n=(8, 8), n_levels=3, gamma_rho=10.0,
             vertices=W.perturbed_vertices(2, (8, 8), seed=3)),
    ]
    Bt = StokesBatch(members, kA=2, kS=2, m=2)
    bs, refs = [], []
    for i, mb in enumerate(members):
        f = W.fourier_forcing(mb["dim"], 2, mb["n"], seed=10 + i).reshape(-1)
        V = mb.get("vertices")
        H = Hierarchy(mb["dim"], 2, mb["n"], mb["n_levels"],
                      V if V is not None else W.lattice_vertices(mb["dim"], mb["n"]))
        lev = H.levels[-1]
        ops = assemble(lev, 1.0, mb["gamma_rho"])
        b = load_vector_nodal(lev, ops, f)
        bs.append(torch.as_tensor(b, device="cuda"))
        refs.append((lev, ops, b))
    xs, its, rels = Bt.solve(bs, rtol=1e-10)
    for i, mb in enumerate(members):
        lev, ops, b = refs[i]
        x = xs[i].cpu().numpy()
        assert np.linalg.norm(b - ops["K"] @ x) <= 1.01e-10 * np.linalg.norm(b), i
        S = StokesMG(dim=mb["dim"], n=mb["n"], n_levels=mb["n_levels"], gamma_rho=mb["gamma_rho"],
                     vertices=mb.get("vertices"), kA=2, kS=2, m=2)
        xs1, its1, _ = S.solve(bs[i], rtol=1e-10)
        assert its[i] == its1, (i, its, its1)
        assert np.abs(xs1.cpu().numpy() - x).max() <= 1e-8 * np.abs(x).max(), i


@pytest.mark.parametrize("host", [False, True])
def test_batch_device_krylov_loop_matches_host_loop(monkeypatch, host):
    """The batch's inner FGMRES iterations on the device (one graph launch per restart cycle, a
    conditional node per member) and host-driven: same iteration counts as single-mesh solves,
    with members of different lengths (a restart of 3 forces several cycles)."""
    from paper_2205_15770_gb300 import StokesBatch, StokesMG
    if host:
        monkeypatch.setenv("STOKES_HOST_KRYLOV", "1")
    else:
        monkeypatch.delenv("STOKES_HOST_KRYLOV", raising=False)
    members = [dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=0.0),
               dict(dim=3, n=(8, 8, 8), n_levels=3, gamma_rho=1e3),
               dict(dim=3, n=(6, 6, 6), n_levels=2, gamma_rho=10.0)]
    Bt = StokesBatch(members, kA=1, kS=1, m=2, schur_diag="d", restart=3)
    bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=20 + i).reshape(-1), device="cuda"))
          for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    xs, its, rels = Bt.solve(bs, rtol=1e-10)
    assert Bt.krylov_mode == (0 if host else 1)
    for i, mb in enumerate(members):
        assert rels[i] <= 1e-10
        S = StokesMG(dim=3, n=mb["n"], n_levels=mb["n_levels"], gamma_rho=mb["gamma_rho"], kA=1, kS=1, m=2,
                     schur_diag="d", restart=3)
        xs1, its1, _ = S.solve(bs[i], rtol=1e-10)
        assert its[i] == its1, (i, its, its1)
        assert np.abs(xs1.cpu().numpy() - xs[i].cpu().numpy()).max() <= 1e-8 * xs1.abs().max().item()
        S.close()
    Bt.close()


def test_batch_zero_rhs_member():
    from paper_2205_15770_gb300 import StokesBatch
    members = [dict(dim=3, n=(4, 4, 4), n_levels=2), dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=5.0)]
    Bt = StokesBatch(members)
    N = Bt.members[0].size()
    b0 = torch.zeros(N, dtype=torch.float64, device="cuda")
    b1 = Bt.members[1].mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, (4, 4, 4), seed=1).reshape(-1),
                                                device="cuda"))
    xs, its, rels = Bt.solve([b0, b1], rtol=1e-9)
    assert its[0] == 0 and rels[0] == 0.0 and torch.count_nonzero(xs[0]).item() == 0
    assert rels[1] <= 1e-9 and its[1] > 0


def test_autotuned_launch_shapes_are_valid():
    from paper_2205_15770_gb300 import StokesMG
    S = StokesMG(dim=3, n=(16, 16, 16), n_levels=4, k=2)
    for prec in (32, 64):
        shapes = S.launch_shapes(prec)
        assert len(shapes) == 4 and all(s in (1, 3, 4, -1, 5) for s in shapes), shapes


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("blocks", [1, 2, 4, 3, 7])
def test_every_launch_shape_gives_the_same_blocks(k, blocks):
    from paper_2205_15770_gb300 import StokesMG
    n = (4, 6, 2) if k < 4 else (2, 4, 2)
    V = W.perturbed_vertices(3, n, seed=5)
    S = StokesMG(dim=3, n=n, n_levels=1, k=k, vertices=V, gamma_rho=2.0)
    nu, npr = S.sizes()
    u = torch.as_tensor(W.random_vector(nu, 11), device="cuda")
    p = torch.as_tensor(W.random_vector(npr, 12), device="cuda")
    ref = None
    for shape in (4, 1, 3, -1, 5):
        S.set_launch_shape(0, shape, precision=64)
        yu, yp = S.apply_blocks(blocks, u=u, p=p)
        y = torch.cat([t for t in (yu, yp) if t is not None]).cpu().numpy()
        if ref is None:
            ref = y
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), (shape, k, blocks)


def test_every_launch_shape_gives_the_same_operator():
    from paper_2205_15770_gb300 import StokesMG
    V = W.perturbed_vertices(3, (8, 8, 8), seed=4)
    S = StokesMG(dim=3, n=(8, 8, 8), n_levels=2, k=2, vertices=V, gamma_rho=3.0)
    x = torch.as_tensor(W.random_vector(S.size(), 9), device="cuda")
    ref = None
    for shape in (4, 1, 3, -1, 5):
        S.set_launch_shape(1, shape, precision=64)
        y = S.vmult(x).cpu().numpy()
        if ref is None:
            ref = y
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), shape


def test_tuning_string_pins_shapes_and_smoother_forms(monkeypatch):
    from paper_2205_15770_gb300 import StokesError, StokesMG
    monkeypatch.setenv("STOKES_TUNING", "s32=4,1,3;s64=-1,3,1;f32=0,0,1;f64=0,1,0")
    S = StokesMG(dim=3, n=(8, 8, 8), n_levels=3, k=2, kA=1, kS=2, m=2)
    assert S.launch_shapes(32) == [4, 1, 3] and S.launch_shapes(64) == [-1, 3, 1]
    assert S.fused_levels(32) == [False, False, True]
    assert S.fused_levels(64) == [False, True, False]
    monkeypatch.setenv("STOKES_TUNING", "s32=4,4;s64=4,4,4;f32=0,1,1;f64=0,1,1")  # wrong length
    with pytest.raises(StokesError):
        StokesMG(dim=3, n=(8, 8, 8), n_levels=3, k=2, kA=1, kS=2, m=2)


def _queue_members():
    return [dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=0.0),
            dict(dim=3, n=(8, 8, 8), n_levels=3, gamma_rho=1e3),
            dict(dim=3, n=(6, 6, 6), n_levels=2, gamma_rho=10.0),
            dict(dim=3, n=(8, 8, 8), n_levels=3, gamma_rho=0.0, vertices=W.perturbed_vertices(3, (8, 8, 8), seed=7)),
            dict(dim=3, n=(16, 16, 16), n_levels=4, gamma_rho=1e2)]


@pytest.mark.parametrize("restart", [30, 3])
def test_batch_work_queue_solves(monkeypatch, restart):
    """Work-queue mode (krylov_mode 2): every member's FP32 cycle of an iteration is run by one
    persistent kernel taking (member, operation, brick) items from one queue.  Each member reaches
    the FP64 residual rtol (checked through the member's own FP64 operator) in the iteration count of
    its single-mesh solve, give or take one (the queue records the unfused smoother, the single solve
    may fuse some levels: the FP32 cycles differ by rounding), with Cartesian and trilinear members
    of different depths and a short restart that forces several restart cycles."""
    from paper_2205_15770_gb300 import StokesBatch, StokesMG
    monkeypatch.setenv("STOKES_BATCH_QUEUE", "1")
    members = _queue_members()
    kw = dict(kA=1, kS=1, m=2, schur_diag="d", restart=restart)
    Bt = StokesBatch(members, **kw)
    bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=30 + i).reshape(-1), device="cuda"))
          for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    for rep in range(2):  # the second solve replays the built graph
        xs, its, rels = Bt.solve(bs, rtol=1e-10)
        assert Bt.krylov_mode == 2
        for i, (mb, mv) in enumerate(zip(members, Bt.members)):
            r = bs[i] - mv.vmult(xs[i])
            assert torch.linalg.norm(r).item() <= 1.01e-10 * torch.linalg.norm(bs[i]).item(), (rep, i)
            if rep == 0:
                S = StokesMG(dim=3, n=mb["n"], n_levels=mb["n_levels"], gamma_rho=mb["gamma_rho"],
                             vertices=mb.get("vertices"), **kw)
                _, its1, _ = S.solve(bs[i], rtol=1e-10)
                assert abs(its[i] - its1) <= 1, (i, its, its1)
                S.close()
    Bt.close()


def test_batch_work_queue_matches_graph_branches(monkeypatch):
    """The same batch in work-queue mode and in graph-branch mode (krylov_mode 1): solutions within the
    solver tolerance of each other."""
    from paper_2205_15770_gb300 import StokesBatch
    members = _queue_members()
    kw = dict(kA=1, kS=1, m=2, schur_diag="d")
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("STOKES_BATCH_QUEUE", mode)
        Bt = StokesBatch(members, **kw)
        bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=40 + i).reshape(-1), device="cuda"))
              for i, (mb, mv) in enumerate(zip(members, Bt.members))]
        xs, its, rels = Bt.solve(bs, rtol=1e-10)
        assert Bt.krylov_mode == (2 if mode == "1" else 1)
        out[mode] = [x.cpu().numpy() for x in xs]
        Bt.close()
    for a, b in zip(out["0"], out["1"]):
        assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max()


def test_batch_work_queue_wait_budget_returns_etimeout(monkeypatch):
    """A one-cycle budget makes the first dependency wait of the queue kernel run out: the launch
    ends (no GPU fault), solve reports STOKES_ETIMEOUT, and the batch solves normally once the
    budget is restored."""
    from paper_2205_15770_gb300 import StokesBatch
    monkeypatch.setenv("STOKES_BATCH_QUEUE", "1")
    members = [dict(dim=3, n=(16, 16, 16), n_levels=4, gamma_rho=0.0), dict(dim=3, n=(8, 8, 8), n_levels=3)]
    Bt = StokesBatch(members, kA=1, kS=1, m=2, schur_diag="d")
    bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=50 + i).reshape(-1), device="cuda"))
          for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    Bt.set_wait_cycles(1)
    _, _, _, st = Bt.solve(bs, rtol=1e-8, check=False)
    assert st == 6 and "budget" in Bt.last_error
    Bt.set_wait_cycles(0)
    xs, its, rels = Bt.solve(bs, rtol=1e-8)
    assert Bt.krylov_mode == 2 and max(rels) <= 1e-8
    Bt.close()


def test_batch_work_queue_vcycle_matches_member_cycles():
    """stokes_batch_vcycle: one launch of the work-queue kernel runs the FP32 cycle of every member
    (Cartesian and trilinear, different depths).  Measured against the member's own FP64 cycle, each
    queue result is as accurate as the member's own FP32 cycle (within twice its error; FP32 cycles
    of these small pure-Stokes members drift by up to ~1e-2 in the pressure), and the queue cycle is
    a fixed function of its input (two launches agree up to the order of the atomic sums: 1e-5)."""
    from paper_2205_15770_gb300 import StokesBatch
    members = _queue_members()
    Bt = StokesBatch(members, kA=1, kS=1, m=2, schur_diag="d")
    b64 = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=60 + i).reshape(-1), device="cuda"))
           for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    bs = [b.float() for b in b64]
    first = Bt.vcycle(bs)
    first = [x.clone() for x in first]
    xs = Bt.vcycle(bs)
    for i, (mv, b) in enumerate(zip(Bt.members, b64)):
        ref = mv.vcycle(b, torch.zeros_like(b))
        own = mv.vcycle(bs[i], torch.zeros_like(bs[i])).double()
        scale = ref.abs().max().item()
        err_own = (own - ref).abs().max().item()
        assert (xs[i].double() - ref).abs().max().item() <= max(2 * err_own, 1e-5 * scale), i
        assert (xs[i] - first[i]).abs().max().item() <= 1e-5 * scale, i
    Bt.close()


def test_batch_work_queue_w_cycle(monkeypatch):
    """Work-queue mode with W-cycles (the recorded cycle visits the coarser levels twice): every
    member reaches rtol through its own FP64 operator."""
    from paper_2205_15770_gb300 import StokesBatch
    monkeypatch.setenv("STOKES_BATCH_QUEUE", "1")
    members = _queue_members()[:4]
    Bt = StokesBatch(members, kA=1, kS=1, m=2, schur_diag="d", cycle="W")
    bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, 2, mb["n"], seed=70 + i).reshape(-1), device="cuda"))
          for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    xs, its, rels = Bt.solve(bs, rtol=1e-10)
    assert Bt.krylov_mode == 2
    for i, mv in enumerate(Bt.members):
        r = bs[i] - mv.vmult(xs[i])
        assert torch.linalg.norm(r).item() <= 1.01e-10 * torch.linalg.norm(bs[i]).item(), i
    Bt.close()


def test_batch_work_queue_not_served_falls_back(monkeypatch):
    """A member the work-queue kernel does not serve (k = 3) keeps the batch on the graph branches
    (krylov_mode 1), and stokes_batch_vcycle reports STOKES_EINVAL."""
    from paper_2205_15770_gb300 import StokesBatch, StokesError
    monkeypatch.setenv("STOKES_BATCH_QUEUE", "1")
    members = [dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=0.0),
               dict(dim=3, n=(4, 4, 4), n_levels=2, gamma_rho=1.0, k=3)]
    Bt = StokesBatch(members, kA=1, kS=1, m=2, schur_diag="d")
    bs = [mv.mass_rhs(torch.as_tensor(W.fourier_forcing(3, mb.get("k", 2), mb["n"], seed=80 + i).reshape(-1),
                                      device="cuda"))
          for i, (mb, mv) in enumerate(zip(members, Bt.members))]
    xs, its, rels = Bt.solve(bs, rtol=1e-9)
    assert Bt.krylov_mode == 1 and max(rels) <= 1e-9
    with pytest.raises(StokesError) as e:
        Bt.vcycle([b.float() for b in bs])
    assert e.value.status == 1
    Bt.close()
