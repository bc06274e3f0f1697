"""Pins of the oracle's flexible GMRES (CPU only) against properties that fix it independently of its
own arithmetic: with a fixed preconditioner M its j-th iterate minimises ||b - A x|| over
x in M K_j(A M, b) (computed here by least squares on the explicit Krylov matrix), a restarted run
reaches the tolerance with a non-increasing residual estimate, and a zero right-hand side returns
zero at once."""
import numpy as np
import pytest

from oracle.krylov import fgmres


def _system(n=40, seed=0):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4.0 + rng.standard_normal((n, n)) / np.sqrt(n)  # nonsymmetric, well conditioned
    M = np.diag(1.0 / np.diag(A) * rng.uniform(0.5, 1.5, n))     # a fixed (non-flexible) preconditioner
    b = rng.standard_normal(n)
    return A, M, b


@pytest.mark.parametrize("j", [1, 2, 3, 4, 5])
def test_iterate_minimises_the_residual_over_the_krylov_space(j):
    A, M, b = _system()
    x, its, _ = fgmres(lambda v: A @ v, lambda v: M @ v, b, rtol=1e-15, restart=30, maxit=j)
    assert its == j
    # K_j(A M, b) = span{b, (AM) b, ..., (AM)^(j-1) b}; x = M K y with y minimising ||b - A M K y||
    AM = A @ M
    K = np.empty((len(b), j))
    K[:, 0] = b / np.linalg.norm(b)
    for i in range(1, j):
        K[:, i] = AM @ K[:, i - 1]
        K[:, i] /= np.linalg.norm(K[:, i])
    y = np.linalg.lstsq(AM @ K, b, rcond=None)[0]
    x_ref = M @ (K @ y)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # and no iterate of the space does better
    assert np.linalg.norm(b - A @ x) <= np.linalg.norm(b - A @ x_ref) * (1 + 1e-10)


def test_restarted_run_reaches_the_tolerance_with_a_non_increasing_estimate():
    A, M, b = _system(seed=1)
    x, its, hist = fgmres(lambda v: A @ v, lambda v: M @ v, b, rtol=1e-10, restart=3, maxit=200)
    assert np.linalg.norm(b - A @ x) <= 1.0001e-10 * np.linalg.norm(b)
    assert its > 3  # it restarted
    # estimates relative to ||b||; the explicit residual recomputed at a restart carries rounding of
    # order eps ||b||, so the sequence is non-increasing up to that
    assert all(h1 <= h0 + 1e-14 for h0, h1 in zip(hist, hist[1:]))
    # the full-length run needs no more iterations than the restarted one
    _, its_full, _ = fgmres(lambda v: A @ v, lambda v: M @ v, b, rtol=1e-10, restart=40, maxit=200)
    assert its_full <= its


def test_zero_right_hand_side_and_iteration_limit():
    A, M, b = _system(seed=2)
    x, its, hist = fgmres(lambda v: A @ v, lambda v: M @ v, np.zeros_like(b))
    assert its == 0 and not x.any() and hist == [0.0]
    _, its, hist = fgmres(lambda v: A @ v, lambda v: M @ v, b, rtol=1e-14, restart=5, maxit=7)
    assert its == 7 and hist[-1] > 1e-14
