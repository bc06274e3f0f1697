"""The seeded synthetic inputs shared by the oracle, the GPU path and the benchmark (CPU only): each
recipe is deterministic per seed and has the properties the workloads are described by (the perturbed
meshes keep the box and fold no cell, the forcings vanish where they are sampled on the boundary, the
random field is normalised, the batch coarsens to 2^3, 3^3 or 5^3)."""
import numpy as np
import pytest

import workloads as W


def _corner_dets(V):
    """det J at the 8 corners of every cell of an (nz+1, ny+1, nx+1, 3) vertex array, from the
    cell's edges leaving each corner along +x, +y, +z."""
    out = []
    for c in range(8):
        bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        s = [1 - 2 * bx, 1 - 2 * by, 1 - 2 * bz]
        corner = V[bz:V.shape[0] - 1 + bz, by:V.shape[1] - 1 + by, bx:V.shape[2] - 1 + bx]
        ex = s[0] * (V[bz:V.shape[0] - 1 + bz, by:V.shape[1] - 1 + by, 1 - bx:V.shape[2] - bx] - corner)
        ey = s[1] * (V[bz:V.shape[0] - 1 + bz, 1 - by:V.shape[1] - by, bx:V.shape[2] - 1 + bx] - corner)
        ez = s[2] * (V[1 - bz:V.shape[0] - bz, by:V.shape[1] - 1 + by, bx:V.shape[2] - 1 + bx] - corner)
        out.append(np.einsum("...i,...i->...", ex, np.cross(ey, ez)))
    return np.stack(out)


def test_perturbed_vertices_keep_the_box_and_fold_no_cell():
    n = (8, 6, 4)
    hi = (4.0, 1.0, 1.0)
    V = W.perturbed_vertices(3, n, seed=0, amplitude=0.1, hi=hi)
    X = W.lattice_vertices(3, n, hi=hi)
    assert V.shape == (5, 7, 9, 3)
    np.testing.assert_array_equal(V, W.perturbed_vertices(3, n, seed=0, amplitude=0.1, hi=hi))
    assert not np.array_equal(V, W.perturbed_vertices(3, n, seed=1, amplitude=0.1, hi=hi))
    # every boundary vertex stays where it was (the bubble factor vanishes there)
    for sl in ((0,), (-1,)):
        np.testing.assert_allclose(V[sl[0]], X[sl[0]], atol=1e-15)
        np.testing.assert_allclose(V[:, sl[0]], X[:, sl[0]], atol=1e-15)
        np.testing.assert_allclose(V[:, :, sl[0]], X[:, :, sl[0]], atol=1e-15)
    # |zeta| <= 1: no vertex moves by more than amplitude x its axis' cell size
    h = np.array(hi) / np.array(n)
    assert np.all(np.abs(V - X) <= 0.1 * h + 1e-15)
    assert np.abs(V - X).max() > 0.01 * h.min()
    np.testing.assert_allclose(_corner_dets(X), np.prod(h), rtol=1e-12)
    folded = X.copy()
    folded[2, 3, 4, 0] += 1.5 * h[0]  # pushed past its +x neighbour
    assert (_corner_dets(folded) < 0).any()
    dets = _corner_dets(V)
    assert np.all(dets > 0)
    # a cell of the unperturbed box has det J = h_x h_y h_z at each corner; 0.1 h moves stay close
    assert dets.min() > 0.5 * np.prod(h) and dets.max() < 1.5 * np.prod(h)


def test_fourier_forcing_is_seeded_smooth_and_zero_on_the_boundary():
    f = W.fourier_forcing(3, 2, (4, 4, 4), seed=0)
    assert f.shape == (3, 9, 9, 9)
    np.testing.assert_array_equal(f, W.fourier_forcing(3, 2, (4, 4, 4), seed=0))
    assert not np.array_equal(f, W.fourier_forcing(3, 2, (4, 4, 4), seed=1))
    # products of sin(pi w x) with integer w vanish on every face of the unit box
    for face in (f[:, 0], f[:, -1], f[:, :, 0], f[:, :, -1], f[:, :, :, 0], f[:, :, :, -1]):
        assert np.abs(face).max() < 1e-12
    assert np.isfinite(f).all() and np.abs(f).max() > 0.1


def test_gaussian_field_is_normalised_and_seeded():
    g = W.gaussian_field_cells(16, seed=0)
    assert g.shape == (16, 16, 16)
    assert abs(g.mean()) < 1e-12 and g.std() == pytest.approx(1.0, rel=1e-12)
    np.testing.assert_array_equal(g, W.gaussian_field_cells(16, seed=0))
    # correlation length 0.2 of a unit box on 16 cells: neighbouring cells are strongly correlated,
    # cells half the box apart are not
    near = np.mean(g[:, :, 1:] * g[:, :, :-1])
    far = np.mean(g[:, :, 8:] * g[:, :, :8])
    assert near > 0.8 and abs(far) < 0.2


def test_batch_recipe_coarsens_to_the_stated_coarse_meshes():
    B = W.batch_meshes(16, seed=0)
    assert len(B) == 16
    assert B == W.batch_meshes(16, seed=0)
    for m in B:
        assert m["n"] in (8, 16, 24, 32, 40) and m["gamma"] in (0.0, 1e3)
        assert m["coarse_n"] in (2, 3, 5)
        assert m["coarse_n"] * 2 ** (m["levels"] - 1) == m["n"]
    assert {m["n"] for m in B} != {B[0]["n"]}  # uneven sizes


def test_laser_beam_forcing_peaks_at_the_beam_centre():
    f = W.laser_beam_forcing((16, 16))
    assert f.shape == (2, 33, 33)
    assert np.all(f[0] == 0.0)
    j, i = np.unravel_index(np.argmax(f[1]), f[1].shape)
    assert (i, j) == (24, 24)  # x0 = (0.75, 0.75) on the 33-point lattice
    assert f[1, 24, 24] == pytest.approx(1e-3)
    assert f[1, 0, 0] == pytest.approx(1e-3 * np.exp(-100 * 2 * 0.75 ** 2))


def test_random_vector_range_and_seed():
    x = W.random_vector(1000, 5)
    assert x.min() >= -1.0 and x.max() < 1.0
    np.testing.assert_array_equal(x, W.random_vector(1000, 5))
    assert W.random_vector(10, 5, dtype=np.float32).dtype == np.float32
