"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the multigrid method itself: it only draws
the problem data (mesh vertex coordinates, forcing fields, viscosity fields)
that both the CPU oracle and the CUDA path take as inputs.  Every generator is
deterministic in its seed.

Layout conventions (shared with the C-ABI):
  * vertex arrays: shape (n_z+1, n_y+1, n_x+1, d) in 3D, (n_y+1, n_x+1, d) in 2D,
    x fastest, coordinates interleaved; flattened C-order they are the
    ``vertices`` argument of ``stokes_setup``.
  * velocity nodal fields: shape (d, N_z, N_y, N_x) with N = k*n+1 nodes per
    direction, component-blocked.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "lattice_vertices",
    "perturbed_vertices",
    "fourier_forcing",
    "mms2d_forcing",
    "laser_beam_forcing",
    "velocity_lattice",
    "gaussian_field_cells",
    "random_vector",
    "batch_meshes",
]


def _axes(dim, n, lo, hi, per_cell):
    return [np.linspace(lo[a], hi[a], per_cell * n[a] + 1) for a in range(dim)]


def lattice_vertices(dim, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Unperturbed vertex coordinates of an n[0] x n[1] (x n[2]) box mesh."""
    ax = _axes(dim, n, lo, hi, 1)
    grids = np.meshgrid(*ax[::-1], indexing="ij")[::-1]  # x fastest in memory
    return np.stack(grids, axis=-1).astype(np.float64)


def perturbed_vertices(dim, n, seed, amplitude=0.1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), modes=3):
    """Vertices moved by a smooth seeded field: x + amplitude * h * zeta(x).

    zeta_c(x) = (1/modes) * sum_m sin(2 pi kappa_m . xhat + phi_m) * prod_i sin(pi xhat_i),
    xhat the coordinates scaled to the unit box, kappa_m integer wave vectors in
    {0,1,2}^d (not all zero), phi_m uniform phases.  zeta vanishes on the
    boundary, so boundary faces stay planar and the domain is unchanged.
    h is the cell size of this (finest) mesh along each axis.  Coarser levels of
    a uniformly refined hierarchy take every 2^j-th vertex of this array.
    """
    rng = np.random.default_rng(seed)
    X = lattice_vertices(dim, n, lo, hi)
    lo_a = np.asarray(lo[:dim], dtype=np.float64)
    hi_a = np.asarray(hi[:dim], dtype=np.float64)
    xh = (X - lo_a) / (hi_a - lo_a)
    bubble = np.prod(np.sin(np.pi * xh), axis=-1)
    h = (hi_a - lo_a) / np.asarray(n[:dim], dtype=np.float64)
    out = X.copy()
    for c in range(dim):
        zeta = np.zeros(X.shape[:-1])
        for _ in range(modes):
            kappa = rng.integers(0, 3, size=dim)
            if not kappa.any():
                kappa[rng.integers(0, dim)] = 1
            phi = rng.uniform(0.0, 2.0 * np.pi)
            zeta += np.sin(2.0 * np.pi * (xh @ kappa) + phi)
        out[..., c] += amplitude * h[c] * bubble * zeta / modes
    return out


def velocity_lattice(dim, k, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Equispaced points of the velocity node lattice, (k*n+1) per direction.

    Returned as a list of 1D coordinate arrays (x, y[, z]).  For k = 2 these
    are exactly the Taylor-Hood velocity nodes of a Cartesian mesh; for k > 2
    they are just sample positions for drawing smooth nodal fields.
    """
    return _axes(dim, n, lo, hi, k)


def fourier_forcing(dim, k, n, seed, modes=4, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Smooth random forcing sampled on the velocity lattice.

    f_c(x) = sum_{m<modes} a_cm prod_i sin(pi w_cmi xhat_i), a_cm ~ N(0,1),
    integer wave numbers w in {1,2,3}.  Shape (d, N_z, N_y, N_x) (3D).
    """
    rng = np.random.default_rng(seed)
    ax = velocity_lattice(dim, k, n, lo, hi)
    axh = [(ax[a] - lo[a]) / (hi[a] - lo[a]) for a in range(dim)]
    shape = tuple(len(a) for a in ax[::-1])
    f = np.zeros((dim,) + shape)
    for c in range(dim):
        for _ in range(modes):
            amp = rng.standard_normal()
            w = rng.integers(1, 4, size=dim)
            term = np.ones(shape)
            for a in range(dim):
                s = np.sin(np.pi * w[a] * axh[a])
                bshape = [1] * dim
                bshape[dim - 1 - a] = len(s)
                term = term * s.reshape(bshape)
            f[c] += amp * term
    return f


def mms2d_forcing(x, y, mu=1.0):
    """Forcing f = -mu Lap u + grad p of the smooth 2D Stokes solution on (0,1)^2.

    psi = sin^2(pi x) sin^2(pi y), u = (d psi/dy, -d psi/dx), p = cos(pi x) cos(pi y).
    x, y broadcastable arrays; returns (f1, f2).
    """
    pi = np.pi
    sx, cx = np.sin(pi * x), np.cos(pi * x)
    sy, cy = np.sin(pi * y), np.cos(pi * y)
    # u1 = 2 pi sx^2 sy cy = pi sx^2 sin(2 pi y); u2 = -pi sin(2 pi x) sy^2
    s2x, c2x = np.sin(2 * pi * x), np.cos(2 * pi * x)
    s2y, c2y = np.sin(2 * pi * y), np.cos(2 * pi * y)
    # Laplacians: d2/dx2 (sx^2) = 2 pi^2 cos(2 pi x); d2/dy2 sin(2 pi y) = -4 pi^2 sin(2 pi y)
    lap_u1 = pi * (2 * pi**2 * c2x) * s2y + pi * sx**2 * (-4 * pi**2 * s2y)
    lap_u2 = -(pi * (-4 * pi**2 * s2x) * sy**2 + pi * s2x * (2 * pi**2 * c2y))
    dpdx = -pi * sx * cy
    dpdy = -pi * cx * sy
    return -mu * lap_u1 + dpdx, -mu * lap_u2 + dpdy


def laser_beam_forcing(n, k=2, x0=(0.75, 0.75), c1=1e-3, c2=100.0):
    """The laser-beam test of the paper (Sec. 4.2.1) on the unit square, Q_k velocity nodes of an
    n[0] x n[1] Cartesian mesh: f = (0, c1 exp(-c2 |x - x0|^2)) with x0 = (0.75, 0.75),
    c1 = 1e-3, c2 = 100 (the paper's mu = 0.0022 and homogeneous Dirichlet data are set by the
    caller).  Shape (2, N_y, N_x).  Equispaced lattice points are the velocity nodes for k = 2."""
    ax = velocity_lattice(2, k, n)
    Y, X = np.meshgrid(ax[1], ax[0], indexing="ij")
    f = np.zeros((2,) + X.shape)
    f[1] = c1 * np.exp(-c2 * ((X - x0[0]) ** 2 + (Y - x0[1]) ** 2))
    return f


def gaussian_field_cells(n, seed, corr_length=0.2, std=1.0):
    """Seeded Gaussian random field at the cell centres of an n^3 unit-cube mesh.

    White noise on the n^3 cell grid is filtered in Fourier space by the square
    root of a squared-exponential spectrum with correlation length corr_length,
    then shifted/scaled to zero sample mean and sample standard deviation std.
    Returns shape (n, n, n) (z, y, x order), x fastest.
    """
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n, n))
    kf = np.fft.fftfreq(n, d=1.0 / n) * 2 * np.pi
    kz, ky, kx = np.meshgrid(kf, kf, kf, indexing="ij")
    k2 = kx**2 + ky**2 + kz**2
    spec = np.exp(-0.25 * corr_length**2 * k2)  # sqrt of exp(-l^2 k^2 / 2)
    g = np.real(np.fft.ifftn(np.fft.fftn(w) * spec))
    g = (g - g.mean()) / g.std() * std
    return g


def random_vector(size, seed, dtype=np.float64):
    """Uniform(-1, 1) entries, seeded."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=size).astype(dtype)


def batch_meshes(count=16, seed=0, sizes=(8, 16, 24, 32, 40), gammas=(0.0, 1e3)):
    """Seeded recipe of a batch of independent unit-cube meshes of uneven size.

    Each member: n cells per direction drawn from `sizes`, gamma drawn from `gammas`, a forcing
    seed, and the number of levels that coarsens n by halving down to 2, 3 or 5 cells.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        g = float(rng.choice(gammas))
        levels = 1
        m = n
        while m % 2 == 0 and m // 2 >= 2:
            m //= 2
            levels += 1
        out.append({"n": n, "levels": levels, "coarse_n": m, "gamma": g, "forcing_seed": int(seed * 1000 + i)})
    return out
