"""GB300 matrix-free monolithic multigrid for Q_k-Q_{k-1} Taylor-Hood (generalized) Stokes.

Python face of the C ABI in include/stokes_mf.h.  Every computation runs in the CUDA
library libstokes_mf.so; this module only marshals torch tensors (device memory and
streams) into the C calls.  If the library is missing, constructing a solver raises.

    from paper_2205_15770_gb300 import StokesMG
    S = StokesMG(dim=3, n=(32, 32, 32), n_levels=5, k=2, vertices=V, gamma_rho=100.0)
    b = S.mass_rhs(f)                      # f: velocity nodal forcing, torch.float64 on cuda
    x, iters, rel = S.solve(b, rtol=1e-8)
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

__all__ = ["StokesMG", "StokesBatch", "StokesError", "ALL_FACES", "stokes_solve_fn", "fma_peak"]

ALL_FACES = {2: 0xF, 3: 0x3F}
BLOCK_A, BLOCK_BT, BLOCK_B = 1, 2, 4


class StokesError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{L.STATUS.get(status, status)}: {msg}")
        self.status = status


def _torch():
    import torch
    return torch


def _ptr(t, dtype, n=None, device=None, what="vector"):
    """Device pointer of a contiguous CUDA tensor of the given dtype; with n / device, also checks
    its entry count and its device (the C ABI takes bare pointers: a short vector or one on another
    GPU would be read out of bounds there)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what}: expected {n} entries, got {t.numel()}")
    if device is not None and t.device != device:
        raise ValueError(f"{what}: tensor on {t.device}, the solver's context on {device}")
    return C.c_void_p(t.data_ptr())


def _host_doubles(a, n, what):
    """Contiguous float64 copy of a host array with exactly n entries (the setup reads n values)."""
    v = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if v.size != n:
        raise ValueError(f"{what}: expected {n} values, got {v.size}")
    return v


def fma_peak(precision=32):
    """Measured FMA throughput of the current device in TFLOP/s (stokes_fma_peak; precision 32, 64, or 2 for
    FP32 in packed pairs)."""
    torch = _torch()
    lib = L.load()
    out = C.c_double()
    st = lib.stokes_fma_peak(int(precision), C.byref(out), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise StokesError(st, lib.stokes_global_last_error().decode())
    return out.value


class StokesMG:
    """One hierarchy + smoother setup (Algorithm 2) + coarse factorisation on the current CUDA device."""

    def __init__(self, dim, n, n_levels, k=2, mu=1.0, gamma_rho=0.0, vertices=None, lo=(0.0, 0.0, 0.0),
                 hi=(1.0, 1.0, 1.0), dirichlet_faces=None, mu_cell=None, kA=3, kS=3, m=2, cycle="V",
                 schur_diag="loc", vcycle_fp32=True, restart=30, eig_iters=40, eig_safety=1.1, seed=0x5EED,
                 c_mass=0.0, c_grad=0.0, sym_grad=False, rho_cell=None, deterministic=False, wait_cycles=0):
        self._lib = L.load()
        torch = _torch()
        self.dim, self.k, self.n_levels = dim, k, n_levels
        self._n = tuple(int(v) for v in n[:dim])
        mesh = L.StokesMesh()
        mesh.dim = dim
        nn = list(n) + [1] * (3 - len(n))
        for a in range(3):
            mesh.n[a] = int(nn[a])
            mesh.lo[a] = float(lo[a]) if a < len(lo) else 0.0
            mesh.hi[a] = float(hi[a]) if a < len(hi) else 1.0
        mesh.n_levels = n_levels
        mesh.dirichlet_faces = ALL_FACES[dim] if dirichlet_faces is None else int(dirichlet_faces)
        self._keep = []
        n_cells, n_vert = 1, 1
        for a in range(dim):
            n_cells *= int(nn[a])
            n_vert *= int(nn[a]) + 1
        if vertices is not None:
            v = _host_doubles(vertices, n_vert * dim, "vertices")
            self._keep.append(v)
            mesh.vertices = v.ctypes.data_as(C.POINTER(C.c_double))
        mu_ptr = None
        if mu_cell is not None:
            mc = _host_doubles(mu_cell, n_cells, "mu_cell")
            self._keep.append(mc)
            mu_ptr = mc.ctypes.data_as(C.POINTER(C.c_double))
        opts = L.StokesOpts()
        self._lib.stokes_default_opts(C.byref(opts))
        opts.kA, opts.kS, opts.m = kA, kS, m
        opts.cycle = {"V": 0, "W": 1}[cycle]
        opts.schur_diag = {"loc": 0, "p": 1, "d": 2, "exact": 3}[schur_diag]
        opts.vcycle_fp32 = 1 if vcycle_fp32 else 0
        opts.gmres_restart = restart
        opts.eig_iters = eig_iters
        opts.eig_safety = eig_safety
        opts.seed = seed
        opts.c_mass, opts.c_grad = float(c_mass), float(c_grad)
        opts.sym_grad = 1 if sym_grad else 0
        # True / 1: owner-computes, 2 or "colour": colour classes with bounded grid barriers
        opts.deterministic = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, "owner": 1, "colour": 2}[deterministic]
        opts.wait_cycles = int(wait_cycles)
        if rho_cell is not None:
            rc = _host_doubles(rho_cell, n_cells, "rho_cell")
            self._keep.append(rc)
            opts.rho_cell = rc.ctypes.data_as(C.POINTER(C.c_double))
        ctx = C.c_void_p()
        st = self._lib.stokes_setup(C.byref(mesh), k, float(mu), float(gamma_rho), mu_ptr, C.byref(opts),
                                    self._stream(), C.byref(ctx))
        if st != 0:
            raise StokesError(st, self._lib.stokes_global_last_error().decode())
        self._ctx = ctx
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.sizes_all = [self.sizes(l) for l in range(n_levels)]

    # --- plumbing ------------------------------------------------------------------------------
    @staticmethod
    def _stream():
        torch = _torch()
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def _check(self, st):
        if st != 0:
            raise StokesError(st, self._lib.stokes_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.stokes_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _level(self, level):
        return self.n_levels - 1 if level is None else level

    def sizes(self, level=None):
        """(n_u, n_p) of a level (fixed for the context's lifetime, so asked once per level)."""
        lv = self._level(level)
        cache = self.__dict__.setdefault("_sizes", {})
        if lv not in cache:
            nu, npr = C.c_longlong(), C.c_longlong()
            self._check(self._lib.stokes_sizes(self._ctx, lv, C.byref(nu), C.byref(npr)))
            cache[lv] = (nu.value, npr.value)
        return cache[lv]

    def size(self, level=None):
        nu, npr = self.sizes(level)
        return nu + npr

    @staticmethod
    def _prec(t):
        torch = _torch()
        if t.dtype == torch.float64:
            return 64
        if t.dtype == torch.float32:
            return 32
        raise TypeError("vectors must be float32 or float64")

    def empty(self, level=None, dtype=None):
        torch = _torch()
        return torch.empty(self.size(level), dtype=dtype or torch.float64, device=self.device)

    # --- operators ------------------------------------------------------------------------------
    def _v(self, t, dtype, n, what):
        """_ptr with the entry count and the context's device checked."""
        return _ptr(t, dtype, n=n, device=self.device, what=what)

    @staticmethod
    def _distinct(a, b, names):
        """An input the library reads while it writes the other vector must not be that vector."""
        if a.data_ptr() == b.data_ptr():
            raise ValueError(f"{names[0]} and {names[1]} must be different vectors")

    def vmult(self, x, y=None, level=None):
        """y = K x (Sec. 3.1 matrix-free operator)."""
        torch = _torch()
        y = torch.empty_like(x) if y is None else y
        pr = self._prec(x)
        lv = self._level(level)
        n = self.size(lv)
        self._distinct(x, y, ("x", "y"))
        self._check(self._lib.stokes_vmult(self._ctx, lv, pr, self._v(x, x.dtype, n, "x"), self._v(y, x.dtype, n, "y"),
                                           self._stream()))
        return y

    def apply_blocks(self, blocks, u=None, p=None, level=None, dtype=None):
        """Returns (yu, yp) with yu = [A u] + [B^T p], yp = [B u] - [C p] according to the block bit set
        (1 A, 2 B^T, 4 B, 64 C; 8 / 16 mass)."""
        torch = _torch()
        lv = self._level(level)
        nu, npr = self.sizes(lv)
        ref = u if u is not None else p
        dt = ref.dtype
        yu = torch.empty(nu, dtype=dt, device=self.device) if blocks & (1 | 2 | 8 | 16) else None
        yp = torch.empty(npr, dtype=dt, device=self.device) if blocks & (4 | 64) else None
        self._check(self._lib.stokes_apply_blocks(
            self._ctx, lv, self._prec(ref), blocks, self._v(u, dt, nu, "u") if u is not None else None,
            self._v(p, dt, npr, "p") if p is not None else None, _ptr(yu, dt) if yu is not None else None,
            _ptr(yp, dt) if yp is not None else None, self._stream()))
        return yu, yp

    def mass_rhs(self, f, level=None):
        """b = [Z M_v f ; 0] for velocity nodal values f (n_u entries)."""
        torch = _torch()
        lv = self._level(level)
        b = torch.empty(self.size(lv), dtype=f.dtype, device=self.device)
        self._check(self._lib.stokes_mass_rhs(self._ctx, lv, self._prec(f), self._v(f, f.dtype, self.sizes(lv)[0], "f"),
                                              _ptr(b, f.dtype), self._stream()))
        return b

    def smooth(self, b, x, steps=1, level=None):
        """x <- S^steps (x, b): inexact symmetric Uzawa smoother (in place)."""
        lv = self._level(level)
        n = self.size(lv)
        self._distinct(b, x, ("b", "x"))
        self._check(self._lib.stokes_smooth(self._ctx, lv, self._prec(x), steps, self._v(b, x.dtype, n, "b"),
                                            self._v(x, x.dtype, n, "x"), self._stream()))
        return x

    def smooth_noalloc(self, b, x, steps=1, level=None):
        """Same as smooth(), but the smoother's work vectors live in the library's static 16 MiB device
        array instead of the context's memory: for callers that must not allocate at this point.
        Overlapping calls race on that array; levels that need more scratch raise StokesError."""
        lv = self._level(level)
        n = self.size(lv)
        self._distinct(b, x, ("b", "x"))
        self._check(self._lib.stokes_smooth_noalloc(self._ctx, lv, self._prec(x), steps,
                                                    self._v(b, x.dtype, n, "b"), self._v(x, x.dtype, n, "x"),
                                                    self._stream()))
        return x

    def restrict(self, r_fine, fine_level):
        torch = _torch()
        out = torch.empty(self.size(fine_level - 1), dtype=r_fine.dtype, device=self.device)
        self._check(self._lib.stokes_transfer(self._ctx, fine_level, self._prec(r_fine), 0,
                                              self._v(r_fine, r_fine.dtype, self.size(fine_level), "r_fine"),
                                              _ptr(out, r_fine.dtype), self._stream()))
        return out

    def prolongate(self, w_coarse, fine_level):
        torch = _torch()
        out = torch.empty(self.size(fine_level), dtype=w_coarse.dtype, device=self.device)
        self._check(self._lib.stokes_transfer(self._ctx, fine_level, self._prec(w_coarse), 1,
                                              self._v(w_coarse, w_coarse.dtype, self.size(fine_level - 1), "w_coarse"),
                                              _ptr(out, w_coarse.dtype), self._stream()))
        return out

    def coarse_solve(self, b):
        torch = _torch()
        x = torch.empty_like(b)
        self._check(self._lib.stokes_coarse_solve(self._ctx, self._prec(b), self._v(b, b.dtype, self.size(0), "b"),
                                                  _ptr(x, b.dtype), self._stream()))
        return x

    def vcycle(self, b, x=None):
        """x <- MG(x, b), one cycle of Algorithm 1 on the finest level (FP32 or FP64 by dtype)."""
        torch = _torch()
        x = torch.zeros_like(b) if x is None else x
        n = self.size()
        self._distinct(b, x, ("b", "x"))
        self._check(self._lib.mg_vcycle(self._ctx, self._prec(b), self._v(b, b.dtype, n, "b"),
                                        self._v(x, b.dtype, n, "x"), self._stream()))
        return x

    def solve(self, b, x=None, rtol=1e-8, maxit=200):
        """FP64 FGMRES right-preconditioned by one cycle per iteration; returns (x, iterations, rel. residual)."""
        torch = _torch()
        x = torch.zeros_like(b) if x is None else x
        it, rel = C.c_int(), C.c_double()
        n = self.size()
        self._distinct(b, x, ("b", "x"))
        st = self._lib.stokes_solve(self._ctx, self._v(b, torch.float64, n, "b"), self._v(x, torch.float64, n, "x"),
                                    float(rtol), int(maxit), C.byref(it), C.byref(rel), self._stream())
        self._check(st)
        return x, it.value, rel.value

    def solve_host(self, b, rtol=1e-8, maxit=200, out=None):
        """stokes_solve_host: numpy float64 b in (pinned or pageable host memory), numpy x out."""
        b = _host_doubles(b, self.size(), "b")
        x = np.empty_like(b) if out is None else out
        if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.size == b.size and x.flags.c_contiguous):
            raise ValueError(f"out: expected a contiguous float64 array of {b.size} entries")
        it, rel = C.c_int(), C.c_double()
        st = self._lib.stokes_solve_host(self._ctx, b.ctypes.data_as(C.POINTER(C.c_double)),
                                         x.ctypes.data_as(C.POINTER(C.c_double)), float(rtol), int(maxit),
                                         C.byref(it), C.byref(rel), self._stream())
        self._check(st)
        return x, it.value, rel.value

    def mass(self, u, full_rows=True, level=None):
        """Velocity mass: full_rows -> M_v Z u (every row, constrained u read as 0); else Z M_v u."""
        yu, _ = self.apply_blocks(16 if full_rows else 8, u=u, level=level)
        return yu

    def set_viscosity(self, mu_cell):
        """Replace the per-cell viscosity of the finest level and rebuild the hierarchy's setup."""
        n_cells = 1
        for v in self._n:
            n_cells *= v
        mc = _host_doubles(mu_cell, n_cells, "mu_cell")
        self._check(self._lib.stokes_set_viscosity(self._ctx, mc.ctypes.data_as(C.POINTER(C.c_double)),
                                                   self._stream()))

    def cell_grad(self, x, lam):
        """dJ/dmu_c = -lam^T (dK/dmu_c) x per finest-level cell (adjoint viscosity gradient)."""
        torch = _torch()
        n = 1
        for v in self._n:
            n *= v
        g = torch.empty(n, dtype=torch.float64, device=self.device)
        N = self.size()
        self._check(self._lib.stokes_cell_grad(self._ctx, self._v(x, torch.float64, N, "x"),
                                               self._v(lam, torch.float64, N, "lam"), _ptr(g, torch.float64),
                                               self._stream()))
        return g

    def velocity_nodes(self, level=None):
        """(nv, dim) float64 CUDA tensor of the physical velocity-node coordinates of a level."""
        torch = _torch()
        lv = self._level(level)
        nu, _ = self.sizes(lv)
        xyz = torch.empty(nu, dtype=torch.float64, device=self.device)
        self._check(self._lib.stokes_velocity_nodes(self._ctx, lv, _ptr(xyz, torch.float64), self._stream()))
        return xyz.view(nu // self.dim, self.dim)

    def lift_rhs(self, uD, b):
        """b -= Z K_full u_D in place (inhomogeneous Dirichlet data by lifting); returns b."""
        torch = _torch()
        n = self.size()
        self._distinct(uD, b, ("uD", "b"))
        self._check(self._lib.stokes_lift_rhs(self._ctx, self._v(uD, torch.float64, n, "uD"),
                                              self._v(b, torch.float64, n, "b"), self._stream()))
        return b

    def mg_iterate(self, b, x=None, max_iter=15, reduction=1e-10, allow_divergence=False):
        """Stationary multigrid iteration (FP64 cycle); returns (x, iterations, residual history, rate q).

        Not reaching the reduction in max_iter cycles is not an error (the paper's protocol); a
        diverging iteration raises StokesError unless allow_divergence, in which case q = inf."""
        torch = _torch()
        x = torch.zeros_like(b) if x is None else x
        it, q = C.c_int(), C.c_double()
        hist = (C.c_double * (max_iter + 1))()
        n = self.size()
        self._distinct(b, x, ("b", "x"))
        st = self._lib.stokes_mg_iterate(self._ctx, self._v(b, torch.float64, n, "b"), self._v(x, torch.float64, n, "x"),
                                         int(max_iter), float(reduction), C.byref(it), hist, C.byref(q), self._stream())
        if st == 5 and allow_divergence:
            return x, it.value, [], float("inf")
        if st not in (0, 4):
            self._check(st)
        return x, it.value, list(hist)[: it.value + 1], q.value

    def level_params(self, level):
        vals = [C.c_double() for _ in range(4)]
        self._check(self._lib.stokes_get_level_params(self._ctx, level, *[C.byref(v) for v in vals]))
        return dict(zip(("beta_A", "beta_S", "sigma", "tau"), (v.value for v in vals)))

    def diagonals(self, level):
        torch = _torch()
        nu, npr = self.sizes(level)
        DA = torch.empty(nu, dtype=torch.float64, device=self.device)
        DS = torch.empty(npr, dtype=torch.float64, device=self.device)
        self._check(self._lib.stokes_get_diagonals(self._ctx, level, _ptr(DA, torch.float64), _ptr(DS, torch.float64),
                                                   self._stream()))
        return DA, DS

    def time_apply(self, blocks, level=None, precision=32, reps=100):
        """Average duration (ms) of the cell kernel for `blocks`, timed with CUDA events on the launching stream."""
        ms = C.c_double()
        self._check(self._lib.stokes_time_apply(self._ctx, self._level(level), precision, blocks, reps, C.byref(ms),
                                                self._stream()))
        return ms.value

    def launch_shapes(self, precision=32):
        """Autotuned 3D cell-kernel launch shape per level (1 / 4 warps per CTA, 3 = components split over
        3 warps, -1 = point kernel, 5 = cell-component kernel)."""
        out = []
        for l in range(self.n_levels):
            v = C.c_int()
            self._check(self._lib.stokes_get_launch_shape(self._ctx, l, precision, C.byref(v)))
            out.append(v.value)
        return out

    def geometry_stored(self, precision=64):
        """Per level: True where the column kernels of that precision read the per-point geometry stored
        at setup (stokes_get_geometry_stored)."""
        out = []
        for l in range(self.n_levels):
            v = C.c_int()
            self._check(self._lib.stokes_get_geometry_stored(self._ctx, l, precision, C.byref(v)))
            out.append(bool(v.value))
        return out

    def fused_levels(self, precision=32):
        """Per level: True where smoothing runs in the fused form (stokes_get_smoother_fusion)."""
        out = []
        for l in range(self.n_levels):
            v = C.c_int()
            self._check(self._lib.stokes_get_smoother_fusion(self._ctx, l, precision, C.byref(v)))
            out.append(bool(v.value))
        return out

    def set_launch_shape(self, level, shape, precision=32):
        """Override the autotuned launch shape (1 or 4 warps per CTA column kernel, 3 component split,
        -1 point kernel, 5 cell-component kernel)."""
        self._check(self._lib.stokes_set_launch_shape(self._ctx, level, precision, shape))

    @property
    def launch_count(self):
        return int(self._lib.stokes_launch_count(self._ctx))

    @property
    def krylov_mode(self):
        """1: inner FGMRES iterations on the device (one graph launch per restart cycle), 0: host-driven,
        -1: no solve yet (stokes_krylov_mode)."""
        return int(self._lib.stokes_krylov_mode(self._ctx))

    def set_wait_cycles(self, cycles):
        """Deterministic mode: the grid-barrier wait budget in clock cycles (0: the default)."""
        self._check(self._lib.stokes_set_wait_cycles(self._ctx, int(cycles)))


class StokesBatch:
    """Independent meshes solved together (stokes_setup_batch / stokes_solve_batch).

    members: list of dicts with keys dim, n, n_levels and optionally k, mu, gamma_rho,
    vertices, lo, hi, dirichlet_faces.  Options (kA, kS, m, ...) are shared.
    """

    def __init__(self, members, kA=3, kS=3, m=2, cycle="V", schur_diag="loc", vcycle_fp32=True, restart=30,
                 eig_iters=40, eig_safety=1.1, seed=0x5EED, c_mass=0.0, c_grad=0.0):
        self._lib = L.load()
        torch = _torch()
        nm = len(members)
        meshes = (L.StokesMesh * nm)()
        self._keep = []
        ks = (C.c_int * nm)()
        mus = (C.c_double * nm)()
        gs = (C.c_double * nm)()
        for i, mb in enumerate(members):
            ms = meshes[i]
            dim = mb["dim"]
            ms.dim = dim
            nn = list(mb["n"]) + [1] * (3 - len(mb["n"]))
            lo = mb.get("lo", (0.0, 0.0, 0.0))
            hi = mb.get("hi", (1.0, 1.0, 1.0))
            for a in range(3):
                ms.n[a] = int(nn[a])
                ms.lo[a] = float(lo[a])
                ms.hi[a] = float(hi[a])
            ms.n_levels = mb["n_levels"]
            ms.dirichlet_faces = mb.get("dirichlet_faces", ALL_FACES[dim])
            if mb.get("vertices") is not None:
                n_vert = 1
                for a in range(dim):
                    n_vert *= int(nn[a]) + 1
                v = _host_doubles(mb["vertices"], n_vert * dim, f"member {i} vertices")
                self._keep.append(v)
                ms.vertices = v.ctypes.data_as(C.POINTER(C.c_double))
            ks[i] = mb.get("k", 2)
            mus[i] = mb.get("mu", 1.0)
            gs[i] = mb.get("gamma_rho", 0.0)
        opts = L.StokesOpts()
        self._lib.stokes_default_opts(C.byref(opts))
        opts.kA, opts.kS, opts.m = kA, kS, m
        opts.cycle = {"V": 0, "W": 1}[cycle]
        opts.schur_diag = {"loc": 0, "p": 1, "d": 2, "exact": 3}[schur_diag]
        opts.vcycle_fp32 = 1 if vcycle_fp32 else 0
        opts.gmres_restart = restart
        opts.eig_iters = eig_iters
        opts.eig_safety = eig_safety
        opts.seed = seed
        opts.c_mass, opts.c_grad = float(c_mass), float(c_grad)
        bt = C.c_void_p()
        st = self._lib.stokes_setup_batch(nm, meshes, ks, mus, gs, C.byref(opts), StokesMG._stream(), C.byref(bt))
        if st != 0:
            raise StokesError(st, self._lib.stokes_global_last_error().decode())
        self._bt = bt
        self.n_meshes = nm
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.members = []
        for i in range(nm):
            ctx = C.c_void_p()
            self._check(self._lib.stokes_batch_context(bt, i, C.byref(ctx)))
            self.members.append(_MemberView(self._lib, ctx, members[i]["n_levels"], members[i]["dim"],
                                            members[i]["n"], self.device))

    def _check(self, st):
        if st != 0:
            raise StokesError(st, self._lib.stokes_batch_last_error(self._bt).decode())

    def _member_ptrs(self, bs, xs, dtype):
        """Pointer arrays of one vector per member, each checked against its member's size."""
        nm = self.n_meshes
        if len(bs) != nm or len(xs) != nm:
            raise ValueError(f"expected {nm} right-hand sides and {nm} solution vectors, got {len(bs)} and {len(xs)}")
        bp = (C.c_void_p * nm)(*[_ptr(b, dtype, n=M.size(), device=self.device, what=f"b[{i}]").value
                                 for i, (b, M) in enumerate(zip(bs, self.members))])
        xp = (C.c_void_p * nm)(*[_ptr(x, dtype, n=M.size(), device=self.device, what=f"x[{i}]").value
                                 for i, (x, M) in enumerate(zip(xs, self.members))])
        return bp, xp

    def solve(self, bs, xs=None, rtol=1e-8, maxit=200, check=True):
        """Solve all members; bs, xs: lists of float64 CUDA tensors.  Returns (xs, iterations, rel residuals);
        with check=False a failing member raises nothing and the status (the first non-OK member's,
        0 if none) is returned as a fourth value."""
        torch = _torch()
        xs = [torch.zeros_like(b) for b in bs] if xs is None else xs
        nm = self.n_meshes
        bp, xp = self._member_ptrs(bs, xs, torch.float64)
        its = (C.c_int * nm)()
        rel = (C.c_double * nm)()
        st = self._lib.stokes_solve_batch(self._bt, bp, xp, float(rtol), int(maxit), its, rel, StokesMG._stream())
        if not check:
            return xs, list(its), list(rel), st
        self._check(st)
        return xs, list(its), list(rel)

    @property
    def last_error(self):
        return self._lib.stokes_batch_last_error(self._bt).decode()

    @property
    def krylov_mode(self):
        """1: every member's inner FGMRES iterations on the device in one graph launch per restart cycle
        (one while node per member, independent branches), 2: device iterations in lockstep with the
        members' FP32 cycles in one persistent work-queue kernel per iteration (STOKES_BATCH_QUEUE=1),
        0: host-driven lockstep, -1: no solve yet (stokes_batch_krylov_mode)."""
        return int(self._lib.stokes_batch_krylov_mode(self._bt))

    def vcycle(self, bs, xs=None):
        """One FP32 cycle of every member in one launch of the persistent work-queue kernel
        (stokes_batch_vcycle); bs, xs: lists of float32 CUDA tensors.  Returns xs."""
        torch = _torch()
        xs = [torch.empty_like(b) for b in bs] if xs is None else xs
        bp, xp = self._member_ptrs(bs, xs, torch.float32)
        st = self._lib.stokes_batch_vcycle(self._bt, bp, xp, StokesMG._stream())
        if st != 0:
            raise StokesError(st, self._lib.stokes_global_last_error().decode())
        return xs

    def set_wait_cycles(self, cycles):
        """Work-queue mode: the clock64() budget of each dependency wait (0: 2^31); a wait that runs out
        makes solve() raise STOKES_ETIMEOUT (stokes_batch_set_wait_cycles)."""
        st = self._lib.stokes_batch_set_wait_cycles(self._bt, int(cycles))
        self._check(st)

    def close(self):
        if getattr(self, "_bt", None):
            self._lib.stokes_destroy_batch(self._bt)
            self._bt = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _MemberView(StokesMG):
    """A batch member's context seen through the StokesMG interface (owned by the batch)."""

    def __init__(self, lib, ctx, n_levels, dim, n, device):  # noqa: D401 - no setup here
        self._lib = lib
        self._ctx = ctx
        self.n_levels = n_levels
        self.dim = dim
        self._n = tuple(int(v) for v in n[:dim])
        self.device = device

    def close(self):
        self._ctx = None


class StokesSolveFunction:
    """torch.autograd.Function for x = K(mu)^{-1} (Z M_v f) with adjoint gradients.

    forward(mu_cell, f): FP64 FGMRES solve on a StokesMG whose finest-level per-cell viscosity is
    mu_cell (rebuilt through set_viscosity when mu changes).  backward(dJ/dx): one adjoint solve
    K lam = dJ/dx with the same multigrid (K is symmetric), then
        dJ/dmu_c = -lam^T (dK/dmu_c) x          (stokes_cell_grad)
        dJ/df    = (Z M_v)^T lam_u = M_v Z lam_u  (velocity mass, every row)
    Use through ``stokes_solve_fn(solver, mu_cell, f, rtol)``.
    """


def _make_function():
    import torch

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, mu_cell, f, solver, rtol):
            solver.set_viscosity(mu_cell.detach().cpu().numpy())
            b = solver.mass_rhs(f.detach())
            x, _, _ = solver.solve(b, rtol=rtol)
            ctx.solver, ctx.rtol = solver, rtol
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            S = ctx.solver
            lam, _, _ = S.solve(gx.detach().contiguous().clone(), rtol=ctx.rtol)
            gmu = S.cell_grad(x, lam)
            nu, _ = S.sizes()
            gf = S.mass(lam[:nu].contiguous(), full_rows=True)  # (Z M_v)^T lam_u = M_v Z lam_u
            return gmu, gf, None, None

    return _Fn


_FN = None


def stokes_solve_fn(solver, mu_cell, f, rtol=1e-12):
    """Differentiable solve: returns x(mu_cell, f) with gradients w.r.t. mu_cell and f."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(mu_cell, f, solver, rtol)
