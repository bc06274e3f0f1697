"""The C-ABI library builds, loads and exports every entry point of include/stokes_mf.h (CPU only).

No compute call is made here: argument validation that returns before any CUDA work
is exercised, nothing else.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stokes_mf.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "for", "return", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_15770_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("stokes_setup", "stokes_vmult", "mg_vcycle", "stokes_solve", "stokes_destroy",
                     "stokes_sizes", "stokes_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2205_15770_gb300 import _lib
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    from paper_2205_15770_gb300 import _lib
    ctx = C.c_void_p()
    opts = _lib.StokesOpts()
    lib.stokes_default_opts(C.byref(opts))
    assert (opts.kA, opts.kS, opts.m, opts.gmres_restart, opts.eig_iters) == (3, 3, 2, 30, 40)
    mesh = _lib.StokesMesh()
    mesh.dim = 3
    for a in range(3):
        mesh.n[a] = 6
        mesh.hi[a] = 1.0
    mesh.n_levels = 3  # 6 is not divisible by 4
    mesh.dirichlet_faces = 0x3F
    assert lib.stokes_setup(C.byref(mesh), 2, 1.0, 0.0, None, C.byref(opts), None, C.byref(ctx)) == 1
    assert b"multiple" in lib.stokes_global_last_error()
    mesh.n_levels = 2
    assert lib.stokes_setup(C.byref(mesh), 5, 1.0, 0.0, None, C.byref(opts), None, C.byref(ctx)) == 1
    assert lib.stokes_setup(C.byref(mesh), 2, -1.0, 0.0, None, C.byref(opts), None, C.byref(ctx)) == 1
    assert lib.stokes_setup(None, 2, 1.0, 0.0, None, C.byref(opts), None, C.byref(ctx)) == 1
    mu = np.full(216, 1.0)
    mu[7] = 0.0
    assert lib.stokes_setup(C.byref(mesh), 2, 1.0, 0.0, mu.ctypes.data_as(C.POINTER(C.c_double)),
                            C.byref(opts), None, C.byref(ctx)) == 1
    assert ctx.value is None
    assert lib.stokes_vmult(None, 0, 64, None, None, None) == 1
    assert lib.stokes_solve(None, None, None, 1e-8, 10, None, None, None) == 1
    lib.stokes_destroy(None)


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2205_15770_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(OSError):
        _lib.load(str(tmp_path / "missing.so"))


def test_sampled_oracle_rows_match_assembled_operator():
    import workloads as W
    from oracle.assemble import assemble
    from oracle.mesh import Level
    from oracle.sampled import apply_rows
    V = W.perturbed_vertices(3, (3, 4, 2), seed=2, amplitude=0.3)
    lev = Level(3, 2, (3, 4, 2), V, dirichlet_faces=0x3F & ~0x2)
    ops = assemble(lev, mu=0.7, gamma_rho=5.0)
    x = W.random_vector(lev.size, 1)
    rows = np.random.default_rng(0).choice(lev.size, 60, replace=False)
    np.testing.assert_allclose(apply_rows(lev, x, rows, 0.7, 5.0), (ops["K"] @ x)[rows], rtol=1e-12, atol=1e-12)


def _declared_arity():
    """Parameter count of every prototype in the header (comments stripped)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name in _declared_functions():
        m = re.search(r"\b" + name + r"\s*\(([^;{]*?)\)\s*;", text, flags=re.S)
        assert m, name
        params = m.group(1).strip()
        assert "(" not in params, name  # no function-pointer parameters in this ABI
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every ctypes declaration of the binding takes as many arguments as the header's prototype
    (a changed entry point must change both)."""
    from paper_2205_15770_gb300 import _lib
    for name, n in _declared_arity().items():
        assert len(_lib.SIGNATURES[name][1]) == n, (name, n, len(_lib.SIGNATURES[name][1]))


def test_every_entry_point_rejects_a_null_context(lib):
    """Each entry point taking a context or batch handle returns STOKES_EINVAL for a null handle
    (null pointers and zero sizes elsewhere), before any device work, and keeps the reason as the
    thread's last error; the mode queries answer -1, the launch counter 0, the error-text queries of
    a null handle the thread's last error, and the destroy calls accept null."""
    from paper_2205_15770_gb300 import _lib
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    checked = 0
    for name, n in _declared_arity().items():
        m = re.search(r"\b" + name + r"\s*\(([^;{]*?)\)\s*;", text, flags=re.S)
        first = m.group(1).split(",")[0]
        restype, argtypes = _lib.SIGNATURES[name]
        if restype is not C.c_int or not ("stokes_ctx" in first or "stokes_batch" in first):
            continue
        args = [0 if t in (C.c_int, C.c_uint, C.c_longlong, C.c_size_t) else 0.0 if t in (C.c_double, C.c_float)
                else None for t in argtypes]
        expect = -1 if name in ("stokes_krylov_mode", "stokes_batch_krylov_mode") else 1
        assert getattr(lib, name)(*args) == expect, name
        if expect == 1:
            assert lib.stokes_global_last_error() != b"", name
        checked += 1
    assert checked >= 30
    assert lib.stokes_last_error(None) == lib.stokes_global_last_error()
    assert lib.stokes_batch_last_error(None) == lib.stokes_global_last_error()
    assert lib.stokes_launch_count(None) == 0
    lib.stokes_destroy(None)
    lib.stokes_destroy_batch(None)


def test_every_declaration_cites_its_passage():
    """The comment above each prototype names the paper passage it implements (a section, an
    algorithm, a lemma, a reading of the paper) or says that it has no counterpart in the paper."""
    text = open(HEADER).read()
    for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
        before = text[:m.start()]
        end = before.rfind("*/")
        comment = before[before.rfind("/*", 0, end):end]
        assert re.search(r"Sec\.|Algorithm|Lemma|reading|counterpart", comment), m.group(1)



def test_binding_checks_host_arrays_before_setup():
    """Host arrays whose size the setup would trust (vertices, per-cell mu and rho) are checked by
    the binding before any device work: a short array would otherwise be read past its end."""
    from paper_2205_15770_gb300 import StokesBatch, StokesMG, _ptr
    torch = pytest.importorskip("torch")
    n = (2, 2, 2)
    with pytest.raises(ValueError, match="vertices"):
        StokesMG(dim=3, n=n, n_levels=1, vertices=np.zeros(3 * 3 * 3 * 3 - 1))
    with pytest.raises(ValueError, match="mu_cell"):
        StokesMG(dim=3, n=n, n_levels=1, mu_cell=np.ones(7))
    with pytest.raises(ValueError, match="rho_cell"):
        StokesMG(dim=3, n=n, n_levels=1, rho_cell=np.ones(9))
    with pytest.raises(ValueError, match="member 0 vertices"):
        StokesBatch([dict(dim=2, n=(4, 4), n_levels=2, vertices=np.zeros(10))])
    with pytest.raises(TypeError, match="CUDA"):
        _ptr(torch.zeros(4, dtype=torch.float64), torch.float64, n=4)


def test_setup_rejects_inverted_or_non_finite_cells(lib):
    """A vertex-given mesh whose cell maps are not proper images of the reference cell (det J <= 0 at
    a corner) or whose coordinates are not finite is rejected before any device work."""
    import workloads as W
    from paper_2205_15770_gb300 import _lib

    def setup(V, n, dim):
        mesh = _lib.StokesMesh()
        mesh.dim = dim
        for a in range(3):
            mesh.n[a] = n[a] if a < dim else 1
            mesh.hi[a] = 1.0
        mesh.n_levels = 1
        mesh.dirichlet_faces = 0x3F if dim == 3 else 0xF
        v = np.ascontiguousarray(V.reshape(-1))
        mesh.vertices = v.ctypes.data_as(C.POINTER(C.c_double))
        opts = _lib.StokesOpts()
        lib.stokes_default_opts(C.byref(opts))
        ctx = C.c_void_p()
        return lib.stokes_setup(C.byref(mesh), 2, 1.0, 0.0, None, C.byref(opts), None, C.byref(ctx))

    V = W.lattice_vertices(3, (2, 2, 2))
    V[1, 1, 1, 0] += 1.0  # the middle vertex pushed past its +x neighbour: cell (1, 0, 0) folds
    assert setup(V, (2, 2, 2), 3) == 1
    assert b"cell (1, 0, 0) is inverted" in lib.stokes_global_last_error()
    V = W.lattice_vertices(3, (2, 2, 2))
    V[0, 0, 0, 2] = np.nan
    assert setup(V, (2, 2, 2), 3) == 1 and b"not finite" in lib.stokes_global_last_error()
    V = W.lattice_vertices(2, (4, 4))
    V[2, 2, 1] += 0.6  # 2D: the vertex (2, 2) moved past the next row
    assert setup(V, (4, 4), 2) == 1 and b"cell (1, 2) is inverted" in lib.stokes_global_last_error()


def test_header_is_plain_c_and_a_c_program_links(lib, tmp_path):
    """The boundary is a C ABI: the header compiles as strict C99 (no C++ or torch types), and a C
    program links against the library and calls it (the defaults, and a rejected setup)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_abi.c"
    src.write_text(
        '#include "stokes_mf.h"\n'
        "#include <stdio.h>\n"
        "int main(void) {\n"
        "  stokes_opts o; stokes_ctx *ctx = 0; stokes_mesh m = {0};\n"
        "  stokes_default_opts(&o);\n"
        "  if (o.kA != 3 || o.kS != 3 || o.m != 2) return 1;\n"
        "  m.dim = 3; m.n[0] = m.n[1] = m.n[2] = 6; m.hi[0] = m.hi[1] = m.hi[2] = 1.0; m.n_levels = 3;\n"
        "  if (stokes_setup(&m, 2, 1.0, 0.0, 0, &o, 0, &ctx) != STOKES_EINVAL || ctx) return 2;\n"
        '  printf("%s\\n", stokes_global_last_error());\n'
        "  return 0;\n"
        "}\n")
    libdir = os.path.join(ROOT, "paper_2205_15770_gb300")
    exe = tmp_path / "use_abi"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lstokes_mf", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert "multiple" in r.stdout
