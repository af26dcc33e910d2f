"""CPU checks of the C-ABI library: it builds, loads, and exports every entry point
declared in include/pfq4.h (no compute calls: no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pfq4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", src)) - {"pf_alloc_fn", "pf_free_fn"})


@pytest.fixture(scope="module")
def lib_path():
    from paper_2512_12232_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pf_[a-z_]+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_ctypes_binding_covers_the_header(lib_path):
    from paper_2512_12232_gb300 import _lib
    lib = _lib.load(lib_path)
    assert sorted(_lib.EXPORTED) == declared_functions()
    for name in _lib.EXPORTED:
        assert hasattr(lib, name)


def test_error_path_without_gpu(lib_path):
    """Argument validation happens before any device work and reports PF_EINVAL."""
    import ctypes as C
    from paper_2512_12232_gb300 import _lib
    lib = _lib.load(lib_path)
    assert lib.pf_batch_build(None, None, None, 0, 0, None, None, None) == _lib.PF_EINVAL
    assert b"NULL" in lib.pf_last_error() or len(lib.pf_last_error()) > 0
    assert lib.pf_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None) == _lib.PF_OK
    assert lib.pf_workspace_bytes(None) == 0
    n = C.c_longlong()
    assert lib.pf_mesh_info(None, C.byref(n), None, None, None) == _lib.PF_EINVAL
    assert lib.pf_batch_solve(None, 1.0, None, None, None, None) == _lib.PF_EINVAL
    assert lib.pf_batch_grad(None, 0, 3, 4, 1.0, 1e-12, None, None, None, None) == _lib.PF_EINVAL
    lib.pf_mesh_destroy(None)  # a NULL handle is a no-op, as for pf_batch_destroy
    assert lib.pf_velocity_field(None, 0, None, None, None) == _lib.PF_EINVAL
    assert lib.pf_mesh_set_coords(None, 0, None, None) == _lib.PF_EINVAL
    assert lib.pf_coords_vjp(None, None, None, None) == _lib.PF_EINVAL
    # the mixed-cell mesh: refused before any device work without an output, and its
    # surface-point export without a handle
    assert lib.pf_batch_build_cut(None, None, None, 1, 0, None, 0.0, None, None) == _lib.PF_EINVAL
    assert lib.pf_mesh_cut_points(None, 0, None, None) == _lib.PF_EINVAL
    # general shapes: refused on the host before any device work
    assert lib.pf_batch_build_shapes(None, None, None, 1, 0, None, None, None) == _lib.PF_EINVAL
    g = (_lib.pf_grid * 1)(_lib.pf_grid(-1.0, 1.0, -1.0, 1.0, 16, 16))
    off = (C.c_int * 2)(0, 1)
    bc = (C.c_int * 4)(0, 0, 0, 0)
    h = C.c_void_p()
    xy = (C.c_double * 4)(0.0, 0.0, 0.5, 0.0)
    for shape, msg in [(_lib.pf_shape(7, 0.0, 0.0, 0.3, 0, None, -1), b"kind"),
                       (_lib.pf_shape(_lib.PF_SHAPE_POLYGON, 0.0, 0.0, 0.0, 2, C.cast(xy, C.POINTER(C.c_double)), -1),
                        b"3 vertices")]:
        shapes = (_lib.pf_shape * 1)(shape)
        assert lib.pf_batch_build_shapes(g, off, shapes, 1, 4, bc, None, C.byref(h)) == _lib.PF_EINVAL
        assert msg in lib.pf_last_error()


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2512_12232_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_header_compiles_as_c99_and_cxx(tmp_path):
    """include/pfq4.h is a C header: it compiles alone as pedantic C99 and as C++17."""
    import shutil
    src = tmp_path / "use.c"
    src.write_text('#include "pfq4.h"\nint main(void) { pf_shape s = {0}; pf_batch* b = 0; (void)s; (void)b; return 0; }\n')
    inc = os.path.join(ROOT, "include")
    for cc, args in (("gcc", ["-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror"]),
                     ("g++", ["-std=c++17", "-Wall", "-Werror", "-x", "c++"])):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not installed")
        r = subprocess.run([cc, *args, "-I", inc, "-c", str(src), "-o", str(tmp_path / "use.o")],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def declared_arities():
    """Number of parameters of every function declared in include/pfq4.h."""
    src = open(os.path.join(ROOT, "include", "pfq4.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(pf_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src):
        name, args = m.group(1), m.group(2).strip()
        if name in ("pf_alloc_fn", "pf_free_fn"):
            continue
        depth, n = 0, (0 if args in ("", "void") else 1)
        for ch in args:
            depth += ch == "("
            depth -= ch == ")"
            n += ch == "," and depth == 0
        out[name] = n
    return out


def test_ctypes_signatures_match_the_header_arities():
    """Every ctypes declaration passes as many arguments as the C prototype takes."""
    from paper_2512_12232_gb300 import _lib
    ar = declared_arities()
    assert ar, "no prototypes parsed"
    bad = {k: (n, len(_lib._SIGS[k][1])) for k, n in ar.items() if k in _lib._SIGS and len(_lib._SIGS[k][1]) != n}
    assert not bad, bad
