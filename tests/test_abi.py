"""The C ABI on the CPU: the shared library loads and exports every function
include/fvm.h declares, the binding's structures match the header, and the
host-only parameter checks reject bad input (no CUDA call is made)."""
import ctypes
import os
import re

import pytest

import cases

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fvm.h")


def _lib():
    import paper_2209_09671_gb300 as P
    from paper_2209_09671_gb300 import fvm
    if not os.path.exists(fvm.LIB_PATH):
        from paper_2209_09671_gb300 import _build
        _build.build()
    return P, fvm, P.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fvm_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("fvm_workspace_size", "fvm_create", "fvm_destroy", "fvm_step", "fvm_poisson_solve",
              "fvm_step_adjoint", "fvm_poisson_solve_noalloc"):
        assert n in names


def test_library_exports_every_declared_function():
    P, fvm, lib = _lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(fvm.EXPORTS) <= set(declared_functions())


def test_params_struct_matches_header_field_order():
    _, fvm, _ = _lib()
    text = open(HEADER).read()
    body = text[text.index("typedef struct {\n  int nx, ny, nz;"):text.index("} fvm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b([A-Za-z_][A-Za-z_0-9]*)(?:\[\d\])?\s*[,;]", body)
    fields = ["lam" if f == "lambda" else f for f in fields]
    assert fields == [f[0] for f in fvm.fvm_params._fields_]


def test_workspace_size_and_validation_on_host():
    _, fvm, lib = _lib()
    p, _ = cases.static_drop()
    n = fvm.fvm_workspace_size(p)
    assert n > 0
    bad = [p.replace(h=0.0), p.replace(nx=2), p.replace(precision=7), p.replace(rho=(0.0, 1.0)),
           p.replace(smooth_passes=3), p.replace(mg_levels=0),
           p.replace(tbc=(1, 1, 1, 1, 0, 0), tbc_T0=(1.0,) * 6),
           p.replace(nz=3), p.replace(bc=(0, 1, 0), nx=63)]   # odd periodic axes
    for q in bad:
        with pytest.raises(fvm.FvmError):
            fvm.fvm_workspace_size(q)
    # null pointers are rejected before any CUDA call
    cp = fvm.make_params(p)
    out = ctypes.c_void_p()
    assert lib.fvm_create(ctypes.byref(cp), None, ctypes.c_size_t(n), None, ctypes.byref(out)) == 1
    assert lib.fvm_poisson_solve_noalloc(ctypes.byref(cp), None, None, None, None, None) == 1
    assert lib.fvm_status_string(0) == b"ok"
    assert lib.fvm_version().startswith(b"fvm-gb300")


def test_workspace_grows_with_the_grid_and_precision():
    _, fvm, _ = _lib()
    small = cases.Params(nx=32, ny=32, nz=32, h=1.0 / 32)
    big = small.replace(nx=64, ny=64, nz=64, h=1.0 / 64)
    assert fvm.fvm_workspace_size(big) > 7 * fvm.fvm_workspace_size(small)
    assert fvm.fvm_workspace_size(small.replace(precision=cases.MIXED)) < fvm.fvm_workspace_size(small)


def test_adjoint_buffers_are_reserved_only_on_request():
    """adjoint = 1 adds 21 double fields of N cells (the adjoint step's
    buffers) and 22 coefficient slots of N doubles; it is rejected with the
    MIXED precision and for values other than 0 and 1."""
    _, fvm, _ = _lib()
    p = cases.Params(nx=32, ny=16, nz=8, h=1.0 / 32, precision=cases.F64)
    n0 = fvm.fvm_workspace_size(p)
    n1 = fvm.fvm_workspace_size(p.replace(adjoint=1))
    assert n1 - n0 >= 43 * 8 * p.nx * p.ny * p.nz
    assert n1 - n0 <= 43 * 8 * p.nx * p.ny * p.nz + 22 * 256
    for q in (p.replace(adjoint=1, precision=cases.MIXED), p.replace(adjoint=2)):
        with pytest.raises(fvm.FvmError):
            fvm.fvm_workspace_size(q)
