"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(monc_proj_[A-Za-z0-9_]+)\s*\(",
                                    text, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("monc_proj_plan", "monc_proj_solve", "monc_proj_destroy", "monc_proj_workspace_size",
                 "monc_proj_solve_batch", "monc_proj_status_string"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    L = lib.load_library()
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name
        assert getattr(L, name) is not None


def test_binding_names_match_header(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_without_gpu(lib):
    assert lib.monc_proj_status_string(0) == "ok"
    assert "unsupported" in lib.monc_proj_status_string(2)
    assert lib.monc_proj_status_string(99) == "unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    L = lib.load_library()
    assert L.monc_proj_plan(None, 8, 8, 4, 1.0, 1.0, None, None, None, 0, None) == lib.MONC_PROJ_EINVAL
    assert L.monc_proj_workspace_size(None, None) == lib.MONC_PROJ_EINVAL
    assert L.monc_proj_destroy(None) == lib.MONC_PROJ_OK


def test_krylov_entry_points_reject_bad_arguments_without_gpu(lib):
    L = lib.load_library()
    assert L.monc_proj_krylov_workspace_size(None, None) == lib.MONC_PROJ_EINVAL
    assert L.monc_proj_solve_krylov(None, None, None, None, None, None, None, None, None, 1e-4, 10, 1,
                                    None, None, None) == lib.MONC_PROJ_EINVAL
    assert "iteration limit" in lib.monc_proj_status_string(lib.MONC_PROJ_ENOCONV)
    assert "broke down" in lib.monc_proj_status_string(lib.MONC_PROJ_EBREAKDOWN)


def test_plan_validation_without_gpu(lib):
    import ctypes
    L = lib.load_library()
    h = ctypes.c_void_p()
    nz = 4
    dz = (ctypes.c_double * nz)(*([25.0] * nz))
    rc = (ctypes.c_double * nz)(*([1.0] * nz))
    rf = (ctypes.c_double * (nz + 1))(*([1.0] * (nz + 1)))
    # 7 and 14 are not of the form 2^a 3^b 5^c
    assert L.monc_proj_plan(ctypes.byref(h), 7, 8, nz, 10.0, 10.0, dz, rc, rf, 1, None) == lib.MONC_PROJ_EUNSUPPORTED
    assert L.monc_proj_plan(ctypes.byref(h), 8, 14, nz, 10.0, 10.0, dz, rc, rf, 1, None) == lib.MONC_PROJ_EUNSUPPORTED
    # non-positive or non-finite spacings, an unknown precision
    assert L.monc_proj_plan(ctypes.byref(h), 8, 8, nz, 0.0, 10.0, dz, rc, rf, 1, None) == lib.MONC_PROJ_EINVAL
    assert L.monc_proj_plan(ctypes.byref(h), 8, 8, nz, 10.0, float("nan"), dz, rc, rf, 1, None) == lib.MONC_PROJ_EINVAL
    bad = (ctypes.c_double * nz)(*([25.0, -1.0, 25.0, 25.0]))
    assert L.monc_proj_plan(ctypes.byref(h), 8, 8, nz, 10.0, 10.0, bad, rc, rf, 1, None) == lib.MONC_PROJ_EINVAL
    assert L.monc_proj_plan(ctypes.byref(h), 8, 8, nz, 10.0, 10.0, dz, rc, rf, 7, None) == lib.MONC_PROJ_EINVAL
    assert h.value is None
