"""Failure detection without a GPU fault, host side (no GPU needed).

The allocator hook of plan tables (monc_proj_set_allocator): an allocator that
fails makes monc_proj_plan return MONC_PROJ_ENOMEM before it touches the
device, and the hook's arguments are checked.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_12849_gb300 import workloads as W


@pytest.fixture(scope="module")
def mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return (ctypes.c_double * a.size)(*a.tolist())


def _plan(mp, g, prec="mixed"):
    L = mp.load_library()
    h = ctypes.c_void_p()
    rc = L.monc_proj_plan(ctypes.byref(h), g.nx, g.ny, g.nz, g.dx, g.dy, _dbl(g.dz), _dbl(g.rho_c), _dbl(g.rho_f),
                          mp.PRECISIONS[prec], None)
    return rc, h


def test_failing_allocator_gives_enomem(mp):
    calls = []
    released = []
    mp.monc_proj_set_allocator(lambda n: calls.append(n) or 0, lambda ptr: released.append(ptr))
    try:
        g = W.make_grid(32, 24, 8, 25.0, 25.0, W.uniform_dz(8, 20.0))
        for prec in ("fp64", "mixed", "refined"):
            rc, h = _plan(mp, g, prec)
            assert rc == mp.MONC_PROJ_ENOMEM, mp.monc_proj_status_string(rc)
            assert not h.value
        assert len(calls) == 3 and all(n > 0 for n in calls)
        assert released == []
    finally:
        mp.monc_proj_set_allocator()


def test_allocator_arguments_checked(mp):
    L = mp.load_library()
    assert L.monc_proj_set_allocator(mp.ALLOC_FN(lambda n, u: 0), mp.FREE_FN(), None) == mp.MONC_PROJ_EINVAL
    assert L.monc_proj_set_allocator(mp.ALLOC_FN(), mp.FREE_FN(lambda p, u: None), None) == mp.MONC_PROJ_EINVAL
    assert L.monc_proj_set_allocator(mp.ALLOC_FN(), mp.FREE_FN(), None) == mp.MONC_PROJ_OK


def test_argument_checks_come_before_allocation(mp):
    calls = []
    mp.monc_proj_set_allocator(lambda n: calls.append(n) or 0, lambda ptr: None)
    try:
        g = W.make_grid(14, 16, 4, 25.0, 25.0, W.uniform_dz(4, 10.0))      # 14 = 2 * 7
        rc, _ = _plan(mp, g)
        assert rc == mp.MONC_PROJ_EUNSUPPORTED
        assert calls == []
    finally:
        mp.monc_proj_set_allocator()
