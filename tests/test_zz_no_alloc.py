"""monc_proj_solve_noalloc: a projection that allocates no device memory.

Callers that cannot allocate (a host application that owns all device memory
through its own pool, a model component handed finished device arrays, a
latency-critical loop that cannot afford cudaMalloc's device-wide
synchronisation) use this entry point; its tables and workspace live in a
static device array inside the library.  This test calls it through the C ABI
and checks it against monc_proj_solve, on two calls in a row so that the
second runs on scratch the first one left behind.  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2009_12849_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5, "refined": 1e-11}
DTYPE = {"fp64": torch.float64, "mixed": torch.float32, "refined": torch.float64}


def _lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return (ctypes.c_double * a.size)(*a.tolist())


def _call_noalloc(mp, g, prec, u, v, w, outs, stream=None):
    L = mp.load_library()
    ptr = lambda t: ctypes.c_void_p(None if t is None else t.data_ptr())
    st = torch.cuda.current_stream() if stream is None else stream
    return L.monc_proj_solve_noalloc(g.nx, g.ny, g.nz, g.dx, g.dy, _dbl(g.dz), _dbl(g.rho_c), _dbl(g.rho_f),
                                     mp.PRECISIONS[prec], ptr(u), ptr(v), ptr(w), ptr(outs[0]), ptr(outs[1]),
                                     ptr(outs[2]), ptr(outs[3]), ctypes.c_void_p(st.cuda_stream))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "refined"])
def test_noalloc_matches_solve_on_two_calls_in_a_row(prec):
    mp = _lib()
    dev = torch.device("cuda", 0)
    dt = DTYPE[prec]
    grids = [W.make_grid(48, 40, 12, 25.0, 20.0, W.geometric_dz(12, 10.0, 100.0)),
             W.make_grid(30, 32, 9, 50.0, 50.0, W.uniform_dz(9, 20.0))]
    for call, g in enumerate(grids):
        u, v, w = (torch.tensor(a, dtype=dt, device=dev) for a in W.random_fields(g, 10 + call, True))
        P = mp.Projector.from_grid(g, prec, dev)
        ref = P.solve(u, v, w, phi=True)
        outs = (torch.full_like(u, np.nan), torch.full_like(v, np.nan), torch.full_like(w, np.nan),
                torch.full_like(u, np.nan))
        rc = _call_noalloc(mp, g, prec, u, v, w, outs)
        assert rc == mp.MONC_PROJ_OK, mp.monc_proj_status_string(rc)
        torch.cuda.synchronize()
        got = torch.cat([o.double().flatten() for o in outs[:3]])
        exp = torch.cat([r.double().flatten() for r in ref[:3]])
        err = float(torch.linalg.norm(got - exp) / torch.linalg.norm(exp))
        assert err <= TOL[prec], f"call {call}: rel err {err:.3e}"
        ephi = float(torch.linalg.norm(outs[3].double() - ref[3].double()) / torch.linalg.norm(ref[3].double()))
        assert ephi <= 10 * TOL[prec]
        P.close()


def test_noalloc_without_phi():
    """phi_out may be NULL, as for monc_proj_solve."""
    mp = _lib()
    dev = torch.device("cuda", 0)
    g = W.make_grid(40, 36, 10, 25.0, 25.0, W.geometric_dz(10, 10.0, 60.0))
    u, v, w = (torch.tensor(a, dtype=torch.float32, device=dev) for a in W.random_fields(g, 7, True))
    P = mp.Projector.from_grid(g, "mixed", dev)
    ref = P.solve(u, v, w)
    outs = (torch.full_like(u, np.nan), torch.full_like(v, np.nan), torch.full_like(w, np.nan), None)
    rc = _call_noalloc(mp, g, "mixed", u, v, w, outs)
    assert rc == mp.MONC_PROJ_OK, mp.monc_proj_status_string(rc)
    torch.cuda.synchronize()
    got = torch.cat([o.double().flatten() for o in outs[:3]])
    exp = torch.cat([r.double().flatten() for r in ref[:3]])
    assert float(torch.linalg.norm(got - exp) / torch.linalg.norm(exp)) <= TOL["mixed"]
    P.close()


def test_noalloc_refuses_a_capturing_stream():
    """Its table upload reads host memory owned by the call alone, so a
    stream under graph capture is refused before anything is enqueued."""
    mp = _lib()
    dev = torch.device("cuda", 0)
    g = W.make_grid(16, 16, 4, 25.0, 25.0, W.uniform_dz(4, 10.0))
    u = torch.zeros((4, 16, 16), dtype=torch.float32, device=dev)
    w = torch.zeros((5, 16, 16), dtype=torch.float32, device=dev)
    outs = (torch.empty_like(u), torch.empty_like(u), torch.empty_like(w), None)
    side = torch.cuda.Stream(device=dev)
    x = torch.zeros(8, device=dev)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        x.add_(1.0)
        rc = _call_noalloc(mp, g, "mixed", u, u, w, outs, stream=side)
    assert rc == mp.MONC_PROJ_EUNSUPPORTED
    graph.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    # outside the capture the same call runs
    rc = _call_noalloc(mp, g, "mixed", u, u, w, outs)
    assert rc == mp.MONC_PROJ_OK
    torch.cuda.synchronize()


def test_noalloc_rejects_oversized_grid():
    mp = _lib()
    g = W.make_grid(256, 256, 128, 25.0, 25.0, W.uniform_dz(128, 25.0))
    t = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = _call_noalloc(mp, g, "mixed", t, t, t, (t, t, t, t))
    assert rc == mp.MONC_PROJ_ESCRATCH
    assert "static scratch" in mp.monc_proj_status_string(rc)
