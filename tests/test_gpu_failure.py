"""Failure detection on the GPU without a fault: a bounded wait that runs out
and an allocator supplied by the caller.

MONC_PROJ_SPIN_LIMIT=0 (read when the plan is made) makes the persistent
pipelines' dependency waits give up at the first poll that finds their
producer tasks unfinished; with a lag of zero levels the first consumer tasks
always find them unfinished.  The kernels then latch the timeout bit and run
to the end (their indices never depend on the data), the host reads
MONC_PROJ_ETIMEOUT from monc_proj_sync_status, and the context stays usable:
the status is cleared and the next plan solves correctly.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2009_12849_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def test_wait_that_runs_out_reports_timeout_and_the_context_recovers(monkeypatch):
    mp = _mp()
    dev = torch.device("cuda", 0)
    g = W.make_grid(256, 256, 8, 25.0, 25.0, W.geometric_dz(8, 10.0, 60.0))
    u, v, w = (a.astype(np.float32).astype(np.float64) for a in W.random_fields(g, 3, True))
    tu, tv, tw = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (u, v, w))
    for k, val in (("MONC_PROJ_PIPE", "1"), ("MONC_PROJ_SPIN_LIMIT", "0"), ("MONC_PROJ_PIPE_LAG_FWD", "0"),
                   ("MONC_PROJ_PIPE_LAG_INV", "0")):
        monkeypatch.setenv(k, val)
    P = mp.Projector.from_grid(g, "mixed", dev)
    P.solve(tu, tv, tw)
    torch.cuda.synchronize()
    assert P.sync_status() == mp.MONC_PROJ_ETIMEOUT
    assert P.sync_status() == mp.MONC_PROJ_OK          # read once, then cleared
    P.close()
    for k in ("MONC_PROJ_PIPE", "MONC_PROJ_SPIN_LIMIT", "MONC_PROJ_PIPE_LAG_FWD", "MONC_PROJ_PIPE_LAG_INV"):
        monkeypatch.delenv(k)
    Q = mp.Projector.from_grid(g, "mixed", dev)
    out = Q.solve(tu, tv, tw)
    torch.cuda.synchronize()
    assert Q.sync_status() == mp.MONC_PROJ_OK
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    got = np.concatenate([o.double().cpu().numpy().ravel() for o in out])
    exp = np.concatenate([r.ravel() for r in ref[:3]])
    assert np.linalg.norm(got - exp) / np.linalg.norm(exp) < 1e-5
    Q.close()


def test_caller_allocator_serves_plan_tables():
    mp = _mp()
    dev = torch.device("cuda", 0)
    live = {}

    def alloc(n):
        ptr = torch.cuda.caching_allocator_alloc(n, device=0)
        live[ptr] = n
        return ptr

    def release(ptr):
        torch.cuda.caching_allocator_delete(ptr)
        live.pop(ptr)

    g = W.make_grid(96, 64, 10, 25.0, 25.0, W.geometric_dz(10, 10.0, 60.0))
    u, v, w = (torch.tensor(a, dtype=torch.float32, device=dev) for a in W.random_fields(g, 5, True))
    P0 = mp.Projector.from_grid(g, "mixed", dev)
    ref = P0.solve(u, v, w)
    mp.monc_proj_set_allocator(alloc, release)
    try:
        P = mp.Projector.from_grid(g, "mixed", dev)
        assert len(live) == 1
        out = P.solve(u, v, w)
        torch.cuda.synchronize()
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
        P.close()
        assert live == {}
    finally:
        mp.monc_proj_set_allocator()
    P0.close()
