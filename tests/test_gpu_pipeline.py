"""The persistent pipelines of the transforms (opt-in, MONC_PROJ_PIPE=1: one
kernel per transform, row and column tasks taken by ticket with per-level
counters, the intermediate spectra handed over in L2 and discarded once read)
against the oracle and against the one-launch-per-pass path.

The pipelines run the same task bodies with the same arithmetic per element,
so they must equal the one-launch-per-pass solve bit for bit; that solve is
the one the parity tests pin to the FP64 oracle.  Lags leave ragged ends.
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


def solve(g, u, v, w, phi=True, inplace=False):
    """Mixed solve; returns the outputs (FP64 numpy) and the phases that ran."""
    mp = _mp()
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, "mixed", dev)
    tu, tv, tw = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (u, v, w))
    mp.monc_proj_profile(P.plan, 1)
    res = P.solve(tu, tv, tw, out=(tu, tv, tw) if inplace else None, phi=phi)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    prof = mp.monc_proj_profile_read(P.plan)
    ran = {k for k, t in prof["phases"].items() if t > 0}
    out = [r.double().cpu().numpy() for r in res]
    P.close()
    return out, ran


def f32_fields(g, seed):
    u, v, w = W.random_fields(g, seed, True)
    return tuple(a.astype(np.float32).astype(np.float64) for a in (u, v, w))


def use(monkeypatch, variant, a=0, b=0):
    """Select the pipelines (lags a, b) or the one-launch-per-pass kernels."""
    if variant == "pipe":
        monkeypatch.setenv("MONC_PROJ_PIPE", "1")
        monkeypatch.setenv("MONC_PROJ_PIPE_LAG_FWD", str(a))
        monkeypatch.setenv("MONC_PROJ_PIPE_LAG_INV", str(b))
        return {"fwd_pipe", "inv_pipe"}
    monkeypatch.setenv("MONC_PROJ_PIPE", "0")
    return {"fwd_rows", "inv_rows"}


@pytest.mark.parametrize("shape,a,b", [((256, 256, 7), 3, 2), ((512, 512, 5), 2, 3), ((1024, 1024, 3), 1, 1),
                                       ((256, 256, 2), 4, 4), ((512, 512, 1), 2, 2)])
def test_pipe_vs_oracle(shape, a, b, monkeypatch):
    nx, ny, nz = shape
    want = use(monkeypatch, "pipe", a, b)
    g = W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))
    u, v, w = f32_fields(g, 21)
    got, ran = solve(g, u, v, w)
    assert want <= ran, ran
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    a_ = np.concatenate([x.ravel() for x in got[:3]])
    b_ = np.concatenate([x.ravel() for x in ref[:3]])
    err = np.linalg.norm(a_ - b_) / np.linalg.norm(b_)
    assert err < 1e-5, f"rel err {err:.3e}"
    div = O.divergence_residual(*got[:3], u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert div < 1e-6, f"divergence residual {div:.3e}"
    assert np.all(got[2][0] == 0) and np.all(got[2][-1] == 0)


@pytest.mark.parametrize("variant,shape,a,b,phi,inplace", [
    ("pipe", (1024, 1024, 9), 4, 2, False, False), ("pipe", (1024, 1024, 5), 3, 3, True, True),
    ("pipe", (512, 512, 13), 4, 2, True, False), ("pipe", (256, 256, 6), 5, 1, False, True),
    ("pipe", (1024, 1024, 4), 9, 9, True, False)])
def test_equals_one_launch_per_pass_bitwise(variant, shape, a, b, phi, inplace, monkeypatch):
    nx, ny, nz = shape
    g = W.make_grid(nx, ny, nz, 10.0, 10.0, W.geometric_dz(nz, 5.0, 50.0))
    u, v, w = f32_fields(g, 2)
    use(monkeypatch, "plain")
    plain, ran0 = solve(g, u, v, w, phi=phi, inplace=inplace)
    assert {"fwd_rows", "inv_rows"} <= ran0, ran0
    want = use(monkeypatch, variant, a, b)
    other, ran1 = solve(g, u, v, w, phi=phi, inplace=inplace)
    assert want <= ran1, ran1
    for x, y in zip(plain, other):
        assert np.array_equal(x, y)


def test_repeated_solves_on_one_workspace(monkeypatch):
    """Tickets and counters are cleared per solve: many solves back to back
    on one plan and workspace give the same result every time and no
    timeout."""
    mp = _mp()
    use(monkeypatch, "pipe", 2, 2)
    g = W.make_grid(256, 256, 11, 25.0, 25.0, W.geometric_dz(11, 10.0, 60.0))
    u, v, w = f32_fields(g, 4)
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, "mixed", dev)
    tu, tv, tw = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (u, v, w))
    first = P.solve(tu, tv, tw)
    for _ in range(20):
        again = P.solve(tu, tv, tw)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    for x, y in zip(first, again):
        assert torch.equal(x, y)
    P.close()
