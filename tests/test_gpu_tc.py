"""The tensor-core split-precision forward column transforms (two radix-32
stages of the length-1024 y transform as tcgen05 matrix products) against the
FP64 oracle, inside the mixed solve.

- BF16 x 6 (MONC_PROJ_TC=2): three BF16 parts per operand, six products
  accumulated in FP32 -- FP32-level accuracy, held to the mixed path's
  tolerances (1e-5 relative error, 1e-6 divergence residual);
- TF32 x 3 (MONC_PROJ_TC=1): two TF32 parts, three products -- about 2^-21
  relative error per product, which puts the divergence residual at about
  1e-6: held to 1e-5 and 2e-6.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2009_12849_gb300 import workloads as W
from tests.oracle_checks import divergence_residual_levels, sampled_mode_error, sampled_modes

pytestmark = pytest.mark.gpu


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


TOL = {1: (1e-5, 2e-6), 2: (1e-5, 1e-6)}


def _solve(g, ins, monkeypatch, tc):
    mp = _mp()
    monkeypatch.setenv("MONC_PROJ_TC", str(tc))
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, "mixed", dev)
    mp.monc_proj_profile(P.plan, 1)
    out = P.solve(*(torch.from_numpy(a).to(dev) for a in ins))
    torch.cuda.synchronize()
    st = P.sync_status()
    prof = mp.monc_proj_profile_read(P.plan)
    ran = {k for k, t in prof["phases"].items() if t > 0}
    res = [o.double().cpu().numpy() for o in out]
    P.close()
    return res, st, ran


@pytest.mark.parametrize("fmt", [2, 1])
@pytest.mark.parametrize("shape", [(64, 1024, 3), (1024, 1024, 2), (250, 1024, 4)])
def test_tc_columns_against_full_oracle(shape, fmt, monkeypatch):
    nx, ny, nz = shape
    g = W.make_grid(nx, ny, nz, 10.0, 10.0, W.geometric_dz(nz, 5.0, 50.0))
    ins = tuple(np.asarray(a, np.float32) for a in W.random_fields(g, 6, True))
    got, st, ran = _solve(g, ins, monkeypatch, tc=fmt)
    assert st == 0
    assert "fwd_cols_tc" in ran and "fwd_cols" not in ran, ran
    u, v, w = (a.astype(np.float64) for a in ins)
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    a = np.concatenate([x.ravel() for x in got])
    b = np.concatenate([x.ravel() for x in ref[:3]])
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    div = O.divergence_residual(*got, u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    print(f"tensor-core columns, format {fmt}, {shape}: rel err {err:.2e}, divergence residual {div:.2e}")
    assert err <= TOL[fmt][0] and div <= TOL[fmt][1]


@pytest.mark.parametrize("fmt", [2, 1])
def test_tc_columns_at_1024_sampled(fmt, monkeypatch):
    g = W.make_grid(1024, 1024, 24, 10.0, 10.0, W.geometric_dz(24, 5.0, 50.0))
    ins = W.random_fields_f32(g, 2, True)
    got, st, ran = _solve(g, ins, monkeypatch, tc=fmt)
    assert st == 0 and "fwd_cols_tc" in ran
    u, v, w = (np.asarray(a, np.float64) for a in ins)
    kx, ky = sampled_modes(g)
    err = sampled_mode_error(g, u, v, w, got, kx, ky)
    div = divergence_residual_levels(g, u, v, w, got)
    print(f"tensor-core columns, format {fmt}, 1024^2 x 24: rel err {err:.2e} at {len(kx)} modes, "
          f"divergence residual {div:.2e}")
    assert err <= TOL[fmt][0] and div <= TOL[fmt][1]
