"""Full-size parity: the 1024x1024x256 mixed workload in the launch
configuration bench.py times (default plan shapes, out-of-place solve),
checked against the FP64 oracle where it can compute outputs one by one.

The projection decouples by horizontal wavenumber, so the oracle solves the
sampled modes (kx, ky) alone (``project_modes``) and the GPU output's DFT at
those modes is compared with them (relative L2 over u, v, w, tolerance 1e-5);
the divergence residual is taken over every cell in FP64 on the host
(tolerance 1e-6).  The inputs are FP32 draws that both sides read.  The
checker itself is exercised on the CPU against the full oracle at a small size.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2009_12849_gb300 import workloads as W
from tests.oracle_checks import divergence_residual_levels, sampled_mode_error, sampled_modes


def test_checker_against_the_full_oracle():
    # the sampled-mode checker on a small grid: the full oracle's own output
    # passes at rounding level, and a planted error in one mode fails it
    g = W.make_grid(24, 20, 6, 10.0, 10.0, W.geometric_dz(6, 5.0, 50.0))
    u, v, w = (a.astype(np.float64) for a in W.random_fields_f32(g, 2, True))
    uo, vo, wo, _ = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    kx, ky = sampled_modes(g)
    assert sampled_mode_error(g, u, v, w, (uo, vo, wo), kx, ky) < 1e-12
    assert divergence_residual_levels(g, u, v, w, (uo, vo, wo)) < 1e-12
    x = np.arange(g.nx) * 2 * np.pi / g.nx
    bad = uo + 1e-3 * np.cos(x)[None, None, :]            # mode (1, 0), sampled
    assert sampled_mode_error(g, u, v, w, (bad, vo, wo), kx, ky) > 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["mixed", "mixed_z64"])
def test_1024x256_mixed_sampled_modes_and_divergence(prec):
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj as mp
    g, seed, mode = W.workload_1024()
    u_h, v_h, w_h = W.random_fields_f32(g, seed, mode)
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, prec, dev)
    u, v, w = (torch.from_numpy(a).to(dev) for a in (u_h, v_h, w_h))
    out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
    P.solve(u, v, w, out=out)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    outs = [t.cpu().numpy() for t in out]
    P.close()
    del u, v, w, out
    kx, ky = sampled_modes(g)
    err = sampled_mode_error(g, u_h, v_h, w_h, outs, kx, ky)
    div = divergence_residual_levels(g, u_h, v_h, w_h, outs)
    print(f"1024x1024x256 {prec}: rel err {err:.3e} at {len(kx)} modes, divergence residual {div:.3e}")
    assert err < 1e-5
    assert div < 1e-6
    assert np.all(outs[2][0] == 0) and np.all(outs[2][-1] == 0)
