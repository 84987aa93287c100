"""Accuracy margins of the mixed path against the FP64 oracle on every workload
of the set: the 64^3 and 256^2 x 128 grids, the 64 instances of the uneven
batch (solved as one batch) and a sample of 20 served requests (solved by the
serving loop), each at <= 1e-5 relative error and <= 1e-6 divergence
residual; the full-size 1024^2 x 256 case is tests/test_z_fullsize.py.

Both readings of the vertical solve run: MONC_PROJ_MIXED (FP32-pair
elimination with FP64 pivots for the near-zero wavenumbers, FP32 for the rest)
and MONC_PROJ_MIXED_Z64 (FP64 elimination on every column).  Small grids are checked against the full
oracle element by element, the others at sampled modes (the oracle solves
each (kx, ky) alone) plus the residual over every cell.  Inputs are FP32
draws that both sides read.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2009_12849_gb300 import workloads as W
from tests.oracle_checks import divergence_residual_levels, sampled_mode_error, sampled_modes

pytestmark = pytest.mark.gpu

ERR, DIV = 1e-5, 1e-6


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def f32(fields):
    return tuple(np.asarray(a, np.float32) for a in fields)


def check(g, ins, outs, full_oracle, extra_modes=10):
    """(relative error, divergence residual) of host outputs against the oracle."""
    u, v, w = (np.asarray(a, np.float64) for a in ins)
    outs = [np.asarray(o, np.float64) for o in outs]
    if full_oracle:
        ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
        a = np.concatenate([x.ravel() for x in outs])
        b = np.concatenate([x.ravel() for x in ref[:3]])
        err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        div = O.divergence_residual(*outs, u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    else:
        kx, ky = sampled_modes(g, extra=extra_modes)
        err = sampled_mode_error(g, u, v, w, outs, kx, ky)
        div = divergence_residual_levels(g, u, v, w, outs)
    return err, div


@pytest.mark.parametrize("prec", ["mixed", "mixed_z64"])
@pytest.mark.parametrize("case", ["proj64", "proj256x128"])
def test_configs(case, prec):
    mp = _mp()
    g, seed, mode = W.workload_64cube() if case == "proj64" else W.workload_256()
    ins = f32(W.random_fields(g, seed, mode))
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, prec, dev)
    out = P.solve(*(torch.from_numpy(a).to(dev) for a in ins))
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    assert P.info()["precision"] == mp.PRECISIONS[prec]
    err, div = check(g, ins, [o.cpu().numpy() for o in out], full_oracle=case == "proj64")
    print(f"{case} {prec}: rel err {err:.2e}, divergence residual {div:.2e}")
    assert err <= ERR and div <= DIV
    P.close()


def test_batch_instances_against_oracle():
    mp = _mp()
    dev = torch.device("cuda", 0)
    inst = W.batch_instances(64, 3)
    grids = [g for g, _ in inst]
    B = mp.BatchProjector(grids, "mixed", dev)
    host = [f32(W.random_fields(g, sd, False)) for g, sd in inst]
    args = []
    for h in host:
        u, v, w = (torch.from_numpy(a).to(dev) for a in h)
        args.append((u, v, w, torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)))
    B.solve(args)
    torch.cuda.synchronize()
    worst = (0.0, 0.0)
    for (g, _), h, a in zip(inst, host, args):
        err, div = check(g, h, [t.cpu().numpy() for t in a[3:6]], full_oracle=g.nx <= 64, extra_modes=4)
        assert err <= ERR and div <= DIV, f"{g.nx}x{g.ny}x{g.nz}: err {err:.2e} div {div:.2e}"
        worst = (max(worst[0], err), max(worst[1], div))
    print(f"64 batch instances: worst rel err {worst[0]:.2e}, worst divergence residual {worst[1]:.2e}")
    B.close()


def test_batch_instances_fp64_elimination():
    """Every eighth batch instance with the FP64 elimination on all columns."""
    mp = _mp()
    dev = torch.device("cuda", 0)
    for g, sd in W.batch_instances(64, 3)[::8]:
        h = f32(W.random_fields(g, sd, False))
        P = mp.Projector.from_grid(g, "mixed_z64", dev)
        out = P.solve(*(torch.from_numpy(a).to(dev) for a in h))
        torch.cuda.synchronize()
        err, div = check(g, h, [o.cpu().numpy() for o in out], full_oracle=g.nx <= 64, extra_modes=4)
        assert err <= ERR and div <= DIV, f"{g.nx}x{g.ny}x{g.nz}: err {err:.2e} div {div:.2e}"
        P.close()


def test_served_requests_against_oracle():
    """20 requests of the serving recipe (distinct sizes spread over the
    envelope), served by the loop, checked one by one."""
    mp = _mp()
    from paper_2009_12849_gb300 import serve as S
    dev = torch.device("cuda", 0)
    pool = sorted(S.requests_from_recipe(4000, 2000.0, 4), key=lambda r: r.points)
    seen, picked = set(), []
    for r in pool[:: max(1, len(pool) // 200)]:
        if (r.n, r.nz) not in seen:
            seen.add((r.n, r.nz))
            picked.append(r)
    idx = np.linspace(0, len(picked) - 1, 20).round().astype(int)
    reqs = [picked[i] for i in sorted(set(idx))]
    assert len(reqs) >= 20
    # replay them as a fast stream (all overlapping on the device)
    reqs = [S.Request(t=0.0005 * i, n=r.n, nz=r.nz, seed=r.seed) for i, r in enumerate(reqs)]
    srv = S.ProjectionServer(dev, hbm_budget=40e9, slots=8)
    stats = srv.run(reqs, keep_outputs=True)
    assert stats["served"] == len(reqs)
    gen = torch.Generator(device=dev)
    worst = (0.0, 0.0)
    for r, out in zip(sorted(reqs, key=lambda q: q.t), stats["outputs"]):
        g = W.serving_grid(r.n, r.nz)
        ins = [t.cpu().numpy() for t in S.make_fields(r, torch.float32, dev, gen)]
        err, div = check(g, ins, [t.cpu().numpy() for t in out], full_oracle=False, extra_modes=4)
        assert err <= ERR and div <= DIV, f"{r.n}^2 x {r.nz}: err {err:.2e} div {div:.2e}"
        worst = (max(worst[0], err), max(worst[1], div))
    print(f"{len(reqs)} served requests: worst rel err {worst[0]:.2e}, worst divergence residual {worst[1]:.2e}")
    srv.close()


@pytest.mark.parametrize("prec", ["mixed", "mixed_z64"])
def test_ill_conditioned_columns(prec):
    """A grid whose columns are badly conditioned: wide cells (dx = dy = 200 m,
    so |lambda| <= 2e-4 against a vertical operator bound near 1), 256 levels
    from 2 m at the ground to 100 m at the top (kappa up to ~2e6).  Every
    column falls below the near-zero threshold and takes the FP32-pair path;
    against the full FP64 oracle at the mixed tolerances."""
    mp = _mp()
    nz = 256
    g = W.make_grid(48, 40, nz, 200.0, 200.0, W.geometric_dz(nz, 2.0, 100.0))
    ins = f32(W.random_fields(g, 31, True))
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, prec, dev)
    info = P.info()
    out = P.solve(*(torch.from_numpy(a).to(dev) for a in ins))
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    err, div = check(g, ins, [o.cpu().numpy() for o in out], full_oracle=True)
    print(f"ill-conditioned {prec}: {info['fp64_columns']} of {info['total_columns']} near-zero columns, "
          f"rel err {err:.2e}, divergence residual {div:.2e}")
    if prec == "mixed":
        assert info["fp64_columns"] > info["total_columns"] // 4
    assert err <= ERR and div <= DIV
    P.close()
