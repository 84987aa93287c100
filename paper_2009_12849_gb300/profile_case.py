"""Run a few projections of one synthetic grid, for profiling under ncu.

    python -m paper_2009_12849_gb300.profile_case --grid 512,512,64 --precision mixed --solves 3
    python -m paper_2009_12849_gb300.profile_case --grid 256,256,128 --krylov 3
    python -m paper_2009_12849_gb300.profile_case --batch 2 [--per-instance]

Inputs are the seeded workload recipe (N(0,1) plus the large-scale mode,
dx = dy = 10 m, dz geometric 5 -> 50 m).  Prints the wall time per solve.
With --krylov N each solve is N BiCGStab iterations (vertical-line
preconditioner, no stopping test) instead of the FFT projection.  With
--batch N the 64-instance uneven batch of the benchmark (seed 3) is solved N
times with grouped launches (or per-instance launches with --per-instance).
"""
from __future__ import annotations

import argparse
import time

import torch

from paper_2009_12849_gb300 import monc_proj as MP
from paper_2009_12849_gb300 import workloads as W


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", default="512,512,64")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "refined", "mixed_z64"])
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--krylov", type=int, default=0, help="BiCGStab iterations per solve (0: FFT solve)")
    ap.add_argument("--batch", type=int, default=0, help="solve the 64-instance batch this many times")
    ap.add_argument("--per-instance", action="store_true", help="batch: per-instance launches")
    a = ap.parse_args()
    if a.batch > 0:
        return run_batch(a.batch, not a.per_instance)
    nx, ny, nz = (int(x) for x in a.grid.split(","))
    g = W.make_grid(nx, ny, nz, 10.0, 10.0, W.geometric_dz(nz, 5.0, 50.0))
    dt = torch.float32 if a.precision in ("mixed", "mixed_z64") else torch.float64
    dev = torch.device("cuda", 0)
    u, v, w = (torch.from_numpy(x).to(dev, dt) for x in W.random_fields_f32(g, 2, True))
    P = MP.Projector.from_grid(g, a.precision, dev)
    out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
    ws = None
    if a.krylov > 0:
        ws = torch.empty(MP.monc_proj_krylov_workspace_size(P.plan), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.solves):
        if a.krylov > 0:
            P.solve_krylov(u, v, w, 0.0, a.krylov, "line", out=out, workspace=ws)
        else:
            P.solve(u, v, w, out=out)
    torch.cuda.synchronize()
    dt_s = (time.perf_counter() - t0) / a.solves
    st = P.sync_status()
    kind = f" krylov x{a.krylov}" if a.krylov > 0 else ""
    print(f"{nx}x{ny}x{nz} {a.precision}{kind}: {dt_s * 1e3:.3f} ms/solve (wall), status {st}")
    if st != 0:
        raise SystemExit(1)


def run_batch(reps, grouped):
    dev = torch.device("cuda", 0)
    inst = W.batch_instances(64, 3)
    B = MP.BatchProjector([g for g, _ in inst], "mixed", dev)
    args = []
    for g, sd in inst:
        u, v, w = (torch.from_numpy(x).to(dev) for x in W.random_fields_f32(g, sd, False))
        args.append((u, v, w, torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        B.solve(args, grouped=grouped)
    torch.cuda.synchronize()
    dt_s = (time.perf_counter() - t0) / reps
    st = max(MP.monc_proj_sync_status(p.handle) for p in B.plans)
    print(f"batch of 64 ({'grouped' if grouped else 'per-instance'}): {dt_s * 1e3:.3f} ms/batch (wall), status {st}")
    B.close()
    if st != 0:
        raise SystemExit(1)


if __name__ == "__main__":
    main()
