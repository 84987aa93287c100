#!/usr/bin/env python3
"""Benchmark of the anelastic pressure projection on one GB300.

One step = one full projection (divergence, forward 2D FFT per level,
vertical tridiagonal solve per wavenumber, inverse FFT, gradient correction)
of the 1024 x 1024 x 256 mixed-precision workload (dx = dy = 10 m, dz 5 -> 50 m
geometric, rho0 = 1.2 exp(-z/8000 m), N(0,1) velocities plus a smooth
large-scale mode, seed 2).  Inputs (1.07 GB per field) are larger than L2,
so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --impl reference the FP64 CPU oracle is
timed on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "projection Mpts/s, mixed vs FP64 on one GB300 at <=1e-5 rel err; p50/p99 latency"
UNIT = "Mpts/s"
WORKLOAD = "proj1024x256_mixed"
FALLBACK_HBM_GBS = 6800.0
CPU_SAMPLE_LEVELS = 48          # oracle sample for the cpu_baseline key
REF_SAMPLE_LEVELS = 4           # oracle sample per step of --impl reference


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-check", action="store_true", help="skip the accuracy check")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batch measurement")
    ap.add_argument("--no-refined", action="store_true", help="skip the refinement (mixed passes on FP64 fields) leg")
    ap.add_argument("--no-krylov", action="store_true", help="skip the BiCGStab pressure-solver leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 64^3 and 256^2 x 128 legs (the other configurations of the workload set)")
    ap.add_argument("--e2e-lanes", type=int, default=4,
                    help="streams (each with its own staging area and workspace) taking turns in the e2e leg")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the serving measurement (0 skips it; the full recipe is 10000)")
    return ap.parse_args()


def workload_grid():
    from paper_2009_12849_gb300 import workloads as W
    g, seed, mode = W.workload_1024()
    return g, seed, mode


def sample_grid(g, nlev):
    from paper_2009_12849_gb300 import workloads as W
    return W.make_grid(g.nx, g.ny, nlev, g.dx, g.dy, g.dz[:nlev])


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"monc_clocks_{os.getpid()}.csv")

    INTERVAL_MS = 50

    def start(self):
        """Start sampling and wait (up to 5 s) for the first sample, so the
        sampler is running when the timed region begins."""
        self.window = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t_end = time.time() + 5.0
        while time.time() < t_end:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def mark(self, t0: float, t1: float):
        """Host times (time.time()) bracketing the timed region."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        # samples inside the timed region (plus one sampling interval either
        # side); if it was too short to catch any, the nearest three
        window = "timed region"
        sel = rows
        if self.window is not None and rows:
            pad = self.INTERVAL_MS / 1000.0
            sel = [r for r in rows if self.window[0] - pad <= r[0] <= self.window[1] + pad]
            if not sel:
                mid = 0.5 * (self.window[0] + self.window[1])
                sel = sorted(rows, key=lambda r: abs(r[0] - mid))[:3]
                window = "nearest samples"
        reasons = set()
        for r in sel:
            for nm, val in zip(names, r[3]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median([r[1] for r in sel]) if sel else None,
                "sm_max_mhz": max(r[2] for r in sel) if sel else None,
                "reasons": sorted(reasons), "samples": len(sel), "window": window,
                "interval_ms": self.INTERVAL_MS}


# ------------------------------------------------------------------ roofline bookkeeping

def phase_bytes(g, phase: str, elem: int) -> float:
    """Algorithmic DRAM bytes of one launch of a phase (inputs read once, outputs
    written once).  elem = bytes of one real value (4 mixed, 8 FP64)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    n = nx * ny * nz
    nw = nx * ny * (nz + 1)
    spec = (nx // 2 + 1) * ny * nz * 2 * elem      # one half-spectrum array
    fields_in = (2 * n + nw) * elem
    return {
        "fwd_rows": fields_in + spec,                   # u,v,w -> x-spectrum
        "fwd_cols": 2 * spec,                           # x-spectrum -> D^
        "tridiag": 3 * spec,                            # D^ -> p^, gz^
        "inv_cols": 5 * spec,                           # p^, gz^ -> 3 channel spectra
        "inv_rows": 3 * spec + 2 * fields_in,           # 3 spectra + u,v,w -> u,v,w
        "fwd_fused": fields_in + spec,                  # u,v,w -> D^ (x-spectra stay in L2)
        "inv_fused": 2 * spec + 2 * fields_in,          # p^, gz^, u,v,w -> u,v,w
        "fwd_pipe": fields_in + spec,                   # u,v,w -> D^ (x-spectra handed off in L2)
        "inv_pipe": 2 * spec + 2 * fields_in,           # p^, gz^, u,v,w -> u,v,w (channel spectra in L2)
    }[phase]


def path_bytes_per_point(elem: int) -> float:
    """Algorithmic bytes per grid point of the whole projection: read u,v,w (3
    reals), write D^ (a half spectrum: 1 real per point), read D^, write p^,
    read p^, read u,v,w again, write u,v,w -- 13 reals per point (52 B in
    FP32).  The spectral w-gradient the mixed path also writes and reads is
    not counted, nor any hand-off between the passes of a 2D transform."""
    return 13.0 * elem


# Dense FP64 arithmetic rate of one GB300 (nominal; the FP64 path is bound by it)
FP64_PEAK_TFLOPS = 1.25


def fp64_flops_per_point(nx, ny):
    """Algorithmic FP64 flops per grid point of one projection: the forward
    real 2D transform and the three inverse real 2D transforms at 5 n log2 n per
    complex transform of n points (a real transform of n points as half of one:
    2.5 log2(nx ny) per point each, 10 log2(nx ny) for the four), the vertical
    solve at 21 flops per complex column and level over nx/2 + 1 of nx columns
    (11 per point), the divergence (10) and the correction (3)."""
    return 10.0 * math.log2(nx * ny) + 24.0


def recorded_path_traffic():
    """DRAM bytes of one whole step (all five kernels) from the committed ncu
    summary, or None if the kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("csrc_hash") != csrc_hash() or rec.get("workload") != WORKLOAD:
        return None
    ks = rec.get("kernels", {})
    vals = [k.get("dram_bytes_per_launch") for k in ks.values()]
    return None if not vals or any(v is None for v in vals) else float(sum(vals))


# Sources of the BiCGStab solver: no kernel of the FFT path includes them, so
# they are left out of the hash that dates the recorded DRAM traffic.
KRYLOV_SOURCES = ("kern_krylov.cu", "krylov.h")


def csrc_hash() -> str:
    """Hash of the sources the FFT path's kernels are built from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2009_12849_gb300", "csrc")
    for fn in sorted(os.listdir(d)):
        if fn in KRYLOV_SOURCES:
            continue
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    if the kernels changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    if rec.get("csrc_hash") != csrc_hash() or rec.get("workload") != WORKLOAD:
        return None
    k = rec.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        rec = json.load(open(path))
        v = rec.get("hbm_gbs")
        if v:
            return float(v), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ CPU oracle timing

def time_oracle(g, seed, mode, nlev, repeats=1):
    """Time the FP64 oracle on the first nlev levels of the workload."""
    import oracle as O
    from paper_2009_12849_gb300 import workloads as W
    gs = sample_grid(g, nlev)
    u, v, w = (a.astype(np.float64) for a in W.random_fields_f32(gs, seed, mode))
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        O.project(u, v, w, gs.dx, gs.dy, gs.dz, gs.rho_c, gs.rho_f)
        times.append(time.perf_counter() - t0)
    return gs, times


def cpu_threads():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


# ------------------------------------------------------------------ replicas (N > 1)

def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values: the slowest replica's time."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(seed: int, rank: int) -> int:
    """Each rank projects its own replica of the workload (independent inputs)."""
    return seed + 1000 * rank


def job_throughput(world: int, npts: int, ms: float) -> float:
    """Whole-job Mpts/s: the points all replicas projected over the slowest one's time."""
    return world * npts / (ms * 1e-3) / 1e6


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    if rank != 0:
        return
    g, seed, mode = workload_grid()
    gs, _ = time_oracle(g, seed, mode, REF_SAMPLE_LEVELS, repeats=max(args.warmup, 0) or 1)
    _, times = time_oracle(g, seed, mode, REF_SAMPLE_LEVELS, repeats=args.steps)
    pts = gs.nx * gs.ny * gs.nz
    value = pts * len(times) / sum(times) / 1e6
    sample = (f"{gs.nx}x{gs.ny}x{gs.nz}: the first {gs.nz} levels of the {g.nx}x{g.ny}x{g.nz} workload "
              f"per step (same dx, dz, rho0, seed)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": g.nx, "ny": g.ny, "nz": g.nz, "sample_levels": gs.nz},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2009_12849_gb300 import workloads as W
    from paper_2009_12849_gb300 import monc_proj as MP

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    g, seed, mode = workload_grid()
    npts = g.nx * g.ny * g.nz
    # each rank projects its own replica of the workload (independent problems)
    u_h, v_h, w_h = W.random_fields_f32(g, replica_seed(seed, rank), mode)
    u = torch.from_numpy(u_h).to(dev)
    v = torch.from_numpy(v_h).to(dev)
    w = torch.from_numpy(w_h).to(dev)
    P = MP.Projector.from_grid(g, "mixed", dev)
    out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        P.solve(u, v, w, out=out)
    torch.cuda.synchronize(dev)
    if P.sync_status() != 0:
        raise SystemExit("device error during warm-up")

    clocks = ClockSampler(local_rank)
    MP.monc_proj_profile(P.plan, True)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_region0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        P.solve(u, v, w, out=out)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(t_region0, time.time())
    barrier()
    clk = clocks.stop()
    MP.monc_proj_profile(P.plan, False)
    prof = MP.monc_proj_profile_read(P.plan)
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    value = job_throughput(world, npts, ms)
    status = P.sync_status()

    # ---- end to end through the C ABI with host buffers (monc_proj_solve_host):
    # every step copies its fields in from page-locked host memory, projects
    # them and copies them back; --e2e-lanes streams with their own staging
    # areas and workspaces take turns, so one step's copies back overlap the
    # next step's copies in
    uh = torch.from_numpy(u_h).pin_memory()
    vh = torch.from_numpy(v_h).pin_memory()
    wh = torch.from_numpy(w_h).pin_memory()
    lanes = []
    nl = max(1, args.e2e_lanes)
    for li in range(nl):
        outs_h = tuple(torch.empty_like(x).pin_memory() for x in (uh, vh, wh))
        stg = torch.empty(MP.monc_proj_host_staging_size(P.plan), dtype=torch.uint8, device=dev)
        ws = P.workspace if li == 0 else torch.empty_like(P.workspace)
        lanes.append((torch.cuda.Stream(dev), outs_h, stg, ws))
    e2e_steps = max(2 * nl, min(args.steps, 20))

    def e2e_step(i):
        s_, o_, stg_, ws_ = lanes[i % nl]
        MP.monc_proj_solve_host(P.plan, uh, vh, wh, o_[0], o_[1], o_[2], None, stg_, ws_, s_)

    # every lane's staging area and host buffers are used several times
    # before the timed steps (the first passes over freshly page-locked host
    # memory run slower)
    for i in range(max(3 * nl, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(lanes[0][0])
    for ln in lanes[1:]:
        ln[0].wait_event(e0)
    for i in range(e2e_steps):
        e2e_step(i)
    for ln in lanes[1:]:
        lanes[0][0].wait_stream(ln[0])
    e1.record(lanes[0][0])
    torch.cuda.synchronize(dev)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world, dev)
    e2e_match = bool(torch.equal(lanes[0][1][0], out[0].cpu()))
    del lanes
    field_bytes = sum(x.numel() * x.element_size() for x in (uh, vh, wh))

    # ---- FP64 path on the same grid (the plain FP64 GPU path to beat)
    fp64 = None
    if not args.no_fp64:
        P64 = MP.Projector.from_grid(g, "fp64", dev)
        u64, v64, w64 = u.double(), v.double(), w.double()
        o64 = (torch.empty_like(u64), torch.empty_like(v64), torch.empty_like(w64))
        for _ in range(2):
            P64.solve(u64, v64, w64, out=o64)
        torch.cuda.synchronize(dev)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        n64 = 5
        a0.record(stream)
        for _ in range(n64):
            P64.solve(u64, v64, w64, out=o64)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = a0.elapsed_time(a1) / n64
        fp64 = {"value": npts / (ms64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms64, "steps": n64}
        fpp = fp64_flops_per_point(g.nx, g.ny)
        ach = fpp * npts / (ms64 * 1e-3) / 1e12
        fp64["roofline"] = {"bound": "alu", "flops_per_point": fpp, "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                            "peak_kind": "nominal FP64 FMA rate of a GB300", "unit": "TFLOP/s",
                            "frac": ach / FP64_PEAK_TFLOPS}
        if not args.no_check and rank == 0:
            fp64["accuracy"] = verify(g, (u64, v64, w64), o64)
        P64.close()

    # ---- the vertical solve with FP64 elimination on every column (FP32
    # storage): the reading of a3 in which no column runs FP32 arithmetic
    # (the default: FP32 elimination, near-zero-wavenumber columns in FP32-pair
    # arithmetic with FP64 pivots from the plan)
    a3_variants = {"fp32_with_pair_near_zero": {"ms_per_step": ms, "value": value, "unit": UNIT,
                                                "near_zero_columns": P.info().get("fp64_columns"),
                                                "columns": P.info().get("total_columns")}}
    if not args.no_fp64:
        PZ = MP.Projector.from_grid(g, "mixed_z64", dev)
        oz = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        for _ in range(2):
            PZ.solve(u, v, w, out=oz)
        torch.cuda.synchronize(dev)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        nzr = 5
        MP.monc_proj_profile(PZ.plan, True)
        a0.record(stream)
        for _ in range(nzr):
            PZ.solve(u, v, w, out=oz)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        MP.monc_proj_profile(PZ.plan, False)
        pz = MP.monc_proj_profile_read(PZ.plan)
        msz = a0.elapsed_time(a1) / nzr
        leg = {"ms_per_step": msz, "value": npts / (msz * 1e-3) / 1e6, "unit": UNIT,
               "tridiag_ms": pz["phases"].get("tridiag", 0.0) / max(pz["solves"], 1),
               "fp64_columns": PZ.info().get("fp64_columns")}
        if not args.no_check and rank == 0:
            leg["accuracy"] = verify(g, (u, v, w), oz, o64)
        a3_variants["fp64_all_columns"] = leg
        PZ.close()
        del oz

    # ---- the forward column transforms on the tensor cores (split TF32 x 3
    # and BF16 x 6, opt-in): time and accuracy of the whole mixed solve
    tensor_cols = None
    if not args.no_fp64:
        tensor_cols = {}
        for fmt, name in ((1, "tf32x3"), (2, "bf16x6")):
            os.environ["MONC_PROJ_TC"] = str(fmt)
            PT = MP.Projector.from_grid(g, "mixed", dev)
            os.environ.pop("MONC_PROJ_TC", None)
            ot = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
            for _ in range(2):
                PT.solve(u, v, w, out=ot)
            torch.cuda.synchronize(dev)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            MP.monc_proj_profile(PT.plan, True)
            a0.record(stream)
            for _ in range(5):
                PT.solve(u, v, w, out=ot)
            a1.record(stream)
            torch.cuda.synchronize(dev)
            MP.monc_proj_profile(PT.plan, False)
            pt = MP.monc_proj_profile_read(PT.plan)
            mst = a0.elapsed_time(a1) / 5
            leg = {"ms_per_step": mst, "value": npts / (mst * 1e-3) / 1e6, "unit": UNIT,
                   "fwd_cols_tc_ms": pt["phases"].get("fwd_cols_tc", 0.0) / max(pt["solves"], 1),
                   "device_status": PT.sync_status()}
            if not args.no_check and rank == 0:
                leg["accuracy"] = verify(g, (u, v, w), ot, o64)
            tensor_cols[name] = leg
            PT.close()
            del ot

    # ---- refinement: mixed passes on FP64 fields (FP64-level accuracy)
    refined = None
    if not args.no_fp64 and not args.no_refined:
        PR = MP.Projector.from_grid(g, "refined", dev)
        o_r = (torch.empty_like(u64), torch.empty_like(v64), torch.empty_like(w64))
        for _ in range(2):
            PR.solve(u64, v64, w64, out=o_r)
        torch.cuda.synchronize(dev)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        nr = 5
        a0.record(stream)
        for _ in range(nr):
            PR.solve(u64, v64, w64, out=o_r)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        msr = a0.elapsed_time(a1) / nr
        refined = {"value": npts / (msr * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": msr, "steps": nr,
                   "passes": int(os.environ.get("MONC_PROJ_REFINE_PASSES", 3)), "device_status": PR.sync_status()}
        if not args.no_check and rank == 0:
            refined["accuracy"] = verify(g, (u64, v64, w64), o_r, o64)
        PR.close()
        del o_r

    # ---- accuracy of the timed result: divergence residual, and the error
    # against the FP64 GPU path (which the parity tests pin to the FP64 oracle);
    # the FP64 fields are freed before the batch and serving legs
    check = None
    if not args.no_check and rank == 0:
        check = verify(g, (u, v, w), out, o64 if not args.no_fp64 else None)
    if not args.no_fp64:
        del u64, v64, w64, o64
    torch.cuda.empty_cache()

    # ---- uneven batch of 64 projections (one batched call, and its CUDA-graph replay)
    batch = None
    if not args.no_batch and rank == 0:
        batch = measure_batch(dev, stream, check=not args.no_check)

    # ---- serving: Poisson arrivals, continuous batching, HBM admission
    serving = None
    if args.serve_requests > 0 and rank == 0:
        serving = measure_serving(dev, args.serve_requests, args.no_check)

    # ---- BiCGStab pressure solver to the paper's stopping criterion
    krylov = None
    if not args.no_krylov and rank == 0:
        krylov = measure_krylov(dev, stream, args.no_check)

    # ---- the other configurations: 64^3 and 256^2 x 128 (FP64 workloads; the
    # mixed path timed beside them)
    configs = None
    if not args.no_configs and rank == 0:
        configs = measure_configs(dev, stream, args.no_check)

    # ---- the host link the e2e leg runs over: plain page-locked copies of the
    # step's bytes, each direction alone and both at once
    link = measure_link(dev, field_bytes) if rank == 0 else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel
    phases = {k: v for k, v in prof["phases"].items() if v > 0}
    nsolves = prof["solves"]
    dom = max(phases, key=lambda k: phases[k])
    dom_ms = phases[dom] / max(nsolves, 1)
    peak, peak_kind = hbm_peak()
    dom_bytes = phase_bytes(g, dom, 4)
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    traffic = recorded_traffic(dom)
    path_bpp = path_bytes_per_point(4)
    path_gbs = path_bpp * npts / (ms * 1e-3) / 1e9
    path_traffic = recorded_path_traffic()

    cpu = None
    if not args.no_cpu_baseline:
        gs, times = time_oracle(g, seed, mode, CPU_SAMPLE_LEVELS)
        pts = gs.nx * gs.ny * gs.nz
        cpu = {"value": pts / times[0] / 1e6, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
               "sample": f"first {gs.nz} levels of the workload ({gs.nx}x{gs.ny}x{gs.nz}, "
                         f"{times[0]:.1f} s), FP64 naive-DFT + Thomas oracle"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": g.nx, "ny": g.ny, "nz": g.nz, "dx": g.dx,
                   "dz": "geometric 5->50 m", "precision": "mixed", "seed": seed,
                   "l2": "inputs larger than L2 (1.07 GB per field), no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "scope": "whole projection step (all kernels)",
                     "bytes_per_point": path_bpp, "achieved": path_gbs, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": path_gbs / peak, "traffic": path_traffic,
                     "algorithmic_bytes": path_bpp * npts,
                     "kernel": {"name": dom, "achieved": achieved, "frac": achieved / peak, "traffic": traffic,
                                "algorithmic_bytes": dom_bytes, "ms_per_launch": dom_ms}},
        "phases_ms": {k: v / max(nsolves, 1) for k, v in phases.items()},
        "cpu_baseline": cpu,
        "e2e": {"value": job_throughput(world, npts, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": field_bytes, "d2h_bytes_per_step": field_bytes,
                "ms_per_step": e2e_ms, "api": f"monc_proj_solve_host, {nl} streams",
                "matches_device_solve": e2e_match},
        "clocks": clk,
        "gpu_launches": nsolves * len(phases),
        "fp64_path": fp64,
        "a3_variants": a3_variants,
        "tensor_core_columns": tensor_cols,
        "refined_path": refined,
        "configs": configs,
        "link": link,
        "krylov_path": krylov,
        "batch": batch,
        "serving": serving,
        "accuracy": check,
        "device_status": status,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_batch(dev, stream, count=64, reps=5, check=True):
    """64 uneven projections (n from {64,96,128,192,256}, nz from
    {64,96,128,160}, mixed precision, seed 3): time of one batched call and of
    a CUDA-graph replay of it, with per-instance launches on the stream pool
    and with grouped launches (one launch per phase and size group)."""
    import torch
    from paper_2009_12849_gb300 import monc_proj as MP
    from paper_2009_12849_gb300 import workloads as W
    inst = W.batch_instances(count, 3)
    grids = [g for g, _ in inst]
    B = MP.BatchProjector(grids, "mixed", dev)
    args = []
    for g, sd in inst:
        u, v, w = (torch.from_numpy(a).to(dev) for a in W.random_fields_f32(g, sd, False))
        args.append((u, v, w, torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)))
    pts = sum(g.npoints for g in grids)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(grouped=False):
        for _ in range(2):
            B.solve(args, stream=stream, grouped=grouped)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            B.solve(args, stream=stream, grouped=grouped)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        side = torch.cuda.Stream(dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                B.solve(args, stream=side, grouped=grouped)
        graph.replay()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return ms, e0.elapsed_time(e1) / reps

    ms0, ms_graph0 = timed()
    gms0, gms_graph0 = timed(grouped=True)
    grouped_out = [tuple(t.clone() for t in a[3:6]) for a in args]
    B.solve(args, stream=stream)
    torch.cuda.synchronize(dev)
    grouped_same = all(torch.equal(x, y) for a, o in zip(args, grouped_out) for x, y in zip(a[3:6], o))
    # task shapes picked per instance by the library's autotuner, then timed again
    shapes = B.autotune(args, stream=stream)
    torch.cuda.synchronize(dev)
    scheds = {}
    for pl in B.plans:
        sc = MP.monc_proj_plan_schedule(pl.handle)
        key = f"n={pl.grid.nx} rows {sc['row_threads']}thr cols {sc['col_threads']}thr E={sc['col_elems']}"
        scheds[key] = scheds.get(key, 0) + 1
    ms, ms_graph = timed()
    B.close()
    tuned = sorted({tuple(x) for x in shapes})
    res = {"instances": count, "points": pts, "ms_per_batch": ms, "mpts_per_s": pts / (ms * 1e-3) / 1e6,
           "graph_ms_per_batch": ms_graph, "graph_mpts_per_s": pts / (ms_graph * 1e-3) / 1e6,
           "autotuned": True, "shapes_kept": [list(x) for x in tuned],
           "schedules_kept": dict(sorted(scheds.items())),
           "default_shapes": {"ms_per_batch": ms0, "graph_ms_per_batch": ms_graph0},
           "grouped": {"api": "monc_proj_solve_batch_grouped (one launch per phase and size group)",
                       "ms_per_batch": gms0, "graph_ms_per_batch": gms_graph0,
                       "graph_mpts_per_s": pts / (gms_graph0 * 1e-3) / 1e6,
                       "bitwise_equal_to_per_instance": grouped_same}}
    if check:
        # every instance against its own FP64 GPU solve (the path the parity
        # tests pin to the FP64 oracle) and its divergence residual
        errs, divs = [], []
        for g, a in zip(grids, args):
            P64 = MP.Projector.from_grid(g, "fp64", dev)
            ref = P64.solve(*(t.double() for t in a[:3]))
            acc = verify(g, a[:3], a[3:6], ref)
            errs.append(acc["rel_err_vs_fp64_path"])
            divs.append(acc["div_residual"])
            P64.close()
        res["accuracy"] = {"max_rel_err_vs_fp64_path": max(errs), "max_div_residual": max(divs),
                           "instances": len(errs)}
    return res


def measure_serving(dev, nreq, no_check, samples=20):
    """The serving recipe: plans for the whole size envelope built first
    (every 2^a3^b5^c n in [128, 512] x nz in [64, 192], chosen without the
    request list), then the process's first serving pass (2000 requests of
    another seed: the cold p50/p99) and the measured pass (nreq requests, seed
    4), with every (nreq // samples)-th output kept and checked."""
    import torch
    from paper_2009_12849_gb300 import monc_proj as MP
    from paper_2009_12849_gb300 import serve as S
    from paper_2009_12849_gb300 import workloads as W
    srv = S.ProjectionServer(dev, hbm_budget=40e9, slots=32)
    setup = srv.prewarm_envelope()
    cold = srv.run(sorted(S.requests_from_recipe(min(2000, nreq), 2000.0, 5), key=lambda r: r.t))
    reqs = sorted(S.requests_from_recipe(nreq, 2000.0, 4), key=lambda r: r.t)
    every = max(1, nreq // samples)
    stats = srv.run(reqs, keep_outputs=not no_check, keep_every=every)
    outputs = stats.pop("outputs", None)
    stats.update({"rate_per_s": 2000.0, "prewarm_s": setup,
                  "recipe": "sizes 128-512 log-uniform (nearest 2^a3^b5^c) x nz 64-192, seed 4, mixed precision",
                  "prewarm": "every 2^a3^b5^c n in [128, 512] x nz in [64, 192], built before any request",
                  "cold": {k: cold[k] for k in ("requests", "served", "p50_ms", "p99_ms", "max_ms", "mean_ms",
                                                "mpts_per_s")}})
    if outputs is not None:
        gen = torch.Generator(device=dev)
        errs, divs, sizes = [], [], []
        for i, o in enumerate(outputs):
            if o is None:
                continue
            r = reqs[i]
            g = W.serving_grid(r.n, r.nz)
            ins = S.make_fields(r, torch.float32, dev, gen)
            P64 = MP.Projector.from_grid(g, "fp64", dev)
            ref = P64.solve(*(t.double() for t in ins))
            acc = verify(g, ins, o, ref)
            errs.append(acc["rel_err_vs_fp64_path"])
            divs.append(acc["div_residual"])
            sizes.append([r.n, r.n, r.nz])
            P64.close()
        stats["accuracy"] = {"max_rel_err_vs_fp64_path": max(errs), "max_div_residual": max(divs),
                             "requests_checked": len(errs), "sizes": sizes}
    srv.close()
    return stats


def measure_configs(dev, stream, no_check, reps=30):
    """The 64^3 (seed 0) and 256^2 x 128 (seed 1, with the large-scale mode)
    workloads, FP64 as specified and mixed beside them; accuracy of the mixed
    path against the FP64 path and the divergence residual of both."""
    import torch
    from paper_2009_12849_gb300 import monc_proj as MP
    from paper_2009_12849_gb300 import workloads as W
    out = {}
    for name, (g, seed, mode) in (("proj64_fp64", W.workload_64cube()), ("proj256x128_fp64", W.workload_256())):
        npts = g.nx * g.ny * g.nz
        host = W.random_fields(g, seed, mode)
        leg = {"nx": g.nx, "ny": g.ny, "nz": g.nz, "points": npts}
        ref = None
        for prec in ("fp64", "mixed"):
            P = MP.Projector.from_grid(g, prec, dev)
            u, v, w = (torch.tensor(a, dtype=P.dtype, device=dev) for a in host)
            o = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
            for _ in range(3):
                P.solve(u, v, w, out=o)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                P.solve(u, v, w, out=o)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            msr = e0.elapsed_time(e1) / reps
            r = {"ms_per_step": msr, "value": npts / (msr * 1e-3) / 1e6, "unit": UNIT,
                 "device_status": P.sync_status()}
            if not no_check:
                r["accuracy"] = verify(g, (u, v, w), o, ref)
            if prec == "fp64":
                ref = tuple(t.clone() for t in o)
            leg[prec] = r
            P.close()
        out[name] = leg
    return out


def measure_link(dev, total_bytes, chunk=1 << 30):
    """Page-locked host <-> device copy rates (GB/s) over up to 1 GiB: each
    direction alone, then both at once on two streams (the pattern of the e2e
    leg, whose copies in and out of different steps overlap)."""
    import torch
    n = int(min(total_bytes, chunk))
    h_in = torch.empty(n, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(n, dtype=torch.uint8).pin_memory()
    d_in = torch.empty(n, dtype=torch.uint8, device=dev)
    d_out = torch.empty(n, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed(h2d, d2h, reps=3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(s1)
        s2.wait_event(e0)
        for _ in range(reps):
            if h2d:
                with torch.cuda.stream(s1):
                    d_in.copy_(h_in, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    h_out.copy_(d_out, non_blocking=True)
        s1.wait_stream(s2)
        e1.record(s1)
        torch.cuda.synchronize(dev)
        return reps * n * (int(h2d) + int(d2h)) / (e0.elapsed_time(e1) * 1e-3) / 1e9

    for _ in range(2):
        timed(True, True, 1)
    res = {"bytes_per_copy": n, "h2d_gbs": timed(True, False), "d2h_gbs": timed(False, True),
           "both_directions_gbs": timed(True, True)}
    del h_in, h_out, d_in, d_out
    return res


def _divergence(g, u, v, w, k0, k1):
    """D(u, v, w) at levels k0..k1-1 in FP64 with torch (verification only:
    the bottom and top faces count as w = 0)."""
    import torch
    dev = u.device
    ud = u[k0:k1].double()
    vd = v[k0:k1].double()
    d = (ud - torch.roll(ud, 1, dims=2)) / g.dx + (vd - torch.roll(vd, 1, dims=1)) / g.dy
    rc = np.asarray(g.rho_c, np.float64)
    rf = np.asarray(g.rho_f, np.float64)
    dz = np.asarray(g.dz, np.float64)
    ks = np.arange(k0, k1)
    fhi = np.where(ks < g.nz - 1, rf[ks + 1], 0.0) / (rc[ks] * dz[ks])
    flo = np.where(ks > 0, rf[ks], 0.0) / (rc[ks] * dz[ks])
    fhi_t = torch.tensor(fhi, device=dev)[:, None, None]
    flo_t = torch.tensor(flo, device=dev)[:, None, None]
    return d + fhi_t * w[k0 + 1:k1 + 1].double() - flo_t * w[k0:k1].double()


def verify(g, ins, outs, ref=None, chunk=16):
    """Divergence residual ||D(out)|| / ||D(in)|| over all cells and, given a
    reference projection, the relative L2 error over u, v, w stacked; FP64,
    on the device, level chunk by level chunk."""
    dn = dd = 0.0
    for k0 in range(0, g.nz, chunk):
        k1 = min(g.nz, k0 + chunk)
        dn += float((_divergence(g, *outs, k0, k1) ** 2).sum())
        dd += float((_divergence(g, *ins, k0, k1) ** 2).sum())
    res = {"div_residual": (dn / dd) ** 0.5}
    if ref is not None:
        num = den = 0.0
        for a, b in zip(outs, ref):
            for k0 in range(0, a.shape[0], chunk):
                x = a[k0:k0 + chunk].double()
                y = b[k0:k0 + chunk].double()
                num += float(((x - y) ** 2).sum())
                den += float((y ** 2).sum())
        res["rel_err_vs_fp64_path"] = (num / den) ** 0.5
    return res


def measure_krylov(dev, stream, no_check, tol=1e-4):
    """BiCGStab with the vertical-line preconditioner to the paper's 1e-4
    criterion on the 256^2 x 128 workload, FP32 (mixed plan) and FP64
    vectors, beside the FFT path on the same grid."""
    import torch
    from paper_2009_12849_gb300 import monc_proj as MP
    from paper_2009_12849_gb300 import workloads as W
    g, seed, mode = W.workload_256()
    npts = g.nx * g.ny * g.nz
    fields = [torch.from_numpy(a).to(dev) for a in W.random_fields(g, seed, mode)]
    peak, peak_kind = hbm_peak()
    res = {"workload": "proj256x128", "nx": g.nx, "ny": g.ny, "nz": g.nz, "precond": "line", "tol": tol}
    ref = None
    for prec in ("fp64", "mixed"):
        P = MP.Projector.from_grid(g, prec, dev)
        u, v, w = (t.to(P.dtype) for t in fields)
        out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        ws = torch.empty(MP.monc_proj_krylov_workspace_size(P.plan), dtype=torch.uint8, device=dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            P.solve(u, v, w, out=out)
        e0.record(stream)
        for _ in range(10):
            P.solve(u, v, w, out=out)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        fft_ms = e0.elapsed_time(e1) / 10
        if prec == "fp64":
            ref = tuple(x.clone() for x in out)
        P.solve_krylov(u, v, w, tol, 5000, "line", out=out, workspace=ws)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        _, _, _, _, st, it, rr = P.solve_krylov(u, v, w, tol, 5000, "line", out=out, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        kms = e0.elapsed_time(e1)
        elem = 4 if prec == "mixed" else 8
        # algorithmic bytes per point and iteration: p update 4, two line
        # solves 2 each, two stencil applications 3 each, s 3, update 7 reads
        # and 3 writes (the FP32 iterate is a pair) -- in field elements
        bpp = elem * (4 + 2 + 3 + 3 + 2 + 3 + (10 if prec == "mixed" else 8))
        gbs = bpp * npts * it / (kms * 1e-3) / 1e9 if it else 0.0
        leg = {"ms_per_solve": kms, "status": st, "iterations": it, "rel_residual": rr,
               "ms_per_iteration": kms / max(it, 1), "fft_ms_per_solve": fft_ms,
               "roofline": {"bound": "hbm", "bytes_per_point_iteration": bpp, "achieved": gbs, "peak": peak,
                            "peak_kind": peak_kind, "unit": "GB/s", "frac": gbs / peak}}
        if not no_check:
            leg["accuracy"] = verify(g, (u, v, w), out, ref)
        res["fp32" if prec == "mixed" else "fp64"] = leg
        P.close()
    return res


if __name__ == "__main__":
    main()
