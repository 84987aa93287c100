"""Batched and served projections equal standalone solves of the same inputs."""
import numpy as np
import pytest
import torch

from paper_2009_12849_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_equals_individual_solves(prec):
    mp = _mp()
    dev = torch.device("cuda", 0)
    dt = torch.float32 if prec == "mixed" else torch.float64
    grids = [W.make_grid(n, n, nz, 25.0, 25.0, W.geometric_dz(nz, 10.0, 100.0))
             for n, nz in ((96, 20), (64, 33), (128, 12), (48, 9), (192, 6), (30, 7))]
    B = mp.BatchProjector(grids, prec, dev)
    ins, outs, refs = [], [], []
    for i, g in enumerate(grids):
        u, v, w = (torch.tensor(a, dtype=dt, device=dev) for a in W.random_fields(g, 40 + i, True))
        ins.append((u, v, w))
        outs.append((torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)))
        P = mp.Projector.from_grid(g, prec, dev)
        refs.append([t.clone() for t in P.solve(u, v, w)])
        torch.cuda.synchronize()
        P.close()
    B.solve([(a[0], a[1], a[2], o[0], o[1], o[2]) for a, o in zip(ins, outs)])
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        for x, y in zip(o, r):
            assert torch.equal(x, y)
    B.close()


def test_grouped_batch_equals_individual_solves():
    """Grouped launches: instances of one size share each phase's launch
    (a group of 25 spans two chunks); sizes without a compile-time plan and
    FP64 plans run alone; with and without phi.  Bit for bit against
    standalone solves, also when the call is captured into a CUDA graph."""
    mp = _mp()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(21)
    spec = [(64, int(rng.integers(3, 12)), "mixed") for _ in range(25)]
    spec += [(96, 20, "mixed"), (96, 7, "mixed"), (128, 12, "mixed"), (256, 5, "mixed"), (48, 9, "mixed"),
             (30, 7, "mixed"), (64, 6, "fp64")]
    plans, fields, refs, ins = [], [], [], []
    for i, (n, nz, prec) in enumerate(spec):
        g = W.make_grid(n, n, nz, 25.0, 25.0, W.geometric_dz(nz, 10.0, 100.0))
        dt = torch.float32 if prec == "mixed" else torch.float64
        u, v, w = (torch.tensor(a, dtype=dt, device=dev) for a in W.random_fields(g, 70 + i, True))
        phi = i % 3 == 0
        P = mp.Projector.from_grid(g, prec, dev)
        refs.append([t.clone() for t in P.solve(u, v, w, phi=phi)])
        torch.cuda.synchronize()
        P.close()
        pl = mp.Plan(g, prec, dev)
        plans.append(pl)
        out = [torch.empty_like(u), torch.empty_like(v), torch.empty_like(w)]
        if phi:
            out.append(torch.empty_like(u))
        fields.append((u, v, w, *out) + (None,) * (4 - len(out)))
    handles = [p.handle for p in plans]
    ws = torch.empty(max(mp.monc_proj_batch_workspace_size(handles), 256), dtype=torch.uint8, device=dev)
    mp.monc_proj_solve_batch_grouped(handles, fields, ws)
    torch.cuda.synchronize()

    def check():
        for f, r in zip(fields, refs):
            got = [t for t in f[3:] if t is not None]
            assert len(got) == len(r)
            for x, y in zip(got, r):
                assert torch.equal(x, y)

    check()
    # and every grouped instance against the FP64 oracle (inputs as the GPU saw them)
    import oracle as O
    for i, ((n, nz, prec), f) in enumerate(zip(spec, fields)):
        g = W.make_grid(n, n, nz, 25.0, 25.0, W.geometric_dz(nz, 10.0, 100.0))
        u, v, w = (t.double().cpu().numpy() for t in f[:3])
        ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
        got = [t.double().cpu().numpy() for t in f[3:6]]
        num = sum(np.linalg.norm(a - b) ** 2 for a, b in zip(got, ref[:3]))
        den = sum(np.linalg.norm(b) ** 2 for b in ref[:3])
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert (num / den) ** 0.5 < tol, f"instance {i} ({n}x{n}x{nz} {prec})"
        assert O.divergence_residual(*got, u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f) < \
            (1e-10 if prec == "fp64" else 1e-6)
    for f in fields:
        for t in f[3:]:
            if t is not None:
                t.zero_()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            mp.monc_proj_solve_batch_grouped(handles, fields, ws, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    check()
    for p in plans:
        p.close()


def test_batch_capturable_in_cuda_graph():
    mp = _mp()
    dev = torch.device("cuda", 0)
    grids = [W.make_grid(n, n, 8, 25.0, 25.0, W.uniform_dz(8, 25.0)) for n in (64, 96, 128)]
    B = mp.BatchProjector(grids, "mixed", dev)
    ins = [tuple(torch.tensor(a, dtype=torch.float32, device=dev) for a in W.random_fields(g, 3, False))
           for g in grids]
    outs = [tuple(torch.empty_like(t) for t in f) for f in ins]
    args = [(a[0], a[1], a[2], o[0], o[1], o[2]) for a, o in zip(ins, outs)]
    B.solve(args)                      # warm-up outside capture
    torch.cuda.synchronize()
    ref = [tuple(t.clone() for t in o) for o in outs]
    for o in outs:
        for t in o:
            t.zero_()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            B.solve(args, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        for x, y in zip(o, r):
            assert torch.equal(x, y)
    B.close()


def test_served_results_equal_standalone_and_overlap():
    mp = _mp()
    from paper_2009_12849_gb300 import serve as S
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(11)
    reqs = [S.Request(t=0.0002 * i, n=int(rng.choice([64, 96, 120, 128])), nz=int(rng.integers(8, 24)),
                      seed=500 + i) for i in range(16)]
    srv = S.ProjectionServer(dev, hbm_budget=8e9, slots=8)
    stats = srv.run(reqs, keep_outputs=True)
    assert stats["served"] == len(reqs)
    assert stats["max_inflight"] > 1            # requests overlapped on the device
    gen = torch.Generator(device=dev)
    for i, r in enumerate(sorted(reqs, key=lambda r: r.t)):
        plan = srv.plans.get(r.n, r.nz, "mixed")
        u, v, w = S.make_fields(r, torch.float32, dev, gen)
        ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device=dev)
        mp.monc_proj_solve(plan.handle, u, v, w, u, v, w, None, ws)
        torch.cuda.synchronize()
        for x, y in zip(stats["outputs"][i], (u, v, w)):
            assert torch.equal(x, y)
    srv.close()


def test_admission_respects_budget():
    _mp()
    from paper_2009_12849_gb300 import serve as S
    dev = torch.device("cuda", 0)
    small = [S.Request(t=0.0, n=64, nz=16, seed=i) for i in range(6)]
    one = S.field_bytes(64, 16) + 1
    srv = S.ProjectionServer(dev, hbm_budget=2.2 * (one + 64 * 64 * 16 * 40), slots=8)
    huge = S.Request(t=0.0, n=512, nz=192, seed=99)
    stats = srv.run(small + [huge])
    assert stats["rejected"] == 1 and stats["served"] == 6
    assert stats["max_inflight"] <= 2
    assert stats["peak_hbm_gb"] <= stats["hbm_budget_gb"]
    srv.close()


@pytest.mark.parametrize("shape", [(256, 192, 8), (384, 480, 4), (96, 1024, 3)])
def test_autotune_keeps_results_bitwise(shape):
    """The autotuner changes how work is split into blocks, never the
    arithmetic: results before and after tuning are bitwise equal, and the
    shapes kept are among the candidates."""
    import torch
    mp = _mp()
    nx, ny, nz = shape
    g = W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))
    dev = torch.device("cuda", 0)
    u, v, w = (torch.from_numpy(a).to(dev) for a in W.random_fields_f32(g, 3, True))
    P = mp.Projector.from_grid(g, "mixed", dev)
    ref = [x.clone() for x in P.solve(u, v, w, phi=True)]
    rt, ct = P.autotune(u, v, w, reps=2)
    assert rt in (32, 64, 128) and ct in (128, 256, 512)
    got = P.solve(u, v, w, phi=True)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    P.close()


@pytest.mark.parametrize("n,nz", [(256, 12), (512, 6), (1024, 3)])
def test_radix_schedules_match_the_oracle(n, nz):
    """The column transforms' E = 16 schedule (1024 = 16*16*4) against the FP64
    oracle at the mixed tolerance, with and without phi; the autotuner keeps
    one of the candidates and, when it keeps the default schedule, results
    bitwise equal to the untuned plan's."""
    import torch
    import oracle as O
    mp = _mp()
    g = W.make_grid(n, n, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))
    dev = torch.device("cuda", 0)
    u, v, w = W.random_fields(g, 12, True)
    u, v, w = (a.astype(np.float32).astype(np.float64) for a in (u, v, w))
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    tu, tv, tw = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (u, v, w))
    P = mp.Projector.from_grid(g, "mixed", dev)
    assert mp.monc_proj_plan_schedule(P.plan)["col_elems"] == 32
    base = [x.clone() for x in P.solve(tu, tv, tw, phi=True)]
    mp.monc_proj_set_schedule(P.plan, 128, 256, 16)
    sch = mp.monc_proj_plan_schedule(P.plan)
    assert sch["col_elems"] == 16 and sch["col_threads"] == 256
    got = P.solve(tu, tv, tw, phi=True)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    num = sum(np.linalg.norm(a.double().cpu().numpy() - b) ** 2 for a, b in zip(got[:3], ref[:3]))
    den = sum(np.linalg.norm(b) ** 2 for b in ref[:3])
    assert (num / den) ** 0.5 < 1e-5
    div = O.divergence_residual(*(a.double().cpu().numpy() for a in got[:3]), u, v, w, g.dx, g.dy, g.dz,
                                g.rho_c, g.rho_f)
    assert div < 1e-6
    assert not all(torch.equal(a, b) for a, b in zip(base, got))     # a different summation order
    with pytest.raises(mp.ProjError):
        mp.monc_proj_set_schedule(P.plan, 128, 512, 16)              # no kernels for that tile
    assert mp.monc_proj_plan_schedule(P.plan)["col_elems"] == 16    # kept on refusal
    mp.monc_proj_set_schedule(P.plan, 128, 256, 32)
    again = P.solve(tu, tv, tw, phi=True)
    torch.cuda.synchronize()
    for a, b in zip(base, again):
        assert torch.equal(a, b)
    rt, ct = P.autotune(tu, tv, tw, reps=2)
    sch = mp.monc_proj_plan_schedule(P.plan)
    assert (ct, sch["col_elems"]) in ((128, 32), (256, 32), (512, 32), (256, 16))
    tuned = P.solve(tu, tv, tw, phi=True)
    torch.cuda.synchronize()
    if sch["col_elems"] == 32:
        for a, b in zip(base, tuned):
            assert torch.equal(a, b)
    P.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_host_buffer_solve_matches_device_solve(prec):
    """monc_proj_solve_host (host arrays in and out through a device staging
    area) gives bitwise the device solve's result, with and without phi."""
    import torch
    mp = _mp()
    g = W.make_grid(96, 80, 10, 25.0, 25.0, W.geometric_dz(10, 10.0, 60.0))
    dev = torch.device("cuda", 0)
    dt = mp.DTYPES[mp.PRECISIONS[prec]]
    hu, hv, hw = (torch.from_numpy(a).to(dt).pin_memory() for a in W.random_fields(g, 4, True))
    P = mp.Projector.from_grid(g, prec, dev)
    ref = P.solve(hu.to(dev), hv.to(dev), hw.to(dev), phi=True)
    outs = tuple(torch.empty_like(x).pin_memory() for x in (hu, hv, hw, hu))
    stg = torch.empty(mp.monc_proj_host_staging_size(P.plan, True), dtype=torch.uint8, device=dev)
    mp.monc_proj_solve_host(P.plan, hu, hv, hw, *outs, stg, P.workspace)
    torch.cuda.synchronize()
    for a, b in zip(ref, outs):
        assert torch.equal(a.cpu(), b)
    out3 = tuple(torch.empty_like(x).pin_memory() for x in (hu, hv, hw))
    P.solve_host(hu, hv, hw, out3)
    torch.cuda.synchronize()
    for a, b in zip(ref[:3], out3):
        assert torch.equal(a.cpu(), b)
    short = torch.empty(256, dtype=torch.uint8, device=dev)
    with pytest.raises(mp.ProjError):
        mp.monc_proj_solve_host(P.plan, hu, hv, hw, *out3, None, short, P.workspace)
    P.close()
