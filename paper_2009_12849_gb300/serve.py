"""Continuous-batching server for projection requests of different grid sizes.

Requests arrive over time (each with an arrival time, a square horizontal
size n, a level count nz and a seed for its synthetic fields).  The loop

* moves arrived requests into a FIFO queue,
* admits queued requests while the HBM budget (fields + workspace of every
  request on the device) and the stream slots allow, even while earlier
  requests are still running: each admitted request runs on its own stream,
  so the work of requests admitted at different times overlaps on the GPU,
* keeps plans (twiddles, wavenumbers, rho0-weighted coefficients) resident in
  an LRU cache keyed by the grid, so repeated sizes do not rebuild them,
* retires finished requests (their memory goes back to the budget) and
  records each request's latency on the device clock:
  completion event - start event - arrival time.

Latency therefore covers queueing, admission, the generation of the request's
input fields on the device, and the projection.
"""
from __future__ import annotations

import collections
import dataclasses
import statistics
import time

import torch

from . import monc_proj as MP
from . import workloads as W


@dataclasses.dataclass
class Request:
    t: float            # arrival time [s] after the start of the run
    n: int              # nx = ny
    nz: int
    seed: int

    @property
    def points(self) -> int:
        return self.n * self.n * self.nz


@dataclasses.dataclass
class _Inflight:
    req: Request
    slot: int
    event: torch.cuda.Event
    nbytes: int
    tensors: tuple


class PlanCache:
    """LRU cache of resident plans keyed by (n, nz, precision)."""

    def __init__(self, device, capacity=256, grid_fn=W.serving_grid):
        self.device = device
        self.capacity = capacity
        self.grid_fn = grid_fn
        self.plans = collections.OrderedDict()
        self.created = 0

    def get(self, n, nz, precision):
        key = (n, nz, precision)
        p = self.plans.get(key)
        if p is not None:
            self.plans.move_to_end(key)
            return p
        p = MP.Plan(self.grid_fn(n, nz), precision, self.device)
        self.created += 1
        self.plans[key] = p
        while len(self.plans) > self.capacity:
            _, old = self.plans.popitem(last=False)
            old.close()
        return p

    def close(self):
        for p in self.plans.values():
            p.close()
        self.plans.clear()


def field_bytes(n, nz, elem=4):
    return elem * n * n * (3 * nz + 1)


def make_fields(req: Request, dtype, device, generator, out=None):
    """Synthetic N(0,1) provisional velocities of a request, generated on the
    device from the request's seed (w's bottom and top faces are zero), into
    `out` = (u, v, w) when given."""
    generator.manual_seed(req.seed)
    n, nz = req.n, req.nz
    if out is None:
        out = (torch.empty((nz, n, n), dtype=dtype, device=device),
               torch.empty((nz, n, n), dtype=dtype, device=device),
               torch.empty((nz + 1, n, n), dtype=dtype, device=device))
    u, v, w = out
    torch.randn((nz, n, n), dtype=dtype, device=device, generator=generator, out=u)
    torch.randn((nz, n, n), dtype=dtype, device=device, generator=generator, out=v)
    torch.randn((nz + 1, n, n), dtype=dtype, device=device, generator=generator, out=w)
    w[0].zero_()
    w[nz].zero_()
    return u, v, w


class ProjectionServer:
    def __init__(self, device=None, hbm_budget=40e9, slots=32, precision="mixed", plan_capacity=256):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.hbm_budget = float(hbm_budget)
        self.precision = precision
        self.dtype = MP.DTYPES[MP.PRECISIONS[precision]]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.plans = PlanCache(self.device, plan_capacity)
        self.generator = torch.Generator(device=self.device)

    def request_bytes(self, req, plan):
        return field_bytes(req.n, req.nz, torch.tensor([], dtype=self.dtype).element_size()) + plan.workspace_bytes

    def prewarm(self, sizes):
        """Build the plans of the given (n, nz) sizes so they are resident
        before requests arrive; run one solve per horizontal size (the
        kernels depend on n only), so that the CUDA runtime has loaded every
        kernel the stream will use before the first arrival (it loads a
        kernel on its first launch, a few ms each); and grow the allocator's
        pool to the HBM budget once (request buffers are carved from it, so
        the serving loop makes no device allocation).  The serving loop's
        own first-use work is done here too: one request's fields generated
        and one solve run on every slot stream with an event recorded (the
        field generator's kernels load on their first launch as well).
        Returns the set-up time [s]."""
        t = time.perf_counter()
        for n, nz in sizes:
            self.plans.get(n, nz, self.precision)
        smallest = {}
        for n, nz in sizes:
            smallest[n] = min(nz, smallest.get(n, nz))
        for n, nz in sorted(smallest.items()):
            plan = self.plans.get(n, nz, self.precision)
            u = torch.zeros((nz, n, n), dtype=self.dtype, device=self.device)
            v = torch.zeros_like(u)
            w = torch.zeros((nz + 1, n, n), dtype=self.dtype, device=self.device)
            ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device=self.device)
            MP.monc_proj_solve(plan.handle, u, v, w, u, v, w, None, ws, torch.cuda.current_stream(self.device))
            del u, v, w, ws
        if smallest:
            n, nz = min(smallest.items())
            plan = self.plans.get(n, nz, self.precision)
            u = torch.empty((nz, n, n), dtype=self.dtype, device=self.device)
            v = torch.empty_like(u)
            w = torch.empty((nz + 1, n, n), dtype=self.dtype, device=self.device)
            ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device=self.device)
            for stream in self.streams:
                with torch.cuda.stream(stream):
                    make_fields(Request(0.0, n, nz, 0), self.dtype, self.device, self.generator, out=(u, v, w))
                    MP.monc_proj_solve(plan.handle, u, v, w, u, v, w, None, ws, stream)
                    torch.cuda.Event(enable_timing=True).record(stream)
                stream.synchronize()
            del u, v, w, ws
        free, _ = torch.cuda.mem_get_info(self.device)
        pool = int(min(self.hbm_budget, 0.8 * free))
        if pool > 0:
            block = torch.empty(pool, dtype=torch.uint8, device=self.device)
            del block
        torch.cuda.synchronize(self.device)
        return time.perf_counter() - t

    def prewarm_envelope(self, n_range=(128, 512), nz_range=(64, 192)):
        """Prewarm the service's whole size envelope, chosen without looking
        at any request: every 2^a 3^b 5^c horizontal size in n_range times
        every level count in nz_range.  Returns the set-up time [s]."""
        ns = [n for n in W.smooth_sizes(n_range[1]) if n >= n_range[0]]
        sizes = [(n, nz) for n in ns for nz in range(nz_range[0], nz_range[1] + 1)]
        self.plans.capacity = max(self.plans.capacity, len(sizes))
        return self.prewarm(sizes)

    def run(self, requests, keep_outputs=False, time_scale=1.0, keep_every=0):
        """Serve the requests (sorted by arrival time).  Returns a stats dict;
        with keep_outputs, stats["outputs"][i] holds request i's (u, v, w)
        (with keep_every = m > 0, only every m-th request's, None for the
        rest).  Plans that are not resident (see prewarm) are built when a
        request first needs them."""
        reqs = sorted(requests, key=lambda r: r.t)
        created_before = self.plans.created
        pending = collections.deque(enumerate(reqs))
        queue = collections.deque()
        inflight: list[_Inflight] = []
        free_slots = list(range(len(self.streams)))
        used = 0.0
        latencies = [None] * len(reqs)
        outputs = [None] * len(reqs) if keep_outputs else None
        peak_used = 0.0
        max_inflight = 0
        rejected = 0
        start_ev = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        start_ev.record(torch.cuda.current_stream(self.device))
        done_events = [None] * len(reqs)
        while pending or queue or inflight:
            now = (time.perf_counter() - t0) / time_scale
            while pending and pending[0][1].t <= now:
                queue.append(pending.popleft())
            # retire finished requests
            still = []
            for f in inflight:
                if f.event.query():
                    used -= f.nbytes
                    free_slots.append(f.slot)
                else:
                    still.append(f)
            inflight = still
            # admit in arrival order while memory and slots allow
            progressed = False
            while queue and free_slots:
                idx, req = queue[0]
                plan = self.plans.get(req.n, req.nz, self.precision)
                nbytes = self.request_bytes(req, plan)
                if nbytes > self.hbm_budget:
                    queue.popleft()             # can never fit: reject
                    rejected += 1
                    continue
                if used + nbytes > self.hbm_budget and inflight:
                    break
                queue.popleft()
                slot = free_slots.pop()
                stream = self.streams[slot]
                # buffers come from the current stream's pool (one pool for
                # every slot, grown once by prewarm); record_stream below
                # keeps a buffer from reuse until its slot's work is done
                n, nz = req.n, req.nz
                u = torch.empty((nz, n, n), dtype=self.dtype, device=self.device)
                v = torch.empty((nz, n, n), dtype=self.dtype, device=self.device)
                w = torch.empty((nz + 1, n, n), dtype=self.dtype, device=self.device)
                ws = torch.empty(max(plan.workspace_bytes, 256), dtype=torch.uint8, device=self.device)
                with torch.cuda.stream(stream):
                    make_fields(req, self.dtype, self.device, self.generator, out=(u, v, w))
                    MP.monc_proj_solve(plan.handle, u, v, w, u, v, w, None, ws, stream)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(stream)
                for t in (u, v, w, ws):
                    t.record_stream(stream)
                done_events[idx] = ev
                if keep_outputs and (keep_every <= 0 or idx % keep_every == 0):
                    outputs[idx] = (u, v, w)
                used += nbytes
                peak_used = max(peak_used, used)
                inflight.append(_Inflight(req, slot, ev, nbytes, (u, v, w, ws)))
                max_inflight = max(max_inflight, len(inflight))
                progressed = True
            if not progressed:
                # nothing admitted: wait a little (until the next arrival when idle)
                wait = 20e-6
                if pending and not queue and not inflight:
                    wait = min(1e-3, max(0.0, pending[0][1].t * time_scale - (time.perf_counter() - t0)))
                if wait > 0:
                    time.sleep(wait)
        torch.cuda.synchronize(self.device)
        wall = time.perf_counter() - t0
        served = [i for i, e in enumerate(done_events) if e is not None]
        for i in served:
            latencies[i] = start_ev.elapsed_time(done_events[i]) / 1e3 - reqs[i].t * time_scale
        lat = sorted(latencies[i] for i in served)
        pts = sum(reqs[i].points for i in served)
        last = max(start_ev.elapsed_time(done_events[i]) / 1e3 for i in served) if served else 0.0
        first = reqs[0].t * time_scale if reqs else 0.0
        pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))] if lat else None
        stats = {
            "requests": len(reqs), "served": len(served), "rejected": rejected,
            "p50_ms": 1e3 * pct(0.50) if lat else None, "p99_ms": 1e3 * pct(0.99) if lat else None,
            "max_ms": 1e3 * lat[-1] if lat else None,
            "mean_ms": 1e3 * statistics.fmean(lat) if lat else None,
            "points": pts, "mpts_per_s": pts / max(last - first, 1e-9) / 1e6,
            "wall_s": wall, "peak_hbm_gb": peak_used / 1e9, "hbm_budget_gb": self.hbm_budget / 1e9,
            "max_inflight": max_inflight, "plans_created_in_loop": self.plans.created - created_before,
            "plans_resident": len(self.plans.plans),
        }
        if keep_outputs:
            stats["outputs"] = outputs
        return stats

    def close(self):
        self.plans.close()


def requests_from_recipe(count=10000, rate=2000.0, seed=4):
    return [Request(r["t"], r["n"], r["nz"], r["seed"]) for r in W.serving_requests(count, rate, seed)]


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--slots", type=int, default=32)
    a = ap.parse_args()
    srv = ProjectionServer(hbm_budget=a.budget_gb * 1e9, slots=a.slots)
    setup = srv.prewarm_envelope()
    stats = srv.run(requests_from_recipe(a.requests, a.rate))
    stats["prewarm_s"] = setup
    srv.close()
    print(json.dumps(stats))


if __name__ == "__main__":
    main()
