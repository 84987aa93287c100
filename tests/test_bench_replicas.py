"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks.

bench.py runs one independent replica of the workload per rank (no data-path
collective); its only cross-rank steps are the barrier and the max over ranks
of the timed region, and rank 0 alone prints (and runs the reference arm).
"""
import importlib.util
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out_dir):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    b = _bench()
    ms = b.max_over_ranks(times[rank], world, torch.device("cpu"))
    dist.barrier()
    seed = b.replica_seed(2, rank)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{ms} {seed}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    port = _free_port()
    times = [3.25, 5.5]
    tmp.spawn(_rank, args=(2, port, times, str(tmp_path)), nprocs=2, join=True)
    got = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    assert [float(g[0]) for g in got] == [5.5, 5.5]
    seeds = [int(g[1]) for g in got]
    assert seeds[0] != seeds[1]                  # independent replicas


def test_job_throughput_counts_every_replica():
    b = _bench()
    assert b.job_throughput(1, 1_000_000, 1.0) == pytest.approx(1000.0)
    assert b.job_throughput(4, 1_000_000, 2.0) == pytest.approx(2000.0)
    assert b.max_over_ranks(7.0, 1, torch.device("cpu")) == 7.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    b = _bench()

    class A:
        steps, warmup = 1, 1

    assert b.run_reference(A(), 1, 2) is None
    assert capsys.readouterr().out == ""
