"""The pencil decomposition's collectives on CPU: world-size 2 and 3 gloo ranks.

Each rank runs the distributed driver (paper_2009_12849_gb300.pencil) with the
phases restated from the oracle (tests/pencil_phases.py); the gathered slabs
must equal the oracle's whole-grid projection.  A second driver run carries
exact labels through the all-to-alls to check the slab <-> pencil index maps
bit for bit, and the halo exchange of w's face k1.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle as O
from paper_2009_12849_gb300 import workloads as W
from paper_2009_12849_gb300.pencil import PencilProjector, block_range
from tests.pencil_phases import OraclePhases, part_rows

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _grid(shape):
    nx, ny, nz = shape
    return W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))


def _slab_inputs(g, k0, k1, seed):
    """This rank's u, v and w (faces k0 .. k1, face k1 poisoned with NaN: the
    halo exchange must overwrite it, or, on the last rank, nothing reads it)."""
    u, v, w = W.random_fields(g, seed, True)
    nzl = k1 - k0
    ws = np.full((nzl + 1, g.ny, g.nx), np.nan)
    ws[:nzl] = w[k0:k1]
    return torch.tensor(u[k0:k1]), torch.tensor(v[k0:k1]), torch.tensor(ws)


def _solve_rank(rank, world, port, shape, seed, out_dir):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    g = _grid(shape)
    ph = OraclePhases(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    pp = PencilProjector(ph, g.nx, g.ny, g.nz)
    u, v, w = _slab_inputs(g, pp.k0, pp.k1, seed)
    uo, vo, wo = pp.solve(u, v, w)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), k0=pp.k0, k1=pp.k1, u=uo.numpy(), v=vo.numpy(),
             w=wo.numpy())
    dist.barrier()
    dist.destroy_process_group()


class LabelPhases(OraclePhases):
    """Phases that write exact labels of (level, row, kx, part) and check, on
    the receiving side, that every value arrived where the index maps say."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.errors = []

    def label(self, k, j):
        kx = torch.arange(self.nxp, dtype=torch.float64)[:, None]
        c = torch.arange(2, dtype=torch.float64)[None, :]
        return ((k * 1000.0 + j) * 1000.0 + kx) * 2.0 + c

    def forward_slab(self, k0, k1, u, v, w, dhat):
        for k in range(k1 - k0):
            for j in range(self.ny):
                dhat[k, j] = self.label(k0 + k, j)
        # the halo: face k1 arrived from the next rank (no NaN left)
        if k1 < self.nz and not torch.isfinite(w[k1 - k0]).all():
            self.errors.append("halo face not received")

    def vertical_pencil(self, j0, j1, spec, gz):
        for k in range(self.nz):
            for jl in range(j1 - j0):
                if not torch.equal(spec[k, jl], self.label(k, j0 + jl)):
                    self.errors.append(f"pencil ({k}, {j0 + jl})")
                spec[k, jl] = -self.label(k, j0 + jl)
                gz[k, jl] = self.label(k, j0 + jl) + 0.5

    def inverse_slab(self, k0, k1, phat, gz, u, v, w, u_out, v_out, w_out):
        for k in range(k1 - k0):
            for j in range(self.ny):
                if not torch.equal(phat[k, j], -self.label(k0 + k, j)):
                    self.errors.append(f"p^ slab ({k0 + k}, {j})")
                if not torch.equal(gz[k, j], self.label(k0 + k, j) + 0.5):
                    self.errors.append(f"gz^ slab ({k0 + k}, {j})")


def _label_rank(rank, world, port, shape, out_dir):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    g = _grid(shape)
    ph = LabelPhases(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    pp = PencilProjector(ph, g.nx, g.ny, g.nz)
    u, v, w = _slab_inputs(g, pp.k0, pp.k1, 3)
    # the face each rank sends down is finite and distinct from the poison
    pp.solve(u, v, w)
    with open(os.path.join(out_dir, f"labels{rank}.txt"), "w") as f:
        f.write("\n".join(ph.errors))
    dist.barrier()
    dist.destroy_process_group()


def _gather(out_dir, world, g):
    u = np.empty((g.nz, g.ny, g.nx))
    v = np.empty_like(u)
    w = np.full((g.nz + 1, g.ny, g.nx), np.nan)
    for r in range(world):
        d = np.load(os.path.join(out_dir, f"rank{r}.npz"))
        k0, k1 = int(d["k0"]), int(d["k1"])
        u[k0:k1], v[k0:k1] = d["u"], d["v"]
        w[k0:k1] = d["w"][:k1 - k0]
        if k1 == g.nz and k1 > k0:
            w[g.nz] = d["w"][k1 - k0]
    return u, v, w


@pytest.mark.parametrize("world,shape", [(2, (12, 9, 5)), (2, (16, 8, 4)), (3, (10, 9, 2)), (3, (12, 2, 7))])
def test_distributed_solve_matches_oracle(world, shape, tmp_path):
    """Slabs and pencils of uneven size, an empty slab (nz < ranks) and an
    empty pencil (ny < ranks)."""
    port = _free_port()
    tmp.spawn(_solve_rank, args=(world, port, shape, 5, str(tmp_path)), nprocs=world, join=True)
    g = _grid(shape)
    got = _gather(str(tmp_path), world, g)
    u, v, w = W.random_fields(g, 5, True)
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    for a, b in zip(got, ref[:3]):
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-12
    assert np.all(got[2][0] == 0) and np.all(got[2][-1] == 0)


@pytest.mark.parametrize("world,shape", [(2, (8, 7, 5)), (3, (6, 5, 4)), (3, (4, 2, 2))])
def test_transposes_move_every_value_exactly(world, shape, tmp_path):
    port = _free_port()
    tmp.spawn(_label_rank, args=(world, port, shape, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        errs = open(tmp_path / f"labels{r}.txt").read()
        assert errs == "", f"rank {r}: {errs[:400]}"


def test_block_range_is_the_balanced_split():
    for n in range(0, 23):
        for parts in range(1, 7):
            assert [block_range(n, parts, s) for s in range(parts)] == part_rows(n, parts)


def test_single_rank_runs_the_phases_back_to_back():
    """Without torch.distributed the driver is the whole solve (no reordering)."""
    g = _grid((12, 10, 6))
    ph = OraclePhases(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    pp = PencilProjector(ph, g.nx, g.ny, g.nz)
    assert (pp.size, pp.k0, pp.k1, pp.j0, pp.j1) == (1, 0, 6, 0, 10)
    u, v, w = W.random_fields(g, 2, True)
    got = pp.solve(torch.tensor(u), torch.tensor(v), torch.tensor(w))
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    for a, b in zip(got, ref[:3]):
        assert np.linalg.norm(a.numpy() - b) / np.linalg.norm(b) < 1e-12
