"""One projection sharded over the processes of a torch.distributed group:
the pencil decomposition (paper, Section 4: the model's FFT pressure solver
decomposes the domain into 2D pencils, and every transform needs a global
all-to-all between the processes).

Rank s of P holds the z-slab of cell levels [k0_s, k1_s) and, in spectral
space, the pencil of spectral rows [j0_s, j1_s) over all levels (both split
in contiguous blocks, the first n % P ranks one item more).  One solve is

  halo      the top face k1 of w from rank s+1 (point to point)
  a1-a2     forward transform of the slab            monc_proj_forward_slab
  A2A 1     slab -> pencil: the rows of rank t of every slab go to rank t
            (send buffer packed by monc_proj_pack_pencils; the receive buffer,
            the slabs' blocks one after the other, is the pencil itself)
  a3        vertical solve of the pencil             monc_proj_vertical_pencil
  A2A 2, 3  pencil -> slab for p^ and gz^ (the levels of slab t are one block
            of the pencil; the receive buffer is unpacked by
            monc_proj_unpack_pencils)
  a4-a5     inverse transform and correction         monc_proj_inverse_slab

The compute phases are an object with the methods of ``GpuPhases``; the
collectives are torch.distributed calls on that group (NCCL for CUDA
tensors, gloo for CPU ones).  With one rank there is no collective and no
reordering: the phases run back to back on one buffer, with results bitwise
equal to monc_proj_solve.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import monc_proj as mp


def block_range(n: int, parts: int, s: int) -> tuple[int, int]:
    """Items [lo, hi) of part s when n items are split into `parts` contiguous
    blocks, the first n % parts blocks one item longer."""
    q, r = divmod(n, parts)
    lo = s * q + min(s, r)
    return lo, lo + q + (1 if s < r else 0)


class GpuPhases:
    """The compute phases on one device: a plan of the whole grid and its
    workspace, calling the slab and pencil entry points of the C ABI."""

    def __init__(self, nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision="mixed", device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(self.device):
            self.plan = mp.monc_proj_plan(nx, ny, nz, dx, dy, dz, rho_c, rho_f, precision)
            prec = mp.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
            self.dtype = mp.DTYPES[prec]
            self.nxp = mp.monc_proj_spectral_pitch(self.plan)
            nbytes = mp.monc_proj_workspace_size(self.plan)
            self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)

    def forward_slab(self, k0, k1, u, v, w, dhat):
        mp.monc_proj_forward_slab(self.plan, k0, k1, u, v, w, dhat, self.workspace)

    def vertical_pencil(self, j0, j1, spec, gz):
        mp.monc_proj_vertical_pencil(self.plan, j0, j1, spec, gz, self.workspace)

    def inverse_slab(self, k0, k1, phat, gz, u, v, w, u_out, v_out, w_out):
        mp.monc_proj_inverse_slab(self.plan, k0, k1, phat, gz, u, v, w, u_out, v_out, w_out, self.workspace)

    def pack(self, nzl, parts, slab, packed):
        mp.monc_proj_pack_pencils(self.plan, nzl, parts, slab, packed)

    def unpack(self, nzl, parts, packed, slab):
        mp.monc_proj_unpack_pencils(self.plan, nzl, parts, packed, slab)

    def close(self):
        if getattr(self, "plan", None):
            mp.monc_proj_destroy(self.plan)
            self.plan = None


class PencilProjector:
    """The distributed projection of an nx x ny x nz grid on the ranks of
    `group` (the default group if None; one rank if torch.distributed is not
    initialised).  `phases` provides the compute (``GpuPhases`` on a GPU)."""

    def __init__(self, phases, nx, ny, nz, group=None):
        self.ph = phases
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.group = group
        if dist.is_available() and dist.is_initialized():
            self.rank = dist.get_rank(group)
            self.size = dist.get_world_size(group)
        else:
            self.rank, self.size = 0, 1
        P = self.size
        self.slabs = [block_range(self.nz, P, s) for s in range(P)]
        self.pencils = [block_range(self.ny, P, s) for s in range(P)]
        self.k0, self.k1 = self.slabs[self.rank]
        self.j0, self.j1 = self.pencils[self.rank]
        self.nzl = self.k1 - self.k0
        self.nyl = self.j1 - self.j0
        nxp = phases.nxp
        row = nxp * 2                                   # reals per spectral row
        dt, dev = phases.dtype, phases.device
        # spectral buffers (real views of complex rows: [..., nxp, 2])
        self.dhat = torch.empty((self.nzl, self.ny, nxp, 2), dtype=dt, device=dev)
        if P == 1:
            self.pencil = self.dhat
            self.gzp = torch.empty_like(self.dhat)
            self.phat, self.gz = self.pencil, self.gzp
        else:
            self.packed = torch.empty(max(self.nzl * self.ny * row, 1), dtype=dt, device=dev)
            self.pencil = torch.empty((self.nz, self.nyl, nxp, 2), dtype=dt, device=dev)
            self.gzp = torch.empty_like(self.pencil)
            self.recv_p = torch.empty_like(self.packed)
            self.recv_g = torch.empty_like(self.packed)
            self.phat = torch.empty_like(self.dhat)
            self.gz = torch.empty_like(self.dhat)
        # element counts of the all-to-alls: slab -> pencil sends rank t the
        # slab's rows of pencil t and receives from rank s the pencil's rows
        # of slab s
        self.to_pencil = [self.nzl * (j1 - j0) * row for j0, j1 in self.pencils]
        self.from_slab = [(k1 - k0) * self.nyl * row for k0, k1 in self.slabs]

    # -- collectives --------------------------------------------------------
    def _halo(self, w):
        """Face k1 of w (slot nzl) from the next rank, face k0 to the previous."""
        ops = []
        if self.nzl > 0 and self.rank > 0:
            ops.append(dist.P2POp(dist.isend, w[0].contiguous(), self.rank - 1, self.group))
        if self.nzl > 0 and self.k1 < self.nz:
            self._face = torch.empty_like(w[self.nzl])
            ops.append(dist.P2POp(dist.irecv, self._face, self.rank + 1, self.group))
        for req in dist.batch_isend_irecv(ops) if ops else []:
            req.wait()
        if self.nzl > 0 and self.k1 < self.nz:
            w[self.nzl].copy_(self._face)

    def _a2a(self, out, inp, out_splits, in_splits):
        dist.all_to_all_single(out, inp, out_splits, in_splits, group=self.group)

    # -- the solve ------------------------------------------------------------
    def solve(self, u, v, w, out=None):
        """Project this rank's slab.  u, v: [nzl][ny][nx]; w: [nzl+1][ny][nx],
        faces k0 .. k1, whose face k1 is filled here from the next rank.
        Returns (u_out, v_out, w_out) of the same shapes (faces k0 .. k1-1 of
        w_out, and the zero top face on the last rank); `out` may alias the
        inputs."""
        ph, P = self.ph, self.size
        if out is None:
            out = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        if P > 1:
            self._halo(w)
        if self.nzl > 0:
            ph.forward_slab(self.k0, self.k1, u, v, w, self.dhat)
        if P > 1:
            if self.nzl > 0:
                ph.pack(self.nzl, P, self.dhat, self.packed)
            self._a2a(self.pencil.view(-1), self.packed[:sum(self.to_pencil)], self.from_slab, self.to_pencil)
        if self.nyl > 0:
            ph.vertical_pencil(self.j0, self.j1, self.pencil, self.gzp)
        if P > 1:
            n = sum(self.to_pencil)
            self._a2a(self.recv_p[:n], self.pencil.view(-1), self.to_pencil, self.from_slab)
            self._a2a(self.recv_g[:n], self.gzp.view(-1), self.to_pencil, self.from_slab)
            if self.nzl > 0:
                ph.unpack(self.nzl, P, self.recv_p, self.phat)
                ph.unpack(self.nzl, P, self.recv_g, self.gz)
        if self.nzl > 0:
            ph.inverse_slab(self.k0, self.k1, self.phat, self.gz, u, v, w, out[0], out[1], out[2])
        return out
