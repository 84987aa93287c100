"""The slab and pencil entry points of the distributed projection on one GPU.

* Each phase against the same phase restated from the oracle
  (tests/pencil_phases.py), FP64, on a slab and a pencil inside the grid.
* The pack / unpack kernels against the reordering written out from its
  definition, bit for bit.
* P ranks emulated in one process (the all-to-alls done by copies between
  the ranks' buffers, exactly as torch.distributed.all_to_all_single moves
  them): the result equals monc_proj_solve bit for bit, for FP64 and mixed
  plans, uneven slabs and pencils and an empty slab.
* The driver with one rank (no collective) equals monc_proj_solve bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2009_12849_gb300 import workloads as W
from tests.pencil_phases import OraclePhases

pytestmark = pytest.mark.gpu


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj, pencil
    return monc_proj, pencil


def _grid(shape):
    nx, ny, nz = shape
    return W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))


def _phases(g, prec):
    _, pencil = _mp()
    return pencil.GpuPhases(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, prec, "cuda:0")


def _whole(g, prec, u, v, w):
    mp, _ = _mp()
    P = mp.Projector.from_grid(g, prec, "cuda:0")
    out = P.solve(u, v, w)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    P.close()
    return out


def _fields(g, prec, seed):
    mp, _ = _mp()
    dt = mp.DTYPES[mp.PRECISIONS[prec]]
    u, v, w = W.random_fields(g, seed, True)
    if prec == "mixed":
        u, v, w = (a.astype(np.float32).astype(np.float64) for a in (u, v, w))
    return (u, v, w), tuple(torch.tensor(a, dtype=dt, device="cuda:0") for a in (u, v, w))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(64, 48, 7), (30, 45, 9)])
def test_each_phase_matches_the_oracle_phase(shape):
    g = _grid(shape)
    ph = _phases(g, "fp64")
    orc = OraclePhases(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, nxp=ph.nxp)
    (u, v, w), _ = _fields(g, "fp64", 4)
    nxp, nxh = ph.nxp, g.nx // 2 + 1
    dev = "cuda:0"
    # a1-a2 on levels [2, 6)
    k0, k1 = 2, 6
    us, vs, wsl = (torch.tensor(a) for a in (u[k0:k1], v[k0:k1], w[k0:k1 + 1]))
    d_gpu = torch.zeros((k1 - k0, g.ny, nxp, 2), dtype=torch.float64, device=dev)
    ph.forward_slab(k0, k1, us.to(dev), vs.to(dev), wsl.to(dev), d_gpu)
    d_ref = torch.zeros((k1 - k0, g.ny, nxp, 2), dtype=torch.float64)
    orc.forward_slab(k0, k1, us, vs, wsl, d_ref)
    torch.cuda.synchronize()
    assert _rel(d_gpu.cpu().numpy()[..., :nxh, :], d_ref.numpy()[..., :nxh, :]) < 1e-12
    # a3 on spectral rows [3, 8) of every level, from the oracle's D^
    j0, j1 = 3, 8
    d_all = torch.zeros((g.nz, g.ny, nxp, 2), dtype=torch.float64)
    orc.forward_slab(0, g.nz, *(torch.tensor(a) for a in (u, v, w)), d_all)
    spec = d_all[:, j0:j1].contiguous()
    s_gpu = spec.to(dev)
    gz_gpu = torch.zeros_like(s_gpu)
    ph.vertical_pencil(j0, j1, s_gpu, gz_gpu)
    gz_ref = torch.zeros_like(spec)
    orc.vertical_pencil(j0, j1, spec, gz_ref)
    torch.cuda.synchronize()
    assert _rel(s_gpu.cpu().numpy()[..., :nxh, :], spec.numpy()[..., :nxh, :]) < 1e-12
    assert _rel(gz_gpu.cpu().numpy()[1:, :, :nxh, :], gz_ref.numpy()[1:, :, :nxh, :]) < 1e-12
    # a4-a5 on levels [k0, k1) from the oracle's p^ and gz^ of every row
    p_all = d_all.clone()
    g_all = torch.zeros_like(p_all)
    orc.vertical_pencil(0, g.ny, p_all, g_all)
    ps, gs = p_all[k0:k1].contiguous(), g_all[k0:k1].contiguous()
    outs_gpu = [torch.zeros_like(x, device=dev) for x in (us, vs, wsl)]
    ph.inverse_slab(k0, k1, ps.to(dev), gs.to(dev), us.to(dev), vs.to(dev), wsl.to(dev), *outs_gpu)
    outs_ref = [torch.zeros_like(x) for x in (us, vs, wsl)]
    orc.inverse_slab(k0, k1, ps, gs, us, vs, wsl, *outs_ref)
    torch.cuda.synchronize()
    for a, b in zip(outs_gpu[:2], outs_ref[:2]):
        assert _rel(a.cpu().numpy(), b.numpy()) < 1e-12
    # faces k0 .. k1-1 of w (face k1 belongs to the next slab)
    assert _rel(outs_gpu[2].cpu().numpy()[:k1 - k0], outs_ref[2].numpy()[:k1 - k0]) < 1e-12
    ph.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("ny,nzl", [(9, 3), (10, 1), (2, 4)])
def test_pack_kernels_match_the_definition(prec, ny, nzl):
    g = _grid((24, ny, 5))
    ph = _phases(g, prec)
    orc = OraclePhases(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, nxp=ph.nxp)
    gen = torch.Generator().manual_seed(ny * 7 + nzl)
    slab = torch.randn((nzl, ny, ph.nxp, 2), generator=gen, dtype=torch.float64).to(ph.dtype)
    for parts in (1, 2, 3, 5):
        packed_gpu = torch.empty(slab.numel(), dtype=ph.dtype, device="cuda:0")
        ph.pack(nzl, parts, slab.to("cuda:0"), packed_gpu)
        packed_ref = torch.empty(slab.numel(), dtype=ph.dtype)
        orc.pack(nzl, parts, slab, packed_ref)
        back = torch.empty_like(slab, device="cuda:0")
        ph.unpack(nzl, parts, packed_gpu, back)
        torch.cuda.synchronize()
        assert torch.equal(packed_gpu.cpu(), packed_ref)
        assert torch.equal(back.cpu(), slab)
    ph.close()


def _emulated(g, prec, ph, pencil, world, u, v, w):
    """The driver's data movement for `world` ranks, run rank by rank on one GPU."""
    blk = pencil.block_range
    slabs = [blk(g.nz, world, s) for s in range(world)]
    pens = [blk(g.ny, world, s) for s in range(world)]
    row = ph.nxp * 2
    dev, dt = "cuda:0", ph.dtype
    # a1-a2 and the pack, per rank
    packed = []
    for (k0, k1) in slabs:
        nzl = k1 - k0
        d = torch.empty((nzl, g.ny, ph.nxp, 2), dtype=dt, device=dev)
        buf = torch.empty(nzl * g.ny * row, dtype=dt, device=dev)
        if nzl:
            # each rank's own (aligned) arrays
            ph.forward_slab(k0, k1, u[k0:k1].clone(), v[k0:k1].clone(), w[k0:k1 + 1].clone(), d)
            ph.pack(nzl, world, d, buf)
        packed.append(buf)
    # all-to-all 1: rank t receives, from every s in order, s's block for t
    pencils, gzs = [], []
    for t, (j0, j1) in enumerate(pens):
        chunks = []
        for s, (k0, k1) in enumerate(slabs):
            off = (k1 - k0) * pens[t][0] * row
            chunks.append(packed[s][off:off + (k1 - k0) * (j1 - j0) * row])
        pen = torch.cat(chunks).view(g.nz, j1 - j0, ph.nxp, 2)
        gz = torch.empty_like(pen)
        if j1 > j0:
            ph.vertical_pencil(j0, j1, pen, gz)
        pencils.append(pen)
        gzs.append(gz)
    # all-to-alls 2 and 3, the unpack, a4-a5, per rank
    outs = []
    for s, (k0, k1) in enumerate(slabs):
        nzl = k1 - k0
        rp = torch.cat([pencils[t][k0:k1].reshape(-1) for t in range(world)])
        rg = torch.cat([gzs[t][k0:k1].reshape(-1) for t in range(world)])
        if not nzl:
            continue
        phat = torch.empty((nzl, g.ny, ph.nxp, 2), dtype=dt, device=dev)
        gzs_ = torch.empty_like(phat)
        ph.unpack(nzl, world, rp, phat)
        ph.unpack(nzl, world, rg, gzs_)
        wo = torch.empty((nzl + 1, g.ny, g.nx), dtype=dt, device=dev)
        uo, vo = torch.empty_like(u[k0:k1]), torch.empty_like(v[k0:k1])
        ph.inverse_slab(k0, k1, phat, gzs_, u[k0:k1].clone(), v[k0:k1].clone(), w[k0:k1 + 1].clone(), uo, vo, wo)
        outs.append((k0, k1, uo, vo, wo))
    torch.cuda.synchronize()
    uo = torch.empty_like(u)
    vo = torch.empty_like(v)
    wo = torch.empty_like(w)
    for k0, k1, a, b, c in outs:
        uo[k0:k1], vo[k0:k1], wo[k0:k1] = a, b, c[:k1 - k0]
        if k1 == g.nz:
            wo[g.nz] = c[k1 - k0]
    return uo, vo, wo


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape,world", [((64, 48, 7), 2), ((96, 64, 10), 3), ((30, 45, 9), 4), ((128, 40, 3), 4),
                                         ((1024, 64, 5), 2)])
def test_emulated_ranks_equal_the_whole_solve(shape, world, prec):
    _, pencil = _mp()
    g = _grid(shape)
    ph = _phases(g, prec)
    _, (u, v, w) = _fields(g, prec, 6)
    got = _emulated(g, prec, ph, pencil, world, u, v, w)
    ref = _whole(g, prec, u, v, w)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    ph.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_rank_driver_equals_the_whole_solve(prec):
    _, pencil = _mp()
    g = _grid((256, 128, 12))
    ph = _phases(g, prec)
    _, (u, v, w) = _fields(g, prec, 8)
    pp = pencil.PencilProjector(ph, g.nx, g.ny, g.nz)
    got = pp.solve(u, v, w.clone())
    torch.cuda.synchronize()
    ref = _whole(g, prec, u, v, w)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    ph.close()


def test_invalid_ranges_rejected():
    mp, _ = _mp()
    g = _grid((32, 16, 6))
    ph = _phases(g, "fp64")
    t = torch.zeros(1 << 16, dtype=torch.float64, device="cuda:0")
    for k0, k1 in ((-1, 2), (3, 3), (4, 2), (0, 7)):
        with pytest.raises(mp.ProjError) as e:
            ph.forward_slab(k0, k1, t, t, t, t)
        assert e.value.status == mp.MONC_PROJ_EINVAL
    for j0, j1 in ((0, 0), (0, 17), (-2, 3)):
        with pytest.raises(mp.ProjError) as e:
            ph.vertical_pencil(j0, j1, t, t)
        assert e.value.status == mp.MONC_PROJ_EINVAL
    with pytest.raises(mp.ProjError) as e:
        ph.pack(0, 2, t, t)
    assert e.value.status == mp.MONC_PROJ_EINVAL
    ph.close()
    ref = _phases(g, "refined")
    with pytest.raises(mp.ProjError) as e:
        ref.forward_slab(0, 2, t, t, t, t)
    assert e.value.status == mp.MONC_PROJ_EUNSUPPORTED
    ref.close()
