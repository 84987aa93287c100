"""GPU projection vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (relative L2 over u, v, w stacked; see the projection's error
statement): FP64 path 1e-12; mixed path 1e-5 with the divergence residual
||D(u_out)|| / ||D(u_in)|| <= 1e-6, evaluated in FP64 on the host.  For the
mixed path the oracle is fed the same FP32-rounded inputs, upcast, so the
error measured is the solver's alone.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2009_12849_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5, "refined": 1e-12}
DIV_TOL = {"fp64": 1e-10, "mixed": 1e-6, "refined": 1e-10}


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def run_gpu(g, u, v, w, prec, phi=True, inplace=False):
    mp = _mp()
    dev = torch.device("cuda", 0)
    dt = mp.DTYPES[mp.PRECISIONS[prec]]
    P = mp.Projector.from_grid(g, prec, dev)
    tu, tv, tw = (torch.tensor(a, dtype=dt, device=dev) for a in (u, v, w))
    out = (tu, tv, tw) if inplace else None
    res = P.solve(tu, tv, tw, out=out, phi=phi)
    torch.cuda.synchronize()
    assert P.sync_status() == 0
    res = [r.double().cpu().numpy() for r in res]
    P.close()
    return res


def rounded_inputs(u, v, w, prec):
    if prec != "mixed":
        return u, v, w
    return tuple(a.astype(np.float32).astype(np.float64) for a in (u, v, w))


def rel(a_list, b_list):
    a = np.concatenate([x.ravel() for x in a_list])
    b = np.concatenate([x.ravel() for x in b_list])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_case(g, seed, mode, prec, phi=True, inplace=False):
    u, v, w = W.random_fields(g, seed, mode)
    u, v, w = rounded_inputs(u, v, w, prec)
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    got = run_gpu(g, u, v, w, prec, phi=phi, inplace=inplace)
    err = rel(got[:3], ref[:3])
    assert err < TOL[prec], f"{prec} {g.nx}x{g.ny}x{g.nz}: rel err {err:.3e}"
    div = O.divergence_residual(*got[:3], u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert div < DIV_TOL[prec], f"divergence residual {div:.3e}"
    if phi:
        # phi carries the same pin (level-0 horizontal mean zero) in both
        ephi = np.linalg.norm(got[3] - ref[3]) / np.linalg.norm(ref[3])
        assert ephi < {"fp64": 1e-11, "refined": 1e-9}.get(prec, 1e-4), f"phi rel err {ephi:.3e}"
    # the bottom and top faces of w are zero
    assert np.all(got[2][0] == 0) and np.all(got[2][-1] == 0)
    return err, div


@pytest.mark.parametrize("prec", ["fp64", "mixed", "refined"])
def test_64cube_uniform(prec):
    g, seed, mode = W.workload_64cube()
    check_case(g, seed, mode, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(48, 40, 12), (96, 96, 20), (30, 45, 7), (75, 64, 9),
                                   (15, 16, 5), (160, 20, 6), (2, 8, 3), (8, 2, 4),
                                   (128, 192, 8), (192, 128, 5), (512, 256, 3), (256, 512, 3),
                                   (1024, 64, 3), (64, 1024, 2),
                                   # extended compile-time lengths (FP32), odd and radix-3/5 ones
                                   (135, 150, 4), (375, 243, 3), (500, 405, 2), (162, 486, 2),
                                   (225, 288, 3), (480, 320, 2), (250, 243, 2)])
def test_ragged_and_mixed_radix(shape, prec):
    nx, ny, nz = shape
    g = W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))
    check_case(g, 5, True, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "refined"])
def test_single_level(prec):
    g = W.make_grid(32, 16, 1, 25.0, 25.0, W.uniform_dz(1, 30.0))
    check_case(g, 9, False, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "refined"])
def test_in_place_and_no_phi(prec):
    g = W.make_grid(64, 48, 10, 25.0, 25.0, W.geometric_dz(10, 10.0, 50.0))
    check_case(g, 3, True, prec, phi=False, inplace=True)


def test_256x128_fp64_full_oracle():
    g, seed, mode = W.workload_256()
    err, div = check_case(g, seed, mode, "fp64", phi=False)
    print(f"256x256x128 fp64: rel err {err:.3e}, div {div:.3e}")


def test_deterministic_bitwise():
    g = W.make_grid(96, 64, 16, 25.0, 25.0, W.geometric_dz(16, 10.0, 80.0))
    u, v, w = W.random_fields(g, 1, True)
    for prec in ("fp64", "mixed"):
        a = run_gpu(g, u, v, w, prec)
        b = run_gpu(g, u, v, w, prec)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_invalid_arguments_rejected():
    mp = _mp()
    g = W.make_grid(14, 16, 4, 25.0, 25.0, W.uniform_dz(4, 10.0))   # 14 = 2*7
    with pytest.raises(mp.ProjError) as e:
        mp.Projector.from_grid(g, "fp64")
    assert e.value.status == mp.MONC_PROJ_EUNSUPPORTED
    g = W.make_grid(16, 16, 4, 25.0, 25.0, W.uniform_dz(4, 10.0))
    bad = g.dz.copy()
    bad[2] = -1.0
    with pytest.raises(mp.ProjError) as e:
        mp.Projector(16, 16, 4, 25.0, 25.0, bad, g.rho_c, g.rho_f)
    assert e.value.status == mp.MONC_PROJ_EINVAL
    with pytest.raises(mp.ProjError):
        mp.Projector(16, 16, 4, float("nan"), 25.0, g.dz, g.rho_c, g.rho_f)
    P = mp.Projector.from_grid(g, "fp64")
    t = torch.zeros((4, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(mp.ProjError):
        P.solve(t, t, torch.zeros((5, 16, 16), dtype=torch.float32, device="cuda"))
    rc = mp.load_library().monc_proj_solve(None, None, None, None, None, None, None, None, None, None)
    assert rc == mp.MONC_PROJ_EINVAL
    P.close()


@pytest.mark.parametrize("shape", [(128, 192, 8), (256, 512, 3), (96, 1024, 4)])
def test_opt_in_kernel_variants(shape, monkeypatch):
    """The opt-in column kernels (TMA-staged tiles; persistent cp.async
    tiles) give the same projection as the default kernels."""
    nx, ny, nz = shape
    g = W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))
    for var in ("MONC_PROJ_TMA", "MONC_PROJ_PERSIST_COLS"):
        monkeypatch.setenv(var, "1")
        check_case(g, 5, True, "mixed")
        monkeypatch.delenv(var)


@pytest.mark.parametrize("shape", [(48, 40, 12), (30, 45, 7), (128, 192, 8), (384, 96, 4), (1024, 64, 3),
                                   (256, 256, 16)])
def test_refined_reaches_fp64_accuracy(shape):
    """The refinement passes on FP64 fields agree with the FP64 oracle at FP64
    tolerance, on compile-time and run-time lengths."""
    nx, ny, nz = shape
    g = W.make_grid(nx, ny, nz, 25.0, 20.0, W.geometric_dz(nz, 10.0, 100.0))
    err, div = check_case(g, 11, True, "refined")
    print(f"refined {shape}: rel err {err:.3e}, div {div:.3e}")
