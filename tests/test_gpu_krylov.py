"""GPU BiCGStab pressure solver vs the FP64 CPU oracles, through the C ABI.

* A fixed number of iterations (tol = 0): the GPU iterate, projected, against
  the Krylov oracle's after the same iterations, element by element (both
  FP64; they differ by rounding order only, 1e-9 relative allowed).
* Converged (tol = 1e-12): against the FFT oracle's exact discrete solution
  (1e-9 relative L2 on u, v, w); iterations to 1e-6 within 10% of the
  oracle's.
* The paper's stopping criterion (1e-4) on a larger grid against the GPU FFT
  path, edge cases and argument checks.
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.krylov as K
from paper_2009_12849_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mp():
    import __graft_entry__ as ge
    ge.build()
    from paper_2009_12849_gb300 import monc_proj
    return monc_proj


def grid(nx, ny, nz, dx=40.0, dy=30.0):
    return W.make_grid(nx, ny, nz, dx, dy, W.geometric_dz(nz, 10.0, 60.0))


def run(g, u, v, w, tol, max_iter, precond, inplace=False, precision="fp64"):
    mp = _mp()
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, precision, dev)
    dt = mp.DTYPES[mp.PRECISIONS[precision]]
    tu, tv, tw = (torch.tensor(a, dtype=dt, device=dev) for a in (u, v, w))
    out = (tu, tv, tw) if inplace else None
    uo, vo, wo, phi, st, it, rr = P.solve_krylov(tu, tv, tw, tol, max_iter, precond, out=out, phi=True)
    torch.cuda.synchronize()
    res = [t.double().cpu().numpy() for t in (uo, vo, wo, phi)]
    P.close()
    return res, st, it, rr


def relmax(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("precond", ["line", "none"])
@pytest.mark.parametrize("iters", [1, 4, 10])
def test_fixed_iterations_match_oracle(precond, iters):
    mp = _mp()
    g = grid(24, 20, 16)
    u, v, w = W.random_fields(g, 21, True)
    ref = K.project_krylov(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, 0.0, iters, precond)
    got, st, it, rr = run(g, u, v, w, 0.0, iters, precond)
    assert st == mp.MONC_PROJ_ENOCONV and ref[6] == K.KRYLOV_MAX_ITER
    assert it == iters == ref[4]
    assert abs(rr - ref[5]) <= 1e-8 * ref[5]
    assert relmax(got[3], ref[3]) < 1e-9
    for a, b in zip(got[:3], ref[:3]):
        assert relmax(a, b) < 1e-9
    assert np.all(got[2][0] == 0) and np.all(got[2][-1] == 0)


@pytest.mark.parametrize("precond", ["line", "none"])
def test_converged_matches_fft_oracle(precond):
    mp = _mp()
    g = grid(32, 30, 20)
    u, v, w = W.random_fields(g, 22, True)
    fft = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    kry = K.project_krylov(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, 1e-12, 5000, precond)
    got, st, it, rr = run(g, u, v, w, 1e-12, 5000, precond)
    assert st == mp.MONC_PROJ_OK and rr <= 1e-12
    assert kry[6] == K.KRYLOV_CONVERGED
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got[:3], fft[:3])))
    den = np.sqrt(sum(np.sum(b ** 2) for b in fft[:3]))
    assert num / den < 1e-9
    assert np.linalg.norm(got[3] - fft[3]) / np.linalg.norm(fft[3]) < 1e-8
    assert abs(np.mean(got[3][0])) < 1e-12 * np.max(np.abs(got[3]))
    div = O.divergence_residual(*got[:3], u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert div < 1e-11


@pytest.mark.parametrize("precond", ["line", "none"])
def test_iterations_to_tolerance_match_oracle(precond):
    # Rounding-order differences grow over hundreds of BiCGStab steps (the
    # fixed-iteration test above bounds them over the first ten), so the
    # counts to a moderate tolerance agree to 10%, not exactly.
    mp = _mp()
    g = grid(32, 30, 20)
    u, v, w = W.random_fields(g, 26, True)
    kry = K.project_krylov(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, 1e-6, 5000, precond)
    got, st, it, rr = run(g, u, v, w, 1e-6, 5000, precond)
    assert st == mp.MONC_PROJ_OK and rr <= 1e-6 and kry[6] == K.KRYLOV_CONVERGED
    assert abs(it - kry[4]) <= max(2, 0.1 * kry[4])


def test_paper_tolerance_against_gpu_fft_path():
    # the paper solves to 1e-4; the divergence left is the Krylov residual
    mp = _mp()
    g = grid(128, 96, 48, dx=25.0, dy=25.0)
    u, v, w = W.random_fields(g, 23, True)
    got, st, it, rr = run(g, u, v, w, 1e-4, 2000, "line")
    assert st == mp.MONC_PROJ_OK and rr <= 1e-4 and it > 0
    dev = torch.device("cuda", 0)
    P = mp.Projector.from_grid(g, "fp64", dev)
    tu, tv, tw = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (u, v, w))
    ref = [t.cpu().numpy() for t in P.solve(tu, tv, tw)]
    P.close()
    div = O.divergence_residual(*got[:3], u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert div <= 1.01e-4 and abs(div - rr) <= 1e-3 * rr
    num = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got[:3], ref)))
    den = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip((u, v, w), ref)))
    assert num / den < 5e-2          # error in the removed gradient part, relative to it


def test_in_place_matches_out_of_place():
    g = grid(20, 18, 12)
    u, v, w = W.random_fields(g, 24, True)
    a, st_a, it_a, _ = run(g, u, v, w, 1e-10, 500, "line")
    b, st_b, it_b, _ = run(g, u, v, w, 1e-10, 500, "line", inplace=True)
    assert st_a == st_b and it_a == it_b
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_divergence_free_input_needs_no_iteration():
    mp = _mp()
    g = grid(16, 12, 10)
    u = np.full((g.nz, g.ny, g.nx), 2.5)
    v = np.full((g.nz, g.ny, g.nx), -1.25)
    w = np.zeros((g.nz + 1, g.ny, g.nx))
    got, st, it, rr = run(g, u, v, w, 1e-8, 100, "line")
    assert st == mp.MONC_PROJ_OK and it == 0 and rr == 0.0
    assert np.array_equal(got[0], u) and np.array_equal(got[1], v) and not np.any(got[2]) and not np.any(got[3])


def test_refined_plan_is_accepted():
    mp = _mp()
    g = grid(16, 16, 8)
    u, v, w = W.random_fields(g, 25, False)
    a, st_a, it_a, _ = run(g, u, v, w, 1e-10, 500, "line")
    b, st_b, it_b, _ = run(g, u, v, w, 1e-10, 500, "line", precision="refined")
    assert st_a == st_b == mp.MONC_PROJ_OK and it_a == it_b
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_invalid_arguments():
    mp = _mp()
    dev = torch.device("cuda", 0)
    g = grid(16, 16, 8)
    P = mp.Projector.from_grid(g, "fp64", dev)
    c = torch.zeros((g.nz, g.ny, g.nx), dtype=torch.float64, device=dev)
    f = torch.zeros((g.nz + 1, g.ny, g.nx), dtype=torch.float64, device=dev)
    ws = torch.empty(mp.monc_proj_krylov_workspace_size(P.plan), dtype=torch.uint8, device=dev)
    for kw in ({"tol": -1.0}, {"tol": float("nan")}, {"tol": float("inf")}, {"max_iter": -1}, {"precond": 7}):
        args = {"tol": 1e-6, "max_iter": 10, "precond": "line"}
        args.update(kw)
        with pytest.raises(mp.ProjError) as e:
            mp.monc_proj_solve_krylov(P.plan, c, c, f, c, c, f, None, ws, args["tol"], args["max_iter"],
                                      args["precond"])
        assert e.value.status == mp.MONC_PROJ_EINVAL
    with pytest.raises(mp.ProjError) as e:
        mp.monc_proj_solve_krylov(P.plan, c, c, f, c, c, f, None, None, 1e-6, 10, "line")
    assert e.value.status == mp.MONC_PROJ_EINVAL
    P.close()


# ---------------------------------------------------------------- FP32 vectors (mixed plans)

def fp32_inputs(g, seed):
    return tuple(a.astype(np.float32).astype(np.float64) for a in W.random_fields(g, seed, True))


@pytest.mark.parametrize("precond", ["line", "none"])
def test_fp32_fixed_iterations_close_to_oracle(precond):
    # FP32 vectors against the FP64 oracle on the same (FP32-rounded) inputs:
    # after a few iterations the two differ by FP32 rounding only
    mp = _mp()
    g = grid(24, 20, 16)
    u, v, w = fp32_inputs(g, 27)
    ref = K.project_krylov(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, 0.0, 4, precond)
    got, st, it, rr = run(g, u, v, w, 0.0, 4, precond, precision="mixed")
    assert st == mp.MONC_PROJ_ENOCONV and it == 4
    assert abs(rr - ref[5]) <= 1e-3 * ref[5]
    assert relmax(got[3], ref[3]) < 1e-4
    for a, b in zip(got[:3], ref[:3]):
        assert relmax(a, b) < 1e-4


@pytest.mark.parametrize("tol", [1e-4, 1e-5])
def test_fp32_converged_against_fft_oracle(tol):
    mp = _mp()
    g = grid(32, 30, 20)
    u, v, w = fp32_inputs(g, 28)
    fft = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    kry = K.project_krylov(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, tol, 5000, "line")
    got, st, it, rr = run(g, u, v, w, tol, 5000, "line", precision="mixed")
    assert st == mp.MONC_PROJ_OK and rr <= tol
    assert abs(it - kry[4]) <= max(2, 0.2 * kry[4])
    # the divergence left is the Krylov residual (FP32 recurrence vs true residual)
    div = O.divergence_residual(*got[:3], u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert div <= 3 * tol
    # the error against the exact solution is that of the FP64 solver at the same tolerance
    e64 = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(kry[:3], fft[:3])))
    e32 = np.sqrt(sum(np.sum((a - b) ** 2) for a, b in zip(got[:3], fft[:3])))
    den = np.sqrt(sum(np.sum(b ** 2) for b in fft[:3]))
    assert e32 / den <= 3 * e64 / den + 1e-6
