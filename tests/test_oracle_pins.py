"""Pins of the FP64 CPU oracle against mathematics that does not come from it.

Each test ties one part of the oracle to something independent of its own
code path: closed-form transforms, a direct double sum, a dense least-squares
solve of the assembled operator, second-order convergence of the stencils to
calculus, summation by parts, a divergence-free field built from a
streamfunction, manufactured solutions, and projection invariants.
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_12849_gb300 import workloads as W


def small_grid(nx, ny, nz, stretched=True, dx=50.0, dy=40.0):
    dz = W.geometric_dz(nz, 10.0, 60.0) if stretched else W.uniform_dz(nz, 25.0)
    return W.make_grid(nx, ny, nz, dx, dy, dz)


def fields(g, seed, mode=False):
    return W.random_fields(g, seed, mode)


# ---------------------------------------------------------------- DFT pins

@pytest.mark.parametrize("n,m", [(8, 1), (8, 3), (12, 5), (15, 2), (16, 8)])
def test_dft_single_cosine_closed_form(n, m):
    # f(i) = cos(2 pi m i / n) has DFT n/2 at +-m (n at m=n/2), zero elsewhere.
    ny = 3
    i = np.arange(n)
    f = np.tile(np.cos(2 * np.pi * m * i / n), (1, ny, 1))
    X = O.forward_dft2(f)[0]                  # (ny, nxh)
    expect = np.zeros_like(X)
    expect[0, m] = n * ny * (1.0 if 2 * m == n else 0.5)
    assert np.max(np.abs(X - expect)) < 1e-11 * n * ny


def test_dft2_against_direct_double_sum():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((2, 6, 8))
    X = O.forward_dft2(f)
    nz, ny, nx = f.shape
    j = np.arange(ny)[:, None]
    i = np.arange(nx)[None, :]
    for k in range(nz):
        for ky in range(ny):
            for kx in range(nx // 2 + 1):
                s = np.sum(f[k] * np.exp(-2j * np.pi * (kx * i / nx + ky * j / ny)))
                assert abs(X[k, ky, kx] - s) < 1e-12 * 48


@pytest.mark.parametrize("shape", [(2, 8, 8), (3, 9, 10), (1, 5, 7), (2, 6, 15)])
def test_dft_roundtrip_and_parseval(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape)
    X = O.forward_dft2(f)
    back = O.inverse_dft2(X, shape[2])
    assert np.max(np.abs(back - f)) < 1e-12
    # Parseval on the half spectrum: interior kx count twice.
    nx, ny = shape[2], shape[1]
    wts = np.full(nx // 2 + 1, 2.0)
    wts[0] = 1.0
    if nx % 2 == 0:
        wts[-1] = 1.0
    e_spec = np.sum(wts[None, None, :] * np.abs(X) ** 2) / (nx * ny)
    assert abs(e_spec - np.sum(f ** 2)) < 1e-10 * np.sum(f ** 2)


def test_mode_dft_matches_full_transform():
    rng = np.random.default_rng(2)
    f = rng.standard_normal((3, 10, 12))
    X = O.forward_dft2(f)
    kx = np.array([0, 1, 6, 3])
    ky = np.array([0, 9, 5, 2])
    S = O.mode_dft(f, kx, ky)
    assert np.max(np.abs(S - X[:, ky, kx])) < 1e-11


# ---------------------------------------------------------------- Thomas pin

def test_thomas_against_dense_solve():
    rng = np.random.default_rng(3)
    n, m = 17, 5
    sub = rng.uniform(0.1, 1.0, (n, m))
    sup = rng.uniform(0.1, 1.0, (n, m))
    diag = -(sub + sup) - rng.uniform(0.0, 0.5, (n, m))
    rhs = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    x = O.thomas(sub, diag, sup, rhs)
    for c in range(m):
        A = np.diag(diag[:, c]) + np.diag(sub[1:, c], -1) + np.diag(sup[:-1, c], 1)
        ref = np.linalg.solve(A, rhs[:, c])
        assert np.max(np.abs(x[:, c] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_modified_wavenumber_is_second_difference_eigenvalue():
    n, d = 12, 7.0
    lam = O.modified_wavenumbers(n, d)
    i = np.arange(n)
    for k in range(n):
        e = np.exp(2j * np.pi * k * i / n)
        lap = (np.roll(e, -1) - 2 * e + np.roll(e, 1)) / d ** 2
        assert np.max(np.abs(lap - lam[k] * e)) < 1e-14


# ---------------------------------------------------------------- stencils vs calculus

def _convergence_ratio(errs):
    return errs[0] / errs[1]


def test_divergence_second_order_against_analytic():
    # Smooth periodic-in-x,y fields on a uniform vertical grid; compare the
    # discrete D with the analytic (1/rho0) d(rho0 w)/dz + du/dx + dv/dy at
    # the cell centres.  Halving the spacing must cut the error about 4x.
    errs = []
    for n in (16, 32):
        nz = n
        lx, ly, h = 1000.0, 800.0, 600.0
        dz = W.uniform_dz(nz, h / nz)
        g = W.make_grid(n, n, nz, lx / n, ly / n, dz, scale_height=500.0)
        zf, zc, _ = O.grid_metrics(g.dz)
        xe = (np.arange(n) + 1.0) * g.dx
        xc = (np.arange(n) + 0.5) * g.dx
        yn = (np.arange(n) + 1.0) * g.dy
        yc = (np.arange(n) + 0.5) * g.dy
        kx, ky = 2 * np.pi / lx, 2 * np.pi / ly
        u = np.sin(kx * xe)[None, None, :] * np.cos(ky * yc)[None, :, None] * np.ones((nz, 1, 1))
        v = np.cos(kx * xc)[None, None, :] * np.sin(ky * yn)[None, :, None] * np.ones((nz, 1, 1))
        wz = np.sin(np.pi * zf / h)
        w = wz[:, None, None] * np.cos(kx * xc)[None, None, :] * np.cos(ky * yc)[None, :, None]
        D = O.divergence(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
        # analytic: du/dx + dv/dy + (1/rho) d(rho w)/dz, rho = 1.2 exp(-z/Hs)
        hs = 500.0
        dwdz = (np.pi / h) * np.cos(np.pi * zc / h) - np.sin(np.pi * zc / h) / hs
        exact = (kx * np.cos(kx * xc)[None, None, :] * np.cos(ky * yc)[None, :, None]
                 + ky * np.cos(kx * xc)[None, None, :] * np.cos(ky * yc)[None, :, None]
                 + dwdz[:, None, None] * np.cos(kx * xc)[None, None, :] * np.cos(ky * yc)[None, :, None])
        errs.append(np.max(np.abs(D - exact)))
    assert 3.3 < _convergence_ratio(errs) < 4.8


def test_gradient_second_order_against_analytic():
    errs = []
    for n in (16, 32):
        nz = n
        lx, ly, h = 1000.0, 800.0, 600.0
        g = W.make_grid(n, n, nz, lx / n, ly / n, W.geometric_dz(nz, h / nz * 0.8, h / nz * 1.25))
        zf, zc, _ = O.grid_metrics(g.dz)
        xc = (np.arange(n) + 0.5) * g.dx
        yc = (np.arange(n) + 0.5) * g.dy
        kx, ky = 2 * np.pi / lx, 2 * np.pi / ly
        f = lambda z: np.cos(np.pi * z / zf[-1])
        df = lambda z: -np.pi / zf[-1] * np.sin(np.pi * z / zf[-1])
        phi = f(zc)[:, None, None] * np.sin(kx * xc)[None, None, :] * np.sin(ky * yc)[None, :, None]
        gx, gy, gz = O.gradient(phi, g.dx, g.dy, g.dz)
        xe = xc + 0.5 * g.dx
        yn = yc + 0.5 * g.dy
        ex = f(zc)[:, None, None] * kx * np.cos(kx * xe)[None, None, :] * np.sin(ky * yc)[None, :, None]
        ey = f(zc)[:, None, None] * ky * np.sin(kx * xc)[None, None, :] * np.cos(ky * yn)[None, :, None]
        ez = df(zf)[1:-1, None, None] * np.sin(kx * xc)[None, None, :] * np.sin(ky * yc)[None, :, None]
        # the vertical difference is centred at the midpoint of the two centres
        zm = 0.5 * (zc[1:] + zc[:-1])
        ezm = df(zm)[:, None, None] * np.sin(kx * xc)[None, None, :] * np.sin(ky * yc)[None, :, None]
        errs.append(max(np.max(np.abs(gx - ex)), np.max(np.abs(gy - ey)),
                        np.max(np.abs(gz[1:-1] - ezm))))
        assert np.all(gz[0] == 0) and np.all(gz[-1] == 0)
        del ez
    assert 3.3 < _convergence_ratio(errs) < 4.8


def test_gradient_is_negative_weighted_adjoint_of_divergence():
    # sum_W (G phi) . u = - sum_{rho_c dz} phi D(u), W_u = W_v = rho_c dz,
    # W_w = rho_f dzn on interior faces (summation by parts, periodic x, y).
    g = small_grid(6, 5, 7)
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((7, 5, 6))
    u, v, w = fields(g, 11)
    _, _, dzn = O.grid_metrics(g.dz)
    gx, gy, gz = O.gradient(phi, g.dx, g.dy, g.dz)
    wc = (g.rho_c * g.dz)[:, None, None]
    wf = (g.rho_f[1:-1] * dzn[1:-1])[:, None, None]
    lhs = np.sum(wc * gx * u) + np.sum(wc * gy * v) + np.sum(wf * gz[1:-1] * w[1:-1])
    rhs = -np.sum(wc * phi * O.divergence(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)


# ---------------------------------------------------------------- whole solve vs dense

def dense_laplacian(g):
    """L = D o G assembled column by column from the oracle's stencils."""
    n = g.nx * g.ny * g.nz
    L = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        gx, gy, gz = O.gradient(e.reshape(g.nz, g.ny, g.nx), g.dx, g.dy, g.dz)
        L[:, c] = O.divergence(gx, gy, gz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f).ravel()
    return L


@pytest.mark.parametrize("shape", [(4, 4, 3), (6, 5, 4), (8, 8, 8), (9, 6, 7)])
def test_projection_against_dense_least_squares(shape):
    nx, ny, nz = shape
    g = small_grid(nx, ny, nz)
    u, v, w = fields(g, 7, mode=True)
    L = dense_laplacian(g)
    b = O.divergence(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f).ravel()
    # the pin: horizontal mean of phi at level 0 is zero
    pin = np.zeros(L.shape[1])
    pin[: nx * ny] = 1.0
    A = np.vstack([L, pin])
    phi_ref = np.linalg.lstsq(A, np.append(b, 0.0), rcond=None)[0].reshape(nz, ny, nx)
    gx, gy, gz = O.gradient(phi_ref, g.dx, g.dy, g.dz)
    uo, vo, wo, phi = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    scale = np.max(np.abs(phi_ref))
    assert np.max(np.abs(phi - phi_ref)) < 1e-11 * scale
    w_in = w.copy()
    w_in[0] = 0
    w_in[-1] = 0
    for out, ref in ((uo, u - gx), (vo, v - gy), (wo, w_in - gz)):
        assert np.max(np.abs(out - ref)) < 1e-11


# ---------------------------------------------------------------- manufactured solutions

def test_manufactured_single_mode():
    # u* = G phi_exact with phi_exact = cos(2 pi x/Lx) cos(2 pi y/Ly) f(z):
    # the solve returns phi_exact (its level-0 mean is zero) and u = 0; the
    # divergence's spectrum lives only at (kx, ky) = (+-1, +-1).
    nx, ny, nz = 16, 12, 10
    g = small_grid(nx, ny, nz)
    zf, zc, _ = O.grid_metrics(g.dz)
    xc = (np.arange(nx) + 0.5) * g.dx
    yc = (np.arange(ny) + 0.5) * g.dy
    f = np.exp(-zc / 300.0) + 0.3 * zc / zf[-1]
    phi_ex = (f[:, None, None] * np.cos(2 * np.pi * xc / (nx * g.dx))[None, None, :]
              * np.cos(2 * np.pi * yc / (ny * g.dy))[None, :, None])
    u, v, w = O.gradient(phi_ex, g.dx, g.dy, g.dz)
    D = O.divergence(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    Dh = O.forward_dft2(D)
    mask = np.ones(Dh.shape[1:], bool)
    mask[1, 1] = False
    mask[ny - 1, 1] = False
    assert np.max(np.abs(Dh[:, mask])) < 1e-9 * np.max(np.abs(Dh))
    uo, vo, wo, phi = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert np.max(np.abs(phi - phi_ex)) < 1e-11 * np.max(np.abs(phi_ex))
    vmax = max(np.max(np.abs(u)), np.max(np.abs(v)), np.max(np.abs(w)))
    for out in (uo, vo, wo):
        assert np.max(np.abs(out)) < 1e-11 * vmax


def streamfunction_field(g, seed):
    """Horizontally divergence-free velocities from a corner streamfunction."""
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((g.nz, g.ny, g.nx))     # at (x=(i+1)dx, y=(j+1)dy)
    u = (psi - np.roll(psi, 1, axis=1)) / g.dy
    v = -(psi - np.roll(psi, 1, axis=2)) / g.dx
    w = np.zeros((g.nz + 1, g.ny, g.nx))
    return u, v, w


def test_divergence_free_part_is_preserved():
    g = small_grid(12, 10, 9)
    u_df, v_df, w_df = streamfunction_field(g, 21)
    assert np.max(np.abs(O.divergence(u_df, v_df, w_df, g.dx, g.dy, g.dz, g.rho_c, g.rho_f))) < 1e-13
    rng = np.random.default_rng(22)
    phi_ex = rng.standard_normal((g.nz, g.ny, g.nx))
    phi_ex -= phi_ex[0].mean()
    gx, gy, gz = O.gradient(phi_ex, g.dx, g.dy, g.dz)
    uo, vo, wo, phi = O.project(u_df + gx, v_df + gy, w_df + gz, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert np.max(np.abs(uo - u_df)) < 1e-12 * np.max(np.abs(u_df))
    assert np.max(np.abs(vo - v_df)) < 1e-12 * np.max(np.abs(v_df))
    assert np.max(np.abs(wo)) < 1e-12 * np.max(np.abs(gz))
    assert np.max(np.abs(phi - phi_ex)) < 1e-11 * np.max(np.abs(phi_ex))


# ---------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def projected():
    g = small_grid(16, 12, 11)
    u, v, w = fields(g, 3, mode=True)
    out = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    return g, (u, v, w), out


def test_divergence_free_output(projected):
    g, (u, v, w), (uo, vo, wo, _) = projected
    r = O.divergence_residual(uo, vo, wo, u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert r < 1e-10


def test_idempotent(projected):
    g, _, (uo, vo, wo, _) = projected
    u2, v2, w2, phi2 = O.project(uo, vo, wo, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    for a, b in ((u2, uo), (v2, vo), (w2, wo)):
        assert np.max(np.abs(a - b)) < 1e-12
    assert np.max(np.abs(phi2)) < 1e-9


def _wdot(g, a, b):
    _, _, dzn = O.grid_metrics(g.dz)
    wc = (g.rho_c * g.dz)[:, None, None]
    wf = (g.rho_f[1:-1] * dzn[1:-1])[:, None, None]
    return (np.sum(wc * a[0] * b[0]) + np.sum(wc * a[1] * b[1])
            + np.sum(wf * a[2][1:-1] * b[2][1:-1]))


def test_self_adjoint_and_energy(projected):
    g, a, pa = projected
    b = fields(g, 99)
    pb = O.project(*b, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    lhs = _wdot(g, pa, b)
    rhs = _wdot(g, a, pb)
    assert abs(lhs - rhs) < 1e-11 * abs(_wdot(g, a, a))
    assert _wdot(g, pa, pa) <= _wdot(g, a, a)


def test_horizontal_mean_w_vanishes(projected):
    _, _, (_, _, wo, _) = projected
    assert np.max(np.abs(wo.mean(axis=(1, 2)))) < 1e-13


def test_linearity():
    g = small_grid(8, 10, 6)
    a = fields(g, 1)
    b = fields(g, 2)
    pa = O.project(*a, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    pb = O.project(*b, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    c = tuple(2.5 * x - 0.75 * y for x, y in zip(a, b))
    pc = O.project(*c, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    for i in range(4):
        assert np.max(np.abs(pc[i] - (2.5 * pa[i] - 0.75 * pb[i]))) < 1e-11 * (1 + np.max(np.abs(pc[i])))


def test_project_modes_matches_full_projection(projected):
    g, (u, v, w), (uo, vo, wo, phi) = projected
    kx = np.array([0, 1, 3, 8, 2])
    ky = np.array([0, 11, 6, 0, 5])
    ref = O.project_modes(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, kx, ky)
    for name, out in (("u", uo), ("v", vo), ("w", wo)):
        got = O.mode_dft(out, kx, ky)
        assert np.max(np.abs(got - ref[name])) < 1e-10 * (1 + np.max(np.abs(ref[name])))
