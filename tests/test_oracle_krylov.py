"""Pins of the Krylov oracle (oracle/krylov.py) against mathematics outside it.

* the stencil L against the operator assembled column by column from the
  (separately pinned) divergence and gradient;
* the line preconditioner against numpy's dense solve of the assembled line
  matrix;
* BiCGStab against numpy's dense solve of a small nonsymmetric system, one
  iteration with an exact preconditioner, and finite termination on a matrix
  with three distinct eigenvalues;
* the whole Krylov projection against the FFT oracle, itself pinned by a dense
  least-squares solve (test_oracle_pins).

Planted mistakes in the Krylov oracle (at the bottom) must each fail a pin.
"""
import numpy as np
import pytest

import oracle as O
import oracle.krylov as K
from tests.test_oracle_pins import dense_laplacian, fields, small_grid


def test_laplacian_matches_assembled_divergence_of_gradient():
    g = small_grid(6, 5, 7)
    L = dense_laplacian(g)
    x = np.random.default_rng(3).standard_normal((g.nz, g.ny, g.nx))
    ref = (L @ x.ravel()).reshape(x.shape)
    out = K.laplacian(x, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))


def test_line_solve_against_dense_solve():
    g = small_grid(4, 3, 9)
    sub, diag, sup = K.line_operator(g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    # the line matrix from the assembled operator: the vertical couplings of
    # one column plus the diagonal of the whole operator
    L = dense_laplacian(g)
    col = np.arange(g.nz) * g.nx * g.ny            # column (i, j) = (0, 0)
    M = np.zeros((g.nz, g.nz))
    for a in range(g.nz):
        for b in range(g.nz):
            if abs(a - b) <= 1:
                M[a, b] = L[col[a], col[b]]
    assert np.allclose(np.diag(M), diag, rtol=1e-14, atol=0)
    r = np.random.default_rng(4).standard_normal((g.nz, g.ny, g.nx))
    z = K.line_solve(r, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    ref = np.linalg.solve(M, r.reshape(g.nz, -1)).reshape(r.shape)
    assert np.max(np.abs(z - ref)) < 1e-12 * np.max(np.abs(ref))


def test_bicgstab_against_dense_solve():
    rng = np.random.default_rng(5)
    n = 40
    A = rng.standard_normal((n, n)) + 12.0 * np.eye(n)
    b = rng.standard_normal(n)
    d = np.diag(A).copy()
    x, it, relres, status = K.bicgstab(b, lambda y: A @ y, lambda r: r / d, 1e-13, 200)
    assert status == K.KRYLOV_CONVERGED
    assert relres <= 1e-13
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(x - ref)) < 1e-11 * np.max(np.abs(ref))
    # the reported residual is the true residual up to the recurrence's rounding
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 10 * 1e-13


def test_bicgstab_exact_preconditioner_converges_in_one_iteration():
    rng = np.random.default_rng(6)
    d = rng.uniform(1.0, 3.0, 30)
    b = rng.standard_normal(30)
    x, it, _, status = K.bicgstab(b, lambda y: d * y, lambda r: r / d, 1e-14, 10)
    assert status == K.KRYLOV_CONVERGED and it == 1
    assert np.max(np.abs(x - b / d)) < 1e-14 * np.max(np.abs(b / d))


def test_bicgstab_finite_termination_with_three_distinct_eigenvalues():
    # The BiCGStab residual is Q_i(A) P_i(A) r_0 with P_i the BiCG residual
    # polynomial of degree i; with three distinct eigenvalues the BiCG
    # polynomial of degree 3 annihilates r_0, so the method ends within three
    # iterations (exact arithmetic; here to rounding).
    rng = np.random.default_rng(8)
    d = np.repeat([1.0, 2.5, 7.0], 10)
    rng.shuffle(d)
    b = rng.standard_normal(30)
    x, it, relres, status = K.bicgstab(b, lambda y: d * y, lambda r: r, 1e-12, 10)
    assert status == K.KRYLOV_CONVERGED and it <= 3
    assert np.max(np.abs(x - b / d)) < 1e-11


def test_bicgstab_zero_rhs_and_max_iter():
    x, it, relres, status = K.bicgstab(np.zeros(5), lambda y: 2 * y, lambda r: r, 1e-10, 10)
    assert it == 0 and status == K.KRYLOV_CONVERGED and not np.any(x)
    rng = np.random.default_rng(7)
    A = rng.standard_normal((30, 30)) + 3.0 * np.eye(30)
    x, it, relres, status = K.bicgstab(rng.standard_normal(30), lambda y: A @ y, lambda r: r, 0.0, 3)
    assert status == K.KRYLOV_MAX_ITER and it == 3 and relres > 0


@pytest.mark.parametrize("precond", ["line", "none"])
def test_krylov_projection_matches_fft_oracle(precond):
    g = small_grid(8, 6, 5)
    u, v, w = fields(g, 11, mode=True)
    ref = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    uo, vo, wo, phi, it, relres, status = K.project_krylov(
        u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, 1e-13, 2000, precond)
    assert status == K.KRYLOV_CONVERGED and relres <= 1e-13
    assert np.max(np.abs(phi - ref[3])) < 1e-9 * np.max(np.abs(ref[3]))
    vmax = max(np.max(np.abs(a)) for a in (u, v, w))
    for out, r in zip((uo, vo, wo), ref[:3]):
        assert np.max(np.abs(out - r)) < 1e-9 * vmax


def test_line_preconditioner_cuts_iterations_on_a_stretched_grid():
    g = small_grid(12, 10, 16, dx=25.0, dy=25.0)
    u, v, w = fields(g, 12, mode=True)
    its = {}
    for pc in ("line", "none"):
        its[pc] = K.project_krylov(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, 1e-8, 3000, pc)[4]
    assert its["line"] < its["none"]


# ---------------------------------------------------------------- planted mistakes

def _pins():
    return [
        test_laplacian_matches_assembled_divergence_of_gradient,
        test_line_solve_against_dense_solve,
        test_bicgstab_against_dense_solve,
        test_bicgstab_exact_preconditioner_converges_in_one_iteration,
        test_bicgstab_finite_termination_with_three_distinct_eigenvalues,
        lambda: test_krylov_projection_matches_fft_oracle("line"),
    ]


def _some_pin_fails():
    for pin in _pins():
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError, ZeroDivisionError):
            return True
    return False


_orig = {name: getattr(K, name) for name in ("vertical_operator", "line_operator", "bicgstab", "_dot")}


def _vertical_sign_flipped(dz, rho_c, rho_f):
    sub, diag0, sup = _orig["vertical_operator"](dz, rho_c, rho_f)
    return sub, diag0, -sup


def _line_without_horizontal_diagonal(dx, dy, dz, rho_c, rho_f):
    sub, diag, sup = _orig["line_operator"](dx, dy, dz, rho_c, rho_f)
    return sub, diag + 2.0 / (dx * dx) + 2.0 / (dy * dy), sup


def _bicgstab_beta_without_omega(b, apply_a, apply_m, tol, max_iter):
    # the search-direction update p = r + beta (p - omega v) written as r + beta p
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b)
    bnorm = np.sqrt(np.sum(b * b))
    r = b.copy()
    rt = r.copy()
    p = np.zeros_like(b)
    rho_prev = alpha = omega = 1.0
    relres = 1.0
    for i in range(1, max_iter + 1):
        rho = float(np.sum(rt * r))
        p = r.copy() if i == 1 else r + (rho / rho_prev) * (alpha / omega) * p
        ph = apply_m(p)
        vv = apply_a(ph)
        alpha = rho / float(np.sum(rt * vv))
        s = r - alpha * vv
        if np.sqrt(np.sum(s * s)) <= tol * bnorm:
            return x + alpha * ph, i, 0.0, K.KRYLOV_CONVERGED
        sh = apply_m(s)
        t = apply_a(sh)
        omega = float(np.sum(t * s)) / float(np.sum(t * t))
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        relres = np.sqrt(np.sum(r * r)) / bnorm
        if relres <= tol:
            return x, i, relres, K.KRYLOV_CONVERGED
        rho_prev = rho
    return x, max_iter, relres, K.KRYLOV_MAX_ITER


MUTATIONS = {
    "vertical coupling sign": ("vertical_operator", _vertical_sign_flipped),
    "line preconditioner without the horizontal diagonal": ("line_operator", _line_without_horizontal_diagonal),
    "search direction without the omega v term": ("bicgstab", _bicgstab_beta_without_omega),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_krylov_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(K, attr, fn)
    assert _some_pin_fails(), f"no pin caught: {name}"


def test_unmutated_krylov_oracle_passes_every_pin():
    assert not _some_pin_fails()
