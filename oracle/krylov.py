"""FP64 CPU oracle of the Krylov pressure solver (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It shares no code with the CUDA path.

What it computes (paper, Section 4): besides the FFT solver, the model solves
the same Poisson problem with a Krylov subspace method, BiCGStab with an ILU
preconditioner, whose only global communication is the reduction behind the
residual norm; the paper's closing section names a bespoke preconditioner that
exploits the problem's known structure as further work.  The readings used
here:

* The operator is L = D o G of the FFT solver (``projection.py``), written out
  as its stencil: periodic 3-point second differences in x and y plus the
  vertical rows of ``vertical_operator`` (Neumann at the bottom and top faces).
* Preconditioner ``"line"``: the vertical lines of L, i.e. its vertical part
  plus the diagonal of its horizontal part (-2/dx^2 - 2/dy^2), inverted column
  by column with the Thomas algorithm.  It stands in for ILU: an incomplete
  factorisation sweeps the whole grid one cell after another, while the line
  preconditioner keeps the strong vertical coupling of a stretched grid and
  inverts ny*nx independent columns.  ``"none"`` runs the method without one.
* BiCGStab (H. A. van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) with the
  preconditioner applied to the search directions, in the order of the
  preconditioned algorithm of Barrett et al., "Templates for the Solution of
  Linear Systems" (SIAM, 1994): starting guess 0, shadow residual equal to the
  first residual, and the stopping test ||r||_2 <= tol ||b||_2 on the
  recurrence residual, also taken after the half step on s.
* L is singular (constants); the right-hand side D(u*) is compatible up to
  rounding.  The solution is pinned afterwards as in the FFT solver: the
  horizontal mean of phi at level 0 is made zero, which leaves G phi unchanged.
"""
from __future__ import annotations

import numpy as np

from .projection import divergence, gradient, thomas, vertical_operator

__all__ = [
    "laplacian", "line_operator", "line_solve", "bicgstab", "project_krylov",
    "KRYLOV_CONVERGED", "KRYLOV_MAX_ITER", "KRYLOV_BREAKDOWN",
]

KRYLOV_CONVERGED = 0
KRYLOV_MAX_ITER = 1
KRYLOV_BREAKDOWN = 2


def laplacian(phi, dx, dy, dz, rho_c, rho_f):
    """L phi = D(G phi) as a 7-point stencil, shape (nz, ny, nx).

    (phi_{i+1} - 2 phi_i + phi_{i-1})/dx^2 + (phi_{j+1} - 2 phi_j + phi_{j-1})/dy^2
      + sub[k] phi[k-1] + diag0[k] phi[k] + sup[k] phi[k+1]."""
    phi = np.asarray(phi, np.float64)
    nz = phi.shape[0]
    out = (np.roll(phi, -1, axis=2) - 2.0 * phi + np.roll(phi, 1, axis=2)) / (dx * dx)
    out = out + (np.roll(phi, -1, axis=1) - 2.0 * phi + np.roll(phi, 1, axis=1)) / (dy * dy)
    sub, diag0, sup = vertical_operator(dz, rho_c, rho_f)
    for k in range(nz):
        out[k] = out[k] + diag0[k] * phi[k]
        if k > 0:
            out[k] = out[k] + sub[k] * phi[k - 1]
        if k < nz - 1:
            out[k] = out[k] + sup[k] * phi[k + 1]
    return out


def line_operator(dx, dy, dz, rho_c, rho_f):
    """Rows (sub, diag, sup) of one vertical line of L with the diagonal of its
    horizontal part: the same matrix for every column (i, j)."""
    sub, diag0, sup = vertical_operator(dz, rho_c, rho_f)
    diag = diag0 - 2.0 / (dx * dx) - 2.0 / (dy * dy)
    return sub, diag, sup


def line_solve(r, dx, dy, dz, rho_c, rho_f):
    """M^-1 r for the vertical-line preconditioner: Thomas down every column."""
    r = np.asarray(r, np.float64)
    nz = r.shape[0]
    sub, diag, sup = line_operator(dx, dy, dz, rho_c, rho_f)
    return thomas(sub, diag, sup, r.reshape(nz, -1)).reshape(r.shape)


def _dot(a, b):
    return float(np.sum(a * b))


def bicgstab(b, apply_a, apply_m, tol, max_iter):
    """Preconditioned BiCGStab for A x = b from x = 0.

    apply_a(x) -> A x, apply_m(r) -> M^-1 r.  Returns (x, iterations,
    relative residual ||r||/||b|| of the recurrence, status) with status
    KRYLOV_CONVERGED, KRYLOV_MAX_ITER or KRYLOV_BREAKDOWN (a denominator that
    is zero, or not finite once rounding has driven the method past its
    attainable accuracy).  b = 0 returns x = 0 after no iterations."""
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b)
    bnorm = np.sqrt(_dot(b, b))
    if bnorm == 0.0:
        return x, 0, 0.0, KRYLOV_CONVERGED
    r = b.copy()                                  # r_0 = b - A x_0 with x_0 = 0
    r_tilde = r.copy()
    p = np.zeros_like(b)
    v = np.zeros_like(b)
    rho_prev = alpha = omega = 1.0
    relres = 1.0
    for i in range(1, max_iter + 1):
        rho = _dot(r_tilde, r)
        if rho == 0.0 or not np.isfinite(rho):
            return x, i - 1, relres, KRYLOV_BREAKDOWN
        if i == 1:
            p = r.copy()
        else:
            beta = (rho / rho_prev) * (alpha / omega)
            p = r + beta * (p - omega * v)
        p_hat = apply_m(p)
        v = apply_a(p_hat)
        rv = _dot(r_tilde, v)
        if rv == 0.0 or not np.isfinite(rv):
            return x, i - 1, relres, KRYLOV_BREAKDOWN
        alpha = rho / rv
        s = r - alpha * v
        snorm = np.sqrt(_dot(s, s))
        if snorm <= tol * bnorm:
            x = x + alpha * p_hat
            return x, i, snorm / bnorm, KRYLOV_CONVERGED
        s_hat = apply_m(s)
        t = apply_a(s_hat)
        tt = _dot(t, t)
        if tt == 0.0 or not np.isfinite(tt):
            return x + alpha * p_hat, i, snorm / bnorm, KRYLOV_BREAKDOWN
        omega = _dot(t, s) / tt
        x = x + alpha * p_hat + omega * s_hat
        r = s - omega * t
        relres = np.sqrt(_dot(r, r)) / bnorm
        if relres <= tol:
            return x, i, relres, KRYLOV_CONVERGED
        if omega == 0.0 or not np.isfinite(omega):
            return x, i, relres, KRYLOV_BREAKDOWN
        rho_prev = rho
    return x, max_iter, relres, KRYLOV_MAX_ITER


def project_krylov(u, v, w, dx, dy, dz, rho_c, rho_f, tol, max_iter, precond="line"):
    """The projection with the Poisson problem solved by BiCGStab.

    Returns (u_out, v_out, w_out, phi, iterations, relative residual, status);
    phi carries the pin of the FFT solver (level-0 horizontal mean zero)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    w = np.array(w, np.float64)
    nz = u.shape[0]
    b = divergence(u, v, w, dx, dy, dz, rho_c, rho_f)

    def apply_a(x):
        return laplacian(x, dx, dy, dz, rho_c, rho_f)

    if precond == "line":
        def apply_m(r):
            return line_solve(r, dx, dy, dz, rho_c, rho_f)
    elif precond == "none":
        def apply_m(r):
            return r.copy()
    else:
        raise ValueError(precond)
    phi, iters, relres, status = bicgstab(b, apply_a, apply_m, tol, max_iter)
    phi = phi - np.mean(phi[0])
    gx, gy, gz = gradient(phi, dx, dy, dz)
    w_in = w.copy()
    w_in[0] = 0.0
    w_in[nz] = 0.0
    return u - gx, v - gy, w_in - gz, phi, iters, relres, status
