"""FP64 CPU oracle of the anelastic pressure projection.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
it is used by ``tests/``, by ``__graft_entry__.smoke()`` (to check one small
GPU solve) and by ``bench.py``'s CPU-baseline leg.  It shares no code,
constants or tables with the CUDA path.

What it computes (paper, Section 4: pressure terms are handled by a forward
FFT, a vertical ODE solved in Fourier space for each horizontal wavenumber,
and a backward FFT).  The paper states no stencil, staggering or boundary
treatment; the readings used here are:

* Arakawa-C staggering: u[k,j,i] on the east face of cell (i,j,k), v on the
  north face, w[k,j,i] on the horizontal face at height zf[k] (k = 0..nz, so
  w has nz+1 levels); the pressure-like potential phi at cell centres.
  Periodic in x and y.  Face heights zf[0]=0, zf[k+1]=zf[k]+dz[k]; centres
  zc[k]; centre-to-centre spacing dzn[k] = (dz[k-1]+dz[k])/2 for faces
  k = 1..nz-1.
* Divergence (step a1):  D = (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy
  + (rho_f[k+1] w[k+1] - rho_f[k] w[k]) / (rho_c[k] dz[k]), with the bottom
  and top faces taken as w = 0 whatever the input holds there.
* Gradient (step a5): (phi_{i+1}-phi_i)/dx on u faces, (phi_{j+1}-phi_j)/dy
  on v faces, (phi_k - phi_{k-1})/dzn[k] on interior w faces, zero on the
  bottom and top faces (Neumann).
* The Poisson problem L phi = D(u*) with L = D o G; the projected velocity is
  u = u* - G phi.
* The horizontal mean mode (kx,ky) = (0,0) is singular; it is pinned by
  phi_hat(0,0)[k=0] = 0 and the (redundant, by compatibility) first equation
  of that column is dropped.
* Forward DFT unnormalised, inverse scaled by 1/(nx ny).

Every step is written in the plain form of its definition: the horizontal
transforms are naive O(n^2) DFTs (a dense DFT matrix built from a cos/sin
table of 2 pi m / n, applied with a matrix product), the vertical problem is
the textbook Thomas algorithm, one column at a time in the sense of the
recurrence (vectorised over columns only for speed).  No blocking, fusion or
reordering.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_metrics", "divergence_level", "divergence", "gradient", "twiddle_table", "dft_matrix",
    "forward_dft2", "inverse_dft2", "modified_wavenumbers", "vertical_operator",
    "thomas", "solve_spectral", "project", "mode_dft", "project_modes",
    "divergence_residual",
]


# --------------------------------------------------------------------------
# Grid metrics
# --------------------------------------------------------------------------

def grid_metrics(dz):
    """Face heights zf (nz+1), centre heights zc (nz), centre spacing dzn (nz+1).

    dzn[k] for k = 1..nz-1 is the distance between the centres of cells k-1
    and k; dzn[0] and dzn[nz] are unused (set to nan)."""
    dz = np.asarray(dz, dtype=np.float64)
    nz = dz.shape[0]
    zf = np.zeros(nz + 1)
    for k in range(nz):
        zf[k + 1] = zf[k] + dz[k]
    zc = 0.5 * (zf[:-1] + zf[1:])
    dzn = np.full(nz + 1, np.nan)
    for k in range(1, nz):
        dzn[k] = zc[k] - zc[k - 1]
    return zf, zc, dzn


# --------------------------------------------------------------------------
# Step a1: divergence, step a5: gradient
# --------------------------------------------------------------------------

def divergence_level(u_k, v_k, w_below, w_above, dx, dy, dz_k, rho_c_k, rho_f_below, rho_f_above):
    """Step a1 at one level k: the cell-centre divergence (ny, nx).

    (u_i - u_{i-1})/dx + (v_j - v_{j-1})/dy
      + (rho_f[k+1] w[k+1] - rho_f[k] w[k]) / (rho_c[k] dz[k])."""
    d = (u_k - np.roll(u_k, 1, axis=1)) / dx
    d = d + (v_k - np.roll(v_k, 1, axis=0)) / dy
    d = d + (rho_f_above * w_above - rho_f_below * w_below) / (rho_c_k * dz_k)
    return d


def divergence(u, v, w, dx, dy, dz, rho_c, rho_f):
    """(1/rho_c) div(rho0 u) at cell centres, shape (nz, ny, nx).

    The bottom and top faces count as w = 0 whatever the input holds there."""
    nz, ny, nx = np.shape(u)
    zero = np.zeros((ny, nx))
    d = np.empty((nz, ny, nx))
    for k in range(nz):
        w_below = zero if k == 0 else np.asarray(w[k], np.float64)
        w_above = zero if k == nz - 1 else np.asarray(w[k + 1], np.float64)
        d[k] = divergence_level(np.asarray(u[k], np.float64), np.asarray(v[k], np.float64),
                                w_below, w_above, dx, dy, float(dz[k]), float(rho_c[k]),
                                float(rho_f[k]), float(rho_f[k + 1]))
    return d


def gradient(phi, dx, dy, dz):
    """G phi: (gx on u faces, gy on v faces, gz on w faces with gz[0]=gz[nz]=0)."""
    phi = np.asarray(phi, np.float64)
    nz = phi.shape[0]
    _, _, dzn = grid_metrics(dz)
    gx = (np.roll(phi, -1, axis=2) - phi) / dx
    gy = (np.roll(phi, -1, axis=1) - phi) / dy
    gz = np.zeros((nz + 1,) + phi.shape[1:])
    for k in range(1, nz):
        gz[k] = (phi[k] - phi[k - 1]) / dzn[k]
    return gx, gy, gz


# --------------------------------------------------------------------------
# Step a2 / a4: naive DFTs
# --------------------------------------------------------------------------

def twiddle_table(n):
    """cos and sin of 2 pi m / n for m = 0..n-1 (FP64, libm)."""
    m = np.arange(n, dtype=np.float64)
    ang = 2.0 * np.pi * m / n
    return np.cos(ang), np.sin(ang)


def dft_matrix(n, nout=None, sign=-1):
    """F[a, b] = exp(sign * 2 pi i a b / n) for a < n (input), b < nout (output)."""
    nout = n if nout is None else nout
    c, s = twiddle_table(n)
    idx = (np.arange(n)[:, None] * np.arange(nout)[None, :]) % n
    return c[idx] + 1j * sign * s[idx]


def forward_dft2(field):
    """Real field (nz, ny, nx) -> half spectrum (nz, ny, nx//2+1).

    X[k, ky, kx] = sum_j sum_i field[k, j, i] exp(-2 pi i (kx i/nx + ky j/ny)).
    Along x first (real input, the nx//2+1 non-negative kx), then along y."""
    nz, ny, nx = field.shape
    fx = dft_matrix(nx, nx // 2 + 1, -1)          # (nx, nxh)
    fy = dft_matrix(ny, ny, -1)                   # (ny, ny) symmetric
    out = np.empty((nz, ny, nx // 2 + 1), np.complex128)
    for k in range(nz):
        t = field[k] @ fx                         # (ny, nxh): transform along x
        out[k] = fy.T @ t                         # along y
    return out


def inverse_dft2(spec, nx):
    """Half spectrum (nz, ny, nx//2+1) -> real field (nz, ny, nx), scaled 1/(nx ny).

    The missing negative kx are restored by Hermitian symmetry
    X[ky, nx-kx] = conj(X[(ny-ky) % ny, kx]); then a full complex inverse DFT
    is taken along y and along x and the real part is returned."""
    nz, ny, nxh = spec.shape
    gy = dft_matrix(ny, ny, +1)
    gx = dft_matrix(nx, nx, +1)
    out = np.empty((nz, ny, nx))
    ky_neg = (-np.arange(ny)) % ny
    for k in range(nz):
        full = np.empty((ny, nx), np.complex128)
        full[:, :nxh] = spec[k]
        for kx in range(nxh, nx):
            full[:, kx] = np.conj(spec[k][ky_neg, nx - kx])
        t = gy.T @ full                           # inverse along y
        t = t @ gx                                # inverse along x
        out[k] = t.real / (nx * ny)
    return out


# --------------------------------------------------------------------------
# Step a3: vertical problem per horizontal wavenumber
# --------------------------------------------------------------------------

def modified_wavenumbers(n, d):
    """Eigenvalue of the periodic 3-point second difference: 2(cos(2 pi k/n) - 1)/d^2."""
    c, _ = twiddle_table(n)
    return 2.0 * (c - 1.0) / (d * d)


def vertical_operator(dz, rho_c, rho_f):
    """Rows of the vertical part of L: (sub, diag0, sup) with

    (L_z phi)[k] = sub[k] phi[k-1] + diag0[k] phi[k] + sup[k] phi[k+1],
    A[k] = rho_f[k]/dzn[k] on interior faces, A[0] = A[nz] = 0 (Neumann), and
    row k divided by rho_c[k] dz[k]."""
    dz = np.asarray(dz, np.float64)
    rho_c = np.asarray(rho_c, np.float64)
    rho_f = np.asarray(rho_f, np.float64)
    nz = dz.shape[0]
    _, _, dzn = grid_metrics(dz)
    a = np.zeros(nz + 1)
    for k in range(1, nz):
        a[k] = rho_f[k] / dzn[k]
    vol = rho_c * dz
    sub = a[:nz] / vol
    sup = a[1:] / vol
    diag0 = -(a[:nz] + a[1:]) / vol
    return sub, diag0, sup


def thomas(sub, diag, sup, rhs):
    """Textbook Thomas algorithm for tridiagonal systems.

    Row k: sub[k] x[k-1] + diag[k] x[k] + sup[k] x[k+1] = rhs[k]; sub[0] and
    sup[n-1] are ignored.  Leading axis is the row index; trailing axes batch
    independent systems (each with its own coefficients)."""
    n = rhs.shape[0]
    cp = np.empty(diag.shape, np.float64)
    dp = np.empty(rhs.shape, rhs.dtype)
    cp[0] = sup[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for k in range(1, n):
        den = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / den if k < n - 1 else 0.0
        dp[k] = (rhs[k] - sub[k] * dp[k - 1]) / den
    x = np.empty(rhs.shape, rhs.dtype)
    x[n - 1] = dp[n - 1]
    for k in range(n - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def solve_spectral(dhat, nx, ny, dx, dy, dz, rho_c, rho_f, kx=None, ky=None):
    """Solve L_lambda phi_hat = dhat for every horizontal wavenumber column.

    dhat: (nz, m) complex, column c belonging to wavenumber (kx[c], ky[c]);
    by default all (ky, kx) of the half spectrum, flattened ky-major.
    The (0,0) column has its first row replaced by phi_hat[0] = 0."""
    nz = dhat.shape[0]
    if kx is None:
        kyy, kxx = np.meshgrid(np.arange(ny), np.arange(nx // 2 + 1), indexing="ij")
        kx, ky = kxx.ravel(), kyy.ravel()
    kx = np.asarray(kx)
    ky = np.asarray(ky)
    lam = modified_wavenumbers(nx, dx)[kx % nx] + modified_wavenumbers(ny, dy)[ky % ny]
    sub, diag0, sup = vertical_operator(dz, rho_c, rho_f)
    m = dhat.shape[1]
    sub2 = np.repeat(sub[:, None], m, axis=1)
    sup2 = np.repeat(sup[:, None], m, axis=1)
    diag2 = diag0[:, None] + lam[None, :]
    rhs = np.array(dhat, np.complex128)
    mean = (kx % nx == 0) & (ky % ny == 0)
    if np.any(mean):
        diag2[0, mean] = 1.0
        sup2[0, mean] = 0.0
        rhs[0, mean] = 0.0
    return thomas(sub2, diag2, sup2, rhs)


# --------------------------------------------------------------------------
# The whole projection
# --------------------------------------------------------------------------

def project(u, v, w, dx, dy, dz, rho_c, rho_f):
    """Return (u_out, v_out, w_out, phi), all FP64.

    a1 divergence -> a2 forward DFT per level -> a3 Thomas per column ->
    a4 inverse DFT per level -> a5 u = u* - G phi."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    w = np.array(w, np.float64)
    nz, ny, nx = u.shape
    d = divergence(u, v, w, dx, dy, dz, rho_c, rho_f)
    dhat = forward_dft2(d)
    nxh = nx // 2 + 1
    phat = solve_spectral(dhat.reshape(nz, ny * nxh), nx, ny, dx, dy, dz, rho_c, rho_f)
    phi = inverse_dft2(phat.reshape(nz, ny, nxh), nx)
    gx, gy, gz = gradient(phi, dx, dy, dz)
    w_in = w.copy()
    w_in[0] = 0.0
    w_in[nz] = 0.0
    return u - gx, v - gy, w_in - gz, phi


def divergence_residual(u_out, v_out, w_out, u_in, v_in, w_in, dx, dy, dz, rho_c, rho_f):
    """||D(u_out)||_2 / ||D(u_in)||_2 over all cells, in FP64."""
    d_out = divergence(u_out, v_out, w_out, dx, dy, dz, rho_c, rho_f)
    d_in = divergence(u_in, v_in, w_in, dx, dy, dz, rho_c, rho_f)
    return float(np.linalg.norm(d_out) / np.linalg.norm(d_in))


# --------------------------------------------------------------------------
# Sampled modes at sizes where the full oracle is too slow
# --------------------------------------------------------------------------

def mode_dft(field, kx, ky, x_shift=0.0, y_shift=0.0):
    """Direct DFT of a (nlev, ny, nx) real field at the listed (kx, ky) pairs.

    Returns (nlev, m) complex: sum_j sum_i f[., j, i] exp(-2 pi i (kx i/nx + ky j/ny)).
    Computed level by level in FP64 straight from the sum's definition (as a
    matrix product with the m exponential vectors)."""
    nlev, ny, nx = field.shape
    kx = np.asarray(kx)
    ky = np.asarray(ky)
    cx, sx = twiddle_table(nx)
    cy, sy = twiddle_table(ny)
    ex = cx[(np.arange(nx)[:, None] * kx[None, :]) % nx] - 1j * sx[(np.arange(nx)[:, None] * kx[None, :]) % nx]
    ey = cy[(np.arange(ny)[:, None] * ky[None, :]) % ny] - 1j * sy[(np.arange(ny)[:, None] * ky[None, :]) % ny]
    out = np.empty((nlev, kx.shape[0]), np.complex128)
    for k in range(nlev):
        t = np.asarray(field[k], np.float64) @ ex       # (ny, m)
        out[k] = np.sum(t * ey, axis=0)
    return out


def project_modes(u, v, w, dx, dy, dz, rho_c, rho_f, kx, ky):
    """Spectral coefficients of the projected velocities at the listed modes.

    The projection decouples by horizontal wavenumber, so the output at mode
    (kx, ky) needs only the input at that mode.  Returns a dict with the
    expected DFTs of u_out (nz, m), v_out (nz, m), w_out (nz+1, m) and of the
    divergence of the input (nz, m).  Used to check one output at a time on
    domains where the full oracle would take too long."""
    nz, ny, nx = np.asarray(u).shape
    kx = np.asarray(kx)
    ky = np.asarray(ky)
    d = divergence(u, v, w, dx, dy, dz, rho_c, rho_f)
    dhat = mode_dft(d, kx, ky)
    phat = solve_spectral(dhat, nx, ny, dx, dy, dz, rho_c, rho_f, kx=kx, ky=ky)
    _, _, dzn = grid_metrics(dz)
    cx, sx = twiddle_table(nx)
    cy, sy = twiddle_table(ny)
    # spectral symbols of the forward differences (phi_{i+1} - phi_i)/dx etc.
    sym_x = ((cx[kx % nx] + 1j * sx[kx % nx]) - 1.0) / dx
    sym_y = ((cy[ky % ny] + 1j * sy[ky % ny]) - 1.0) / dy
    u_hat = mode_dft(u, kx, ky) - phat * sym_x[None, :]
    v_hat = mode_dft(v, kx, ky) - phat * sym_y[None, :]
    w_in = mode_dft(w, kx, ky)
    w_hat = np.zeros((nz + 1, kx.shape[0]), np.complex128)
    for k in range(1, nz):
        w_hat[k] = w_in[k] - (phat[k] - phat[k - 1]) / dzn[k]
    return {"u": u_hat, "v": v_hat, "w": w_hat, "div": dhat, "phi": phat}
