"""Seeded synthetic inputs for the anelastic pressure projection.

This module only *generates* inputs: grid profiles (layer thicknesses and the
reference density at cell centres and faces) and provisional velocity fields
on the Arakawa-C grid.  It holds none of the projection's arithmetic, so both
the CUDA path and the FP64 CPU oracle can be fed from it without sharing any
of the method.

The paper (Section 4) runs the dry boundary layer case on a Cartesian grid of
64 levels with square horizontal domains; that case and its data are not
available, so the workloads below are synthetic fields with the same kind of
shape: square horizontal domains, tens to hundreds of levels, a stretched
vertical grid and an exponentially decaying reference density.

Recipe (every draw from ``numpy.random.default_rng(seed)``, FP64):
  * ``u``  shape (nz, ny, nx): standard normal, then ``v`` (nz, ny, nx), then
    ``w`` (nz+1, ny, nx); the boundary faces w[0] and w[nz] are set to zero.
  * Optionally a smooth large-scale mode of 1 m/s,
    ``sin(2 pi x/Lx) cos(2 pi y/Ly) sin(pi z/H)``, is added to each component
    at that component's own staggered position (u on east faces, v on north
    faces, w on horizontal faces; it vanishes at the bottom and top faces).
  * Reference density ``rho0(z) = 1.2 exp(-z / Hs)`` evaluated at the cell
    centres ``zc`` and at the faces ``zf``; ``Hs`` = 8000 m unless stated.
  * Layer thickness either uniform or geometric: ``dz[k] = a r^k`` with
    ``r = (b/a)^(1/(nz-1))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: np.ndarray      # (nz,)   layer thickness [m]
    rho_c: np.ndarray   # (nz,)   reference density at cell centres
    rho_f: np.ndarray   # (nz+1,) reference density at w faces

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def uniform_dz(nz: int, dz: float) -> np.ndarray:
    return np.full(nz, float(dz))


def geometric_dz(nz: int, dz_bottom: float, dz_top: float) -> np.ndarray:
    """Layer thicknesses growing geometrically from dz_bottom to dz_top."""
    if nz == 1:
        return np.array([float(dz_bottom)])
    r = (dz_top / dz_bottom) ** (1.0 / (nz - 1))
    return dz_bottom * r ** np.arange(nz, dtype=np.float64)


def face_heights(dz: np.ndarray) -> np.ndarray:
    """Heights of the nz+1 horizontal faces, zf[0] = 0."""
    return np.concatenate([[0.0], np.cumsum(dz)])


def make_grid(nx, ny, nz, dx, dy, dz, scale_height=8000.0, rho_surface=1.2) -> Grid:
    dz = np.asarray(dz, dtype=np.float64)
    zf = face_heights(dz)
    zc = 0.5 * (zf[:-1] + zf[1:])
    rho_c = rho_surface * np.exp(-zc / scale_height)
    rho_f = rho_surface * np.exp(-zf / scale_height)
    return Grid(nx, ny, nz, float(dx), float(dy), dz, rho_c, rho_f)


def random_fields(grid: Grid, seed: int, large_scale_mode: bool = False):
    """Provisional velocities u, v, w (FP64) for the recipe in the module doc."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    u = rng.standard_normal((nz, ny, nx))
    v = rng.standard_normal((nz, ny, nx))
    w = rng.standard_normal((nz + 1, ny, nx))
    w[0] = 0.0
    w[nz] = 0.0
    if large_scale_mode:
        add_large_scale_mode(grid, u, v, w)
    return u, v, w


def random_fields_f32(grid: Grid, seed: int, large_scale_mode: bool = False):
    """The same fields as ``random_fields(...)`` rounded to float32, drawn level
    by level so that FP64 copies of whole fields are never held at once."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    out = (np.empty((nz, ny, nx), np.float32), np.empty((nz, ny, nx), np.float32),
           np.empty((nz + 1, ny, nx), np.float32))
    modes = _mode_factors(grid) if large_scale_mode else None
    for f, arr in enumerate(out):
        for k in range(arr.shape[0]):
            lev = rng.standard_normal((ny, nx))
            if modes is not None:
                lev += modes[f](k)
            if f == 2 and (k == 0 or k == nz):
                lev[:] = 0.0
            arr[k] = lev
    return out


def _mode_factors(grid: Grid, amplitude: float = 1.0):
    nx, ny = grid.nx, grid.ny
    lx, ly = nx * grid.dx, ny * grid.dy
    zf = face_heights(grid.dz)
    zc = 0.5 * (zf[:-1] + zf[1:])
    h = zf[-1]
    xc = (np.arange(nx) + 0.5) * grid.dx
    xe = (np.arange(nx) + 1.0) * grid.dx
    yc = (np.arange(ny) + 0.5) * grid.dy
    yn = (np.arange(ny) + 1.0) * grid.dy
    hu = np.cos(2 * np.pi * yc / ly)[:, None] * np.sin(2 * np.pi * xe / lx)[None, :]
    hv = np.cos(2 * np.pi * yn / ly)[:, None] * np.sin(2 * np.pi * xc / lx)[None, :]
    hw = np.cos(2 * np.pi * yc / ly)[:, None] * np.sin(2 * np.pi * xc / lx)[None, :]
    return (lambda k: amplitude * np.sin(np.pi * zc[k] / h) * hu,
            lambda k: amplitude * np.sin(np.pi * zc[k] / h) * hv,
            lambda k: amplitude * np.sin(np.pi * zf[k] / h) * hw)


def add_large_scale_mode(grid: Grid, u, v, w, amplitude: float = 1.0):
    nx, ny = grid.nx, grid.ny
    lx, ly = nx * grid.dx, ny * grid.dy
    zf = face_heights(grid.dz)
    zc = 0.5 * (zf[:-1] + zf[1:])
    h = zf[-1]
    xc = (np.arange(nx) + 0.5) * grid.dx      # cell centres in x
    xe = (np.arange(nx) + 1.0) * grid.dx      # east faces
    yc = (np.arange(ny) + 0.5) * grid.dy
    yn = (np.arange(ny) + 1.0) * grid.dy      # north faces

    def mode(x, y, z):
        return (amplitude * np.sin(np.pi * z / h)[:, None, None]
                * np.cos(2 * np.pi * y / ly)[None, :, None]
                * np.sin(2 * np.pi * x / lx)[None, None, :])

    u += mode(xe, yc, zc)
    v += mode(xc, yn, zc)
    w += mode(xc, yc, zf)
    w[0] = 0.0
    w[-1] = 0.0


# --------------------------------------------------------------------------
# The five workloads: shapes, spacings and seeds.
# --------------------------------------------------------------------------

def workload_64cube():
    """64x64x64, dx=dy=50 m, uniform dz=25 m, white-noise velocities, seed 0."""
    g = make_grid(64, 64, 64, 50.0, 50.0, uniform_dz(64, 25.0))
    return g, 0, False


def workload_256():
    """256x256x128, dx=dy=25 m, dz 10->100 m geometric, noise + mode, seed 1."""
    g = make_grid(256, 256, 128, 25.0, 25.0, geometric_dz(128, 10.0, 100.0))
    return g, 1, True


def workload_1024():
    """1024x1024x256, dx=dy=10 m, dz 5->50 m geometric, noise + mode, seed 2."""
    g = make_grid(1024, 1024, 256, 10.0, 10.0, geometric_dz(256, 5.0, 50.0))
    return g, 2, True


WORKLOADS = {
    "proj64_fp64": (workload_64cube, "fp64"),
    "proj256x128_fp64": (workload_256, "fp64"),
    "proj1024x256_mixed": (workload_1024, "mixed"),
}


def smooth_sizes(limit: int = 4096):
    """Sorted list of 2^a 3^b 5^c <= limit (the lengths the GPU transforms take)."""
    out = []
    a = 1
    while a <= limit:
        b = a
        while b <= limit:
            c = b
            while c <= limit:
                out.append(c)
                c *= 5
            b *= 3
        a *= 2
    return sorted(out)


def nearest_smooth(n: float, limit: int = 4096) -> int:
    s = smooth_sizes(limit)
    return min(s, key=lambda m: (abs(m - n), m))


def batch_instances(count: int = 64, seed: int = 3):
    """Uneven batch: nx=ny from {64,96,128,192,256}, nz from {64,96,128,160},
    dx=dy=25 m, dz uniform 25 m or geometric 10->100 m (coin flip), rho0 scale
    height uniform in [7000, 9000] m.  Returns (grid, field_seed) pairs."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([64, 96, 128, 192, 256]))
        nz = int(rng.choice([64, 96, 128, 160]))
        stretched = bool(rng.integers(0, 2))
        hs = float(rng.uniform(7000.0, 9000.0))
        dz = geometric_dz(nz, 10.0, 100.0) if stretched else uniform_dz(nz, 25.0)
        out.append((make_grid(n, n, nz, 25.0, 25.0, dz, scale_height=hs), 1000 * seed + i))
    return out


def serving_requests(count: int = 10000, rate: float = 2000.0, seed: int = 4,
                     n_min: int = 128, n_max: int = 512, nz_min: int = 64, nz_max: int = 192):
    """Poisson arrivals (rate per second) with log-uniform sizes.

    Horizontal size is drawn log-uniformly in [n_min, n_max] and rounded to the
    nearest 2^a 3^b 5^c; nz is drawn log-uniformly in [nz_min, nz_max] and
    rounded to the nearest integer.  Returns a list of dicts with the arrival
    time [s], nx=ny, nz and a field seed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    ln = rng.uniform(math.log(n_min), math.log(n_max), size=count)
    lz = rng.uniform(math.log(nz_min), math.log(nz_max), size=count)
    out = []
    for i in range(count):
        n = nearest_smooth(math.exp(ln[i]))
        nz = int(round(math.exp(lz[i])))
        out.append({"t": float(t[i]), "n": n, "nz": nz, "seed": 100000 * seed + i})
    return out


def serving_grid(n: int, nz: int) -> Grid:
    """Grid of a served request: dx=dy=25 m, dz geometric 10->100 m."""
    return make_grid(n, n, nz, 25.0, 25.0, geometric_dz(nz, 10.0, 100.0))
