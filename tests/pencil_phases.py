"""The phases of the distributed projection restated on the CPU from the
oracle's steps (test infrastructure): the same interface as the product's
GpuPhases, FP64, on CPU torch tensors.

Each phase follows the contract of its C entry point (paper, Section 4:
forward transform, a vertical problem per wavenumber, backward transform):
  forward_slab     D^ = DFT2(rho_c dz D) of levels [k0, k1)   (a1-a2)
  vertical_pencil  p^ / (nx ny) and gz^ = (p^_k - p^_{k-1}) / dzn_k / (nx ny)
                   of spectral rows [j0, j1)                    (a3)
  inverse_slab     u - G_x phi, v - G_y phi, w - IDFT2(gz^)     (a4-a5)
and pack / unpack are the row reordering written out from its definition
(rows of part s at [s q + min(s, r), ...) of ny = q parts + r).
"""
import numpy as np
import torch

import oracle as O


def part_rows(n, parts):
    """Brute-force split: part s gets q + 1 items for s < r, else q, in order."""
    q, r = n // parts, n % parts
    bounds, lo = [], 0
    for s in range(parts):
        hi = lo + q + (1 if s < r else 0)
        bounds.append((lo, hi))
        lo = hi
    return bounds


def to_complex(t, nxh):
    a = t.numpy()
    return a[..., :nxh, 0] + 1j * a[..., :nxh, 1]


def put_complex(t, z):
    t.zero_()
    nxh = z.shape[-1]
    t[..., :nxh, 0] = torch.from_numpy(np.ascontiguousarray(z.real))
    t[..., :nxh, 1] = torch.from_numpy(np.ascontiguousarray(z.imag))


class OraclePhases:
    def __init__(self, nx, ny, nz, dx, dy, dz, rho_c, rho_f, nxp=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dy = dx, dy
        self.dz = np.asarray(dz, np.float64)
        self.rho_c = np.asarray(rho_c, np.float64)
        self.rho_f = np.asarray(rho_f, np.float64)
        self.nxh = nx // 2 + 1
        self.nxp = nxp if nxp is not None else (self.nxh + 3) // 4 * 4
        self.dtype = torch.float64
        self.device = torch.device("cpu")
        self.dzn = O.grid_metrics(self.dz)[2]

    def forward_slab(self, k0, k1, u, v, w, dhat):
        zero = np.zeros((self.ny, self.nx))
        d = np.empty((k1 - k0, self.ny, self.nx))
        for k in range(k1 - k0):
            kg = k0 + k
            below = zero if kg == 0 else w[k].numpy()
            above = zero if kg == self.nz - 1 else w[k + 1].numpy()
            d[k] = O.divergence_level(u[k].numpy(), v[k].numpy(), below, above, self.dx, self.dy, self.dz[kg],
                                      self.rho_c[kg], self.rho_f[kg], self.rho_f[kg + 1])
            d[k] *= self.rho_c[kg] * self.dz[kg]
        put_complex(dhat, O.forward_dft2(d))

    def vertical_pencil(self, j0, j1, spec, gz):
        nz, nyl, nxh = self.nz, j1 - j0, self.nxh
        vol = self.rho_c * self.dz
        rhs = to_complex(spec, nxh) / vol[:, None, None]
        ky, kx = np.meshgrid(np.arange(j0, j1), np.arange(nxh), indexing="ij")
        ph = O.solve_spectral(rhs.reshape(nz, nyl * nxh), self.nx, self.ny, self.dx, self.dy, self.dz,
                              self.rho_c, self.rho_f, kx=kx.ravel(), ky=ky.ravel()).reshape(nz, nyl, nxh)
        ph = ph / (self.nx * self.ny)
        g = np.zeros_like(ph)
        for k in range(1, nz):
            g[k] = (ph[k] - ph[k - 1]) / self.dzn[k]
        put_complex(spec, ph)
        put_complex(gz, g)

    def inverse_slab(self, k0, k1, phat, gz, u, v, w, u_out, v_out, w_out):
        n = self.nx * self.ny
        phi = O.inverse_dft2(to_complex(phat, self.nxh), self.nx) * n
        gx, gy, _ = O.gradient(phi, self.dx, self.dy, self.dz[k0:k1])
        gzr = O.inverse_dft2(to_complex(gz, self.nxh), self.nx) * n
        wo = w.numpy()[:k1 - k0] - gzr
        if k0 == 0:
            wo[0] = 0.0
        u_out.copy_(torch.from_numpy(u.numpy() - gx))
        v_out.copy_(torch.from_numpy(v.numpy() - gy))
        w_out[:k1 - k0] = torch.from_numpy(wo)
        if k1 == self.nz:
            w_out[k1 - k0] = 0.0

    def pack(self, nzl, parts, slab, packed):
        off = 0
        for j0, j1 in part_rows(self.ny, parts):
            for k in range(nzl):
                for j in range(j0, j1):
                    m = slab[k, j].numel()
                    packed[off:off + m] = slab[k, j].reshape(-1)
                    off += m

    def unpack(self, nzl, parts, packed, slab):
        off = 0
        for j0, j1 in part_rows(self.ny, parts):
            for k in range(nzl):
                for j in range(j0, j1):
                    m = slab[k, j].numel()
                    slab[k, j] = packed[off:off + m].reshape(slab[k, j].shape)
                    off += m
