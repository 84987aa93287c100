"""Checks of GPU outputs against the FP64 oracle at sizes where the full oracle
is slow: the projection decouples by horizontal wavenumber, so the oracle
solves sampled modes (kx, ky) alone (``project_modes``) and the output's DFT
at those modes is compared with them; the divergence residual is taken over
every cell in FP64.  Test infrastructure only."""
import numpy as np

import oracle as O


def sampled_modes(g, extra=10, seed=7):
    """The mean-adjacent, Nyquist and a few random modes of a grid."""
    rng = np.random.default_rng(seed)
    nxh = g.nx // 2 + 1
    kx = np.concatenate([[0, 1, 0, 1, 2, nxh - 1], rng.integers(0, nxh, extra)])
    ky = np.concatenate([[0, 0, 1, g.ny - 1, 3, g.ny // 2], rng.integers(0, g.ny, extra)])
    return kx, ky


def sampled_mode_error(g, u, v, w, outs, kx, ky):
    """Relative L2 error of the outputs' DFTs at (kx, ky) against the oracle."""
    ref = O.project_modes(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f, kx, ky)
    num = den = 0.0
    for name, arr in zip(("u", "v", "w"), outs):
        got = O.mode_dft(arr, kx, ky)
        num += float(np.sum(np.abs(got - ref[name]) ** 2))
        den += float(np.sum(np.abs(ref[name]) ** 2))
    return (num / den) ** 0.5


def divergence_residual_levels(g, u, v, w, outs):
    """||D(out)|| / ||D(in)|| over all cells, one level at a time (FP64)."""
    dn = dd = 0.0
    zero = np.zeros((g.ny, g.nx))
    for k in range(g.nz):
        for fields, is_out in ((outs, True), ((u, v, w), False)):
            fu, fv, fw = fields
            lo = np.asarray(fw[k], np.float64) if k > 0 else zero
            hi = np.asarray(fw[k + 1], np.float64) if k < g.nz - 1 else zero
            d = O.divergence_level(np.asarray(fu[k], np.float64), np.asarray(fv[k], np.float64), lo, hi,
                                   g.dx, g.dy, g.dz[k], g.rho_c[k], g.rho_f[k], g.rho_f[k + 1])
            if is_out:
                dn += float(np.sum(d * d))
            else:
                dd += float(np.sum(d * d))
    return (dn / dd) ** 0.5
