"""Planted mistakes in the oracle must be caught by its pins.

Each case swaps one oracle function for a plausibly wrong variant (on the CPU,
inside this test only) and checks that at least one pin of
``test_oracle_pins`` then fails.  This is what makes the pins worth trusting.
"""
import numpy as np
import pytest

import oracle.projection as P
import tests.test_oracle_pins as pins


def _pins():
    return [
        lambda: pins.test_projection_against_dense_least_squares((6, 5, 4)),
        lambda: pins.test_manufactured_single_mode(),
        lambda: pins.test_divergence_free_part_is_preserved(),
        lambda: pins.test_divergence_second_order_against_analytic(),
        lambda: pins.test_gradient_second_order_against_analytic(),
        lambda: pins.test_gradient_is_negative_weighted_adjoint_of_divergence(),
        lambda: pins.test_dft_roundtrip_and_parseval((2, 6, 15)),
        lambda: pins.test_dft2_against_direct_double_sum(),
        lambda: pins.test_thomas_against_dense_solve(),
    ]


def _some_pin_fails():
    for pin in _pins():
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            return True
    return False


def _wrong_sign_wavenumber(n, d):
    c, _ = P.twiddle_table(n)
    return 2.0 * (1.0 - c) / (d * d)


def _unweighted_vertical(dz, rho_c, rho_f):
    return _orig["vertical_operator"](dz, np.ones_like(rho_c), np.ones_like(rho_f))


def _divergence_level_wrong_offset(u_k, v_k, w_below, w_above, dx, dy, dz_k, rc, rfb, rfa):
    d = (np.roll(u_k, -1, axis=1) - u_k) / dx
    d = d + (v_k - np.roll(v_k, 1, axis=0)) / dy
    return d + (rfa * w_above - rfb * w_below) / (rc * dz_k)


def _grid_metrics_dzn_is_dz(dz):
    zf, zc, dzn = _orig["grid_metrics"](dz)
    dzn = dzn.copy()
    dzn[1:-1] = np.asarray(dz)[1:]
    return zf, zc, dzn


def _inverse_without_negative_ky(spec, nx):
    nz, ny, nxh = spec.shape
    out = np.empty((nz, ny, nx))
    gy = P.dft_matrix(ny, ny, +1)
    gx = P.dft_matrix(nx, nx, +1)
    for k in range(nz):
        full = np.empty((ny, nx), np.complex128)
        full[:, :nxh] = spec[k]
        for kx in range(nxh, nx):
            full[:, kx] = np.conj(spec[k][:, nx - kx])      # forgot ky -> -ky
        out[k] = ((gy.T @ full) @ gx).real / (nx * ny)
    return out


def _thomas_drops_back_substitution(sub, diag, sup, rhs):
    n = rhs.shape[0]
    cp = np.empty(diag.shape)
    dp = np.empty(rhs.shape, rhs.dtype)
    cp[0] = sup[0] / diag[0]
    dp[0] = rhs[0] / diag[0]
    for k in range(1, n):
        den = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / den if k < n - 1 else 0.0
        dp[k] = (rhs[k] - sub[k] * dp[k - 1]) / den
    return dp


def _twiddle_transposed(n):
    c, s = _orig["twiddle_table"](n)
    return c, -s


_orig = {name: getattr(P, name) for name in
         ("vertical_operator", "grid_metrics", "twiddle_table")}

MUTATIONS = {
    "modified wavenumber sign": ("modified_wavenumbers", _wrong_sign_wavenumber),
    "rho0 weighting dropped": ("vertical_operator", _unweighted_vertical),
    "u difference one cell off": ("divergence_level", _divergence_level_wrong_offset),
    "dz used for centre spacing": ("grid_metrics", _grid_metrics_dzn_is_dz),
    "Hermitian fill without -ky": ("inverse_dft2", _inverse_without_negative_ky),
    "Thomas back-substitution dropped": ("thomas", _thomas_drops_back_substitution),
    "twiddle sign flipped": ("twiddle_table", _twiddle_transposed),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(P, attr, fn)
    assert _some_pin_fails(), f"no pin caught: {name}"


def test_unmutated_oracle_passes_every_pin():
    assert not _some_pin_fails()
