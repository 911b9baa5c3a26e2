"""Pins of the oracle's one-FFT propagator (Eq. intens, Eq. Gxy) and its passband co-addition.

  * off critical sampling: a brute-force discrete Fresnel sum (Eq. hxy) evaluated at the
    output points x_0 = (k - N/2) lambda z / (N Delta_1), written out here term by term;
  * at critical sampling N Delta^2 = lambda z: the transfer-function pattern, index for index
    (the chirp kernel exp(i pi m^2 / N) is N-periodic for even N, so the plain Fresnel sum is
    the circular one), itself pinned in test_oracle_propagation.py;
  * a uniform untapered screen at critical sampling gives exactly 1 (|Gauss sum|^2 = N);
  * energy: sum h Delta_0^2 = sum |A_in|^2 Delta_1^2 (Parseval);
  * the resampling onto the reference grid: the identity for the reference wavelength and the
    scaled coordinates about the optical axis for the others.
"""
import math

import numpy as np
import pytest

import oracle as O


def _critical(n, lam=500.0, z=160.0, **kw):
    lz = lam * O.KM_PER_NM * z * O.KM_PER_PC
    pix = math.sqrt(lz / n)
    return O.ScreenParams(n=n, pixel_km=pix, lambda_nm=lam, lambda_ref_nm=lam, z_pc=z, **kw)


def test_brute_force_fresnel_sum_off_critical():
    p = O.ScreenParams(n=16, pixel_km=700.0, r_diff_km=900.0, lambda_nm=620.0, lambda_ref_nm=550.0,
                       z_pc=160.0, seed=31, margin_km=2000.0)
    phi = O.make_screen(p)
    lam = 620.0
    lz = lam * O.KM_PER_NM * p.z_pc * O.KM_PER_PC
    a_in = O.screen_field(phi, p, lam)
    x1 = (np.arange(p.n) - p.n // 2) * p.pixel_km
    d0 = lz / (p.n * p.pixel_km)
    x0 = (np.arange(p.n) - p.n // 2) * d0
    want = np.zeros((p.n, p.n))
    for ky in range(p.n):
        for kx in range(p.n):
            acc = 0j
            for iy in range(p.n):
                for ix in range(p.n):
                    r2 = (x0[kx] - x1[ix]) ** 2 + (x0[ky] - x1[iy]) ** 2
                    acc += a_in[iy, ix] * np.exp(1j * math.pi * r2 / lz)
            want[ky, kx] = abs(acc * p.pixel_km ** 2 / lz) ** 2
    np.testing.assert_allclose(O.propagate_conjugate(phi, p, lam), want, rtol=1e-10, atol=1e-12)
    assert O.observer_pixel_km(p, lam) == pytest.approx(d0, rel=1e-15)


@pytest.mark.parametrize("n", [32, 64])
def test_critical_sampling_equals_transfer_function(n):
    p = _critical(n, r_diff_km=0.0, seed=8)
    p = p.with_(r_diff_km=3.0 * p.pixel_km)
    phi = O.make_screen(p)
    np.testing.assert_allclose(O.propagate_conjugate(phi, p), O.intensity_mono(phi, p), rtol=1e-9, atol=1e-12)
    assert O.observer_pixel_km(p, p.lambda_nm) == pytest.approx(p.pixel_km, rel=1e-14)


def test_uniform_screen_at_critical_sampling_is_flat():
    p = _critical(64, r_diff_km=100.0, margin_km=0.0)
    h = O.propagate_conjugate(np.zeros((64, 64)), p)
    np.testing.assert_allclose(h, 1.0, atol=1e-12)


def test_energy_is_conserved():
    p = O.ScreenParams(n=64, pixel_km=40.0, r_diff_km=90.0, lambda_nm=800.0, lambda_ref_nm=550.0, seed=4)
    phi = O.make_screen(p)
    h = O.propagate_conjugate(phi, p)
    a_in = O.screen_field(phi, p, 800.0)
    d0 = O.observer_pixel_km(p, 800.0)
    assert np.sum(h) * d0 ** 2 == pytest.approx(np.sum(np.abs(a_in) ** 2) * p.pixel_km ** 2, rel=1e-12)


def test_passband_resampling():
    p = O.ScreenParams(n=32, pixel_km=60.0, r_diff_km=120.0, lambda_nm=550.0, lambda_ref_nm=550.0, seed=12)
    phi = O.make_screen(p)
    # the grid wavelength alone: the pattern itself
    np.testing.assert_allclose(O.sum_passband_conjugate(phi, p, [550.0]), O.propagate_conjugate(phi, p), rtol=1e-14)
    # another wavelength: output pixel k samples the pattern at (k - N/2) lambda_grid/lambda + N/2
    lam = 700.0
    h = O.propagate_conjugate(phi, p, lam)
    out = O.sum_passband_conjugate(phi, p, [lam])
    r = 550.0 / lam
    for ky, kx in [(16, 16), (3, 29), (30, 1), (17, 8)]:
        u = (kx - 16) * r + 16
        v = (ky - 16) * r + 16
        x0, y0 = int(math.floor(u)), int(math.floor(v))
        tx, ty = u - x0, v - y0
        g = lambda yy, xx: h[yy % 32, xx % 32]
        want = ((1 - tx) * (1 - ty) * g(y0, x0) + tx * (1 - ty) * g(y0, x0 + 1)
                + (1 - tx) * ty * g(y0 + 1, x0) + tx * ty * g(y0 + 1, x0 + 1))
        assert out[ky, kx] == pytest.approx(want, rel=1e-13)
    # the optical axis is a pixel centre of every grid
    assert out[16, 16] == pytest.approx(h[16, 16], rel=1e-14)
    # weights
    two = O.sum_passband_conjugate(phi, p, [550.0, lam], weights=[0.25, 0.75])
    np.testing.assert_allclose(two, 0.25 * O.propagate_conjugate(phi, p) + 0.75 * out, rtol=1e-13)
