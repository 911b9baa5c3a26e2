"""Pins of the oracle's source smoothing, light curves, modulation index and gradient (CPU only)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O


@pytest.mark.parametrize("q,R", [(0.0, 50.0), (0.003, 50.0), (0.011, 80.0), (0.04, 120.0)])
def test_disk_kernel_matches_quadrature(q, R):
    """K(q) is the Fourier transform of the unit-integral uniform disk (Eq. iprh):
    (1/pi R^2) int_{-R}^{R} 2 sqrt(R^2 - x^2) cos(2 pi q x) dx, by quadrature."""
    val = integrate.quad(lambda x: 2.0 * math.sqrt(R * R - x * x) * math.cos(2 * math.pi * q * x),
                         -R, R, limit=400)[0] / (math.pi * R * R)
    n, pix = 256, 1.0 / (256 * 0.0005)    # frequency grid containing q exactly
    k = O.fft_freqs(n, pix)
    j = int(round(q / (k[1] - k[0])))
    K = O.source_kernel(n, pix, R)
    assert K[0, j] == pytest.approx(val, abs=1e-10)
    assert K[j, 0] == pytest.approx(val, abs=1e-10)


def test_smoothing_eigenfunction_and_mean():
    n, pix, R = 128, 10.0, 90.0
    L = n * pix
    x = (np.arange(n) + 0.5) * pix
    for m in (1, 3, 7):
        I = np.tile(1.0 + 0.3 * np.cos(2 * np.pi * m * x / L), (n, 1))
        out = O.smooth_source(I, pix, R)
        u = 2 * np.pi * (m / L) * R
        Kq = integrate.quad(lambda t: 2.0 * math.sqrt(1 - t * t) * math.cos(u * t), -1, 1)[0] / math.pi
        np.testing.assert_allclose(out, np.tile(1.0 + 0.3 * Kq * np.cos(2 * np.pi * m * x / L), (n, 1)), atol=1e-12)
    rng = np.random.default_rng(5)
    I = rng.uniform(0, 3, (n, n))
    assert O.smooth_source(I, pix, R).mean() == pytest.approx(I.mean(), rel=1e-13)
    np.testing.assert_allclose(O.smooth_source(I, pix, 0.0), I, atol=1e-13)


def test_smoothing_commutes_with_passband_sum():
    p = O.ScreenParams(n=64, pixel_km=10.0, r_diff_km=15.0, seed=6, lambda_ref_nm=550.0)
    phi = O.make_screen(p)
    lams = [500.0, 600.0]
    a = O.smooth_source(O.sum_passband(phi, p, lams), p.pixel_km, 70.0)
    b = 0.5 * O.smooth_source(O.intensity_mono(phi, p, 500.0), p.pixel_km, 70.0) \
        + 0.5 * O.smooth_source(O.intensity_mono(phi, p, 600.0), p.pixel_km, 70.0)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_lightcurve_integer_positions_are_pixels():
    rng = np.random.default_rng(7)
    I = rng.uniform(0, 2, (32, 32))
    c = O.lightcurves(I, [(3.0, 5.0, 0.0, 1.0)], 40)[0]
    np.testing.assert_array_equal(c, I[5, (3 + np.arange(40)) % 32])


def test_lightcurve_bilinear_exact_on_bilinear_map():
    n = 32
    iy, ix = np.mgrid[0:n, 0:n].astype(float)
    a, b, cc, d = 0.3, 0.07, -0.05, 0.002
    I = a + b * ix + cc * iy + d * ix * iy
    tr = (2.3, 4.6, 0.61, 0.37)
    x, y = O.track_positions(tr, 50)
    assert x.max() < n - 1 and y.max() < n - 1        # interior: no wrap
    np.testing.assert_allclose(O.lightcurves(I, [tr], 50)[0], a + b * x + cc * y + d * x * y, atol=1e-13)


def test_lightcurve_periodic_wrap_and_adjoint():
    rng = np.random.default_rng(8)
    n = 16
    I = rng.uniform(0, 2, (n, n))
    x = rng.uniform(-40, 40, 200)
    y = rng.uniform(-40, 40, 200)
    np.testing.assert_allclose(O.bilinear_periodic(I, x, y), O.bilinear_periodic(I, x + n, y - 2 * n), atol=1e-12)
    g = rng.standard_normal(200)
    lhs = np.dot(O.bilinear_periodic(I, x, y), g)
    rhs = np.sum(I * O.bilinear_periodic_adjoint((n, n), x, y, g))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_modulation_index_closed_form():
    n = 256
    x = np.arange(n)
    A = 0.37
    I = np.tile(1.0 + A * np.cos(2 * np.pi * 5 * x / n), (n, 1))
    assert O.modulation_index(I) == pytest.approx(A / math.sqrt(2.0), rel=1e-12)


def test_fiducial_zone():
    # like the 4096^2 single screens, R_diff = 30 km: margin exceeds L/2 -> whole map, flagged
    p = O.ScreenParams(n=4096, pixel_km=10.0, r_diff_km=30.0)
    assert O.fiducial_slice(p) == (0, 4096, True)
    p = O.ScreenParams(n=4096, pixel_km=10.0, r_diff_km=300.0)
    i0, i1, flag = O.fiducial_slice(p)
    m = O.fiducial_margin_km(p)
    assert not flag and (i0 + 0.5) * 10.0 >= m and (i0 - 0.5) * 10.0 < m and i1 == 4096 - i0
    assert O.fiducial_slice(p.with_(margin_km=0.0)) == (0, 4096, False)


def _grad_case():
    p = O.ScreenParams(n=32, pixel_km=10.0, r_diff_km=20.0, seed=9, lambda_ref_nm=550.0,
                       source_radius_km=25.0)
    lams = [520.0, 580.0]
    tracks = [(1.5, 3.25, 0.4, 0.7), (20.0, 2.0, 2.2, 1.1)]
    ns = 30
    _, _, target = O.forward(p.with_(seed=509), lams, tracks, ns)
    return p, lams, tracks, ns, target


def test_gradient_matches_central_differences():
    p, lams, tracks, ns, target = _grad_case()
    phi = O.make_screen(p)
    loss, g, g_rd = O.misfit_gradient(p, phi, lams, tracks, ns, target)
    rng = np.random.default_rng(10)
    h = 1e-5
    for _ in range(12):
        iy, ix = rng.integers(0, p.n, 2)
        e = np.zeros_like(phi)
        e[iy, ix] = h
        lp = O.misfit_loss(O.forward(p, lams, tracks, ns, phi=phi + e)[2], target)
        lm = O.misfit_loss(O.forward(p, lams, tracks, ns, phi=phi - e)[2], target)
        fd = (lp - lm) / (2 * h)
        assert g[iy, ix] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max())
    # R_diff: phi is regenerated from the same seed (phi ~ R_diff^((2-beta)/2))
    d = 1e-5 * p.r_diff_km
    lp = O.misfit_loss(O.forward(p.with_(r_diff_km=p.r_diff_km + d), lams, tracks, ns)[2], target)
    lm = O.misfit_loss(O.forward(p.with_(r_diff_km=p.r_diff_km - d), lams, tracks, ns)[2], target)
    assert g_rd == pytest.approx((lp - lm) / (2 * d), rel=1e-5)
    assert loss > 0
