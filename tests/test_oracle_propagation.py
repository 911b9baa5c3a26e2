"""Pins of the oracle's Fresnel propagation (CPU only).

Each check is fixed outside the oracle: a direct DFT, the direct Fresnel sum
of Eq. hxy, the Jacobi-Anger/Talbot closed forms of a phase grating,
energy conservation and the paper's uniform-screen check.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle as O


def test_fft_sign_and_scale_conventions():
    rng = np.random.default_rng(1)
    n = 8
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    j = np.arange(n)
    Wf = np.exp(-2j * np.pi * np.outer(j, j) / n)
    np.testing.assert_allclose(O.fft2(x), Wf @ x @ Wf.T, atol=1e-12)
    np.testing.assert_allclose(O.ifft2(x) * n * n, Wf.conj() @ x @ Wf.conj().T, atol=1e-12)
    # Parseval
    assert np.sum(np.abs(O.fft2(x)) ** 2) == pytest.approx(n * n * np.sum(np.abs(x) ** 2), rel=1e-13)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64])
@pytest.mark.parametrize("inverse", [False, True])
def test_own_radix2_fft_equals_the_direct_dft(n, inverse):
    rng = np.random.default_rng(n + 3)
    x = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    j = np.arange(n)
    W = np.exp((2j if inverse else -2j) * np.pi * np.outer(j, j) / n)
    np.testing.assert_allclose(O.fft_radix2(x, inverse), x @ W.T, atol=1e-12 * max(1, n))


@pytest.mark.parametrize("workers", [1, 4])
def test_library_fft_equals_the_own_radix2_fft(workers, monkeypatch):
    """The library primitive (one thread and several) against the oracle's own transform at
    sizes the direct DFT cannot reach."""
    monkeypatch.setattr(O, "FFT_WORKERS", workers)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((4096, 4)) + 1j * rng.standard_normal((4096, 4))
    ref = np.swapaxes(O.fft_radix2(np.swapaxes(x, 0, 1)), 0, 1)
    lib = O.fft2(x)[:, :1]                      # along y (4096 points), then 4 columns summed
    assert np.abs(lib[:, 0] - ref.sum(axis=1)).max() <= 1e-11 * np.abs(ref).max()
    x2 = rng.standard_normal((128, 128)) + 1j * rng.standard_normal((128, 128))
    np.testing.assert_allclose(O.fft2(x2), O.fft2_radix2(x2), atol=1e-10)
    np.testing.assert_allclose(O.ifft2(x2) * 128 * 128, O.fft2_radix2(x2, inverse=True), atol=1e-10)
    x3 = rng.standard_normal((3, 256, 512)) + 1j * rng.standard_normal((3, 256, 512))
    np.testing.assert_allclose(O.fft2(x3), O.fft2_radix2(x3), atol=1e-9)


def test_propagation_through_the_own_fft():
    """propagate_field (the library FFT) equals IDFT(DFT(A_in) H) / N^2 with the own radix-2 FFT."""
    p = O.ScreenParams(n=64, pixel_km=10.0, r_diff_km=20.0, seed=3)
    a_in = O.screen_field(O.make_screen(p), p, 520.0)
    H = O.transfer_function(64, 10.0, 520.0, p.z_pc)
    own = O.fft2_radix2(O.fft2_radix2(a_in) * H, inverse=True) / (64 * 64)
    np.testing.assert_allclose(O.propagate_field(a_in, 10.0, 520.0, p.z_pc), own, atol=1e-12)


def test_uniform_untapered_screen_is_exactly_one():
    p = O.ScreenParams(n=64, pixel_km=20.0, r_diff_km=100.0, margin_km=0.0)
    I = O.intensity_mono(np.zeros((64, 64)), p)
    np.testing.assert_allclose(I, 1.0, atol=1e-12)


def test_uniform_tapered_screen_flat_in_fiducial_zone():
    """Sect. 3.2.1: a point source through a uniform screen with the L_m = 10 R_F taper is flat to <1%."""
    n, pix, z = 1024, 20.0, 50.0
    p = O.ScreenParams(n=n, pixel_km=pix, r_diff_km=100.0, z_pc=z)
    lm = O.taper_margin_km(p, 500.0)
    rf = O.fresnel_radius_km(500.0, z)
    assert lm == pytest.approx(10.0 * rf)          # the paper's margin, not clamped here
    I = O.intensity_mono(np.zeros((n, n)), p)
    x = (np.arange(n) + 0.5) * pix
    # along a profile through the centre: flat to <1% everywhere past the taper
    flat = (x >= lm) & (x <= n * pix - lm)
    assert np.abs(I[n // 2, flat] - 1.0).max() < 0.01
    # in 2D the x and y edge ripples multiply near the corners; 2 R_F further in it is <1% again
    zone = (x >= lm + 2 * rf) & (x <= n * pix - lm - 2 * rf)
    assert np.abs(I[np.ix_(zone, zone)] - 1.0).max() < 0.01
    # and the ripple is a real effect of the finite taper, not noise: it decays inward
    deep = (x >= lm + 6 * rf) & (x <= n * pix - lm - 6 * rf)
    assert np.abs(I[np.ix_(deep, deep)] - 1.0).max() < 0.1 * np.abs(I[np.ix_(flat, flat)] - 1.0).max()
    # energy: the mean intensity is the mean transmitted power <SF^2>^2
    sf = O.taper_1d(n, pix, lm)
    assert I.mean() == pytest.approx(np.mean(sf ** 2) ** 2, rel=1e-12)


def test_propagation_conserves_energy_random_screen():
    p = O.ScreenParams(n=128, pixel_km=10.0, r_diff_km=20.0, seed=11)
    phi = O.make_screen(p)
    a_in = O.screen_field(phi, p, 500.0)
    a_out = O.propagate_field(a_in, p.pixel_km, 500.0, p.z_pc)
    assert np.sum(np.abs(a_out) ** 2) == pytest.approx(np.sum(np.abs(a_in) ** 2), rel=1e-12)


def test_transfer_function_equals_direct_fresnel_sum_at_critical_sampling():
    """With N Delta^2 = lambda z the FFT propagator equals the direct Fresnel-Huygens sum (Eq. hxy)."""
    n, lam, z = 32, 500.0, 160.0
    lz = lam * O.KM_PER_NM * z * O.KM_PER_PC
    pix = math.sqrt(lz / n)
    rng = np.random.default_rng(2)
    a_in = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    tf = O.propagate_field(a_in, pix, lam, z)
    direct = O.fresnel_direct(a_in, pix, lam, z)
    np.testing.assert_allclose(tf, direct, atol=1e-11 * np.abs(direct).max())


def test_transfer_function_is_circular_convolution_off_critical():
    n, pix, lam, z = 16, 15.0, 620.0, 90.0
    rng = np.random.default_rng(3)
    a_in = np.exp(1j * rng.uniform(0, 6.3, (n, n)))
    h = np.fft.ifft2(O.transfer_function(n, pix, lam, z))
    direct = np.zeros((n, n), complex)
    for oy in range(n):
        for ox in range(n):
            direct[oy, ox] = np.sum(h[(oy - np.arange(n))[:, None] % n, (ox - np.arange(n))[None, :] % n] * a_in)
    np.testing.assert_allclose(O.propagate_field(a_in, pix, lam, z), direct, atol=1e-12)


@pytest.mark.parametrize("lam,lam_ref", [(500.0, 500.0), (500.0, 550.0), (700.0, 550.0)])
def test_sinusoidal_phase_grating_closed_form(lam, lam_ref):
    """phi = a sin(2 pi x / p): A_out = sum_n J_n(a s) e^{2 pi i n x/p} e^{-i pi lambda z n^2/p^2} (Jacobi-Anger)."""
    n, pix, z, a = 64, 20.0, 160.0, 1.3
    L = n * pix
    per = L / 4.0
    x = (np.arange(n) + 0.5) * pix
    phi = np.tile(a * np.sin(2.0 * np.pi * x / per), (n, 1))
    p = O.ScreenParams(n=n, pixel_km=pix, r_diff_km=100.0, lambda_nm=lam, lambda_ref_nm=lam_ref,
                       z_pc=z, margin_km=0.0)
    I = O.intensity_mono(phi, p)
    s = lam_ref / lam
    lz = lam * O.KM_PER_NM * z * O.KM_PER_PC
    orders = np.arange(-20, 21)
    amp = sum(special.jv(m, a * s) * np.exp(2j * np.pi * m * x / per) * np.exp(-1j * np.pi * lz * m * m / per ** 2)
              for m in orders)
    I_ref = np.tile(np.abs(amp) ** 2, (n, 1))
    # residual = harmonics |m| >= 8 aliased by the grid, ~J_8(a s)
    np.testing.assert_allclose(I, I_ref, atol=2e-5)


def test_talbot_self_imaging():
    """At the Talbot distance z_T = 2 p^2 / lambda a phase grating re-images: I = 1."""
    n, pix, lam = 64, 20.0, 500.0
    per = n * pix / 4.0
    z_pc = 2.0 * per ** 2 / (lam * O.KM_PER_NM) / O.KM_PER_PC
    x = (np.arange(n) + 0.5) * pix
    phi = np.add.outer(0.7 * np.cos(2 * np.pi * x / per), 2.1 * np.sin(2 * np.pi * x / per + 0.3))
    p = O.ScreenParams(n=n, pixel_km=pix, r_diff_km=100.0, z_pc=z_pc, margin_km=0.0)
    np.testing.assert_allclose(O.intensity_mono(phi, p), 1.0, atol=1e-10)
    # a quarter of the Talbot distance does not (the check has teeth)
    I4 = O.intensity_mono(phi, p.with_(z_pc=z_pc / 4.0))
    assert np.abs(I4 - 1.0).max() > 0.1


def test_taper_shape():
    """SF of Sect. 3.2.1: 1/2 [1 + sin(pi x/L_m - pi/2)] = sin^2(pi x / 2 L_m) on the rising edge."""
    n, pix, lm = 200, 7.0, 300.0
    sf = O.taper_1d(n, pix, lm)
    x = (np.arange(n) + 0.5) * pix
    L = n * pix
    rise = x <= lm
    np.testing.assert_allclose(sf[rise], np.sin(np.pi * x[rise] / (2 * lm)) ** 2, atol=1e-14)
    np.testing.assert_allclose(sf, sf[::-1], atol=1e-14)       # symmetric about L/2
    assert np.all(sf[(x > lm) & (x < L - lm)] == 1.0)
    assert np.all((sf >= 0) & (sf <= 1))
    np.testing.assert_allclose(O.taper_1d(n, pix, 0.0), 1.0)


def test_passband_sum_weights():
    p = O.ScreenParams(n=64, pixel_km=10.0, r_diff_km=15.0, seed=4, margin_km=0.0, lambda_ref_nm=550.0)
    phi = O.make_screen(p)
    lams = [480.0, 550.0, 610.0]
    I = O.sum_passband(phi, p, lams)
    assert I.mean() == pytest.approx(1.0, rel=1e-12)     # sum w = 1, untapered: unit mean
    Iw = O.sum_passband(phi, p, lams, [0.2, 0.5, 0.3])
    ref = 0.2 * O.intensity_mono(phi, p, 480.0) + 0.5 * O.intensity_mono(phi, p, 550.0) \
        + 0.3 * O.intensity_mono(phi, p, 610.0)
    np.testing.assert_allclose(Iw, ref, atol=1e-12)


def test_point_source_strong_regime_modulation_near_one():
    """Loose sanity only (parity unpinned): a point source in the strong regime has m ~ 1 (Sect. 4.1)."""
    p = O.ScreenParams(n=256, pixel_km=20.0, r_diff_km=100.0, seed=20131514, margin_km=0.0)
    m = O.modulation_index(O.intensity_mono(O.make_screen(p), p))
    assert 0.7 < m < 1.4
