"""Pins of the oracle's random draws and spectrum (CPU only).

The oracle is checked against things fixed outside itself: the generator's
published known answers, the moments of the normal distribution, the paper's
printed normalisation results and closed forms of the structure function.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O


def test_philox_known_answers(golden):
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(*[np.uint64(x) for x in v[:6]])
        assert [int(o) for o in out] == v[6:]


def test_philox_vectorised_matches_scalar():
    c0 = np.arange(17, dtype=np.uint64)
    out = O.philox4x32_10(c0, np.uint64(3), np.uint64(5), np.uint64(0), np.uint64(11), np.uint64(13))
    for i in range(17):
        o = O.philox4x32_10(np.uint64(i), np.uint64(3), np.uint64(5), np.uint64(0), np.uint64(11), np.uint64(13))
        assert [int(w[i]) for w in out] == [int(x) for x in o]


def test_uniform53_range_and_resolution():
    hi = np.array([0, 0xFFFFFFFF, 0x80000000], dtype=np.uint64)
    lo = np.array([0, 0xFFFFFFFF, 0], dtype=np.uint64)
    u = O.uniform53(hi, lo)
    assert u[0] == 0.5 * 2.0 ** -53          # never zero: log stays finite
    assert u[1] == 1.0 - 0.5 * 2.0 ** -53    # never one
    assert u[2] == 0.5 + 0.5 * 2.0 ** -53


def test_gaussian_moments():
    w = O.noise_words(1024, seed=7, screen_id=1)
    g_re, g_im = O.gaussian_pair(w)
    n = g_re.size
    for g in (g_re, g_im):
        assert abs(g.mean()) < 5.0 / math.sqrt(n)
        assert abs(g.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
        # fourth moment of N(0,1) is 3
        assert abs(np.mean(g ** 4) - 3.0) < 0.05
    assert abs(np.mean(g_re * g_im)) < 5.0 / math.sqrt(n)
    # distinct seeds / screen ids give different streams
    w2 = O.noise_words(8, seed=8, screen_id=1)
    w3 = O.noise_words(8, seed=7, screen_id=2)
    assert not np.array_equal(w2[0], O.noise_words(8, 7, 1)[0])
    assert not np.array_equal(w3[0], O.noise_words(8, 7, 1)[0])


@pytest.mark.parametrize("beta", [11.0 / 3.0, 3.3, 3.1])
def test_spectrum_normalisation_continuum(beta):
    """2 int_0^inf 2 pi q S(q) (1 - J0(2 pi q r)) dq = (r / R_diff)^(beta-2) (Eq. dphi with Eq. spectre)."""
    r_diff = 100.0
    for r in (30.0, 100.0, 400.0):
        # substitute u = 2 pi q r; split the range to handle the oscillating tail
        def integrand(u):
            q = u / (2.0 * math.pi * r)
            return 2.0 * 2.0 * math.pi * q * O.phase_spectrum(q, r_diff, beta) * (1.0 - special.j0(u)) / (2.0 * math.pi * r)
        total = integrate.quad(integrand, 0.0, 1.0, limit=200)[0]
        a = 1.0
        while a < 4000.0:
            total += integrate.quad(integrand, a, 2.0 * a, limit=400)[0]
            a *= 2.0
        # tail beyond 4000: J0 averages out, integrand ~ 2 * 2 pi q S(q) / (2 pi r)
        c = 2.0 * 2.0 * math.pi * r_diff ** 2 / (2.0 * (2.0 * math.pi) ** (beta - 1.0) * O.f_beta(beta)) \
            * r_diff ** (-beta) / (2.0 * math.pi * r) ** (2.0 - beta) / (2.0 * math.pi * r)
        total += c * a ** (2.0 - beta) / (beta - 2.0)
        assert total == pytest.approx((r / r_diff) ** (beta - 2.0), rel=2e-3)


def test_rdiff_reconstructed_matches_paper(golden):
    """Sect. 3.1.1: the spectrum sampled on N ~ 14000, Delta = 28.85 km, R_diff = 500 km gives R_diff^rec ~ 540 km."""
    vals = {r[0]: (float(r[1]), float(r[2])) for r in golden("paper_worked_numbers.txt")}
    target, tol = vals["rdiff_rec_km_14000_28p85_500"]
    r = np.linspace(500.0, 580.0, 81)
    D = O.structure_function_discrete(14000, 28.85, 500.0, 11.0 / 3.0, r)
    r_rec = np.interp(1.0, D, r)
    assert r_rec == pytest.approx(target, rel=tol)
    # and the sampling can only lose variance: D_disc < continuum everywhere
    assert np.all(D < (r / 500.0) ** (5.0 / 3.0))


def test_spectrum_power_per_bin():
    """<|F|^2> = L_x L_y S(q) (Eq. densite): the mean of |F|^2 / (L^2 S) over bins is 1."""
    p = O.ScreenParams(n=256, pixel_km=10.0, r_diff_km=50.0, seed=3)
    F = O.noise_spectrum(p)
    L = p.n * p.pixel_km
    k = O.fft_freqs(p.n, p.pixel_km)
    Q = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    S = O.phase_spectrum(Q, p.r_diff_km, p.beta)
    ratio = (np.abs(F) ** 2)[Q > 0] / (L * L * S[Q > 0])
    assert F[0, 0] == 0.0
    assert ratio.mean() == pytest.approx(1.0, abs=5.0 / math.sqrt(ratio.size))


def test_screen_structure_function_matches_sampled_spectrum():
    """Mean empirical D(r) of synthesised screens equals the sampled-spectrum sum (Sect. 3.1.1)."""
    n, pix, rd = 128, 10.0, 40.0
    lags = [1, 2, 4, 8, 16]
    emp = np.zeros(len(lags))
    nseed = 24
    var = 0.0
    for s in range(nseed):
        phi = O.make_screen(O.ScreenParams(n=n, pixel_km=pix, r_diff_km=rd, seed=1000 + s))
        var += phi.var() + phi.mean() ** 2
        for j, lag in enumerate(lags):
            d = phi - np.roll(phi, -lag, axis=1)
            emp[j] += np.mean(d * d)
    emp /= nseed
    var /= nseed
    theory = O.structure_function_discrete(n, pix, rd, 11.0 / 3.0, np.array(lags) * pix)
    np.testing.assert_allclose(emp, theory, rtol=0.12)
    # phase variance = sum S dq^2 (Sect. 3.1)
    k = O.fft_freqs(n, pix)
    Q = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    S = O.phase_spectrum(Q, rd, 11.0 / 3.0)
    S[0, 0] = 0.0
    assert var == pytest.approx(S.sum() / (n * pix) ** 2, rel=0.35)


def test_screen_is_real_part_times_sqrt2():
    """phi = sqrt(2)/(L^2) Re sum F exp(+2 pi i k x): compare with a direct double sum on a tiny grid."""
    p = O.ScreenParams(n=8, pixel_km=25.0, r_diff_km=30.0, seed=5, screen_id=9)
    F = O.noise_spectrum(p)
    L = p.n * p.pixel_km
    j = np.arange(p.n)
    E = np.exp(2j * np.pi * np.outer(j, j) / p.n)       # E[x, k]
    direct = np.sqrt(2.0) / L ** 2 * np.real(E @ F @ E.T)  # rows y, cols x
    np.testing.assert_allclose(O.make_screen(p), direct, atol=1e-12)


def test_paper_parameter_numbers(golden):
    vals = {r[0]: (float(r[1]), float(r[2])) for r in golden("paper_worked_numbers.txt")}
    v, t = vals["fresnel_radius_km_2160nm_160pc"]
    assert O.fresnel_radius_km(2160.0, 160.0) == pytest.approx(v, rel=t)
    v, t = vals["fresnel_radius_km_1um_1kpc"]
    assert O.fresnel_radius_km(1000.0, 1000.0) == pytest.approx(v, rel=t)
    p = O.ScreenParams(n=8, pixel_km=1.0, r_diff_km=100.0, lambda_nm=2160.0, lambda_ref_nm=2160.0, z_pc=160.0)
    v, t = vals["refraction_radius_km_2160nm_160pc_rdiff100"]
    assert O.refraction_radius_km(p, 2160.0) == pytest.approx(v, rel=t)
    p = O.ScreenParams(n=8, pixel_km=1.0, r_diff_km=1000.0, lambda_nm=1000.0, lambda_ref_nm=1000.0, z_pc=1000.0)
    v, t = vals["refraction_radius_km_1um_1kpc_rdiff1000"]
    assert O.refraction_radius_km(p, 1000.0) == pytest.approx(v, rel=t)
    v, t = vals["alias_onset_px_rf1000_pix22"]
    assert O.aliasing_onset_px(1000.0, 22.0) == pytest.approx(v, rel=t)


def test_rdiff_wavelength_scaling_kolmogorov():
    """For a fixed column density R_diff grows as lambda^(6/5) (footnote of Sect. 3.2.4)."""
    p = O.ScreenParams(n=8, pixel_km=1.0, r_diff_km=100.0, lambda_ref_nm=500.0)
    assert O.diffraction_radius_km(p, 1000.0) == pytest.approx(100.0 * 2.0 ** 1.2, rel=1e-12)
