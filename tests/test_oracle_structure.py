"""Pins of the oracle's screen check (Sect. 3.1.1, Eq. crec): the annulus-averaged
spectrum S_rec, the recomputed structure function D_rec and R_diff^rec.

What fixes each part independently of the oracle itself:
  * the annulus average: a brute-force loop over every bin of a tiny grid, and
    its expectation <|F|^2> = L^2 S (Eq. densite) within the sampling error;
  * the Hankel integral of Eq. crec: a Gaussian spectrum, whose 2D Fourier
    transform is a Gaussian in closed form, xi(r) = exp(-pi r^2 / a^2) / a^2;
  * the root D_rec(R) = 1: the same Gaussian, whose root is closed form too;
  * the whole chain with the sampled theoretical spectrum: the paper's
    R_diff^rec ~ 540 km for N ~ 14000, Delta = 28.85 km, R_diff = 500 km.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_annulus_average_brute_force():
    p = O.ScreenParams(n=10, pixel_km=7.0, r_diff_km=20.0, seed=77, screen_id=3)
    F = O.noise_spectrum(p)
    L = p.n * p.pixel_km
    sums, counts = {}, {}
    for iy in range(p.n):
        for ix in range(p.n):
            my = iy if iy < p.n // 2 else iy - p.n
            mx = ix if ix < p.n // 2 else ix - p.n
            j = int(round(math.sqrt(mx * mx + my * my)))
            sums[j] = sums.get(j, 0.0) + abs(F[iy, ix]) ** 2
            counts[j] = counts.get(j, 0) + 1
    s, c = O.spectrum_rec(p)
    assert len(s) == max(counts) + 1 == O.max_annulus(p.n) + 1
    for j in range(len(s)):
        assert c[j] == counts.get(j, 0)
        want = sums[j] / counts[j] / (L * L) if counts.get(j) else 0.0
        assert s[j] == pytest.approx(want, rel=1e-13, abs=0.0)
    assert s[0] == 0.0 and c[0] == 1            # only the DC bin, F_0 = 0


def test_partial_annuli_equal_full_computation():
    p = O.ScreenParams(n=96, pixel_km=10.0, r_diff_km=30.0, seed=5)
    s_all, c_all = O.spectrum_rec(p)
    s_12, c_12 = O.spectrum_rec(p, j_max=12)
    np.testing.assert_array_equal(c_12, c_all[:13])
    np.testing.assert_allclose(s_12, s_all[:13], rtol=1e-13)


def test_rec_spectrum_is_unbiased():
    """<|F|^2> = L_x L_y S(q) per bin (Eq. densite): S_rec over its expectation is 1 on average."""
    p = O.ScreenParams(n=512, pixel_km=10.0, r_diff_km=50.0, seed=11)
    s, c = O.spectrum_rec(p)
    # expectation of each annulus: the mean of S over the annulus' own bins
    m = np.rint(np.fft.fftfreq(p.n) * p.n).astype(np.int64)
    j = O.annulus_index(m[None, :], m[:, None])
    L = p.n * p.pixel_km
    Q = np.sqrt((m[None, :] ** 2 + m[:, None] ** 2).astype(float)) / L
    S = O.phase_spectrum(np.where(Q > 0, Q, 1.0), p.r_diff_km, p.beta)
    S[Q == 0] = 0.0
    expect = np.bincount(j.ravel(), weights=S.ravel()) / np.maximum(np.bincount(j.ravel()), 1)
    sel = np.arange(1, len(s))
    ratio = s[sel] / expect[sel]
    w = c[sel].astype(float)                     # |F|^2 / (L^2 S) is Exp(1): variance 1 per bin
    mean = np.sum(w * ratio) / np.sum(w)
    assert mean == pytest.approx(1.0, abs=5.0 / math.sqrt(w.sum()))
    # per annulus, the relative scatter is 1/sqrt(count)
    z = (ratio - 1.0) * np.sqrt(w)
    assert np.abs(z).max() < 6.0


def _gaussian_s(n, pixel_km, a):
    L = n * pixel_km
    q = np.arange(0, n // 2 + 1) / L
    return np.exp(-math.pi * a * a * q * q)


def test_hankel_sum_gaussian_closed_form():
    """S = exp(-pi a^2 q^2) has xi(r) = exp(-pi r^2/a^2)/a^2, so D(r) = 2 (1 - exp(-pi r^2/a^2))/a^2."""
    n, pix, a = 4096, 2.0, 50.0
    s = _gaussian_s(n, pix, a)
    r = np.array([1.0, 10.0, 37.5, 80.0, 400.0])
    want = 2.0 * (1.0 - np.exp(-math.pi * r * r / (a * a))) / (a * a)
    np.testing.assert_allclose(O.structure_function_rec(s, n, pix, r), want, rtol=1e-4)
    # the limits matter: q_max = 1/(2 Delta) cuts the Gaussian when Delta is coarse
    cut = O.structure_function_rec(_gaussian_s(64, 40.0, a), 64, 40.0, r)
    assert np.abs(cut / want - 1.0).max() > 0.05


def test_rdiff_rec_gaussian_root():
    """D(R) = 1 for the Gaussian: R = a sqrt(-ln(1 - a^2/2) / pi)."""
    n, pix, a = 4096, 0.1, 1.2
    s = _gaussian_s(n, pix, a)
    want = a * math.sqrt(-math.log(1.0 - a * a / 2.0) / math.pi)
    assert O.rdiff_rec(s, n, pix) == pytest.approx(want, rel=1e-5)
    # a screen that never reaches 1 rad^2 has no R_diff^rec
    assert math.isnan(O.rdiff_rec(0.1 * s, n, pix))


def test_rdiff_rec_of_sampled_spectrum_matches_paper(golden):
    """Sect. 3.1.1: Eq. crec with the theoretical spectrum sampled as in the simulation
    (N ~ 14000, Delta = 28.85 km, R_diff = 500 km) gives R_diff^rec ~ 540 km."""
    vals = {r[0]: (float(r[1]), float(r[2])) for r in golden("paper_worked_numbers.txt")}
    target, tol = vals["rdiff_rec_hankel_km_14000_28p85_500"]
    n, pix, rd = 14000, 28.85, 500.0
    q = np.arange(0, n // 2 + 1) / (n * pix)
    s = np.zeros_like(q)
    s[1:] = O.phase_spectrum(q[1:], rd, 11.0 / 3.0)
    r_rec = O.rdiff_rec(s, n, pix)
    assert r_rec == pytest.approx(target, rel=tol)
    # finite sampling loses large and small scales: D_rec < (r/R_diff)^(5/3), so R_rec > R_diff
    r = np.array([100.0, 500.0, 2000.0])
    assert np.all(O.structure_function_rec(s, n, pix, r) < (r / rd) ** (5.0 / 3.0))
    assert r_rec > rd
