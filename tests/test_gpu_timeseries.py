"""Light-curve time analysis (Sect. 5) on the GPU vs the FP64 oracle, and the
two-telescope decorrelation of a simulated pattern.

Periodograms: within 1e-5 of the largest bin (FP32 transform after an FP64 mean
removal).  Correlations: 1e-12 (FP64 sums of the same FP32 curves).  On a
8192^2 disk-source pattern the curves of parallel tracks stay correlated at
separations well below R_ref and decorrelate beyond 2 max(R_ref, R_s).
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1301_0514_gb300 as S
import paper_1301_0514_gb300.timeseries as TS

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [16, 64, 512, 4096, 8192])
def test_power_spectrum_matches_oracle(n):
    rng = np.random.default_rng(n)
    c = (1.0 + 0.05 * rng.standard_normal((7, n)) + 0.2 * np.cos(2 * np.pi * 3 * np.arange(n) / n)).astype(np.float32)
    P = S.curve_power_spectrum(torch.from_numpy(c).cuda()).cpu().numpy()
    want = O.periodogram(c.astype(np.float64))
    assert P.shape == want.shape
    assert np.abs(P - want).max() <= 1e-5 * want.max()
    assert P[:, 0].max() == 0.0


def test_correlation_matches_oracle():
    rng = np.random.default_rng(7)
    a = (1.0 + rng.standard_normal((5, 3000))).astype(np.float32)
    b = (0.3 * a + rng.standard_normal((5, 3000))).astype(np.float32)
    r = S.curve_correlation(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    np.testing.assert_allclose(r, O.pearson(a.astype(np.float64), b.astype(np.float64)), rtol=1e-12)
    r1 = S.curve_correlation(torch.from_numpy(a[:1]).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    np.testing.assert_allclose(r1, O.pearson(np.repeat(a[:1], 5, 0).astype(np.float64), b.astype(np.float64)),
                               rtol=1e-12)
    # groups: rows 0 and 3 of a strided view against pairs (0, 1, 2) and (3, 4, ... ) of b
    big = torch.from_numpy(np.concatenate([a, b[:1]], 0)).cuda()
    b6 = torch.from_numpy(np.concatenate([b, b[:1]], 0)).cuda()
    r2 = S.curve_correlation(big, b6, a_rows=2, a_stride=3 * 3000).cpu().numpy()
    want = O.pearson(np.repeat(np.stack([a[0], a[3]]), 3, 0).astype(np.float64),
                     np.concatenate([b, b[:1]], 0).astype(np.float64))
    np.testing.assert_allclose(r2, want, rtol=1e-12)


def test_parallel_tracks_match_oracle():
    tr = (100.5, 7.25, 1.1, 0.9)
    sep = [0.0, 3.0, 250.0]
    np.testing.assert_allclose(TS.parallel_tracks(tr, sep), O.parallel_tracks(tr, sep), rtol=0, atol=1e-12)


def test_two_telescopes_decorrelate_beyond_refraction_scale():
    """8192^2, 10 km pixels, R_diff = 300 km at 550 nm: R_ref = 9050 km (905 px); disk R_s = R_ref/2."""
    n, pix = 8192, 10.0
    r_ref = 550.0 * 1e-12 * 160.0 * 3.0856775814913673e13 / 300.0
    p = S.params(n=n, pixel_km=pix, r_diff_km=300.0, lambda_nm=550.0, source_radius_km=0.5 * r_ref,
                 seed=20130514 + 9600)
    I = S.propagate(p, S.make_screen(p))
    S.smooth_source(p, I)
    rng = np.random.default_rng(5)
    base = np.stack([np.full(48, 900.0), rng.uniform(0.0, n, 48), np.zeros(48), np.ones(48)], axis=1)
    sep_km = np.array([0.0, 0.05, 0.2, 2.5, 3.0, 4.0]) * r_ref
    r = TS.decorrelation(p, I, base, sep_km / pix, 6000).cpu().numpy().mean(axis=0)
    assert r[0] == pytest.approx(1.0, abs=1e-12)
    assert r[1] > 0.9 and r[2] > 0.6
    assert r[1] > r[2] > max(abs(r[3]), abs(r[4]), abs(r[5]))
    assert np.all(np.abs(r[3:]) < 0.2)
