"""Host-side helpers of the package (no GPU): the m-sweep layout and Eq. xparam of sweeps.py, the
grouping of sweep results, and the parallel tracks of timeseries.py, against the oracle and
geometry."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import sweeps as SW
from paper_1301_0514_gb300 import timeseries as TS


def test_xparam_matches_the_papers_numerical_form():
    """The package's Eq. xparam (first form) against the oracle's printed numerical form
    (coefficient 0.035, read to 2 %) over the sweep's range."""
    for rd in (50.0, 200.0, 500.0):
        for rs_rsun in (0.25, 1.0, 1.5):
            for lam in (1000.0, 2162.0):
                z0, z1_kpc = 160.0, 1.0
                rs_km = rs_rsun * SW.R_SUN_KM * z0 / (z1_kpc * 1000.0)
                got = SW.xparam_m(rd, lam, z0, rs_km)
                ratio = rs_rsun / z1_kpc / 0.1                  # (r_s/z1) / (R_sun / 10 kpc)
                want = O.xparam_m_numeric(rd, lam, z0, ratio)
                assert got == pytest.approx(want, rel=0.02)
                assert got == pytest.approx(O.xparam_m(rd, lam, z0, rs_km), rel=1e-13)


def test_sweep_points_layout():
    pts = SW.sweep_points(r_diffs=(100.0, 300.0), radii_rsun=(0.5, 1.0, 1.5), betas=(3.1, 3.9), n=2048)
    assert len(pts) == 12
    assert len({(p.params.seed, p.params.screen_id) for p in pts}) == 12
    for pt in pts:
        p = pt.params
        assert p.pixel_km == pytest.approx(pt.r_diff_km / 3.0)
        assert p.source_radius_km == pytest.approx(pt.r_s_rsun * SW.R_SUN_KM * 160.0 / 1000.0, rel=1e-14)
        assert p.lambda_nm == p.lambda_ref_nm == SW.KS_CENTRE_NM
        assert p.beta == pt.beta
        po = O.ScreenParams(n=p.n, pixel_km=p.pixel_km, r_diff_km=p.r_diff_km, beta=p.beta, lambda_nm=p.lambda_nm,
                            lambda_ref_nm=p.lambda_ref_nm, z_pc=p.z_pc, source_radius_km=p.source_radius_km,
                            margin_km=p.margin_km)
        assert pt.n_regions == pytest.approx(O.refractive_regions(po), rel=1e-12)
    # the K_s band: 21 wavelengths over [2.08, 2.28] um
    assert len(SW.KS_BAND_NM) == 21 and SW.KS_BAND_NM[0] == 2080.0 and SW.KS_BAND_NM[-1] == 2280.0


def test_summarize_groups_by_prediction_and_drops_small_zones():
    pts = SW.sweep_points(r_diffs=(100.0, 200.0, 400.0), radii_rsun=(0.25, 1.0), n=1024)
    m = np.array([pt.m_theory * 1.1 for pt in pts])
    rows = SW.summarize(pts, m, min_regions=0.0)
    assert sum(r[3] for r in rows) == sum(1 for pt in pts if 0.004 <= pt.m_theory < 0.6)
    for centre, mean, rms, count in rows:
        assert count >= 1 and rms >= 0.0
        assert 0.004 <= centre < 0.6
    # a threshold no zone reaches leaves nothing
    assert SW.summarize(pts, m, min_regions=1e30) == []


@pytest.mark.parametrize("theta", [0.0, 0.7, math.pi / 2, 2.9])
def test_parallel_tracks_are_parallel_and_offset_perpendicularly(theta):
    base = (12.5, -3.0, theta, 0.8)
    seps = [0.0, 1.5, -4.0, 100.0]
    tr = TS.parallel_tracks(base, seps)
    assert tr.shape == (4, 4)
    d = np.array([math.cos(theta), math.sin(theta)])
    for (x, y, th, ds), s in zip(tr, seps):
        assert th == theta and ds == 0.8
        off = np.array([x - base[0], y - base[1]])
        assert abs(off @ d) < 1e-12                              # perpendicular to the motion
        assert np.linalg.norm(off) == pytest.approx(abs(s), abs=1e-12)
    np.testing.assert_allclose(tr, O.parallel_tracks(base, seps), rtol=0, atol=1e-12)
