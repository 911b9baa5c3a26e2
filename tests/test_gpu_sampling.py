"""The sampling condition of Sect. 3.2.2 (pixel < R_diff(lambda)/2) on the propagating calls:
violating parameters leave a warning (SamplingWarning in Python) and the call still runs; compliant
ones leave none.  The ratio itself is pinned on the host in test_abi.py."""
import warnings

import pytest
import torch

import paper_1301_0514_gb300 as S

pytestmark = pytest.mark.gpu


def test_propagate_warns_when_the_pixel_exceeds_half_rdiff():
    bad = S.params(n=64, pixel_km=60.0, r_diff_km=100.0, seed=5)
    phi = S.make_screen(bad)
    with pytest.warns(S.SamplingWarning, match=r"Sect\. 3\.2\.2"):
        I = S.propagate(bad, phi)
    assert "at 500 nm" in S.last_warning()
    assert torch.isfinite(I).all()
    good = S.params(n=64, pixel_km=20.0, r_diff_km=100.0, seed=5)
    with warnings.catch_warnings():
        warnings.simplefilter("error", S.SamplingWarning)
        S.propagate(good, S.make_screen(good))
    assert S.last_warning() == ""


def test_passband_warns_at_its_shortest_wavelength():
    # 2 x 45 / 100 = 0.9 at lambda_ref = 550 nm, but R_diff(400 nm) = 100 (400/550)^1.2 = 68 km
    p = S.params(n=64, pixel_km=45.0, r_diff_km=100.0, lambda_nm=550.0, lambda_ref_nm=550.0, seed=6)
    phi = S.make_screen(p)
    with pytest.warns(S.SamplingWarning, match="at 400 nm"):
        S.sum_passband(p, phi, [700.0, 400.0, 550.0])
    with warnings.catch_warnings():
        warnings.simplefilter("error", S.SamplingWarning)
        S.sum_passband(p, phi, [550.0, 700.0])
    with pytest.warns(S.SamplingWarning, match="at 400 nm"):
        S.sum_passband_conjugate(p, phi, [400.0, 550.0])


def test_batch_names_the_first_item_that_warns():
    good = S.params(n=64, pixel_km=20.0, r_diff_km=100.0, seed=7, screen_id=0)
    bad = S.params(n=64, pixel_km=60.0, r_diff_km=100.0, seed=7, screen_id=1)
    items = [dict(params=p, intensity=torch.empty((64, 64), device="cuda")) for p in (good, bad, bad)]
    with pytest.warns(S.SamplingWarning, match="item 1:"):
        S.run_batch(items, [500.0], n_lanes=2)
    with warnings.catch_warnings():
        warnings.simplefilter("error", S.SamplingWarning)
        S.run_batch(items[:1], [500.0], n_lanes=1)
