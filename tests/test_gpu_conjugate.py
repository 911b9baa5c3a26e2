"""The paper's one-FFT propagator (Eq. intens, Eq. Gxy) on the GPU vs the FP64 oracle.

Patterns are compared with an absolute bound of 2e-4 of the pattern's maximum (the
intensity tolerance, on the scale of the pattern: off critical sampling a pattern's
mean is (Delta_1/Delta_0)^2 <SF^2>, not 1).  At critical sampling the pattern must
equal the transfer-function pattern pixel for pixel, which is checked on the GPU up
to N = 16384 (lines split over two-block clusters) where the oracle cannot run.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1301_0514_gb300 as S

pytestmark = pytest.mark.gpu

TOL = 2e-4


def _pair(n, pix, rd, lam=550.0, lam_ref=550.0, margin=-1.0, seed=20130514 + 9300, sid=1, z=160.0):
    kw = dict(n=n, pixel_km=pix, r_diff_km=rd, lambda_nm=lam, lambda_ref_nm=lam_ref, z_pc=z, margin_km=margin,
              seed=seed, screen_id=sid)
    return S.params(**kw), O.ScreenParams(**kw)


def _critical_pixel(n, lam=550.0, z=160.0):
    return math.sqrt(lam * O.KM_PER_NM * z * O.KM_PER_PC / n)


def _close(got, want):
    scale = max(float(np.abs(want).max()), 1e-30)
    assert np.abs(got - want).max() <= TOL * scale, (np.abs(got - want).max(), scale)


@pytest.mark.parametrize("n,pix,rd,margin", [(16, 700.0, 900.0, 2000.0), (64, 40.0, 90.0, -1.0),
                                             (256, 25.0, 60.0, 0.0), (1024, 12.0, 40.0, -1.0)])
def test_conjugate_matches_oracle(n, pix, rd, margin):
    pg, po = _pair(n, pix, rd, lam=620.0, margin=margin)
    phi = O.make_screen(po)
    h = S.propagate_conjugate(pg, torch.from_numpy(phi).cuda()).cpu().numpy()
    _close(h, O.propagate_conjugate(phi, po))
    assert S.conjugate_pixel_km(pg) == pytest.approx(O.observer_pixel_km(po, 620.0), rel=1e-15)


@pytest.mark.parametrize("n", [64, 512, 2048])
def test_conjugate_equals_transfer_function_at_critical_sampling(n):
    pg, po = _pair(n, _critical_pixel(n), 3.0 * _critical_pixel(n))
    phi = S.make_screen(pg)
    h = S.propagate_conjugate(pg, phi).cpu().numpy()
    I = S.propagate(pg, phi).cpu().numpy()
    assert np.abs(h - I).max() <= TOL * max(1.0, float(I.max()))
    if n <= 512:
        _close(h, O.propagate_conjugate(O.make_screen(po), po))


def test_conjugate_16384_split_lines_at_critical_sampling():
    n = 16384
    pix = _critical_pixel(n, lam=500.0)
    pg = S.params(n=n, pixel_km=pix, r_diff_km=4.0 * pix, lambda_nm=500.0, seed=20130514 + 9310)
    phi = S.make_screen(pg)
    h = S.propagate_conjugate(pg, phi)
    I = S.propagate(pg, phi)
    for y in (0, 77, 8192, 16383):
        assert (h[y] - I[y]).abs().max().item() <= TOL * max(1.0, I[y].max().item())
    assert abs(h.double().mean().item() - I.double().mean().item()) < 1e-5


def test_conjugate_16384_pattern_mode_equals_direct():
    """Two copies of the grid wavelength go through the stored patterns and the resampling
    (ratio 1: the identity) and must give the direct single-wavelength pattern."""
    n = 16384
    pix = _critical_pixel(n, lam=500.0)
    pg = S.params(n=n, pixel_km=pix, r_diff_km=4.0 * pix, lambda_nm=500.0, seed=20130514 + 9320)
    phi = S.make_screen(pg)
    h = S.propagate_conjugate(pg, phi)
    two = S.sum_passband_conjugate(pg, phi, [500.0, 500.0], [0.5, 0.5])
    for y in (0, 5, 8191, 8192, 16383):
        assert (two[y] - h[y]).abs().max().item() <= 1e-6 * max(1.0, h[y].max().item())
    assert (two[:, 777] - h[:, 777]).abs().max().item() <= 1e-6 * max(1.0, h[:, 777].max().item())


@pytest.mark.parametrize("lams,weights", [((550.0,), None), ((480.0, 550.0, 640.0), None),
                                          ((450.0, 520.0, 600.0, 700.0), (0.1, 0.2, 0.3, 0.4))])
def test_conjugate_passband_matches_oracle(lams, weights):
    pg, po = _pair(128, 30.0, 70.0)
    phi = O.make_screen(po)
    got = S.sum_passband_conjugate(pg, torch.from_numpy(phi).cuda(), lams, weights).cpu().numpy()
    _close(got, O.sum_passband_conjugate(phi, po, lams, weights))


def test_conjugate_passband_groups_and_accumulate():
    pg, po = _pair(256, 20.0, 50.0, lam=600.0)
    lams = (480.0, 530.0, 600.0, 690.0, 700.0)
    phi = O.make_screen(po)
    ws = torch.empty(S.workspace_bytes(pg, 1), dtype=torch.uint8, device="cuda")      # one wavelength per group
    out = torch.full((256, 256), 0.5, device="cuda")
    S.sum_passband_conjugate(pg, torch.from_numpy(phi).cuda(), lams, out=out, accumulate=True, workspace=ws)
    want = O.sum_passband_conjugate(phi, po, lams)
    _close(out.cpu().numpy() - 0.5, want)
