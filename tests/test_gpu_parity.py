"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Tolerances (fixed by the required accuracy of the FP32 path, not tuned):
  * Philox words: bit-exact.
  * Shaped spectrum: bins with |mx|, |my| <= 32 are FP64 on both sides (1e-13
    relative; the GPU widens its FP64 square up to 256 for screens with large
    phases); the other bins may be drawn in FP32 on the GPU (2e-6 relative).
  * Phase screen: 2e-6 rad absolute.  The screen's error is ~1e-7 of the rms
    phase carried by the FP32 bins (a few rad at most); the intensity bound
    needs the phase to ~4e-6 rad (2e-4 / (2 |A|_max * 5 sigma), |A|^2 <= 20).
  * Intensity, normalised to the unobstructed wave: 2e-4 max absolute.
  * Modulation index: 1e-4 relative.
  * Line FFT: 2e-6 (FP32) / 1e-13 (FP64) relative to the line's l2 norm.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import workloads as W
from conftest import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

I_TOL = 2e-4
M_TOL = 1e-4
PHI_TOL = 2e-6


def _item(n=256, pixel_km=20.0, r_diff_km=100.0, **kw):
    return W._item(n, pixel_km, r_diff_km, **kw)


# ---------------------------------------------------------------------------
def test_noise_words_bit_exact():
    for n, seed, sid in [(64, 0, 0), (256, 2**40 + 12345, 7)]:
        it = _item(n=n, seed=seed, screen_id=sid)
        g = S.noise_words(gpu_params(it)).cpu().numpy().view(np.uint32)
        w = O.noise_words(n, seed, sid)
        for j in range(4):
            np.testing.assert_array_equal(g[..., j].astype(np.uint64), w[j])


@pytest.mark.parametrize("beta", [11.0 / 3.0, 3.3, 3.9])
def test_noise_spectrum(beta):
    n = 1024    # both kinds of bins: |mx|, |my| <= 32 are always drawn in FP64, the rest may be FP32
    it = _item(n=n, pixel_km=15.0, r_diff_km=40.0, beta=beta, seed=99, screen_id=3)
    g = S.noise_spectrum(gpu_params(it)).cpu().numpy()
    o = O.noise_spectrum(oracle_params(it))
    m = np.abs(np.fft.fftfreq(n, 1.0 / n))
    low = (m[:, None] <= 32) & (m[None, :] <= 32)
    rel = np.abs(g - o) / np.maximum(np.abs(o), 1e-300)
    assert rel[low].max() <= 1e-13
    assert rel[~low].max() <= 2e-6
    assert g[0, 0] == 0


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192])
@pytest.mark.parametrize("direction", [-1, 1])
def test_fft_lines_fp32(n, direction):
    rng = np.random.default_rng(n)
    lines = 3 if n >= 1024 else 37          # several blocks and a partly filled last one
    x = (rng.standard_normal((lines, n)) + 1j * rng.standard_normal((lines, n))).astype(np.complex64)
    t = torch.from_numpy(x).cuda()
    S.fft_lines(t, direction)
    ref = np.fft.fft(x.astype(np.complex128), axis=1) if direction < 0 else np.fft.ifft(x.astype(np.complex128), axis=1) * n
    err = np.linalg.norm(t.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < 2e-6


@pytest.mark.parametrize("n", [16, 32, 256, 2048, 4096, 8192])
def test_fft_lines_fp64(n):
    rng = np.random.default_rng(n + 1)
    x = rng.standard_normal((5, n)) + 1j * rng.standard_normal((5, n))
    t = torch.from_numpy(x.copy()).cuda()
    S.fft_lines(t, 1)
    ref = np.fft.ifft(x, axis=1) * n
    err = np.linalg.norm(t.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < 1e-13


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,pixel,rd,beta", [(256, 20.0, 100.0, 11 / 3), (1024, 10.0, 30.0, 11 / 3),
                                             (512, 10.0, 50.0, 3.1), (64, 30.0, 70.0, 3.9),
                                             (16, 40.0, 100.0, 11 / 3)])
def test_make_screen(n, pixel, rd, beta):
    it = _item(n=n, pixel_km=pixel, r_diff_km=rd, beta=beta, seed=W.SEED_BASE + n, screen_id=1)
    phi_g = S.make_screen(gpu_params(it)).cpu().numpy()
    phi_o = O.make_screen(oracle_params(it))
    assert np.abs(phi_g - phi_o).max() <= PHI_TOL


def _intensity_case(it, lam=None):
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi = O.make_screen(p_o)
    I_o = O.intensity_mono(phi, p_o, lam)
    phi_t = torch.from_numpy(phi).cuda()
    I_g = S.propagate(p_g if lam is None else p_g.replace(lambda_nm=lam), phi_t).cpu().numpy()
    return I_g, I_o


def test_small_screen_256_full_path():
    """256^2, 20 km, R_diff = 100 km, 500 nm, 160 pc: GPU screen + propagation + track vs oracle."""
    it = W.small_screen_256()[0]
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi_t = S.make_screen(p_g)
    I_g = S.propagate(p_g, phi_t)
    c_g = S.lightcurve(p_g, I_g, it["tracks"], it["n_samples"]).cpu().numpy()
    m_g = S.modulation_index(p_g, I_g).cpu().numpy()
    phi_o = O.make_screen(p_o)
    I_o = O.intensity_mono(phi_o, p_o)
    c_o = O.lightcurves(I_o, it["tracks"], it["n_samples"])
    err = np.abs(I_g.cpu().numpy() - I_o).max()
    assert err <= I_TOL, err
    assert np.abs(c_g - c_o).max() <= I_TOL
    assert m_g[0] == pytest.approx(O.modulation_index_map(I_o, p_o), rel=M_TOL)


@pytest.mark.parametrize("case", [
    dict(n=128, pixel_km=20.0, r_diff_km=60.0, margin_km=0.0),               # untapered
    dict(n=512, pixel_km=10.0, r_diff_km=25.0),                             # several row/column blocks
    dict(n=2048, pixel_km=10.0, r_diff_km=40.0, lambda_nm=700.0, lambda_ref_nm=550.0),
    dict(n=32, pixel_km=50.0, r_diff_km=120.0, margin_km=200.0),            # explicit margin
    dict(n=16, pixel_km=50.0, r_diff_km=120.0),
    dict(n=256, pixel_km=10.0, r_diff_km=15.0, beta=3.9),
])
def test_propagate_matches_oracle(case):
    it = _item(seed=W.SEED_BASE + 77, **case)
    I_g, I_o = _intensity_case(it)
    err = np.abs(I_g - I_o).max()
    assert err <= I_TOL, err


def test_uniform_screen_gpu():
    """phi = 0 without taper gives exactly 1 (to FP32 rounding); with taper the zone is flat (Sect. 3.2.1)."""
    n = 256
    phi = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    I = S.propagate(S.params(n=n, pixel_km=20.0, r_diff_km=100.0, margin_km=0.0), phi).cpu().numpy()
    assert np.abs(I - 1.0).max() < 1e-5
    p = S.params(n=1024, pixel_km=20.0, r_diff_km=100.0, z_pc=50.0)
    I = S.propagate(p, torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")).cpu().numpy()
    I_o = O.intensity_mono(np.zeros((1024, 1024)), O.ScreenParams(n=1024, pixel_km=20.0, r_diff_km=100.0, z_pc=50.0))
    assert np.abs(I - I_o).max() <= I_TOL


@pytest.mark.parametrize("workspace_groups", [None, 2])
def test_sum_passband(workspace_groups):
    lams = np.array([480.0, 515.0, 550.0, 590.0, 640.0])
    wts = np.array([0.1, 0.3, 0.2, 0.25, 0.15])
    it = _item(n=256, pixel_km=10.0, r_diff_km=30.0, lambda_nm=550.0, lambda_ref_nm=550.0, seed=5)
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi = O.make_screen(p_o)
    ws = None
    if workspace_groups:
        ws = torch.empty(S.workspace_bytes(p_g, workspace_groups), dtype=torch.uint8, device="cuda")
    I_g = S.sum_passband(p_g, torch.from_numpy(phi).cuda(), lams, wts, workspace=ws).cpu().numpy()
    I_o = O.sum_passband(phi, p_o, lams, wts)
    assert np.abs(I_g - I_o).max() <= I_TOL
    # accumulate onto an existing map; flat weights
    base = torch.full((256, 256), 0.5, device="cuda")
    S.sum_passband(p_g, torch.from_numpy(phi).cuda(), lams, out=base, accumulate=True)
    assert np.abs(base.cpu().numpy() - 0.5 - O.sum_passband(phi, p_o, lams)).max() <= I_TOL


@pytest.mark.parametrize("n,rs", [(256, 150.0), (1024, 900.0), (64, 60.0), (4096, 20000.0)])
def test_smooth_source(n, rs):
    rng = np.random.default_rng(n)
    I = rng.uniform(0.0, 3.0, (n, n))
    p = S.params(n=n, pixel_km=10.0, r_diff_km=50.0, source_radius_km=rs)
    t = torch.from_numpy(I.astype(np.float32)).cuda()
    out = S.smooth_source(p, t).cpu().numpy()
    ref = O.smooth_source(I.astype(np.float32).astype(np.float64), 10.0, rs)
    assert np.abs(out - ref).max() <= I_TOL


def test_smooth_point_source_is_identity():
    t = torch.rand((128, 128), device="cuda")
    before = t.clone()
    S.smooth_source(S.params(n=128, pixel_km=10.0, r_diff_km=50.0), t)
    assert torch.equal(t, before)


def test_lightcurves_edge_cases():
    n = 512
    rng = np.random.default_rng(3)
    I = rng.uniform(0, 2, (n, n)).astype(np.float32)
    t = torch.from_numpy(I).cuda()
    p = S.params(n=n, pixel_km=10.0, r_diff_km=50.0)
    tracks = W.random_tracks(rng, n, 70, 0.37)          # more than one launch of tracks
    tracks[0] = (-3.5, -700.25, 2.0, 1.7)               # negative coordinates: periodic wrap
    tracks[1] = (5.0, 9.0, 0.0, 1.0)                    # integer positions
    ns = 1001                                           # ragged sample count
    c = S.lightcurve(p, t, tracks, ns).cpu().numpy()
    ref = O.lightcurves(I.astype(np.float64), tracks, ns)
    assert np.abs(c - ref).max() <= 1e-5
    np.testing.assert_array_equal(c[1], I[9, (5 + np.arange(ns)) % n])
    assert S.lightcurve(p, t, np.zeros((0, 4)), 10).shape == (0, 10)
    cm = S.curve_modulation(torch.from_numpy(c).cuda()).cpu().numpy()
    for k in range(0, 70, 9):
        assert cm[k, 0] == pytest.approx(O.modulation_index(c[k].astype(np.float64)), rel=1e-9)


def test_modulation_index_fiducial_zone():
    n = 2048
    rng = np.random.default_rng(4)
    I = rng.uniform(0.5, 1.5, (n, n)).astype(np.float32)
    t = torch.from_numpy(I).cuda()
    for rd, rs, margin in [(300.0, 0.0, -1.0), (30.0, 0.0, -1.0), (300.0, 2000.0, -1.0), (300.0, 0.0, 0.0)]:
        it = _item(n=n, pixel_km=10.0, r_diff_km=rd, source_radius_km=rs, margin_km=margin)
        m = S.modulation_index(gpu_params(it), t).cpu().numpy()
        p_o = oracle_params(it)
        i0, i1, _ = O.fiducial_slice(p_o)
        assert m[3] == (i1 - i0) ** 2
        assert m[0] == pytest.approx(O.modulation_index_map(I.astype(np.float64), p_o), rel=1e-9)


# ---------------------------------------------------------------------------
def test_largest_phase_screen_full_path():
    """R_diff = 30 km (phase rms ~ 60 rad, peaks ~ 300 rad), 2048^2: screen, intensity, m vs oracle."""
    it = W.single_screens_4096(r_diffs=(30.0,), n=2048)[0]
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi_g = S.make_screen(p_g)
    phi_o = O.make_screen(p_o)
    assert np.abs(phi_o).max() > 100.0
    assert np.abs(phi_g.cpu().numpy() - phi_o).max() <= PHI_TOL
    I_g = S.propagate(p_g, phi_g)
    I_o = O.intensity_mono(phi_o, p_o)
    assert np.abs(I_g.cpu().numpy() - I_o).max() <= I_TOL
    assert S.modulation_index(p_g, I_g).cpu().numpy()[0] == pytest.approx(O.modulation_index_map(I_o, p_o), rel=M_TOL)


def test_batched_polychromatic_screen_passband_and_disk():
    """One 1024^2 screen of the batched workload: 32 wavelengths, disk source, tracks."""
    it = [x for x in W.batched_polychromatic() if x["n"] == 1024][0]
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi_g = S.make_screen(p_g)
    I_g = S.sum_passband(p_g, phi_g, it["lambdas_nm"])
    S.smooth_source(p_g, I_g)
    phi_o = O.make_screen(p_o)
    I_o = O.smooth_source(O.sum_passband(phi_o, p_o, it["lambdas_nm"]), p_o.pixel_km, p_o.source_radius_km)
    assert np.abs(I_g.cpu().numpy() - I_o).max() <= I_TOL
    c_g = S.lightcurve(p_g, I_g, it["tracks"], it["n_samples"]).cpu().numpy()
    c_o = O.lightcurves(I_o, it["tracks"], it["n_samples"])
    assert np.abs(c_g - c_o).max() <= I_TOL
    assert S.modulation_index(p_g, I_g).cpu().numpy()[0] == pytest.approx(O.modulation_index_map(I_o, p_o), rel=M_TOL)


def test_passband_at_the_wavelength_limit():
    """SCINT_MAX_LAMBDA wavelengths in one call (one group when the workspace allows, else groups)."""
    it = W._item(64, 20.0, 50.0, lambda_nm=550.0, lambda_ref_nm=550.0, seed=W.SEED_BASE + 77, screen_id=3)
    p_g, p_o = gpu_params(it), oracle_params(it)
    lams = np.linspace(420.0, 690.0, S.MAX_LAMBDA)
    w = np.linspace(1.0, 2.0, S.MAX_LAMBDA)
    w /= w.sum()
    phi = O.make_screen(p_o)
    got = S.sum_passband(p_g, torch.from_numpy(phi).cuda(), lams, w).cpu().numpy()
    assert np.abs(got - O.sum_passband(phi, p_o, lams, w)).max() <= I_TOL
    ws = torch.empty(S.workspace_bytes(p_g, 7), dtype=torch.uint8, device="cuda")   # groups of 7
    got7 = S.sum_passband(p_g, torch.from_numpy(phi).cuda(), lams, w, workspace=ws).cpu().numpy()
    assert np.abs(got7 - got).max() <= 1e-5


def test_empty_batch_and_empty_curves():
    S.run_batch([], [550.0])
    p = gpu_params(W._item(64, 20.0, 50.0))
    I = torch.ones((64, 64), device="cuda")
    assert S.lightcurve(p, I, np.zeros((0, 4)), 10).shape == (0, 10)
    out = S.curve_modulation(torch.empty((0, 5), device="cuda"))
    assert out.shape == (0, 3)
    torch.cuda.synchronize()
