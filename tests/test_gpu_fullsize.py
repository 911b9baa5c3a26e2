"""Whole-map parity at the full sizes of the single-screen and large-screen workloads.

Every output is compared element by element with the FP64 oracle run on the
same seeded inputs on the host (the oracle at 16384^2 holds ~30 GB; its 2D
transforms run on every host core):

  * 4096^2, 10 km pixels, R_diff in {30, 100, 300} km, 500 nm, point source,
    64 tracks of 2048 samples: phase screen, intensity map, curves, m of the
    map's fiducial zone and of every curve;
  * 8192^2, 5 km pixels, R_diff = 100 km, Kolmogorov, a disk of one R_ref,
    16 tracks of 4096 samples (the largest lines that are not split);
  * 16384^2, 5 km pixels, R_diff = 100 km: beta = 3.67 with a disk of one
    R_ref and beta = 3.3 with a point source, 16 tracks of 8192 samples;
  * the gradient of a light-curve misfit at 16384^2 (two wavelengths, disk
    source) against the oracle's reverse-mode gradient.

Each test prints the largest errors it saw (run pytest with -rP to see them).
Tolerances: 2e-6 rad for the phase screen (it enters the 2e-4 intensity bound
through |dI| ~ 2|A| |dphi|), 2e-4 absolute for intensities and curves, 1e-4
relative for m, 1e-4 of max |dL/dphi| for the gradient and 1e-3 relative for
dL/dR_diff.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import workloads as W
from conftest import gpu_params, oracle_params

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

PHI_TOL = 2e-6
I_TOL = 2e-4
M_TOL = 1e-4
G_TOL = 1e-4


@pytest.fixture(autouse=True, scope="module")
def _oracle_threads():
    """The oracle's 2D transforms at 4096^2 and 16384^2 on every host core."""
    old = O.FFT_WORKERS
    O.FFT_WORKERS = os.cpu_count() or 1
    yield
    O.FFT_WORKERS = old


def _forward_parity(it, label):
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi_g = S.make_screen(p_g)
    phi_o = O.make_screen(p_o)
    e_phi = float(np.abs(phi_g.cpu().numpy() - phi_o).max())
    phi_rms = float(np.sqrt(np.mean(phi_o ** 2)))
    I_g = S.propagate(p_g, phi_g)
    I_o = O.intensity_mono(phi_o, p_o)
    if p_o.source_radius_km > 0.0:
        S.smooth_source(p_g, I_g)
        I_o = O.smooth_source(I_o, p_o.pixel_km, p_o.source_radius_km)
    e_I = float(np.abs(I_g.cpu().numpy() - I_o).max())
    c_g = S.lightcurve(p_g, I_g, it["tracks"], it["n_samples"]).cpu().numpy()
    c_o = O.lightcurves(I_o, it["tracks"], it["n_samples"])
    e_c = float(np.abs(c_g - c_o).max())
    m_g = float(S.modulation_index(p_g, I_g).cpu().numpy()[0])
    m_o = O.modulation_index_map(I_o, p_o)
    cm_g = S.curve_modulation(torch.from_numpy(c_g).cuda()).cpu().numpy()[:, 0]
    cm_o = np.array([O.modulation_index(c) for c in c_o])
    e_m = abs(m_g - m_o) / m_o
    e_cm = float(np.max(np.abs(cm_g - cm_o) / cm_o))
    print(f"{label}: phi rms {phi_rms:.3g} rad, max |phi| {np.abs(phi_o).max():.4g} rad, phi err {e_phi:.3e} rad; "
          f"I max {I_o.max():.4g}, I err {e_I:.3e}; curve err {e_c:.3e}; m {m_o:.6f} rel err {e_m:.2e}; "
          f"curve m rel err {e_cm:.2e}")
    assert e_phi <= PHI_TOL
    assert e_I <= I_TOL
    assert e_c <= I_TOL
    assert e_m <= M_TOL
    assert e_cm <= M_TOL


@pytest.mark.parametrize("r_diff", [30.0, 100.0, 300.0])
def test_single_screen_4096_whole_map(r_diff):
    """4096^2, R_diff in {30, 100, 300} km: the R_diff = 30 km screen has phases of ~60 rad rms."""
    it = W.single_screens_4096(r_diffs=(30.0, 100.0, 300.0))[(30.0, 100.0, 300.0).index(r_diff)]
    _forward_parity(it, f"4096^2 R_diff {r_diff:g} km")


def test_screen_8192_whole_map():
    """8192^2, 5 km pixels, Kolmogorov, a disk of one R_ref: the largest unsplit lines (one
    512-thread block per line in every pass), used by the modulation-index sweeps."""
    it = W.large_screen_16384(beta=11.0 / 3.0, disk=True, n=8192)
    _forward_parity(it, "8192^2 Kolmogorov disk")


@pytest.mark.parametrize("beta,disk", [(3.67, True), (3.3, False)])
def test_large_screen_16384_whole_map(beta, disk):
    """16384^2, 5 km pixels (the lines split over two-block clusters), beta = 3.67 with a disk of
    one R_ref and beta = 3.3 (the largest phase variance of the three indices) with a point source."""
    it = W.large_screen_16384(beta=beta, disk=disk)
    _forward_parity(it, f"16384^2 beta {beta:g} {'disk' if disk else 'point'}")


def test_gradient_16384_vs_oracle():
    """dL/dphi and dL/dR_diff at 16384^2 (split adjoint passes), two wavelengths, disk source,
    16 curves of 8192 samples, L = mean (c - 0)^2: GPU adjoint vs the oracle's reverse mode on the
    oracle's own screen."""
    it = W.large_screen_16384(beta=3.67, disk=True)
    p_g, p_o = gpu_params(it), oracle_params(it)
    lams = np.array([480.0, 520.0])
    tracks, ns = it["tracks"], 8192
    phi = O.make_screen(p_o)
    target = np.zeros((len(tracks), ns))
    _, g_o, gr_o, c_o = O.misfit_gradient(p_o, phi, lams, tracks, ns, target, return_curves=True)
    gc = 2.0 * (c_o - target) / c_o.size
    phi_t = torch.from_numpy(phi).cuda()
    g_g = S.lightcurve_adjoint(p_g, phi_t, lams, tracks, ns, torch.from_numpy(gc.astype(np.float32)).cuda())
    scale = float(np.abs(g_o).max())
    e_g = float(np.abs(g_g.cpu().numpy() - g_o).max())
    gr = S.rdiff_gradient(p_g, phi_t, g_g).item()
    print(f"16384^2 gradient: max |dL/dphi| {scale:.3e}, err {e_g:.3e} ({e_g / scale:.2e} of max); "
          f"dL/dR_diff {gr_o:.6e}, rel err {abs(gr - gr_o) / abs(gr_o):.2e}")
    assert e_g <= G_TOL * scale
    assert gr == pytest.approx(gr_o, rel=1e-3)
