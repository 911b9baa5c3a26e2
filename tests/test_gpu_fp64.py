"""The plain method in FP64 on the GPU (scint_propagate64) against the FP64 oracle.

The small-screen workload (256^2 Kolmogorov screen, 20 km pixels, R_diff = 100 km,
500 nm, 160 pc, point source, taper margin clamped to L/4, one horizontal track
through row 128) runs every step in double precision on both sides, so the maps
agree to FP64 rounding: two 256-point line transforms per axis (relative error
~1e-15 each), FP64 sines and cosines of the screen phase (|phi| < 60 rad here,
absolute error ~1e-14) and an exactly reduced chirp.  The bound 1e-10 leaves four
orders of margin above that; a dropped taper factor, a wrong sign of H or a missed
normalisation fails it by many orders.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import workloads as W
from conftest import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def test_small_screen_256_fp64_map_and_track():
    it = W.small_screen_256()[0]
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi = O.make_screen(p_o)
    I_o = O.intensity_mono(phi, p_o)
    I_g = S.propagate64(p_g, torch.from_numpy(phi).cuda()).cpu().numpy()
    err = np.abs(I_g - I_o).max()
    print(f"256^2 FP64 plain method: max |I| {I_o.max():.4g}, max abs err {err:.3e}")
    assert err <= TOL64
    # the horizontal track samples integer positions: the curve is row 128 of the map
    c_o = O.lightcurves(I_o, it["tracks"], it["n_samples"])[0]
    assert np.abs(I_g[128, :] - c_o).max() <= TOL64
    # the FP32 path agrees at its own tolerance
    I_32 = S.propagate(p_g, torch.from_numpy(phi).cuda()).cpu().numpy()
    assert np.abs(I_32 - I_g).max() <= 2e-4


@pytest.mark.parametrize("n,pix,rd,lam,lam_ref,margin", [(16, 40.0, 100.0, 500.0, 500.0, -1.0),
                                                          (128, 20.0, 60.0, 620.0, 550.0, 0.0),
                                                          (1024, 10.0, 40.0, 450.0, 550.0, -1.0),
                                                          (4096, 10.0, 100.0, 500.0, 500.0, -1.0)])
def test_fp64_path_sizes_scales_and_tapers(n, pix, rd, lam, lam_ref, margin):
    it = W._item(n, pix, rd, lambda_nm=lam, lambda_ref_nm=lam_ref, margin_km=margin, seed=W.SEED_BASE + 61 + n)
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi = O.make_screen(p_o)
    I_o = O.intensity_mono(phi, p_o)
    I_g = S.propagate64(p_g, torch.from_numpy(phi).cuda()).cpu().numpy()
    assert np.abs(I_g - I_o).max() <= TOL64 * max(1.0, np.abs(I_o).max() / 10.0)


def test_fp64_chirp_reduction_is_exact_for_large_lambda_z():
    """z = 10 kpc (lambda z / 2 L^2 >> 1): the split chirp constant still gives the oracle's map."""
    it = W._item(256, 20.0, 100.0, z_pc=10000.0, margin_km=0.0, seed=W.SEED_BASE + 62)
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi = O.make_screen(p_o)
    I_o = O.intensity_mono(phi, p_o)
    I_g = S.propagate64(p_g, torch.from_numpy(phi).cuda()).cpu().numpy()
    assert np.abs(I_g - I_o).max() <= TOL64


def test_small_screen_256_whole_configuration_in_fp64():
    """Synthesis (every bin drawn in FP64 up to 512^2; double-float transform) and the FP64
    propagation against the oracle's screen and map: phase ~1e-12 rad, map ~1e-10."""
    it = W.small_screen_256()[0]
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi_g = S.make_screen(p_g)
    phi_o = O.make_screen(p_o)
    e_phi = np.abs(phi_g.cpu().numpy() - phi_o).max()
    I_g = S.propagate64(p_g, phi_g).cpu().numpy()
    e_I = np.abs(I_g - O.intensity_mono(phi_o, p_o)).max()
    print(f"256^2 whole configuration: phase err {e_phi:.3e} rad, map err {e_I:.3e}")
    assert e_phi <= 1e-11
    assert e_I <= TOL64


def test_fp64_path_rejects_grids_above_4096():
    p = S.params(n=8192, pixel_km=10.0, r_diff_km=100.0)
    phi = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        S.propagate64(p, phi)      # the binding checks the tensor size first
    out = torch.empty((1,), dtype=torch.float64, device="cuda")
    import ctypes
    rc = S.lib().scint_propagate64(ctypes.byref(p), ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   None, 0, None)
    assert rc == 5 and "4096" in S.lib().scint_last_error().decode()
