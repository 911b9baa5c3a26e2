"""N = 16384 (the large single-screen configuration): lines split over a two-block cluster.

At this size the oracle cannot run the whole map in seconds, so the checks are
(a) sampled outputs the oracle computes one by one, and (b) closed forms and
identities that hold at any size:
  * line FFTs vs numpy on whole 16384-point lines (FP32 and FP64);
  * screen pixels vs the oracle's direct double sum over all 2.7e8 bins;
  * sinusoidal phase gratings (along x, y and obliquely) vs the Jacobi-Anger closed form;
  * a two-wavelength passband split into groups and accumulated vs its single-wavelength maps;
  * cosine eigenfunctions of the disk filter (along x, y and obliquely) vs quadrature;
  * the full pipeline (beta in {3.3, 3.67, 3.9}, point and disk source):
    energy conservation of the periodic propagation (mean I = <SF^2>^2) and
    of the disk filter (mean preserved).
"""
import math

import numpy as np
import pytest
import torch
from scipy import integrate, special

import oracle as O
import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import workloads as W
from conftest import gpu_params, oracle_params
from oracle_pool import screen_pixels_direct

pytestmark = pytest.mark.gpu

N = 16384
I_TOL = 2e-4
PHI_TOL = 2e-6


@pytest.mark.parametrize("dtype,tol", [(torch.complex64, 2e-6), (torch.complex128, 1e-13)])
@pytest.mark.parametrize("direction", [-1, 1])
def test_fft_lines_16384(dtype, tol, direction):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, N)) + 1j * rng.standard_normal((3, N))
    t = torch.from_numpy(x).to(dtype).cuda()
    xin = t.cpu().numpy().astype(np.complex128)
    S.fft_lines(t, direction)
    ref = np.fft.fft(xin, axis=1) if direction < 0 else np.fft.ifft(xin, axis=1) * N
    err = np.linalg.norm(t.cpu().numpy() - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() < tol


def test_screen_16384_sampled_pixels():
    it = W.large_screen_16384(beta=3.67, disk=False)
    p_g, p_o = gpu_params(it), oracle_params(it)
    phi = S.make_screen(p_g)
    pix = [(0, 0), (1, 8191), (8192, 8192), (16383, 1), (5000, 12345), (12001, 777)]
    ref = screen_pixels_direct(p_o, pix)
    got = np.array([phi[y, x].item() for y, x in pix])
    assert np.abs(got - ref).max() <= PHI_TOL
    assert np.abs(ref).max() > 1.0


@pytest.mark.parametrize("fx,fy", [(64, 0), (0, 48), (40, -24)])
def test_grating_16384_closed_form(fx, fy):
    """phi = a sin(2 pi (fx x + fy y) / L) on 16384^2, untapered: Jacobi-Anger closed form
    (orders |m| <= 20); fy != 0 puts the column pass (its split radix-2 steps) to work."""
    pix_km, a, lam, lam_ref, z = 5.0, 1.7, 500.0, 550.0, 160.0
    L = N * pix_km
    c = (torch.arange(N, dtype=torch.float64, device="cuda") + 0.5) * pix_km
    phi = a * torch.sin(2.0 * np.pi * (fx * c[None, :] + fy * c[:, None]) / L)
    p = S.params(n=N, pixel_km=pix_km, r_diff_km=100.0, lambda_nm=lam, lambda_ref_nm=lam_ref, z_pc=z, margin_km=0.0)
    I = S.propagate(p, phi.contiguous())
    s = lam_ref / lam
    lz = lam * O.KM_PER_NM * z * O.KM_PER_PC
    k2 = (fx * fx + fy * fy) / L ** 2
    x = (np.arange(N) + 0.5) * pix_km
    for y in (0, 4097, 8192, 16383):
        u = 2.0 * np.pi * (fx * x + fy * x[y]) / L
        amp = sum(special.jv(m, a * s) * np.exp(1j * m * u) * np.exp(-1j * np.pi * lz * m * m * k2) for m in range(-20, 21))
        assert np.abs(I[y].cpu().numpy() - np.abs(amp) ** 2).max() <= I_TOL
    # a column as well (the transposed write of the column pass)
    xc = 12345
    u = 2.0 * np.pi * (fx * x[xc] + fy * x) / L
    amp = sum(special.jv(m, a * s) * np.exp(1j * m * u) * np.exp(-1j * np.pi * lz * m * m * k2) for m in range(-20, 21))
    assert np.abs(I[:, xc].cpu().numpy() - np.abs(amp) ** 2).max() <= I_TOL


def test_passband_16384_groups_accumulate():
    """Two wavelengths in two groups (the workspace holds one) added onto a prior map equal
    the weighted single-wavelength maps: the accumulating transposed write of the column pass."""
    it = W.large_screen_16384(beta=3.67, disk=False)
    p = gpu_params(it)
    phi = S.make_screen(p)
    lams, wts = (480.0, 530.0), (0.3, 0.7)
    ws = torch.empty(S.workspace_bytes(p, 1), dtype=torch.uint8, device="cuda")
    out = torch.full((N, N), 0.25, device="cuda")
    S.sum_passband(p, phi, lams, wts, out=out, accumulate=True, workspace=ws)
    want = 0.25 + wts[0] * S.sum_passband(p, phi, lams[:1], workspace=ws).double()
    want += wts[1] * S.sum_passband(p, phi, lams[1:], workspace=ws).double()
    for y in (0, 7, 8191, 8192, 16383):
        assert (out[y].double() - want[y]).abs().max().item() <= 1e-5


@pytest.mark.parametrize("mx,my", [(1, 0), (9, 0), (0, 7), (5, -3)])
def test_disk_filter_16384_eigenfunction(mx, my):
    """cos(2 pi (mx x + my y) / L) is an eigenfunction of the periodic disk filter with
    eigenvalue K(q) = 2 J1(2 pi q R)/(2 pi q R), q = |m|/L (K by quadrature here); my != 0
    puts the column passes (their split radix-2 steps) to work."""
    pix_km, R = 5.0, 24686.0
    L = N * pix_km
    c = (torch.arange(N, dtype=torch.float64, device="cuda") + 0.5) * pix_km
    I = (1.0 + 0.25 * torch.cos(2.0 * np.pi * (mx * c[None, :] + my * c[:, None]) / L)).float().contiguous()
    S.smooth_source(S.params(n=N, pixel_km=pix_km, r_diff_km=100.0, source_radius_km=R), I)
    u = 2.0 * np.pi * math.hypot(mx, my) / L * R
    K = integrate.quad(lambda t: 2.0 * math.sqrt(1 - t * t) * math.cos(u * t), -1, 1, limit=200)[0] / math.pi
    x = (np.arange(N) + 0.5) * pix_km
    for y in (0, 9000, 16383):
        ref = 1.0 + 0.25 * K * np.cos(2.0 * np.pi * (mx * x + my * x[y]) / L)
        assert np.abs(I[y].cpu().numpy() - ref).max() <= I_TOL
    ref = 1.0 + 0.25 * K * np.cos(2.0 * np.pi * (mx * x[4321] + my * x) / L)
    assert np.abs(I[:, 4321].cpu().numpy() - ref).max() <= I_TOL


@pytest.mark.parametrize("beta", [3.3, 3.67, 3.9])
@pytest.mark.parametrize("disk", [False, True])
def test_large_16384_pipeline_identities(beta, disk):
    it = W.large_screen_16384(beta=beta, disk=disk)
    p = gpu_params(it)
    phi = S.make_screen(p)
    I = S.propagate(p, phi)
    sf = O.taper_1d(N, p.pixel_km, O.taper_margin_km(oracle_params(it), p.lambda_nm))
    assert I.double().mean().item() == pytest.approx(np.mean(sf ** 2) ** 2, rel=1e-4)
    if disk:
        before = I.double().mean().item()
        S.smooth_source(p, I)
        assert I.double().mean().item() == pytest.approx(before, rel=1e-5)
    curves = S.lightcurve(p, I, it["tracks"], it["n_samples"])
    m = S.modulation_index(p, I).cpu().numpy()
    assert np.isfinite(curves.cpu().numpy()).all() and 0.0 < m[0] < 3.0
