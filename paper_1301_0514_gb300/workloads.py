"""Seeded synthetic workloads shaped like the paper's simulations.

Plain parameter records only: this module draws the random configuration
choices (diffraction radii, source sizes, track placements) and holds none of
the method's arithmetic.  Tests, the bench and the CPU baseline all take their
inputs from here, so the CUDA path and the oracle see identical inputs.

The shapes follow the paper's workloads (Sect. 3, Figs. 3-5): strong
scintillation (R_diff < R_F), z0 = 160 pc, Kolmogorov and non-Kolmogorov
screens, point and extended sources, optical/NIR passbands, long straight
tracks.  Seeds are 20130514 + 1000 * k + item, k = 1..5 for the five workloads below in order.
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

KM_PER_PC = 3.0856775814913673e13
KM_PER_NM = 1.0e-12
SEED_BASE = 20130514


def _item(n, pixel_km, r_diff_km, lambda_nm=500.0, lambda_ref_nm=None, beta=11.0 / 3.0, z_pc=160.0,
          source_radius_km=0.0, seed=0, screen_id=0, margin_km=-1.0, tracks=None, n_samples=0,
          lambdas_nm=None, weights=None) -> Dict:
    return dict(n=int(n), pixel_km=float(pixel_km), r_diff_km=float(r_diff_km), beta=float(beta),
                lambda_nm=float(lambda_nm), lambda_ref_nm=float(lambda_nm if lambda_ref_nm is None else lambda_ref_nm),
                z_pc=float(z_pc), source_radius_km=float(source_radius_km), seed=int(seed),
                screen_id=int(screen_id), margin_km=float(margin_km),
                tracks=np.zeros((0, 4)) if tracks is None else np.asarray(tracks, dtype=np.float64),
                n_samples=int(n_samples),
                lambdas_nm=np.array([float(lambda_nm)]) if lambdas_nm is None
                else np.asarray(lambdas_nm, dtype=np.float64),
                weights=None if weights is None else np.asarray(weights, dtype=np.float64))


def random_tracks(rng: np.random.Generator, n: int, count: int, ds: float) -> np.ndarray:
    """Straight tracks: start uniform on the map, angle uniform in [0, pi), step ds pixels."""
    x0 = rng.uniform(0.0, n, count)
    y0 = rng.uniform(0.0, n, count)
    th = rng.uniform(0.0, math.pi, count)
    return np.stack([x0, y0, th, np.full(count, ds)], axis=1)


def small_screen_256() -> List[Dict]:
    """256^2 Kolmogorov screen, 20 km pixels, R_diff = 100 km, 500 nm, 160 pc, point source,
    one horizontal track through row 128 (1 px steps, 256 samples)."""
    return [_item(256, 20.0, 100.0, seed=SEED_BASE + 1000, tracks=[(0.0, 128.0, 0.0, 1.0)], n_samples=256)]


def single_screens_4096(r_diffs=(30.0, 100.0, 300.0), n: int = 4096) -> List[Dict]:
    """4096^2 screens, 10 km pixels, R_diff in {30, 100, 300} km, 500 nm, point source,
    64 tracks at random angles (1 px steps, 2048 samples)."""
    out = []
    for i, rd in enumerate(r_diffs):
        rng = np.random.default_rng(SEED_BASE + 2000 + i)
        out.append(_item(n, 10.0, rd, seed=SEED_BASE + 2000 + i, screen_id=i,
                         tracks=random_tracks(rng, n, 64, 1.0), n_samples=n // 2))
    return out


def passband_400_700(count: int = 32) -> np.ndarray:
    return np.linspace(400.0, 700.0, count)


def batched_polychromatic(sizes=(1024, 2048, 4096), per_size: int = 16, n_lambda: int = 32, tracks_per_screen: int = 8) -> List[Dict]:
    """Batched polychromatic extended sources: per_size screens of each size, 10 km pixels,
    R_diff ~ U[30, 300] km at lambda_ref = 550 nm, 32 wavelengths in 400-700 nm (flat),
    projected disk radius ~ U[0.1, 2] x R_ref(lambda_ref), R_ref = lambda_ref z / R_diff."""
    rng = np.random.default_rng(SEED_BASE + 3000)
    lams = passband_400_700(n_lambda)
    out = []
    k = 0
    for n in sizes:
        for j in range(per_size):
            rd = rng.uniform(30.0, 300.0)
            r_ref = 550.0 * KM_PER_NM * 160.0 * KM_PER_PC / rd
            rs = rng.uniform(0.1, 2.0) * r_ref
            out.append(_item(n, 10.0, rd, lambda_nm=550.0, lambda_ref_nm=550.0, source_radius_km=rs,
                             seed=SEED_BASE + 3000 + k, screen_id=k,
                             tracks=random_tracks(rng, n, tracks_per_screen, 1.0), n_samples=n // 2,
                             lambdas_nm=lams))
            k += 1
    return out


def large_screen_16384(beta: float, disk: bool, n: int = 16384) -> Dict:
    """16384^2 screen, 5 km pixels, R_diff = 100 km, non-Kolmogorov beta, 500 nm; point source
    or a disk of one R_ref = lambda z / R_diff."""
    r_ref = 500.0 * KM_PER_NM * 160.0 * KM_PER_PC / 100.0
    rng = np.random.default_rng(SEED_BASE + 4000)
    return _item(n, 5.0, 100.0, beta=beta, source_radius_km=r_ref if disk else 0.0,
                 seed=SEED_BASE + 4000 + int(round(beta * 100)), tracks=random_tracks(rng, n, 16, 1.0),
                 n_samples=n // 2)


def gradient_batch_2048(batch: int = 8, n: int = 2048) -> List[Dict]:
    """Differentiation: batch of 2048^2 screens, R_diff = 100 km, 500 nm; one track of 10^4
    samples at 0.2 px steps; the target curve comes from the screen of seed + 500."""
    out = []
    for b in range(batch):
        rng = np.random.default_rng(SEED_BASE + 5000 + b)
        out.append(_item(n, 10.0, 100.0, seed=SEED_BASE + 5000 + b, screen_id=b,
                         tracks=random_tracks(rng, n, 1, 0.2), n_samples=10000))
    return out
