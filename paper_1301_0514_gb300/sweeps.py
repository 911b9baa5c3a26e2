"""Modulation-index sweeps of Sect. 4.1 through the batched path.

The paper checks Eq. xparam,
    m ~ (R_diff / R_F)^(1/3) (R_ref / (2 pi R_s))^(7/6),
with series of screens, R_diff = 50..500 km in steps of 50 km, seen through
sources of radius r_s = 0.25..1.5 R_sun in steps of 0.25 at fixed distances, m
measured over each pattern's fiducial zone; patterns with fewer than five
R_ref-size regions in the zone (N_R = d^2 / R_ref^2 < 5) are discarded, and the
rest are grouped by the predicted m.  Sect. 5 repeats this for beta = 3.1 and
3.9.  Here every pattern is one item of scint_run_batch (synthesis, K_s
passband, disk, m over the fiducial zone, all on the GPU); this module only
lays out the configurations and tabulates the results.  Eq. xparam is host
arithmetic on scalars: the prediction the simulations are compared with.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib

R_SUN_KM = 695700.0
KM_PER_PC = 3.0856775814913673e13
KM_PER_NM = 1.0e-12
# K_s passband of Sect. 3.2.4: 21 wavelengths over [2.08, 2.28] um around 2.162 um
KS_BAND_NM = np.linspace(2080.0, 2280.0, 21)
KS_CENTRE_NM = 2162.0


def xparam_m(r_diff_km: float, lambda_nm: float, z0_pc: float, source_radius_km: float) -> float:
    """Eq. xparam: (R_diff/R_F)^(1/3) (R_ref/(2 pi R_s))^(7/6), R_F^2 = lambda z0 / 2 pi,
    R_ref = lambda z0 / R_diff."""
    lz = lambda_nm * KM_PER_NM * z0_pc * KM_PER_PC
    return ((r_diff_km / math.sqrt(lz / (2.0 * math.pi))) ** (1.0 / 3.0)
            * (lz / r_diff_km / (2.0 * math.pi * source_radius_km)) ** (7.0 / 6.0))


@dataclass
class SweepPoint:
    r_diff_km: float
    r_s_rsun: float
    beta: float
    params: _lib.ScintParams
    m_theory: float          # Eq. xparam
    n_regions: float         # N_R = d^2 / R_ref^2 of the fiducial zone (0 if empty)


def sweep_points(r_diffs: Sequence[float] = tuple(range(50, 501, 50)),
                 radii_rsun: Sequence[float] = (0.25, 0.5, 0.75, 1.0, 1.25, 1.5),
                 betas: Sequence[float] = (11.0 / 3.0,), n: int = 8192, pixels_per_rdiff: float = 3.0,
                 lambda_nm: float = KS_CENTRE_NM, z0_pc: float = 160.0, z1_pc: float = 1000.0,
                 seed: int = 20130514 + 9500) -> List[SweepPoint]:
    """One screen per (R_diff, r_s, beta): pixel R_diff / pixels_per_rdiff (the paper's
    Delta < R_diff / 2), source projected to R_s = r_s z0 / z1 (Eq. iprh)."""
    pts = []
    k = 0
    for beta in betas:
        for rd in r_diffs:
            for rs in radii_rsun:
                p = _lib.params(n=n, pixel_km=rd / pixels_per_rdiff, r_diff_km=rd, beta=beta, lambda_nm=lambda_nm,
                                lambda_ref_nm=lambda_nm, z_pc=z0_pc, source_radius_km=rs * R_SUN_KM * z0_pc / z1_pc,
                                seed=seed + k, screen_id=k)
                i0, i1, r_ref, exists = _lib.fiducial_zone(p)
                d = (i1 - i0) * p.pixel_km
                pts.append(SweepPoint(rd, rs, beta, p, xparam_m(rd, lambda_nm, z0_pc, p.source_radius_km),
                                      d * d / (r_ref * r_ref) if exists else 0.0))
                k += 1
    return pts


def run_m_sweep(points: Sequence[SweepPoint], lambdas_nm=KS_BAND_NM, n_lanes: int = 2,
                workspace: Optional[torch.Tensor] = None, device="cuda", stream=None) -> torch.Tensor:
    """m over the fiducial zone of every point's pattern (device tensor, rows (m, mean,
    sigma, count)), one scint_run_batch call; the maps live in lane scratch."""
    m = torch.empty((len(points), 4), dtype=torch.float64, device=device)
    items = [dict(params=pt.params, m_map=m[i]) for i, pt in enumerate(points)]
    _lib.run_batch(items, lambdas_nm, n_lanes=n_lanes, workspace=workspace, stream=stream)
    return m


def summarize(points: Sequence[SweepPoint], m_sim, min_regions: float = 5.0, bins=None):
    """Keep the patterns with N_R >= min_regions and group them by predicted m (log bins):
    rows (m_theory centre, mean m, rms of m, count), as in the paper's comparison."""
    m_sim = np.asarray(m_sim, dtype=np.float64)
    th = np.array([pt.m_theory for pt in points])
    keep = np.array([pt.n_regions >= min_regions for pt in points])
    if bins is None:
        bins = np.geomspace(0.004, 0.6, 13)
    rows = []
    for lo, hi in zip(bins[:-1], bins[1:]):
        sel = keep & (th >= lo) & (th < hi)
        if sel.any():
            v = m_sim[sel]
            rows.append((float(np.sqrt(lo * hi)), float(v.mean()), float(v.std()), int(sel.sum())))
    return rows
