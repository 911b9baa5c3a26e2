"""Pins of the oracle's modulation-index sweep quantities (Sect. 4.1).

Eq. xparam is printed twice: as radius ratios and as a numerical formula with a
coefficient 0.035.  The ratio form, with R_F and R_ref as the oracle defines them
(pinned against the paper's worked radii in test_oracle_noise.py), must reproduce
that coefficient and the formula's exponents; N_R = d^2/R_ref^2 is checked on a
geometry worked out by hand.
"""
import math

import numpy as np
import pytest

import oracle as O

KPC_PC = 1000.0


def _rs_km(r_s_rsun, z0_pc, z1_pc):
    """Projected source radius R_s = r_s z0 / z1 (Eq. iprh)."""
    return r_s_rsun * O.R_SUN_KM * z0_pc / z1_pc


def test_xparam_forms_agree_with_printed_coefficient(golden):
    vals = {r[0]: (float(r[1]), float(r[2])) for r in golden("paper_worked_numbers.txt")}
    coef, tol = vals["xparam_coefficient"]
    # lambda = 1 um, z0 = 1 kpc, R_diff = 1000 km, r_s / z1 = R_sun / 10 kpc
    m = O.xparam_m(1000.0, 1000.0, KPC_PC, _rs_km(1.0, KPC_PC, 10 * KPC_PC))
    assert m == pytest.approx(coef, rel=tol)


def test_xparam_exponents():
    rng = np.random.default_rng(3)
    base = O.xparam_m(1000.0, 1000.0, KPC_PC, _rs_km(1.0, KPC_PC, 10 * KPC_PC))
    for _ in range(20):
        lam = rng.uniform(400.0, 2500.0)
        z0 = rng.uniform(30.0, 2000.0)
        z1 = rng.uniform(5000.0, 60000.0)
        rd = rng.uniform(30.0, 3000.0)
        rs = rng.uniform(0.2, 3.0)
        ratio = O.xparam_m(rd, lam, z0, _rs_km(rs, z0, z1))
        x = (rs / z1) / (1.0 / (10 * KPC_PC))
        numeric = O.xparam_m_numeric(rd, lam, z0, x, coefficient=base)
        assert ratio == pytest.approx(numeric, rel=1e-12)


def test_refractive_regions_geometry():
    # L = 1024 x 100 km; taper margin 5000 km, R_ref at 500 nm, z 160 pc, R_diff 100 km = 24686 km,
    # R_s = 0: fiducial margin 5000 + 12343 km, zone from 17343 to 85057 km (pixel centres)
    p = O.ScreenParams(n=1024, pixel_km=100.0, r_diff_km=100.0, lambda_nm=500.0, lambda_ref_nm=500.0,
                       margin_km=5000.0)
    r_ref = O.refraction_radius_km(p, 500.0)
    assert r_ref == pytest.approx(500e-12 * 160 * 3.0856775814913673e13 / 100.0, rel=1e-12)
    m = 5000.0 + r_ref / 2
    first = math.ceil(m / 100.0 - 0.5)
    last = math.floor((102400.0 - m) / 100.0 - 0.5)
    d = (last - first + 1) * 100.0
    assert O.refractive_regions(p) == pytest.approx(d * d / r_ref ** 2, rel=1e-12)
    # a zone that does not exist holds no regions
    assert O.refractive_regions(p.with_(source_radius_km=60000.0)) == 0.0
