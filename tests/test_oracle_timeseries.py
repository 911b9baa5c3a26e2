"""Pins of the oracle's light-curve time analysis (Sect. 5).

Periodogram: a sinusoid with an integer number of cycles puts A^2 n / 4 in its
bin and nothing elsewhere; Parseval ties the bins to the variance.  Correlation:
+1 for affine copies, -1 for negated ones, 0 exactly for orthogonal sinusoids.
Parallel tracks: the offset is perpendicular to the track, of the given length.
"""
import math

import numpy as np
import pytest

import oracle as O


def test_periodogram_of_sinusoid_and_parseval():
    n, A, f0 = 256, 1.7, 9
    s = np.arange(n)
    c = 3.0 + A * np.cos(2 * np.pi * f0 * s / n + 0.4)
    P = O.periodogram(c)[0]
    assert P.shape == (n // 2 + 1,)
    assert P[f0] == pytest.approx(A * A * n / 4, rel=1e-12)
    assert np.delete(P, f0).max() < 1e-20 * P[f0] + 1e-18
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n)
    Q = O.periodogram(x)[0]
    # sum over the two-sided spectrum = n * variance (population); one-sided: DC and Nyquist once
    two_sided = Q[0] + Q[n // 2] + 2 * Q[1:n // 2].sum()
    assert two_sided == pytest.approx(n * x.var(), rel=1e-12)
    assert Q[0] == pytest.approx(0.0, abs=1e-20)


def test_pearson():
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3, 500))
    assert O.pearson(a, 2.5 * a + 7.0) == pytest.approx(np.ones(3), rel=1e-14)
    assert O.pearson(a, -a) == pytest.approx(-np.ones(3), rel=1e-14)
    s = np.arange(400)
    u = np.cos(2 * np.pi * 3 * s / 400)
    v = np.sin(2 * np.pi * 5 * s / 400)
    assert abs(O.pearson(u, v)[0]) < 1e-14
    b = rng.standard_normal((3, 500))
    assert np.all(np.abs(O.pearson(a, b)) < 5.0 / math.sqrt(500))


def test_parallel_tracks_are_perpendicular_offsets():
    tr = (10.0, 20.0, 0.3, 0.8)
    sep = np.array([0.0, 5.0, 120.0])
    out = O.parallel_tracks(tr, sep)
    for row, d in zip(out, sep):
        dx, dy = row[0] - tr[0], row[1] - tr[1]
        assert math.hypot(dx, dy) == pytest.approx(d, abs=1e-12)
        assert dx * math.cos(tr[2]) + dy * math.sin(tr[2]) == pytest.approx(0.0, abs=1e-12)
        assert row[2] == tr[2] and row[3] == tr[3]
