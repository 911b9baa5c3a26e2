"""Light-curve time analysis of Sect. 5 on the GPU: time power spectra of light
curves and the decorrelation of two telescopes' curves with their separation.

The curves come from scint_lightcurve on an illumination map; their periodograms
(scint_curve_power_spectrum) show the slope break near 1/t_ref, and curves
along tracks offset perpendicularly by a distance D (two telescopes) decorrelate
(scint_curve_correlation) once D exceeds 2 max(R_ref, R_s).  This module only
lays out the tracks and calls the library.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np
import torch

from . import _lib


def parallel_tracks(track, separations_px: Sequence[float]) -> np.ndarray:
    """Tracks parallel to (x0, y0, theta, ds), offset by each separation (pixels)
    perpendicularly to the direction of motion."""
    x0, y0, th, ds = (float(v) for v in track)
    sep = np.asarray(separations_px, dtype=np.float64)
    return np.stack([x0 - sep * math.sin(th), y0 + sep * math.cos(th), np.full(sep.shape, th),
                     np.full(sep.shape, ds)], axis=1)


def decorrelation(p: _lib.ScintParams, intensity: torch.Tensor, tracks, separations_px: Sequence[float],
                  n_samples: int, stream=None) -> torch.Tensor:
    """Correlation of the curve along each base track with the curves along its parallels at
    each separation: a (n_tracks, n_separations) float64 device tensor."""
    base = np.asarray(tracks, dtype=np.float64).reshape(-1, 4)
    sep = np.asarray(separations_px, dtype=np.float64)
    all_tracks = np.concatenate([parallel_tracks(tr, sep) for tr in base], axis=0)
    curves = _lib.lightcurve(p, intensity, all_tracks, n_samples, stream=stream)
    # one launch: every curve against the first curve of its group (separation 0 first)
    r = _lib.curve_correlation(curves, curves, a_rows=len(base), a_stride=len(sep) * n_samples, stream=stream)
    return r.reshape(len(base), len(sep))


def power_spectra(curves: torch.Tensor, stream=None) -> torch.Tensor:
    """Periodograms of the curves (rows), mean removed: (n_curves, n/2 + 1) float32."""
    return _lib.curve_power_spectrum(curves.contiguous(), stream=stream)
