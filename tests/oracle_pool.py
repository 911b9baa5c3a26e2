"""Test infrastructure: the oracle's direct screen sums split over a spawn-started process pool.

Each worker evaluates, for a block of spectral rows, the partial sums
sum_{ky in block} sum_kx F[ky, kx] exp(2 pi i (kx x + ky y) / N) at the sample
pixels; the parent adds the blocks.  Only oracle code runs in the workers.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _block(args):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    pdict, r0, r1, ys, xs = args
    p = O.ScreenParams(**pdict)
    n = p.n
    rows = np.arange(r0, r1)
    F = O.noise_spectrum(p, rows=rows)
    ex = np.exp(2j * np.pi * np.outer(np.arange(n), xs) / n)
    inner = F @ ex
    return np.sum(inner * np.exp(2j * np.pi * np.outer(rows, ys) / n), axis=0)


def screen_pixels_direct(p, pix, block=256, workers=None):
    """phi at pixels [(y, x), ...] = sqrt(2)/L^2 Re sum_k F_k e^{+2 pi i k.x/N}, over all bins."""
    from dataclasses import asdict
    n = p.n
    L = n * p.pixel_km
    ys = np.array([q[0] for q in pix])
    xs = np.array([q[1] for q in pix])
    jobs = [(asdict(p), r0, min(n, r0 + block), ys, xs) for r0 in range(0, n, block)]
    workers = workers or min(32, os.cpu_count() or 1)
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        acc = sum(ex.map(_block, jobs))
    return np.sqrt(2.0) / (L * L) * np.real(acc)
