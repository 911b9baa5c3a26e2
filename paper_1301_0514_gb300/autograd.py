"""Differentiable screen synthesis and light curves (torch.autograd on the library's kernels).

screen(p, r_diff)            phi as a function of R_diff at a fixed seed; backward
                             gives dL/dR_diff = ((2 - beta)/(2 R_diff)) sum phi dL/dphi.
light_curves(phi, p, ...)    curves = lightcurve(smooth_source(sum_passband(phi)));
                             backward runs scint_lightcurve_adjoint (recomputes the
                             forward fields instead of storing them).
Both forward and backward run in libscint.so; torch only carries the tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


class _Screen(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r_diff, p, workspace):
        q = p.replace(r_diff_km=float(r_diff))
        phi = L.make_screen(q, workspace=workspace)
        ctx.save_for_backward(phi)
        ctx.q, ctx.ws = q, workspace
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        (phi,) = ctx.saved_tensors
        g = L.rdiff_gradient(ctx.q, phi, grad_phi.contiguous().to(torch.float64), workspace=ctx.ws)
        return g.reshape(()).to(device="cpu", dtype=torch.float64), None, None


class _Curves(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, p, lambdas, weights, tracks, n_samples, workspace):
        inten = L.sum_passband(p, phi, lambdas, weights, workspace=workspace)
        if p.source_radius_km > 0.0:
            L.smooth_source(p, inten, workspace=workspace)
        curves = L.lightcurve(p, inten, tracks, n_samples)
        ctx.save_for_backward(phi)
        ctx.args = (p, lambdas, weights, tracks, n_samples, workspace)
        return curves

    @staticmethod
    def backward(ctx, grad_curves):
        (phi,) = ctx.saved_tensors
        p, lambdas, weights, tracks, n_samples, ws = ctx.args
        g = L.lightcurve_adjoint(p, phi, lambdas, tracks, n_samples,
                                 grad_curves.contiguous().to(torch.float32), weights=weights, workspace=ws)
        return g, None, None, None, None, None, None


def screen(p: L.ScintParams, r_diff=None, workspace=None) -> torch.Tensor:
    """Phase screen (N x N float64 on the GPU); differentiable w.r.t. r_diff (a CPU scalar tensor)."""
    if r_diff is None:
        r_diff = torch.tensor(p.r_diff_km, dtype=torch.float64)
    return _Screen.apply(r_diff, p, workspace)


def light_curves(phi: torch.Tensor, p: L.ScintParams, lambdas_nm, tracks, n_samples: int, weights=None,
                 workspace=None) -> torch.Tensor:
    """Light curves (n_tracks x n_samples float32); differentiable w.r.t. phi."""
    lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
    if workspace is None:
        workspace = torch.empty(L.workspace_bytes(p, len(lam)), dtype=torch.uint8, device=phi.device)
    return _Curves.apply(phi, p, lam, weights, np.ascontiguousarray(tracks, dtype=np.float64), n_samples,
                         workspace)
