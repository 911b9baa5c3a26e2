"""scint_propagate_noalloc: propagation for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc, nor hand the library a workspace: hosts
that forbid device allocation once running, or plugins inside a framework that
owns all device memory.  scint_propagate_noalloc serves them from a static
device array inside the library (n <= 1024).  These tests call it through the
C ABI and check it against scint_propagate, the entry point that takes a
workspace, on two calls in a row (so stale scratch from the first call cannot
leak into the second), plus the size limit.  They create every input
themselves, so they pass alone in a fresh process as well as after the rest of
the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1301_0514_gb300 as S

pytestmark = pytest.mark.gpu

I_TOL = 2e-4      # the intensity tolerance used by the parity tests


def _noalloc(p, phi, out):
    lib = S.lib()
    stream = torch.cuda.current_stream().cuda_stream
    return lib.scint_propagate_noalloc(ctypes.byref(p), ctypes.c_void_p(phi.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_noalloc_matches_propagate_on_two_calls_in_a_row():
    cases = [S.params(n=1024, pixel_km=10.0, r_diff_km=40.0, lambda_nm=620.0, lambda_ref_nm=550.0, seed=11),
             S.params(n=256, pixel_km=20.0, r_diff_km=100.0, seed=12, margin_km=0.0)]
    outs = []
    for p in cases:
        phi = S.make_screen(p)
        ref = S.propagate(p, phi)
        out = torch.full((p.n, p.n), float("nan"), dtype=torch.float32, device="cuda")
        rc = _noalloc(p, phi, out)
        assert rc == 0, S.lib().scint_last_error().decode()
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= I_TOL, err
        outs.append(out)
    # the first result is unchanged by the second call (outputs are the caller's)
    p = cases[0]
    again = S.propagate(p, S.make_screen(p))
    assert (outs[0] - again).abs().max().item() <= I_TOL


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    p = S.params(n=2048, pixel_km=10.0, r_diff_km=40.0)
    phi = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    rc = _noalloc(p, phi, out)
    assert rc == 1
    assert "static scratch limit" in S.lib().scint_last_error().decode()
