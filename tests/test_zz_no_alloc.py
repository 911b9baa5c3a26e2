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
    """Both entry points run the same kernels on the same inputs, and the no-allocation one fills
    its twiddle table with the same kernel as the table the other keeps: the maps are identical
    bit for bit, on each of two calls in a row (stale scratch from the first call cannot leak
    into the second)."""
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
        assert torch.equal(out, ref), (out - ref).abs().max().item()
        assert (out - ref).abs().max().item() <= I_TOL
        outs.append(out)
    # the first result is unchanged by the second call (outputs are the caller's)
    p = cases[0]
    again = S.propagate(p, S.make_screen(p))
    assert torch.equal(outs[0], again)


def test_noalloc_allocates_no_device_memory():
    """With the library's pool and kept tables released (scint_release), a call takes no device
    memory: free memory is the same before and after it (the pool or a twiddle table at
    n = 1024 would take at least 8 MiB).  One call first loads the kernels, whose code also
    occupies device memory."""
    p = S.params(n=1024, pixel_km=10.0, r_diff_km=40.0, seed=13)
    phi = S.make_screen(p)
    ref = S.propagate(p, phi)
    out = torch.empty((p.n, p.n), dtype=torch.float32, device="cuda")
    assert _noalloc(p, phi, out) == 0
    torch.cuda.synchronize()
    S.lib().scint_release()
    free0, _ = torch.cuda.mem_get_info()
    out.fill_(float("nan"))
    assert _noalloc(p, phi, out) == 0, S.lib().scint_last_error().decode()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0 - free1)
    assert torch.equal(out, ref)


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    p = S.params(n=2048, pixel_km=10.0, r_diff_km=40.0)
    phi = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    rc = _noalloc(p, phi, out)
    assert rc == 1
    assert "static scratch limit" in S.lib().scint_last_error().decode()
