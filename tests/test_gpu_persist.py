"""The persistent batch kernel (scint_batch_mode 1): one launch propagates every screen.

Checked against the lanes form and the single-screen calls bit for bit (same pass
bodies, same arguments), inside a CUDA graph, and through its failure path: a host
knob withholds one row count so that the waits for that screen cannot succeed; every
wait is bounded, so the launch ends early with SCINT_ETIMEOUT in its status word and
nothing hangs or faults.
"""
import numpy as np
import pytest
import torch

import paper_1301_0514_gb300 as S

pytestmark = pytest.mark.gpu

LAMS = [470.0, 520.0, 560.0, 610.0, 660.0]


def _entries(sizes=(512, 256, 1024, 256, 2048, 512), seed=70):
    out = []
    for i, n in enumerate(sizes):
        kw = dict(n=n, pixel_km=10.0, r_diff_km=45.0 + 20 * i, lambda_nm=560.0, lambda_ref_nm=560.0,
                  source_radius_km=3000.0 * (i % 2), seed=seed + i, screen_id=i)
        tracks = np.array([[1.5, 2.25, 0.3, 0.9], [n / 3, n / 5, 2.0, 1.0]])
        out.append(dict(params=S.params(**kw), phi=torch.empty((n, n), dtype=torch.float64, device="cuda"),
                        intensity=torch.empty((n, n), device="cuda"), tracks=tracks, n_samples=n // 2,
                        curves=torch.empty((2, n // 2), device="cuda"),
                        m_map=torch.empty(4, dtype=torch.float64, device="cuda"),
                        m_curves=torch.empty((2, 3), dtype=torch.float64, device="cuda")))
    return out


def _unpacked(sizes):
    for n in set(sizes):
        S.set_plan(n, 0)


def _copy(entries):
    return [{k: (v.clone() if isinstance(v, torch.Tensor) else v) for k, v in e.items() if k in
             ("phi", "intensity", "curves", "m_map", "m_curves")} for e in entries]


@pytest.fixture
def persistent():
    old = S.batch_mode(1)
    yield
    S.batch_mode(old)
    S.lib().scint_testing_persist(-1, 0)


def test_persistent_equals_lanes_and_single_calls(persistent):
    entries = _entries()
    _unpacked([e["params"].n for e in entries])
    S.run_batch(entries, LAMS, n_lanes=3)
    S.batch_status()
    got = _copy(entries)
    S.batch_mode(0)
    S.run_batch(entries, LAMS, n_lanes=3)
    torch.cuda.synchronize()
    for g, e in zip(got, entries):
        for k in g:
            assert torch.equal(g[k], e[k]), k
    for g, e in zip(got, entries):
        p = e["params"]
        ref = S.sum_passband(p, S.make_screen(p), LAMS)
        S.smooth_source(p, ref)
        assert torch.equal(ref, g["intensity"])


def test_persistent_batch_in_a_cuda_graph(persistent):
    entries = _entries(sizes=(1024, 512, 256, 512), seed=90)
    _unpacked([e["params"].n for e in entries])
    batch = S.batch_items(entries)
    ws = torch.empty(S.batch_workspace_bytes(batch, len(LAMS), 2), dtype=torch.uint8, device="cuda")
    S.run_batch(batch, LAMS, n_lanes=2, workspace=ws)          # outside capture first (tables, attributes)
    torch.cuda.synchronize()
    ref = _copy(entries)
    for e in entries:
        e["intensity"].zero_()
        e["curves"].zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.run_batch(batch, LAMS, n_lanes=2, workspace=ws)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    S.batch_status()
    for r, e in zip(ref, entries):
        assert torch.equal(r["intensity"], e["intensity"])
        assert torch.equal(r["curves"], e["curves"])


def test_persistent_wait_gives_up_with_etimeout(persistent):
    """Screen 1's row count is withheld: its column work and the screens queued behind its
    field slot cannot proceed; each wait gives up after a few thousand reads, the launch
    ends, and the status says SCINT_ETIMEOUT.  The next launch without the knob is complete."""
    entries = _entries(sizes=(256, 512, 256), seed=110)
    _unpacked([e["params"].n for e in entries])
    S.lib().scint_testing_persist(1, 2000)
    S.run_batch(entries, LAMS, n_lanes=2)
    with pytest.raises(S.ScintError) as err:
        S.batch_status()
    assert err.value.code == 4          # SCINT_ETIMEOUT
    S.lib().scint_testing_persist(-1, 0)
    S.run_batch(entries, LAMS, n_lanes=2)
    S.batch_status()
    for e in entries:
        p = e["params"]
        ref = S.sum_passband(p, S.make_screen(p), LAMS)
        S.smooth_source(p, ref)
        assert torch.equal(ref, e["intensity"])


def test_persistent_mode_falls_back_to_lanes(persistent):
    """A packed plan (or a size outside [256, 4096]) runs the batch on lanes: same results."""
    entries = _entries(sizes=(512, 256), seed=130)
    S.set_plan(512, 1, 2, 2, 16)
    S.set_plan(256, 0)
    try:
        S.run_batch(entries, LAMS, n_lanes=2)
        torch.cuda.synchronize()
        for e in entries:
            p = e["params"]
            ref = S.sum_passband(p, S.make_screen(p), LAMS)
            S.smooth_source(p, ref)
            assert torch.equal(ref, e["intensity"])
    finally:
        S.set_plan(512, 0)


def test_batch_mode_rejects_unknown_modes():
    with pytest.raises(S.ScintError):
        S.batch_mode(2)
