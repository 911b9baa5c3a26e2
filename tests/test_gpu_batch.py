"""scint_run_batch: many screens on several lanes give exactly the single-screen results.

The batch executor only schedules the single-screen entry points on internal
streams, so with the same wavelength grouping its outputs are bit-identical to
theirs; one item is also checked against the FP64 oracle at the intensity
tolerance, and a captured graph of the batch replays to the same outputs.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import workloads as W
from conftest import gpu_params, oracle_params

pytestmark = pytest.mark.gpu

I_TOL = 2e-4
LAMS = np.array([480.0, 530.0, 610.0, 690.0])


def _items(sizes=(256, 64, 128, 256, 512, 128)):
    rng = np.random.default_rng(W.SEED_BASE + 7700)
    out = []
    for k, n in enumerate(sizes):
        rd = rng.uniform(30.0, 120.0)
        rs = 0.0 if k % 3 == 0 else rng.uniform(50.0, 300.0)
        out.append(W._item(n, 10.0, rd, lambda_nm=550.0, lambda_ref_nm=550.0, source_radius_km=rs,
                           seed=W.SEED_BASE + 7700 + k, screen_id=k,
                           tracks=W.random_tracks(rng, n, 3 + k, 0.7), n_samples=n // 2 + k, lambdas_nm=LAMS))
    return out


def _outputs(it, with_maps=True):
    n, nt, ns = it["n"], len(it["tracks"]), it["n_samples"]
    d = dict(params=gpu_params(it), tracks=it["tracks"], n_samples=ns,
             curves=torch.full((nt, ns), -1.0, device="cuda"),
             m_map=torch.full((4,), -1.0, dtype=torch.float64, device="cuda"),
             m_curves=torch.full((nt, 3), -1.0, dtype=torch.float64, device="cuda"))
    if with_maps:
        d["phi"] = torch.empty((n, n), dtype=torch.float64, device="cuda")
        d["intensity"] = torch.empty((n, n), dtype=torch.float32, device="cuda")
    return d


def _single(it):
    p = gpu_params(it)
    phi = S.make_screen(p)
    I = S.sum_passband(p, phi, it["lambdas_nm"])
    S.smooth_source(p, I)
    curves = S.lightcurve(p, I, it["tracks"], it["n_samples"])
    return dict(phi=phi, intensity=I, curves=curves, m_map=S.modulation_index(p, I),
                m_curves=S.curve_modulation(curves))


def _same(a, b, keys):
    for k in keys:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("lanes", [1, 3, S.MAX_LANES])
def test_batch_equals_single_screen_calls(lanes):
    items = _items()
    outs = [_outputs(it) for it in items]
    S.run_batch(outs, LAMS, n_lanes=lanes)
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        _same(o, _single(it), ("phi", "intensity", "curves", "m_map", "m_curves"))


def test_batch_item_matches_oracle():
    items = _items((128, 256))
    outs = [_outputs(it) for it in items]
    S.run_batch(outs, LAMS, n_lanes=2)
    it = items[1]
    p = oracle_params(it)
    I = O.smooth_source(O.sum_passband(O.make_screen(p), p, LAMS), p.pixel_km, p.source_radius_km)
    assert np.abs(outs[1]["intensity"].cpu().numpy() - I).max() <= I_TOL
    c = O.lightcurves(I, it["tracks"], it["n_samples"])
    assert np.abs(outs[1]["curves"].cpu().numpy() - c).max() <= I_TOL
    m_ref = O.modulation_index_map(I, p)
    assert outs[1]["m_map"][0].item() == pytest.approx(m_ref, rel=1e-4)


def test_batch_scratch_maps_and_grouped_workspace():
    """phi/intensity left NULL (lane scratch) and a workspace that forces one wavelength per group."""
    items = _items((256, 128, 64))
    ref = [_outputs(it) for it in items]
    S.run_batch(ref, LAMS, n_lanes=2)
    outs = [_outputs(it, with_maps=False) for it in items]
    arr = S.batch_items(outs)
    ws_bytes = S.batch_workspace_bytes(arr, 1, 2)
    assert ws_bytes < S.batch_workspace_bytes(arr, len(LAMS), 2)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    S.run_batch(arr, LAMS, n_lanes=2, workspace=ws)
    for a, b in zip(outs, ref):
        # grouping changes only the FP32 summation order of the passband
        assert torch.allclose(a["curves"], b["curves"], rtol=0, atol=1e-5)
        assert a["m_map"][0].item() == pytest.approx(b["m_map"][0].item(), rel=1e-5)
        assert torch.allclose(a["m_curves"], b["m_curves"], rtol=1e-5, atol=0)


def test_batch_graph_capture_replays():
    items = _items((128, 256, 64, 128))
    eager = [_outputs(it) for it in items]
    S.run_batch(eager, LAMS, n_lanes=3)
    outs = [_outputs(it) for it in items]
    arr = S.batch_items(outs)
    ws = torch.empty(S.batch_workspace_bytes(arr, len(LAMS), 3), dtype=torch.uint8, device="cuda")
    S.run_batch(arr, LAMS, n_lanes=3, workspace=ws)      # kernel attributes set outside the capture
    for o in outs:
        for k in ("curves", "intensity", "m_map"):
            o[k].fill_(-7.0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        S.run_batch(arr, LAMS, n_lanes=3, workspace=ws)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, eager):
        _same(a, b, ("phi", "intensity", "curves", "m_map", "m_curves"))


def test_batch_with_a_16384_screen_equals_single_calls():
    """A 16384^2 screen (persistent two-block-cluster kernels sized to the whole GPU) on one lane
    while the other lanes run small screens: the same bits as the single-screen calls."""
    lams = np.array([500.0, 560.0])
    big = W.large_screen_16384(beta=3.67, disk=True)
    big["tracks"], big["n_samples"] = big["tracks"][:4], 2048
    items = [big] + _items((256, 128, 512))
    for it in items:
        it["lambdas_nm"] = lams
    outs = [_outputs(it) for it in items]
    S.run_batch(outs, lams, n_lanes=3)
    torch.cuda.synchronize()
    for it, o in zip(items, outs):
        _same(o, _single(it), ("phi", "intensity", "curves", "m_map", "m_curves"))
