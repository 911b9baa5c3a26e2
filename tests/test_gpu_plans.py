"""Propagation plans and the autotuner.

Every built variant of the transfer-function passes (one wavelength per thread;
two wavelengths per thread with either twiddle source in either pass) against
the FP64 oracle's passband at 2e-4, with even and odd wavelength counts (an odd
group ends with a half-used pair) and with a workspace that forces groups; the
variants agree with each other to FP32 rounding.  The tuner keeps one of them
and reports what it measured; scint_set_plan rejects variants that are not
built.
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


def _variants(n):
    """The plans built for n (set_plan accepts them); the plan of n is restored afterwards."""
    before = S.get_plan(n)
    out = [(0, 2, 1, 16)]
    for pts in (16, 8):
        for r in (1, 2):
            for c in (1, 2):
                try:
                    S.set_plan(n, 1, r, c, pts)
                except S.ScintError:
                    continue
                out.append((1, r, c, pts))
    _restore(n, before)
    return out


def _restore(n, pl):
    S.set_plan(n, pl["packed"], pl["row_twiddles"], pl["col_twiddles"], pl["points"])


@pytest.mark.parametrize("n,n_lam", [(64, 3), (256, 2), (1024, 5), (2048, 4), (4096, 3)])
def test_every_variant_matches_the_oracle(n, n_lam):
    it = W._item(n, 15.0 if n <= 1024 else 10.0, 60.0, lambda_nm=550.0, lambda_ref_nm=550.0,
                 seed=W.SEED_BASE + 91 + n, screen_id=5)
    p_g, p_o = gpu_params(it), oracle_params(it)
    lams = np.linspace(450.0, 650.0, n_lam)
    w = np.linspace(1.0, 2.0, n_lam)
    w /= w.sum()
    phi = O.make_screen(p_o)
    ref = O.sum_passband(phi, p_o, lams, w)
    phi_t = torch.from_numpy(phi).cuda()
    before = S.get_plan(n)
    maps = {}
    try:
        for v in _variants(n):
            S.set_plan(n, *v)
            got = S.sum_passband(p_g, phi_t, lams, w)
            maps[v] = got
            assert np.abs(got.cpu().numpy() - ref).max() <= I_TOL, v
        assert len(maps) >= (1 if n < 64 else 3)
        base = maps[(0, 2, 1, 16)]
        for v, m in maps.items():
            assert (m - base).abs().max().item() <= 1e-5, v
    finally:
        _restore(n, before)


def test_packed_groups_and_accumulate():
    """Seven wavelengths through a workspace that holds three (groups 3 + 3 + 1: an odd pair, a
    one-wavelength group on the unpacked passes), accumulated onto a prior map."""
    n = 512
    it = W._item(n, 15.0, 50.0, lambda_nm=550.0, lambda_ref_nm=550.0, seed=W.SEED_BASE + 92, screen_id=6)
    p_g, p_o = gpu_params(it), oracle_params(it)
    lams = np.linspace(420.0, 690.0, 7)
    phi = O.make_screen(p_o)
    ref = 0.5 + O.sum_passband(phi, p_o, lams)
    S.set_plan(n, 1, 2, 1, 8)
    ws = torch.empty(S.workspace_bytes(p_g, 3), dtype=torch.uint8, device="cuda")
    out = torch.full((n, n), 0.5, device="cuda")
    S.sum_passband(p_g, torch.from_numpy(phi).cuda(), lams, out=out, accumulate=True, workspace=ws)
    assert np.abs(out.cpu().numpy() - ref).max() <= I_TOL


def test_tune_keeps_a_measured_plan():
    n = 1024
    pl = S.tune(n, 8)
    assert pl["tuned"] == 1 and pl["ms"] > 0.0
    assert S.get_plan(n) == pl
    assert (pl["packed"], pl["row_twiddles"], pl["col_twiddles"], pl["points"]) in _variants(n)
    _restore(n, pl)
    again = S.get_plan(n)
    assert again["tuned"] == 0 and again["packed"] == pl["packed"]


def test_tune_sizes_with_one_variant():
    """N = 16384 has one variant (the split passes): the tuner keeps it without timing."""
    pl = S.tune(16384, 4)
    assert pl["tuned"] == 1 and pl["ms"] == 0.0 and pl["packed"] == 0


def test_set_plan_rejects_variants_not_built():
    with pytest.raises(S.ScintError) as e:
        S.set_plan(16384, 1, 2, 1)
    assert e.value.code == 5      # SCINT_EUNSUPPORTED
    with pytest.raises(S.ScintError) as e:
        S.set_plan(1024, 1, 3, 1)
    assert e.value.code == 1      # SCINT_EINVAL
    with pytest.raises(S.ScintError) as e:
        S.set_plan(64, 1, 2, 1, 8)   # 8 values per thread need N >= 128
    assert e.value.code == 5


def test_batch_autotunes_unplanned_sizes_only_outside_capture():
    """With autotuning on, run_batch measures a plan for each new grid size before it launches;
    the result equals the single-screen calls under that plan bit for bit."""
    n = 256
    lams = [520.0, 560.0, 600.0]
    kw = dict(n=n, pixel_km=15.0, r_diff_km=60.0, lambda_nm=560.0, lambda_ref_nm=560.0, seed=5, screen_id=1)
    item = dict(params=S.params(**kw), phi=torch.empty((n, n), dtype=torch.float64, device="cuda"),
                intensity=torch.empty((n, n), device="cuda"))
    old = S.autotune(True)
    try:
        S.lib().scint_release()
        S.set_plan(n, 0)        # a plan exists: no tuning
        S.run_batch([item], lams)
        assert S.get_plan(n)["tuned"] == 0
        n2 = 128      # no other test plans this size
        item2 = dict(params=S.params(**dict(kw, n=n2)), phi=torch.empty((n2, n2), dtype=torch.float64, device="cuda"),
                     intensity=torch.empty((n2, n2), device="cuda"))
        S.run_batch([item2], lams)
        assert S.get_plan(n2)["tuned"] == 1
        torch.cuda.synchronize()
        p = S.params(**dict(kw, n=n2))
        phi = S.make_screen(p)
        assert torch.equal(phi, item2["phi"])
        ref = S.sum_passband(p, phi, lams)
        S.smooth_source(p, ref)
        assert torch.equal(ref, item2["intensity"])
    finally:
        S.autotune(old)


def test_batch_tuner_keeps_the_fastest_plans_and_lanes():
    """scint_tune_batch times the batch under candidate plan sets and lane counts; afterwards the
    batch's sizes carry measured plans and a run with the returned lanes equals the single calls."""
    lams = [480.0, 540.0, 600.0, 660.0]
    entries = []
    for i, n in enumerate((256, 512, 256, 512, 256)):
        kw = dict(n=n, pixel_km=15.0, r_diff_km=70.0, lambda_nm=540.0, lambda_ref_nm=540.0, seed=40 + i, screen_id=i)
        entries.append(dict(params=S.params(**kw), phi=torch.empty((n, n), dtype=torch.float64, device="cuda"),
                            intensity=torch.empty((n, n), device="cuda")))
    batch = S.batch_items(entries)
    lanes, ms, mode = S.tune_batch(batch, lams)
    S.batch_mode(0)
    assert lanes in (4, 5) and ms > 0.0 and mode in (0, 1)
    for n in (256, 512):
        pl = S.get_plan(n)
        assert pl["tuned"] == 1 and pl["ms"] == pytest.approx(ms)
    S.run_batch(batch, lams, n_lanes=lanes)
    torch.cuda.synchronize()
    for e in entries:
        p = e["params"]
        ref = S.sum_passband(p, S.make_screen(p), lams)
        S.smooth_source(p, ref)
        assert torch.equal(ref, e["intensity"])
