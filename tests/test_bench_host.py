"""bench.py's host logic (no GPU): the clock/throttle record that decides whether a run is kept,
and the workloads the bench lines are measured on."""
import os

import numpy as np
import pytest

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_clocks_and_throttle_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1401.0, 0x0000000000000008, Active, Not Active, Not Active, Active",
    ]
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    open(s.path, "w").write("\n".join(rows) + "\n")
    s.proc = _Proc()
    rec = s.stop()
    assert rec == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"], "samples": 3}


def test_clock_sampler_without_samples(tmp_path):
    s = bench.ClockSampler(0)
    assert s.stop() is None                     # never started (no nvidia-smi)
    s.path = str(tmp_path / "empty.csv")
    open(s.path, "w").write("")
    s.proc = _Proc()
    assert s.stop() is None


@pytest.mark.parametrize("name,count,sizes,n_lam", [
    ("batched", 48, {1024, 2048, 4096}, 32),
    ("profile", 1, {4096}, 8),
    ("large16384", 1, {16384}, 1),
    ("single4096", 1, {4096}, 1),
])
def test_workloads(name, count, sizes, n_lam):
    items, desc = bench._workload(name, 0)
    assert len(items) == count and {it["n"] for it in items} == sizes and desc
    assert all(len(it["lambdas_nm"]) == n_lam for it in items)
    # ranks draw disjoint seeds for the same shapes
    other, _ = bench._workload(name, 1)
    assert {it["seed"] for it in items}.isdisjoint({it["seed"] for it in other})
    assert [it["n"] for it in items] == [it["n"] for it in other]
    if name == "batched":
        units = sum(it["n"] ** 2 * len(it["lambdas_nm"]) for it in items)
        assert units == pytest.approx(1.127e10, rel=1e-3)


def test_peaks_and_source_hash():
    hbm, mhz, src = bench._peaks()
    assert hbm > 1000.0 and mhz > 1000.0 and src in ("measured", "fallback")
    h = bench._kernel_source_hash(["fft.cuh", "common.cuh"])
    assert len(h) == 16 and h == bench._kernel_source_hash(["fft.cuh", "common.cuh"])
    assert h != bench._kernel_source_hash(["common.cuh", "fft.cuh"])
