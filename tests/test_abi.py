"""The C-ABI library loads and exports every declared entry point; host-side checks (CPU only).

No compute is launched here: invalid parameters are rejected on the host
before any CUDA call, so these run without a GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1301_0514_gb300 as S
from paper_1301_0514_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for h in os.listdir(INCLUDE):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(scint_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1301_0514_gb300 import build
        build.build()
    return S.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert lib.scint_version() >= 100


def test_params_struct_layout_matches_header():
    # int32 n, int32 reserved, 8 doubles, uint64 seed, uint32 id, uint32 reserved
    assert ctypes.sizeof(_lib.ScintParams) == 4 + 4 + 8 * 8 + 8 + 4 + 4
    assert _lib.ScintParams.seed.offset == 72


@pytest.mark.parametrize("kw,msg", [
    (dict(n=100), "power of two"),
    (dict(n=8), "power of two"),
    (dict(n=32768), "power of two"),
    (dict(pixel_km=0.0), "pixel_km"),
    (dict(r_diff_km=-1.0), "r_diff_km"),
    (dict(beta=2.0), "beta"),
    (dict(beta=4.5), "beta"),
    (dict(lambda_nm=0.0), "lambda_nm"),
    (dict(z_pc=float("nan")), "z_pc"),
    (dict(source_radius_km=-3.0), "source_radius_km"),
    (dict(margin_km=1e9), "margin_km"),
])
def test_invalid_parameters_rejected_on_host(lib, kw, msg):
    p = S.params(n=256, pixel_km=20.0, r_diff_km=100.0).replace(**kw)
    rc = lib.scint_make_screen(ctypes.byref(p), ctypes.c_void_p(16), None, 0, None)
    assert rc == 1
    assert msg in lib.scint_last_error().decode()
    rc = lib.scint_propagate(ctypes.byref(p), ctypes.c_void_p(16), ctypes.c_void_p(16), None, 0, None)
    assert rc == 1


def test_reserved_fields_and_null_pointers(lib):
    p = S.params(n=256, pixel_km=20.0, r_diff_km=100.0)
    bad = p.replace(reserved0=1)
    assert lib.scint_make_screen(ctypes.byref(bad), ctypes.c_void_p(16), None, 0, None) == 1
    assert lib.scint_make_screen(ctypes.byref(p), None, None, 0, None) == 1
    assert lib.scint_make_screen(None, ctypes.c_void_p(16), None, 0, None) == 1
    lam = np.array([500.0])
    assert lib.scint_sum_passband(ctypes.byref(p), ctypes.c_void_p(16), lam.ctypes.data_as(ctypes.c_void_p),
                                  None, 0, ctypes.c_void_p(16), 0, None, 0, None) == 1
    lam = np.array([500.0, -1.0])
    assert lib.scint_sum_passband(ctypes.byref(p), ctypes.c_void_p(16), lam.ctypes.data_as(ctypes.c_void_p),
                                  None, 2, ctypes.c_void_p(16), 0, None, 0, None) == 1
    tr = np.array([0.0, 0.0, float("inf"), 1.0])
    assert lib.scint_lightcurve(ctypes.byref(p), ctypes.c_void_p(16), tr.ctypes.data_as(ctypes.c_void_p),
                                1, 10, ctypes.c_void_p(16), None) == 1


def test_workspace_too_small_rejected(lib):
    p = S.params(n=1024, pixel_km=10.0, r_diff_km=50.0)
    need1 = S.workspace_bytes(p, 1)
    assert need1 > 1024 * 1024 * 8
    assert S.workspace_bytes(p, 32) > S.workspace_bytes(p, 8) > need1 - 1
    # a workspace that cannot hold even one wavelength group
    rc = lib.scint_propagate(ctypes.byref(p), ctypes.c_void_p(256), ctypes.c_void_p(256),
                             ctypes.c_void_p(256), 1024, None)
    assert rc == 2 and "workspace" in lib.scint_last_error().decode()


def test_workloads_are_seeded_and_shaped():
    from paper_1301_0514_gb300 import workloads as W
    c3 = W.batched_polychromatic()
    assert len(c3) == 48 and sorted({it["n"] for it in c3}) == [1024, 2048, 4096]
    assert all(len(it["lambdas_nm"]) == 32 for it in c3)
    assert all(30.0 <= it["r_diff_km"] <= 300.0 for it in c3)
    again = W.batched_polychromatic()
    assert all(a["seed"] == b["seed"] and a["r_diff_km"] == b["r_diff_km"] for a, b in zip(c3, again))
    c2 = W.single_screens_4096()
    assert [it["r_diff_km"] for it in c2] == [30.0, 100.0, 300.0] and c2[0]["tracks"].shape == (64, 4)


def _c_layout(struct, fields):
    """offsetof/sizeof of a struct of include/scint.h, compiled with the host C compiler."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    body = "".join(f'printf("%zu ", offsetof({struct}, {f}));' for f in fields)
    src = f'#include <stdio.h>\n#include <stddef.h>\n#include "scint.h"\nint main(void){{{body}printf("%zu", sizeof({struct}));return 0;}}\n'
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "p.c"), os.path.join(d, "p")
        open(c, "w").write(src)
        subprocess.run([cc, "-I", INCLUDE, c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(x) for x in out]


def test_struct_layouts_match_the_c_compiler():
    for struct, cls in (("scint_params", _lib.ScintParams), ("scint_batch_item", _lib.BatchItem),
                        ("scint_kernel_stat", _lib.KernelStat), ("scint_plan", _lib.ScintPlan)):
        fields = [f for f, _ in cls._fields_]
        got = _c_layout(struct, fields)
        assert got[:-1] == [getattr(cls, f).offset for f in fields], struct
        assert got[-1] == ctypes.sizeof(cls), struct


def _batch_entry(n=256, **kw):
    return dict(params=S.params(n=n, pixel_km=20.0, r_diff_km=100.0, **kw))


def test_batch_rejected_on_host(lib):
    good = _batch_entry()
    lam = [500.0, 600.0]
    cases = [
        ([good, _batch_entry(n=100)], {}, "item 1: n=100"),
        ([good], dict(n_lanes=S.MAX_LANES + 1), "n_lanes"),
        ([dict(good, tracks=np.array([[0.0, 1.0, float("nan"), 1.0]]), n_samples=4)], {}, "item 0"),
        ([dict(good, tracks=np.array([[0.0, 1.0, 0.5, 1.0]]), n_samples=4)], {}, "tracks and curves"),
    ]
    for items, kw, msg in cases:
        with pytest.raises(S.ScintError) as e:
            S.run_batch(items, lam, stream=0, **kw)
        assert e.value.code == 1 and msg in str(e.value), (msg, str(e.value))
    with pytest.raises(S.ScintError):
        S.run_batch([good], [], stream=0)


def test_batch_workspace_bytes(lib):
    items = [_batch_entry(n=256), _batch_entry(n=1024), _batch_entry(n=512)]
    one = S.batch_workspace_bytes(items, 4, 1)
    assert one > 0
    # lanes split the workspace into equal slices sized for the largest screen
    assert S.batch_workspace_bytes(items, 4, 3) == 3 * one
    assert S.batch_workspace_bytes(items, 4, 5) == 3 * one       # never more lanes than items
    assert S.batch_workspace_bytes(items, 8, 1) > one            # a larger wavelength group
    assert S.batch_workspace_bytes([_batch_entry(n=100)], 4, 1) == 0


@pytest.mark.parametrize("n,msg", [(15, "even"), (8, "even"), (32770, "even")])
def test_screen_check_rejected_on_host(lib, n, msg):
    p = S.params(n=n, pixel_km=10.0, r_diff_km=50.0)
    rc = lib.scint_spectrum_rec(ctypes.byref(p), ctypes.c_void_p(16), ctypes.c_void_p(16), 10, None)
    assert rc == 1 and msg in lib.scint_last_error().decode()


def test_screen_check_arguments_rejected_on_host(lib):
    p = S.params(n=14000, pixel_km=28.85, r_diff_km=500.0)
    assert lib.scint_spectrum_rec(ctypes.byref(p), ctypes.c_void_p(16), ctypes.c_void_p(16), 0, None) == 1
    assert lib.scint_spectrum_rec(ctypes.byref(p), None, ctypes.c_void_p(16), 10, None) == 1
    assert lib.scint_structure_function_rec(ctypes.byref(p), ctypes.c_void_p(16), 1, None, 0, None,
                                            ctypes.c_void_p(16), None, 0, None) == 1
    assert lib.scint_structure_function_rec(ctypes.byref(p), ctypes.c_void_p(16), 100, None, 3, None,
                                            None, None, 0, None) == 1
    assert S.max_annulus(14000) == O_max_annulus(14000)


def O_max_annulus(n):
    import oracle as O
    return O.max_annulus(n)


def test_conjugate_host_checks(lib):
    p = S.params(n=64, pixel_km=10.0, r_diff_km=50.0, lambda_nm=500.0)
    assert lib.scint_conjugate_pixel_km(ctypes.byref(p), 500.0) == pytest.approx(
        500.0 * 1e-12 * 160.0 * 3.0856775814913673e13 / 640.0, rel=1e-15)
    import math
    assert math.isnan(lib.scint_conjugate_pixel_km(ctypes.byref(p.replace(n=100)), 500.0))
    assert lib.scint_propagate_conjugate(ctypes.byref(p.replace(beta=5.0)), ctypes.c_void_p(16),
                                         ctypes.c_void_p(16), None, 0, None) == 1
    assert lib.scint_propagate_conjugate(ctypes.byref(p), None, ctypes.c_void_p(16), None, 0, None) == 1


def test_timeseries_host_checks(lib):
    assert lib.scint_curve_power_spectrum(ctypes.c_void_p(16), 3, 1000, ctypes.c_void_p(16), None, 0, None) == 1
    assert "power of two" in lib.scint_last_error().decode()
    assert lib.scint_curve_power_spectrum(ctypes.c_void_p(16), 3, 16384, ctypes.c_void_p(16), None, 0, None) == 1
    assert lib.scint_curve_power_spectrum(None, 0, 256, None, None, 0, None) == 0      # nothing to do
    assert lib.scint_curve_correlation(ctypes.c_void_p(16), 2, 100, ctypes.c_void_p(16), 3, 100,
                                       ctypes.c_void_p(16), None) == 1          # 2 does not divide 3
    assert lib.scint_curve_correlation(ctypes.c_void_p(16), 3, 50, ctypes.c_void_p(16), 3, 100,
                                       ctypes.c_void_p(16), None) == 1          # rows of a overlap
    assert lib.scint_curve_correlation(ctypes.c_void_p(16), 1, 0, ctypes.c_void_p(16), 3, 1,
                                       ctypes.c_void_p(16), None) == 1


def test_wavelength_count_limits(lib):
    p = S.params(n=64, pixel_km=20.0, r_diff_km=50.0)
    lam = (ctypes.c_double * (S.MAX_LAMBDA + 1))(*([500.0] * (S.MAX_LAMBDA + 1)))
    for count in (0, S.MAX_LAMBDA + 1):
        rc = lib.scint_sum_passband(ctypes.byref(p), ctypes.c_void_p(16), lam, None, count, ctypes.c_void_p(16), 0,
                                    None, 0, None)
        assert rc == 1 and "n_lambda" in lib.scint_last_error().decode()
    bad = (ctypes.c_double * 2)(500.0, -1.0)
    assert lib.scint_sum_passband(ctypes.byref(p), ctypes.c_void_p(16), bad, None, 2, ctypes.c_void_p(16), 0,
                                  None, 0, None) == 1
    nan_w = (ctypes.c_double * 2)(0.5, float("nan"))
    assert lib.scint_sum_passband(ctypes.byref(p), ctypes.c_void_p(16), lam, nan_w, 2, ctypes.c_void_p(16), 0,
                                  None, 0, None) == 1


def test_sampling_ratio_closed_form(lib):
    """Sect. 3.2.2 asks pixel < R_diff(lambda)/2, R_diff(lambda) = R_diff (lambda/lambda_ref)^(2/(beta-2))
    (phase ~ lambda_ref/lambda; Kolmogorov R_diff ~ lambda^(6/5)); the ratio is checked on the host."""
    p = S.params(n=256, pixel_km=20.0, r_diff_km=100.0, lambda_nm=500.0, lambda_ref_nm=500.0)
    assert S.sampling_ratio(p) == pytest.approx(0.4, rel=1e-15)
    q = S.params(n=256, pixel_km=20.0, r_diff_km=100.0, beta=11.0 / 3.0, lambda_nm=550.0, lambda_ref_nm=550.0)
    want = 40.0 / (100.0 * (400.0 / 550.0) ** 1.2)           # the shortest wavelength has the smallest R_diff
    assert S.sampling_ratio(q, [700.0, 400.0, 550.0]) == pytest.approx(want, rel=1e-13)
    b = S.params(n=256, pixel_km=20.0, r_diff_km=100.0, beta=3.1, lambda_nm=550.0, lambda_ref_nm=550.0)
    assert S.sampling_ratio(b, [800.0]) == pytest.approx(40.0 / (100.0 * (800.0 / 550.0) ** (2.0 / 1.1)), rel=1e-13)
    # pixel = R_diff/2 exactly is on the violating side
    assert S.sampling_ratio(S.params(n=256, pixel_km=50.0, r_diff_km=100.0)) == pytest.approx(1.0, rel=1e-15)
    with pytest.raises(S.ScintError):
        S.sampling_ratio(S.params(n=256, pixel_km=-1.0, r_diff_km=100.0))
    with pytest.raises(S.ScintError):
        S.sampling_ratio(p, [500.0, -3.0])
    assert S.last_warning() == ""     # nothing propagated on this thread


def test_cpu_tensors_are_refused_no_fallback(lib):
    """The product path has no CPU fallback: the binding refuses host tensors loudly before any
    library call (the oracle is test infrastructure, never a substitute)."""
    import torch
    p = S.params(n=64, pixel_km=20.0, r_diff_km=100.0)
    phi = torch.zeros((64, 64), dtype=torch.float64)
    I = torch.ones((64, 64), dtype=torch.float32)
    calls = [
        lambda: S.make_screen(p, out=phi),
        lambda: S.propagate(p, phi),
        lambda: S.sum_passband(p, phi, [500.0, 550.0]),
        lambda: S.smooth_source(p, I),
        lambda: S.lightcurve(p, I, np.array([[1.0, 2.0, 0.3, 1.0]]), 10),
        lambda: S.propagate_conjugate(p, phi),
        lambda: S.phase_fixed(phi.reshape(-1)),
        lambda: S.fft_lines(torch.zeros((2, 64), dtype=torch.complex64), -1),
    ]
    for call in calls:
        with pytest.raises(ValueError):
            call()


def test_plan_host_checks(lib):
    """Plan calls reject bad grid sizes and variants on the host (no GPU call is made)."""
    pl = _lib.ScintPlan(packed=1, points=16, row_twiddles=3, col_twiddles=1)
    assert lib.scint_set_plan(1024, ctypes.byref(pl)) == 1
    assert lib.scint_set_plan(1000, ctypes.byref(pl)) == 1
    assert lib.scint_get_plan(1000, ctypes.byref(pl)) == 1
    assert lib.scint_get_plan(1024, None) == 1
    assert lib.scint_tune(999, 8, None, None) == 1
    assert lib.scint_autotune(0) in (0, 1)


def test_screen_must_be_16_byte_aligned(lib):
    """The synthesis writes two phases per 16-byte store: an unaligned phi is refused on the host."""
    p = _lib.params(n=64, pixel_km=20.0, r_diff_km=100.0)
    assert lib.scint_make_screen(ctypes.byref(p), ctypes.c_void_p(8), None, 0, None) == 1
    assert "16-byte aligned" in lib.scint_last_error().decode()
