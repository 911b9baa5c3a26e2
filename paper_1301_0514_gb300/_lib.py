"""ctypes binding of libscint.so: argument marshalling only.

Every function here forwards to the C entry point of the same name in
include/scint.h (or include/scint_testing.h).  PyTorch supplies device memory,
the current CUDA stream and workspace buffers; all computation happens in the
library's CUDA kernels.  If the library is missing or fails to load, every
call raises: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import warnings
import os
from typing import Optional, Sequence

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libscint.so")

SCINT_OK = 0
ERRORS = {1: "SCINT_EINVAL", 2: "SCINT_ENOMEM", 3: "SCINT_ECUDA", 4: "SCINT_ETIMEOUT", 5: "SCINT_EUNSUPPORTED"}
MAX_LAMBDA = 128
MAX_CHECK_N = 32768


class ScintError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class ScintParams(ctypes.Structure):
    """Mirror of struct scint_params (include/scint.h)."""
    _fields_ = [
        ("n", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("pixel_km", ctypes.c_double),
        ("r_diff_km", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("lambda_nm", ctypes.c_double),
        ("lambda_ref_nm", ctypes.c_double),
        ("z_pc", ctypes.c_double),
        ("source_radius_km", ctypes.c_double),
        ("margin_km", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("screen_id", ctypes.c_uint32),
        ("reserved1", ctypes.c_uint32),
    ]

    def replace(self, **kw) -> "ScintParams":
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d.update(kw)
        return ScintParams(**d)

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


def params(n: int, pixel_km: float, r_diff_km: float, beta: float = 11.0 / 3.0, lambda_nm: float = 500.0,
           lambda_ref_nm: Optional[float] = None, z_pc: float = 160.0, source_radius_km: float = 0.0,
           seed: int = 0, screen_id: int = 0, margin_km: float = -1.0) -> ScintParams:
    return ScintParams(n=n, reserved0=0, pixel_km=pixel_km, r_diff_km=r_diff_km, beta=beta,
                       lambda_nm=lambda_nm, lambda_ref_nm=lambda_nm if lambda_ref_nm is None else lambda_ref_nm,
                       z_pc=z_pc, source_radius_km=source_radius_km, margin_km=margin_km,
                       seed=seed, screen_id=screen_id, reserved1=0)


class BatchItem(ctypes.Structure):
    """Mirror of struct scint_batch_item (include/scint.h)."""
    _fields_ = [
        ("params", ScintParams),
        ("phi", ctypes.c_void_p),
        ("intensity", ctypes.c_void_p),
        ("tracks", ctypes.c_void_p),
        ("n_tracks", ctypes.c_int32),
        ("n_samples", ctypes.c_int32),
        ("curves", ctypes.c_void_p),
        ("m_map", ctypes.c_void_p),
        ("m_curves", ctypes.c_void_p),
    ]


MAX_LANES = 8


class KernelStat(ctypes.Structure):
    """Mirror of struct scint_kernel_stat (include/scint.h)."""
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class ScintPlan(ctypes.Structure):
    """Mirror of struct scint_plan (include/scint.h)."""
    _fields_ = [("packed", ctypes.c_int32), ("points", ctypes.c_int32), ("row_twiddles", ctypes.c_int32),
                ("col_twiddles", ctypes.c_int32), ("tuned", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_lib = None
_P = ctypes.POINTER(ScintParams)
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i = ctypes.c_int


def lib() -> ctypes.CDLL:
    """Load libscint.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1301_0514_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "scint_version": ([], _i),
        "scint_last_error": ([], ctypes.c_char_p),
        "scint_last_warning": ([], ctypes.c_char_p),
        "scint_sampling_ratio": ([_P, _vp, _i], ctypes.c_double),
        "scint_workspace_bytes": ([_P, _i], _sz),
        "scint_make_screen": ([_P, _vp, _vp, _sz, _vp], _i),
        "scint_propagate": ([_P, _vp, _vp, _vp, _sz, _vp], _i),
        "scint_propagate_noalloc": ([_P, _vp, _vp, _vp], _i),
        "scint_propagate64": ([_P, _vp, _vp, _vp, _sz, _vp], _i),
        "scint_sum_passband": ([_P, _vp, _vp, _vp, _i, _vp, _i, _vp, _sz, _vp], _i),
        "scint_smooth_source": ([_P, _vp, _vp, _sz, _vp], _i),
        "scint_lightcurve": ([_P, _vp, _vp, _i, _i, _vp, _vp], _i),
        "scint_modulation_index": ([_P, _vp, _vp, _vp, _sz, _vp], _i),
        "scint_curve_modulation": ([_vp, _i, _i, _vp, _vp], _i),
        "scint_release": ([], None),
        "scint_noise_words": ([_P, _vp, _vp], _i),
        "scint_noise_spectrum": ([_P, _vp, _vp], _i),
        "scint_fft_lines32": ([_i, _i, _vp, _i, _vp], _i),
        "scint_phase_fixed": ([_vp, _vp, ctypes.c_int64, _vp], _i),
        "scint_fft_lines64": ([_i, _i, _vp, _i, _vp], _i),
        "scint_lightcurve_adjoint": ([_P, _vp, _vp, _vp, _i, _vp, _i, _i, _vp, _vp, _i, _vp, _sz, _vp], _i),
        "scint_rdiff_gradient": ([_P, _vp, _vp, _vp, _vp, _sz, _vp], _i),
        "scint_batch_workspace_bytes": ([ctypes.POINTER(BatchItem), _i, _i, _i], _sz),
        "scint_run_batch": ([ctypes.POINTER(BatchItem), _i, _vp, _vp, _i, _i, _vp, _sz, _vp], _i),
        "scint_spectrum_rec": ([_P, _vp, _vp, _i, _vp], _i),
        "scint_curve_power_spectrum": ([_vp, _i, _i, _vp, _vp, _sz, _vp], _i),
        "scint_curve_correlation": ([_vp, _i, ctypes.c_int64, _vp, _i, _i, _vp, _vp], _i),
        "scint_fiducial_zone": ([_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_double)], _i),
        "scint_propagate_conjugate": ([_P, _vp, _vp, _vp, _sz, _vp], _i),
        "scint_sum_passband_conjugate": ([_P, _vp, _vp, _vp, _i, _vp, _i, _vp, _sz, _vp], _i),
        "scint_conjugate_pixel_km": ([_P, ctypes.c_double], ctypes.c_double),
        "scint_structure_function_rec": ([_P, _vp, _i, _vp, _i, _vp, _vp, _vp, _sz, _vp], _i),
        "scint_get_plan": ([_i, ctypes.POINTER(ScintPlan)], _i),
        "scint_set_plan": ([_i, ctypes.POINTER(ScintPlan)], _i),
        "scint_tune": ([_i, _i, ctypes.POINTER(ScintPlan), _vp], _i),
        "scint_autotune": ([_i], _i),
        "scint_batch_mode": ([_i], _i),
        "scint_batch_status": ([_vp], _i),
        "scint_testing_persist": ([_i, _i], None),
        "scint_tune_batch": ([ctypes.POINTER(BatchItem), _i, _vp, _vp, _i, _vp, _sz, ctypes.POINTER(_i),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i), _vp], _i),
        "scint_profile_enable": ([_i], _i),
        "scint_profile_read": ([ctypes.POINTER(KernelStat), _i, ctypes.POINTER(_i)], _i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc: int):
    if rc != SCINT_OK:
        raise ScintError(rc, lib().scint_last_error().decode())


class SamplingWarning(UserWarning):
    """The pixel does not resolve the screen's phase variations (Sect. 3.2.2:
    pixel < R_diff(lambda)/2); the call still ran."""


def _check_warn(rc: int):
    """_check, then the library's sampling warning (if any) as a SamplingWarning."""
    _check(rc)
    msg = lib().scint_last_warning().decode()
    if msg:
        warnings.warn(msg, SamplingWarning, stacklevel=3)


def last_warning() -> str:
    return lib().scint_last_warning().decode()


def sampling_ratio(p: "ScintParams", lambdas_nm=None) -> float:
    """Worst 2 pixel / R_diff(lambda) over the wavelengths (>= 1 violates Sect. 3.2.2)."""
    if lambdas_nm is None:
        r = lib().scint_sampling_ratio(ctypes.byref(p), None, 0)
    else:
        lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
        r = lib().scint_sampling_ratio(ctypes.byref(p), lam.ctypes.data_as(ctypes.c_void_p), len(lam))
    if r < 0:
        raise ScintError(1, lib().scint_last_error().decode())   # SCINT_EINVAL
    return r


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, numel: int, name: str):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
            and t.numel() == numel):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor with {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def workspace_bytes(p: ScintParams, n_lambda: int = 1) -> int:
    return int(lib().scint_workspace_bytes(ctypes.byref(p), n_lambda))


def _workspace(p: ScintParams, n_lambda: int, workspace, device):
    if workspace is None:
        workspace = torch.empty(workspace_bytes(p, n_lambda), dtype=torch.uint8, device=device)
    return workspace, ctypes.c_void_p(workspace.data_ptr()), workspace.numel()


def make_screen(p: ScintParams, out: Optional[torch.Tensor] = None, workspace=None, stream=None,
                device="cuda") -> torch.Tensor:
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float64, device=device)
    ws, wp, wb = _workspace(p, 1, workspace, out.device)
    _check(lib().scint_make_screen(ctypes.byref(p), _dev(out, torch.float64, p.n * p.n, "phi"),
                                   wp, wb, _stream(stream)))
    return out


def propagate(p: ScintParams, phi: torch.Tensor, out: Optional[torch.Tensor] = None, workspace=None,
              stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float32, device=phi.device)
    ws, wp, wb = _workspace(p, 1, workspace, phi.device)
    _check_warn(lib().scint_propagate(ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"),
                                 _dev(out, torch.float32, p.n * p.n, "intensity"), wp, wb, _stream(stream)))
    return out


def propagate64(p: ScintParams, phi: torch.Tensor, out: Optional[torch.Tensor] = None, workspace=None,
                stream=None) -> torch.Tensor:
    """The plain method in FP64 (scint_propagate64): an FP64 intensity map, n <= 4096."""
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float64, device=phi.device)
    ws, wp, wb = _workspace(p, 1, workspace, phi.device)
    _check_warn(lib().scint_propagate64(ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"),
                                   _dev(out, torch.float64, p.n * p.n, "intensity"), wp, wb, _stream(stream)))
    return out


def sum_passband(p: ScintParams, phi: torch.Tensor, lambdas_nm: Sequence[float], weights=None,
                 out: Optional[torch.Tensor] = None, accumulate: bool = False, workspace=None,
                 stream=None) -> torch.Tensor:
    lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and w.shape != lam.shape:
        raise ValueError("weights must match lambdas")
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float32, device=phi.device)
    ws, wp, wb = _workspace(p, len(lam), workspace, phi.device)
    _check_warn(lib().scint_sum_passband(
        ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"),
        lam.ctypes.data_as(ctypes.c_void_p), None if w is None else w.ctypes.data_as(ctypes.c_void_p),
        len(lam), _dev(out, torch.float32, p.n * p.n, "intensity"), int(bool(accumulate)), wp, wb,
        _stream(stream)))
    return out


def curve_power_spectrum(curves: torch.Tensor, out: Optional[torch.Tensor] = None, workspace=None,
                         stream=None) -> torch.Tensor:
    """Periodogram (n_curves, n/2 + 1) of light curves (n_curves, n), mean removed (Sect. 5)."""
    nc, ns = curves.shape
    if out is None:
        out = torch.empty((nc, ns // 2 + 1), dtype=torch.float32, device=curves.device)
    if workspace is None:
        wp, wb = None, 0
    else:
        wp, wb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
    _check(lib().scint_curve_power_spectrum(_dev(curves, torch.float32, nc * ns, "curves"), nc, ns,
                                            _dev(out, torch.float32, nc * (ns // 2 + 1), "power"), wp, wb,
                                            _stream(stream)))
    return out


def curve_correlation(a: torch.Tensor, b: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None,
                      a_rows: Optional[int] = None, a_stride: Optional[int] = None) -> torch.Tensor:
    """Correlation coefficient of row i of b with row i // (n_pairs // a_rows) of a (Sect. 5).
    By default a's rows are contiguous and a_rows is its row count; a strided view of a
    larger tensor can be given with a_rows and a_stride (in floats)."""
    b2 = b.reshape(-1, b.shape[-1])
    n_pairs, ns = b2.shape
    if a_rows is None:
        a2 = a.reshape(-1, a.shape[-1])
        _dev(a2, torch.float32, a2.numel(), "a")
        a_rows, a_stride = a2.shape[0], ns
    elif not (a.is_cuda and a.dtype == torch.float32):
        raise ValueError("a must be a float32 CUDA tensor")
    if out is None:
        out = torch.empty(n_pairs, dtype=torch.float64, device=b.device)
    _check(lib().scint_curve_correlation(ctypes.c_void_p(a.data_ptr()), int(a_rows), int(a_stride),
                                         _dev(b2, torch.float32, b2.numel(), "b"), n_pairs, ns,
                                         _dev(out, torch.float64, n_pairs, "r"), _stream(stream)))
    return out


def fiducial_zone(p: ScintParams):
    """(i0, i1, r_ref_km, exists): the fiducial pixel range of scint_modulation_index."""
    i0, i1, rr = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0.0)
    rc = lib().scint_fiducial_zone(ctypes.byref(p), ctypes.byref(i0), ctypes.byref(i1), ctypes.byref(rr))
    if rc not in (SCINT_OK, 5):
        _check(rc)
    return i0.value, i1.value, rr.value, rc == SCINT_OK


def conjugate_pixel_km(p: ScintParams, lambda_nm: Optional[float] = None) -> float:
    """Observer pixel lambda z / (N Delta) of the one-FFT method (km)."""
    return float(lib().scint_conjugate_pixel_km(ctypes.byref(p), p.lambda_nm if lambda_nm is None else lambda_nm))


def propagate_conjugate(p: ScintParams, phi: torch.Tensor, out: Optional[torch.Tensor] = None, workspace=None,
                        stream=None) -> torch.Tensor:
    """One-FFT pattern at p.lambda_nm (Eq. intens), optical axis at element (N/2, N/2)."""
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float32, device=phi.device)
    ws, wp, wb = _workspace(p, 1, workspace, phi.device)
    _check_warn(lib().scint_propagate_conjugate(ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"),
                                           _dev(out, torch.float32, p.n * p.n, "intensity"), wp, wb,
                                           _stream(stream)))
    return out


def sum_passband_conjugate(p: ScintParams, phi: torch.Tensor, lambdas_nm: Sequence[float], weights=None,
                           out: Optional[torch.Tensor] = None, accumulate: bool = False, workspace=None,
                           stream=None) -> torch.Tensor:
    """Passband of one-FFT patterns resampled onto the grid of p.lambda_nm."""
    lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and w.shape != lam.shape:
        raise ValueError("weights must match lambdas")
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float32, device=phi.device)
    if workspace is None:
        wp, wb = None, 0
    else:
        wp, wb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
    _check_warn(lib().scint_sum_passband_conjugate(
        ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"),
        lam.ctypes.data_as(ctypes.c_void_p), None if w is None else w.ctypes.data_as(ctypes.c_void_p),
        len(lam), _dev(out, torch.float32, p.n * p.n, "intensity"), int(bool(accumulate)), wp, wb,
        _stream(stream)))
    return out


def smooth_source(p: ScintParams, intensity: torch.Tensor, workspace=None, stream=None) -> torch.Tensor:
    ws, wp, wb = _workspace(p, 1, workspace, intensity.device)
    _check(lib().scint_smooth_source(ctypes.byref(p), _dev(intensity, torch.float32, p.n * p.n, "intensity"),
                                     wp, wb, _stream(stream)))
    return intensity


def lightcurve(p: ScintParams, intensity: torch.Tensor, tracks, n_samples: int,
               out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    tr = np.ascontiguousarray(tracks, dtype=np.float64).reshape(-1, 4)
    if out is None:
        out = torch.empty((tr.shape[0], n_samples), dtype=torch.float32, device=intensity.device)
    _check(lib().scint_lightcurve(ctypes.byref(p), _dev(intensity, torch.float32, p.n * p.n, "intensity"),
                                  tr.ctypes.data_as(ctypes.c_void_p), tr.shape[0], n_samples,
                                  _dev(out, torch.float32, tr.shape[0] * n_samples, "curves"),
                                  _stream(stream)))
    return out


def modulation_index(p: ScintParams, intensity: torch.Tensor, out: Optional[torch.Tensor] = None,
                     workspace=None, stream=None) -> torch.Tensor:
    """Device tensor (m, mean, sigma, count) over the fiducial zone."""
    if out is None:
        out = torch.empty(4, dtype=torch.float64, device=intensity.device)
    ws, wp, wb = _workspace(p, 1, workspace, intensity.device)
    _check(lib().scint_modulation_index(ctypes.byref(p), _dev(intensity, torch.float32, p.n * p.n, "intensity"),
                                        _dev(out, torch.float64, 4, "out"), wp, wb, _stream(stream)))
    return out


def curve_modulation(curves: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    nc, ns = curves.shape
    if out is None:
        out = torch.empty((nc, 3), dtype=torch.float64, device=curves.device)
    _check(lib().scint_curve_modulation(_dev(curves, torch.float32, nc * ns, "curves"), nc, ns,
                                        _dev(out, torch.float64, nc * 3, "out"), _stream(stream)))
    return out


def lightcurve_adjoint(p: ScintParams, phi: torch.Tensor, lambdas_nm, tracks, n_samples: int,
                       grad_curves: torch.Tensor, weights=None, out: Optional[torch.Tensor] = None,
                       accumulate: bool = False, workspace=None, stream=None) -> torch.Tensor:
    """dL/dphi (N x N float64) for the forward curves = lightcurve(smooth(sum_passband(phi)))."""
    lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    tr = np.ascontiguousarray(tracks, dtype=np.float64).reshape(-1, 4)
    if out is None:
        out = torch.empty((p.n, p.n), dtype=torch.float64, device=phi.device)
    ws, wp, wb = _workspace(p, len(lam), workspace, phi.device)
    _check_warn(lib().scint_lightcurve_adjoint(
        ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"), lam.ctypes.data_as(ctypes.c_void_p),
        None if w is None else w.ctypes.data_as(ctypes.c_void_p), len(lam),
        tr.ctypes.data_as(ctypes.c_void_p), tr.shape[0], n_samples,
        _dev(grad_curves, torch.float32, tr.shape[0] * n_samples, "grad_curves"),
        _dev(out, torch.float64, p.n * p.n, "grad_phi"), int(bool(accumulate)), wp, wb, _stream(stream)))
    return out


def rdiff_gradient(p: ScintParams, phi: torch.Tensor, grad_phi: torch.Tensor, workspace=None,
                   out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """dL/dR_diff (1-element float64 device tensor) from dL/dphi at a fixed seed."""
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=phi.device)
    ws, wp, wb = _workspace(p, 1, workspace, phi.device)
    _check(lib().scint_rdiff_gradient(ctypes.byref(p), _dev(phi, torch.float64, p.n * p.n, "phi"),
                                      _dev(grad_phi, torch.float64, p.n * p.n, "grad_phi"),
                                      _dev(out, torch.float64, 1, "out"), wp, wb, _stream(stream)))
    return out


def _opt_dev(t: Optional[torch.Tensor], dtype, numel: int, name: str):
    return None if t is None else _dev(t, dtype, numel, name)


def batch_items(entries) -> "ctypes.Array":
    """ctypes array of scint_batch_item from dicts with keys params and, optionally,
    phi, intensity, tracks (n x 4 host array), n_samples, curves, m_map, m_curves
    (device tensors or None).  The track arrays are kept alive on the result."""
    arr = (BatchItem * len(entries))()
    keep = []
    for i, e in enumerate(entries):
        p = e["params"]
        nn = p.n * p.n
        tr = np.ascontiguousarray(e.get("tracks", np.zeros((0, 4))), dtype=np.float64).reshape(-1, 4)
        keep.append(tr)
        ns = int(e.get("n_samples", 0))
        arr[i].params = p
        arr[i].phi = _opt_dev(e.get("phi"), torch.float64, nn, "phi")
        arr[i].intensity = _opt_dev(e.get("intensity"), torch.float32, nn, "intensity")
        arr[i].tracks = tr.ctypes.data if tr.shape[0] else None
        arr[i].n_tracks = tr.shape[0]
        arr[i].n_samples = ns
        arr[i].curves = _opt_dev(e.get("curves"), torch.float32, tr.shape[0] * ns, "curves")
        arr[i].m_map = _opt_dev(e.get("m_map"), torch.float64, 4, "m_map")
        arr[i].m_curves = _opt_dev(e.get("m_curves"), torch.float64, 3 * tr.shape[0], "m_curves")
    arr._keep = keep
    return arr


def batch_workspace_bytes(items, n_lambda: int, n_lanes: int = 0) -> int:
    arr = items if isinstance(items, ctypes.Array) else batch_items(items)
    return int(lib().scint_batch_workspace_bytes(arr, len(arr), n_lambda, n_lanes))


def run_batch(items, lambdas_nm, weights=None, n_lanes: int = 0, workspace: Optional[torch.Tensor] = None,
              stream=None):
    """Forward path of every item (see scint_run_batch); outputs are written into the
    items' tensors.  `items` is a list of dicts (batch_items) or its ctypes array."""
    arr = items if isinstance(items, ctypes.Array) else batch_items(items)
    lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if workspace is None:
        wp, wb = None, 0
    else:
        if not (workspace.is_cuda and workspace.is_contiguous()):
            raise ValueError("workspace must be a contiguous CUDA tensor")
        wp, wb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
    _check_warn(lib().scint_run_batch(arr, len(arr), lam.ctypes.data_as(ctypes.c_void_p),
                                 None if w is None else w.ctypes.data_as(ctypes.c_void_p), len(lam),
                                 int(n_lanes), wp, wb, _stream(stream)))
    return arr


def max_annulus(n: int) -> int:
    """Largest annulus index of an n x n grid (its corner, |m| = sqrt(2) n/2)."""
    return int(np.floor(np.sqrt(2.0 * (n // 2) ** 2) + 0.5))


def spectrum_rec(p: ScintParams, n_bins: Optional[int] = None, out=None, stream=None, device="cuda"):
    """(S_rec, counts) over annuli j = 0..n_bins-1 (Sect. 3.1.1); all annuli by default.
    `out` = (float64, int64) device tensors of n_bins elements to write into."""
    if out is not None:
        s, c = out
        n_bins = s.numel()
        _dev(s, torch.float64, n_bins, "s_rec"), _dev(c, torch.int64, n_bins, "counts")
    else:
        n_bins = max_annulus(p.n) + 1 if n_bins is None else int(n_bins)
        s = torch.empty(n_bins, dtype=torch.float64, device=device)
        c = torch.empty(n_bins, dtype=torch.int64, device=device)
    _check(lib().scint_spectrum_rec(ctypes.byref(p), ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                    n_bins, _stream(stream)))
    return s, c


def structure_function_rec(p: ScintParams, s_rec: torch.Tensor, r_km=None, root: bool = True, workspace=None,
                           out=None, stream=None):
    """(D_rec at r_km, R_diff^rec) by Eq. crec from a spectrum on the annuli (Sect. 3.1.1).
    r_km: lags (host array or float64 device tensor); `out` = (d, root) device tensors."""
    dev = s_rec.device
    if isinstance(r_km, torch.Tensor):
        r = r_km
    else:
        r = torch.as_tensor(np.zeros(0) if r_km is None else np.asarray(r_km, dtype=np.float64), device=dev)
    r = r.to(torch.float64).contiguous()
    if out is not None:
        d, out = out
    else:
        d = torch.empty(r.numel(), dtype=torch.float64, device=dev)
        out = torch.empty(1, dtype=torch.float64, device=dev) if root else None
    if workspace is None:
        wp, wb = None, 0
    else:
        wp, wb = ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()
    _check(lib().scint_structure_function_rec(
        ctypes.byref(p), _dev(s_rec, torch.float64, s_rec.numel(), "s_rec"), s_rec.numel(),
        ctypes.c_void_p(r.data_ptr()) if r.numel() else None, r.numel(),
        ctypes.c_void_p(d.data_ptr()) if r.numel() else None,
        None if out is None else ctypes.c_void_p(out.data_ptr()), wp, wb, _stream(stream)))
    return d, out


def noise_words(p: ScintParams, stream=None, device="cuda") -> torch.Tensor:
    out = torch.empty((p.n, p.n, 4), dtype=torch.int32, device=device)
    _check(lib().scint_noise_words(ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def noise_spectrum(p: ScintParams, stream=None, device="cuda") -> torch.Tensor:
    out = torch.empty((p.n, p.n), dtype=torch.complex128, device=device)
    _check(lib().scint_noise_spectrum(ctypes.byref(p), ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def phase_fixed(phi: torch.Tensor, stream=None) -> torch.Tensor:
    """The propagation passes' fixed-point phase round(phi 2^32 / 2 pi) (int64) of a CUDA
    float64 tensor (test hook)."""
    if not (phi.is_cuda and phi.is_contiguous() and phi.dtype == torch.float64):
        raise ValueError("phi must be a contiguous float64 CUDA tensor")
    out = torch.empty(phi.shape, dtype=torch.int64, device=phi.device)
    _check(lib().scint_phase_fixed(ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   phi.numel(), _stream(stream)))
    return out


def fft_lines(x: torch.Tensor, direction: int, stream=None) -> torch.Tensor:
    """In-place line FFT of a contiguous (lines, n) complex64/complex128 CUDA tensor."""
    if not (x.is_cuda and x.is_contiguous() and x.dim() == 2):
        raise ValueError("x must be a contiguous 2-D CUDA tensor")
    n_lines, n = x.shape
    if x.dtype == torch.complex64:
        _check(lib().scint_fft_lines32(n, direction, ctypes.c_void_p(x.data_ptr()), n_lines, _stream(stream)))
    elif x.dtype == torch.complex128:
        _check(lib().scint_fft_lines64(n, direction, ctypes.c_void_p(x.data_ptr()), n_lines, _stream(stream)))
    else:
        raise ValueError("complex64 or complex128 expected")
    return x


def get_plan(n: int) -> dict:
    """The propagation plan of grid n on the current device (scint_get_plan)."""
    pl = ScintPlan()
    _check(lib().scint_get_plan(n, ctypes.byref(pl)))
    return pl.as_dict()


def set_plan(n: int, packed: int, row_twiddles: int = 2, col_twiddles: int = 1, points: int = 16):
    """Fix the propagation plan of grid n on the current device (scint_set_plan)."""
    pl = ScintPlan(packed=packed, points=points, row_twiddles=row_twiddles, col_twiddles=col_twiddles, tuned=0,
                   reserved=0, ms=0.0)
    _check(lib().scint_set_plan(n, ctypes.byref(pl)))


def tune(n: int, n_lambda: int = 32, stream=None) -> dict:
    """Time the built propagation variants for grid n and keep the fastest (scint_tune)."""
    pl = ScintPlan()
    _check(lib().scint_tune(n, n_lambda, ctypes.byref(pl), ctypes.c_void_p(_stream(stream))))
    return pl.as_dict()


def tune_batch(items, lambdas_nm, weights=None, workspace: Optional[torch.Tensor] = None, stream=None):
    """Time the batch under candidate plan sets and lane counts and keep the fastest
    (scint_tune_batch).  Returns (lanes, ms, mode); the plans of the batch's grid sizes and the
    batch mode are set."""
    arr = items if isinstance(items, ctypes.Array) else batch_items(items)
    lam = np.ascontiguousarray(lambdas_nm, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    wp, wb = (None, 0) if workspace is None else (ctypes.c_void_p(workspace.data_ptr()),
                                                  workspace.numel() * workspace.element_size())
    lanes, ms, mode = _i(0), ctypes.c_double(0.0), _i(0)
    _check(lib().scint_tune_batch(arr, len(arr), lam.ctypes.data_as(ctypes.c_void_p),
                                  None if w is None else w.ctypes.data_as(ctypes.c_void_p), len(lam), wp, wb,
                                  ctypes.byref(lanes), ctypes.byref(ms), ctypes.byref(mode), _stream(stream)))
    return lanes.value, ms.value, mode.value


def batch_mode(mode: int) -> int:
    """Batch execution form (scint_batch_mode): 0 lanes, 1 persistent propagation; returns the old one."""
    old = lib().scint_batch_mode(int(mode))
    if old < 0:
        raise ScintError(1, lib().scint_last_error().decode())
    return old


def batch_status(stream=None):
    """Raise ScintError (SCINT_ETIMEOUT) if the last persistent batch gave up a wait (scint_batch_status)."""
    _check(lib().scint_batch_status(ctypes.c_void_p(_stream(stream))))


def autotune(on: bool = True) -> bool:
    """Tune unplanned grid sizes on first use in run_batch (scint_autotune); returns the old setting."""
    return bool(lib().scint_autotune(1 if on else 0))


def release():
    lib().scint_release()


def profile_enable(on: bool = True):
    """Start (clearing old records) or stop the library's per-kernel event timing."""
    _check(lib().scint_profile_enable(int(bool(on))))


def profile_read():
    """Per kernel class: dict(launches, total_ms, bytes, flops) of the recorded launches."""
    arr = (KernelStat * 32)()
    cnt = ctypes.c_int(0)
    _check(lib().scint_profile_read(arr, 32, ctypes.byref(cnt)))
    return {arr[i].name.decode(): dict(launches=int(arr[i].launches), total_ms=float(arr[i].total_ms),
                                       bytes=float(arr[i].bytes), flops=float(arr[i].flops))
            for i in range(cnt.value)}
