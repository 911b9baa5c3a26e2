"""GB300-native Fresnel-scintillation library (Habibi et al. 2013, arXiv:1301.0514).

The computation runs in libscint.so (hand-written CUDA for sm_103a) behind the
C ABI of include/scint.h; this package only marshals arguments to it.
"""
from ._lib import (  # noqa: F401
    MAX_CHECK_N,
    MAX_LAMBDA,
    MAX_LANES,
    BatchItem,
    ScintPlan,
    autotune,
    get_plan,
    set_plan,
    tune,
    tune_batch,
    batch_items,
    batch_workspace_bytes,
    SamplingWarning,
    ScintError,
    ScintParams,
    conjugate_pixel_km,
    curve_correlation,
    curve_modulation,
    curve_power_spectrum,
    fft_lines,
    fiducial_zone,
    last_warning,
    lib,
    lightcurve,
    lightcurve_adjoint,
    make_screen,
    max_annulus,
    modulation_index,
    noise_spectrum,
    noise_words,
    params,
    phase_fixed,
    profile_enable,
    profile_read,
    propagate,
    propagate_conjugate,
    rdiff_gradient,
    release,
    run_batch,
    sampling_ratio,
    smooth_source,
    spectrum_rec,
    structure_function_rec,
    sum_passband,
    sum_passband_conjugate,
    workspace_bytes,
)

from .autograd import light_curves, screen  # noqa: F401,E402

__version__ = "0.1.0"
