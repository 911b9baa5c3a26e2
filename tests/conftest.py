import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled scint library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    """Rows of a whitespace-separated golden file, comments stripped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def golden():
    return read_golden


_PARAM_KEYS = ("n", "pixel_km", "r_diff_km", "beta", "lambda_nm", "lambda_ref_nm", "z_pc",
               "source_radius_km", "seed", "screen_id", "margin_km")


def oracle_params(item, **kw):
    """Workload record -> oracle ScreenParams."""
    import oracle as O
    d = {k: item[k] for k in _PARAM_KEYS}
    d.update(kw)
    return O.ScreenParams(**d)


def gpu_params(item, **kw):
    """Workload record -> library ScintParams."""
    import paper_1301_0514_gb300 as S
    d = {k: item[k] for k in _PARAM_KEYS}
    d.update(kw)
    return S.params(**d)
