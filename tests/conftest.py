import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2201_01446_gb300 import inputs  # noqa: E402


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


# copper model of the paper's shape (embedding 1-32-64-128, M<=16, fitting
# 2048-240-240-240-1); std 0.1 is the configured synthetic model, std 1.0 a
# stress model whose forces are O(0.1-1) eV/A so that error bounds bite
CU_RC, CU_RCS, CU_SEL = 8.0, 0.5, 256
CU_SMAX = 2.0  # table domain s <= 2 (r >= 0.5 A)
TABLE_H = 0.01


@pytest.fixture(scope="session")
def model_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("models")


@pytest.fixture(scope="session")
def cu_model_path(model_dir):
    p = model_dir / "cu_std0.1.model"
    inputs.write_seeded_model(p, inputs.COPPER_SPEC, seed=0, std=0.1)
    return str(p)


@pytest.fixture(scope="session")
def cu_stress_path(model_dir):
    p = model_dir / "cu_std1.0.model"
    inputs.write_seeded_model(p, inputs.COPPER_SPEC, seed=0, std=1.0)
    return str(p)


@pytest.fixture(scope="session")
def water_model_path(model_dir):
    p = model_dir / "water_std1.0.model"
    inputs.write_seeded_model(p, inputs.WATER_SPEC, seed=4, std=1.0)
    return str(p)


F_ABS = 1e-5  # eV/A: the stated force RMSE tolerance of the FP32 path
F_REL = 1e-3  # at most this fraction of the reference RMS force


def force_bar(frms):
    """Force-RMSE bar of the configured models: the stated 1e-5 eV/A, and no
    more than 1e-3 of the reference RMS force.  The configured N(0, 0.1)
    models exert only 1e-6-1e-4 eV/A, below the absolute bar, where a kernel
    returning F = 0 (RMSE = RMS force) would pass it; with the relative cap the
    bar is below the RMS force by construction, which this asserts.  A
    reference without any force gives a bar of 0 (exact zeros expected)."""
    if frms == 0.0:
        return 0.0
    bar = min(F_ABS, F_REL * frms)
    assert bar < frms, (bar, frms)
    return bar


def rmse(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.sqrt(np.mean((a - b) ** 2))) if a.size else 0.0


# measured parity errors, written to $DP_PARITY_REPORT (JSON) when set
PARITY_LOG = []


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("DP_PARITY_REPORT")
    if path and PARITY_LOG:
        import json
        with open(path, "w") as f:
            json.dump(PARITY_LOG, f, indent=1)
