import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA device (GB300) and the built library")


@pytest.fixture(scope="session")
def mfp():
    """The built CUDA library's binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_03029_gb300 import build
    build.build()
    from paper_1611_03029_gb300 import mfpoisson
    return mfpoisson


def rel_err(y, ref):
    import numpy as np
    y, ref = np.asarray(y), np.asarray(ref)
    return float(np.abs(y - ref).max() / max(np.abs(ref).max(), 1e-300))
