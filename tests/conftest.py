import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test taking more than a few seconds")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, loaded through the Python binding; skips without a GPU."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_00315_gb300 import capi

    return capi.load()
