import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library's binding; fails (not skips) when the extension is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a test marked gpu ran without a visible CUDA device")
    import paper_2208_12350_gb300 as swgb
    swgb.load()
    return swgb
