import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def sf():
    """The CUDA library binding (built in-tree).  Only for gpu-marked tests."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_04148_gb300 as sfpkg
    sfpkg.load()
    return sfpkg
