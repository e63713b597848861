import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled libblsh")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def B():
    """The libblsh binding; builds the library if it is missing."""
    import paper_1110_1328_gb300 as B
    from paper_1110_1328_gb300 import build as _b
    _b.build()
    return B


@pytest.fixture(scope="session")
def ctx(B):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return B.Context(0)
