import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and librve.so")


@pytest.fixture(scope="session")
def lib():
    """librve.so built for sm_103a (built on first use)."""
    from paper_2402_09996_gb300 import build_lib, rve

    build_lib.build()
    return rve.load_library()


@pytest.fixture(scope="session")
def cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch.device("cuda:0")
