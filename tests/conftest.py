import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def ctx():
    """A liblch context on cuda:0 (GPU tests only)."""
    import torch

    from paper_1404_3458_gb300 import build as B
    from paper_1404_3458_gb300 import lch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    c = lch.Context(0)
    yield c
    c.close()
