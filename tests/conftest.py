import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def built_lib():
    from paper_1901_10559_gb300 import build
    return build.build()


@pytest.fixture(scope="session")
def ctx(built_lib):
    import torch
    import paper_1901_10559_gb300 as idl
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    torch.cuda.init()
    c = idl.Context(0)
    yield c
    c.close()
