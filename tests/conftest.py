import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def built_lib():
    """Build libcbp.so in-tree if needed (nvcc works without a GPU)."""
    from paper_1203_4874_gb300 import build
    build.build()
    from paper_1203_4874_gb300 import cbp
    return cbp.lib()


@pytest.fixture(scope="session")
def gpu_ctx(built_lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_4874_gb300 import cbp
    torch.cuda.init()
    ctx = cbp.cbp_create(0, 0)
    yield ctx
    cbp.cbp_destroy(ctx)
