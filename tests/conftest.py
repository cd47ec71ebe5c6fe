import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _default_dtype_guard(request):
    """A GPU test must start with torch's stock float32 default dtype: a module
    that changes the default for its own tests restores it, and this guard makes
    a leak fail loudly at the first GPU test it would reach."""
    if "gpu" in request.keywords:
        import torch
        assert torch.get_default_dtype() == torch.float32, (
            f"torch default dtype leaked into a GPU test: {torch.get_default_dtype()}")
    yield
