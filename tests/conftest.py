import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def tgctx():
    """A library context on cuda:0 (builds libtg.so first if a source changed)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_21095_gb300 as tg

    tg.build()
    torch.zeros(1, device="cuda")  # PyTorch's runtime and context come first
    ctx = tg.tg_create(0)
    yield ctx
    tg.tg_destroy(ctx)
