import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libagcm")


@pytest.fixture(scope="session")
def cuda_ok():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True


@pytest.fixture(params=["column", "row"])
def stage_kernel(request, cuda_ok):
    """Run a GPU test with each design of the stage kernel (the row-segment
    kernel forced onto grids it would otherwise leave to the column kernel)."""
    from paper_2103_10114_gb300 import agcm

    agcm.build()
    agcm.set_stage_kernel(agcm.STAGE_COLUMN if request.param == "column" else agcm.STAGE_ROW)
    yield request.param
    agcm.set_stage_kernel(agcm.STAGE_AUTO)
