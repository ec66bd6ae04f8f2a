import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def lib():
    """The product library through its Python binding (GPU tests only)."""
    import paper_2605_04178_gb300 as pm
    return pm


@pytest.fixture(params=[0, 1], ids=["literal", "measured"])
def reading(request):
    """Runs a test under each reading of the stage model's open points (the
    literal equations, and the readings measured on the GPU's kernels), in the
    oracle and, when the library is loaded, in the library; restores the
    literal default afterwards."""
    import oracle as O
    O.set_reading(request.param)
    pm = sys.modules.get("paper_2605_04178_gb300")
    if pm is not None:
        pm.pm_model_set_reading(request.param)
    yield request.param
    O.set_reading(1)
    if pm is not None:
        pm.pm_model_set_reading(1)
