import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size case, minutes of CPU oracle time")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O

    O.lib()
    return O


def pytest_collection_finish(session):
    """Start the minutes-long oracle runs of the target-size tests in spawned
    processes as soon as one of those tests is selected (and a GPU is
    present), so that they overlap the GPU tests that run before them."""
    if not any("test_gpu_target" in it.nodeid for it in session.items):
        return
    try:
        import torch

        if not torch.cuda.is_available():
            return
    except Exception:
        return
    import target_oracle

    target_oracle.start()
