import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: full-size workload (minutes)")


@pytest.fixture(scope="session", autouse=True)
def _host_libs():
    """The generator and the oracle are plain C/C++ compiled with gcc on first use."""
    import synth
    import oracle
    synth.build()
    oracle.build()
    yield
