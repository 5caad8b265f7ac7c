import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@pytest.fixture(scope="session", autouse=True)
def _built_libraries(request):
    """Build the CUDA library (when GPU tests are selected) and the oracle once."""
    if any(item.get_closest_marker("gpu") for item in request.session.items):
        from paper_1611_02967_gb300 import build as lib_build
        lib_build.build()
    from oracle import build as oracle_build
    oracle_build.build()
