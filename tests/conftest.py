import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


@pytest.fixture(scope="session")
def O():
    from oracle import oracle as _O

    _O.lib()
    return _O


@pytest.fixture(scope="session")
def I():
    from paper_2106_00282_gb300 import inputs as _I

    return _I
