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


# full-size oracle runs shared by the FP64 and FP32-bulk parity tests of the
# benchmark workloads (each takes from seconds to minutes of host time)
FULL_SIZE_STEPS = {"impact": 100, "conduction": 20}
_full_size_cache = {}


@pytest.fixture(scope="session")
def oracle_full_size(O, I):
    """oracle_full_size(which) -> (workload, U after FULL_SIZE_STEPS[which]
    oracle steps from the initial state, status word)."""

    def run(which):
        if which not in _full_size_cache:
            wl = I.impact() if which == "impact" else I.conduction_disc()
            Uo, st, dto, ph = O.step(wl.params, O.from_primitive(wl.params, wl.prim), wl.dx, wl.dy,
                                     FULL_SIZE_STEPS[which])
            _full_size_cache[which] = (wl, Uo, st)
        return _full_size_cache[which]

    return run
