import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle pin (still CPU-only)")


_REPORT = []


@pytest.fixture
def report():
    """Lines a test wants shown in the run's summary (measured figures)."""
    return _REPORT


def pytest_terminal_summary(terminalreporter):
    if _REPORT:
        terminalreporter.write_sep("-", "measured")
        for line in _REPORT:
            terminalreporter.write_line(line)
