"""Test configuration: the ``gpu`` marker selects tests that need a CUDA device and the built library.

Run the CPU suite with ``pytest -m "not gpu"`` and the device parity suite with ``pytest -m gpu``.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the compiled library")
    config.addinivalue_line("markers", "timeout(seconds): per-test time limit (pytest-timeout, when installed)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Print the measured ambiguity shares and plain gradient pass rates of the parity tests."""
    try:
        from helpers import REPORT
    except ImportError:
        return
    if not REPORT:
        return
    tr = terminalreporter
    tr.section("parity measurements")
    for kind, test, what, value, limit in REPORT:
        op = "<" if kind.startswith("ambiguous") else ">="
        tr.write_line(f"{kind:22s} {value:.6f} ({op} {limit:g})  {test}  {what}")
