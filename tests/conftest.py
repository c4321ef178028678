import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle
    oracle.build()
    return oracle


_REPORTS = []


@pytest.fixture(scope="session")
def report():
    """report(name, record): keeps a parity record (measured errors, counts
    of checked and skipped items) for the end-of-run summary and, when
    GS_PARITY_REPORT names a file, appends it there as one JSON line."""
    import json

    path = os.environ.get("GS_PARITY_REPORT")

    def _report(name, record):
        line = json.dumps({"test": name, **record}, default=float)
        _REPORTS.append(line)
        if path:
            with open(path, "a") as f:
                f.write(line + "\n")
    return _report


def pytest_terminal_summary(terminalreporter):
    if _REPORTS:
        terminalreporter.write_sep("-", f"parity records ({len(_REPORTS)})")
        for line in _REPORTS:
            terminalreporter.write_line(line[:400])
