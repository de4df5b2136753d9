import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libpamd.so")
    config.addinivalue_line("markers", "slow: long-running statistical or full-size check")


def pytest_addoption(parser):
    parser.addoption("--parity-report", default=None,
                     help="write the measured errors of the GPU path against the oracle, "
                          "per workload, to this JSON file")


class ParityReport:
    """Largest error seen per workload and quantity (relative errors of S, of the
    gradient in 2-norm and in max-abs, finite differences, ...), with the test that
    measured it."""

    def __init__(self):
        self.rows = {}

    def record(self, workload: str, test: str, **errors):
        row = self.rows.setdefault(workload, {})
        for key, val in errors.items():
            val = float(val)
            old = row.get(key)
            if old is None or val > old["value"]:
                row[key] = {"value": val, "test": test}


@pytest.fixture(scope="session")
def parity_report(request):
    rep = ParityReport()
    yield rep
    path = request.config.getoption("--parity-report")
    if path and rep.rows:
        with open(path, "w") as fh:
            json.dump(rep.rows, fh, indent=1, sort_keys=True)
