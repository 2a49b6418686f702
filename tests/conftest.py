import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_printed_values():
    """key = value pairs of tests/golden/printed_values.txt."""
    out = {}
    with open(os.path.join(GOLDEN, "printed_values.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = [s.strip() for s in line.split("=")]
            out[k] = float(v)
    return out


@pytest.fixture(scope="session")
def printed():
    return read_printed_values()
