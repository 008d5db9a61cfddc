import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built librexi")


@pytest.fixture(scope="session")
def golden():
    """Values printed in the paper, parsed from tests/golden/paper_values.txt."""
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=", 1)
                vals[k.strip()] = float(v)
    return vals
