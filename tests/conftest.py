import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def sigma_grid():
    # The 6-level roughness grid the workloads use (Eq. 8 reading: sigma = 0
    # is a delta lobe, so the grid starts at 0.02, the value Fig. 3 shows).
    return [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]
