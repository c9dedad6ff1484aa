import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TABLE = os.path.join(ROOT, "paper_2210_05547_gb300", "data", "air5.dat")
TABLE11 = os.path.join(ROOT, "paper_2210_05547_gb300", "data", "air11.dat")
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


@pytest.fixture(scope="session")
def table():
    from oracle import gas
    return gas.load_table(TABLE)


@pytest.fixture(scope="session")
def table11():
    from oracle import gas
    return gas.load_table(TABLE11)
