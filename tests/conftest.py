import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    """Rows of a tab-separated golden file under tests/golden (comments and
    the header line skipped), as lists of ints/floats."""
    path = os.path.join(ROOT, "tests", "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split("\t")
            try:
                rows.append([int(p) if p.lstrip("-").isdigit() else float(p) for p in parts])
            except ValueError:
                continue  # header
    return rows


@pytest.fixture(scope="session")
def table1():
    return {n: m for n, m in read_golden("table1.txt")}
