import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    """Parse a tests/golden fixture: minsup, transactions, and (flag, itemset, support) rows."""
    path = os.path.join(ROOT, "tests", "golden", name)
    minsup, txs, rows = None, [], []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("minsup"):
            minsup = int(line.split()[1])
        elif line.startswith("tx"):
            txs.append([int(v) for v in line.split(":")[1].split()])
        else:
            flag, rest = line.split(None, 1)
            items, supp = rest.split(":")
            rows.append((flag, tuple(int(v) for v in items.split()), int(supp)))
    return minsup, txs, rows


@pytest.fixture
def golden():
    return read_golden
