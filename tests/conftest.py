import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_published_splitmix64():
    path = os.path.join(ROOT, "tests", "golden", "splitmix64_published.txt")
    seqs, cur = {}, None
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("seed"):
                cur = int(line.split()[1], 0)
                seqs[cur] = []
            else:
                seqs[cur].append(int(line, 0))
    return seqs


@pytest.fixture(scope="session")
def published_splitmix64():
    return load_published_splitmix64()
