import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libprobesim.so")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


NODES = "abcdefgh"


def load_toy():
    src, dst = [], []
    with open(os.path.join(GOLDEN, "toy_graph.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            a, b = line.split()
            src.append(NODES.index(a))
            dst.append(NODES.index(b))
    return 8, np.array(src, np.int32), np.array(dst, np.int32)


def load_printed():
    rows = []
    with open(os.path.join(GOLDEN, "toy_printed.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            kind, path, node, val, tol = line.split()[:5]
            rows.append((kind, [NODES.index(x) for x in path.split(",")], NODES.index(node), float(val), float(tol)))
    return rows


@pytest.fixture(scope="session")
def toy():
    return load_toy()


@pytest.fixture(scope="session")
def printed():
    return load_printed()
