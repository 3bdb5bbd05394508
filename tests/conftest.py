import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def load_paper_table(section):
    """Rows of tests/golden/paper_example1_iterations.txt: {p: (mg[6], gmres[6])}."""
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_example1_iterations.txt")
    rows, cur = {}, None
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                continue
            if cur != section:
                continue
            tok = line.split()
            vals = [None if t == "*" else int(t) for t in tok[1:]]
            rows[int(tok[0])] = (vals[:6], vals[6:])
    return rows
