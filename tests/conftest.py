import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_sessionstart(session):
    # Build the CUDA library and the oracle's C library in-tree if stale (fast;
    # the same step __graft_entry__.build() runs).
    from paper_1208_0274_gb300 import build as b
    b.build()
    import oracle
    oracle.build()
