"""Shared pytest configuration.

Markers: ``gpu`` -- needs a CUDA device (parity tests through the C ABI).
Everything else runs on CPU.  The oracle under ``oracle/`` is compiled once
per session on first use.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (parity tests through the C ABI)")
    config.addinivalue_line("markers", "slow: statistical tests that take more than a few seconds")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
