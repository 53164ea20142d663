"""Shared pytest configuration.

Markers:
  gpu -- needs a CUDA device (GB300); run with ``-m gpu``.  Everything else runs
         on a CPU-only machine with ``-m "not gpu"``.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: test needs a CUDA GPU (GB300)")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    return oracle.load()
