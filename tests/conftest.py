"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA GPU and the compiled library; run with ``-m gpu``.
Everything unmarked runs on a CPU-only machine.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: requires a CUDA GPU (GB300, sm_103a) and the built libmd")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle
