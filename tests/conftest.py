"""Shared pytest configuration.

Markers (registered in pytest.ini):
  gpu  -- needs a CUDA device (GB300, sm_103a); a CPU-only run deselects
          these with ``-m "not gpu"``.  They fail, not skip, without a GPU.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle
