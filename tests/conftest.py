import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libfe.so")
    config.addinivalue_line("markers", "slow: larger CPU case (still minutes at most)")


def pytest_collection_modifyitems(config, items):
    # GPU tests fail loudly (not skip) when the GPU is missing but selected;
    # on a CPU-only box run them only when explicitly asked with -m gpu.
    pass
