import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: longer CPU test")
    # PyTorch's notices that two of its APIs the tests use for checks (index_reduce_, sparse CSR
    # tensors) are in beta
    config.addinivalue_line("filterwarnings", "ignore:index_reduce\\(\\) is in beta:UserWarning")
    config.addinivalue_line("filterwarnings", "ignore:Sparse CSR tensor support is in beta:UserWarning")
