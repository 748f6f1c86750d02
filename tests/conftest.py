import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libfks.so")
    config.addinivalue_line("markers", "slow: oracle work of more than a few seconds")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.build()
    return O


# Parity bounds: relative L2 of Q per cell against the FP64 oracle.  The FP32
# and split-BF16 paths meet them on every cell through their precision
# escalation (cells whose error bound exceeds the tolerance are recomputed at
# higher precision), including cells near equilibrium where the gain and the
# loss cancel.
FP64_REL = 1e-10
FP32_REL = 1e-5
BF16_REL = 1e-3
