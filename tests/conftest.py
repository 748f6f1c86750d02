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


# FP32 parity bound.  Q = G - L is a difference of two terms of size ||L||;
# FP32 rounds both, so the attainable error is a fraction of the loss scale,
# not of Q: relative L2 <= 1e-5 wherever ||L|| / ||Q|| <= 40 (cells away from
# equilibrium), and ||dQ|| <= 2.5e-7 ||L|| / Kn in general.
FP32_REL = 1e-5
FP32_LOSS = 2.5e-7


# split-BF16 tensor-core transforms: each split keeps ~16 bits (2^-17 ~ 7.6e-6
# relative) and the errors of the products scale with the gain and loss
# magnitudes, not with Q = G - L.  Relative L2 <= 1e-3 of Q (the stated
# bound) wherever ||L|| / ||Q|| <= 40; in general ||dQ|| <= 2.5e-5 ||L|| / Kn
# (the two coincide at ||L|| / ||Q|| = 40).
BF16_REL = 1e-3
BF16_LOSS = 2.5e-5


def bf16_within(Q_gpu, Q_ref, loss_ref_over_kn):
    import numpy as np
    err = float(np.linalg.norm(np.asarray(Q_gpu) - np.asarray(Q_ref)))
    return err <= max(BF16_REL * float(np.linalg.norm(Q_ref)), BF16_LOSS * float(np.linalg.norm(loss_ref_over_kn)))


def fp32_within(Q_gpu, Q_ref, loss_ref_over_kn):
    import numpy as np
    err = float(np.linalg.norm(np.asarray(Q_gpu) - np.asarray(Q_ref)))
    return err <= max(FP32_REL * float(np.linalg.norm(Q_ref)), FP32_LOSS * float(np.linalg.norm(loss_ref_over_kn)))
