"""Host-side checks of the C-ABI library (no GPU): it builds, loads, exports
every symbol include/fks.h declares, and its table arithmetic (evaluated on
the host by the same code the device table kernel runs) agrees with the
oracle's independent kernel transforms."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fks():
    from paper_1701_01608_gb300 import fks
    fks.lib()
    return fks


def test_exports_every_declared_symbol(fks):
    hdr = open(os.path.join(ROOT, "include", "fks.h")).read()
    declared = set(re.findall(r"\b(fks_[a-z_]+)\s*\(", hdr))
    assert declared, "no declarations found"
    lib = fks.lib()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(fks.EXPORTS)


@pytest.mark.parametrize("ktype", [0, 1])
@pytest.mark.parametrize("s", [0.0, 1e-6, 0.3, 1.7, 4.9, 8.2])
def test_kernel_transforms_match_oracle(fks, oracle, ktype, s):
    L = 10.0
    R = 2.0 / (3.0 + np.sqrt(2.0)) * L
    phi, psi = fks.kernel_transform(ktype, 0.25, L, s)
    assert abs(phi - oracle.phi(ktype, 0.25, R, s)) < 1e-12 * R * R
    assert abs(psi - oracle.psi(ktype, 0.25, R, s)) < 1e-12 * R * R


def test_status_strings(fks):
    lib = fks.lib()
    assert lib.fks_status_string(0) == b"ok"
    assert lib.fks_status_string(1) == b"invalid argument"
