"""The library's register FFTs (csrc/fks_fft.cuh), compiled for the host,
against numpy.fft: mixed radix 2/3/4/8 transforms and the packed C2R, in float,
double and double-float (csrc/fks_dfloat.cuh) arithmetic."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1701_01608_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("fft") / "libfft_host.so")
    cmd = ["nvcc", "-std=c++17", "-O2", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", "--expt-relaxed-constexpr",
           "-I", CSRC, os.path.join(HERE, "harness", "fft_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.fks_test_fft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P]
    lib.fks_test_c2r.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
    lib.fks_test_fft_radix.argtypes = [ctypes.c_int] * 4 + [P, P]
    return lib


TOL = {0: 1e-6, 1: 1e-14, 2: 1e-13}   # float, double, double-float (~48 bits)


@pytest.mark.parametrize("fp64", [1, 0, 2])
@pytest.mark.parametrize("n", [2, 3, 4, 8, 12, 16, 24, 32])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_numpy(harness, n, sign, fp64):
    rng = np.random.default_rng(n * 7 + sign)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    inp = np.ascontiguousarray(x).view(np.float64).copy()
    out = np.empty(2 * n)
    assert harness.fks_test_fft(n, sign, fp64, inp.ctypes.data, out.ctypes.data) == 0
    got = out.view(np.complex128)
    xin = inp.view(np.complex128) if fp64 else inp.astype(np.float32).astype(np.float64).view(np.complex128)
    want = np.fft.fft(xin) if sign < 0 else n * np.fft.ifft(xin)
    assert np.abs(got - want).max() < TOL[fp64] * np.abs(want).max()


@pytest.mark.parametrize("fp64", [1, 0, 2])
@pytest.mark.parametrize("n", [8, 16, 24, 32])
def test_c2r_matches_numpy(harness, n, fp64):
    rng = np.random.default_rng(n)
    X = rng.standard_normal(n // 2 + 1) + 1j * rng.standard_normal(n // 2 + 1)
    X[0] = X[0].real
    X[n // 2] = X[n // 2].real
    packed = np.empty(n // 2, dtype=np.complex128)
    packed[0] = X[0].real + 1j * X[n // 2].real
    packed[1:] = X[1:n // 2]
    inp = packed.view(np.float64).copy()
    out = np.empty(n)
    assert harness.fks_test_c2r(n, fp64, inp.ctypes.data, out.ctypes.data) == 0
    want = n * np.fft.irfft(X, n)
    assert np.abs(out - want).max() < TOL[fp64] * np.abs(want).max()


@pytest.mark.parametrize("prec", [1, 0, 2])
@pytest.mark.parametrize("n,r0", [(8, 2), (8, 4), (16, 2), (16, 8), (24, 2), (24, 4), (24, 8), (32, 2), (32, 8)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_radix_schedules_match_numpy(harness, n, r0, sign, prec):
    """The alternative radix schedules (top radix r0 of the n-point transform) the autotuner can
    choose give the same transform."""
    rng = np.random.default_rng(n * 31 + r0 + sign)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    inp = np.ascontiguousarray(x).view(np.float64).copy()
    out = np.empty(2 * n)
    assert harness.fks_test_fft_radix(n, r0, sign, prec, inp.ctypes.data, out.ctypes.data) == 0
    got = out.view(np.complex128)
    xin = inp.view(np.complex128) if prec else inp.astype(np.float32).astype(np.float64).view(np.complex128)
    want = np.fft.fft(xin) if sign < 0 else n * np.fft.ifft(xin)
    assert np.abs(got - want).max() < TOL[prec] * np.abs(want).max()
