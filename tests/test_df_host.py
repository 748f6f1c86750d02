"""The compensated FP32 sums (csrc/fks_df.cuh) of the collision epilogue, the moments, the
single-read BGK kernel and the variant-B truncation, compiled for the host and held to the
published error bounds of compensated summation (Ogita, Rump and Oishi, "Accurate sum and dot
product", SIAM J. Sci. Comput. 26 (2005): Sum2 and Dot2), against exactly rounded sums."""
import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1701_01608_gb300", "csrc")
U = 2.0 ** -24                      # unit roundoff of FP32


def gamma(k):
    return k * U / (1 - k * U)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("df") / "libdf_host.so")
    cmd = ["nvcc", "-std=c++17", "-O2", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
           "-I", CSRC, os.path.join(HERE, "harness", "df_host.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.fks_test_df_sum.argtypes = [P, I, P]
    lib.fks_test_df_dot.argtypes = [P, P, P, I, P]
    lib.fks_test_df_tree.argtypes = [P, P, I, P]
    lib.fks_test_df_tree2.argtypes = [P, P, I, P]
    lib.fks_test_df_mul.argtypes = [ctypes.c_float] * 4 + [P]
    return lib


def _call(fn, *args):
    out = ctypes.c_double()
    assert fn(*args, ctypes.byref(out)) == 0
    return out.value


def _ill_conditioned(rng, n):
    """Large terms that cancel plus small ones: the sum is far below the sum of magnitudes."""
    big = rng.standard_normal(n // 2) * 1e4
    x = np.concatenate([big, -big * (1 + rng.standard_normal(n // 2) * 1e-6),
                        rng.standard_normal(n - 2 * (n // 2))])
    rng.shuffle(x)
    return x.astype(np.float32)


@pytest.mark.parametrize("n", [1, 7, 256, 4096])
@pytest.mark.parametrize("kind", ["normal", "positive", "ill"])
def test_sum_within_sum2_bound(harness, n, kind):
    """Sum2: |res - s| <= u|s| + gamma_{n-1}^2 sum|x|; the result is read as hi + lo in FP64, so
    the u|s| term (the final rounding to FP32) becomes the FP64 rounding of hi + lo."""
    rng = np.random.default_rng(n + len(kind))
    x = {"normal": lambda: rng.standard_normal(n),
         "positive": lambda: rng.random(n) * 10 ** rng.uniform(-3, 3, n),
         "ill": lambda: _ill_conditioned(rng, n)}[kind]().astype(np.float32)
    exact = math.fsum(x.astype(np.float64))
    got = _call(harness.fks_test_df_sum, x.ctypes.data, n)
    abs_sum = float(np.abs(x.astype(np.float64)).sum())
    bound = gamma(n - 1) ** 2 * abs_sum + 2.0 ** -52 * abs(exact)
    assert abs(got - exact) <= bound
    if kind == "ill" and n >= 256:
        naive = float(np.float32(0))
        for v in x:
            naive = float(np.float32(naive) + v)
        # the plain FP32 loop loses the small terms; the compensated one keeps them
        assert abs(naive - exact) > 1e3 * max(abs(got - exact), 1e-30)


def test_sum_cancellation_exact(harness):
    """2^24 + 1 - 2^24: the plain FP32 sum is 0, the compensated one exactly 1."""
    x = np.array([2.0 ** 24, 1.0, -2.0 ** 24], dtype=np.float32)
    assert _call(harness.fks_test_df_sum, x.ctypes.data, 3) == 1.0


@pytest.mark.parametrize("n", [32, 1024, 4096])
def test_dot_within_dot2_bound(harness, n):
    """Dot2 with weights carried as (hi, lo) pairs, as the moment sums carry v and v^2/2:
    |res - x.w| <= u|x.w| + gamma_n^2 |x|.|w|, the lo products adding one more gamma_1 u term."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n).astype(np.float32)
    w = rng.uniform(-8, 8, n)                       # FP64 weights, split into hi + lo
    wh = w.astype(np.float32)
    wl = (w - wh.astype(np.float64)).astype(np.float32)
    xd = x.astype(np.float64)
    # x * wh and x * wl are exact in FP64 (24 x 24 bits), so fsum rounds the exact value once
    exact = math.fsum(list(xd * wh.astype(np.float64)) + list(xd * wl.astype(np.float64)))
    got = _call(harness.fks_test_df_dot, x.ctypes.data, wh.ctypes.data, wl.ctypes.data, n)
    mag = float(np.abs(xd * w).sum())
    bound = U * U * abs(exact) + gamma(n + 1) ** 2 * mag + U * U * mag
    assert abs(got - exact) <= bound
    naive = float(np.dot(x, wh))                    # plain FP32 dot for contrast
    assert abs(naive - exact) > 10 * abs(got - exact)


@pytest.mark.parametrize("fn", ["fks_test_df_tree", "fks_test_df_tree2"])
@pytest.mark.parametrize("n", [2, 5, 32, 1000])
def test_pairwise_tree_of_pairs(harness, fn, n):
    """The warp-shuffle reduction order: a binary tree of pair sums, L = ceil(log2 n) levels.  A
    node's hi sum is exact (two-sum); its lo sum takes two roundings of |a.lo| + |e| + |b.lo|, with
    |e| <= u S and |lo| <= u d S + (sum of leaf lo) for the S of the node's subtree of depth d.
    Over the L levels the error is at most 2 L (L + 1) u^2 M + 2 L u Lambda (first order), with M
    the sum of magnitudes of all parts and Lambda that of the leaf lo parts."""
    rng = np.random.default_rng(n + len(fn))
    hi = _ill_conditioned(rng, n)
    lo = (hi.astype(np.float64) * rng.uniform(-1, 1, n) * 2.0 ** -25).astype(np.float32)
    exact = math.fsum(list(hi.astype(np.float64)) + list(lo.astype(np.float64)))
    got = _call(getattr(harness, fn), hi.ctypes.data, lo.ctypes.data, n)
    mag_lo = float(np.abs(lo.astype(np.float64)).sum())
    mag = float(np.abs(hi.astype(np.float64)).sum()) + mag_lo
    L = max(1, math.ceil(math.log2(n)))
    bound = 1.01 * (2 * L * (L + 1) * U * U * mag + 2 * L * U * mag_lo) + 2.0 ** -52 * abs(exact)
    assert abs(got - exact) <= bound


def test_tree_rejects_oversize(harness):
    x = np.zeros(1025, dtype=np.float32)
    out = ctypes.c_double()
    assert harness.fks_test_df_tree(x.ctypes.data, x.ctypes.data, 1025, ctypes.byref(out)) == 1


def test_mul_relative_error(harness):
    """(ah + al)(bh + bl) with |al| <= u|ah|, |bl| <= u|bh|: relative error at most 4 u^2 (the
    dropped al bl term and two roundings of the lo sum), checked in exact rational arithmetic."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(2000):
        a, b = rng.standard_normal(2) * 10 ** rng.uniform(-5, 5, 2)
        ah, bh = np.float32(a), np.float32(b)
        al, bl = np.float32(a - float(ah)), np.float32(b - float(bh))
        got = _call(harness.fks_test_df_mul, float(ah), float(al), float(bh), float(bl))
        exact = (Fraction(float(ah)) + Fraction(float(al))) * (Fraction(float(bh)) + Fraction(float(bl)))
        rel = abs(Fraction(got) - exact) / abs(exact)
        worst = max(worst, float(rel))
    assert worst <= 4 * U * U
