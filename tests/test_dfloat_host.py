"""The double-float arithmetic (csrc/fks_dfloat.cuh) of the collision kernel's last escalation
tier, compiled for the host, against exact rational arithmetic: the sum of two pairs within
2^-44 (|a| + |b|) (the lo parts are added before one renormalisation: a normwise bound, relative
to the result when there is no cancellation), the product within 2^-45 |a b|, the conversion of
a double within 2^-48 of it, and every result normalised (|lo| <= ulp(hi) / 2).  A planted
mistake (the product error term dropped) breaks the product bound."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1701_01608_gb300", "csrc")


def _build(tmp, src_text=None):
    src = os.path.join(HERE, "harness", "dfloat_host.cu")
    inc = CSRC
    if src_text is not None:   # a planted mistake in a scratch copy of the header
        d = tmp / "planted"
        d.mkdir()
        (d / "fks_dfloat.cuh").write_text(src_text)
        inc = str(d)
    out = str(tmp / ("libdd_planted.so" if src_text else "libdd.so"))
    cmd = ["nvcc", "-std=c++17", "-O2", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
           "--expt-relaxed-constexpr", "-I", inc, "-I", CSRC, src, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    F = ctypes.c_float
    for fn in ("fks_test_dd_add", "fks_test_dd_mul"):
        getattr(lib, fn).argtypes = [F, F, F, F, ctypes.c_void_p]
    lib.fks_test_dd_from_double.argtypes = [ctypes.c_double, ctypes.c_void_p]
    lib.fks_test_dd_dot2.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.fks_test_dd_lazy4.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    return lib


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    return _build(tmp_path_factory.mktemp("dd"))


def pair(rng, scale=1.0):
    x = rng.standard_normal() * scale
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return float(hi), float(lo)


def call(fn, a, b):
    out = np.zeros(2, dtype=np.float32)
    fn(a[0], a[1], b[0], b[1], out.ctypes.data)
    return float(out[0]), float(out[1])


def exact(p):
    return Fraction(p[0]) + Fraction(p[1])


def normalised(r):
    hi, lo = r
    if hi == 0.0:
        return lo == 0.0
    return abs(lo) <= float(np.spacing(np.float32(abs(hi)))) / 2


def cases(seed, n=400):
    rng = np.random.default_rng(seed)
    for i in range(n):
        a = pair(rng, 10.0 ** rng.uniform(-3, 3))
        kind = i % 4
        if kind == 0:
            b = pair(rng, 10.0 ** rng.uniform(-3, 3))
        elif kind == 1:   # near cancellation in the sum (b normalised: |lo| <= |a.lo|)
            b = (-a[0], float(np.float32(a[1] * rng.uniform(-1.0, 1.0))))
        elif kind == 2:   # same hi, opposite lo: the result is the lo parts alone
            b = (-a[0], -a[1] * 0.5)
        else:             # very different magnitudes
            b = pair(rng, 1e-6)
        yield a, b


def test_sum_within_normwise_bound(lib):
    for a, b in cases(1):
        r = call(lib.fks_test_dd_add, a, b)
        err = abs(exact(r) - (exact(a) + exact(b)))
        assert err <= Fraction(2) ** -44 * (abs(exact(a)) + abs(exact(b))), (a, b, r)
        assert normalised(r), (a, b, r)


def test_sum_without_cancellation_is_relative(lib):
    rng = np.random.default_rng(2)
    for _ in range(300):
        a, b = pair(rng), pair(rng)
        b = (abs(b[0]), b[1]) if a[0] > 0 else (-abs(b[0]), -b[1])   # same sign: no cancellation
        r = call(lib.fks_test_dd_add, a, b)
        s = exact(a) + exact(b)
        assert abs(exact(r) - s) <= Fraction(2) ** -46 * abs(s)


def test_product_within_relative_bound(lib):
    for a, b in cases(3):
        r = call(lib.fks_test_dd_mul, a, b)
        p = exact(a) * exact(b)
        assert abs(exact(r) - p) <= Fraction(2) ** -45 * abs(p), (a, b, r)
        assert normalised(r)


def dot2(fn, a, b, c, d):
    inp = np.array([*a, *b, *c, *d], dtype=np.float32)
    out = np.zeros(2, dtype=np.float32)
    fn(inp.ctypes.data, out.ctypes.data)
    return float(out[0]), float(out[1])


def dot2_cases(seed, n=400):
    """(a, b, c, d) with a b + c d generic, cancelling (c d = -a b up to the low parts) or lopsided."""
    rng = np.random.default_rng(seed)
    for i in range(n):
        a = pair(rng, 10.0 ** rng.uniform(-2, 2))
        b = pair(rng, 10.0 ** rng.uniform(-2, 2))
        kind = i % 3
        if kind == 0:
            c, d = pair(rng, 10.0 ** rng.uniform(-2, 2)), pair(rng, 10.0 ** rng.uniform(-2, 2))
        elif kind == 1:   # complex product with a twiddle of modulus one: near cancellation
            c, d = (-a[0], float(np.float32(a[1] * rng.uniform(-1, 1)))), b
        else:
            c, d = pair(rng, 1e-5), pair(rng)
        yield a, b, c, d


def test_dot2_within_normwise_bound(lib):
    """The fused a b + c d of the complex products: error below 2^-45 (|a b| + |c d|), normalised."""
    for a, b, c, d in dot2_cases(6):
        r = dot2(lib.fks_test_dd_dot2, a, b, c, d)
        ab, cd = exact(a) * exact(b), exact(c) * exact(d)
        assert abs(exact(r) - (ab + cd)) <= Fraction(2) ** -45 * (abs(ab) + abs(cd)), (a, b, c, d, r)
        assert normalised(r), (a, b, c, d, r)


def test_unnormalised_inner_sums_keep_the_normwise_bound(lib):
    """(a + b) + (c - d) with the inner sums left unnormalised: error below 2^-44 of the sum of the
    magnitudes (cancelling, lopsided and generic operands), the result normalised."""
    for (a, b), (c, d) in zip(cases(8), cases(9)):
        r = dot2(lib.fks_test_dd_lazy4, a, b, c, d)
        want = exact(a) + exact(b) + exact(c) - exact(d)
        mag = abs(exact(a)) + abs(exact(b)) + abs(exact(c)) + abs(exact(d))
        assert abs(exact(r) - want) <= Fraction(2) ** -44 * mag, (a, b, c, d, r)
        assert normalised(r), (a, b, c, d, r)


def test_planted_mistake_breaks_dot2_bound(tmp_path):
    """Without the cross terms of the low parts the dot product is only single precision."""
    text = open(os.path.join(CSRC, "fks_dfloat.cuh")).read()
    planted = text.replace("    t = fmaf(a.lo, b.hi, t);\n", "")
    assert planted != text
    bad = _build(tmp_path, planted)
    worst = Fraction(0)
    for a, b, c, d in dot2_cases(7, 100):
        r = dot2(bad.fks_test_dd_dot2, a, b, c, d)
        ab, cd = exact(a) * exact(b), exact(c) * exact(d)
        worst = max(worst, abs(exact(r) - (ab + cd)) / (abs(ab) + abs(cd)))
    assert worst > Fraction(2) ** -40


def test_from_double(lib):
    rng = np.random.default_rng(4)
    for x in list(rng.standard_normal(200) * 10.0 ** rng.uniform(-5, 5, 200)) + [np.pi, 1e-30, -7.0]:
        out = np.zeros(2, dtype=np.float32)
        lib.fks_test_dd_from_double(float(x), out.ctypes.data)
        r = (float(out[0]), float(out[1]))
        assert abs(exact(r) - Fraction(float(x))) <= Fraction(2) ** -48 * abs(Fraction(float(x)))
        assert normalised(r)


def test_planted_mistake_breaks_product_bound(tmp_path):
    text = open(os.path.join(CSRC, "fks_dfloat.cuh")).read()
    planted = text.replace("    float e = fmaf(a.hi, b.hi, -p);   // exact: p + e = a.hi b.hi",
                           "    float e = 0.0f;")
    assert planted != text
    bad = _build(tmp_path, planted)
    worst = Fraction(0)
    for a, b in cases(5, 100):
        r = call(bad.fks_test_dd_mul, a, b)
        p = exact(a) * exact(b)
        if p != 0:
            worst = max(worst, abs(exact(r) - p) / abs(p))
    assert worst > Fraction(2) ** -45
