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


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.0, -1.0])
@pytest.mark.parametrize("prec,tol", [(1, 1e-7), (0, 1e-10)])
def test_vhs_expansion_matches_oracle_factor(fks, oracle, alpha, prec, tol):
    """The library's separable expansion of the VHS radial factor H(t, u)
    (eigen-decomposition on its own radial rule, truncated at the precision's
    tolerance) against the oracle's product quadrature of the definition, on
    frequencies of the 32^3 grid of [-10, 10]^3."""
    L, n = 10.0, 32
    R = 2.0 / (3.0 + np.sqrt(2.0)) * L
    tmax = np.pi / L * (n / 2) * np.sqrt(3.0)
    href = abs(oracle.vhs_h(alpha, 0.25, R, 0.0, 0.0))
    rng = np.random.default_rng(7)
    pts = [(0.0, 0.0), (tmax, tmax), (0.0, tmax)] + [tuple(rng.uniform(0, tmax, 2)) for _ in range(6)]
    for t, u in pts:
        H, S, est = fks.vhs_factor(alpha, 0.25, L, n, prec, 0, t, u)
        assert abs(H - oracle.vhs_h(alpha, 0.25, R, t, u)) <= tol * href, (t, u, S)
    # hard spheres are one separable term; the others need several
    assert (S == 1) == (alpha == 1.0)


def test_vhs_expansion_term_count_and_errors(fks):
    L, n = 10.0, 32
    H8, S8, e8 = fks.vhs_factor(0.0, 0.25, L, n, 1, 8, 0.5, 0.5)
    H4, S4, e4 = fks.vhs_factor(0.0, 0.25, L, n, 1, 4, 0.5, 0.5)
    assert (S8, S4) == (8, 4) and e8 < e4
    Ha, Sa, ea = fks.vhs_factor(0.0, 0.25, L, n, 1, 0, 0.5, 0.5)
    Hd, Sd, ed = fks.vhs_factor(0.0, 0.25, L, n, 0, 0, 0.5, 0.5)
    assert ea <= 1e-7 and ed <= 1e-12 and Sd > Sa
    for bad in ((1.5, 0), (-1.5, 0), (0.0, 65), (0.0, -1)):
        with pytest.raises(fks.FKSError):
            fks.vhs_factor(bad[0], 0.25, L, n, 1, bad[1], 0.5, 0.5)


def test_null_context_is_rejected_before_any_device_work(fks):
    """Every context call checks its handle first (FKS_ERR_INVALID_ARG, no CUDA call)."""
    import ctypes
    lib = fks.lib()
    bits = ctypes.c_int()
    assert lib.fks_collide(None, None, None, None) == 1
    assert lib.fks_transport(None, None, None, 0.0, None) == 1
    assert lib.fks_step(None, None, None, 0.0, None) == 1
    assert lib.fks_step_strang(None, None, None, None, 0.0, None) == 1
    assert lib.fks_step_host(None, None, None, 0.0, None) == 1
    assert lib.fks_moments(None, None, None, None) == 1
    assert lib.fks_check(None, None, ctypes.byref(bits)) == 1
    assert lib.fks_set_cluster_size(None, 8) == 1
    assert lib.fks_get_offsets(None, None) == 1
    assert lib.fks_set_offsets(None, None) == 1
    lib.fks_destroy(None)   # a no-op


@pytest.mark.parametrize("change,status", [
    (dict(nx=0), 1), (dict(nx=2048, ny=2048, nz=1024), 1), (dict(n=12), 2), (dict(ktype=7), 1),
    (dict(ktype=3, alpha=1.5), 1), (dict(ktype=3, alpha=-1.5), 1), (dict(ktype=3, terms=65), 1),
    (dict(knudsen=0.0), 1), (dict(A1=128, A2=64), 1), (dict(rule=2), 1), (dict(prec=9), 2),
    (dict(prec=2, ktype=2), 2), (dict(prec=2, n=8), 2), (dict(L=-1.0), 1), (dict(bc=3), 1),
])
def test_init_rejects_invalid_configurations_before_any_device_work(fks, change, status):
    """fks_init validates every argument before it touches the device (no GPU needed)."""
    import ctypes
    p = dict(nx=2, ny=2, nz=2, n=16, L=8.0, ktype=0, C=0.25, knudsen=1.0, alpha=1.0, terms=0,
             A1=4, A2=4, rule=0, prec=1, bc=0)
    p.update(change)
    g = fks._Grid(p["nx"], p["ny"], p["nz"], (ctypes.c_double * 3)(0, 0, 0), (ctypes.c_double * 3)(1, 1, 1),
                  (ctypes.c_int * 3)(p["bc"], 0, 0))
    vb = fks._VBox(p["n"], p["L"])
    k = fks._Kernel(p["ktype"], p["C"], p["knudsen"], p["alpha"], p["terms"])
    d = fks._Dirs(p["A1"], p["A2"], p["rule"])
    h = ctypes.c_void_p()
    st = fks.lib().fks_init(ctypes.byref(g), ctypes.byref(vb), ctypes.byref(k), ctypes.byref(d), p["prec"],
                            ctypes.byref(h))
    assert st == status and not h.value


def test_no_cpu_fallback_without_a_gpu(fks):
    """With no CUDA device the product path fails loudly: a valid context, batch or network cannot be
    created (FKS_ERR_CUDA from the library, raised by the binding), and the binding accepts only CUDA
    tensors.  Nothing computes on the CPU instead."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(fks.FKSError) as e:
        fks.Context(fks.Config(ncell=(2, 1, 1), n=16, L=8.0, precision=fks.FKS_FP32))
    assert e.value.status == 4   # the first device call fails with a CUDA error
    with pytest.raises(TypeError):
        fks._dptr(torch.zeros(16 ** 3), torch.float32)
    with pytest.raises(fks.FKSError) as e:
        fks.Net(16, 2, seed=0)
    assert e.value.status == 4   # a failed allocation reports its CUDA cause, not "out of memory"
