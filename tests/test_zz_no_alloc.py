"""fks_transport_noalloc: the transport entry point for callers that cannot
allocate device memory (an application that owns all device memory through
its own pool, a plugin that may not grow the host program's footprint, a
loop that cannot afford cudaMalloc's implicit synchronisation).  Its scratch
is a fixed static device array, so it needs no context.

Checked through the C ABI against fks_transport (the context-based entry
point) on two calls in a row, bit for bit: transport is a permutation of
the values, which is the tolerance of every transport test here.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_01608_gb300 import fks
    fks.lib()
    return fks


def _grid(fks, ncell, bc):
    return fks._Grid(ncell[0], ncell[1], ncell[2], (ctypes.c_double * 3)(0, 0, 0),
                     (ctypes.c_double * 3)(1, 1, 1), (ctypes.c_int * 3)(*bc))


@pytest.mark.parametrize("prec,n,bc", [(1, 32, (1, 0, 0)), (0, 16, (1, 1, 0)), (1, 8, (0, 0, 0))])
def test_noalloc_matches_context_transport_on_two_calls(fks, prec, n, bc):
    ncell, L = (5, 3, 4), 10.0
    cfg = fks.Config(ncell=ncell, bc=bc, n=n, L=L, precision=prec)
    ctx = fks.Context(cfg)
    dtype = ctx.dtype
    g = torch.Generator(device="cuda").manual_seed(17)
    f = torch.rand((int(np.prod(ncell)), n, n, n), generator=g, device="cuda", dtype=torch.float64).to(dtype)
    ref_in, ref_out = f.clone(), torch.empty_like(f)
    na_in, na_out = f.clone(), torch.empty_like(f)
    s = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    grid = _grid(fks, ncell, bc)
    vbox = fks._VBox(n, L)
    lib = fks.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for dt in (0.41 / (L * 5), -0.93 / (L * 5)):
        ctx.transport(ref_in, ref_out, dt)
        st = lib.fks_transport_noalloc(ctypes.byref(grid), ctypes.byref(vbox), prec,
                                       ctypes.c_void_p(s.data_ptr()), dt, ctypes.c_void_p(na_in.data_ptr()),
                                       ctypes.c_void_p(na_out.data_ptr()), ctypes.c_void_p(stream))
        assert st == 0
        torch.cuda.synchronize()
        assert torch.equal(na_out, ref_out)
        np.testing.assert_array_equal(s.cpu().numpy().reshape(3, n), ctx.offsets())
        ref_in, ref_out = ref_out, ref_in
        na_in, na_out = na_out, na_in


def test_noalloc_rejects_sizes_beyond_its_scratch(fks):
    lib = fks.lib()
    grid = _grid(fks, (2, 2, 2), (0, 0, 0))
    vbox = fks._VBox(64, 10.0)
    x = torch.zeros(8, device="cuda", dtype=torch.float32)
    y = torch.zeros(8, device="cuda", dtype=torch.float32)
    s = torch.zeros(3 * 64, device="cuda", dtype=torch.float64)
    st = lib.fks_transport_noalloc(ctypes.byref(grid), ctypes.byref(vbox), 1, ctypes.c_void_p(s.data_ptr()),
                                   0.01, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 2   # FKS_ERR_UNSUPPORTED, before any work


def test_noalloc_reports_a_shift_out_of_range(fks):
    """Offsets far outside [-dx/2, dx/2) (a corrupted s, written by the host) give cell shifts
    beyond the shift table's range: the call reads its flag word and returns FKS_ERR_NUMERIC;
    the next call with sane offsets succeeds."""
    lib = fks.lib()
    n, ncell, L = 8, (4, 1, 1), 10.0
    grid = _grid(fks, ncell, (0, 0, 0))
    vbox = fks._VBox(n, L)
    f = torch.rand((4, n, n, n), device="cuda", dtype=torch.float32)
    out = torch.empty_like(f)
    dx = 1.0 / ncell[0]
    s = torch.full((3 * n,), 1000.0 * dx, device="cuda", dtype=torch.float64)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.fks_transport_noalloc(ctypes.byref(grid), ctypes.byref(vbox), 1, ctypes.c_void_p(s.data_ptr()), 0.001,
                                   ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 5   # FKS_ERR_NUMERIC
    s.zero_()
    st = lib.fks_transport_noalloc(ctypes.byref(grid), ctypes.byref(vbox), 1, ctypes.c_void_p(s.data_ptr()), 0.001,
                                   ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
    assert st == 0
