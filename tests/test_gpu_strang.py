"""GPU parity of the second-order step (fks_step_strang: Strang splitting with
a Heun collision sub-step) against the oracle's solver, through the C ABI."""
import numpy as np
import pytest

from paper_1701_01608_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_01608_gb300 import fks
    fks.lib()
    return fks


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def host64(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("prec,kernel,n", [(0, 0, 8), (1, 0, 8), (1, 0, 32), (0, 2, 8), (1, 2, 16)])
def test_strang_steps_match_oracle(fks, oracle, prec, kernel, n):
    """3 steps on a ragged grid with a specular wall; spectral (hard spheres) and BGK."""
    ncell, L, bc, kn = (3, 2, 2), 5.0, (1, 0, 0), 0.5
    ctx = fks.Context(fks.Config(ncell=ncell, bc=bc, n=n, L=L, kernel=kernel, C=0.25, kn=kn, A1=4, A2=4,
                                 precision=prec))
    tab = oracle.tables(n, L, 0, 0.25, 4, 4, 0) if kernel == 0 else None
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, kn)
    f = I.two_stream(ncell, n, L, seed=12, noise=0.1)
    fd = torch.from_numpy(f).to(device="cuda", dtype=ctx.dtype).contiguous()
    f = host64(fd)
    out, work = torch.empty_like(fd), torch.empty_like(fd)
    dt = 0.7 * (1.0 / 3) / L
    for _ in range(3):
        ctx.step_strang(fd, out, work, dt)
        fd, out = out, fd
        f = sol.step_strang(f, dt)
    assert ctx.check() & 1 == 0
    assert rel(host64(fd), f) < (1e-10 if prec == 0 else 2e-5)


def test_strang_homogeneous_is_heun(fks, oracle):
    """One periodic cell: transport is the identity and the step is Heun's method,
    b = f + dt Q(f), out = (f + b + dt Q(b)) / 2, evaluated with the library's own collide."""
    n, L = 16, 8.0
    ctx = fks.Context(fks.Config(ncell=(1, 1, 1), n=n, L=L, kernel=0, C=0.25, kn=1.0, A1=4, A2=4, precision=0))
    f = torch.from_numpy(I.two_stream((1, 1, 1), n, L, seed=1)).cuda()
    out, work, Q = torch.empty_like(f), torch.empty_like(f), torch.empty_like(f)
    dt = 0.05
    ctx.step_strang(f, out, work, dt)
    ctx.collide(f, Q)
    b = f + dt * Q
    ctx.collide(b, Q)
    want = 0.5 * (f + b + dt * Q)
    assert rel(host64(out), host64(want)) < 1e-14


def test_strang_rejected_where_unsupported(fks):
    n, L = 16, 8.0
    ctx = fks.Context(fks.Config(ncell=(2, 1, 1), n=n, L=L, precision=fks.FKS_BF16X3))
    f = torch.zeros((2, n, n, n), device="cuda")
    with pytest.raises(fks.FKSError) as e:
        ctx.step_strang(f, torch.empty_like(f), torch.empty_like(f), 0.01)
    assert e.value.status == 2
    ctx = fks.Context(fks.Config(ncell=(2, 1, 1), n=n, L=L))
    with pytest.raises(fks.FKSError) as e:
        ctx.step_strang(f, f, torch.empty_like(f), 0.01)
    assert e.value.status == 1
