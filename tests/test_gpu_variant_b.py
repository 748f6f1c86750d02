"""GPU parity of variant B (fks_set_dealias: Eq. CF1 without reduction mod n,
2n transforms) against the oracle's collide_b: FP64 <= 1e-10, FP32 <= 1e-5
(the FP32 reading of the loss scale), steps with the transport gather,
conservation, more cells than one chunk, unsupported configurations."""
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


def ctx_b(fks, ncell, n, L, prec, kernel=0, kn=1.0, bc=(0, 0, 0)):
    return fks.Context(fks.Config(ncell=tuple(ncell), bc=tuple(bc), n=n, L=L, kernel=kernel, kn=kn, A1=4, A2=4,
                                  precision=prec, dealias=True))


@pytest.mark.parametrize("n,prec,kernel,nc", [
    (8, 0, 0, 5), (8, 0, 1, 3), (16, 0, 0, 3), (8, 1, 0, 7), (16, 1, 0, 5), (16, 1, 1, 3),
])
def test_dealiased_collide_matches_oracle(fks, oracle, n, prec, kernel, nc):
    L, kn = (6.0 if n == 8 else 8.0), 0.4
    ctx = ctx_b(fks, (nc, 1, 1), n, L, prec, kernel=kernel, kn=kn)
    f = I.two_stream((nc, 1, 1), n, L, seed=40 + n + nc, noise=0.05)
    fd = torch.from_numpy(f).to(device="cuda", dtype=ctx.dtype)
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    assert ctx.check() == 0
    fin = fd.double().cpu().numpy()
    tab2 = oracle.tables(2 * n, L, kernel, 0.25, 4, 4, 0)
    Qo = oracle.collide_b(fin, tab2, kn=kn, project=True)
    Qg = Q.double().cpu().numpy()
    for c in range(nc):
        assert rel(Qg[c], Qo[c]) < (1e-10 if prec == 0 else 1e-5), (c, rel(Qg[c], Qo[c]))


def test_dealiased_differs_from_aliased_and_conserves(fks, oracle):
    n, L, nc = 16, 8.0, 3
    f = torch.from_numpy(I.two_stream((nc, 1, 1), n, L, seed=3, noise=0.05)).cuda()
    ca = fks.Context(fks.Config(ncell=(nc, 1, 1), n=n, L=L, kn=1.0, A1=4, A2=4, precision=0))
    cb = ctx_b(fks, (nc, 1, 1), n, L, 0)
    Qa, Qb = torch.empty_like(f), torch.empty_like(f)
    ca.collide(f, Qa)
    cb.collide(f, Qb)
    assert rel(Qa.cpu().numpy(), Qb.cpu().numpy()) > 1e-3
    U = oracle.moments(Qb.cpu().numpy(), n, L)
    Ua = oracle.moments(np.abs(Qb.cpu().numpy()), n, L)
    assert np.all(np.abs(U[:, 0]) < 1e-12 * Ua[:, 0])
    assert np.all(np.abs(U[:, 4]) < 1e-12 * (Ua[:, 4] + Ua[:, 0] * L * L))
    cb.set_dealias(False)   # back to variant A
    cb.collide(f, Qb)
    assert torch.equal(Qa, Qb)


def test_dealiased_more_cells_than_a_chunk(fks, oracle):
    n, L, nc = 8, 6.0, 2100   # chunks of 2048 cells: a ragged second chunk
    ctx = ctx_b(fks, (nc, 1, 1), n, L, 0)
    f = I.two_stream((nc, 1, 1), n, L, seed=12, noise=0.05)
    fd = torch.from_numpy(f).cuda()
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    cells = [0, 1, 2047, 2048, 2099]
    Qo = oracle.collide_b(f[cells], oracle.tables(2 * n, L, 0, 0.25, 4, 4, 0), kn=1.0, project=True)
    Qg = Q.cpu().numpy()[cells]
    for i in range(len(cells)):
        assert rel(Qg[i], Qo[i]) < 1e-10


def test_dealiased_steps_ragged_specular(fks, oracle):
    """The transport gather of step mode inside the pad and truncation kernels."""
    ncell, n, L, bc, kn = (3, 5, 2), 8, 5.0, (1, 1, 0), 0.5
    ctx = ctx_b(fks, ncell, n, L, 0, kn=kn, bc=bc)
    tab2 = oracle.tables(2 * n, L, 0, 0.25, 4, 4, 0)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab2, kn, variant_b=True)
    f = I.two_stream(ncell, n, L, seed=9, noise=0.1)
    fd = torch.from_numpy(f).cuda()
    out = torch.empty_like(fd)
    dt = 0.7 * 0.2 / L
    for _ in range(3):
        ctx.step(fd, out, dt)
        fd, out = out, fd
        f = sol.step(f, dt)
    assert ctx.check() & 1 == 0
    assert rel(fd.cpu().numpy(), f) < 1e-10


def test_dealias_unsupported(fks):
    c32 = fks.Context(fks.Config(ncell=(1, 1, 1), n=32, L=10.0, A1=4, A2=8, precision=0))
    with pytest.raises(fks.FKSError) as e:
        c32.set_dealias(True)
    assert e.value.status == 2
    cb = fks.Context(fks.Config(ncell=(1, 1, 1), n=16, L=8.0, kernel=fks.BGK, precision=1))
    with pytest.raises(fks.FKSError) as e:
        cb.set_dealias(True)
    assert e.value.status == 2
