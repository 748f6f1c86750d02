"""BGK relaxation step (Sec. 2, BGK approximation) on the GPU against the
oracle: collide, fused transport + step on a ragged specular grid, and the
full 32^3 x 32^3 FP32 step on sampled cells."""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ctx(fks, ncell, n, L, prec, kn=0.2, bc=(0, 0, 0)):
    return fks.Context(fks.Config(ncell=ncell, bc=bc, n=n, L=L, kernel=fks.BGK, kn=kn, precision=prec))


@pytest.mark.parametrize("n", [8, 16, 24, 32])
@pytest.mark.parametrize("prec", [0, 1])
def test_bgk_collide_matches_oracle(fks, oracle, n, prec):
    L = 8.0
    c = ctx(fks, (5, 1, 1), n, L, prec)
    f = I.two_stream((5, 1, 1), n, L, seed=n, noise=0.05)
    fd = torch.from_numpy(f).to("cuda", c.dtype).contiguous()
    Q = torch.empty_like(fd)
    c.collide(fd, Q)
    assert c.check() & 1 == 0
    fin = fd.double().cpu().numpy()
    Qo = oracle.bgk(fin, n, L, kn=0.2)
    Qg = Q.double().cpu().numpy()
    for i in range(5):
        assert rel(Qg[i], Qo[i]) < (1e-12 if prec == 0 else 1e-5), (i, rel(Qg[i], Qo[i]))


def test_bgk_steps_ragged_specular(fks, oracle):
    ncell, n, L = (3, 5, 2), 16, 8.0
    bc = (1, 1, 0)
    c = ctx(fks, ncell, n, L, 0, kn=0.1, bc=bc)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, None, 0.1)
    f = I.two_stream(ncell, n, L, seed=2, noise=0.1)
    fd = torch.from_numpy(f).cuda()
    out = torch.empty_like(fd)
    dt = 0.01
    for _ in range(4):
        c.step(fd, out, dt)
        fd, out = out, fd
        f = sol.step(f, dt)
    assert rel(fd.cpu().numpy(), f) < 1e-12


def test_bgk_full_size_fp32_sampled(fks, oracle):
    n, L, kn = 32, 10.0, 0.01
    c = ctx(fks, (32, 32, 32), n, L, 1, kn=kn, bc=(1, 0, 0))
    c2 = ctx(fks, (32, 32, 32), n, L, 1, kn=kn, bc=(1, 0, 0))
    states, which = I.shock_tube_states(n, L, 32)
    st = torch.from_numpy(states).float().cuda()
    f0 = st.index_select(0, torch.from_numpy(np.repeat(which, 1024)).cuda()).contiguous()
    g = torch.Generator(device="cuda").manual_seed(4)
    f0 *= 1.0 + 0.05 * (2.0 * torch.rand(f0.shape, generator=g, device="cuda", dtype=torch.float32) - 1.0)
    f1 = torch.empty_like(f0)
    fs = torch.empty_like(f0)
    dt = 1e-3
    c.step(f0, f1, dt)
    c2.transport(f0, fs, dt)
    sample = [0, 31 * 1024 + 17, 16 * 1024 + 5 * 32 + 7, 32767]
    fsh = fs[sample].double().cpu().numpy()
    Qo = oracle.bgk(fsh, n, L, kn=kn)
    got = f1[sample].double().cpu().numpy()
    for i in range(len(sample)):
        err = np.linalg.norm(got[i] - (fsh[i] + dt * Qo[i]))
        assert err < 1e-5 * np.linalg.norm(dt * Qo[i]) + 2e-7 * np.linalg.norm(fsh[i])


@pytest.mark.parametrize("n,prec", [(32, 1), (16, 0), (32, 0)])
def test_bgk_vacuum_cell_does_not_relax(fks, oracle, n, prec):
    """A vacuum cell (f = 0) has no Maxwellian: Q = 0 there, the other cells as usual."""
    L = 8.0
    c = ctx(fks, (3, 1, 1), n, L, prec)
    f = I.two_stream((3, 1, 1), n, L, seed=7, noise=0.05)
    f[1] = 0.0
    fd = torch.from_numpy(f).to("cuda", c.dtype).contiguous()
    Q = torch.empty_like(fd)
    c.collide(fd, Q)
    assert c.check() & 1 == 0
    Qg = Q.double().cpu().numpy()
    assert np.all(Qg[1] == 0.0)
    Qo = oracle.bgk(fd.double().cpu().numpy(), n, L, kn=0.2)
    assert np.all(Qo[1] == 0.0)
    for i in (0, 2):
        assert rel(Qg[i], Qo[i]) < (1e-12 if prec == 0 else 1e-5), (i, rel(Qg[i], Qo[i]))


@pytest.mark.parametrize("n,prec,kn", [(16, 0, 0.1), (32, 1, 0.01), (32, 1, 1e-6), (16, 0, 1e-6)])
def test_bgk_exponential_step_matches_oracle(fks, oracle, n, prec, kn):
    """fks_step_exp (transport + exact BGK relaxation) against the oracle's solver, 3 steps on a
    ragged specular grid; Kn = 1e-6 is the stiff case (nu dt ~ 1e3, where the Euler step diverges)."""
    ncell, L, bc = (3, 2, 2), 8.0, (1, 0, 0)
    c = ctx(fks, ncell, n, L, prec, kn=kn, bc=bc)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, None, kn)
    f = I.two_stream(ncell, n, L, seed=5, noise=0.1)
    fd = torch.from_numpy(f).to("cuda", c.dtype).contiguous()
    f = fd.double().cpu().numpy()
    out = torch.empty_like(fd)
    dt = 1e-3
    for _ in range(3):
        c.step_exp(fd, out, dt)
        fd, out = out, fd
        f = sol.step_exp(f, dt)
    assert c.check() & 1 == 0
    got = fd.double().cpu().numpy()
    assert rel(got, f) < (1e-11 if prec == 0 else 3e-6)


def test_exponential_step_unsupported_for_split_bf16(fks):
    """The exponential step runs on the BGK and the FP64/FP32 spectral kernels, not on the split-BF16
    tensor-core kernel."""
    c = fks.Context(fks.Config(ncell=(2, 1, 1), n=16, L=8.0, kernel=0, precision=2))
    f = torch.zeros((2, 16, 16, 16), device="cuda")
    with pytest.raises(fks.FKSError) as e:
        c.step_exp(f, torch.empty_like(f), 0.01)
    assert e.value.status == 2
