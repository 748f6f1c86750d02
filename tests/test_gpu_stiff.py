"""The stiff (exponential) step of the spectral operator on the GPU against the oracle: transport,
then the integrating-factor step of the gain-loss split with the loss frequency frozen at f*
(fks_step_exp on FP64 and FP32 spectral contexts), on a ragged specular grid, at Kn = 0.1 and at
Kn = 1e-6 (nu dt ~ 1e4), where the Euler step is unstable."""
import numpy as np
import pytest

from conftest import FP32_REL
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


@pytest.mark.parametrize("kn", [0.1, 1e-6])
def test_fp64_steps_match_oracle(fks, oracle, kn):
    ncell, n, L, bc = (3, 2, 2), 16, 8.0, (1, 0, 0)
    c = fks.Context(fks.Config(ncell=ncell, bc=bc, n=n, L=L, kn=kn, A1=4, A2=4, precision=0))
    tab = oracle.tables(n, L, 0, 0.25, 4, 4, 0)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, kn)
    f = I.two_stream(ncell, n, L, seed=12, noise=0.05)
    fd, out = torch.from_numpy(f).cuda(), torch.empty(f.shape, dtype=torch.float64, device="cuda")
    dt = 0.01
    for _ in range(3):
        c.step_exp(fd, out, dt)
        fd, out = out, fd
        f = sol.step_exp(f, dt)
    assert c.check() & 1 == 0
    assert rel(fd.cpu().numpy(), f) < 1e-10
    # bounded in the stiff case (the Euler step of the same size is not)
    assert np.abs(f).max() < 10 * np.abs(I.two_stream(ncell, n, L, seed=12, noise=0.05)).max()


@pytest.mark.parametrize("kn", [0.1, 1e-6])
def test_fp32_step_matches_oracle(fks, oracle, kn):
    """One FP32 step (with the context's escalation) from the oracle's input: the increment
    f_out - f* against the oracle's, per cell, up to the FP32 rounding of the stored state."""
    ncell, n, L, bc = (3, 2, 2), 32, 10.0, (1, 0, 0)
    c = fks.Context(fks.Config(ncell=ncell, bc=bc, n=n, L=L, kn=kn, A1=4, A2=8, precision=1))
    tab = oracle.tables(n, L, 0, 0.25, 4, 8, 0)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, kn)
    f = I.two_stream(ncell, n, L, seed=13, noise=0.05).astype(np.float32).astype(np.float64)
    fd = torch.from_numpy(f).float().cuda()
    out = torch.empty_like(fd)
    dt = 0.001
    c.step_exp(fd, out, dt)
    assert c.check() & 1 == 0
    fs = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, kn).transport(f, dt)
    want = sol.step_exp(f, dt)
    got = out.double().cpu().numpy()
    for i in range(fs.shape[0]):
        inc_ref = want[i] - fs[i]
        err = np.linalg.norm(got[i] - fs[i] - inc_ref)
        assert err <= FP32_REL * np.linalg.norm(inc_ref) + 2.0 ** -24 * 1.5 * np.linalg.norm(got[i]), i
