"""Oracle variant B (Eq. CF1 with l + m = k over l, m in [-n/2, n/2]^3, not
reduced mod n; 2n transforms as in Sec. 5) pinned by the identity
truncate(pad(f)) = f, exact interpolation of a band-limited function, the
brute-force Galerkin sum, mass conservation and Q(M) = 0."""
import numpy as np
import pytest

from paper_1701_01608_gb300 import inputs as I


def test_truncate_after_pad_is_identity(oracle):
    rng = np.random.Generator(np.random.PCG64(3))
    for n in (8, 16):
        f = rng.standard_normal((n, n, n))
        f2 = oracle.pad(f, n)
        assert np.allclose(f2[::2, ::2, ::2], f, atol=1e-13)   # the interpolant passes through f
        assert np.allclose(oracle.truncate(f2, n), f, atol=1e-12)


def test_pad_interpolates_a_band_limited_function(oracle):
    n, m = 8, 16
    j = np.arange(n)
    j2 = np.arange(m)
    # modes 1 and 3 along x, 2 along z (below the Nyquist index n/2 = 4)
    f = (np.cos(2 * np.pi * 1 * j / n)[:, None, None] + np.sin(2 * np.pi * 3 * j / n)[:, None, None]) \
        * np.cos(2 * np.pi * 2 * j / n)[None, None, :] * np.ones((1, n, 1))
    want = (np.cos(np.pi * 1 * j2 / n)[:, None, None] + np.sin(np.pi * 3 * j2 / n)[:, None, None]) \
        * np.cos(np.pi * 2 * j2 / n)[None, None, :] * np.ones((1, m, 1))
    assert np.allclose(oracle.pad(f, n), want, atol=1e-12)
    # a Nyquist mode (-1)^j is split between +-n/2: cos(pi j2 / 2) on the 2n grid
    g = ((-1.0) ** j)[:, None, None] * np.ones((1, n, n))
    assert np.allclose(oracle.pad(g, n), np.cos(np.pi * j2 / 2)[:, None, None] * np.ones((1, m, m)), atol=1e-12)


@pytest.mark.parametrize("ktype", [0, 1])
def test_fft_evaluation_equals_brute_force_galerkin(oracle, ktype):
    n, L = 8, 6.0
    f = I.two_stream((1, 1, 1), n, L, seed=7, noise=0.05)[0]
    tab2 = oracle.tables(2 * n, L, ktype, 0.25, 4, 4, 0)
    Qf = oracle.collide_b(f[None], tab2, kn=1.0, project=False)[0]
    Qb = oracle.galerkin_b(f, n, L, ktype, 0.25, 4, 4, 0, kn=1.0)
    assert np.linalg.norm(Qf - Qb) < 1e-12 * np.linalg.norm(Qb)


def test_brute_force_differs_from_the_aliased_operator(oracle):
    """A planted mistake: the circular (variant A) operator is not variant B."""
    n, L = 8, 6.0
    f = I.two_stream((1, 1, 1), n, L, seed=7, noise=0.05)[0]
    Qa = oracle.collide(f[None], oracle.tables(n, L, 0, 0.25, 4, 4, 0), kn=1.0, project=False)[0]
    Qb = oracle.galerkin_b(f, n, L, 0, 0.25, 4, 4, 0, kn=1.0)
    assert np.linalg.norm(Qa - Qb) > 1e-3 * np.linalg.norm(Qb)


def test_mass_conserved(oracle):
    n, L = 16, 8.0
    tab2 = oracle.tables(2 * n, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), n, L, seed=2, noise=0.05)[0]
    Q = oracle.collide_b(f[None], tab2, kn=1.0, project=False)[0]
    assert abs(Q.sum()) < 1e-12 * np.abs(Q).sum()


def test_maxwellian_is_equilibrium_spectrally(oracle):
    """Q_B(M) / ||L(M)|| decays spectrally with n on [-8, 8]^3: the Maxwellian's
    spectrum at the cut-off is ~exp(-pi^2/2) at n = 16, ~exp(-2 pi^2) at n = 32."""
    L, r = 8.0, {}
    for n in (16, 32):
        M = I.maxwellian(n, L, 1.0, (0.3, -0.2, 0.1), 1.0)
        QM = oracle.collide_b(M[None], oracle.tables(2 * n, L, 0, 0.25, 4, 4, 0), kn=1.0, project=True)[0]
        _, Lo = oracle.gain_loss(M, oracle.tables(n, L, 0, 0.25, 4, 4, 0))
        r[n] = np.linalg.norm(QM) / np.linalg.norm(Lo)
    assert r[32] < 1e-8 and r[32] < 1e-4 * r[16]
