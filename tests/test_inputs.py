"""The seeded input generators (paper_1701_01608_gb300/inputs.py) against the workloads they stand
for: densities, mean velocities and temperatures of the initial states by quadrature on the velocity
grid, the boundary conditions and parameters of each configuration, the seeded noise bounds, and
determinism under a seed.  The midpoint rule on step h integrates a Gaussian of variance s^2 with a
relative error of about 2 exp(-2 pi^2 s^2 / h^2) (more for the second moment, see quad_tol): ~4e-22
for s^2 = 1 at h = 0.625 (n = 32 on [-10, 10]), ~5e-9 at h = 1 (n = 16 on [-8, 8]); the
tolerances below follow from it."""
import numpy as np
import pytest

from paper_1701_01608_gb300 import inputs as I


def quad_tol(s2, h):
    """a bound on the midpoint rule's relative error for a Gaussian of variance s2 on step h, up to
    its second moment (by Poisson summation the first aliased term of the v^2 moment carries the
    extra factor 1 + 4 pi^2 s2 / h^2)"""
    a = 2.0 * np.pi ** 2 * s2 / h ** 2
    return max(1e-13, 10.0 * (1.0 + 2.0 * a) * np.exp(-a))


def moments(f, n, L):
    """rho, u, T of f[..., n, n, n] by the midpoint rule on [-L, L]^3."""
    v = I.velocity_points(n, L)
    dv3 = (2.0 * L / n) ** 3
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    rho = f.sum(axis=(-3, -2, -1)) * dv3
    u = np.stack([(f * c).sum(axis=(-3, -2, -1)) * dv3 / rho for c in (vx, vy, vz)], axis=-1)
    e = (f * (vx * vx + vy * vy + vz * vz)).sum(axis=(-3, -2, -1)) * dv3 / rho
    T = (e - (u * u).sum(axis=-1)) / 3.0
    return rho, u, T


def test_velocity_points_cell_centred():
    v = I.velocity_points(32, 10.0)
    assert v[0] == pytest.approx(-10.0 + 10.0 / 32) and v[-1] == pytest.approx(10.0 - 10.0 / 32)
    assert np.allclose(np.diff(v), 20.0 / 32) and np.allclose(v, -v[::-1])


@pytest.mark.parametrize("rho,u,T", [(1.0, (0, 0, 0), 1.0), (0.125, (0, 0, 0), 0.8), (2.0, (0.5, -1.0, 0.25), 1.2)])
def test_maxwellian_moments(rho, u, T):
    r, uu, TT = moments(I.maxwellian(32, 10.0, rho, u, T), 32, 10.0)
    assert r == pytest.approx(rho, rel=1e-12)
    assert np.allclose(uu, u, atol=1e-12)
    assert TT == pytest.approx(T, rel=1e-12)


@pytest.mark.parametrize("K", [0.6, 0.8, 1.0])
def test_bkw_has_unit_density_zero_mean_and_temperature_T(K):
    """The BKW family keeps density, momentum and energy for every K (K = 1: the Maxwellian)."""
    for T in (0.8, 1.2):
        r, u, TT = moments(I.bkw(32, 10.0, K, T=T), 32, 10.0)
        tol = 100 * quad_tol(K * T, 0.625)   # the polynomial factor weights the tails
        assert r == pytest.approx(1.0, rel=tol)
        assert np.abs(u).max() < 1e-12
        assert TT == pytest.approx(T, rel=tol)
    assert np.allclose(I.bkw(16, 8.0, 1.0), I.maxwellian(16, 8.0), rtol=1e-13, atol=0)


def test_shock_tube_states_and_config():
    w = I.config_shock_tube(ncell=(8, 2, 2), n=16, L=8.0)
    assert w.bc == (1, 0, 0) and w.kn == 0.01 and w.M == 32 and w.kernel == 0 and w.steps == 100
    f = w.f0.reshape(8, 4, 16, 16, 16)
    rho, u, T = moments(f, 16, 8.0)
    tol = quad_tol(0.8, 1.0)
    assert np.allclose(rho[:4], 1.0, rtol=tol) and np.allclose(rho[4:], 0.125, rtol=tol)
    assert np.allclose(T[:4], 1.0, rtol=tol) and np.allclose(T[4:], 0.8, rtol=tol)
    assert np.abs(u).max() < 1e-12
    states, which = I.shock_tube_states(16, 8.0, 8)
    assert list(which) == [0, 0, 0, 0, 1, 1, 1, 1]
    assert np.array_equal(states[which].repeat(4, axis=0), w.f0)


def test_shock_tube_noise_bounds():
    w0 = I.config_shock_tube(ncell=(4, 1, 1), n=8, L=8.0)
    w = I.config_shock_tube(ncell=(4, 1, 1), n=8, L=8.0, noise=0.02, seed=5)
    ratio = w.f0 / w0.f0
    assert ratio.min() >= 0.98 and ratio.max() <= 1.02 and ratio.std() > 0.005


def test_two_stream_profile():
    f = I.two_stream((8, 1, 1), 16, 8.0, seed=0, noise=0.0)
    rho, u, T = moments(f, 16, 8.0)
    x = (np.arange(8) + 0.5) / 8
    tol = quad_tol(1.0, 1.0)
    assert np.allclose(rho, 1.0 + 0.2 * np.sin(2 * np.pi * x), rtol=tol)
    assert np.abs(u).max() < 1e-12
    # two unit-temperature streams at +-e_x: variance 2 along x, 1 along y and z
    assert np.allclose(T, 4.0 / 3.0, rtol=tol)
    fn = I.two_stream((8, 1, 1), 16, 8.0, seed=0, noise=0.01)
    r = fn / f
    assert r.min() >= 0.99 and r.max() <= 1.01


def test_homogeneous_bkw_config():
    w = I.config_homogeneous_bkw(ncells=8, n=32, seed=1)
    assert w.kernel == 1 and w.M == 32 and w.L == 10.0
    assert (w.T >= 0.8).all() and (w.T <= 1.2).all() and w.T.std() > 0
    rho, u, T = moments(w.f0, 32, 10.0)
    tol = 100 * quad_tol(0.6 * 0.8, 0.625)
    assert np.allclose(rho, 1.0, rtol=tol) and np.allclose(T, w.T, rtol=tol)


def test_uneven_batch_config():
    probs = I.config_uneven_batch(nprob=96, seed=3)
    assert len(probs) == 96
    ns = {p["n"] for p in probs}
    assert ns == {16, 24, 32}
    kn = np.array([p["kn"] for p in probs])
    assert kn.min() >= 1e-3 and kn.max() <= 1.0
    assert {p["kernel"] for p in probs} == {0, 1}
    for p in probs[:8]:
        assert p["f0"].shape == (1, p["n"], p["n"], p["n"])
        rho, _, _ = moments(p["f0"][0], p["n"], p["L"])
        assert rho == pytest.approx(1.0, rel=quad_tol(0.8, 2.0 * p["L"] / p["n"]))


def test_seeded_determinism():
    a = I.two_stream((2, 2, 1), 8, 8.0, seed=7)
    b = I.two_stream((2, 2, 1), 8, 8.0, seed=7)
    c = I.two_stream((2, 2, 1), 8, 8.0, seed=8)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    p1 = I.config_uneven_batch(nprob=4, seed=3)
    p2 = I.config_uneven_batch(nprob=4, seed=3)
    assert all(np.array_equal(x["f0"], y["f0"]) and x["kn"] == y["kn"] for x, y in zip(p1, p2))
