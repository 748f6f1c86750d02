"""Oracle transport (exact shift of the generic-cell particles, Sec. 2.1 and
Sec. 3) and moments, pinned by permutation / conservation facts and closed
forms."""
import numpy as np
import pytest

from paper_1701_01608_gb300 import inputs as I


def _unique_field(nc, n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.permutation(np.arange(np.prod(nc) * n ** 3, dtype=np.float64)).reshape(-1, n, n, n)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 0), (1, 1, 1)])
def test_transport_is_a_bijection(oracle, bc):
    nc, n, L = (5, 3, 4), 8, 4.0
    f = _unique_field(nc, n)
    dx = [1.0 / c for c in nc]
    dt = 0.37 * min(dx) / L
    s = np.zeros((3, n))
    for step in range(4):
        s, delta = oracle.offsets(n, L, dx, dt, s)
        g = oracle.transport(f, nc, bc, delta)
        np.testing.assert_array_equal(np.sort(g.ravel()), np.sort(f.ravel()))
        f = g


def test_offsets_and_shift_rule(oracle):
    n, L, dx = 8, 4.0, 0.25
    v = I.velocity_points(n, L)
    dt = 0.9 * dx / L
    s, delta = oracle.offsets(n, L, [dx] * 3, dt, np.zeros((3, n)))
    # first step from the cell centre: delta = round-half-up(v dt / dx)
    np.testing.assert_array_equal(delta[0], np.floor(v * dt / dx + 0.5).astype(int))
    assert np.all(np.abs(s) <= dx / 2 + 1e-15)
    np.testing.assert_array_equal(s[0][::-1], -s[0])
    # after many steps the cumulative shift + offset equals v t exactly (up to rounding)
    s = np.zeros((3, n))
    tot = np.zeros(n)
    for _ in range(37):
        s, d = oracle.offsets(n, L, [dx] * 3, dt, s)
        tot += d[0]
    np.testing.assert_allclose(tot * dx + s[0], v * 37 * dt, atol=1e-12)


def test_periodic_shift_matches_roll(oracle):
    """A velocity whose offset crosses exactly one face moves its profile by
    one cell: compare with numpy.roll of that velocity's slice."""
    nc, n, L = (6, 5, 4), 8, 4.0
    f = _unique_field(nc, n, 3)
    dx = [1.0 / c for c in nc]
    dt = 0.5 * min(dx) / L
    s, delta = oracle.offsets(n, L, dx, dt, np.zeros((3, n)))
    g = oracle.transport(f, nc, (0, 0, 0), delta)
    F = f.reshape(*nc, n, n, n)
    G = g.reshape(*nc, n, n, n)
    for kx, ky, kz in [(0, 0, 0), (7, 3, 5), (4, 4, 4), (1, 6, 2)]:
        want = np.roll(F[..., kx, ky, kz], (delta[0, kx], delta[1, ky], delta[2, kz]), axis=(0, 1, 2))
        np.testing.assert_array_equal(G[..., kx, ky, kz], want)


def test_round_trip_is_identity(oracle):
    nc, n, L = (4, 4, 4), 8, 4.0
    f = _unique_field(nc, n, 4)
    dx = [0.25] * 3
    dt = 0.61 * 0.25 / L
    s0 = np.zeros((3, n))
    s1, d1 = oracle.offsets(n, L, dx, dt, s0)
    g = oracle.transport(f, nc, (1, 0, 0), d1)
    s2, d2 = oracle.offsets(n, L, dx, -dt, s1)
    h = oracle.transport(g, nc, (1, 0, 0), d2)
    np.testing.assert_array_equal(h, f)


def test_specular_conserves_mass_and_energy(oracle):
    nc, n, L = (8, 2, 2), 8, 4.0
    f = I.two_stream(nc, n, L, seed=1, noise=0.1)
    dx = [1.0 / c for c in nc]
    dt = 0.8 * min(dx) / L
    s = np.zeros((3, n))
    U0 = oracle.moments(f, n, L).sum(axis=0)
    for _ in range(7):
        s, d = oracle.offsets(n, L, dx, dt, s)
        f = oracle.transport(f, nc, (1, 0, 0), d)
    U1 = oracle.moments(f, n, L).sum(axis=0)
    assert abs(U1[0] - U0[0]) < 1e-13 * U0[0]
    assert abs(U1[4] - U0[4]) < 1e-13 * U0[4]


def test_moments_of_maxwellian(oracle):
    n, L = 32, 8.0
    rho, u, T = 1.3, (0.4, -0.2, 0.1), 0.8
    U = oracle.moments(I.maxwellian(n, L, rho, u, T)[None], n, L)[0]
    want = [rho, rho * u[0], rho * u[1], rho * u[2], 0.5 * rho * np.dot(u, u) + 1.5 * rho * T]
    np.testing.assert_allclose(U, want, rtol=1e-10, atol=1e-12)


def test_step_conserves_invariants(oracle):
    """Periodic FKS steps (transport + projected Euler collision) conserve
    mass, momentum and energy to rounding."""
    w = I.config_small_periodic()
    t = oracle.tables(w.n, w.L, w.kernel, w.C, w.A1, w.A2, 0)
    sol = oracle.Solver(w.ncell, w.x0, w.x1, w.bc, w.n, w.L, t, w.kn)
    f = w.f0
    U0 = oracle.moments(f, w.n, w.L).sum(axis=0)
    dt = 0.004
    for _ in range(3):
        f = sol.step(f, dt)
    U1 = oracle.moments(f, w.n, w.L).sum(axis=0)
    scale = np.abs(U0).max()
    assert np.abs(U1 - U0).max() < 1e-12 * scale
