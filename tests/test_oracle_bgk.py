"""Oracle BGK operator pinned by closed forms: the Maxwellian of a mixture
carries the mixture's analytic moments, Q(M) = 0 to spectral accuracy,
conservation after projection, and the relaxation rate nu = rho / Kn."""
import numpy as np

from paper_1701_01608_gb300 import inputs as I


def test_bgk_of_maxwellian_vanishes(oracle):
    n, L = 32, 8.0
    M = I.maxwellian(n, L, 1.3, (0.3, -0.2, 0.1), 0.9)
    Q = oracle.bgk(M, n, L, kn=0.5, project=False)
    assert np.abs(Q).max() < 1e-9 * np.abs(M).max() / 0.5


def test_bgk_targets_the_mixture_maxwellian(oracle):
    """For f = (M1 + M2)/2 with means +-a e_x and temperature T, the
    equilibrium has rho = 1, u = 0 and T_eq = T + a^2 / 3; Q/nu + f must be
    that Maxwellian."""
    n, L, a, T = 32, 8.0, 1.0, 0.8
    f = 0.5 * (I.maxwellian(n, L, u=(a, 0, 0), T=T) + I.maxwellian(n, L, u=(-a, 0, 0), T=T))
    kn = 0.25
    Q = oracle.bgk(f, n, L, kn=kn, project=False)
    Meq = I.maxwellian(n, L, 1.0, (0, 0, 0), T + a * a / 3.0)
    np.testing.assert_allclose(Q * kn + f, Meq, atol=1e-9 * Meq.max())


def test_bgk_conserves_after_projection(oracle):
    n, L = 16, 8.0
    f = I.two_stream((3, 1, 1), n, L, seed=4, noise=0.2)
    Q = oracle.bgk(f, n, L, kn=0.1)
    v = I.velocity_points(n, L)
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    phi = np.stack([np.ones_like(vx), vx, vy, vz, 0.5 * (vx ** 2 + vy ** 2 + vz ** 2)]).reshape(5, -1)
    for c in range(3):
        m = phi @ Q[c].ravel()
        assert np.all(np.abs(m) <= 1e-12 * (np.abs(phi) @ np.abs(Q[c].ravel())))


def test_bgk_vacuum_and_degenerate_cells_do_not_relax(oracle):
    """BGK's Maxwellian needs rho > 0 and T > 0: a vacuum cell (f = 0) and a cell
    whose mass sits on one grid velocity (T = 0) have Q = 0; their neighbours in
    the same call are unaffected."""
    n, L = 8, 6.0
    f = I.two_stream((3, 1, 1), n, L, seed=4, noise=0.05)
    f[1] = 0.0
    f[2] = 0.0
    f[2][3, 4, 5] = 2.0
    Q = oracle.bgk(f, n, L, kn=0.5)
    assert np.all(Q[1] == 0.0) and np.all(Q[2] == 0.0)
    Q0 = oracle.bgk(f[:1], n, L, kn=0.5)
    assert np.array_equal(Q[0], Q0[0])


def _homog_exp(oracle, f, n, L, kn, dt, steps):
    sol = oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), n, L, None, kn)
    for _ in range(steps):
        f = sol.step_exp(f, dt)
    return f


def test_bgk_exponential_step_is_the_exact_relaxation(oracle):
    """The relaxation keeps M[f], nu and the projection term (collision invariants), so
    the exponential step solves it exactly: one step of dt equals two of dt/2."""
    n, L = 16, 8.0
    f = I.two_stream((1, 1, 1), n, L, seed=6, noise=0.05)
    one = _homog_exp(oracle, f, n, L, 0.05, 0.2, 1)
    two = _homog_exp(oracle, f, n, L, 0.05, 0.1, 2)
    assert np.abs(one - two).max() < 1e-12 * np.abs(one).max()
    # it differs from the Euler step by O((nu dt)^2): quartered when dt halves
    sol = oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), n, L, None, 5.0)
    d = [np.abs(sol.step_exp(f, dt) - sol.step(f, dt)).max() for dt in (0.02, 0.01)]
    assert 3.6 < d[0] / d[1] < 4.4


def test_bgk_exponential_step_stiff_limit(oracle):
    """Kn -> 0 with a fixed dt: the step lands on f* + Q/nu, the projected Maxwellian
    (the Euler step would overshoot by nu dt = 1e7)."""
    n, L, kn, dt = 16, 8.0, 1e-8, 0.1
    f = I.two_stream((1, 1, 1), n, L, seed=6, noise=0.05)
    out = _homog_exp(oracle, f, n, L, kn, dt, 1)
    Q = oracle.bgk(f, n, L, kn=kn)
    nu = f.sum() * (2 * L / n) ** 3 / kn
    lim = f + Q / nu
    assert np.abs(out - lim).max() < 1e-12 * np.abs(lim).max()
    # ... which is the cell's Maxwellian to the projection's small correction
    M = I.maxwellian(n, L, *(_moments(oracle, f[0], n, L)))
    assert np.abs(lim[0] - M).max() < 1e-3 * M.max()


def _moments(oracle, f, n, L):
    U = oracle.moments(f[None], n, L)[0]
    rho = U[0]
    u = U[1:4] / rho
    T = (U[4] - 0.5 * rho * (u ** 2).sum()) / (1.5 * rho)
    return rho, tuple(u), T
