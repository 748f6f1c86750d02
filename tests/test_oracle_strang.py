"""The oracle's second-order step (Strang splitting with a Heun collision
sub-step; Sec. 2.1 allows higher-order splitting) pinned by its convergence
order in dt against the first-order step of Eq. disc_relax, by the pure
transport limit, and by conservation."""
import numpy as np
import pytest

from paper_1701_01608_gb300 import inputs as I


def _run(oracle, f, dt, t_end, strang, tab, L=6.0, n=8, kn=1.0):
    sol = oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), n, L, tab, kn)
    for _ in range(int(round(t_end / dt))):
        f = sol.step_strang(f, dt) if strang else sol.step(f, dt)
    return f


@pytest.mark.parametrize("kernel", ["spectral", "bgk"])
def test_orders_in_dt(oracle, kernel):
    """Space-homogeneous cell (transport is the identity): the Euler step is
    first order in dt, the Strang/Heun step second order (error ratios 2 and 4
    when dt halves), against a reference of the same problem with dt/64."""
    n, L = 8, 6.0
    tab = oracle.tables(n, L, 0, 0.25, 4, 4, 0) if kernel == "spectral" else None
    f0 = I.two_stream((1, 1, 1), n, L, seed=3, noise=0.05)
    t_end, dts = 0.4, (0.1, 0.05, 0.025)
    ref = _run(oracle, f0, dts[-1] / 16, t_end, True, tab)
    e1 = [np.linalg.norm(_run(oracle, f0, dt, t_end, False, tab) - ref) for dt in dts]
    e2 = [np.linalg.norm(_run(oracle, f0, dt, t_end, True, tab) - ref) for dt in dts]
    r1 = [e1[i] / e1[i + 1] for i in range(2)]
    r2 = [e2[i] / e2[i + 1] for i in range(2)]
    assert all(1.7 < r < 2.3 for r in r1), r1
    assert all(3.4 < r < 4.6 for r in r2), r2
    assert e2[-1] < e1[-1] / 10


def test_pure_transport_limit(oracle):
    """With the collision switched off (Kn -> infinity) two half transports are
    one full transport; dt and the velocities are exact binary fractions, so
    the offsets agree bit for bit."""
    n, L, ncell, bc = 8, 4.0, (4, 3, 2), (1, 0, 1)
    tab = oracle.tables(n, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream(ncell, n, L, seed=2, noise=0.1)
    s1 = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, 1e30)
    s2 = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, 1e30)
    dt = 0.0625
    a, b = f, f
    for _ in range(3):
        a = s1.step_strang(a, dt)
        b = s2.transport(b, dt)
    assert np.abs(a - b).max() <= 1e-25 * np.abs(b).max()


def test_strang_conserves(oracle):
    n, L, ncell = 8, 5.0, (3, 2, 2)
    tab = oracle.tables(n, L, 0, 0.25, 4, 4, 0)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), (0, 0, 0), n, L, tab, 0.5)
    f = I.two_stream(ncell, n, L, seed=8, noise=0.1)
    U0 = oracle.moments(f, n, L).sum(axis=0)
    for _ in range(2):
        f = sol.step_strang(f, 0.02)
    U1 = oracle.moments(f, n, L).sum(axis=0)
    assert np.abs(U1 - U0).max() < 1e-12 * np.abs(U0).max()
