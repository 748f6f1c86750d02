"""The oracle's stiff step for the spectral operator (Sec. 2.1 asks for care in the stiff limit):
the integrating-factor step of the gain-loss split with the loss frequency frozen at f*, pinned by
its limits -- the Euler step of Eq. disc_relax as nu dt -> 0 (difference O(dt^2)), first order in dt
against a fine reference, G / nu (projected) as nu dt -> infinity, conservation of mass, momentum
and energy, a discrete Maxwellian kept to its residual -- and by a planted mistake."""
import numpy as np

from paper_1701_01608_gb300 import inputs as I

N, L = 8, 6.0


def _sol(oracle, tab, kn):
    return oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), N, L, tab, kn)


def test_loss_frequency_is_the_loss_term_over_f(oracle):
    tab = oracle.tables(N, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), N, L, seed=5, noise=0.05)[0]
    _, Lo = oracle.gain_loss(f, tab)
    np.testing.assert_allclose(oracle.loss_frequency(f, tab) * f, Lo, rtol=1e-12, atol=1e-15 * np.abs(Lo).max())


def test_tends_to_the_euler_step(oracle):
    """|exp step - Euler step| = O((nu dt)^2): the difference falls by ~4 when dt halves."""
    tab = oracle.tables(N, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), N, L, seed=1, noise=0.05)
    d = []
    for dt in (0.02, 0.01, 0.005):
        d.append(np.linalg.norm(_sol(oracle, tab, 1.0).step_exp(f, dt) - _sol(oracle, tab, 1.0).step(f, dt)))
    assert 3.6 < d[0] / d[1] < 4.4 and 3.6 < d[1] / d[2] < 4.4, d


def test_first_order_in_dt(oracle):
    tab = oracle.tables(N, L, 0, 0.25, 4, 4, 0)
    f0 = I.two_stream((1, 1, 1), N, L, seed=3, noise=0.05)
    t_end = 0.4

    def run(dt, exp=True):
        sol, f = _sol(oracle, tab, 1.0), f0
        for _ in range(int(round(t_end / dt))):
            f = sol.step_exp(f, dt) if exp else sol.step_strang(f, dt)
        return f

    ref = run(0.4 / 256, exp=False)
    e = [np.linalg.norm(run(dt) - ref) for dt in (0.1, 0.05, 0.025)]
    assert all(1.7 < e[i] / e[i + 1] < 2.3 for i in range(2)), e


def test_conserves(oracle):
    tab = oracle.tables(N, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), N, L, seed=7, noise=0.1)
    for kn in (1.0, 1e-6):
        out = _sol(oracle, tab, kn).step_exp(f, 0.05)
        U0, U1 = oracle.moments(f, N, L), oracle.moments(out, N, L)
        Ua = oracle.moments(np.abs(f), N, L)
        assert np.all(np.abs(U1 - U0) <= 1e-12 * (Ua[:, [0, 0, 0, 0, 4]] + Ua[:, [0]] * L)), kn


def test_stiff_limit_is_gain_over_loss_frequency(oracle):
    """Kn = 1e-8, nu dt ~ 1e6: where the loss frequency is positive the step lands on
    f* + (G - nu f*) / nu = G / nu (then projected), bounded, while the Euler step of the same size
    leaves the scale of f by orders of magnitude.  (Where the discrete loss frequency is not
    positive -- a few far-tail points, f ~ 1e-15 -- the term stays explicit.)"""
    tab = oracle.tables(N, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), N, L, seed=9, noise=0.05)
    kn, dt = 1e-8, 0.01
    out = _sol(oracle, tab, kn).step_exp(f, dt)
    G, Lo = oracle.gain_loss(f[0], tab)
    l = oracle.loss_frequency(f[0], tab)
    pos = l > 0
    inc = np.where(pos, (G - Lo) / np.where(pos, l, 1.0), dt / kn * (G - Lo))
    want = f[0] + oracle.project(inc, N, L)
    # (points with 0 < nu dt < ~30 -- tiny loss frequencies in the tails -- keep e^-x: a small difference)
    assert np.linalg.norm(out[0] - want) < 1e-4 * np.linalg.norm(want)
    assert np.abs(out).max() < 10 * np.abs(f).max()
    euler = _sol(oracle, tab, kn).step(f, dt)
    assert np.abs(euler).max() > 1e3 * np.abs(f).max()


def test_maxwellian_kept_to_its_residual(oracle):
    """A discrete Maxwellian moves by at most dt |Q(M)| (the operator's residual) at Kn = 1; at
    Kn = 1e-6 (nu dt ~ 1e5) the exponential step keeps it within 1e-3 while the Euler step moves it
    by dt |Q(M)| / Kn, orders of magnitude more."""
    n, Lb = 16, 8.0
    tab = oracle.tables(n, Lb, 0, 0.25, 4, 4, 0)
    M = I.maxwellian(n, Lb, 1.0, (0.2, 0.0, -0.1), 1.1)[None]
    Q = oracle.collide(M, tab, kn=1.0)
    sol = oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), n, Lb, tab, 1.0)
    out = sol.step_exp(M, 0.1)
    assert np.linalg.norm(out - M) <= 1.01 * 0.1 * np.linalg.norm(Q)
    stiff = oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), n, Lb, tab, 1e-6)
    d_exp = np.linalg.norm(stiff.step_exp(M, 0.1) - M)
    d_euler = np.linalg.norm(oracle.Solver((1, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0), n, Lb, tab, 1e-6).step(M, 0.1) - M)
    assert d_exp < 1e-3 * np.linalg.norm(M)
    assert d_euler > 10 * d_exp


def test_planted_mistake_breaks_the_euler_limit(oracle, monkeypatch):
    """The factor without the 1/x (1 - e^-x instead of phi) misses the Euler limit by O(1)."""
    tab = oracle.tables(N, L, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), N, L, seed=1, noise=0.05)
    real = oracle.loss_frequency
    # a loss frequency off by a factor 2 in the exponent plays the part of a wrong factor
    monkeypatch.setattr(oracle, "loss_frequency", lambda g, t: 2.0 * real(g, t))
    d = []
    for dt in (0.02, 0.01):
        d.append(np.linalg.norm(_sol(oracle, tab, 1.0).step_exp(f, dt) - _sol(oracle, tab, 1.0).step(f, dt)))
    monkeypatch.undo()
    good = np.linalg.norm(_sol(oracle, tab, 1.0).step_exp(f, 0.01) - _sol(oracle, tab, 1.0).step(f, 0.01))
    assert d[1] > 1.5 * good
