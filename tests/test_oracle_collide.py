"""Oracle fast spectral operator (Appendix A) pinned against the O(N_v^2)
Galerkin sum, conservation, Q(M) = 0, quadratic scaling, symmetries, the
closed-form loss frequency of a Maxwellian and the BKW solution."""
import numpy as np
import pytest
from scipy.special import erf, gamma

from paper_1701_01608_gb300 import inputs as I


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("ktype,rule,L", [(0, 0, 6.0), (0, 1, 6.0), (1, 0, 7.0)])
def test_fast_operator_equals_galerkin_sum(oracle, ktype, rule, L):
    """Eq. CF1: the fast product form is the circular Galerkin sum with the
    same discrete beta_F, an identity up to rounding."""
    t = oracle.tables(8, L, ktype, 0.25, 4, 4, rule)
    f = I.two_stream((1, 1, 1), 8, L, seed=5, noise=0.05)[0]
    Qf = oracle.collide(f, t, kn=0.5, project=False)
    Qg = oracle.galerkin(f, t, kn=0.5)
    assert relerr(Qf, Qg) < 1e-12


def test_galerkin_catches_a_wrong_operator(oracle):
    """Sanity of the pin: dropping the loss term is detected."""
    t = oracle.tables(8, 6.0, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), 8, 6.0, seed=5, noise=0.05)[0]
    G, Lo = oracle.gain_loss(f, t)
    assert relerr(G, oracle.galerkin(f, t)) > 1e-2


@pytest.mark.parametrize("ktype", [0, 1])
def test_mass_conserved_and_quadratic(oracle, ktype):
    t = oracle.tables(16, 8.0, ktype, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), 16, 8.0, seed=1)[0]
    Q = oracle.collide(f, t, project=False)
    assert abs(Q.sum()) < 1e-13 * np.abs(Q).sum()
    Q3 = oracle.collide(3.0 * f, t, project=False)
    assert relerr(Q3, 9.0 * Q) < 1e-13


def test_translation_and_reflection_covariance(oracle):
    """The discrete operator commutes with grid translations (circular) and
    with the reflection v_x -> -v_x (the direction set is symmetric)."""
    t = oracle.tables(16, 8.0, 0, 0.25, 4, 4, 0)
    f = I.two_stream((1, 1, 1), 16, 8.0, seed=2)[0]
    Q = oracle.collide(f, t, project=False)
    Qs = oracle.collide(np.roll(f, (3, -2, 1), axis=(0, 1, 2)), t, project=False)
    assert relerr(Qs, np.roll(Q, (3, -2, 1), axis=(0, 1, 2))) < 1e-12
    Qr = oracle.collide(f[::-1].copy(), t, project=False)
    assert relerr(Qr, Q[::-1]) < 1e-12


def test_maxwellian_is_equilibrium_spectrally(oracle):
    """Q(M) = 0 up to the spectral error, which falls fast with n."""
    errs = []
    for n in (16, 24, 32):
        t = oracle.tables(n, 8.0, 0, 0.25, 4, 4, 0)
        M = I.maxwellian(n, 8.0, T=0.5)
        G, Lo = oracle.gain_loss(M, t)
        errs.append(np.abs(G - Lo).max() / np.abs(Lo).max())
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 10
    assert errs[2] < 1e-5
    # a non-equilibrium state is far from that level
    f = 0.5 * (I.maxwellian(32, 8.0, u=(1, 0, 0), T=0.5) + I.maxwellian(32, 8.0, u=(-1, 0, 0), T=0.5))
    G, Lo = oracle.gain_loss(f, oracle.tables(32, 8.0, 0, 0.25, 4, 4, 0))
    assert np.abs(G - Lo).max() / np.abs(Lo).max() > 1e-2


def _loss_frequency(oracle, ktype, A, n=24, L=8.0, T=0.5):
    t = oracle.tables(n, L, ktype, 0.25, A, A, 0)
    M = I.maxwellian(n, L, T=T)
    G, Lo = oracle.gain_loss(M, t)
    return Lo / M


@pytest.mark.slow
def test_hard_sphere_loss_frequency_closed_form(oracle):
    """nu(v) = 4 pi C int |v - w| M(w) dw for hard spheres (B = C|g|); for a
    Maxwellian of temperature T, int |v-w| M = sqrt(2T) [exp(-s^2)/sqrt(pi)
    + (s + 1/(2s)) erf(s)], s = |v|/sqrt(2T).  The direction quadrature is
    second order in A; Richardson extrapolation from A = 4, 8 must hit the
    closed form near the centre (where the cut-off R is inactive)."""
    n, L, T = 24, 8.0, 0.5
    v = I.velocity_points(n, L)
    V = np.sqrt(v[:, None, None] ** 2 + v[None, :, None] ** 2 + v[None, None, :] ** 2)
    s = V / np.sqrt(2 * T)
    exact = 4 * np.pi * 0.25 * np.sqrt(2 * T) * (np.exp(-s * s) / np.sqrt(np.pi) + (s + 1 / (2 * s)) * erf(s))
    inner = V < 1.0
    n4 = _loss_frequency(oracle, 0, 4)
    n8 = _loss_frequency(oracle, 0, 8)
    e4 = np.abs(n4 / exact - 1)[inner].max()
    e8 = np.abs(n8 / exact - 1)[inner].max()
    assert 3.0 < e4 / e8 < 5.0          # second-order convergence in A
    rich = (4 * n8 - n4) / 3
    assert np.abs(rich / exact - 1)[inner].max() < 1e-3


@pytest.mark.slow
def test_pseudo_maxwell_loss_frequency_closed_form(oracle):
    """Maxwell-type kernel B = C (sin(theta)/2)^(-1/2): nu = rho int B d omega
    = rho 2 pi C sqrt(2) int_0^pi sin^(1/2)(t) dt, independent of v."""
    const = 2 * np.pi * 0.25 * np.sqrt(2) * np.sqrt(np.pi) * gamma(0.75) / gamma(1.25)
    n, L = 24, 8.0
    v = I.velocity_points(n, L)
    V = np.sqrt(v[:, None, None] ** 2 + v[None, :, None] ** 2 + v[None, None, :] ** 2)
    n4 = _loss_frequency(oracle, 1, 4)
    n8 = _loss_frequency(oracle, 1, 8)
    rich = (4 * n8 - n4) / 3
    assert np.abs(rich / const - 1)[V < 1.0].max() < 1e-3


@pytest.mark.slow
def test_bkw_shape_and_rate(oracle):
    """BKW: for Maxwell-type kernels f(t) = BKW(K(t)), K = 1 - exp(-lam t),
    so Q(f) = lam (1-K) df/dK, with lam = (1/4) int B sin^2(theta) d omega.
    The fitted rate (Richardson in A) must match that value and the shape
    residual must be small."""
    lam_th = 0.25 * 2 * np.pi * 0.25 * np.sqrt(2) * np.sqrt(np.pi) * gamma(1.75) / gamma(2.25)
    n, L, T, K = 24, 8.0, 0.7, 0.7
    f = I.bkw(n, L, K, T=T)
    h = 1e-6
    d = (I.bkw(n, L, K + h, T=T) - I.bkw(n, L, K - h, T=T)) / (2 * h)
    lams = []
    for A in (4, 8):
        Q = oracle.collide(f, oracle.tables(n, L, 1, 0.25, A, A, 0), project=False)
        c = (Q * d).sum() / (d * d).sum()
        lams.append(c / (1 - K))
        resid = np.linalg.norm(Q - c * d) / np.linalg.norm(Q)
    assert resid < 0.02
    lam_rich = (4 * lams[1] - lams[0]) / 3
    assert abs(lam_rich / lam_th - 1) < 5e-3


@pytest.mark.parametrize("n", [8, 16])
def test_projection(oracle, n):
    L = 8.0
    rng = np.random.default_rng(n)
    Q = rng.standard_normal((n, n, n))
    Qc = oracle.project(Q, n, L)
    v = I.velocity_points(n, L)
    dv3 = (2 * L / n) ** 3
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    C = np.stack([np.ones_like(vx), vx, vy, vz, 0.5 * (vx ** 2 + vy ** 2 + vz ** 2)]).reshape(5, -1) * dv3
    m = C @ Qc.ravel()
    assert np.abs(m).max() < 1e-13 * (np.abs(C) @ np.abs(Qc.ravel())).max()
    # idempotent, and the correction lies in the span of the invariants
    np.testing.assert_allclose(oracle.project(Qc, n, L), Qc, atol=1e-13)
    coef, *_ = np.linalg.lstsq(C.T, (Q - Qc).ravel(), rcond=None)
    np.testing.assert_allclose(C.T @ coef, (Q - Qc).ravel(), atol=1e-12)
