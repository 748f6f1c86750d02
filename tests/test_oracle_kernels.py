"""Kernel transforms phi_R, psi_R, directions and tables (Appendix A) pinned
against scipy quadrature / Bessel functions and geometric facts."""
import numpy as np
import pytest
from scipy import integrate, special

R = 2.0 / (3.0 + np.sqrt(2.0)) * 8.0


@pytest.mark.parametrize("x", [0.0, 1e-4, 0.7, 5.0, 22.2, 41.0, 63.0])
def test_bessel_matches_scipy(oracle, x):
    assert abs(oracle.bessel_j(0, x) - special.j0(x)) < 2e-15
    assert abs(oracle.bessel_j(1, x) - special.j1(x)) < 2e-15


def _phi_quad(ktype, C, s):
    a = (lambda r: np.sqrt(4 * C)) if ktype == 0 else (lambda r: np.sqrt(4 * C) / np.sqrt(r))
    # phi(s) = int_{-R}^{R} |rho| a(|rho|) cos(rho s) d rho
    return 2 * integrate.quad(lambda r: r * a(r) * np.cos(r * s), 0, R, limit=400, epsabs=1e-13, epsrel=1e-12)[0]


def _psi_quad(ktype, C, s):
    b = (lambda r: np.sqrt(4 * C)) if ktype == 0 else (lambda r: np.sqrt(4 * C) / np.sqrt(r))
    # psi(s) = int_{disc radius R} b(|y|) exp(i s y_1) dy = 2 pi int_0^R r b(r) J0(r s) dr
    return 2 * np.pi * integrate.quad(lambda r: r * b(r) * special.j0(r * s), 0, R, limit=400,
                                      epsabs=1e-13, epsrel=1e-12)[0]


@pytest.mark.parametrize("ktype", [0, 1])
@pytest.mark.parametrize("s", [0.0, 1e-5, 0.37, 1.9, 6.3, 11.0])
def test_phi_psi_match_defining_integrals(oracle, ktype, s):
    C = 0.25 if ktype == 0 else 0.4
    assert abs(oracle.phi(ktype, C, R, s) - _phi_quad(ktype, C, s)) < 1e-11 * R * R
    assert abs(oracle.psi(ktype, C, R, s) - _psi_quad(ktype, C, s)) < 1e-11 * R * R


def test_hard_sphere_closed_forms(oracle):
    for s in [0.2, 1.0, 3.3]:
        assert abs(oracle.psi(0, 0.25, R, s) - 2 * np.pi * R * special.j1(R * s) / s) < 1e-12
        assert abs(oracle.phi(0, 0.25, R, s) - 2 * (R * np.sin(R * s) / s + (np.cos(R * s) - 1) / s ** 2)) < 1e-12
    assert abs(oracle.phi(0, 0.25, R, 0.0) - R * R) < 1e-13
    assert abs(oracle.psi(0, 0.25, R, 0.0) - np.pi * R * R) < 1e-13


@pytest.mark.parametrize("rule", [0, 1])
def test_directions_cover_half_sphere(oracle, rule):
    e, w = oracle.directions(16, 32, rule)
    np.testing.assert_allclose(np.linalg.norm(e, axis=1), 1.0, atol=1e-15)
    # area of the half sphere, midpoint / trapezoid rule in theta
    assert abs(w.sum() - 2 * np.pi) < 6.0 / 16 ** 2
    # no direction is the antipode of another (each class {e, -e} once)
    d = e @ e.T
    np.fill_diagonal(d, 0.0)
    assert d.min() > -1 + 1e-9
    # weight formula pi^2/(A1 A2) sin(theta)
    np.testing.assert_allclose(w, np.pi ** 2 / (16 * 32) * np.sqrt(1 - e[:, 2] ** 2), atol=1e-15)


@pytest.mark.parametrize("n", [8, 16])
def test_tables_are_hermitian_even(oracle, n):
    t = oracle.tables(n, 8.0, 0, 0.25, 4, 4, 0)
    neg = (-np.arange(n)) % n
    for arr in (t.alpha, t.alphap):
        flipped = arr[:, neg][:, :, neg][:, :, :, neg]
        np.testing.assert_allclose(arr, flipped, rtol=1e-14, atol=1e-14 * np.abs(arr).max())
    # zero mode: alpha(0) = phi(0) = R^2, alphap(0) = psi(0) = pi R^2
    np.testing.assert_allclose(t.alpha[:, 0, 0, 0], R * R, rtol=1e-14)
    np.testing.assert_allclose(t.alphap[:, 0, 0, 0], np.pi * R * R, rtol=1e-14)
    np.testing.assert_allclose(t.betaL, np.einsum("p,pijk,pijk->ijk", t.w, t.alpha, t.alphap), rtol=1e-14)
