"""Plain FP64 CPU oracle of the Fast Kinetic Scheme hot path (arXiv 1701.01608).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_1701_01608_gb300``; the arithmetic lives in
``fks_oracle.c`` (plain C, compiled here with gcc) and this module only
marshals numpy arrays.

Functions and the passage each follows:
  vgrid, moments         -- Sec. 2 (moments U = int phi f dv), Sec. 3 (sum over particles)
  offsets, transport     -- Sec. 2.1 "Transport step" (exact shift), Sec. 3 (generic cell)
  directions, phi, psi,
  tables, collide        -- Appendix A (Carleman form, separable kernel, quadrature
                            over half-sphere directions, fast spectral operator)
  galerkin               -- Appendix A, Eq. CF1 (O(N_v^2) sum), brute force
  project                -- conservation correction (collision invariants, Sec. 2)
  bgk                    -- BGK relaxation nu (M[f] - f) (Sec. 2, BGK approximation)
  step                   -- Eq. disc_relax: transport, then f = f* + dt Q(f*)
  step_strang            -- second-order splitting (Sec. 2.1 allows it): T(dt/2), Heun, T(dt/2)
  step_exp               -- stiff steps (Sec. 2.1, the stiff limit): exact BGK relaxation over dt;
                            for the spectral operator the integrating-factor step of the gain-loss
                            split with the loss frequency (loss_frequency) frozen at f*
  pad, truncate,
  collide_b, galerkin_b  -- variant B: Eq. CF1 with l + m = k not reduced mod n,
                            evaluated with 2n transforms (Sec. 5); brute force
  vhs_h, vhs_gain_loss,
  collide_vhs,
  galerkin_vhs           -- variable hard spheres B = C|g|^alpha: the non-separable
                            Carleman kernel of Eq. Btilde_pl, B_F(l, m) by a product
                            radial quadrature (Appendix A); brute force

Pins: every function is checked against values fixed outside this module by
tests/test_oracle_*.py (numpy.fft, scipy quadrature / Bessel functions, closed
forms, invariants, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile fks_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            D = ctypes.c_double
            I = ctypes.c_int
            Lg = ctypes.c_long
            P = ctypes.c_void_p
            lib.or_vgrid.argtypes = [I, D, P]
            lib.or_fft1d_ri.argtypes = [P, I, I]
            lib.or_fft3d_ri.argtypes = [P, I, I]
            lib.or_directions.argtypes = [I, I, I, P, P]
            lib.or_directions.restype = I
            lib.or_phi.argtypes = [I, D, D, D]
            lib.or_phi.restype = D
            lib.or_psi.argtypes = [I, D, D, D]
            lib.or_psi.restype = D
            lib.or_bessel_j.argtypes = [I, D]
            lib.or_bessel_j.restype = D
            lib.or_tables.argtypes = [I, D, I, D, I, I, I, P, P, P, P]
            lib.or_tables.restype = I
            lib.or_project.argtypes = [I, D, P]
            lib.or_collide.argtypes = [I, D, I, P, P, P, P, D, I, Lg, P, P]
            lib.or_gain_loss.argtypes = [I, I, P, P, P, P, P, P, P]
            lib.or_galerkin.argtypes = [I, I, P, P, P, P, D, P]
            lib.or_moments.argtypes = [I, D, Lg, P, P]
            lib.or_offsets.argtypes = [I, D, D, D, P, P]
            lib.or_transport.argtypes = [P, P, I, P, P, P]
            lib.or_bgk.argtypes = [I, D, D, I, Lg, P, P]
            lib.or_pad.argtypes = [I, P, P]
            lib.or_truncate.argtypes = [I, P, P]
            lib.or_collide_b.argtypes = [I, D, I, P, P, P, P, D, I, Lg, P, P]
            lib.or_galerkin_b.argtypes = [I, D, I, D, I, I, I, D, P, P]
            lib.or_vhs_h.argtypes = [D, D, D, D, D]
            lib.or_vhs_h.restype = D
            lib.or_vhs_gain_loss.argtypes = [I, D, D, D, I, I, I, Lg, P, P, P]
            lib.or_vhs_galerkin.argtypes = [I, D, D, D, I, I, I, D, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- grids / FFT

def vgrid(n: int, L: float) -> np.ndarray:
    v = np.empty(n)
    _L().or_vgrid(n, L, _p(v))
    return v


def fft1d(x, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _L().or_fft1d_ri(_p(a), a.shape[0], sign)
    return a


def fft3d(x, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    n = a.shape[0]
    assert a.shape == (n, n, n)
    _L().or_fft3d_ri(_p(a), n, sign)
    return a


# ---------------------------------------------------------------- kernel tables

HARD_SPHERE = 0
MAXWELL = 1  # separable pseudo-Maxwell kernel B~ = 4C (|x||y|)^(-1/2)

LAMBDA = 2.0 / (3.0 + np.sqrt(2.0))


def directions(A1: int, A2: int, rule: int = 0):
    M = A1 * A2
    e = np.empty((M, 3))
    w = np.empty(M)
    _L().or_directions(A1, A2, rule, _p(e), _p(w))
    return e, w


def phi(ktype: int, C: float, R: float, s: float) -> float:
    return _L().or_phi(ktype, C, R, s)


def psi(ktype: int, C: float, R: float, s: float) -> float:
    return _L().or_psi(ktype, C, R, s)


def bessel_j(nu: int, x: float) -> float:
    return _L().or_bessel_j(nu, x)


class Tables:
    """alpha[p], alphap[p], betaL on the standard DFT index grid, weights w."""

    def __init__(self, n, L, ktype, C, A1, A2, rule):
        self.n, self.L, self.ktype, self.C = n, L, ktype, C
        self.A1, self.A2, self.rule = A1, A2, rule
        M = A1 * A2
        self.M = M
        n3 = n ** 3
        self.alpha = np.empty((M, n, n, n))
        self.alphap = np.empty((M, n, n, n))
        self.betaL = np.empty((n, n, n))
        self.w = np.empty(M)
        _L().or_tables(n, L, ktype, C, A1, A2, rule, _p(self.alpha), _p(self.alphap),
                       _p(self.betaL), _p(self.w))
        assert self.alpha.size == M * n3


_table_cache: dict = {}


def tables(n, L, ktype=HARD_SPHERE, C=0.25, A1=4, A2=4, rule=0) -> Tables:
    key = (n, float(L), ktype, float(C), A1, A2, rule)
    t = _table_cache.get(key)
    if t is None:
        t = Tables(n, L, ktype, C, A1, A2, rule)
        _table_cache[key] = t
    return t


# ---------------------------------------------------------------- operators

def collide(f, tab: Tables, kn: float = 1.0, project: bool = True) -> np.ndarray:
    """Q(f)/Kn for every cell; f has shape (..., n, n, n)."""
    f = _f64(f)
    n = tab.n
    shp = f.shape
    assert shp[-3:] == (n, n, n)
    nc = int(np.prod(shp[:-3])) if len(shp) > 3 else 1
    Q = np.empty_like(f)
    _L().or_collide(n, tab.L, tab.M, _p(tab.alpha), _p(tab.alphap), _p(tab.w), _p(tab.betaL),
                    1.0 / kn, 1 if project else 0, nc, _p(f), _p(Q))
    return Q


def gain_loss(f, tab: Tables):
    f = _f64(f)
    n = tab.n
    G = np.empty((n, n, n))
    Lo = np.empty((n, n, n))
    _L().or_gain_loss(n, tab.M, _p(tab.alpha), _p(tab.alphap), _p(tab.w), _p(tab.betaL),
                      _p(f), _p(G), _p(Lo))
    return G, Lo


def loss_frequency(f, tab: Tables) -> np.ndarray:
    """l(v) = IDFT(betaL DFT(f)) / n^3 of one cell (Appendix A, the B_F(m, m) term): the loss term
    of the operator is f l, the loss frequency l / Kn.  The oracle's own 3-D FFT."""
    n = tab.n
    F = fft3d(np.asarray(f, dtype=np.float64).reshape(n, n, n), -1)
    return fft3d(tab.betaL * F, +1).real / n ** 3


def galerkin(f, tab: Tables, kn: float = 1.0) -> np.ndarray:
    f = _f64(f)
    Q = np.empty_like(f)
    _L().or_galerkin(tab.n, tab.M, _p(tab.alpha), _p(tab.alphap), _p(tab.w), _p(f), 1.0 / kn, _p(Q))
    return Q


def bgk(f, n: int, L: float, kn: float = 1.0, project: bool = True) -> np.ndarray:
    """BGK operator nu (M[f] - f), nu = rho / Kn, projected (Sec. 2, BGK approximation)."""
    f = _f64(f)
    nc = f.size // n ** 3
    Q = np.empty_like(f)
    _L().or_bgk(n, L, 1.0 / kn, 1 if project else 0, nc, _p(f), _p(Q))
    return Q


def pad(f, n: int) -> np.ndarray:
    """Trigonometric interpolant of an n^3 cell on the 2n grid (Nyquist split)."""
    f = _f64(f).reshape(n, n, n)
    f2 = np.empty((2 * n,) * 3)
    _L().or_pad(n, _p(f), _p(f2))
    return f2


def truncate(Q2, n: int) -> np.ndarray:
    """Modes |k| <= n/2 of a (2n)^3 array (+-n/2 folded), on the n grid."""
    Q2 = _f64(Q2).reshape((2 * n,) * 3)
    Q = np.empty((n, n, n))
    _L().or_truncate(n, _p(Q2), _p(Q))
    return Q


def collide_b(f, tab2: Tables, kn: float = 1.0, project: bool = True) -> np.ndarray:
    """Variant B (de-aliased) Q(f)/Kn for every n^3 cell of f; tab2 = tables(2n, L, ...)."""
    f = _f64(f)
    n = tab2.n // 2
    shp = f.shape
    assert shp[-3:] == (n, n, n)
    nc = int(np.prod(shp[:-3])) if len(shp) > 3 else 1
    Q = np.empty_like(f)
    _L().or_collide_b(n, tab2.L, tab2.M, _p(tab2.alpha), _p(tab2.alphap), _p(tab2.w), _p(tab2.betaL),
                      1.0 / kn, 1 if project else 0, nc, _p(f), _p(Q))
    return Q


def galerkin_b(f, n: int, L: float, ktype=HARD_SPHERE, C=0.25, A1=4, A2=4, rule=0, kn: float = 1.0) -> np.ndarray:
    """Brute-force unprojected variant B (Eq. CF1 without mod n) of one n^3 cell; n <= 8."""
    f = _f64(f).reshape(n, n, n)
    Q = np.empty_like(f)
    _L().or_galerkin_b(n, L, ktype, C, A1, A2, rule, 1.0 / kn, _p(f), _p(Q))
    return Q


def vhs_h(alpha: float, C: float, R: float, t: float, u: float) -> float:
    """Direction factor H(t, u) of the VHS kernel B = C|g|^alpha (product radial quadrature)."""
    return _L().or_vhs_h(alpha, C, R, t, u)


def vhs_gain_loss(f, n: int, L: float, alpha: float, C=0.25, A1=4, A2=4, rule=0):
    """Gain and loss of the VHS operator for every n^3 cell of f (no projection, no 1/Kn)."""
    f = _f64(f)
    shp = f.shape
    assert shp[-3:] == (n, n, n)
    nc = int(np.prod(shp[:-3])) if len(shp) > 3 else 1
    G = np.empty_like(f)
    Lo = np.empty_like(f)
    _L().or_vhs_gain_loss(n, L, alpha, C, A1, A2, rule, nc, _p(f), _p(G), _p(Lo))
    return G, Lo


def collide_vhs(f, n: int, L: float, alpha: float, C=0.25, A1=4, A2=4, rule=0, kn: float = 1.0,
                project: bool = True) -> np.ndarray:
    """VHS Q(f)/Kn for every cell, then (optionally) the conservation projection."""
    G, Lo = vhs_gain_loss(f, n, L, alpha, C, A1, A2, rule)
    Q = np.ascontiguousarray((G - Lo) / kn)
    if project:
        Qc = Q.reshape(-1, n, n, n)
        for c in range(Qc.shape[0]):
            _L().or_project(n, L, _p(Qc[c]))
    return Q


def galerkin_vhs(f, n: int, L: float, alpha: float, C=0.25, A1=4, A2=4, rule=0, kn: float = 1.0) -> np.ndarray:
    """Brute-force Eq. CF1 with the VHS B_F of one n^3 cell (unprojected); n <= 8."""
    f = _f64(f).reshape(n, n, n)
    Q = np.empty_like(f)
    _L().or_vhs_galerkin(n, L, alpha, C, A1, A2, rule, 1.0 / kn, _p(f), _p(Q))
    return Q


def project(Q, n: int, L: float) -> np.ndarray:
    Q = _f64(Q).copy()
    cells = Q.reshape(-1, n, n, n)
    for c in range(cells.shape[0]):
        blk = np.ascontiguousarray(cells[c])
        _L().or_project(n, L, _p(blk))
        cells[c] = blk
    return cells.reshape(Q.shape)


def moments(f, n: int, L: float) -> np.ndarray:
    f = _f64(f)
    nc = f.size // n ** 3
    U = np.empty((nc, 5))
    _L().or_moments(n, L, nc, _p(f), _p(U))
    return U


def offsets(n: int, L: float, dx, dt: float, s) -> tuple[np.ndarray, np.ndarray]:
    """Advance per-axis offsets s[3][n] by dt; return (s_new, delta[3][n])."""
    s = _f64(s).reshape(3, n).copy()
    delta = np.empty((3, n), dtype=np.int32)
    for a in range(3):
        sa = np.ascontiguousarray(s[a])
        da = np.empty(n, dtype=np.int32)
        _L().or_offsets(n, L, float(dx[a]), dt, _p(sa), _p(da))
        s[a] = sa
        delta[a] = da
    return s, delta


def transport(f, ncell, bc, delta) -> np.ndarray:
    """f*[j][k] = f[j - delta_k][k'] (exact shift); f shape (nx*ny*nz, n, n, n)."""
    f = _f64(f)
    n = f.shape[-1]
    nc = np.ascontiguousarray(ncell, dtype=np.int32)
    b = np.ascontiguousarray(bc, dtype=np.int32)
    d = np.ascontiguousarray(delta, dtype=np.int32).reshape(3, n)
    out = np.empty_like(f)
    _L().or_transport(_p(nc), _p(b), n, _p(d), _p(f), _p(out))
    return out


class Solver:
    """Plain FKS time loop: transport, then Euler collision step (Eq. disc_relax).
    tab = None: BGK relaxation; variant_b: tab holds the tables of the 2n grid and
    the collision is the de-aliased operator (collide_b); vhs = (alpha, C, A1, A2,
    rule): the variable-hard-sphere operator (collide_vhs), tab unused."""

    def __init__(self, ncell, x0, x1, bc, n, L, tab: Tables, kn: float, variant_b: bool = False,
                 vhs: tuple | None = None):
        self.ncell = tuple(int(c) for c in ncell)
        self.bc = tuple(int(b) for b in bc)
        self.dx = [(x1[a] - x0[a]) / self.ncell[a] for a in range(3)]
        self.n, self.L, self.tab, self.kn = n, L, tab, kn
        self.variant_b = variant_b
        self.vhs = vhs
        self.s = np.zeros((3, n))

    def transport(self, f, dt):
        self.s, delta = offsets(self.n, self.L, self.dx, dt, self.s)
        return transport(f, self.ncell, self.bc, delta)

    def step(self, f, dt):
        fs = self.transport(f, dt)
        if self.vhs is not None:
            Q = collide_vhs(fs, self.n, self.L, *self.vhs, kn=self.kn, project=True)
        elif self.tab is None:   # BGK relaxation
            Q = bgk(fs, self.n, self.L, self.kn, project=True)
        elif self.variant_b:
            Q = collide_b(fs, self.tab, self.kn, project=True)
        else:
            Q = collide(fs, self.tab, self.kn, project=True)
        return fs + dt * Q

    def collision(self, f):
        """Q(f)/Kn, projected, with this solver's operator."""
        if self.vhs is not None:
            return collide_vhs(f, self.n, self.L, *self.vhs, kn=self.kn, project=True)
        if self.tab is None:
            return bgk(f, self.n, self.L, self.kn, project=True)
        if self.variant_b:
            return collide_b(f, self.tab, self.kn, project=True)
        return collide(f, self.tab, self.kn, project=True)

    def step_exp(self, f, dt):
        """Stiff step (Sec. 2.1: care in the stiff limit).  BGK: transport, then the exact solution
        of the BGK relaxation with the cell's Maxwellian, rate nu = rho/Kn and projection term
        fixed: f* + (1 - exp(-nu dt)) / nu * Q(f*) per cell (dt where nu = 0).  Spectral operator:
        transport, then the gain-loss split df/dt = G - nu f with G and the loss frequency
        nu = l / Kn frozen at f*, solved per velocity point: the increment dt phi(nu dt) (G / Kn - nu f*),
        phi(x) = (1 - e^-x) / x, projected onto the constraints.  Where the discrete loss frequency is
        not positive (ringing of the truncated spectrum in the far tails, where f is negligible) the
        term stays explicit: phi(max(x, 0))."""
        assert self.vhs is None and not self.variant_b, "BGK or spectral (variant A) solvers"
        if self.tab is not None:
            fs = self.transport(f, dt)
            n = self.n
            out = np.empty_like(fs)
            cells = fs.reshape(-1, n, n, n)
            for c in range(cells.shape[0]):
                G, Lo = gain_loss(cells[c], self.tab)
                x = np.maximum(loss_frequency(cells[c], self.tab) / self.kn * dt, 0.0)
                safe = np.where(x != 0.0, x, 1.0)
                phi = np.where(x != 0.0, -np.expm1(-x) / safe, 1.0)
                inc = project(dt * phi * (G - Lo) / self.kn, n, self.L)
                out.reshape(-1, n, n, n)[c] = cells[c] + inc
            return out
        fs = self.transport(f, dt)
        Q = bgk(fs, self.n, self.L, self.kn, project=True)
        dv3 = (2.0 * self.L / self.n) ** 3
        shp = fs.shape
        fc = fs.reshape(-1, self.n ** 3)
        nu = fc.sum(axis=1) * dv3 / self.kn
        w = np.where(nu > 0, -np.expm1(-nu * dt) / np.where(nu > 0, nu, 1.0), dt)
        return (fc + w[:, None] * Q.reshape(fc.shape)).reshape(shp)

    def step_strang(self, f, dt):
        """Second-order step (Sec. 2.1 allows higher-order splitting): Strang splitting
        T(dt/2) C(dt) T(dt/2) with the collision sub-step by Heun's method, the
        second-order Runge-Kutta counterpart of Eq. disc_relax."""
        a = self.transport(f, 0.5 * dt)
        b = a + dt * self.collision(a)
        c = 0.5 * (a + b + dt * self.collision(b))
        return self.transport(c, 0.5 * dt)
