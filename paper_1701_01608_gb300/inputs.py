"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method (no transform, no collision
operator, no transport): it only draws initial distributions, from
numpy ``PCG64(seed)``, and returns FP64 numpy arrays.  The same arrays feed
the CUDA library and the CPU oracle.

Layout of every distribution: ``f[cell][ix][iy][iz]`` (iz fastest) with
cell index ``(cx*ny + cy)*nz + cz``; velocities are the cell-centred points
``v_i = (i + 1/2 - n/2) * 2L/n`` of ``[-L, L]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def velocity_points(n: int, L: float) -> np.ndarray:
    return (np.arange(n) + 0.5 - 0.5 * n) * (2.0 * L / n)


def maxwellian(n: int, L: float, rho: float = 1.0, u=(0.0, 0.0, 0.0), T: float = 1.0) -> np.ndarray:
    """rho (2 pi T)^(-3/2) exp(-|v-u|^2 / 2T) at the velocity grid points."""
    v = velocity_points(n, L)
    vx = v[:, None, None] - u[0]
    vy = v[None, :, None] - u[1]
    vz = v[None, None, :] - u[2]
    return rho * (2 * np.pi * T) ** -1.5 * np.exp(-(vx * vx + vy * vy + vz * vz) / (2 * T))


def bkw(n: int, L: float, K: float, T: float = 1.0, rho: float = 1.0) -> np.ndarray:
    """BKW profile for Maxwell-type kernels at similarity parameter K,
    scaled to temperature T:
    f = rho (2 pi K T)^(-3/2) exp(-v^2/(2KT)) [(5K-3)/(2K) + (1-K)/(2K^2) v^2/T]."""
    v = velocity_points(n, L)
    v2 = (v[:, None, None] ** 2 + v[None, :, None] ** 2 + v[None, None, :] ** 2) / T
    return (rho * (2 * np.pi * K * T) ** -1.5 * np.exp(-v2 / (2 * K))
            * ((5 * K - 3) / (2 * K) + (1 - K) / (2 * K * K) * v2))


@dataclass
class Workload:
    name: str
    ncell: tuple            # (nx, ny, nz)
    x0: tuple
    x1: tuple
    bc: tuple               # per axis: 0 periodic, 1 specular
    n: int                  # velocity points per axis
    L: float                # velocity box [-L, L]^3
    kernel: int             # 0 hard spheres, 1 pseudo-Maxwell
    C: float
    kn: float
    A1: int
    A2: int
    steps: int
    f0: np.ndarray = field(repr=False, default=None)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.ncell))

    @property
    def M(self) -> int:
        return self.A1 * self.A2


def two_stream(ncell=(4, 4, 4), n=16, L=8.0, seed=0, noise=0.01, amp=0.2) -> np.ndarray:
    """rho(x) = 1 + amp sin(2 pi x) times the mean of two unit-temperature
    Maxwellians at mean velocities +-e_x, times (1 + noise U(-1,1))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = ncell
    base = 0.5 * (maxwellian(n, L, u=(1.0, 0, 0)) + maxwellian(n, L, u=(-1.0, 0, 0)))
    xc = (np.arange(nx) + 0.5) / nx
    f = np.empty((nx, ny, nz, n, n, n))
    for cx in range(nx):
        f[cx] = (1.0 + amp * np.sin(2 * np.pi * xc[cx])) * base
    f = f.reshape(nx * ny * nz, n, n, n)
    f *= 1.0 + noise * rng.uniform(-1.0, 1.0, size=f.shape)
    return f


def config_small_periodic(seed: int = 0) -> Workload:
    """4^3 periodic cells on [0,1]^3, 16^3 velocities on [-8,8]^3, M = 16,
    hard spheres, Kn = 0.1, two-stream initial data, 10 steps."""
    w = Workload("hs_periodic_4c_16v", (4, 4, 4), (0, 0, 0), (1, 1, 1), (0, 0, 0),
                 16, 8.0, 0, 0.25, 0.1, 4, 4, 10)
    w.f0 = two_stream((4, 4, 4), 16, 8.0, seed)
    return w


def config_homogeneous_bkw(ncells: int = 4096, n: int = 32, seed: int = 1, K0: float = 0.6) -> Workload:
    """ncells independent homogeneous cells, 32^3 velocities on [-10,10]^3,
    M = 32 (4 x 8), pseudo-Maxwell kernel, BKW data at K0 with per-cell
    temperature U[0.8, 1.2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T = rng.uniform(0.8, 1.2, size=ncells)
    w = Workload(f"maxwell_homog_{ncells}c_{n}v", (ncells, 1, 1), (0, 0, 0), (1, 1, 1), (0, 0, 0),
                 n, 10.0, 1, 0.25, 1.0, 4, 8, 50)
    w.f0 = np.stack([bkw(n, 10.0, K0, T=t) for t in T])
    w.T = T
    return w


def config_shock_tube(ncell=(32, 32, 32), n: int = 32, L: float = 10.0, seed: int = 2,
                      noise: float = 0.0) -> Workload:
    """Shock tube on [0,1]^3: Maxwellian rho=1, T=1 for x < 0.5, rho=0.125,
    T=0.8 otherwise; specular walls in x, periodic in y and z; M = 32
    (4 x 8), hard spheres, Kn = 0.01, 100 steps.  ``noise`` > 0 multiplies by
    (1 + noise U(-1,1)) (used by parity tests to leave equilibrium)."""
    nx, ny, nz = ncell
    left = maxwellian(n, L, 1.0, T=1.0)
    right = maxwellian(n, L, 0.125, T=0.8)
    xc = (np.arange(nx) + 0.5) / nx
    f = np.empty((nx, ny * nz, n, n, n))
    for cx in range(nx):
        f[cx] = left if xc[cx] < 0.5 else right
    f = f.reshape(nx * ny * nz, n, n, n)
    if noise > 0:
        rng = np.random.Generator(np.random.PCG64(seed))
        f *= 1.0 + noise * rng.uniform(-1.0, 1.0, size=f.shape)
    w = Workload(f"hs_shocktube_{nx}x{ny}x{nz}c_{n}v", tuple(ncell), (0, 0, 0), (1, 1, 1), (1, 0, 0),
                 n, L, 0, 0.25, 0.01, 4, 8, 100)
    w.f0 = f
    return w


def config_uneven_batch(nprob: int = 96, seed: int = 3):
    """nprob homogeneous problems: n from {16, 24, 32}, Kn log-uniform in
    [1e-3, 1], hard-sphere or pseudo-Maxwell kernel, two-Maxwellian data
    with seeded means in [-1,1] and temperatures in [0.8, 1.2]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    for i in range(nprob):
        n = int(rng.choice([16, 24, 32]))
        kn = float(10 ** rng.uniform(-3, 0))
        kernel = int(rng.integers(0, 2))
        u1 = rng.uniform(-1, 1, size=3)
        u2 = rng.uniform(-1, 1, size=3)
        T1, T2 = rng.uniform(0.8, 1.2, size=2)
        L = 8.0 if n == 16 else 10.0
        f = 0.5 * (maxwellian(n, L, u=u1, T=T1) + maxwellian(n, L, u=u2, T=T2))
        probs.append(dict(n=n, L=L, kn=kn, kernel=kernel, f0=f[None]))
    return probs


def shock_tube_states(n: int = 32, L: float = 10.0, nx: int = 32):
    """The two Maxwellian profiles of the shock tube (left rho=1 T=1, right
    rho=0.125 T=0.8) and, per x index, which one the cells hold (0 left,
    1 right).  Lets a caller assemble the 32^3 x 32^3 state on the device
    without a host copy of the whole array."""
    left = maxwellian(n, L, 1.0, T=1.0)
    right = maxwellian(n, L, 0.125, T=0.8)
    xc = (np.arange(nx) + 0.5) / nx
    return np.stack([left, right]), (xc >= 0.5).astype(np.int64)
