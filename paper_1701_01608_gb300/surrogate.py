"""Training and calibration of the learned collision surrogate.

The surrogate replaces the fast spectral operator on cells near equilibrium;
the spectral operator is its fallback and the measure of its error.  This module
drives the library's kernels (fks.Net, fks.surrogate_inputs,
Context.surrogate_collide): it generates (f, Q) pairs with the spectral solver
itself, trains the network (own BF16 forward/backward/Adam kernels), and
calibrates the error indicator on held-out cells so that the calibrated
indicator bounds the true relative error on >= 99 % of them.  The indicator is
ind_scale / d + defect (d = ||f - M|| / ||M||, defect = relative moment defect of
the raw output): the network's absolute error is about a fixed fraction of its
output scale, while ||Q|| shrinks with d near equilibrium.

Targets: y = Q Kn / (rho^2 s) with a global scale s (the operator is
quadratic: Q(rho g) = rho^2 Q(g)); Q is the hard-sphere operator.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fks
from . import inputs as I


@dataclass
class Surrogate:
    net: "fks.Net"
    out_scale: float
    ind_scale: float
    n: int
    L: float
    train_loss: list
    calib: dict


def shock_tube_cells(torch, n=32, L=10.0, nx=32, ny=2, nz=2, steps=(0, 4, 8, 16), kn=0.01, seed=0):
    """FP32 cells of a (nx, ny, nz) shock tube (specular x walls) after the
    given numbers of FKS steps (spectral FP32), with (1 + 0.02 U(-1,1)) noise."""
    ctx = fks.Context(fks.Config(ncell=(nx, ny, nz), bc=(1, 0, 0), n=n, L=L, kn=kn, A1=4, A2=8,
                                 precision=fks.FKS_FP32))
    states, which = I.shock_tube_states(n, L, nx)
    st = torch.from_numpy(states).float().cuda()
    f = st.index_select(0, torch.from_numpy(np.repeat(which, ny * nz)).cuda()).contiguous()
    g = torch.Generator(device="cuda").manual_seed(seed)
    f *= 1.0 + 0.02 * (2.0 * torch.rand(f.shape, generator=g, device="cuda") - 1.0)
    out, fb = [], torch.empty_like(f)
    dt = min((1.0 / nx) / L, 0.1 * kn)
    done = 0
    for s in sorted(steps):
        while done < s:
            ctx.step(f, fb, dt)
            f, fb = fb, f
            done += 1
        out.append(f.clone())
    return torch.cat(out)


def two_stream_cells(torch, count, n=32, L=10.0, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = []
    for _ in range(count):
        a = rng.uniform(0.2, 1.5)
        T = rng.uniform(0.6, 1.2)
        u = rng.uniform(-0.5, 0.5, 3)
        f = 0.5 * (I.maxwellian(n, L, 1.0, (u[0] + a, u[1], u[2]), T) + I.maxwellian(n, L, 1.0, (u[0] - a, u[1], u[2]), T))
        cells.append(f * rng.uniform(0.3, 2.0))
    return torch.from_numpy(np.stack(cells)).float().cuda()


def labels(torch, f, n=32, L=10.0, kn=1.0):
    """Projected hard-sphere Q (FP32 spectral) of every cell of f, at Knudsen kn."""
    ctx = fks.Context(fks.Config(ncell=(f.shape[0], 1, 1), n=n, L=L, kn=kn, A1=4, A2=8, precision=fks.FKS_FP32))
    Q = torch.empty_like(f)
    ctx.collide(f, Q)
    return Q


def train(torch, f, Q, epochs=20, batch=8, lr=2e-3, seed=0, kn=1.0, n=32, L=10.0, holdout=0.2, log=None,
          steps=None):
    """Train a network on (f, Q) pairs (Q at Knudsen kn); returns the Surrogate.  steps: a fixed
    number of Adam steps on random batches with a cosine learning-rate decay, instead of epochs
    with step decay."""
    nc = f.shape[0]
    x = torch.empty((nc, 2, n, n, n), device="cuda")
    rho = torch.empty(nc, dtype=torch.float64, device="cuda")
    dist = torch.empty(nc, device="cuda")
    fks.surrogate_inputs(n, L, f, x, rho, dist)
    y = (Q.double() * kn / (rho[:, None, None, None] ** 2)).float()
    out_scale = float(y.std().item()) or 1.0
    y = (y / out_scale).reshape(nc, 1, n, n, n).contiguous()
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(nc)
    nh = max(1, int(holdout * nc))
    hold, tr = perm[:nh], perm[nh:]
    net = fks.Net(n, batch, seed=seed)
    losses = []
    if steps:
        loss = torch.zeros(1, device="cuda")
        for it in range(steps):
            idx = torch.from_numpy(rng.choice(tr, batch, replace=len(tr) < batch)).cuda()
            lr_it = lr * 0.5 * (1.0 + np.cos(np.pi * it / steps))
            net.train_step(x.index_select(0, idx).contiguous(), y.index_select(0, idx).contiguous(), lr_it, loss)
            if (it + 1) % 250 == 0 or it + 1 == steps:
                losses.append(loss.item() / ((it % 250) + 1))
                loss.zero_()
                if log:
                    log(f"step {it + 1}: loss {losses[-1]:.4e}")
        epochs = 0
    for ep in range(epochs):
        order = rng.permutation(tr)
        loss = torch.zeros(1, device="cuda")
        nb = 0
        for i in range(0, len(order) - batch + 1, batch):
            idx = torch.from_numpy(order[i:i + batch]).cuda()
            xb = x.index_select(0, idx).contiguous()
            yb = y.index_select(0, idx).contiguous()
            net.train_step(xb, yb, lr * (0.5 ** (ep // max(1, epochs // 3))), loss)
            nb += 1
        losses.append(loss.item() / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    sur = Surrogate(net, out_scale, 1.0, n, L, losses, {})
    sur.calib = calibrate(torch, sur, f[torch.from_numpy(hold).cuda()].contiguous(),
                          Q[torch.from_numpy(hold).cuda()].contiguous(), kn=kn)
    sur.ind_scale = sur.calib["ind_scale"]
    return sur


def surrogate_errors(torch, sur, f, Q, kn=1.0):
    """Relative L2 error of the surrogate's projected Q per cell (every cell inferred), the raw
    indicators (ind_scale = 1: 1 / d + defect) and the distances d from equilibrium."""
    nc = f.shape[0]
    ctx = fks.Context(fks.Config(ncell=(nc, 1, 1), n=sur.n, L=sur.L, kn=kn, A1=4, A2=8, precision=fks.FKS_FP32))
    Qs = torch.empty_like(f)
    ctx.surrogate_collide(sur.net, f, Qs, sur.out_scale, 1.0, 1e30)
    ind = ctx.indicator()
    x = torch.empty((nc, 2, sur.n, sur.n, sur.n), device="cuda")
    rho = torch.empty(nc, dtype=torch.float64, device="cuda")
    dist = torch.empty(nc, device="cuda")
    fks.surrogate_inputs(sur.n, sur.L, f, x, rho, dist)
    err = ((Qs - Q).double().flatten(1).norm(dim=1) / Q.double().flatten(1).norm(dim=1)).cpu().numpy()
    return err, ind, dist.double().cpu().numpy()


def calibrate(torch, sur, f, Q, kn=1.0, quantile=0.99):
    """ind_scale such that the indicator ind_scale / d + defect bounds the relative error on
    `quantile` of the held-out cells: the quantile of (err - defect) d (defect = raw - 1 / d)."""
    err, ind, d = surrogate_errors(torch, sur, f, Q, kn)
    d = np.maximum(d, 1e-30)
    defect = np.maximum(ind - 1.0 / d, 0.0)
    need = np.maximum(err - defect, 0.0) * d
    scale = float(np.quantile(need, quantile))
    cert = scale / d + defect
    return {"ind_scale": scale, "holdout": int(len(err)), "err_median": float(np.median(err)),
            "err_max": float(err.max()), "err_q10": float(np.quantile(err, 0.1)),
            "covered": float(np.mean(cert >= err)),
            "certified_at_1e-3": float(np.mean(cert <= 1e-3))}
