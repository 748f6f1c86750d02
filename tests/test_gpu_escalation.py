"""Precision escalation near equilibrium (the FP64 kept for the gain-loss
subtraction near equilibrium): the FP32 and split-BF16 paths against the FP64
oracle at the plain per-cell bounds (relative L2 of Q <= 1e-5 and <= 1e-3) on
shock-tube cells, n = 32, M = 32, hard spheres, Kn = 0.01:
  - the exact discrete Maxwellians of the initial state (left rho = 1, T = 1;
    right rho = 0.125, T = 0.8), where Q is the discrete operator's own
    residual, ~1e-7 .. 3e-6 of the loss term (||L|| / ||Q|| up to ~1e7);
  - the left state times (1 + eps U(-1, 1)), eps = 1e-2 .. 1e-5;
  - cells of the 32-cell tube after 4 and 16 oracle steps (dt = 1e-3).
Without the escalation the same cells miss the bounds by orders of magnitude."""
import numpy as np
import pytest

from conftest import BF16_REL, FP32_REL
from paper_1701_01608_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, L, KN, A = 32, 10.0, 0.01, (4, 8)


@pytest.fixture(scope="module")
def fks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_01608_gb300 import fks
    fks.lib()
    return fks


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def tab(oracle):
    return oracle.tables(N, L, 0, 0.25, A[0], A[1], 0)


@pytest.fixture(scope="module")
def shock_cells(oracle, tab):
    """FP32-representable cells (the GPU reads FP32) and their FP64 oracle Q."""
    w = I.config_shock_tube(ncell=(32, 1, 1), n=N, L=L)
    cells = [w.f0[3], w.f0[28]]
    rng = np.random.Generator(np.random.PCG64(11))
    for eps in (1e-2, 1e-3, 1e-4, 1e-5):
        cells.append(w.f0[3] * (1.0 + eps * rng.uniform(-1.0, 1.0, size=w.f0[3].shape)))
    sol = oracle.Solver((32, 1, 1), (0, 0, 0), (1, 1, 1), (1, 0, 0), N, L, tab, KN)
    f = w.f0.astype(np.float32).astype(np.float64)
    for k in range(16):
        f = sol.step(f, 1e-3)
        if k + 1 in (4, 16):
            cells += [f[i] for i in (13, 15, 16, 18, 21)]
    f32 = np.stack(cells).astype(np.float32)
    f64 = f32.astype(np.float64)
    Qo = oracle.collide(f64, tab, kn=KN)
    kappa = np.array([np.linalg.norm(oracle.gain_loss(c, tab)[1]) / KN / np.linalg.norm(q) for c, q in zip(f64, Qo)])
    return f32, Qo, kappa


def make_ctx(fks, nc, prec, bc=(0, 0, 0)):
    return fks.Context(fks.Config(ncell=(nc, 1, 1), bc=bc, n=N, L=L, kn=KN, A1=A[0], A2=A[1], precision=prec))


@pytest.mark.parametrize("prec,tol,arith", [(1, FP32_REL, 3), (2, BF16_REL, 3), (1, FP32_REL, 0)])
def test_near_equilibrium_cells_meet_plain_bound(fks, shock_cells, prec, tol, arith):
    f32, Qo, kappa = shock_cells
    # the sample spans the conditioning range of the workload
    assert kappa.max() > 1e5 and kappa.min() < 100
    nc = f32.shape[0]
    ctx = make_ctx(fks, nc, prec)
    assert ctx.escalation()[0] == tol   # on by default at the stated bound
    ctx.set_escalation_arith(arith)   # last tier: double-float (3, the default) or FP64 (0)
    fd = torch.from_numpy(f32).cuda()
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    assert ctx.check() == 0
    Qg = Q.double().cpu().numpy()
    errs = [rel(Qg[c], Qo[c]) for c in range(nc)]
    for c in range(nc):
        assert errs[c] < tol, (c, kappa[c], errs[c])
    _, counts = ctx.escalation()
    assert counts[0] > 0   # the exact Maxwellians at least
    if prec == 2:
        assert counts[1] > 0   # cells beyond the FP32 tier's reach go on to FP64
    # the same cells without escalation: the raw arithmetic misses the bound
    ctx.set_escalation(0.0)
    ctx.collide(fd, Q)
    raw = [rel(Q[c].double().cpu().numpy(), Qo[c]) for c in range(nc)]
    assert max(raw) > 10 * tol
    # the escalated result is deterministic (the order of the device list does not matter)
    ctx.set_escalation(tol)
    Q2 = torch.empty_like(fd)
    ctx.collide(fd, Q2)
    assert torch.equal(Q2, torch.from_numpy(Qg.astype(np.float32)).cuda())


def test_direct_route_to_last_tier_is_identical(fks, shock_cells):
    """Split BF16 at 1e-3: cells whose FP32 bound must exceed the tolerance (the split-BF16 kernel's own
    estimates of ||Q|| and ||L||, its error allowed for) go straight to the last tier.  The results equal
    those of the route through the FP32 tier bit for bit; the last tier receives the same number of
    cells, the FP32 tier fewer (the exact Maxwellians skip it)."""
    f32, Qo, kappa = shock_cells
    nc = f32.shape[0]
    ctx = make_ctx(fks, nc, 2)
    fd = torch.from_numpy(f32).cuda()
    Qa, Qb = torch.empty_like(fd), torch.empty_like(fd)
    ctx.collide(fd, Qa)
    direct = ctx.escalation()[1]
    ctx.set_escalation_direct(False)
    ctx.collide(fd, Qb)
    through = ctx.escalation()[1]
    assert ctx.check() == 0
    assert torch.equal(Qa, Qb)
    assert direct[1] == through[1] > 0
    assert direct[0] < through[0]
    ctx.set_escalation_direct(True)
    ctx.collide(fd, Qb)
    assert torch.equal(Qa, Qb) and ctx.escalation()[1] == direct


@pytest.mark.parametrize("prec,tol", [(2, BF16_REL), (1, FP32_REL)])
def test_direct_route_from_the_classification_is_identical(fks, shock_cells, prec, tol):
    """The surrogate's classification sends cells with d = ||f - M|| / ||M|| below 0.1 c_32 / tol
    (5e-5 at 1e-3, 5e-3 at 1e-5: the exact Maxwellians and the small perturbations) straight to the
    last tier, past the context's own kernel.  Every cell is routed (random network, indicator scale
    1); the results equal those of the route through every tier bit for bit and meet the bound
    against the oracle."""
    f32, Qo, kappa = shock_cells
    nc = f32.shape[0]
    net = fks.Net(N, 2, seed=5)
    fd = torch.from_numpy(f32).cuda()
    outs, counts = [], []
    for direct in (True, False):
        ctx = make_ctx(fks, nc, prec)
        ctx.set_escalation_direct(direct)
        out = torch.empty_like(fd)
        assert ctx.surrogate_collide(net, fd, out, 1.0, 1.0, tol) == nc
        assert ctx.check() == 0
        outs.append(out)
        counts.append(ctx.escalation()[1])
    assert torch.equal(outs[0], outs[1])
    last = 1 if prec == 2 else 0
    assert counts[0][last] == counts[1][last] > 0
    if prec == 2:
        assert counts[0][0] < counts[1][0]
    for c in range(nc):
        assert rel(outs[0][c].double().cpu().numpy(), Qo[c]) < tol, (c, kappa[c])


def test_escalated_step_fp32(fks, oracle, tab, shock_cells):
    """One fused transport + collision step of the 32-cell tube after 4 oracle steps: the
    increment f_out - f* against dt Q of the oracle, per cell, up to the FP32 rounding of the
    stored state."""
    w = I.config_shock_tube(ncell=(32, 1, 1), n=N, L=L)
    sol = oracle.Solver((32, 1, 1), (0, 0, 0), (1, 1, 1), (1, 0, 0), N, L, tab, KN)
    f = w.f0.astype(np.float32).astype(np.float64)
    dt = 1e-3
    for _ in range(4):
        f = sol.step(f, dt)
    f32 = f.astype(np.float32)
    ctx = make_ctx(fks, 32, 1, bc=(1, 0, 0))   # the tube's specular walls in x
    ctx.set_offsets(sol.s.copy())   # continue from the oracle's offsets
    fd = torch.from_numpy(f32).cuda()
    out = torch.empty_like(fd)
    ctx.step(fd, out, dt)
    assert ctx.check() & 1 == 0
    fsh = sol.transport(f32.astype(np.float64), dt)   # f* by the oracle's transport
    Qo = oracle.collide(fsh, tab, kn=KN)
    got = out.double().cpu().numpy()
    for c in range(32):
        err = np.linalg.norm(got[c] - fsh[c] - dt * Qo[c])
        assert err <= FP32_REL * np.linalg.norm(dt * Qo[c]) + 2.0 ** -24 * np.linalg.norm(got[c]) * 1.5, c
    assert ctx.escalation()[1][0] > 0


def test_batch_escalation(fks, oracle):
    """An FP32 batch problem with ||L|| / ||Q|| ~ 270 (two nearby Maxwellians): without the
    escalation its error is above 1e-5, with it the plain bound holds."""
    n, Lb, kn = 16, 8.0, 0.05
    f = 0.5 * (I.maxwellian(n, Lb, u=(0.2, 0.0, 0.0), T=1.0) + I.maxwellian(n, Lb, u=(-0.2, 0.1, 0.0), T=1.05))
    probs = [dict(n=n, L=Lb, kernel=0, kn=kn, f0=f[None]),
             dict(n=32, L=10.0, kernel=0, kn=kn, f0=I.maxwellian(32, 10.0, T=0.9)[None])]
    b = fks.Batch(probs, A1=4, A2=8, precision=1)
    fs = [torch.from_numpy(p["f0"]).to("cuda", torch.float32).contiguous() for p in probs]
    Qs = [torch.empty_like(x) for x in fs]
    b.collide(fs, Qs)
    assert b.escalation()[1] >= 1
    ref = []
    for p, x, Q in zip(probs, fs, Qs):
        t = oracle.tables(p["n"], p["L"], 0, 0.25, 4, 8, 0)
        Qo = oracle.collide(x.double().cpu().numpy(), t, kn=kn)
        ref.append(Qo)
        assert rel(Q.double().cpu().numpy(), Qo) < FP32_REL
    b.set_escalation(0.0)
    b.collide(fs, Qs)
    assert max(rel(Q.double().cpu().numpy(), Qo) for Q, Qo in zip(Qs, ref)) > FP32_REL


@pytest.mark.parametrize("arith,n", [(3, 32), (0, 32), (3, 16), (3, 8), (3, 24)])
def test_last_tier_alone_matches_oracle(fks, oracle, arith, n):
    """A tolerance below any bound sends every cell to the last tier: its arithmetic alone
    (double-float or FP64 over the FP32 state) against the oracle on far-from-equilibrium
    cells, where FP64 accuracy is the reference's own."""
    Ln = 8.0 if n <= 16 else 10.0
    nc = 7
    ctx = fks.Context(fks.Config(ncell=(nc, 1, 1), n=n, L=Ln, kn=0.3, A1=4, A2=8, precision=1))
    ctx.set_escalation(1e-300)
    ctx.set_escalation_arith(arith)
    f = I.two_stream((nc, 1, 1), n, Ln, seed=60 + n, noise=0.05).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    assert ctx.check() == 0
    assert ctx.escalation()[1][0] == nc
    Qo = oracle.collide(f.astype(np.float64), oracle.tables(n, Ln, 0, 0.25, 4, 8, 0), kn=0.3)
    for c in range(nc):
        # the result is stored in FP32: its rounding (6e-8 relative) is the floor
        assert rel(Q[c].double().cpu().numpy(), Qo[c]) < 2e-7, c


def test_full_size_learned_step_sampled(fks, oracle):
    """The benchmark's step at its full size and launch configuration: 32^3 cells x 32^3 velocities of the
    shock tube (left rho = 1, T = 1; right rho = 0.125, T = 0.8; specular x walls), fks_surrogate_step on
    a split-BF16 context at 1e-3 (the classification, its direct route, the split-BF16 kernel, the FP32
    and double-float tiers).  Sampled cells (the walls, the bulk on both sides, the interface) against
    f* (transport, bit-exact) plus dt Q of the oracle, up to the FP32 rounding of the stored state."""
    w = I.config_shock_tube(ncell=(1, 1, 1))        # parameters only
    w.ncell = (32, 32, 32)
    cfg = fks.Config(ncell=w.ncell, bc=w.bc, n=w.n, L=w.L, kernel=w.kernel, kn=w.kn, A1=w.A1, A2=w.A2,
                     precision=fks.FKS_BF16X3)
    ctx = fks.Context(cfg)
    states, which = I.shock_tube_states(w.n, w.L, 32)
    st = torch.from_numpy(states).float().cuda()
    f0 = st.index_select(0, torch.from_numpy(np.repeat(which, 1024)).cuda()).contiguous()
    out, work = torch.empty_like(f0), torch.empty_like(f0)
    net = fks.Net(w.n, 8, seed=4)
    dt = 1e-3
    for _ in range(24):                          # the interface spreads over a few cells
        ctx.surrogate_step(net, f0, out, work, dt, 1.0, 1.0, BF16_REL)
        f0, out = out, f0
    ct = fks.Context(fks.Config(ncell=w.ncell, bc=w.bc, n=w.n, L=w.L, kn=w.kn, A1=w.A1, A2=w.A2,
                                precision=fks.FKS_FP32))
    ct.set_offsets(ctx.offsets())                # the same particle offsets: f* of the checked step
    assert ctx.surrogate_step(net, f0, out, work, dt, 1.0, 1.0, BF16_REL) == f0.shape[0]
    assert ctx.check() & 1 == 0
    counts = ctx.escalation()[1]
    assert counts[1] > 16384                     # the bulk's exact Maxwellians reach the last tier
    fs = torch.empty_like(f0)
    ct.transport(f0, fs, dt)
    assert torch.equal(fs, work)
    # walls, bulk on both sides, the interface region (x = 14 .. 17)
    sample = [0, 5 * 1024 + 17, 14 * 1024 + 9, 15 * 1024 + 31, 16 * 1024 + 5 * 32 + 7, 17 * 1024 + 2,
              26 * 1024 + 3, 32767]
    tab = oracle.tables(32, w.L, 0, 0.25, w.A1, w.A2, 0)
    fsh = fs[sample].double().cpu().numpy()
    Qo = oracle.collide(fsh, tab, kn=w.kn, project=True)
    got = out[sample].double().cpu().numpy()
    for i in range(len(sample)):
        err = np.linalg.norm(got[i] - fsh[i] - dt * Qo[i])
        assert err <= BF16_REL * np.linalg.norm(dt * Qo[i]) + 2.0 ** -24 * np.linalg.norm(got[i]) * 1.5, sample[i]


def test_direct_route_error_behaviour(fks):
    """fks_set_escalation_direct needs a context with escalation tiers: FP64 contexts have none."""
    c64 = fks.Context(fks.Config(ncell=(2, 1, 1), n=16, L=8.0, kn=0.1, A1=4, A2=4, precision=fks.FKS_FP64))
    with pytest.raises(fks.FKSError) as e:
        c64.set_escalation_direct(True)
    assert e.value.status == 2   # FKS_ERR_UNSUPPORTED
    c32 = fks.Context(fks.Config(ncell=(2, 1, 1), n=16, L=8.0, kn=0.1, A1=4, A2=4, precision=fks.FKS_FP32))
    c32.set_escalation_direct(False)
    c32.set_escalation_direct(True)
