"""Learned surrogate on the GPU: network forward and gradients against the
FP64 oracle network (same BF16-rounded weights), training sanity, network
inputs, and the routed surrogate collision (all-routed equals the spectral
operator bit for bit; none-routed equals the oracle network + projection)."""
import numpy as np
import pytest

from oracle import net as onet
from paper_1701_01608_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1701_01608_gb300 import fks
    fks.lib()
    return fks


def oracle_params(p32):
    """FP32 master -> the values the GPU computes with: BF16 weights, FP32 biases."""
    p = p32.astype(np.float64).copy()
    off = 0
    for co, ci in onet.layer_shapes():
        p[off:off + co * ci * 27] = onet.bf16_round(p32[off:off + co * ci * 27])
        off += co * ci * 27 + co
    return p


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [8, 16])
def test_forward_matches_oracle(fks, n):
    net = fks.Net(n, 2, seed=3)
    rng = np.random.default_rng(n)
    x = rng.random((2, 2, n, n, n)).astype(np.float32)
    y = torch.empty((2, 1, n, n, n), device="cuda")
    net.forward(torch.from_numpy(x).cuda(), y)
    yo, _ = onet.forward(oracle_params(net.get_params()), x.astype(np.float64))
    assert rel(y.cpu().numpy(), yo) < 2e-5


@pytest.mark.parametrize("n", [16, 32])
def test_tensor_core_inference_matches_oracle(fks, n):
    """tcgen05 implicit-GEMM inference against the FP64 oracle network with
    the same BF16 weights and BF16-rounded activations (accumulation order
    differences can move an activation by one BF16 unit)."""
    net = fks.Net(n, 2, seed=13)
    rng = np.random.default_rng(n + 1)
    x = rng.random((2, 2, n, n, n)).astype(np.float32)
    y = torch.empty((2, 1, n, n, n), device="cuda")
    net.infer(torch.from_numpy(x).cuda(), y)
    net.check()
    yo, _ = onet.forward(oracle_params(net.get_params()), x.astype(np.float64), act_bf16=True)
    assert rel(y.cpu().numpy(), yo) < 2e-3
    # and close to the FP32-activation path
    y32 = torch.empty_like(y)
    net.forward(torch.from_numpy(x).cuda(), y32)
    assert rel(y.cpu().numpy(), y32.cpu().numpy()) < 2e-2


def test_gradient_matches_oracle(fks):
    n = 16
    net = fks.Net(n, 2, seed=5)
    rng = np.random.default_rng(1)
    x = rng.random((2, 2, n, n, n)).astype(np.float32)
    gy = rng.standard_normal((2, 1, n, n, n)).astype(np.float32)
    grad = torch.empty(net.num_params, device="cuda")
    net.gradient(torch.from_numpy(x).cuda(), torch.from_numpy(gy).cuda(), grad)
    po = oracle_params(net.get_params())
    _, acts = onet.forward(po, x.astype(np.float64))
    go = onet.backward(po, acts, gy.astype(np.float64))
    g = grad.cpu().numpy()
    off = 0
    for co, ci in onet.layer_shapes():
        for size in (co * ci * 27, co):
            assert rel(g[off:off + size], go[off:off + size]) < 1e-4, (co, ci, size)
            off += size


def test_training_reduces_loss(fks):
    n = 8
    net = fks.Net(n, 4, seed=7)
    rng = np.random.default_rng(2)
    xh = rng.random((4, 2, n, n, n)).astype(np.float32)
    x = torch.from_numpy(xh).cuda()
    # a target the network can represent: a relaxation-like difference of its inputs
    t = torch.from_numpy(0.5 * (xh[:, 1:2] - xh[:, 0:1])).cuda()
    losses = []
    for _ in range(60):
        loss = torch.zeros(1, device="cuda")
        net.train_step(x, t, 3e-3, loss)
        losses.append(loss.item())
    assert np.mean(losses[-10:]) < 0.6 * np.mean(losses[:10])


def test_network_inputs(fks, oracle):
    n, L = 16, 8.0
    f = I.two_stream((3, 1, 1), n, L, seed=4, noise=0.05).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    x = torch.empty((3, 2, n, n, n), device="cuda")
    rho = torch.empty(3, dtype=torch.float64, device="cuda")
    dist = torch.empty(3, device="cuda")
    fks.surrogate_inputs(n, L, fd, x, rho, dist)
    U = oracle.moments(f.astype(np.float64), n, L)
    for c in range(3):
        r = U[c, 0]
        u = U[c, 1:4] / r
        T = (U[c, 4] - 0.5 * r * u @ u) / (1.5 * r)
        M = I.maxwellian(n, L, 1.0, u, T)
        g = f[c] / r
        # the moments behind rho are FP32 partial sums (added in FP64)
        assert abs(rho[c].item() - r) < 1e-6 * r
        np.testing.assert_allclose(x[c, 0].cpu().numpy(), g, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(x[c, 1].cpu().numpy(), M, rtol=1e-5, atol=1e-9 * M.max())
        assert abs(dist[c].item() - np.linalg.norm(g - M) / np.linalg.norm(M)) < 1e-5


def test_routed_surrogate_collide(fks, oracle):
    # the routing path infers in chunks of 304 cells: 611 cells make two full
    # chunks and a ragged last one of 3
    n, L, kn = 16, 8.0, 0.3
    nc = 2 * 304 + 3
    ctx = fks.Context(fks.Config(ncell=(nc, 1, 1), n=n, L=L, kn=kn, A1=4, A2=4, precision=fks.FKS_FP32))
    net = fks.Net(n, 2, seed=11)
    f = I.two_stream((nc, 1, 1), n, L, seed=6, noise=0.05).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    Qs = torch.empty_like(fd)
    ctx.collide(fd, Qs)
    Q = torch.empty_like(fd)
    assert ctx.surrogate_collide(net, fd, Q, 1.0, 1.0, -1.0) == nc         # every cell routed
    assert torch.equal(Q, Qs)
    assert ctx.surrogate_collide(net, fd, Q, 2.5, 1.0, 1e30) == 0          # none routed
    ind = ctx.indicator()
    assert np.all(np.isfinite(ind)) and np.all(ind > 0)
    # every cell: the projected output conserves mass, momentum and energy
    Qh = Q.cpu().numpy()
    Um = oracle.moments(Qh.astype(np.float64), n, L)
    Ua = oracle.moments(np.abs(Qh).astype(np.float64), n, L)
    assert np.all(np.abs(Um[:, 0]) < 1e-5 * Ua[:, 0])
    # cells at the chunk boundaries and in the ragged tail against the oracle:
    # network on the same inputs, rho^2 y scale / Kn, projection
    cells = [0, 1, 303, 304, 607, 608, 609, 610]
    po = oracle_params(net.get_params())
    U = oracle.moments(f[cells].astype(np.float64), n, L)
    xs = []
    for i, c in enumerate(cells):
        r = U[i, 0]
        u = U[i, 1:4] / r
        T = (U[i, 4] - 0.5 * r * u @ u) / (1.5 * r)
        xs.append(np.stack([f[c] / r, I.maxwellian(n, L, 1.0, u, T)]))
    # the routing path infers on the tensor cores (BF16 activations)
    yo, _ = onet.forward(po, np.stack(xs), act_bf16=True)
    Qo = np.stack([(U[i, 0] ** 2) * yo[i, 0] * 2.5 / kn for i in range(len(cells))])
    Qo = oracle.project(Qo, n, L)
    assert rel(Qh[cells], Qo) < 2e-3


def test_train_calibrate_route(fks):
    """Train a small surrogate on spectral (f, Q) pairs, calibrate its indicator
    on held-out cells, and check the routing contract: with a threshold, every
    cell is either exact (routed to the spectral operator) or has a calibrated
    indicator below the threshold."""
    from paper_1701_01608_gb300 import surrogate as S
    n, L = 16, 8.0
    f = torch.cat([S.two_stream_cells(torch, 48, n=n, L=L, seed=3)])
    Q = S.labels(torch, f, n=n, L=L, kn=1.0)
    sur = S.train(torch, f, Q, epochs=6, batch=8, lr=2e-3, n=n, L=L, holdout=0.25)
    assert sur.train_loss[-1] < sur.train_loss[0]
    assert sur.calib["covered"] >= 0.9
    ctx = fks.Context(fks.Config(ncell=(f.shape[0], 1, 1), n=n, L=L, kn=1.0, A1=4, A2=8, precision=fks.FKS_FP32))
    out = torch.empty_like(f)
    thr = float(np.median(sur.ind_scale * ctx_indicators(fks, ctx, sur, f)))
    routed = ctx.surrogate_collide(sur.net, f, out, sur.out_scale, sur.ind_scale, thr)
    ind = ctx.indicator()
    assert 0 < routed < f.shape[0]
    Qh, oh = Q.cpu().numpy(), out.cpu().numpy()
    for c in range(f.shape[0]):
        if not ind[c] <= thr:
            assert np.array_equal(oh[c], Qh[c])      # routed: the spectral result itself


def ctx_indicators(fks, ctx, sur, f):
    tmp = torch.empty_like(f)
    ctx.surrogate_collide(sur.net, f, tmp, sur.out_scale, 1.0, 1e30)
    return ctx.indicator()


def test_routed_surrogate_collide_to_tensor_cores(fks):
    """The learned + split-BF16 path: routed cells are recomputed by the
    tensor-core operator, the others keep the surrogate's output."""
    n, L, kn, nc = 16, 8.0, 0.3, 40
    ctx = fks.Context(fks.Config(ncell=(nc, 1, 1), n=n, L=L, kn=kn, A1=4, A2=4, precision=fks.FKS_BF16X3))
    net = fks.Net(n, 2, seed=11)
    fd = torch.from_numpy(I.two_stream((nc, 1, 1), n, L, seed=6, noise=0.05).astype(np.float32)).cuda()
    Qs = torch.empty_like(fd)
    ctx.collide(fd, Qs)
    Q = torch.empty_like(fd)
    assert ctx.surrogate_collide(net, fd, Q, 1.0, 1.0, -1.0) == nc    # every cell routed
    assert torch.equal(Q, Qs)
    Qn = torch.empty_like(fd)
    assert ctx.surrogate_collide(net, fd, Qn, 2.5, 1.0, 1e30) == 0    # none routed
    ind = ctx.indicator()
    thr = float(np.median(ind))
    Qm = torch.empty_like(fd)
    routed = ctx.surrogate_collide(net, fd, Qm, 2.5, 1.0, thr)
    assert 0 < routed < nc
    for c in range(nc):
        want = Qs[c] if not ind[c] <= thr else Qn[c]
        assert torch.equal(Qm[c], want), c


def test_surrogate_step_routes_like_the_spectral_step(fks):
    """fks_surrogate_step: with every cell routed it is the spectral step itself (transport into
    work, then f* + dt Q over the routed list), bit for bit against fks_step; with none routed every
    cell gets f* + dt Q of the network."""
    n, L, kn = 16, 8.0, 0.3
    ncell = (5, 3, 2)
    cfg = fks.Config(ncell=ncell, bc=(1, 0, 0), n=n, L=L, kn=kn, A1=4, A2=4, precision=fks.FKS_FP32)
    ca, cb = fks.Context(cfg), fks.Context(cfg)
    net = fks.Net(n, 2, seed=11)
    f = torch.from_numpy(I.two_stream(ncell, n, L, seed=8, noise=0.05).astype(np.float32)).cuda()
    ref, out, work = torch.empty_like(f), torch.empty_like(f), torch.empty_like(f)
    dt = 0.01
    ca.step(f, ref, dt)
    assert cb.surrogate_step(net, f, out, work, dt, 1.0, 1.0, -1.0) == f.shape[0]
    assert torch.equal(out, ref)
    # none routed: f* + dt Q_net, Q_net as fks_surrogate_collide gives it on f*
    cc = fks.Context(cfg)
    out2, work2 = torch.empty_like(f), torch.empty_like(f)
    assert cc.surrogate_step(net, f, out2, work2, dt, 2.5, 1.0, 1e30) == 0
    assert torch.equal(work2, work)      # the same transport (offsets from zero in both contexts)
    qn = torch.empty_like(f)
    fks.Context(cfg).surrogate_collide(net, work2, qn, 2.5, 1.0, 1e30)
    assert torch.allclose(out2, work2 + dt * qn, rtol=1e-6, atol=1e-7)


def test_trained_surrogate_gain_at_its_certified_tolerance(fks, oracle):
    """What the trained network gains over the method without it.  A network trained on the
    workload's velocity grid (two-stream and shock-tube-like mixtures) is calibrated on held-out
    cells; at a tolerance it can certify, the certified cells are within that tolerance of the
    oracle, the routed ones are the spectral result, and the learned path on the certified cells
    is faster than the FP64 spectral operator on the same cells.  At 1e-3 the calibrated indicator
    certifies none of them (the network's error is >= 1e-2 of ||Q|| at best)."""
    from paper_1701_01608_gb300 import surrogate as S
    n, L = 32, 10.0
    f = S.two_stream_cells(torch, 384, n=n, L=L, seed=21)
    Q = S.labels(torch, f, n=n, L=L, kn=1.0)
    sur = S.train(torch, f, Q, batch=8, lr=2e-3, n=n, L=L, holdout=0.25, steps=1200)
    assert sur.calib["covered"] >= 0.95
    held = S.two_stream_cells(torch, 96, n=n, L=L, seed=22)
    Qh = S.labels(torch, held, n=n, L=L, kn=1.0)
    tol = 0.3
    ctx = fks.Context(fks.Config(ncell=(96, 1, 1), n=n, L=L, kn=1.0, A1=4, A2=8, precision=fks.FKS_FP32))
    out = torch.empty_like(held)
    routed = ctx.surrogate_collide(sur.net, held, out, sur.out_scale, sur.ind_scale, tol)
    ind = ctx.indicator()
    cert = [c for c in range(96) if ind[c] <= tol]
    assert len(cert) > 0 and routed == 96 - len(cert)
    err = ((out - Qh).double().flatten(1).norm(dim=1) / Qh.double().flatten(1).norm(dim=1)).cpu().numpy()
    for c in range(96):
        if c in cert:
            assert err[c] <= tol, (c, err[c])
        else:
            assert err[c] < 1e-5          # routed: the (escalated) FP32 spectral operator
    # two certified cells against the oracle itself
    tab = oracle.tables(n, L, 0, 0.25, 4, 8, 0)
    for c in cert[:2]:
        Qo = oracle.collide(held[c:c + 1].double().cpu().numpy(), tab, kn=1.0)[0]
        assert rel(out[c].double().cpu().numpy(), Qo) <= tol
    # time: the learned path on the certified cells against the FP64 spectral operator on them
    fc = held[torch.tensor(cert, device="cuda")].contiguous()
    k = fc.shape[0]
    cl = fks.Context(fks.Config(ncell=(k, 1, 1), n=n, L=L, kn=1.0, A1=4, A2=8, precision=fks.FKS_FP32))
    c64 = fks.Context(fks.Config(ncell=(k, 1, 1), n=n, L=L, kn=1.0, A1=4, A2=8, precision=fks.FKS_FP64))
    ql, q64, f64 = torch.empty_like(fc), torch.empty(fc.shape, dtype=torch.float64, device="cuda"), fc.double()

    def best(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    t_learn = best(lambda: cl.surrogate_collide(sur.net, fc, ql, sur.out_scale, sur.ind_scale, tol))
    t_fp64 = best(lambda: c64.collide(f64, q64))
    assert t_learn < t_fp64, (t_learn, t_fp64)
    # the stated tolerance of the learned path is out of this network's reach
    assert ctx.surrogate_collide(sur.net, held, out, sur.out_scale, sur.ind_scale, 1e-3) == 96
