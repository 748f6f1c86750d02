"""Uneven batches of homogeneous problems (n in {8, 16, 24, 32}, hard-sphere
and pseudo-Maxwell kernels, per-problem Knudsen numbers) against the oracle;
graph replay against step-by-step launches; the autotuner."""
import numpy as np
import pytest

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problems(seed=3, count=10):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    ns = [8, 16, 24, 32, 16, 24, 8, 32, 16, 24][:count]
    for i, n in enumerate(ns):
        L = 8.0 if n <= 16 else 10.0
        u1, u2 = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
        T1, T2 = rng.uniform(0.8, 1.2, 2)
        f = 0.5 * (I.maxwellian(n, L, u=u1, T=T1) + I.maxwellian(n, L, u=u2, T=T2))
        out.append(dict(n=n, L=L, kernel=i % 2, C=0.25, kn=float(10 ** rng.uniform(-3, 0)), f0=f))
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_batch_collide_and_step_match_oracle(fks, oracle, prec, tol):
    probs = problems()
    b = fks.Batch(probs, A1=4, A2=8, precision=prec)
    fs = [torch.from_numpy(p["f0"]).to("cuda", b.dtype).contiguous() for p in probs]
    Qs = [torch.empty_like(f) for f in fs]
    outs = [torch.empty_like(f) for f in fs]
    b.collide(fs, Qs)
    dts = [0.2 * p["kn"] for p in probs]
    b.step(fs, outs, dts)
    assert b.check() & 1 == 0
    for p, f, Q, o, dt in zip(probs, fs, Qs, outs, dts):
        fin = f.double().cpu().numpy()
        t = oracle.tables(p["n"], p["L"], p["kernel"], 0.25, 4, 8, 0)
        Qo = oracle.collide(fin, t, kn=p["kn"])
        assert rel(Q.double().cpu().numpy(), Qo) < tol, (p["n"], p["kernel"])
        want = fin + dt * Qo
        assert np.linalg.norm(o.double().cpu().numpy() - want) / np.linalg.norm(dt * Qo) < 10 * tol + 1e-6


def test_graph_run_equals_step_by_step(fks):
    probs = problems(seed=5, count=8)
    b = fks.Batch(probs, A1=4, A2=8, precision=1)
    fa = [torch.from_numpy(p["f0"]).to("cuda", torch.float32).contiguous() for p in probs]
    fb = [torch.empty_like(f) for f in fa]
    ga = [f.clone() for f in fa]
    gb = [torch.empty_like(f) for f in fa]
    dts = [0.1 * p["kn"] for p in probs]
    for k in range(5):
        if k % 2 == 0:
            b.step(fa, fb, dts)
        else:
            b.step(fb, fa, dts)
    launches = b.launches
    b.run(ga, gb, dts, 5)
    torch.cuda.synchronize()
    for x, y in zip(fb, gb):   # 5 steps: result in the second buffer
        assert torch.equal(x, y)
    assert b.launches > launches   # the graph was captured from real launches


def test_autotune_keeps_parity(fks, oracle, tmp_path):
    from paper_1701_01608_gb300 import autotune
    probs = problems(seed=7, count=6)
    b = fks.Batch(probs, A1=4, A2=8, precision=1)
    fs = [torch.from_numpy(p["f0"]).to("cuda", torch.float32).contiguous() for p in probs]
    Qs = [torch.empty_like(f) for f in fs]
    chosen = autotune.tune_batch(b, fs, Qs, precision=1, reps=2, cache=str(tmp_path / "tune.json"))
    for n, (C, r) in chosen.items():
        assert (C, r) in autotune.CANDIDATES[(1, n)]
        assert b.cluster_size(n) == C and b.radix(n) == r
    b.collide(fs, Qs)
    for p, f, Q in zip(probs, fs, Qs):
        t = oracle.tables(p["n"], p["L"], p["kernel"], 0.25, 4, 8, 0)
        fin = f.double().cpu().numpy()
        Qo = oracle.collide(fin, t, kn=p["kn"])
        assert rel(Q.double().cpu().numpy(), Qo) < 1e-5
    # a second call reads the cache
    assert autotune.tune_batch(b, fs, Qs, precision=1, cache=str(tmp_path / "tune.json")) == chosen


def test_every_cluster_size_of_a_class(fks, oracle):
    probs = [dict(n=32, L=10.0, kernel=0, kn=0.5, f0=problems(count=4)[3]["f0"])]
    b = fks.Batch(probs, A1=4, A2=8, precision=1)
    f = torch.from_numpy(probs[0]["f0"]).to("cuda", torch.float32).contiguous()
    Qo = oracle.collide(f.double().cpu().numpy(), oracle.tables(32, 10.0, 0, 0.25, 4, 8, 0), kn=0.5)
    for C in (8, 4):
        b.set_cluster_size(32, C)
        Q = torch.empty_like(f)
        b.collide([f], [Q])
        assert rel(Q.double().cpu().numpy(), Qo) < 1e-5


@pytest.mark.parametrize("n", [16, 24, 32])
def test_every_radix_schedule_matches_oracle(fks, oracle, n):
    """Every compiled (cluster size, radix schedule) of an FP32 context: the same operator (relative
    L2 of Q <= 1e-5 per cell against the oracle)."""
    from paper_1701_01608_gb300 import autotune
    L = 8.0 if n == 16 else 10.0
    nc = 5
    ctx = fks.Context(fks.Config(ncell=(nc, 1, 1), n=n, L=L, kn=0.4, A1=4, A2=8, precision=1))
    f = I.two_stream((nc, 1, 1), n, L, seed=70 + n, noise=0.05).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    Qo = oracle.collide(f.astype(np.float64), oracle.tables(n, L, 0, 0.25, 4, 8, 0), kn=0.4)
    for C, r in autotune.CANDIDATES[(1, n)]:
        ctx.set_schedule(C, r)
        assert ctx.cluster_size == C and ctx.radix == r
        Q = torch.empty_like(fd)
        ctx.collide(fd, Q)
        assert ctx.check() == 0
        Qg = Q.double().cpu().numpy()
        for c in range(nc):
            assert rel(Qg[c], Qo[c]) < 1e-5, (C, r, c)
