"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element on the same seeded inputs (FP64 <= 1e-10, FP32 <= 1e-5 relative L2
of Q; transport bit-exact; moments 1e-12)."""
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


TOL = {0: 1e-10, 1: 1e-5}   # fks.FKS_FP64, fks.FKS_FP32


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make_ctx(fks, ncell, n, L, kernel=0, kn=1.0, A=(4, 4), prec=0, bc=(0, 0, 0), rule=0, C=0.25):
    cfg = fks.Config(ncell=tuple(ncell), bc=tuple(bc), n=n, L=L, kernel=kernel, C=C, kn=kn,
                     A1=A[0], A2=A[1], rule=rule, precision=prec)
    return fks.Context(cfg)


def to_dev(f, ctx):
    return torch.from_numpy(np.ascontiguousarray(f)).to(device="cuda", dtype=ctx.dtype).contiguous()


def host64(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("n,prec,kernel,L,A,ncell", [
    (8, 0, 0, 6.0, (4, 4), (5, 1, 1)),
    (16, 0, 0, 8.0, (4, 4), (3, 2, 1)),
    (16, 0, 1, 8.0, (4, 4), (3, 1, 1)),
    (24, 0, 0, 10.0, (4, 8), (3, 1, 1)),
    (32, 0, 0, 10.0, (4, 8), (2, 1, 1)),
    (8, 1, 0, 6.0, (4, 4), (7, 1, 1)),
    (16, 1, 0, 8.0, (4, 4), (9, 1, 1)),
    (16, 1, 1, 8.0, (4, 4), (5, 1, 1)),
    (24, 1, 0, 10.0, (4, 8), (5, 1, 1)),
    (32, 1, 0, 10.0, (4, 8), (5, 1, 1)),
    (32, 1, 1, 10.0, (4, 8), (3, 1, 1)),
])
def test_collide_matches_oracle(fks, oracle, n, prec, kernel, L, A, ncell):
    ctx = make_ctx(fks, ncell, n, L, kernel=kernel, kn=0.3, A=A, prec=prec)
    nc = int(np.prod(ncell))
    f = I.two_stream((nc, 1, 1), n, L, seed=11 + n, noise=0.05)
    fd = to_dev(f, ctx)
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    assert ctx.check() == 0
    fin = host64(fd)   # the oracle sees exactly the values the GPU saw
    tab = oracle.tables(n, L, kernel, 0.25, A[0], A[1], 0)
    Qo = oracle.collide(fin, tab, kn=0.3, project=True)
    Qg = host64(Q)
    for c in range(nc):
        assert rel(Qg[c], Qo[c]) < TOL[prec], (c, rel(Qg[c], Qo[c]))


@pytest.mark.parametrize("prec,C", [(1, 16), (1, 8), (1, 2), (0, 4), (1, 4)])
def test_cluster_size_variants(fks, oracle, prec, C):
    n = {(1, 16): 32, (1, 8): 32, (1, 2): 16, (0, 4): 16, (1, 4): 24}[(prec, C)]
    L, A = 10.0, (4, 4)
    ctx = make_ctx(fks, (3, 1, 1), n, L, A=A, prec=prec)
    ctx.set_cluster_size(C)
    assert ctx.cluster_size == C
    f = I.two_stream((3, 1, 1), n, L, seed=3, noise=0.05)
    fd = to_dev(f, ctx)
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    Qo = oracle.collide(host64(fd), oracle.tables(n, L, 0, 0.25, *A, 0), kn=1.0)
    assert rel(host64(Q), Qo) < TOL[prec]


def test_projection_conserves_in_fp64(fks):
    n, L = 16, 8.0
    ctx = make_ctx(fks, (4, 1, 1), n, L, prec=0)
    f = I.two_stream((4, 1, 1), n, L, seed=5, noise=0.1)
    fd = to_dev(f, ctx)
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    Qh = host64(Q)
    v = I.velocity_points(n, L)
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    phi = np.stack([np.ones_like(vx), vx, vy, vz, 0.5 * (vx ** 2 + vy ** 2 + vz ** 2)]).reshape(5, -1)
    for c in range(4):
        m = phi @ Qh[c].ravel()
        scale = np.abs(phi) @ np.abs(Qh[c].ravel())
        assert np.all(np.abs(m) <= 1e-12 * scale)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 0), (1, 1, 1)])
def test_transport_bit_exact(fks, oracle, prec, bc):
    ncell, n, L = (5, 3, 4), 8, 4.0
    ctx = make_ctx(fks, ncell, n, L, prec=prec, bc=bc)
    rng = np.random.default_rng(7)
    f = rng.random((int(np.prod(ncell)), n, n, n))
    fd = to_dev(f, ctx)
    f = host64(fd)
    dx = [1.0 / c for c in ncell]
    s = np.zeros((3, n))
    out = torch.empty_like(fd)
    for step, dt in enumerate([0.37 * min(dx) / L, 0.9 * min(dx) / L, -0.61 * min(dx) / L, 0.2 / L]):
        ctx.transport(fd, out, dt)
        s, delta = oracle.offsets(n, L, dx, dt, s)
        f = oracle.transport(f, ncell, bc, delta)
        np.testing.assert_array_equal(host64(out), f)
        np.testing.assert_array_equal(ctx.offsets(), s)
        fd, out = out, fd


def test_moments_match_oracle(fks, oracle):
    n, L = 16, 8.0
    ctx = make_ctx(fks, (6, 1, 1), n, L, prec=0)
    f = I.two_stream((6, 1, 1), n, L, seed=2, noise=0.2)
    fd = to_dev(f, ctx)
    U = torch.empty((6, 5), dtype=torch.float64, device="cuda")
    ctx.moments(fd, U)
    Uo = oracle.moments(f, n, L)
    np.testing.assert_allclose(U.cpu().numpy(), Uo, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("prec", [0, 1])
def test_steps_small_periodic_workload(fks, oracle, prec):
    """4^3 periodic cells, 16^3 velocities, M = 16, Kn = 0.1, 10 steps."""
    w = I.config_small_periodic()
    ctx = make_ctx(fks, w.ncell, w.n, w.L, kernel=w.kernel, kn=w.kn, A=(w.A1, w.A2), prec=prec)
    tab = oracle.tables(w.n, w.L, w.kernel, w.C, w.A1, w.A2, 0)
    sol = oracle.Solver(w.ncell, w.x0, w.x1, w.bc, w.n, w.L, tab, w.kn)
    fd = to_dev(w.f0, ctx)
    f = host64(fd)
    out = torch.empty_like(fd)
    dt = 0.25 * 0.25 / 8.0   # dx / max|v|, halved twice
    for _ in range(w.steps):
        ctx.step(fd, out, dt)
        fd, out = out, fd
        f = sol.step(f, dt)
    assert ctx.check() & 1 == 0
    tol = 1e-10 if prec == 0 else 2e-5
    assert rel(host64(fd), f) < tol


def test_step_ragged_specular(fks, oracle):
    ncell, n, L = (3, 5, 2), 8, 5.0
    bc = (1, 1, 0)
    ctx = make_ctx(fks, ncell, n, L, prec=0, bc=bc, kn=0.5)
    tab = oracle.tables(n, L, 0, 0.25, 4, 4, 0)
    sol = oracle.Solver(ncell, (0, 0, 0), (1, 1, 1), bc, n, L, tab, 0.5)
    f = I.two_stream(ncell, n, L, seed=9, noise=0.1)
    fd = to_dev(f, ctx)
    out = torch.empty_like(fd)
    dt = 0.7 * 0.2 / L
    for _ in range(3):
        ctx.step(fd, out, dt)
        fd, out = out, fd
        f = sol.step(f, dt)
    assert rel(host64(fd), f) < 1e-10


def test_single_homogeneous_cell(fks, oracle):
    ctx = make_ctx(fks, (1, 1, 1), 8, 6.0, prec=0)
    f = I.two_stream((1, 1, 1), 8, 6.0, seed=1)
    fd = to_dev(f, ctx)
    out = torch.empty_like(fd)
    ctx.step(fd, out, 0.01)
    Qo = oracle.collide(f, oracle.tables(8, 6.0, 0, 0.25, 4, 4, 0), kn=1.0)
    assert rel(host64(out), f + 0.01 * Qo) < 1e-12


def test_invalid_arguments_rejected(fks):
    with pytest.raises(fks.FKSError) as e:
        make_ctx(fks, (0, 1, 1), 8, 6.0)
    assert e.value.status == 1
    with pytest.raises(fks.FKSError) as e:
        make_ctx(fks, (1, 1, 1), 12, 6.0)
    assert e.value.status == 2
    ctx = make_ctx(fks, (2, 1, 1), 8, 6.0, prec=0)
    fd = torch.zeros((2, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(fks.FKSError) as e:
        ctx.collide(fd, fd)
    assert e.value.status == 1
    with pytest.raises(TypeError):
        ctx.collide(fd.float(), fd.float())


def test_nan_input_is_flagged(fks):
    ctx = make_ctx(fks, (2, 1, 1), 8, 6.0, prec=1)
    f = torch.ones((2, 8, 8, 8), dtype=torch.float32, device="cuda")
    f[1, 3, 3, 3] = float("nan")
    Q = torch.empty_like(f)
    ctx.collide(f, Q)
    with pytest.raises(fks.FKSError) as e:
        ctx.check()
    assert e.value.status == 5
    assert ctx.check() == 0   # bits were cleared


def test_full_size_shock_tube_step_sampled(fks, oracle):
    """32^3 cells x 32^3 velocities FP32, M = 32, specular x walls: the step
    the benchmark times, checked on sampled cells against transport (GPU,
    bit-exact) followed by the oracle's projected operator and Euler step."""
    w = I.config_shock_tube(ncell=(1, 1, 1))        # parameters only (one cell of data)
    w.ncell = (32, 32, 32)
    ctx = make_ctx(fks, w.ncell, w.n, w.L, kernel=w.kernel, kn=w.kn, A=(w.A1, w.A2), prec=1, bc=w.bc)
    ctx2 = make_ctx(fks, w.ncell, w.n, w.L, kernel=w.kernel, kn=w.kn, A=(w.A1, w.A2), prec=1, bc=w.bc)
    states, which = I.shock_tube_states(w.n, w.L, 32)
    st = torch.from_numpy(states).float().cuda()
    f0 = st.index_select(0, torch.from_numpy(np.repeat(which, 1024)).cuda()).contiguous()
    g = torch.Generator(device="cuda").manual_seed(2)
    f0 *= 1.0 + 0.05 * (2.0 * torch.rand(f0.shape, generator=g, device="cuda", dtype=torch.float32) - 1.0)
    f1 = torch.empty_like(f0)
    dt = 1e-3   # explicit-Euler stable for Kn = 0.01 (dt nu / Kn ~ 0.5)
    ctx.step(f0, f1, dt)
    fs = torch.empty_like(f0)
    ctx2.transport(f0, fs, dt)
    assert ctx.check() & 1 == 0
    # transport is a permutation of each velocity's values over the cells
    tot0 = f0.double().sum(dim=0)
    tot1 = fs.double().sum(dim=0)
    assert torch.allclose(tot0.sum(), tot1.sum(), rtol=1e-12)
    sample = [0, 31 * 1024, 16 * 1024 + 5 * 32 + 7, 1023, 15 * 1024 + 31, 32767]
    tab = oracle.tables(32, w.L, 0, 0.25, 4, 8, 0)
    fsh = fs[sample].double().cpu().numpy()
    Qo = oracle.collide(fsh, tab, kn=w.kn, project=True)
    got = f1[sample].double().cpu().numpy()
    want = fsh + dt * Qo
    for i in range(len(sample)):
        # FP32 state: the collision increment must match to the FP32 tolerance
        inc_err = np.linalg.norm(got[i] - want[i]) / np.linalg.norm(dt * Qo[i])
        assert inc_err < 1e-4, (sample[i], inc_err)
    Q = torch.empty((len(sample), 32, 32, 32), dtype=torch.float32, device="cuda")
    ctx3 = make_ctx(fks, (len(sample), 1, 1), 32, w.L, kn=w.kn, A=(4, 8), prec=1)
    ctx3.collide(fs[sample].contiguous(), Q)
    for i in range(len(sample)):
        assert rel(Q[i].double().cpu().numpy(), Qo[i]) < 1e-5


def test_bounded_wait_times_out_and_device_stays_usable(fks, oracle):
    """Failure detection without a GPU fault: a wait that nothing completes runs
    out after its poll limit, the status says so, and the next work is correct."""
    assert fks.selftest_wait(4096) == 6          # FKS_ERR_TIMEOUT
    assert fks.selftest_wait(0) == 1             # FKS_ERR_INVALID_ARG
    ctx = make_ctx(fks, (2, 1, 1), 8, 6.0, prec=0)
    f = I.two_stream((2, 1, 1), 8, 6.0, seed=5)
    fd = to_dev(f, ctx)
    Q = torch.empty_like(fd)
    ctx.collide(fd, Q)
    assert ctx.check() == 0
    Qo = oracle.collide(f, oracle.tables(8, 6.0, 0, 0.25, 4, 4, 0), kn=1.0)
    assert rel(host64(Q), Qo) < 1e-10


@pytest.mark.parametrize("prec", [1, 2])
def test_checkpoint_resume_is_bitwise(fks, prec):
    """Checkpoint after 3 steps (f and the sub-cell offsets), resume in a new
    context: 3 more steps reproduce the uninterrupted run bit for bit."""
    w = I.config_small_periodic()
    mk = lambda: make_ctx(fks, w.ncell, w.n, w.L, kernel=w.kernel, kn=w.kn, A=(w.A1, w.A2), prec=prec)
    dt = 0.25 * 0.25 / 8.0
    a = mk()
    fa = to_dev(w.f0, a)
    fb = torch.empty_like(fa)
    for i in range(6):
        a.step(fa, fb, dt)
        fa, fb = fb, fa
        if i == 2:
            saved_f = fa.clone().cpu()
            saved_s = a.offsets()
    b = mk()
    b.set_offsets(saved_s)
    ga = saved_f.cuda()
    gb = torch.empty_like(ga)
    for _ in range(3):
        b.step(ga, gb, dt)
        ga, gb = gb, ga
    assert torch.equal(ga, fa)


@pytest.mark.parametrize("prec,kernel,n,bc,ncell,dt_scale,pinned", [
    (1, 0, 8, (1, 0, 0), (16, 2, 3), 1.0, True),     # FP32 cluster kernel, specular x: 8 chunks of 2 slabs
    (0, 0, 8, (0, 0, 0), (12, 2, 2), 3.0, True),     # FP64 periodic, shifts reach 4 slabs
    (1, 2, 8, (1, 1, 0), (9, 3, 2), 1.0, True),      # BGK, ragged chunks
    (2, 0, 16, (0, 0, 0), (4, 2, 2), 1.0, True),     # split BF16: one chunk
    (1, 0, 8, (0, 0, 0), (8, 2, 2), 1.0, False),     # pageable host memory
])
def test_step_host_equals_device_step(fks, prec, kernel, n, bc, ncell, dt_scale, pinned):
    """fks_step_host (copies pipelined over x-slab chunks) gives the values of
    fks_step on device copies, bit for bit, over two steps."""
    L = 6.0 if n == 8 else 8.0
    cfg = dict(ncell=ncell, n=n, L=L, kernel=kernel, kn=0.5, A=(4, 4), prec=prec, bc=bc)
    a, b = make_ctx(fks, **cfg), make_ctx(fks, **cfg)
    f = I.two_stream(ncell, n, L, seed=21, noise=0.05)
    fd = to_dev(f, a)
    od = torch.empty_like(fd)
    h_in = fd.cpu()
    h_in = h_in.pin_memory() if pinned else h_in.clone()
    h_out = torch.empty_like(h_in)
    if pinned:
        h_out = h_out.pin_memory()
    dt = dt_scale * (1.0 / ncell[0]) / L
    for _ in range(2):
        a.step(fd, od, dt)
        b.step_host(h_in, h_out, dt)
        torch.cuda.synchronize()
        assert torch.equal(od.cpu(), h_out)
        fd, od = od, fd
        h_in.copy_(h_out)
    assert a.check() & 1 == 0 and b.check() & 1 == 0


@pytest.mark.parametrize("n,prec", [(8, 0), (32, 1), (16, 2)])
def test_zero_distribution_collides_to_zero(fks, n, prec):
    """Q is quadratic: f = 0 gives Q = 0 exactly (transforms, products, projection)."""
    ctx = make_ctx(fks, (2, 1, 1), n, 10.0, prec=prec)
    f = torch.zeros((2, n, n, n), dtype=ctx.dtype, device="cuda")
    Q = torch.full_like(f, 7.0)
    ctx.collide(f, Q)
    assert ctx.check() == 0
    assert bool((Q == 0).all())


def test_alu_peak_measurement_is_plausible(fks):
    """fks_alu_peak: the FMA-chain throughput of the FP32 and FP64 pipes (the
    roofline's measured denominators) lies near GB300's unit counts x clock
    (80.5 and 1.26 TFLOP/s at 2.07 GHz)."""
    t32 = fks.alu_peak(fks.FKS_FP32)
    t64 = fks.alu_peak(fks.FKS_FP64)
    assert 40.0 < t32 < 90.0, t32
    assert 0.5 < t64 < 2.0, t64


@pytest.mark.parametrize("n,L", [(16, 8.0), (32, 10.0)])
def test_fp32_projection_conserves_to_output_rounding(fks, n, L):
    """FP32 output: the moments of Q, summed on the host in FP64, vanish to the rounding of the
    stored values (measured 3-6e-9 of sum |phi Q|): the compensated FP32 moment sums of the
    kernel are as good as FP64 ones."""
    ctx = make_ctx(fks, (6, 1, 1), n, L, kn=0.3, prec=1)
    f = to_dev(I.two_stream((6, 1, 1), n, L, seed=3, noise=0.05), ctx)
    Q = torch.empty_like(f)
    ctx.collide(f, Q)
    q = host64(Q).reshape(6, -1)
    v = I.velocity_points(n, L)
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    phi = np.stack([np.ones_like(vx), vx, vy, vz, 0.5 * (vx ** 2 + vy ** 2 + vz ** 2)]).reshape(5, -1)
    m = np.abs(q @ phi.T) / (np.abs(q) @ np.abs(phi.T))
    assert m.max() < 1e-7, m.max()
