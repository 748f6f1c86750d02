"""Oracle surrogate network: backward pinned by central finite differences,
convolution pinned by a direct 27-point sum at sampled voxels."""
import numpy as np

from oracle import net

SMALL = (2, 3, 4, 1)


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, 5, 5, 5))
    W = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    out = net.conv(x, W, b)
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    for (o, i, j, k) in [(0, 0, 0, 0), (2, 4, 1, 3), (1, 2, 2, 2), (0, 4, 4, 4)]:
        s = b[o]
        for t, (dx, dy, dz) in enumerate(net.TAPS):
            s += sum(W[o, c, t] * xp[0, c, i + 1 + dx, j + 1 + dy, k + 1 + dz] for c in range(2))
        assert abs(out[0, o, i, j, k] - s) < 1e-12


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = net.num_params(SMALL)
    params = 0.3 * rng.standard_normal(P)
    x = rng.standard_normal((2, 2, 4, 4, 4))
    gout = rng.standard_normal((2, 1, 4, 4, 4))
    y, acts = net.forward(params, x, SMALL)
    g = net.backward(params, acts, gout, SMALL)
    idx = rng.choice(P, size=40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(P)
        e[i] = h
        fp = (net.forward(params + e, x, SMALL)[0] * gout).sum()
        fm = (net.forward(params - e, x, SMALL)[0] * gout).sum()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.001953125, -3.14159, 1e-3])
    r = net.bf16_round(vals)
    # bf16 keeps 8 significant bits: rounding error <= half a unit, 2^-8 relative
    assert np.all(np.abs(r - vals) <= 2.0 ** -8 * np.abs(vals))
    assert r[0] == 1.0
    assert r[1] == 1.0            # 1 + 2^-8 is a tie: to even
    assert r[2] == 1.0            # below the tie
