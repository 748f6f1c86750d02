"""Plain FP64 reference of the collision-surrogate network (test infrastructure).

A stack of 3x3x3 convolutions over the velocity grid with zero padding:
channels (2, 32, 32, 32, 32, 32, 1), ReLU after every layer but the last.
Input channels: f / rho and M[f] / rho; output: Q Kn / rho^2 (the operator is
quadratic, Q(rho g) = rho^2 Q(g)).  Weights of layer l: W[co][ci][27] with
tap t = (dx+1)*9 + (dy+1)*3 + (dz+1), then bias[co]; all layers packed in one
flat vector in that order.  Forward and backward are written out plainly
(one shifted view per tap); the backward is pinned by finite differences in
tests/test_oracle_net.py.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 32, 32, 32, 32, 1)


def layer_shapes(channels=CHANNELS):
    return [(channels[i + 1], channels[i]) for i in range(len(channels) - 1)]


def num_params(channels=CHANNELS) -> int:
    return sum(co * ci * 27 + co for co, ci in layer_shapes(channels))


def unpack(params, channels=CHANNELS):
    out, off = [], 0
    for co, ci in layer_shapes(channels):
        W = params[off:off + co * ci * 27].reshape(co, ci, 27)
        off += co * ci * 27
        b = params[off:off + co]
        off += co
        out.append((W, b))
    return out


TAPS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]


def _shift(x, d):
    """y[..., p] = x[..., p + d] with zeros outside (x: [B, C, n, n, n])."""
    n = x.shape[-1]
    y = np.zeros_like(x)
    sl_dst, sl_src = [], []
    for k in d:
        if k >= 0:
            sl_dst.append(slice(0, n - k))
            sl_src.append(slice(k, n))
        else:
            sl_dst.append(slice(-k, n))
            sl_src.append(slice(0, n + k))
    y[(Ellipsis, *sl_dst)] = x[(Ellipsis, *sl_src)]
    return y


def conv(x, W, b):
    """out[b, o, p] = sum_{c, t} W[o, c, t] x[b, c, p + d_t] + bias[o]."""
    out = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
    for t, d in enumerate(TAPS):
        out += np.einsum("oc,bcxyz->boxyz", W[:, :, t], _shift(x, d))
    return out + b[None, :, None, None, None]


def forward(params, x, channels=CHANNELS, act_bf16=False):
    """Returns the output and the list of layer activations (inputs of each layer).
    act_bf16: round the input and every hidden activation to bfloat16 (the
    tensor-core inference path stores activations in that format)."""
    layers = unpack(params, channels)
    h = bf16_round(x) if act_bf16 else x
    acts = [h]
    for l, (W, b) in enumerate(layers):
        h = conv(h, W, b)
        if l < len(layers) - 1:
            h = np.maximum(h, 0.0)
            if act_bf16:
                h = bf16_round(h)
        acts.append(h)
    return h, acts


def backward(params, acts, gout, channels=CHANNELS):
    """Gradient of sum(gout * output) with respect to the flat parameters."""
    layers = unpack(params, channels)
    grads = []
    g = gout
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        if l < len(layers) - 1:
            g = g * (acts[l + 1] > 0)
        xin = acts[l]
        gW = np.zeros_like(W)
        for t, d in enumerate(TAPS):
            gW[:, :, t] = np.einsum("boxyz,bcxyz->oc", g, _shift(xin, d))
        gb = g.sum(axis=(0, 2, 3, 4))
        grads.append((gW, gb))
        # input gradient: transpose of the shifted sums
        gin = np.zeros_like(xin)
        for t, d in enumerate(TAPS):
            gin += _shift(np.einsum("oc,boxyz->bcxyz", W[:, :, t], g), tuple(-k for k in d))
        g = gin
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return np.concatenate(flat)


def bf16_round(a):
    """Round FP32/FP64 values to bfloat16 (round to nearest even), as float64."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)
