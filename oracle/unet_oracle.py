"""FP64 reference of the U-Net pieces that give the forward solves their
initial guess -- TEST INFRASTRUCTURE ONLY (not part of the paper's method).

Definitions written out with numpy: channels-last tensors [n^3, C] of an
n^3 grid (x fastest), 3x3x3 convolutions with zero padding, weights
[27, C_out, C_in] with tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1),
2x2x2 average pooling, nearest upsampling, channel concatenation, and the
round-to-nearest-even bf16 rounding applied where the GPU path stores bf16.
Pinned by tests/test_oracle_unet.py against scipy.ndimage.correlate, the
adjoint identities of the convolution and brute-force sums.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def to_bf16(x) -> np.ndarray:
    """Round float values to the nearest bf16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _grid(x, n):
    return np.asarray(x, dtype=np.float64).reshape(n, n, n, -1)


def _shift(xg, dz, dy, dx):
    """y[z, y, x] = xg[z + dz, y + dy, x + dx] (zero outside)."""
    n = xg.shape[0]
    p = np.pad(xg, ((1, 1), (1, 1), (1, 1), (0, 0)))
    return p[1 + dz:1 + dz + n, 1 + dy:1 + dy + n, 1 + dx:1 + dx + n, :]


def conv3d(x, w, b, n, relu=False):
    """out[v, co] = b[co] + sum_tap sum_ci x[v + off(tap), ci] w[tap, co, ci]."""
    xg = _grid(x, n)
    cout = w.shape[1]
    out = np.zeros((n, n, n, cout))
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += _shift(xg, dz, dy, dx) @ np.asarray(w[t], dtype=np.float64).T
    if b is not None:
        out += np.asarray(b, dtype=np.float64)
    if relu:
        out = np.maximum(out, 0.0)
    return out.reshape(n ** 3, cout)


def conv3d_transpose(dy, w, n):
    """Adjoint of conv3d in its input: dx[u, ci] = sum_tap sum_co dy[u - off(tap), co] w[tap, co, ci]."""
    dyg = _grid(dy, n)
    cin = w.shape[2]
    dx = np.zeros((n, n, n, cin))
    for t, (dz, dy_, dx_) in enumerate(TAPS):
        dx += _shift(dyg, -dz, -dy_, -dx_) @ np.asarray(w[t], dtype=np.float64)
    return dx.reshape(n ** 3, cin)


def conv3d_wgrad(x, dy, n):
    """dw[tap, co, ci] = sum_v dy[v, co] x[v + off(tap), ci];  db[co] = sum_v dy[v, co]."""
    xg = _grid(x, n)
    dyf = np.asarray(dy, dtype=np.float64).reshape(n ** 3, -1)
    cin = xg.shape[3]
    dw = np.stack([dyf.T @ _shift(xg, dz, dy_, dx_).reshape(n ** 3, cin) for (dz, dy_, dx_) in TAPS])
    return dw, dyf.sum(axis=0)


def avgpool(x, n):
    xg = _grid(x, n)
    m = n // 2
    out = xg.reshape(m, 2, m, 2, m, 2, -1).mean(axis=(1, 3, 5))
    return out.reshape(m ** 3, -1)


def upcat(lo, skip, n):
    """Nearest 2x upsampling of lo ((n/2)^3 grid) concatenated with skip (n^3)."""
    m = n // 2
    lg = _grid(lo, m)
    up = lg.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)
    return np.concatenate([up.reshape(n ** 3, -1), np.asarray(skip, dtype=np.float64)], axis=1)


# (c_in, c_out, level, relu) of the 15 convolutions, as in the CUDA runtime
SPEC = [(16, 16, 0, 1), (16, 16, 0, 1), (16, 32, 1, 1), (32, 32, 1, 1), (32, 64, 2, 1),
        (64, 64, 2, 1), (64, 128, 3, 1), (128, 128, 3, 1), (192, 64, 2, 1), (64, 64, 2, 1),
        (96, 32, 1, 1), (32, 32, 1, 1), (48, 16, 0, 1), (16, 16, 0, 1), (16, 16, 0, 0)]


def unpack_params(p):
    """Flat parameter vector -> list of (w [27, co, ci], b [co])."""
    out, o = [], 0
    for ci, co, _, _ in SPEC:
        nw = 27 * co * ci
        out.append((p[o:o + nw].reshape(27, co, ci), p[o + nw:o + nw + co]))
        o += nw + co
    return out


def unet_forward(params, x3, n, bf16: bool = True):
    """U-Net prediction (channel 0 of the last conv) for features x3 [n^3, 3],
    with the bf16 rounding of the GPU path: weights and every stored
    activation are rounded to bf16, accumulation is exact (float64).  With
    bf16=False nothing is rounded (the FP64 network)."""
    rnd = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    P = [(rnd(w), np.asarray(b, np.float64)) for w, b in unpack_params(params)]
    x = np.zeros((n ** 3, 16))
    x[:, :3] = x3
    x = rnd(x)
    n0, n1, n2, n3 = n, n // 2, n // 4, n // 8

    def c(i, inp, m):
        ci, co, _, relu = SPEC[i]
        return rnd(conv3d(inp, P[i][0], P[i][1], m, relu=bool(relu)))

    a0 = c(0, x, n0)
    s0 = c(1, a0, n0)
    a1 = c(2, rnd(avgpool(s0, n0)), n1)
    s1 = c(3, a1, n1)
    a2 = c(4, rnd(avgpool(s1, n1)), n2)
    s2 = c(5, a2, n2)
    a3 = c(6, rnd(avgpool(s2, n2)), n3)
    bt = c(7, a3, n3)
    d2 = c(9, c(8, upcat(bt, s2, n2), n2), n2)
    d1 = c(11, c(10, upcat(d2, s1, n1), n1), n1)
    d0 = c(13, c(12, upcat(d1, s0, n0), n0), n0)
    ci, co, _, _ = SPEC[14]
    y = conv3d(d0, P[14][0], P[14][1], n0, relu=False)
    return y[:, 0]


def _relu_fwd(z):
    return np.maximum(z, 0.0)


def unet_loss_grad(params, x3, target, n):
    """Mean squared error (1/n^3) sum_v (y_v - t_v)^2 of the U-Net prediction
    and its gradient with respect to the flat parameter vector, in FP64
    without any bf16 rounding (the network the GPU's bf16 kernels
    approximate).  Reverse-mode chain rule through the same layers as
    unet_forward: convolutions (weight gradient conv3d_wgrad, data gradient
    conv3d_transpose), ReLU masks, average pooling (each fine voxel gets 1/8
    of its coarse gradient), nearest upsampling (a coarse voxel collects its
    8 fine gradients) and the channel concatenation.  Returns (loss, grad)."""
    P = [(np.asarray(w, np.float64), np.asarray(b, np.float64)) for w, b in unpack_params(params)]
    n0, n1, n2, n3 = n, n // 2, n // 4, n // 8
    x = np.zeros((n ** 3, 16))
    x[:, :3] = x3
    cache = {}

    def c(i, inp, m, key):
        z = conv3d(inp, P[i][0], P[i][1], m, relu=False)
        cache[key] = (i, inp, z, m)
        return _relu_fwd(z) if SPEC[i][3] else z

    a0 = c(0, x, n0, "a0")
    s0 = c(1, a0, n0, "s0")
    a1 = c(2, avgpool(s0, n0), n1, "a1")
    s1 = c(3, a1, n1, "s1")
    a2 = c(4, avgpool(s1, n1), n2, "a2")
    s2 = c(5, a2, n2, "s2")
    a3 = c(6, avgpool(s2, n2), n3, "a3")
    bt = c(7, a3, n3, "bt")
    a4 = c(8, upcat(bt, s2, n2), n2, "a4")
    d2 = c(9, a4, n2, "d2")
    a5 = c(10, upcat(d2, s1, n1), n1, "a5")
    d1 = c(11, a5, n1, "d1")
    a6 = c(12, upcat(d1, s0, n0), n0, "a6")
    d0 = c(13, a6, n0, "d0")
    yall = c(14, d0, n0, "y")
    r = yall[:, 0] - np.asarray(target, np.float64)
    loss = float(np.mean(r * r))
    grads = [None] * len(SPEC)

    def back(key, g_out):
        """Gradient through one convolution (and its ReLU): stores dW, db;
        returns the gradient of its input."""
        i, inp, z, m = cache[key]
        gz = g_out * (z > 0) if SPEC[i][3] else g_out
        dw, db = conv3d_wgrad(inp, gz, m)
        grads[i] = (dw, db)
        return conv3d_transpose(gz, P[i][0], m)

    def pool_back(g, m):
        """Adjoint of avgpool on an m^3 grid: each fine voxel gets 1/8 of its coarse gradient."""
        h = m // 2
        gg = g.reshape(h, h, h, -1) / 8.0
        return gg.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2).reshape(m ** 3, -1)

    def upcat_back(g, m, clo):
        """Adjoint of upcat on an m^3 grid: (gradient of the coarse input, of the skip)."""
        h = m // 2
        gl = g[:, :clo].reshape(h, 2, h, 2, h, 2, clo).sum(axis=(1, 3, 5)).reshape(h ** 3, clo)
        return gl, g[:, clo:]

    gy = np.zeros((n ** 3, 16))
    gy[:, 0] = 2.0 * r / (n ** 3)
    g = back("y", gy)
    g = back("d0", g)
    g_c0 = back("a6", g)
    g_d1, g_s0 = upcat_back(g_c0, n0, 32)
    g = back("d1", g_d1)
    g_c1 = back("a5", g)
    g_d2, g_s1 = upcat_back(g_c1, n1, 64)
    g = back("d2", g_d2)
    g_c2 = back("a4", g)
    g_bt, g_s2 = upcat_back(g_c2, n2, 128)
    g = back("bt", g_bt)
    g = back("a3", g)
    g_s2 = g_s2 + pool_back(g, n2)
    g = back("s2", g_s2)
    g = back("a2", g)
    g_s1 = g_s1 + pool_back(g, n1)
    g = back("s1", g_s1)
    g = back("a1", g)
    g_s0 = g_s0 + pool_back(g, n0)
    g = back("s0", g_s0)
    back("a0", g)
    flat = np.concatenate([np.concatenate([dw.ravel(), db]) for dw, db in grads])
    return loss, flat


def unet_loss(params, x3, target, n):
    """The loss of unet_loss_grad alone (FP64, no rounding)."""
    r = unet_forward(params, x3, n, bf16=False) - np.asarray(target, np.float64)
    return float(np.mean(r * r))
