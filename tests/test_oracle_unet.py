"""Pins of the U-Net reference (oracle/unet_oracle.py) against an independent
library routine, adjoint identities and brute force."""
import numpy as np
import pytest
from scipy import ndimage

import oracle.unet_oracle as U


def test_conv3d_single_channel_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    n = 6
    x = rng.standard_normal(n ** 3)
    k = rng.standard_normal((3, 3, 3))
    w = np.zeros((27, 1, 1))
    for t, (dz, dy, dx) in enumerate(U.TAPS):
        w[t, 0, 0] = k[dz + 1, dy + 1, dx + 1]
    ref = ndimage.correlate(x.reshape(n, n, n), k, mode="constant", cval=0.0)
    np.testing.assert_allclose(U.conv3d(x, w, None, n)[:, 0], ref.ravel(), rtol=1e-12, atol=1e-12)


def test_conv3d_transpose_is_the_adjoint():
    rng = np.random.default_rng(1)
    n, ci, co = 4, 5, 3
    x = rng.standard_normal((n ** 3, ci))
    y = rng.standard_normal((n ** 3, co))
    w = rng.standard_normal((27, co, ci))
    lhs = np.sum(U.conv3d(x, w, None, n) * y)
    rhs = np.sum(x * U.conv3d_transpose(y, w, n))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_wgrad_is_the_weight_adjoint():
    rng = np.random.default_rng(2)
    n, ci, co = 4, 4, 6
    x = rng.standard_normal((n ** 3, ci))
    dy = rng.standard_normal((n ** 3, co))
    w = rng.standard_normal((27, co, ci))
    b = rng.standard_normal(co)
    dw, db = U.conv3d_wgrad(x, dy, n)
    lhs = np.sum(U.conv3d(x, w, b, n) * dy)
    assert abs(lhs - (np.sum(w * dw) + b @ db)) < 1e-10 * abs(lhs)


def test_pool_and_upsample_brute_force():
    rng = np.random.default_rng(3)
    n = 4
    x = rng.standard_normal((n ** 3, 2))
    g = x.reshape(n, n, n, 2)
    p = U.avgpool(x, n).reshape(2, 2, 2, 2)
    for z in range(2):
        for y in range(2):
            for xx in range(2):
                np.testing.assert_allclose(p[z, y, xx], g[2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * xx:2 * xx + 2].mean((0, 1, 2)))
    lo = rng.standard_normal((8, 3))
    cat = U.upcat(lo, x, n).reshape(n, n, n, 5)
    assert np.allclose(cat[3, 2, 1, :3], lo.reshape(2, 2, 2, 3)[1, 1, 0])
    assert np.allclose(cat[..., 3:], g)


def test_bf16_rounding_ties_to_even():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5, 3.0e-3])
    r = U.to_bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0            # halfway -> even mantissa
    assert r[2] == 1.0 + 2.0 ** -6                # halfway -> even mantissa
    assert r[3] == 1.0 + 2.0 ** -7 and r[4] == -2.5
    assert abs(r[5] / 3.0e-3 - 1) < 2.0 ** -8


def _random_net(seed, n):
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, _, _ in U.SPEC:
        parts.append(rng.standard_normal(27 * co * ci) * np.sqrt(2.0 / (27 * ci)))
        parts.append(0.05 * rng.standard_normal(co))
    p = np.concatenate(parts)
    x3 = rng.standard_normal((n ** 3, 3))
    t = rng.standard_normal(n ** 3)
    return p, x3, t


def test_unet_gradient_matches_central_differences():
    """The whole-network reverse pass of unet_loss_grad against central
    differences of the FP64 loss along random directions (8^3 grid: levels 8,
    4, 2, 1), each direction also restricted to one layer so that a wrong or
    missing layer gradient shows; and the plain loss equals the one the
    gradient routine reports."""
    n = 8
    p, x3, t = _random_net(3, n)
    loss, g = U.unet_loss_grad(p, x3, t, n)
    assert abs(loss - U.unet_loss(p, x3, t, n)) <= 1e-14 * loss
    rng = np.random.default_rng(4)
    sizes = [27 * co * ci + co for ci, co, _, _ in U.SPEC]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    dirs = [rng.standard_normal(p.size)]
    for layer in (0, 6, 8, 12, 14):
        d = np.zeros(p.size)
        d[offs[layer]:offs[layer + 1]] = rng.standard_normal(sizes[layer])
        dirs.append(d)
    for d in dirs:
        d = d / np.linalg.norm(d)
        eps = 1e-6
        fd = (U.unet_loss(p + eps * d, x3, t, n) - U.unet_loss(p - eps * d, x3, t, n)) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), 1e-3 * np.linalg.norm(g))
