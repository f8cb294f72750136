"""Pins of the oracle's 3x3x3 convolutions (the learned part): brute-force
loops, shift kernels, the adjoint and bilinear identities, BF16 rounding."""
import numpy as np
import pytest

from oracle import conv


def brute_conv(x, W, b):
    n, Z, Y, X, ci = x.shape
    co = W.shape[4]
    y = np.zeros((n, Z, Y, X, co))
    for nn in range(n):
        for z in range(Z):
            for yy in range(Y):
                for xx in range(X):
                    for o in range(co):
                        s = b[o]
                        for kz in range(3):
                            for ky in range(3):
                                for kx in range(3):
                                    zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                                    if 0 <= zz < Z and 0 <= y2 < Y and 0 <= x2 < X:
                                        s += float(np.dot(x[nn, zz, y2, x2], W[kz, ky, kx, :, o]))
                        y[nn, z, yy, xx, o] = s
    return y


def test_conv_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 4, 5, 2))
    W = rng.standard_normal((3, 3, 3, 2, 3))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(conv.conv3d(x, W, b), brute_conv(x, W, b), rtol=1e-12, atol=1e-12)


def test_shift_kernels():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 4, 5, 6, 3))
    W = np.zeros((3, 3, 3, 3, 3))
    W[1, 1, 1] = np.eye(3)
    np.testing.assert_array_equal(conv.conv3d(x, W), x)
    W = np.zeros((3, 3, 3, 3, 3))
    W[1, 1, 2] = np.eye(3)         # reads x + 1
    y = conv.conv3d(x, W)
    np.testing.assert_array_equal(y[:, :, :, :-1], x[:, :, :, 1:])
    np.testing.assert_array_equal(y[:, :, :, -1], 0)


def test_backward_data_is_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 5, 4, 6, 3))
    W = rng.standard_normal((3, 3, 3, 3, 4))
    y = rng.standard_normal((2, 5, 4, 6, 4))
    lhs = np.sum(conv.conv3d(x, W) * y)
    rhs = np.sum(x * conv.conv3d_backward_data(y, W))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_backward_weight_bilinear_identity():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 4, 5, 3, 2))
    W = rng.standard_normal((3, 3, 3, 2, 3))
    y = rng.standard_normal((1, 4, 5, 3, 3))
    # <conv(x, W), y> is linear in W; its gradient in W is backward_weight(x, y)
    dW = conv.conv3d_backward_weight(x, y)
    assert np.sum(dW * W) == pytest.approx(np.sum(conv.conv3d(x, W) * y), rel=1e-12)
    e = np.zeros_like(W)
    e[0, 2, 1, 1, 2] = 1.0
    assert dW[0, 2, 1, 1, 2] == pytest.approx(np.sum(conv.conv3d(x, e) * y), rel=1e-12)


def test_bf16_round():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-3, 0.0], np.float32)
    r = conv.bf16_round(v)
    np.testing.assert_array_equal(r[[0, 3, 5]], v[[0, 3, 5]])
    assert r[1] == 1.0                    # tie -> even mantissa
    assert r[2] == 1.0 + 4 * 2 ** -8     # tie -> even (up)
    assert abs(r[4] - 3.0e-3) <= 2 ** -8 * 3.0e-3   # half an ulp of an 8-bit significand
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
