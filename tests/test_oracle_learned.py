"""Pins of the oracle's learned-gradient step (oracle.learned): a network
that is the identity on the gradient channel reduces the step to plain
gradient descent, and the hand-written chain rule matches central finite
differences of the step in x, in a weight and in a bias."""
import numpy as np

import oracle
from oracle import learned
from paper_2412_10129_gb300 import inputs


def _geo():
    return inputs.random_geometry((6, 7, 5), (1.1, 0.9, 1.3), (10, 8), (1.4, 1.6), 4, seed=11)


def _net(rng, chans):
    Ws, Bs = [], []
    for ci, co in zip(chans[:-1], chans[1:]):
        Ws.append(rng.standard_normal((3, 3, 3, ci, co)) * 0.3)
        Bs.append(rng.standard_normal(co) * 0.1)
    return Ws, Bs


def test_identity_network_is_gradient_descent():
    geo = _geo()
    rng = np.random.default_rng(0)
    x = rng.random(geo.vol_shape)
    b = rng.random(geo.proj_shape)
    # layer 1: (relu(c1), relu(-c1)); layer 2: pass-through; layer 3: ch0 - ch1
    W1 = np.zeros((3, 3, 3, 3, 2)); W1[1, 1, 1, 1, 0] = 1.0; W1[1, 1, 1, 1, 1] = -1.0
    W2 = np.zeros((3, 3, 3, 2, 2)); W2[1, 1, 1] = np.eye(2)
    W3 = np.zeros((3, 3, 3, 2, 1)); W3[1, 1, 1, 0, 0] = 1.0; W3[1, 1, 1, 1, 0] = -1.0
    Bs = [np.zeros(2), np.zeros(2), np.zeros(1)]
    sx, sg, so = 2.0, 0.37, -1.5
    xn, _ = learned.step(geo, x, b, [W1, W2, W3], Bs, sx, sg, so)
    grad = oracle.backproject(geo, oracle.forward(geo, x) - b)
    np.testing.assert_allclose(xn, x + so * sg * grad, rtol=1e-12, atol=1e-12)


def test_chain_rule_matches_finite_differences():
    geo = _geo()
    rng = np.random.default_rng(1)
    x = rng.random(geo.vol_shape)
    b = rng.random(geo.proj_shape)
    Ws, Bs = _net(rng, (3, 4, 4, 2))
    sx, sg, so = 1.7, 0.05, 0.8
    gbar = rng.standard_normal(geo.vol_shape)
    gx, dWs, dBs = learned.step_backward(geo, x, b, Ws, Bs, sx, sg, so, gbar)

    def L(x_, Ws_=Ws, Bs_=Bs):
        return float(np.sum(gbar * learned.step(geo, x_, b, Ws_, Bs_, sx, sg, so)[0]))

    h = 1e-6
    for _ in range(3):
        d = rng.standard_normal(geo.vol_shape)
        fd = (L(x + h * d) - L(x - h * d)) / (2 * h)
        assert abs(fd - np.sum(gx * d)) <= 1e-6 * max(1.0, abs(fd))
    for li, idx in ((0, (0, 2, 1, 1, 3)), (1, (1, 1, 1, 2, 0)), (2, (2, 0, 1, 3, 1))):
        Wp = [w.copy() for w in Ws]; Wm = [w.copy() for w in Ws]
        Wp[li][idx] += h; Wm[li][idx] -= h
        fd = (L(x, Wp) - L(x, Wm)) / (2 * h)
        assert abs(fd - dWs[li][idx]) <= 1e-6 * max(1.0, abs(fd))
    for li, o in ((0, 2), (2, 1)):
        Bp = [c.copy() for c in Bs]; Bm = [c.copy() for c in Bs]
        Bp[li][o] += h; Bm[li][o] -= h
        fd = (L(x, Ws, Bp) - L(x, Ws, Bm)) / (2 * h)
        assert abs(fd - dBs[li][o]) <= 1e-6 * max(1.0, abs(fd))
