"""Pins of the FP64 network oracle (``oracle/net_oracle.py``) against facts outside it: a library
cross-correlation (scipy.ndimage), hand-built kernels with known outputs, the adjoint identity that
defines the transposed convolution, exact linearity in the weights, central finite differences of the
whole network's loss, and Adam's closed-form first steps."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import net_oracle as no

RNG = np.random.default_rng(2024)


def rand(*shape):
    return RNG.normal(size=shape)


def test_forward_matches_scipy_correlate():
    x, w, b = rand(5, 6, 7, 3), rand(27, 4, 3), rand(4)
    y = no.conv3d_forward(x, w, b)
    for co in range(4):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[:, co, ci].reshape(3, 3, 3)  # tap index (dz, dy, dx) -> kernel[dz, dy, dx]
            ref += ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(y[..., co], ref, rtol=1e-12, atol=1e-12)


def test_identity_and_shift_kernels():
    x = rand(4, 5, 6, 2)
    w = np.zeros((27, 2, 2))
    w[13] = np.eye(2)  # centre tap
    np.testing.assert_array_equal(no.conv3d_forward(x, w), x)
    w = np.zeros((27, 2, 2))
    t = (2 * 3 + 1) * 3 + 1  # offset (+1, 0, 0) along D
    w[t] = np.eye(2)
    y = no.conv3d_forward(x, w)
    np.testing.assert_array_equal(y[:-1], x[1:])
    np.testing.assert_array_equal(y[-1], 0.0)


def test_backward_data_is_the_adjoint():
    x, dy, w = rand(4, 5, 3, 3), rand(4, 5, 3, 5), rand(27, 5, 3)
    lhs = np.sum(no.conv3d_forward(x, w) * dy)
    rhs = np.sum(x * no.conv3d_backward_data(dy, w))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_backward_weight_is_exact_gradient_of_a_linear_form():
    x, dy = rand(3, 4, 5, 2), rand(3, 4, 5, 3)
    dw, db = no.conv3d_backward_weight(x, dy)
    # L(w, b) = <conv(x, w, b), dy> is linear: its gradient is exact and equals the basis responses
    for t, co, ci in [(0, 0, 0), (13, 2, 1), (26, 1, 0), (5, 0, 1)]:
        e = np.zeros((27, 3, 2))
        e[t, co, ci] = 1.0
        assert abs(np.sum(no.conv3d_forward(x, e) * dy) - dw[t, co, ci]) <= 1e-12
    for co in range(3):
        eb = np.zeros(3)
        eb[co] = 1.0
        assert abs(np.sum(no.conv3d_forward(x, np.zeros((27, 3, 2)), eb) * dy) - db[co]) <= 1e-12


def small_net(cin=4, hidden=5, cout=3):
    chans = [cin, hidden, hidden, hidden, cout]
    return [(0.3 * rand(27, chans[i + 1], chans[i]), 0.1 * rand(chans[i + 1])) for i in range(4)]


def test_network_gradient_by_central_differences():
    params = small_net()
    x = rand(4, 4, 5, 4)
    target = rand(4, 4, 5, 3)
    mask = RNG.random((4, 4, 5)) < 0.6

    def loss(ps):
        return no.mse_loss(no.net_forward(ps, x)[-1], target, mask)[0]

    acts = no.net_forward(params, x)
    _, dy = no.mse_loss(acts[-1], target, mask)
    grads = no.net_backward(params, acts, dy)
    h = 1e-6
    checked = 0
    for layer in range(4):
        w, b = params[layer]
        for idx in [(0, 0, 0), (13, w.shape[1] - 1, w.shape[2] - 1), (20, 1, 2 % w.shape[2])]:
            wp, wm = w.copy(), w.copy()
            wp[idx] += h
            wm[idx] -= h
            pp = list(params)
            pp[layer] = (wp, b)
            pm = list(params)
            pm[layer] = (wm, b)
            fd = (loss(pp) - loss(pm)) / (2 * h)
            an = grads[layer][0][idx]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3), (layer, idx, fd, an)
            checked += 1
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        pp = list(params)
        pp[layer] = (w, bp)
        pm = list(params)
        pm[layer] = (w, bm)
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - grads[layer][1][0]) <= 1e-6 * max(abs(fd), 1e-3)
    assert checked == 12


def test_mse_loss_definition():
    p, t = rand(2, 3, 4, 3), rand(2, 3, 4, 3)
    mask = np.zeros((2, 3, 4), bool)
    mask[0, 1, 2] = mask[1, 2, 3] = True
    L, g = no.mse_loss(p, t, mask)
    d = (p - t)[mask]
    assert L == pytest.approx((d ** 2).sum() / (2 * 3))
    assert np.all(g[~mask] == 0)


def test_relu_backward():
    act = np.array([0.0, 1.0, 2.0, 0.0])
    dy = np.array([5.0, 6.0, 7.0, 8.0])
    np.testing.assert_array_equal(no.relu_backward(dy, act), [0.0, 6.0, 7.0, 0.0])


def test_adam_first_steps_closed_form():
    p, g = np.array([1.0, -2.0, 0.5]), np.array([0.3, -4.0, 0.0])
    m = v = np.zeros(3)
    p1, m1, v1 = no.adam_step(p, g, m, v, 1, lr=0.01)
    # step 1: m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    g2 = np.array([0.1, 1.0, -2.0])
    p2, m2, v2 = no.adam_step(p1, g2, m1, v1, 2, lr=0.01)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p2, p1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-12)
