"""Pins of the learned part's oracle (oracle/nn.py) against what fixes it
independently of its own code: a library correlation, the identity kernel,
adjointness, linearity in the weights, finite differences of the loss, and
the closed form of Adam's first step."""
import numpy as np
import pytest

from oracle import nn as O

scipy_signal = pytest.importorskip("scipy.signal")

N3 = (7, 6, 5)  # nx, ny, nz
N = N3[0] * N3[1] * N3[2]


def rnd(*shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv3d_matches_library_correlation():
    x, W, b = rnd(N, 3, seed=1), rnd(4, 27, 3, seed=2), rnd(4, seed=3)
    got = O.conv3d(x, W, b, N3)
    nx, ny, nz = N3
    for co in range(4):
        want = np.full((nz, ny, nx), b[co])
        for ci in range(3):
            k = W[co, :, ci].reshape(3, 3, 3)  # (dz + 1, dy + 1, dx + 1)
            want += scipy_signal.correlate(x[:, ci].reshape(nz, ny, nx), k, mode="same", method="direct")
        np.testing.assert_allclose(got[:, co], want.reshape(-1), rtol=1e-12, atol=1e-12)


def test_identity_kernel():
    x = rnd(N, 2, seed=4)
    W = np.zeros((2, 27, 2))
    W[0, 13, 0] = W[1, 13, 1] = 1.0  # tap 13 is the centre
    np.testing.assert_array_equal(O.conv3d(x, W, None, N3), x)


def test_dgrad_is_the_adjoint_of_the_convolution():
    x, W, dy = rnd(N, 3, seed=5), rnd(4, 27, 3, seed=6), rnd(N, 4, seed=7)
    lhs = np.sum(O.conv3d(x, W, None, N3) * dy)
    rhs = np.sum(x * O.conv3d_dgrad(dy, W, N3))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_wgrad_from_linearity_in_the_weights():
    x, W, b, dy = rnd(N, 3, seed=8), rnd(4, 27, 3, seed=9), rnd(4, seed=10), rnd(N, 4, seed=11)
    dW, db = O.conv3d_wgrad(x, dy, N3)
    # conv3d is linear in (W, b): <conv3d(x, W, b), dy> = <W, dW> + <b, db>
    lhs = np.sum(O.conv3d(x, W, b, N3) * dy)
    assert abs(lhs - (np.sum(W * dW) + np.dot(b, db))) <= 1e-10 * abs(lhs)


def net_params(seed=12):
    r = np.random.default_rng(seed)
    return [(0.3 * r.standard_normal((4, 27, 2)), 0.1 * r.standard_normal(4)),
            (0.2 * r.standard_normal((4, 27, 4)), 0.1 * r.standard_normal(4)),
            (0.2 * r.standard_normal((1, 27, 4)), 0.1 * r.standard_normal(1))]


def test_net_gradient_against_finite_differences():
    params = net_params()
    x = rnd(N, 2, seed=13)
    target = rnd(N, seed=14)
    mask = (np.random.default_rng(15).random(N) < 0.7).astype(float)

    def loss(ps):
        y, _ = O.net_forward(ps, x, N3)
        return O.mse(y, target, mask)[0]

    y, acts = O.net_forward(params, x, N3)
    _, dy = O.mse(y, target, mask)
    grads = O.net_backward(params, acts, dy, N3)
    r = np.random.default_rng(16)
    h = 1e-6
    for layer in range(3):
        for part in range(2):
            arr = params[layer][part]
            for _ in range(4):
                idx = tuple(r.integers(0, s) for s in arr.shape)
                save = arr[idx]
                arr[idx] = save + h
                lp = loss(params)
                arr[idx] = save - h
                lm = loss(params)
                arr[idx] = save
                fd = (lp - lm) / (2 * h)
                an = grads[layer][part][idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (layer, part, idx, fd, an)


def test_mse_gradient_against_finite_differences():
    y = rnd(N, 3, seed=17)
    target = rnd(N, seed=18)
    mask = (np.random.default_rng(19).random(N) < 0.5).astype(float)
    _, g = O.mse(y, target, mask)
    assert np.all(g[:, 1:] == 0.0) and np.all(g[mask == 0, 0] == 0.0)
    v = int(np.flatnonzero(mask)[3])
    h = 1e-6
    yp, ym = y.copy(), y.copy()
    yp[v, 0] += h
    ym[v, 0] -= h
    fd = (O.mse(yp, target, mask)[0] - O.mse(ym, target, mask)[0]) / (2 * h)
    assert abs(fd - g[v, 0]) <= 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    # m-hat = g and v-hat = g^2 after one step: w1 = w0 - lr * g / (|g| + eps)
    w, g = rnd(50, seed=20), rnd(50, seed=21)
    w1, m, v = O.adam(w, g, np.zeros(50), np.zeros(50), 1, 1e-2)
    np.testing.assert_allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)
