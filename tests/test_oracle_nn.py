"""Pins of the learned part's oracle (oracle/nn.py) against what fixes it
independently of its own code: a library correlation, the identity kernel,
adjointness, linearity in the weights, finite differences of the U-Net's
loss, exactness of the interpolation on linear fields, and the closed form
of Adam's first step."""
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


# ------------------------------------------------------------------ U-Net
NU = (17, 9, 9)  # levels (17, 9, 9), (9, 5, 5), (5, 3, 3), (3, 2, 2)


def test_injection_takes_the_even_nodes_and_its_adjoint():
    n = (9, 5, 7)
    a = rnd(9 * 5 * 7, 3, seed=30)
    c = O.inject(a, n)
    g = a.reshape(7, 5, 9, 3)
    for (K, J, I) in [(0, 0, 0), (1, 2, 3), (3, 2, 4)]:
        np.testing.assert_array_equal(c.reshape(4, 3, 5, 3)[K, J, I], g[2 * K, 2 * J, 2 * I])
    cc = rnd(c.shape[0], 3, seed=31)
    assert abs(np.sum(c * cc) - np.sum(a * O.inject_t(cc, n))) <= 1e-12 * np.sum(np.abs(c * cc))


def test_interpolation_exact_on_linear_index_fields_and_adjoint():
    n = (9, 7, 5)
    cx, cy, cz = O.coarse_n(n)
    K, J, I = np.meshgrid(np.arange(cz), np.arange(cy), np.arange(cx), indexing="ij")
    c = (1.5 + 0.3 * I - 0.7 * J + 0.2 * K).reshape(-1, 1)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    want = (1.5 + 0.3 * i / 2 - 0.7 * j / 2 + 0.2 * k / 2).reshape(-1, 1)
    np.testing.assert_allclose(O.prolong(c, n), want, rtol=0, atol=1e-13)
    f = rnd(9 * 7 * 5, 2, seed=32)
    cc = rnd(cx * cy * cz, 2, seed=33)
    lhs, rhs = np.sum(O.prolong(cc, n) * f), np.sum(cc * O.prolong_t(f, n))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(f))


def unet_setup(seed=40):
    r = np.random.default_rng(seed)
    p = []
    for cin, cout, _lvl, _relu in O.UNET_LAYERS:
        p.append(r.standard_normal(cout * 27 * cin) * np.sqrt(2.0 / (27 * cin)))
        p.append(0.05 * r.standard_normal(cout))
    p = np.concatenate(p)
    nvox = NU[0] * NU[1] * NU[2]
    x = r.standard_normal((nvox, 16))
    target = r.standard_normal(nvox)
    mask = (r.random(nvox) < 0.8).astype(float)
    return p, x, target, mask


def test_unet_shapes_and_parameter_count():
    p, x, target, mask = unet_setup()
    assert p.size == 1313968  # sum over the 13 layers of 27 cin cout + cout
    y, (A, ns) = O.unet_forward(O.unet_unflatten(p), x, NU)
    assert y.shape == (x.shape[0], 16) and ns[3] == (3, 2, 2)
    assert A["a7"].shape == (12, 128) and A["u2"].shape == (5 * 3 * 3, 64)


def test_unet_gradient_against_finite_differences():
    p, x, target, mask = unet_setup()
    count = float(mask.sum())

    def loss(pp):
        y, _ = O.unet_forward(O.unet_unflatten(pp), x, NU)
        return O.unet_loss_grad(y, target, mask, count, NU)[0]

    params = O.unet_unflatten(p)
    y, cache = O.unet_forward(params, x, NU)
    _, gy = O.unet_loss_grad(y, target, mask, count, NU)
    g = O.unet_flatten(O.unet_backward(params, cache, gy))
    r = np.random.default_rng(41)
    # two weights and one bias of every layer
    offs, o = [], 0
    for cin, cout, _lvl, _relu in O.UNET_LAYERS:
        nw = cout * 27 * cin
        if cout > 1:
            offs += [o + int(r.integers(0, 27 * cin)), o + int(r.integers(0, nw)), o + nw + 0]
        o += nw + cout
    h = 1e-6
    for k in offs:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - g[k]) <= 2e-6 * max(1e-3, abs(fd)) + 1e-9, (k, fd, g[k])


def test_energy_loss_definition_and_gradient():
    # brute force over the neighbouring pairs, the error zero outside the grid
    n = (4, 3, 5)
    N = 60
    y = rnd(N, 16, seed=50)
    t = rnd(N, seed=51)
    m = (np.random.default_rng(52).random(N) < 0.7).astype(float)
    L, g = O.unet_loss_grad(y, t, m, 7.0, n)
    d = ((y[:, 0] - t) * m).reshape(5, 3, 4)
    want = 0.0
    for k in range(-1, 5):
        for j in range(-1, 3):
            for i in range(-1, 4):
                v = d[k, j, i] if (0 <= k < 5 and 0 <= j < 3 and 0 <= i < 4) else 0.0
                for dk, dj, di in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
                    kk, jj, ii = k + dk, j + dj, i + di
                    w = d[kk, jj, ii] if (0 <= kk < 5 and 0 <= jj < 3 and 0 <= ii < 4) else 0.0
                    want += (v - w) ** 2
    assert abs(L - want / 7.0) <= 1e-12 * want
    assert np.all(g[:, 1:] == 0.0) and np.all(g[m == 0, 0] == 0.0)
    v = int(np.flatnonzero(m)[2])
    h = 1e-6
    yp, ym = y.copy(), y.copy()
    yp[v, 0] += h
    ym[v, 0] -= h
    fd = (O.unet_loss_grad(yp, t, m, 7.0, n)[0] - O.unet_loss_grad(ym, t, m, 7.0, n)[0]) / (2 * h)
    assert abs(fd - g[v, 0]) <= 1e-6 * max(1.0, abs(fd))
