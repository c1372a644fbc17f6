"""Oracle of the learned part: a small 3D convolutional network on the grid.

TEST INFRASTRUCTURE ONLY (imported by tests/ and nothing in the product).
Plain numpy in FP64, written from the definitions, with no blocking or
reordering beyond them.

Fields live on the solver's grid: node (i, j, k) at linear index
i + nx*(j + ny*k); an activation is an array of shape (N, C), channels last.
A 3x3x3 convolution with zero padding and stride 1 has weights W of shape
(Co, 27, Ci); tap t stands for the offset
    (dz, dy, dx) = (t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1),
and
    out[v, co] = bias[co] + sum_t sum_ci W[co, t, ci] * in[v + off(t), ci],
where in[...] is zero outside the grid.  The network maps two input
channels (a residual and the unknowns' mask) through three such layers
(ReLU after the first two) to one output channel, the predicted error.
"""
import numpy as np

TAPS = [(t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1) for t in range(27)]


def shift(a, n, off):
    """a[v + off] with zero outside the grid: a has shape (N, C) on the grid
    n = (nx, ny, nz); off = (dz, dy, dx)."""
    nx, ny, nz = n
    g = a.reshape(nz, ny, nx, -1)
    out = np.zeros_like(g)
    dz, dy, dx = off
    zs, ys, xs = (slice(max(0, -d), m - max(0, d)) for d, m in ((dz, nz), (dy, ny), (dx, nx)))
    zd, yd, xd = (slice(max(0, d), m - max(0, -d)) for d, m in ((dz, nz), (dy, ny), (dx, nx)))
    out[zs, ys, xs] = g[zd, yd, xd]
    return out.reshape(a.shape)


def conv3d(x, W, bias, n):
    """Forward convolution: (N, Ci) -> (N, Co)."""
    out = np.zeros((x.shape[0], W.shape[0])) + (0.0 if bias is None else bias[None, :])
    for t, off in enumerate(TAPS):
        out += shift(x, n, off) @ W[:, t, :].T
    return out


def conv3d_dgrad(dy, W, n):
    """Gradient of sum(dy * conv3d(x, W)) with respect to x: the adjoint of the
    convolution, dx[v, ci] = sum_t sum_co W[co, t, ci] * dy[v - off(t), co]."""
    dx = np.zeros((dy.shape[0], W.shape[2]))
    for t, off in enumerate(TAPS):
        dx += shift(dy, n, tuple(-d for d in off)) @ W[:, t, :]
    return dx


def conv3d_wgrad(x, dy, n):
    """Gradients with respect to W and bias:
    dW[co, t, ci] = sum_v dy[v, co] * x[v + off(t), ci], db[co] = sum_v dy[v, co]."""
    dW = np.zeros((dy.shape[1], 27, x.shape[1]))
    for t, off in enumerate(TAPS):
        dW[:, t, :] = dy.T @ shift(x, n, off)
    return dW, dy.sum(axis=0)


def relu(a):
    return np.maximum(a, 0.0)


def mse(y, target, mask):
    """Masked mean squared error of output channel 0 and its gradient (N, Co)."""
    d = (y[:, 0] - target) * mask
    cnt = mask.sum()
    g = np.zeros_like(y)
    g[:, 0] = 2.0 * d / cnt
    return float((d * d).sum() / cnt), g


def net_forward(params, x, n):
    """params: [(W1, b1), (W2, b2), (W3, b3)]; returns (output, activations)."""
    (W1, b1), (W2, b2), (W3, b3) = params
    a1 = relu(conv3d(x, W1, b1, n))
    a2 = relu(conv3d(a1, W2, b2, n))
    return conv3d(a2, W3, b3, n), (x, a1, a2)


def net_backward(params, acts, dy, n):
    """Gradients [(dW1, db1), (dW2, db2), (dW3, db3)] of the network for dL/dy."""
    (W1, _), (W2, _), (W3, _) = params
    x, a1, a2 = acts
    g3 = conv3d_wgrad(a2, dy, n)
    d2 = conv3d_dgrad(dy, W3, n) * (a2 > 0)
    g2 = conv3d_wgrad(a1, d2, n)
    d1 = conv3d_dgrad(d2, W2, n) * (a1 > 0)
    g1 = conv3d_wgrad(x, d1, n)
    return [g1, g2, g3]


def adam(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1) on flat arrays; returns the new
    (w, m, v).  step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
