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


def adam(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1) on flat arrays; returns the new
    (w, m, v).  step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ U-Net
# Four levels; level l+1 has (n_l + 1) // 2 nodes per axis (odd sizes), its
# node I on node 2I of level l.  Written from the definitions: injection R,
# linear interpolation P in index space, and the network
#   a0 = relu(conv(x)), a1 = relu(conv(a0))          level 0, 16 channels
#   a2 = relu(conv(R a1)), a3 = relu(conv(a2))       level 1, 32
#   a4 = relu(conv(R a3)), a5 = relu(conv(a4))       level 2, 64
#   a6 = relu(conv(R a5)), a7 = relu(conv(a6))       level 3, 128
#   u2 = P conv(a7) + a5, a8 = relu(conv(u2))
#   u1 = P conv(a8) + a3, a9 = relu(conv(u1))
#   c0 = conv(a9) at level 1,  y = P c0 (its channel 0) on level 0.
UNET_LAYERS = [(16, 16, 0, 1), (16, 16, 0, 1), (16, 32, 1, 1), (32, 32, 1, 1), (32, 64, 2, 1), (64, 64, 2, 1),
               (64, 128, 3, 1), (128, 128, 3, 1), (128, 64, 3, 0), (64, 64, 2, 1), (64, 32, 2, 0), (32, 32, 1, 1),
               (32, 16, 1, 0)]  # (cin, cout, level, relu)


def coarse_n(n):
    return tuple((m + 1) // 2 for m in n)


def unet_unflatten(p):
    """The flat parameter vector (per layer W [cout][27][cin] then b [cout])
    as [(W, b)] per layer."""
    out, o = [], 0
    for cin, cout, _lvl, _relu in UNET_LAYERS:
        W = p[o:o + cout * 27 * cin].reshape(cout, 27, cin)
        o += cout * 27 * cin
        b = p[o:o + cout]
        o += cout
        out.append((W, b))
    assert o == p.size
    return out


def unet_flatten(grads):
    return np.concatenate([np.concatenate([dW.reshape(-1), db.reshape(-1)]) for dW, db in grads])


def inject(a, n):
    """R: the coarse grid's node (I, J, K) takes the fine node (2I, 2J, 2K)."""
    nx, ny, nz = n
    g = a.reshape(nz, ny, nx, -1)
    return np.ascontiguousarray(g[::2, ::2, ::2]).reshape(-1, a.shape[1])


def inject_t(c, n):
    """R^T: coarse node I placed on fine node 2I, zero elsewhere."""
    nx, ny, nz = n
    out = np.zeros((nz, ny, nx, c.shape[1]))
    cx, cy, cz = coarse_n(n)
    out[::2, ::2, ::2] = c.reshape(cz, cy, cx, -1)
    return out.reshape(-1, c.shape[1])


def _interp_matrix(nf):
    """P along one axis (nf odd): fine 2I = coarse I, fine 2I+1 = the mean of
    coarse I and I+1."""
    nc = (nf + 1) // 2
    M = np.zeros((nf, nc))
    for i in range(nf):
        if i % 2 == 0:
            M[i, i // 2] = 1.0
        else:
            M[i, i // 2] = M[i, i // 2 + 1] = 0.5
    return M


def prolong(c, n):
    """P: coarse -> fine (n the fine sizes), trilinear in index space."""
    nx, ny, nz = n
    Mx, My, Mz = _interp_matrix(nx), _interp_matrix(ny), _interp_matrix(nz)
    cx, cy, cz = coarse_n(n)
    g = c.reshape(cz, cy, cx, -1)
    f = np.einsum("zk,yj,xi,kjic->zyxc", Mz, My, Mx, g)
    return f.reshape(-1, c.shape[1])


def prolong_t(f, n):
    """P^T: fine -> coarse."""
    nx, ny, nz = n
    Mx, My, Mz = _interp_matrix(nx), _interp_matrix(ny), _interp_matrix(nz)
    g = f.reshape(nz, ny, nx, -1)
    c = np.einsum("zk,yj,xi,zyxc->kjic", Mz, My, Mx, g)
    return c.reshape(-1, f.shape[1])


def _bf16(a):
    """Round to the nearest BF16 value (ties to even), as the tensor cores'
    activations are stored."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unet_forward(params, x, n, store=None):
    """params: [(W, b)] per layer; x (N0, 16) on the level-0 grid n = (nx, ny,
    nz).  store: None (FP64 throughout) or a rounding applied wherever an
    activation is stored (the kernels store BF16).  Returns (y, acts)."""
    s = store or (lambda a: a)
    ns = [tuple(n)]
    for _ in range(3):
        ns.append(coarse_n(ns[-1]))

    def layer(l, inp):
        W, b = params[l]
        out = conv3d(inp, W, b, ns[UNET_LAYERS[l][2]])
        return relu(out) if UNET_LAYERS[l][3] else out

    A = {"x": x}
    A["a0"] = s(layer(0, A["x"]))
    A["a1"] = s(layer(1, A["a0"]))
    A["b0"] = inject(A["a1"], ns[0])
    A["a2"] = s(layer(2, A["b0"]))
    A["a3"] = s(layer(3, A["a2"]))
    A["b1"] = inject(A["a3"], ns[1])
    A["a4"] = s(layer(4, A["b1"]))
    A["a5"] = s(layer(5, A["a4"]))
    A["b2"] = inject(A["a5"], ns[2])
    A["a6"] = s(layer(6, A["b2"]))
    A["a7"] = s(layer(7, A["a6"]))
    A["c2"] = s(layer(8, A["a7"]))
    A["u2"] = s(prolong(A["c2"], ns[2]) + A["a5"])
    A["a8"] = s(layer(9, A["u2"]))
    A["c1"] = s(layer(10, A["a8"]))
    A["u1"] = s(prolong(A["c1"], ns[1]) + A["a3"])
    A["a9"] = s(layer(11, A["u1"]))
    A["c0"] = s(layer(12, A["a9"]))
    y = np.zeros((x.shape[0], 16))
    y[:, 0] = prolong(A["c0"][:, :1], ns[0])[:, 0]
    return y, (A, ns)


def unet_backward(params, cache, gy, store=None):
    """Gradients [(dW, db)] per layer of sum(gy * y) (gy: dL/dy, (N0, 16)),
    by the chain rule through unet_forward's graph in reverse.  store rounds
    the gradient activations as the kernels store them."""
    s = store or (lambda a: a)
    A, ns = cache
    grads = [None] * len(UNET_LAYERS)

    def back(l, inp, gout, act_in):
        """gout: the gradient at layer l's pre-activation output; returns the
        gradient at its input (times [act_in > 0] when act_in is given)."""
        W, _ = params[l]
        grads[l] = conv3d_wgrad(inp, gout, ns[UNET_LAYERS[l][2]])
        gin = conv3d_dgrad(gout, W, ns[UNET_LAYERS[l][2]])
        return s(gin * (act_in > 0) if act_in is not None else gin)

    g = np.zeros((A["c0"].shape[0], 16))
    g[:, 0] = prolong_t(s(gy)[:, :1], ns[0])[:, 0]   # of c0 (channel 0 feeds y)
    g = s(g)
    g = back(12, A["a9"], g, A["a9"])
    gu1 = back(11, A["u1"], g, None)
    g = s(prolong_t(gu1, ns[1]))                 # of c1
    g = back(10, A["a8"], g, A["a8"])
    gu2 = back(9, A["u2"], g, None)
    g = s(prolong_t(gu2, ns[2]))                 # of c2
    g = back(8, A["a7"], g, A["a7"])
    g = back(7, A["a6"], g, A["a6"])
    gb2 = back(6, A["b2"], g, None)              # of b2
    g = s((gu2 + inject_t(gb2, ns[2])) * (A["a5"] > 0))
    g = back(5, A["a4"], g, A["a4"])
    gb1 = back(4, A["b1"], g, None)
    g = s((gu1 + inject_t(gb1, ns[1])) * (A["a3"] > 0))
    g = back(3, A["a2"], g, A["a2"])
    gb0 = back(2, A["b0"], g, None)
    g = s(inject_t(gb0, ns[0]) * (A["a1"] > 0))
    g = back(1, A["a0"], g, A["a0"])
    grads[0] = conv3d_wgrad(A["x"], g, ns[0])
    return grads


def unet_loss_grad(y, target, mask, count, n):
    """The energy norm of the error d = mask (y[:, 0] - target) on the grid n,
    the error being zero outside it (Dirichlet):
        L = (1 / count) sum over neighbouring pairs (p, q) (d_p - d_q)^2,
    pairs of the grid padded by one zero node on every side; and dL/dy."""
    nx, ny, nz = n
    d = ((y[:, 0] - target) * mask).reshape(nz, ny, nx)
    dp = np.zeros((nz + 2, ny + 2, nx + 2))
    dp[1:-1, 1:-1, 1:-1] = d
    L = sum(float(np.sum(np.diff(dp, axis=a) ** 2)) for a in range(3)) / count
    lap = 6.0 * dp[1:-1, 1:-1, 1:-1] - (dp[2:, 1:-1, 1:-1] + dp[:-2, 1:-1, 1:-1] + dp[1:-1, 2:, 1:-1] +
                                        dp[1:-1, :-2, 1:-1] + dp[1:-1, 1:-1, 2:] + dp[1:-1, 1:-1, :-2])
    g = np.zeros_like(y)
    g[:, 0] = 2.0 / count * mask * lap.reshape(-1)
    return L, g
