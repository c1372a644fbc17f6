"""The learned part's tensor-core kernels (include/cfp_nn.h) against the FP64
oracle (oracle/nn.py) on the same BF16-rounded inputs, the whole U-Net's
output and gradients, and determinism of the weight gradient.

Tolerances: the kernels accumulate in FP32, so an FP32 output may differ
from the FP64 value by a few units of 2^-24 times the sum of the absolute
terms (bounded here by 1e-5 of it); a BF16 output adds its own rounding,
2^-8 of the value.  Through the whole network, where every stored
activation is BF16 and an FP32 rounding difference can flip a BF16 rounding
that the later layers carry along, the output and every layer's gradient
agree with the oracle storing BF16 at the same points within twice the
distance between that oracle and the exact FP64 one (the size of the BF16
noise itself), plus 1e-2, in the relative 2-norm."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import nn as O  # noqa: E402
from paper_1901_08269_gb300 import cfp  # noqa: E402
from paper_1901_08269_gb300 import workloads as W  # noqa: E402

DIMS = (21, 13, 9)  # nx, ny, nz: 4095 padded voxels, 32 tiles of 128 and a ragged tail
PAIRS = [(16, 16), (16, 32), (32, 16), (32, 32), (32, 64), (64, 32), (64, 64), (64, 128), (128, 64), (128, 128)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def ctx():
    c = cfp.Context(W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), [])
    yield c
    c.close()


def npad(d):
    return (d[0] + 2) * (d[1] + 2) * (d[2] + 2)


def pad(a, d):
    """(N, C) on the grid d -> the padded (Np, C) layout, zero padding."""
    nx, ny, nz = d
    out = np.zeros((nz + 2, ny + 2, nx + 2, a.shape[1]))
    out[1:-1, 1:-1, 1:-1] = a.reshape(nz, ny, nx, -1)
    return out.reshape(-1, a.shape[1])


def unpad(a, d, c):
    nx, ny, nz = d
    g = a.reshape(nz + 2, ny + 2, nx + 2, c)
    return g, g[1:-1, 1:-1, 1:-1].reshape(-1, c)


def bf16(a):
    """(device bfloat16 tensor, the same values as float64 numpy)."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda().reshape(-1), t.double().numpy().reshape(np.shape(a))


def rnd(shape, seed, s=1.0):
    return s * np.random.default_rng(seed).standard_normal(shape)


def act_in(d, c, seed, relu=False):
    a = rnd((d[0] * d[1] * d[2], c), seed)
    if relu:
        a = np.maximum(a, 0.0)
    t, v = bf16(pad(a, d))
    return t, unpad(v, d, c)[1]


def close(got, want, scale, bf, what):
    tol = 1e-5 * scale + (2.0 ** -8) * np.abs(want) * (1 if bf else 0) + 1e-30
    err = np.abs(got - want)
    assert np.all(err <= tol), (what, float(np.max(err / tol)))


@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv_forward(ctx, cin, cout):
    d = DIMS
    x_d, x = act_in(d, cin, 1)
    w_d, w = bf16(rnd((cout, 27, cin), 2, 0.3))
    b = rnd(cout, 3, 0.5).astype(np.float32).astype(np.float64)
    b_d = torch.as_tensor(b, dtype=torch.float32).cuda()
    out = torch.empty(npad(d) * cout, dtype=torch.float32, device="cuda")
    ctx.nn_conv3d(d, cin, cout, x_d, w_d, out, bias=b_d, flags=cfp.NN_OUT_F32)
    g, got = unpad(out.double().cpu().numpy(), d, cout)
    want = O.conv3d(x, w, b, d)
    scale = O.conv3d(np.abs(x), np.abs(w), np.abs(b), d)
    close(got, want, scale, False, "forward")
    border = g.copy()
    border[1:-1, 1:-1, 1:-1] = 0.0
    assert np.all(border == 0.0)  # the padding rows are written as zeros
    # BF16 output with the ReLU
    outb = torch.empty(npad(d) * cout, dtype=torch.bfloat16, device="cuda")
    ctx.nn_conv3d(d, cin, cout, x_d, w_d, outb, bias=b_d, flags=cfp.NN_RELU)
    got = unpad(outb.double().cpu().numpy(), d, cout)[1]
    close(got, O.relu(want), scale, True, "forward bf16 relu")


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 64), (64, 32), (128, 128), (16, 32)])
def test_conv_input_gradient(ctx, cin, cout):
    # the input gradient of a (cin -> cout) layer: a (cout -> cin) call on
    # the forward weights, times [act > 0]
    d = DIMS
    g_d, g = act_in(d, cout, 4)
    w_d, w = bf16(rnd((cout, 27, cin), 5, 0.3))
    a_d, a = act_in(d, cin, 6, relu=True)
    out = torch.empty(npad(d) * cin, dtype=torch.bfloat16, device="cuda")
    ctx.nn_conv3d(d, cout, cin, g_d, w_d, out, act=a_d, flags=cfp.NN_DGRAD | cfp.NN_MASK)
    got = unpad(out.double().cpu().numpy(), d, cin)[1]
    want = O.conv3d_dgrad(g, w, d) * (a > 0)
    scale = O.conv3d_dgrad(np.abs(g), np.abs(w), d)
    close(got, want, scale, True, "dgrad")


@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv_weight_gradient(ctx, cin, cout):
    d = DIMS
    x_d, x = act_in(d, cin, 7)
    g_d, g = act_in(d, cout, 8)
    dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    ctx.nn_wgrad(d, cin, cout, x_d, g_d, dw, db)
    want, wantb = O.conv3d_wgrad(x, g, d)
    scale, scaleb = O.conv3d_wgrad(np.abs(x), np.abs(g), d)
    close(dw.double().cpu().numpy().reshape(cout, 27, cin), want, scale, False, "wgrad")
    close(db.double().cpu().numpy(), wantb, scaleb, False, "bias grad")
    # deterministic: a second call adds exactly the same values
    dw2 = dw.clone()
    ctx.nn_wgrad(d, cin, cout, x_d, g_d, dw2)
    assert torch.equal(dw2, 2 * dw)


def test_transfers(ctx):
    d = (17, 9, 13)
    dc = tuple((n + 1) // 2 for n in d)
    c = 32
    f_d, f = act_in(d, c, 9)
    c_d, cv = act_in(dc, c, 10)
    s_d, sv = act_in(d, c, 11)
    a_d, a = act_in(d, c, 12, relu=True)
    out_c = torch.empty(npad(dc) * c, dtype=torch.bfloat16, device="cuda")
    ctx.nn_transfer(cfp.NN_INJECT, d, c, f_d, out_c)
    np.testing.assert_array_equal(unpad(out_c.double().cpu().numpy(), dc, c)[1], O.inject(f, d))
    ctx.nn_transfer(cfp.NN_PROLONG_T, d, c, f_d, out_c)
    close(unpad(out_c.double().cpu().numpy(), dc, c)[1], O.prolong_t(f, d), O.prolong_t(np.abs(f), d), True, "P^T")
    out_f = torch.empty(npad(d) * c, dtype=torch.bfloat16, device="cuda")
    ctx.nn_transfer(cfp.NN_PROLONG_ADD, d, c, c_d, out_f, b=s_d)
    close(unpad(out_f.double().cpu().numpy(), d, c)[1], O.prolong(cv, d) + sv, O.prolong(np.abs(cv), d) + np.abs(sv),
          True, "P + skip")
    ctx.nn_transfer(cfp.NN_SKIP_GRAD, d, c, s_d, out_f, b=c_d, act=a_d)
    want = (sv + O.inject_t(cv, d)) * (a > 0)
    close(unpad(out_f.double().cpu().numpy(), d, c)[1], want, np.abs(sv) + O.inject_t(np.abs(cv), d), True, "skip")


def rel2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_unet_forward_and_gradients_match_the_oracle(ctx):
    d = (17, 9, 9)
    net = cfp.UNet(ctx, seed=3)
    p32 = net.params()
    # BF16 weights as the kernels use them, FP32 biases
    params = []
    o = 0
    for cin, cout, _l, _r in O.UNET_LAYERS:
        nw = cout * 27 * cin
        Wt = torch.as_tensor(p32[o:o + nw]).to(torch.bfloat16).double().numpy().reshape(cout, 27, cin)
        o += nw
        params.append((Wt, p32[o:o + cout].astype(np.float64)))
        o += cout
    nvox = d[0] * d[1] * d[2]
    r = np.random.default_rng(13)
    x = r.standard_normal((nvox, 16))
    x[:, 6:] = 0.0
    x_d, xv = bf16(pad(x, d))
    xv = unpad(xv, d, 16)[1]
    target = r.standard_normal(nvox).astype(np.float32).astype(np.float64)
    mask = (r.random(nvox) < 0.8).astype(np.float64)
    count = int(mask.sum())
    t_d = torch.as_tensor(pad(target[:, None], d).reshape(-1), dtype=torch.float32).cuda()
    m_d = torch.as_tensor(pad(mask[:, None], d).reshape(-1), dtype=torch.float32).cuda()
    y_d = torch.empty(npad(d) * 16, dtype=torch.float32, device="cuda")
    loss = net.forward_raw(d, x_d, y=y_d, target=t_d, mask=m_d, count=count)
    _, grads = net.params(grads=True)
    y = unpad(y_d.double().cpu().numpy(), d, 16)[1]
    yo, cache = O.unet_forward(params, xv, d, store=O._bf16)
    lo, gy = O.unet_loss_grad(yo, target, mask, count, d)
    go = O.unet_flatten(O.unet_backward(params, cache, gy, store=O._bf16))
    y64, cache64 = O.unet_forward(params, xv, d)  # exact: the BF16 noise level
    _, gy64 = O.unet_loss_grad(y64, target, mask, count, d)
    g64 = O.unet_flatten(O.unet_backward(params, cache64, gy64))
    assert rel2(y[:, 0], yo[:, 0]) <= 2 * rel2(yo[:, 0], y64[:, 0]) + 1e-2
    assert abs(loss - lo) <= 3e-2 * lo
    o = 0
    for li, (cin, cout, _l, _r) in enumerate(O.UNET_LAYERS):
        n = cout * 27 * cin + cout
        gw, gwo, gw64 = grads[o:o + n], go[o:o + n], g64[o:o + n]
        if li == len(O.UNET_LAYERS) - 1:  # only output channel 0 carries a gradient
            gw, gwo, gw64 = (a.reshape(-1)[:27 * cin] for a in (gw, gwo, gw64))
        bar = 2 * rel2(gwo, gw64) + 1e-2
        assert rel2(gw, gwo) <= bar, (li, rel2(gw, gwo), bar)
        o += n
    # the same call again: the same gradients added (deterministic kernels)
    net.forward_raw(d, x_d, target=t_d, mask=m_d, count=count)
    _, grads2 = net.params(grads=True)
    np.testing.assert_array_equal(grads2, 2 * grads)
    net.close()
