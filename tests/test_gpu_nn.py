"""The learned part's kernels (include/cfp_nn.h) against the FP64 oracle
(oracle/nn.py) on the same BF16-rounded inputs, and a training run on pairs
the solver generates.

Tolerances: the kernels accumulate in FP32, so an FP32 output may differ
from the FP64 value by a few units of 2^-24 times the sum of the absolute
terms; a BF16 output adds its own rounding, 2^-8 of the value."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import nn as O  # noqa: E402
from paper_1901_08269_gb300 import cfp  # noqa: E402
from paper_1901_08269_gb300 import learned  # noqa: E402
from paper_1901_08269_gb300 import workloads as W  # noqa: E402

NX, NY, NZ = 21, 13, 9  # two x tiles of 16, the second ragged
N = NX * NY * NZ


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def ctx():
    c = cfp.Context(W.uniform_grid(0, 1, NX), W.uniform_grid(0, 1, NY), W.uniform_grid(0, 1, NZ), [])
    yield c
    c.close()


def bf16(a):
    """(device bfloat16 tensor, the same values as float64 numpy)."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda().reshape(-1), t.double().numpy().reshape(np.shape(a))


def host(t, shape):
    return t.double().cpu().numpy().reshape(shape)


def rnd(shape, seed, s=1.0):
    return s * np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("relu,out32,with_bias", [(False, True, True), (True, True, False), (True, False, True),
                                                  (False, False, False)])
def test_conv3d_forward(ctx, relu, out32, with_bias):
    x_d, x = bf16(rnd((N, 16), 1))
    w_d, w = bf16(rnd((16, 27, 16), 2, 0.2))
    b = rnd(16, 3, 0.5).astype(np.float32).astype(np.float64)
    b_d = torch.as_tensor(b, dtype=torch.float32).cuda() if with_bias else None
    out = torch.empty(N * 16, dtype=torch.float32 if out32 else torch.bfloat16, device="cuda")
    ctx.nn_conv3d(x_d, w_d, b_d, int(relu), out)
    got = host(out, (N, 16))
    pre = O.conv3d(x, w, b if with_bias else None, (NX, NY, NZ))
    want = O.relu(pre) if relu else pre
    scale = O.conv3d(np.abs(x), np.abs(w), np.abs(b) if with_bias else None, (NX, NY, NZ))
    tol = 4e-7 * scale + 1e-6 + (0.0 if out32 else 2.0 ** -8 * np.abs(want))
    assert np.all(np.abs(got - want) <= tol), np.max(np.abs(got - want) - tol)


def test_conv3d_dgrad_with_relu_mask(ctx):
    dy_d, dy = bf16(rnd((N, 16), 4))
    w_d, w = bf16(rnd((16, 27, 16), 5, 0.2))
    act_d, act = bf16(rnd((N, 16), 6))  # about half positive
    din = torch.empty(N * 16, dtype=torch.bfloat16, device="cuda")
    ctx.nn_dgrad(dy_d, w_d, act_d, din)
    got = host(din, (N, 16))
    want = O.conv3d_dgrad(dy, w, (NX, NY, NZ)) * (act > 0)
    scale = O.conv3d_dgrad(np.abs(dy), np.abs(w), (NX, NY, NZ))
    assert np.all(got[act <= 0] == 0.0)
    assert np.all(np.abs(got - want) <= 4e-7 * scale + 2.0 ** -8 * np.abs(want) + 1e-6)


def test_conv3d_wgrad_and_bias_grad(ctx):
    x_d, x = bf16(rnd((N, 16), 7))
    dy_d, dy = bf16(rnd((N, 16), 8))
    dw = torch.full((16 * 27 * 16,), 0.25, dtype=torch.float32, device="cuda")  # accumulates onto this
    db = torch.full((16,), -0.5, dtype=torch.float32, device="cuda")
    ctx.nn_wgrad(x_d, dy_d, dw, db)
    want_w, want_b = O.conv3d_wgrad(x, dy, (NX, NY, NZ))
    scale_w, scale_b = O.conv3d_wgrad(np.abs(x), np.abs(dy), (NX, NY, NZ))
    got_w = host(dw, (16, 27, 16)) - 0.25
    got_b = db.double().cpu().numpy() + 0.5
    assert np.all(np.abs(got_w - want_w) <= 2e-6 * scale_w + 1e-6)
    assert np.all(np.abs(got_b - want_b) <= 2e-6 * scale_b + 1e-6)


def test_mse_and_adam(ctx):
    y = rnd((N, 16), 9).astype(np.float32).astype(np.float64)
    target = rnd(N, 10).astype(np.float32).astype(np.float64)
    mask = (np.random.default_rng(11).random(N) < 0.6).astype(np.float64)
    dy = torch.empty(N * 16, dtype=torch.bfloat16, device="cuda")
    loss = ctx.nn_mse(torch.as_tensor(y, dtype=torch.float32).cuda().reshape(-1),
                      torch.as_tensor(target, dtype=torch.float32).cuda(),
                      torch.as_tensor(mask, dtype=torch.float32).cuda(), 1.0 / mask.sum(), dy)
    want_loss, want_g = O.mse(y, target, mask)
    assert abs(loss - want_loss) <= 1e-6 * want_loss
    got_g = host(dy, (N, 16))
    assert np.all(np.abs(got_g - want_g) <= 2.0 ** -8 * np.abs(want_g) + 1e-9)
    # two Adam steps against the oracle's
    w0, g1, g2 = rnd(500, 12), rnd(500, 13), rnd(500, 14)
    w = torch.as_tensor(w0, dtype=torch.float32).cuda()
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    wb = torch.empty(500, dtype=torch.bfloat16, device="cuda")
    ow, om, ov = w0.astype(np.float32).astype(np.float64), np.zeros(500), np.zeros(500)
    for step, g in ((1, g1), (2, g2)):
        gd = torch.as_tensor(g, dtype=torch.float32).cuda()
        ctx.nn_adam(w, gd, m, v, step, 1e-2, wb)
        assert torch.all(gd == 0)
        ow, om, ov = O.adam(ow, g.astype(np.float32).astype(np.float64), om, ov, step, 1e-2)
    np.testing.assert_allclose(w.double().cpu().numpy(), ow, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(wb.double().cpu().numpy(), ow, rtol=2.0 ** -8, atol=1e-6)


def test_pack_scale_and_unpack():
    w = W.config2(17)
    c = cfp.Context(w.x, w.y, w.z, w.bodies)
    ty = torch.empty(w.N, dtype=torch.uint8, device="cuda")
    c.classify_points(ty)
    unk = ((ty == cfp.REGULAR) | (ty == cfp.IRREGULAR)).cpu().numpy()
    r = torch.as_tensor(rnd(w.N, 15), device="cuda")
    e = torch.as_tensor(rnd(w.N, 16), device="cuda")
    x = torch.empty(w.N * 16, dtype=torch.bfloat16, device="cuda")
    tgt = torch.empty(w.N, dtype=torch.float32, device="cuda")
    msk = torch.empty(w.N, dtype=torch.float32, device="cuda")
    scale = c.nn_pack(r, e, 0.0, 3.0, x, tgt, msk)
    rn, en = r.cpu().numpy(), e.cpu().numpy()
    assert scale == pytest.approx(1.0 / np.max(np.abs(rn[unk])), rel=1e-7)  # max taken in FP32
    xs = host(x, (w.N, 16))
    np.testing.assert_allclose(xs[:, 0], np.where(unk, scale * rn, 0.0), rtol=2.0 ** -8, atol=0)
    np.testing.assert_array_equal(xs[:, 1], unk.astype(float))
    assert np.all(xs[:, 2:] == 0)
    np.testing.assert_allclose(tgt.double().cpu().numpy(), np.where(unk, 3.0 * scale * en, 0.0), rtol=1e-6, atol=0)
    np.testing.assert_array_equal(msk.cpu().numpy(), unk.astype(np.float32))
    y = torch.zeros(w.N * 16, dtype=torch.float32, device="cuda")
    y[0::16] = tgt
    u = torch.full((w.N,), 9.0, dtype=torch.float64, device="cuda")
    c.nn_unpack(y, 1.0 / (3.0 * scale), u)
    np.testing.assert_allclose(u.cpu().numpy(), np.where(unk, en, 0.0), rtol=1e-6, atol=0)
    c.close()


@pytest.fixture(scope="module")
def trained():
    """The network trained on solver-generated pairs (random bodies at 33^3)."""
    train_w = [W.random_problem(s, sizes=(33,)) for s in range(6)]
    samples, escale = learned.make_samples(train_w)
    net = learned.ConvNet(seed=0, escale=escale)
    losses = learned.train(net, samples, 600, lr=2e-3)
    return net, losses


def test_training_on_solver_pairs_and_the_guess_it_gives(trained):
    """Training lowers the loss; on held-out problems compare the network's
    initial guess with zero: its error and the iterations of the same solve
    from it."""
    net, losses = trained
    first, last = float(np.mean(losses[:6])), float(np.mean(losses[-30:]))
    assert np.isfinite(last) and last < 0.5 * first, (first, last)
    report = []
    for s in (100, 101):
        w = W.random_problem(s, sizes=(33,))
        smp = learned.Sample(w)
        u0 = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        net.guess(smp.ctx, smp.rhs, u0)
        err0 = float((smp.u).abs().max())
        errn = float((u0 - smp.u).abs().max())
        its = {}
        for name, guess in (("zero", torch.zeros_like(u0)), ("net", u0.clone())):
            info = smp.ctx.solve(smp.f, smp.g, smp.gi, guess, tol=1e-10, precision=cfp.PREC_MIXED,
                                 precond=cfp.PRECOND_MG)
            assert info.status == 0
            its[name] = info.iterations
            np.testing.assert_allclose(guess.cpu().numpy(), smp.u.cpu().numpy(), rtol=0, atol=1e-8 * err0)
        report.append((s, errn / err0, its))
    print("learned initial guess: loss %.3e -> %.3e; held-out (seed, error ratio, iterations): %s"
          % (first, last, report))
    assert all(r[1] < 1.0 for r in report), report


def test_network_as_preconditioner_in_flexible_gmres(trained):
    """FGMRES whose first direction comes from the network (z = net(v) +
    V(v - B net(v)), the V-cycle V alone afterwards) against FGMRES with the
    V-cycle alone; both reach the solution of the plain BiCGSTAB solve (the
    reference) on a held-out problem."""
    net, _ = trained
    w = W.random_problem(100, sizes=(33,))
    smp = learned.Sample(w, tol=1e-12)
    ctx = smp.ctx
    ref = smp.u.cpu().numpy()
    opts = cfp.default_opts(precond=cfp.PRECOND_MG, mg_smooth=2)
    its = {}
    for name, prec in (("mg", learned.mg_precond(ctx, opts)), ("net+mg", learned.net_mg_precond(ctx, net, opts))):
        x = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        n_it, rel = learned.fgmres(ctx, smp.rhs, x, prec, m=30, tol=1e-11, maxit=200)
        assert rel <= 1e-11, (name, rel)
        assert np.max(np.abs(x.cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref)), name
        its[name] = n_it
    print("FGMRES iterations to 1e-11:", its)
