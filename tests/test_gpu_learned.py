"""The flexible GMRES of the learned part (cfp_solve_fgmres) and the U-Net's
training through the C ABI.

Without a network the flexible GMRES is right-preconditioned GMRES: its
solution must equal the preconditioned BiCGSTAB's (and so the oracle's,
which the BiCGSTAB parity tests pin) within the solve tolerance.  With a
network (trained or not) the preconditioner changes from step to step and
the flexible method must still converge to the same solution.  Training is
deterministic: the same seed and pairs give the same parameters bit for
bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pyoracle as O  # noqa: E402
from paper_1901_08269_gb300 import cfp  # noqa: E402
from paper_1901_08269_gb300 import learned  # noqa: E402
from paper_1901_08269_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def setup(w):
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    t = torch.empty(w.N, dtype=torch.uint8, device="cuda")
    ctx.classify_points(t)
    xyz = ctx.ibi_points()
    f, g = w.fields(torch, "cuda")
    gi = w.g_at(xyz, torch).contiguous() if ctx.n_ibi else None
    return ctx, t, f, g, gi


@pytest.mark.parametrize("precond,prec", [(cfp.PRECOND_RBGS, cfp.PREC_FP64), (cfp.PRECOND_MG, cfp.PREC_FP64),
                                          (cfp.PRECOND_MG, cfp.PREC_MIXED)])
def test_fgmres_without_network_matches_bicgstab_and_oracle(precond, prec):
    w = W.config2(33)
    ctx, t, f, g, gi = setup(w)
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    info = ctx.solve_fgmres(f, g, gi, u, tol=1e-12, m=20, precond=precond, precision=prec, sweeps=8)
    assert info.status == 0 and info.rel_residual <= 1e-12
    ub = torch.zeros_like(u)
    ctx.solve(f, g, gi, ub, tol=1e-12, precond=precond, sweeps=8)
    d = float((u - ub).abs().max() / ub.abs().max())
    assert d <= 1e-9, d
    P = O.Problem(w.x, w.y, w.z, w.bodies)
    P.classify()
    _, _, oxyz = P.ibi()
    fo, go = w.fields()
    uo, st, it, rel = P.solve(fo, go, w.g_at(oxyz), tol=1e-12)
    assert st == 0
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-9 * np.max(np.abs(uo))
    ctx.close()


def test_fgmres_with_an_untrained_network_still_converges():
    w = W.random_problem(101, sizes=(33,))
    ctx, t, f, g, gi = setup(w)
    net = cfp.UNet(ctx, seed=1)
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    info = ctx.solve_fgmres(f, g, gi, u, tol=1e-10, net=net, m=20, net_guess=True, precond=cfp.PRECOND_RBGS,
                            sweeps=8)
    assert info.status == 0 and info.rel_residual <= 1e-10
    ub = torch.zeros_like(u)
    ctx.solve(f, g, gi, ub, tol=1e-12, precond=cfp.PRECOND_MG)
    assert float((u - ub).abs().max() / ub.abs().max()) <= 1e-7
    net.close()
    ctx.close()


def test_training_is_deterministic_and_lowers_the_loss():
    host = cfp.Context(W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), [])
    runs = []
    for _ in range(2):
        net = cfp.UNet(host, seed=7)
        n, secs, tail = learned.train(net, seeds=[11, 12, 13, 14], sizes=(33,), lr=3e-4, lr_end=1e-4)
        runs.append((net.params(), tail))
        net.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1]
    net = cfp.UNet(host, seed=7)
    first = []
    p = learned.Problem(11, (33,))
    for r, e in p.pairs():
        first.append(net.train_step(p.ctx, r, e, 0.0, want_loss=True))  # lr 0: the initial loss
    p.close()
    assert np.mean(runs[0][1]) < np.mean(first), (np.mean(runs[0][1]), np.mean(first))
    net.close()
    host.close()


def test_trained_network_learns_the_error_and_the_flexible_solve_converges():
    """Trained on the smoothed pairs of 150 random geometries at 65^3, the
    network's correction (with the energy step of the cycle) reduces the
    error of every held-out smoothed residual, and by at least 5 % on
    average;
    the flexible GMRES with it converges on held-out 129^3 geometries with
    1-3 bodies to the same solution as a tight multigrid-preconditioned
    solve, and the per-step fallback keeps it within a quarter of GMRES
    with the red-black sweeps alone.  The iterations of the paper's method
    (BiCGSTAB with the same sweeps), of GMRES and of the flexible GMRES with
    the network are printed: what the network gains in the solve."""
    import time
    host = cfp.Context(W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), [])
    net = cfp.UNet(host, seed=5)
    n, secs, tail = learned.train(net, seeds=list(range(2000, 2150)), sizes=(65,))
    assert n == 150 * len(learned.PAIR_ITERS)
    # prediction on held-out pairs: |e - alpha y| / |e| with the cycle's step
    p = learned.Problem(9001, (65,))
    ratios = []
    for r, e in p.pairs():
        y = torch.zeros_like(r)
        net.apply(p.ctx, r, y)
        By = torch.zeros_like(r)
        p.ctx.apply(y, By)
        alpha = float((y * r).sum() / (y * By).sum())
        ratios.append(float((e - alpha * y).norm() / e.norm()))
    p.close()
    print("held-out error ratios", [round(q, 3) for q in ratios])
    assert max(ratios) < 1.0 and np.mean(ratios) < 0.95, ratios
    rows = []
    for seed in (9001, 9002):
        w = W.random_problem(seed, sizes=(129,))
        assert 1 <= len(w.bodies) <= 3
        ctx, t, f, g, gi = setup(w)
        ref = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        ctx.solve(f, g, gi, ref, tol=1e-13, precond=cfp.PRECOND_MG)
        out = {}
        for name in ("bicgstab", "gmres", "fgmres+net"):
            u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "bicgstab":
                info = ctx.solve(f, g, gi, u, tol=1e-10, precond=cfp.PRECOND_RBGS, sweeps=8)
            else:
                info = ctx.solve_fgmres(f, g, gi, u, tol=1e-10, net=net if name == "fgmres+net" else None, m=20,
                                        net_guess=name == "fgmres+net", precond=cfp.PRECOND_RBGS, sweeps=8)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            assert info.status == 0 and info.rel_residual <= 1e-10, (name, info.as_dict())
            diff = float((u - ref).abs().max() / ref.abs().max())
            assert diff <= 1e-7, (name, diff)
            out[name] = (info.iterations, info.refinements, round(dt, 3))
        rows.append(out)
        print("seed %d (iterations, steps with the network's direction, s): %s" % (seed, out))
        ctx.close()
    net.close()
    host.close()
    for out in rows:
        assert out["fgmres+net"][0] <= 1.25 * out["gmres"][0], rows
