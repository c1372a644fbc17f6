"""Batched solves (many uneven random problems at once) and the autotuner,
through the C ABI.  A batched result must be bitwise the lone solve's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pyoracle as O  # noqa: E402
from paper_1901_08269_gb300 import cfp  # noqa: E402
from paper_1901_08269_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _problems(seeds):
    out = []
    for s in seeds:
        w = W.random_problem(s, sizes=(33, 41, 49))
        ctx = cfp.Context(w.x, w.y, w.z, w.bodies, stream=torch.cuda.Stream())
        ctx.classify_points()
        xyz = ctx.ibi_points()
        f, g = w.fields(torch, "cuda")
        gi = w.g_at(xyz, torch).contiguous() if ctx.n_ibi else None
        out.append((w, ctx, f, g, gi))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precision", [cfp.PREC_FP64, cfp.PREC_MIXED])
def test_batch_equals_lone_solves(precision):
    probs = _problems(range(100, 106))
    opts = dict(precision=precision, precond=cfp.PRECOND_MG)
    lone = []
    for w, ctx, f, g, gi in probs:
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        info = ctx.solve(f, g, gi, u, tol=1e-12, **opts)
        assert info.status == 0
        lone.append(u)
    us = [torch.full((w.N,), 0.0, dtype=torch.float64, device="cuda") for w, *_ in probs]
    torch.cuda.synchronize()
    infos = cfp.solve_batch([p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs],
                            [p[4] for p in probs], us, tol=1e-12, nthreads=4, **opts)
    torch.cuda.synchronize()
    for u, ul, info in zip(us, lone, infos):
        assert info.status == 0
        assert torch.equal(u, ul)


def test_batch_member_matches_oracle():
    probs = _problems([7])
    w, ctx, f, g, gi = probs[0]
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    cfp.solve_batch([ctx], [f], [g], [gi], [u], tol=1e-13, precond=cfp.PRECOND_MG)
    P = O.Problem(w.x, w.y, w.z, w.bodies)
    P.classify()
    key, t, xyz = P.ibi()
    fo, go = w.fields()
    uo, st, it, rel = P.solve(fo, go, w.g_at(xyz), tol=1e-13)
    assert st == 0
    scale = max(np.max(np.abs(uo)), 1e-300)
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-10 * scale


def test_batch_rejects_repeated_context():
    probs = _problems([3])
    w, ctx, f, g, gi = probs[0]
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    with pytest.raises(cfp.CfpError) as e:
        cfp.solve_batch([ctx, ctx], [f, f], [g, g], [gi, gi], [u, u])
    assert e.value.status == cfp.EINVAL


def test_autotune_picks_a_converging_setting():
    probs = _problems([11])
    w, ctx, f, g, gi = probs[0]
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    o, ms = ctx.autotune(f, g, gi, u, tol=1e-12, precision=cfp.PREC_MIXED)
    assert o.precond == cfp.PRECOND_MG and o.mg_smooth in (1, 2, 3) and o.inner_tol in (1e-2, 1e-3, 1e-4)
    assert ms > 0
    u.zero_()
    info = ctx.solve(f, g, gi, u, tol=1e-12, opts=o)
    assert info.status == 0


# ----------------------------------------------- the batch as one graph launch
def _lone(probs, opts, tol):
    out = []
    for w, ctx, f, g, gi in probs:
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        info = ctx.solve(f, g, gi, u, tol=tol, opts=opts)
        assert info.status == 0
        out.append((u, info))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("precond", [cfp.PRECOND_MG, cfp.PRECOND_RBGS])
def test_graph_batch_is_bitwise_the_lone_solves(precond):
    # uneven sizes and bodies; every refinement decision taken on the device
    probs = _problems(range(100, 106))
    opts = cfp.default_opts(precision=cfp.PREC_MIXED, precond=precond, inner_tol=1e-3)
    lone = _lone(probs, opts, 1e-12)
    us = [torch.zeros(w.N, dtype=torch.float64, device="cuda") for w, *_ in probs]
    b = cfp.Batch([p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs], [p[4] for p in probs], us,
                  tol=1e-12, opts=opts)
    infos = b.run()
    for u, (ul, il), info in zip(us, lone, infos):
        assert info.status == 0
        assert (info.iterations, info.refinements) == (il.iterations, il.refinements)
        assert info.rel_residual == il.rel_residual
        assert torch.equal(u, ul)
        assert info.launches > 0
    # a second run: the same graph on new data (the source scaled and shifted)
    for p in probs:
        p[2].mul_(0.5).add_(0.25)
    lone2 = _lone(probs, opts, 1e-12)
    for u in us:
        u.zero_()
    infos = b.run()
    for u, (ul, il), info in zip(us, lone2, infos):
        assert info.status == 0 and info.iterations == il.iterations
        assert torch.equal(u, ul)
    b.close()


def test_graph_batch_recaptures_after_a_reclassification():
    probs = _problems([7, 11, 3])
    opts = cfp.default_opts(precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG)
    us = [torch.zeros(w.N, dtype=torch.float64, device="cuda") for w, *_ in probs]
    b = cfp.Batch([p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs], [p[4] for p in probs], us,
                  tol=1e-12, opts=opts)
    b.run()
    probs[1][1].classify_points()  # frees and rebuilds its side data and hierarchy
    for u in us:
        u.zero_()
    infos = b.run()
    lone = _lone(probs, opts, 1e-12)
    for u, (ul, il), info in zip(us, lone, infos):
        assert info.status == 0
        assert torch.equal(u, ul)
    b.close()


def test_graph_batch_reports_a_failing_member_and_solves_the_others():
    probs = _problems([100, 101])
    good = cfp.default_opts(precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG)
    bad = cfp.default_opts(precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG, max_refine=1)
    us = [torch.zeros(w.N, dtype=torch.float64, device="cuda") for w, *_ in probs]
    b = cfp.Batch([p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs], [p[4] for p in probs], us,
                  tol=1e-13, opts=[good, bad])
    infos = b.run(check=False)
    assert infos[0].status == 0
    assert infos[1].status == cfp.ENOCONV and infos[1].refinements == 1
    with pytest.raises(cfp.CfpError) as e:
        b.run()
    assert e.value.status == cfp.ENOCONV and "problem 1" in str(e.value)
    (ul, il), = _lone(probs[:1], good, 1e-13)
    assert torch.equal(us[0], ul)
    b.close()


def test_graph_batch_rejects_fp64_and_repeated_contexts():
    probs = _problems([3])
    w, ctx, f, g, gi = probs[0]
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    with pytest.raises(cfp.CfpError) as e:
        cfp.Batch([ctx], [f], [g], [gi], [u], opts=cfp.default_opts(precision=cfp.PREC_FP64))
    assert e.value.status == cfp.EINVAL
    with pytest.raises(cfp.CfpError) as e:
        cfp.Batch([ctx, ctx], [f, f], [g, g], [gi, gi], [u, u], opts=cfp.default_opts(precision=cfp.PREC_MIXED))
    assert e.value.status == cfp.EINVAL
