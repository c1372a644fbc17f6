"""The multigrid preconditioner (CFP_PRECOND_MG) against a plain numpy
V-cycle written from its definition.

The V-cycle is not the paper's (Sec. 3.3 uses a fixed number of red-black
Gauss-Seidel inner iterations on K); it is this library's alternative
approximate solve of the same system K phi = rho.  The definition checked
here, step by step on whole arrays in natural node order:

  levels      n_c = (n + 2) // 2 per axis while every axis of the finer level
              has >= 17 nodes; coarse node I sits on fine node min(2I, n - 1)
  types       injected from the fine node (irregular becomes regular)
  K           the fine level's K is the oracle's (Eq. A7 and the
              Shortley-Weller rows); a coarse K is the 7-point operator of
              the coarse coordinates (Eq. 2ndorder_coef), unknowns only
  smoother    red-black Gauss-Seidel (red = even i + j + k), red first
  transfers   P: piecewise-linear interpolation in the coordinates per axis,
              tensor product; restriction (P^T r) / (P^T 1)
  cycle       nu sweeps from zero, residual, restriction; 16 sweeps from zero
              on the coarsest level; prolongation added, post sweeps
              (mg_smooth = nu, mg_post = post)

The CUDA path stores colours in separate arrays and skips the black
residuals and the red prolongation (both exact for red-black smoothing), so
the two agree to rounding."""
import numpy as np
import pytest
import scipy.sparse as sp

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


def second_difference(X):
    n = len(X)
    rows, cols, vals = [], [], []
    for i in range(1, n - 1):
        f, b = X[i + 1] - X[i], X[i] - X[i - 1]
        for c, v in ((i - 1, 2.0 / (b * (f + b))), (i, -2.0 / (b * f)), (i + 1, 2.0 / (f * (f + b)))):
            rows.append(i)
            cols.append(c)
            vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def interpolation(Xf, Xc, n):
    """P (n_f x n_c): fine node i from the two coarse nodes around it."""
    nc = len(Xc)
    fine_of = np.minimum(2 * np.arange(nc), n - 1)
    P = np.zeros((n, nc))
    for I in range(nc - 1):
        a, b = fine_of[I], fine_of[I + 1]
        for i in range(a, b + 1):
            t = (Xf[i] - Xf[a]) / (Xf[b] - Xf[a])
            P[i, I] = 1.0 - t
            P[i, I + 1] = t
    return sp.csr_matrix(P)


def build_levels(x, y, z, otype, K0):
    n = (len(x), len(y), len(z))
    levels = [dict(n=n, X=[np.asarray(x), np.asarray(y), np.asarray(z)], type=otype, K=K0)]
    while min(levels[-1]["n"]) >= 17:
        F = levels[-1]
        nc = tuple((m + 2) // 2 for m in F["n"])
        idx = [np.minimum(2 * np.arange(nc[d]), F["n"][d] - 1) for d in range(3)]
        Xc = [F["X"][d][idx[d]] for d in range(3)]
        t3 = F["type"].reshape(F["n"][2], F["n"][1], F["n"][0])
        tc = t3[np.ix_(idx[2], idx[1], idx[0])].reshape(-1).copy()
        tc[tc == O.IRREGULAR] = O.REGULAR
        Ix, Iy, Iz = (sp.identity(m, format="csr") for m in nc)
        K3 = (sp.kron(Iz, sp.kron(Iy, second_difference(Xc[0]))) + sp.kron(Iz, sp.kron(second_difference(Xc[1]), Ix)) +
              sp.kron(second_difference(Xc[2]), sp.kron(Iy, Ix)))
        M = sp.diags(((tc == O.REGULAR) | (tc == O.IRREGULAR)).astype(float))
        F["P"] = sp.kron(interpolation(F["X"][2], Xc[2], F["n"][2]),
                         sp.kron(interpolation(F["X"][1], Xc[1], F["n"][1]),
                                 interpolation(F["X"][0], Xc[0], F["n"][0]))).tocsr()
        levels.append(dict(n=nc, X=Xc, type=tc, K=(M @ K3 @ M).tocsr()))
    for L in levels:
        nx, ny, nz = L["n"]
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        unk = ((L["type"] == O.REGULAR) | (L["type"] == O.IRREGULAR))
        red = ((i + j + k) % 2 == 0).reshape(-1)
        L["colour"] = [unk & red, unk & ~red]
        L["unk"] = unk
        L["diag"] = L["K"].diagonal()
    return levels


def sweep(L, b, e):
    for m in L["colour"]:
        off = L["K"] @ e - L["diag"] * e
        e[m] = (b[m] - off[m]) / L["diag"][m]


def vcycle(levels, rho, nu, l=0, post=None):
    post = nu if post is None else post
    L = levels[l]
    e = np.zeros(len(rho))
    if l == len(levels) - 1:
        for _ in range(16):
            sweep(L, rho, e)
        return e
    for _ in range(nu):
        sweep(L, rho, e)
    r = np.where(L["unk"], rho - L["K"] @ e, 0.0)
    P = L["P"]
    C = levels[l + 1]
    bc = np.where(C["unk"], (P.T @ r) / (P.T @ np.ones(len(r))), 0.0)
    e += np.where(L["unk"], P @ vcycle(levels, bc, nu, l + 1, post), 0.0)
    for _ in range(post):
        sweep(L, rho, e)
    return e


def ragged(n=41):
    return (W.tanh_grid(-1, 1, n, 1.1), W.tanh_grid(-1, 1, n + 12, 0.7), W.uniform_grid(-1, 1, n - 6))


CASES = {
    "c2-33": lambda: W.config2(33),
    "ragged-torus": lambda: W.Workload("ragged-torus", *ragged(),
                                       [W.torus((0.02, 0.01, -0.03), 0.45, 0.16, W.rot_euler(0.1, 0.5, 0.3))],
                                       W._c3_u, W._c3_f),
    "interior-sphere": lambda: W.interior_sphere(41),
    "even-48": lambda: W.Workload("even", W.tanh_grid(-1, 1, 48, 1.2), W.uniform_grid(-1, 1, 34),
                                  W.tanh_grid(-1, 1, 40, 0.8), [W.sphere((0.04, -0.02, 0.03), 0.35)],
                                  W._c2_u, W._c2_f),
    "tiny-one-level": lambda: W.Workload("tiny", W.uniform_grid(-1, 1, 8), W.uniform_grid(-1, 1, 11),
                                         W.uniform_grid(-1, 1, 9), [W.sphere((0.1, 0.0, 0.05), 0.4)],
                                         W._c2_u, W._c2_f),
}


@pytest.mark.parametrize("nu,post", [(1, 1), (2, 2), (3, 3), (2, 1), (1, 3)])
@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_matches_definition(name, nu, post):
    w = CASES[name]()
    P = O.Problem(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    otype = P.classify()
    P.ibi()
    P.assemble()
    levels = build_levels(w.x, w.y, w.z, otype, P.export(O.MAT_K))
    if name == "tiny-one-level":
        assert len(levels) == 1
    else:
        assert len(levels) >= 3
    rng = np.random.default_rng(11 + nu)
    rho = np.where(levels[0]["unk"], rng.standard_normal(w.N), 0.0)
    want = vcycle(levels, rho, nu, post=post)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    ctx.classify_points()
    phi = torch.full((w.N,), 7.0, dtype=torch.float64, device="cuda")  # overwritten: zeroed, then the V-cycle
    opts = dict(precond=cfp.PRECOND_MG, mg_smooth=nu, mg_post=post)
    ctx.precondition_ex(torch.as_tensor(rho, device="cuda"), phi, **opts)
    got = phi.cpu().numpy()
    u = levels[0]["unk"]
    assert np.all(got[~u] == 0.0)
    err = np.max(np.abs(got[u] - want[u])) / np.max(np.abs(want[u]))
    assert err <= 1e-12, err
    # a second call reuses the level vectors: nothing stale may leak in
    phi2 = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    ctx.precondition_ex(torch.as_tensor(rho, device="cuda"), phi2, **opts)
    assert torch.equal(phi, phi2)
    ctx.close()


# levels of >= 192 nodes per row run their FP32 half-sweeps through the
# TMA-fed kernel: one x tile (257), a ragged second x tile with an even row
# (300), two such levels (513, then 257); ragged y tiles and z chunks in all
WIDE = {
    "wide-257": lambda: W.Workload("wide-257", W.tanh_grid(-1, 1, 257, 1.1), W.uniform_grid(-1, 1, 27),
                                   W.tanh_grid(-1, 1, 45, 0.8), [W.sphere((0.03, -0.02, 0.01), 0.4)],
                                   W._c2_u, W._c2_f),
    "wide-300": lambda: W.Workload("wide-300", W.uniform_grid(-1, 1, 300), W.tanh_grid(-1, 1, 21, 0.6),
                                   W.uniform_grid(-1, 1, 70), [W.sphere((-0.05, 0.02, 0.04), 0.42)],
                                   W._c2_u, W._c2_f),
    "wide-513": lambda: W.Workload("wide-513", W.tanh_grid(-1, 1, 513, 1.4), W.uniform_grid(-1, 1, 18),
                                   W.uniform_grid(-1, 1, 18), [W.sphere((0.01, 0.02, -0.03), 0.45)],
                                   W._c2_u, W._c2_f),
}


@pytest.mark.parametrize("nu,post", [(2, 2), (4, 3)])
@pytest.mark.parametrize("name", list(WIDE))
def test_fp32_vcycle_tma_smoother(name, nu, post):
    """The FP32 V-cycle (the mixed solve's inner preconditioner) with the
    TMA-fed half-sweeps (mg_tma 1), and with the fused black-then-red passes
    as well (mg_tma 2: nu - 1 before the coarse correction, post - 1 after
    it, on every level of >= 192 nodes per row, the fine level's
    Shortley-Weller rows inside the pass): bitwise equal to the plain-load
    half-sweeps (same arithmetic), and the numpy V-cycle in FP64 to FP32
    accuracy."""
    w = WIDE[name]()
    P = O.Problem(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    otype = P.classify()
    P.ibi()
    P.assemble()
    levels = build_levels(w.x, w.y, w.z, otype, P.export(O.MAT_K))
    rng = np.random.default_rng(5)
    rho = np.where(levels[0]["unk"], rng.standard_normal(w.N), 0.0)
    want = vcycle(levels, rho, nu, post=post)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    ctx.classify_points()
    rho_t = torch.as_tensor(rho, device="cuda")
    got = {}
    for tma in (1, 0, 2, 1, 2):
        phi = torch.full((w.N,), 7.0, dtype=torch.float64, device="cuda")
        ctx.precondition_ex(rho_t, phi, precond=cfp.PRECOND_MG, mg_smooth=nu, mg_post=post,
                            precision=cfp.PREC_MIXED, mg_tma=tma)
        if tma in got:
            assert torch.equal(phi, got[tma])  # repeatable
        got[tma] = phi
    assert torch.equal(got[1], got[0])
    assert torch.equal(got[2], got[0])
    g = got[1].cpu().numpy()
    u = levels[0]["unk"]
    assert np.all(g[~u] == 0.0)
    err = np.max(np.abs(g[u] - want[u])) / np.max(np.abs(want[u]))
    assert err <= 1e-5, err
    ctx.close()


@pytest.mark.parametrize("name", list(WIDE))
def test_fp32_rbgs_fused_passes(name):
    """The red-black preconditioner in FP32 with the fused passes (mg_tma 2;
    8 sweeps on the fine level: the first red half-sweep, seven fused
    black-then-red passes, the last black half-sweep) bitwise equal to the
    same sweeps as one launch per half-sweep, TMA-fed or plain, and within
    FP32 rounding of the FP64 sweeps."""
    w = WIDE[name]()
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    types = torch.empty(w.N, dtype=torch.uint8, device="cuda")
    ctx.classify_points(types)
    unk = (types == cfp.REGULAR) | (types == cfp.IRREGULAR)
    rng = np.random.default_rng(9)
    rho_t = torch.as_tensor(rng.standard_normal(w.N), device="cuda") * unk
    got = {}
    for tma in (2, 0, 1):
        phi = torch.full((w.N,), 7.0, dtype=torch.float64, device="cuda")
        ctx.precondition_ex(rho_t, phi, precond=cfp.PRECOND_RBGS, sweeps=8, precision=cfp.PREC_MIXED, mg_tma=tma)
        got[tma] = phi
    assert torch.equal(got[2], got[0]) and torch.equal(got[1], got[0])
    ref = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    ctx.precondition_ex(rho_t, ref, precond=cfp.PRECOND_RBGS, sweeps=8, precision=cfp.PREC_FP64)
    err = (got[1] - ref).abs().max().item() / ref.abs().max().item()
    assert err <= 1e-5, err
    ctx.close()


def test_mixed_solve_with_fused_passes_is_bitwise_the_default():
    """The whole mixed solve (graph-captured V-cycles, refinement) with the
    fused black-then-red passes gives the default solve's bits."""
    w = WIDE["wide-300"]()
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
    ctx.classify_points()
    f, g = w.fields(torch, "cuda")
    gi = w.g_at(ctx.ibi_points(), torch)
    out = {}
    for tma in (1, 2):
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        info = ctx.solve(f, g, gi, u, tol=1e-12, precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG,
                         mg_smooth=4, mg_post=3, mg_tma=tma)
        assert info.status == 0 and info.rel_residual <= 1e-12
        out[tma] = (u, info.iterations, info.refinements)
    assert torch.equal(out[1][0], out[2][0]) and out[1][1:] == out[2][1:]
    ctx.close()


def test_kernel_timer_covers_every_kernel():
    w = W.config2(33)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
    ctx.classify_points()
    nint = 31 ** 3
    for prec, size in ((cfp.PREC_FP64, 8), (cfp.PREC_MIXED, 4)):
        for kid, per in ((cfp.KERNEL_APPLY, 3.0 * nint * size), (cfp.KERNEL_RBGS, 1.5 * nint * size),
                         (cfp.KERNEL_MG_SWEEP, 1.5 * nint * size), (cfp.KERNEL_UPDATE, 8.0 * w.N * size),
                         (cfp.KERNEL_PROLONG, (0.5 * (1 + 2 * size) + size / 8) * nint),
                         (cfp.KERNEL_RESTRICT, (0.5 * size + (1 + size) / 8) * nint)):
            ms, by = ctx.time_kernel(kid, prec, reps=2)
            assert ms > 0.0 and by == per
    with pytest.raises(cfp.CfpError):
        ctx.time_kernel(7, cfp.PREC_FP64, reps=1)
    # the fused pass needs a fine level of >= 192 nodes per row, in FP32
    for prec in (cfp.PREC_MIXED, cfp.PREC_FP64):
        with pytest.raises(cfp.CfpError) as e:
            ctx.time_kernel(cfp.KERNEL_MG_PAIR, prec, reps=1)
        assert e.value.status == cfp.EINVAL
    ctx.close()
    wide = WIDE["wide-257"]()
    wc = cfp.Context(wide.x, wide.y, wide.z, wide.bodies, wide.fluid_inside)
    wc.classify_points()
    ms, by = wc.time_kernel(cfp.KERNEL_MG_PAIR, cfp.PREC_MIXED, reps=2)
    assert ms > 0.0 and by == 2.5 * 4 * (len(wide.x) - 2) * (len(wide.y) - 2) * (len(wide.z) - 2)
    wc.close()
    # a grid with a single multigrid level has no transfer to time
    x = W.uniform_grid(0, 1, 9)
    small = cfp.Context(x, x, x, [])
    small.classify_points()
    with pytest.raises(cfp.CfpError) as e:
        small.time_kernel(cfp.KERNEL_PROLONG, cfp.PREC_MIXED, reps=1)
    assert e.value.status == cfp.EINVAL
    small.close()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The pipeline waits of the TMA-fed smoother are bounded: a wait on an
    mbarrier phase that nothing completes gives up after one second, the call
    reports CFP_ECUDA with the recorded code, the wait word is cleared, and
    the same context then solves normally."""
    import time
    w = W.config2(33)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
    ctx.classify_points()
    t0 = time.perf_counter()
    st, msg = ctx.diag_bounded_wait()
    dt = time.perf_counter() - t0
    assert st == cfp.ECUDA and "code 5" in msg, (st, msg)
    assert 0.9 <= dt < 30.0, dt
    f, g = w.fields(torch, "cuda")
    gi = w.g_at(ctx.ibi_points(), torch)
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    info = ctx.solve(f, g, gi, u, tol=1e-10, precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG)
    assert info.status == 0 and info.rel_residual <= 1e-10
    ctx.close()
