"""Parity at the benchmark's full size: config 3 (513^3, ellipsoid + torus on
the tanh grid), through the C ABI, in the configuration bench.py times.

At this size the oracle can classify and locate the IBIs (a few seconds) but
not assemble the system (its CSR would need ~44 GB), so:
  - the point types and the IBI coordinates are compared with the oracle's
    over the whole grid, bit for bit;
  - the FP64 apply is compared on a seeded sample of regular rows with the
    27-term definition of the regular row (Eq. A27: Rx Ly Lz + Lx Ry Lz +
    Lx Ly Rz with the oracle's 1D coefficients of Eq. app_xxx), summed here
    in numpy;
  - every irregular row of B x (the modified stencils of Secs. 2.2-2.3, the
    degenerate operators included) and of the right-hand side, plus a seeded
    sample of regular and non-unknown rows, is compared element by element
    with the oracle's rows, which it builds one by one without assembling
    the system (cfo_rows);
  - the preconditioned solve is checked through what holds at any size: the
    mixed-precision solve with the multigrid V(5,3) preconditioner (the
    bench's) reaches a true relative residual of 1e-15 and the FP64 solve's
    max-norm error within 2 %."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pyoracle as O  # noqa: E402
from paper_1901_08269_gb300 import cfp  # noqa: E402
from paper_1901_08269_gb300 import workloads as W  # noqa: E402

N513 = 513


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    w = W.config3(N513)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
    ty = torch.empty(w.N, dtype=torch.uint8, device="cuda")
    ctx.classify_points(ty)
    xyz = ctx.ibi_points()
    yield w, ctx, ty, xyz
    ctx.close()


@pytest.fixture(scope="module")
def oracle(full):
    w = full[0]
    P = O.Problem(w.x, w.y, w.z, w.bodies)
    otype = P.classify()
    _, _, oxyz = P.ibi()
    return P, otype, oxyz


def test_full_size_classification_and_ibi_points_bit_exact(full, oracle):
    w, ctx, ty, xyz = full
    P, otype, oxyz = oracle
    assert ctx.n_irregular == P.n_irr and ctx.n_ibi == P.n_ibi
    np.testing.assert_array_equal(ty.cpu().numpy(), otype)
    np.testing.assert_array_equal(xyz.cpu().numpy(), oxyz)


def test_full_size_apply_on_sampled_regular_rows(full):
    w, ctx, ty, xyz = full
    nx, ny, nz = w.x.size, w.y.size, w.z.size
    gen = torch.Generator(device="cuda")
    gen.manual_seed(513)
    x = torch.randn(w.N, generator=gen, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ctx.apply(x, y)
    # seeded sample of regular rows (no solid node among the 26 neighbours)
    rng = np.random.default_rng(7)
    i = rng.integers(1, nx - 1, 6000)
    j = rng.integers(1, ny - 1, 6000)
    k = rng.integers(1, nz - 1, 6000)
    lin = (k * ny + j) * nx + i
    regular = ty[torch.as_tensor(lin, device="cuda")].cpu().numpy() == O.REGULAR
    i, j, k, lin = i[regular][:4000], j[regular][:4000], k[regular][:4000], lin[regular][:4000]
    assert lin.size == 4000
    coef = [O.compact_coefs(a) for a in (w.x, w.y, w.z)]  # a, c, ar, br, cr per axis

    def lr(d, idx):
        a, c, ar, br, cr = coef[d]
        L = np.stack([a[idx], np.ones(idx.size), c[idx]], axis=1)
        R = np.stack([ar[idx], br[idx], cr[idx]], axis=1)
        return L, R

    (Lx, Rx), (Ly, Ry), (Lz, Rz) = lr(0, i), lr(1, j), lr(2, k)
    offs = np.array([(o - 1) + (p - 1) * nx + (r - 1) * nx * ny for r in range(3) for p in range(3) for o in range(3)])
    xs = x[torch.as_tensor(lin[:, None] + offs[None, :], device="cuda")].cpu().numpy()  # (rows, 27)
    want = np.zeros(lin.size)
    scale = np.zeros(lin.size)
    q = 0
    for r in range(3):
        for p in range(3):
            for o in range(3):
                wgt = (Rx[:, o] * Ly[:, p] * Lz[:, r] + Lx[:, o] * Ry[:, p] * Lz[:, r] + Lx[:, o] * Ly[:, p] * Rz[:, r])
                want += wgt * xs[:, q]
                scale += np.abs(wgt * xs[:, q])
                q += 1
    got = y[torch.as_tensor(lin, device="cuda")].cpu().numpy()
    err = np.abs(got - want) / scale
    assert np.max(err) <= 1e-13, np.max(err)


def _rows_under_test(otype, seed):
    """Every irregular row plus a seeded sample of 20000 other nodes (regular,
    solid and box rows)."""
    rng = np.random.default_rng(seed)
    irr = np.flatnonzero(otype == O.IRREGULAR)
    return np.concatenate([irr, rng.integers(0, otype.size, 20000)]), irr.size


def test_full_size_irregular_rows_of_the_apply(full, oracle):
    w, ctx, ty, xyz = full
    P, otype, oxyz = oracle
    rows, n_irr = _rows_under_test(otype, 17)
    assert n_irr == ctx.n_irregular and n_irr > 300000
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5130)
    x = torch.randn(w.N, generator=gen, dtype=torch.float64, device="cuda")
    x[ty == O.SOLID] = 0.0  # box values stay: the rows next to the box read them
    y = torch.empty_like(x)
    ctx.apply(x, y)
    bx, ba, _, ndeg = P.rows(rows, x=x.cpu().numpy())
    assert ndeg > 0  # the degenerate operators of this geometry are among the rows
    got = y[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    err = np.abs(got - bx)
    # the bar of the small parity cases: an irregular row is the regular row
    # plus merged corrections, rounding bounded by 1e-12 |B||x|
    assert np.all(err <= 1e-12 * ba + 1e-300), np.max(err / (ba + 1e-300))
    assert np.all(got[otype[rows] == O.SOLID] == 0.0)


def test_full_size_rhs_rows(full, oracle):
    w, ctx, ty, xyz = full
    P, otype, oxyz = oracle
    rows, _ = _rows_under_test(otype, 18)
    f, g = w.fields(torch, "cuda")
    gi = w.g_at(xyz, torch).contiguous()
    rhs = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    ctx.assemble_rhs(f, g, gi, rhs)
    X, Y, Z = w.mesh(torch, "cuda")
    u = w.u(X, Y, Z, torch).reshape(-1)
    u[ty == O.SOLID] = 0.0
    del X, Y, Z
    # the same g at the IBI points on both sides (the coordinates are
    # bit-equal; the values are evaluated once, on the device)
    _, ba, ro, _ = P.rows(rows, x=u.cpu().numpy(), f=f.cpu().numpy(), g_nodes=g.cpu().numpy(),
                          g_ibi=gi.cpu().numpy())
    got = rhs[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    scale = ba + np.abs(ro) + 1.0  # the bar of the small parity cases
    err = np.abs(got - ro)
    assert np.all(err <= 1e-12 * scale), np.max(err / scale)


def test_full_size_mixed_multigrid_solve_reaches_fp64_error(full):
    w, ctx, ty, xyz = full
    f, g = w.fields(torch, "cuda")
    gi = w.g_at(xyz, torch)
    X, Y, Z = w.mesh(torch, "cuda")
    ue = w.u(X, Y, Z, torch).reshape(-1)
    fluid = ty != O.SOLID
    errs = {}
    for name, prec in (("fp64", cfp.PREC_FP64), ("mixed", cfp.PREC_MIXED)):
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        info = ctx.solve(f, g, gi, u, tol=1e-15, precision=prec, precond=cfp.PRECOND_MG, mg_smooth=5,
                         mg_post=3, inner_tol=3e-3)
        assert info.status == 0 and info.rel_residual <= 1e-15, (name, info.as_dict())
        errs[name] = float((u - ue)[fluid].abs().max())
    # fourth-order scheme at 513^3 on this geometry: E* of a few 1e-9
    assert 1e-10 < errs["fp64"] < 1e-8, errs
    assert errs["mixed"] <= 1.02 * errs["fp64"], errs
