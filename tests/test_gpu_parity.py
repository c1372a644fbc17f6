"""GPU path versus the CPU oracle, through the C ABI.

Bars: classification and IBI order bit-exact; IBI coordinates and the
operators within rounding (scaled by the sum of absolute terms); FP64
solutions within 1e-10 relative max-norm; fourth-order convergence; the
mixed-precision solve reaching the FP64 discretisation error."""
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


def ragged(n=37):
    # deliberately uneven sizes: several apply tiles plus a ragged tail in x,
    # y and z chunks
    return (W.tanh_grid(-1, 1, n, 1.1), W.tanh_grid(-1, 1, n + 12, 0.7), W.uniform_grid(-1, 1, n - 6))


CASES = {
    "c1-17": lambda: W.config1(17),
    "c2-33": lambda: W.config2(33),
    "ragged-sphere": lambda: W.Workload("ragged", *ragged(), [W.sphere((0.05, -0.03, 0.02), 0.33)], W._c2_u, W._c2_f),
    "ragged-torus": lambda: W.Workload("ragged-torus", *ragged(41),
                                       [W.torus((0.02, 0.01, -0.03), 0.45, 0.16, W.rot_euler(0.1, 0.5, 0.3))],
                                       W._c3_u, W._c3_f),
    "c3-bodies-65": lambda: W.Workload("c3b", W.tanh_grid(-1, 1, 65, 1.0), W.tanh_grid(-1, 1, 65, 0.6),
                                       W.tanh_grid(-1, 1, 65, 0.6), W.config3_bodies(), W._c3_u, W._c3_f),
    "random-3": lambda: W.random_problem(3, sizes=(33, 49)),
    "interior-sphere": lambda: W.interior_sphere(41),
    "random-8": lambda: W.random_problem(8, sizes=(33, 49)),
    # even sizes, n_x / 2 a multiple of 8: rows of the red/black split arrays
    # without padding (the speculative x+ load of a row's last pair reads the
    # next row)
    "even-48": lambda: W.Workload("even", W.tanh_grid(-1, 1, 48, 1.2), W.uniform_grid(-1, 1, 34),
                                  W.tanh_grid(-1, 1, 40, 0.8), [W.sphere((0.04, -0.02, 0.03), 0.35)],
                                  W._c2_u, W._c2_f),
}


class Pair:
    def __init__(self, w):
        self.w = w
        self.ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
        self.type = torch.empty(w.N, dtype=torch.uint8, device="cuda")
        self.ctx.classify_points(self.type)
        self.xyz = self.ctx.ibi_points()
        self.P = O.Problem(w.x, w.y, w.z, w.bodies, w.fluid_inside)
        self.otype = self.P.classify()
        self.okey, self.ot, self.oxyz = self.P.ibi()
        self.P.assemble()
        self.unk = np.flatnonzero((self.otype == O.REGULAR) | (self.otype == O.IRREGULAR))

    def rand_field(self, seed, zero_off=True):
        rng = np.random.default_rng(seed)
        x = rng.standard_normal(self.w.N)
        if zero_off:
            m = np.zeros(self.w.N, bool)
            m[self.unk] = True
            x[~m] = 0.0
        else:
            x[self.otype == O.SOLID] = 0.0
        return x


_pairs = {}


def pair(name):
    if name not in _pairs:
        _pairs[name] = Pair(CASES[name]())
    return _pairs[name]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_classification_bit_exact(name):
    p = pair(name)
    np.testing.assert_array_equal(p.type.cpu().numpy(), p.otype)
    assert p.ctx.n_irregular == p.P.n_irr and p.ctx.n_ibi == p.P.n_ibi


@pytest.mark.parametrize("name", list(CASES))
def test_ibi_points(name):
    p = pair(name)
    g = p.xyz.cpu().numpy()
    assert g.shape == p.oxyz.shape
    # same bisection on bit-identical level-set values: equal coordinates
    np.testing.assert_array_equal(g, p.oxyz)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("zero_off", [True, False])
def test_apply_parity(name, zero_off):
    p = pair(name)
    x = p.rand_field(1, zero_off)
    y = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    p.ctx.apply(dev(x), y)
    yo = p.P.apply_B(x)
    scale = p.P.apply_B(x, absval=True)
    err = np.abs(y.cpu().numpy() - yo)
    # The GPU forms an irregular row as the regular 27-point row plus the
    # merged corrections of its modified lines (the split of Eq. Bdec), whose
    # intermediate terms can exceed the merged coefficients behind |B||x|:
    # rounding relative to |B||x| is bounded by 1e-12 rather than 1e-13.
    assert np.all(err <= 1e-12 * scale + 1e-300), np.max(err / (scale + 1e-300))
    nonunk = np.ones(p.w.N, bool)
    nonunk[p.unk] = False
    assert np.all(y.cpu().numpy()[nonunk] == 0.0)


# FP32 apply kernels and tile shapes (kernel, rows, planes per z chunk): the
# streaming kernel in both row counts and the bulk-copy ring in every depth
SHAPES_F32 = [(cfp.APPLY_STREAM, 2, 64), (cfp.APPLY_STREAM, 4, 16), (cfp.APPLY_RING, 2, 32),
              (cfp.APPLY_RING, 2, 64)]


# grids around the ring's span limit (rows of up to 514 nodes are copied as
# whole-plane spans, wider ones row by row)
WIDE = {
    "span-514": lambda: W.Workload("span-514", W.uniform_grid(-1, 1, 514), W.tanh_grid(-1, 1, 15, 0.5),
                                   W.uniform_grid(-1, 1, 12), [W.sphere((0.1, 0.02, -0.03), 0.4)], W._c2_u, W._c2_f),
    "rows-530": lambda: W.Workload("rows-530", W.tanh_grid(-1, 1, 530, 0.6), W.tanh_grid(-1, 1, 14, 0.5),
                                   W.uniform_grid(-1, 1, 11), [W.sphere((-0.05, 0.0, 0.04), 0.35)], W._c2_u, W._c2_f),
}


def _apply_f32_case(p):
    x = p.rand_field(2, zero_off=False).astype(np.float32)
    x64 = x.astype(np.float64)
    yo = p.P.apply_B(x64)
    scale = p.P.apply_B(x64, absval=True)
    xd = torch.as_tensor(x, device="cuda")
    outs = []
    for kernel, rows, planes in SHAPES_F32:
        p.ctx.tune_apply(cfp.PREC_MIXED, rows, planes, kernel=kernel)
        y = torch.full((p.w.N,), float("nan"), dtype=torch.float32, device="cuda")
        p.ctx.apply_f32(xd, y)
        outs.append(y)
    p.ctx.tune_apply(cfp.PREC_MIXED, 2, 64, kernel=cfp.APPLY_STREAM)
    y = outs[0].double().cpu().numpy()
    err = np.abs(y - yo)
    reg = p.otype == O.REGULAR
    irr = p.otype == O.IRREGULAR
    assert np.all(err[reg] <= 64 * 2.0 ** -24 * scale[reg] + 1e-30), np.max(err[reg] / (scale[reg] + 1e-30))
    assert np.all(err[irr] <= 2.0 ** 29 * 1e-12 * scale[irr] + 1e-30), np.max(err[irr] / (scale[irr] + 1e-30))
    nonunk = np.ones(p.w.N, bool)
    nonunk[p.unk] = False
    assert np.all(y[nonunk] == 0.0)
    for shape, o in zip(SHAPES_F32[1:], outs[1:]):
        assert torch.equal(o, outs[0]), shape


@pytest.mark.parametrize("name", list(CASES))
def test_apply_f32_parity_and_tile_shapes(name):
    """The FP32 apply of the mixed solve's inner iterations against the FP64
    oracle on the same FP32 input.  Regular rows: the rounding of the 1D
    metrics to FP32 and of the FP32 sum-factorised arithmetic are a few units
    of 2^-24 relative to |B||x|, bounded here by 64 * 2^-24.  Irregular rows
    carry the split form's larger intermediate terms (the FP64 test's 1e-12
    bar), scaled here from 2^-53 to 2^-24.  Every kernel and tile shape gives
    the same bits: each row is the same chain of fused multiply-adds."""
    _apply_f32_case(pair(name))


@pytest.mark.parametrize("name", list(WIDE))
def test_apply_f32_ring_copy_patterns(name):
    """The same on grids at and beyond the width the ring copies as
    whole-plane spans (514 nodes per row): its row-by-row copies and ragged
    second column tile."""
    _apply_f32_case(Pair(WIDE[name]()))


@pytest.mark.parametrize("name", ["c2-33", "ragged-torus", "random-3"])
@pytest.mark.parametrize("sweeps", [0, 1, 8])
def test_preconditioner_parity(name, sweeps):
    p = pair(name)
    rho = p.rand_field(2)
    phi = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    p.ctx.precondition(dev(rho), phi, sweeps)
    po = p.P.precond(rho, sweeps)
    err = np.max(np.abs(phi.cpu().numpy() - po))
    assert err <= 1e-12 * np.max(np.abs(po)), err


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_parity(name):
    p = pair(name)
    f, g = p.w.fields()
    gi = p.w.g_at(p.oxyz)
    rhs = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    p.ctx.assemble_rhs(dev(f), dev(g), dev(gi), rhs)
    ro = p.P.rhs(f, g, gi)
    X, Y, Z = p.w.mesh()
    u = p.w.u(X, Y, Z, np).reshape(-1)
    u[p.otype == O.SOLID] = 0.0
    scale = p.P.apply_B(u, absval=True) + np.abs(ro) + 1.0
    err = np.abs(rhs.cpu().numpy() - ro)
    assert np.all(err <= 1e-12 * scale), np.max(err / scale)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("graph", [1, 0])
def test_solve_parity_fp64(name, graph):
    p = pair(name)
    f, g = p.w.fields()
    gi = p.w.g_at(p.oxyz)
    tol = 1e-13
    uo, st, it, rel = p.P.solve(f, g, gi, tol=tol)
    assert st == 0
    u = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    info = p.ctx.solve(dev(f), dev(g), dev(gi), u, tol=tol, use_graph=graph)
    assert info.status == 0 and info.rel_residual <= tol
    ug = u.cpu().numpy()
    assert np.max(np.abs(ug - uo)) <= 1e-10 * np.max(np.abs(uo))
    assert np.all(ug[p.otype == O.SOLID] == 0.0)
    bd = p.otype == O.BOUNDARY
    np.testing.assert_array_equal(ug[bd], g[bd])
    assert abs(info.iterations - it) <= max(3, it // 5)


def test_solve_fourth_order_gpu():
    errs, ns = [], (33, 65, 129)
    for n in ns:
        w = W.config2(n)
        ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
        t = torch.empty(w.N, dtype=torch.uint8, device="cuda")
        ctx.classify_points(t)
        xyz = ctx.ibi_points()
        f, g = w.fields(torch, "cuda")
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        ctx.solve(f, g, w.g_at(xyz, torch), u, tol=1e-13)
        X, Y, Z = w.mesh(torch, "cuda")
        ue = w.u(X, Y, Z, torch).reshape(-1)
        m = t != cfp.SOLID
        errs.append(float((u - ue).abs()[m].max()))
    p = [np.log(errs[q] / errs[q + 1]) / np.log((ns[q + 1] - 1) / (ns[q] - 1)) for q in range(2)]
    assert 3.7 < p[0] < 4.3 and 3.8 < p[1] < 4.2, (errs, p)


@pytest.mark.parametrize("name", ["c2-33", "ragged-torus", "c3-bodies-65"])
def test_mixed_precision_reaches_fp64_error(name):
    p = pair(name)
    f, g = p.w.fields()
    gi = p.w.g_at(p.oxyz)
    X, Y, Z = p.w.mesh()
    ue = p.w.u(X, Y, Z, np).reshape(-1)
    m = p.otype != O.SOLID
    u64 = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    p.ctx.solve(dev(f), dev(g), dev(gi), u64, tol=1e-12)
    u32 = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    info = p.ctx.solve(dev(f), dev(g), dev(gi), u32, tol=1e-12, precision=cfp.PREC_MIXED)
    assert info.status == 0 and info.refinements >= 1
    e64 = np.max(np.abs(u64.cpu().numpy() - ue)[m])
    e32 = np.max(np.abs(u32.cpu().numpy() - ue)[m])
    assert e32 <= 1.02 * e64 + 1e-14, (e32, e64)
    assert np.max(np.abs(u32.cpu().numpy() - u64.cpu().numpy())) <= 1e-9 * np.max(np.abs(ue))


def test_errors_are_reported_not_raised_on_device():
    w = W.config1(17)
    ctx = cfp.Context(w.x, w.y, w.z, [W.sphere((0.5, 0.5, 0.97), 0.2)])  # body through the box
    with pytest.raises(cfp.CfpError) as e:
        ctx.classify_points()
    assert e.value.status == cfp.EGEOM
    ctx2 = cfp.Context(w.x, w.y, w.z)
    ctx2.classify_points()
    f, g = w.fields(torch, "cuda")
    f[100] = float("nan")
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    info = ctx2.solve(f, g, None, u, tol=1e-12, check=False)
    assert info.status == cfp.ENAN
    wq = W.quartic_workload(w.x, w.y, w.z, seed=2)
    f2, g2 = wq.fields(torch, "cuda")
    u.zero_()
    info = ctx2.solve(f2, g2, None, u, tol=1e-15, maxit=3, max_restarts=0, check=False)
    assert info.status == cfp.ENOCONV and info.iterations == 3
    u.zero_()
    info = ctx2.solve(f2, g2, None, u, tol=1e-12)
    assert info.status == 0


# ---------------------------------------------------------------- multigrid
@pytest.mark.parametrize("name", ["c2-33", "ragged-torus", "c3-bodies-65", "random-8"])
def test_solve_parity_multigrid(name):
    # The converged solution does not depend on the preconditioner: the
    # V-cycle solve must match the oracle's red-black solve like the others.
    p = pair(name)
    f, g = p.w.fields()
    gi = p.w.g_at(p.oxyz)
    uo, st, it, rel = p.P.solve(f, g, gi, tol=1e-13)
    u = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    info = p.ctx.solve(dev(f), dev(g), dev(gi), u, tol=1e-13, precond=cfp.PRECOND_MG)
    assert info.status == 0 and info.rel_residual <= 1e-13
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-10 * np.max(np.abs(uo))
    assert info.iterations < it


def test_multigrid_iterations_do_not_grow_with_n():
    its = []
    for n in (33, 65, 129):
        w = W.config2(n)
        ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
        ctx.classify_points()
        xyz = ctx.ibi_points()
        f, g = w.fields(torch, "cuda")
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        info = ctx.solve(f, g, w.g_at(xyz, torch), u, tol=1e-12, precond=cfp.PRECOND_MG)
        assert info.status == 0
        its.append(info.iterations)
    assert its[-1] <= 2 * its[0] + 4, its


@pytest.mark.parametrize("name", ["c2-33", "ragged-torus"])
def test_multigrid_preconditioner_is_linear_and_approximates_K_inverse(name):
    p = pair(name)
    K = p.P.export(O.MAT_K)
    a, b = p.rand_field(5), p.rand_field(6)
    outs = []
    for v in (a, b, 2.0 * a - 3.0 * b):
        phi = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
        p.ctx.precondition_ex(dev(v), phi, precond=cfp.PRECOND_MG)
        outs.append(phi.cpu().numpy())
    np.testing.assert_allclose(outs[2], 2.0 * outs[0] - 3.0 * outs[1], atol=1e-11 * np.max(np.abs(outs[2])))
    # residual of K phi = rho after one V-cycle, versus 8 red-black sweeps
    res_mg = np.linalg.norm((a - K @ outs[0])[p.unk]) / np.linalg.norm(a[p.unk])
    phi = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    p.ctx.precondition(dev(a), phi, 8)
    res_gs = np.linalg.norm((a - K @ phi.cpu().numpy())[p.unk]) / np.linalg.norm(a[p.unk])
    assert res_mg < 0.5 and res_mg < res_gs, (res_mg, res_gs)


@pytest.mark.parametrize("pinned", [True, False])
def test_solve_with_host_buffers_equals_the_device_solve(pinned):
    """cfp_solve_host on page-locked buffers (used in place by the kernels)
    and on pageable ones (copied through the context's device buffers) gives
    bitwise the solution of cfp_solve on device buffers, and leaves the
    caller's inputs unchanged."""
    p = pair("c3-bodies-65")
    f, g = p.w.fields()
    gi = p.w.g_at(p.oxyz)
    u_dev = torch.zeros(p.w.N, dtype=torch.float64, device="cuda")
    ref = p.ctx.solve(dev(f), dev(g), dev(gi), u_dev, tol=1e-12, precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG)
    hf, hg, hgi = (torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64) for a in (f, g, gi))
    hu = torch.zeros(p.w.N, dtype=torch.float64)
    if pinned:
        hf, hg, hgi, hu = (t.pin_memory() for t in (hf, hg, hgi, hu))
    f0 = hf.clone()
    info = p.ctx.solve_host(hf, hg, hgi, hu, tol=1e-12, precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG)
    assert info.status == 0 and info.iterations == ref.iterations
    assert torch.equal(hu, u_dev.cpu())
    assert torch.equal(hf, f0)
