"""The ILU(0)-Richardson inner iteration (CFP_PRECOND_ILU) against the
oracle's, through the C ABI: the preconditioner map itself, and solves with
it in FP64 and mixed precision (the converged solution does not depend on
the preconditioner, so it must match the oracle's red-black solve)."""
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
    return (W.tanh_grid(-1, 1, n, 1.1), W.tanh_grid(-1, 1, n + 12, 0.7), W.uniform_grid(-1, 1, n - 6))


CASES = {
    "c2-33": lambda: W.config2(33),
    "ragged-torus": lambda: W.Workload("ragged-torus", *ragged(41),
                                       [W.torus((0.02, 0.01, -0.03), 0.45, 0.16, W.rot_euler(0.1, 0.5, 0.3))],
                                       W._c3_u, W._c3_f),
    "interior-sphere": lambda: W.interior_sphere(41),
    "random-3": lambda: W.random_problem(3, sizes=(33, 49)),
}

_cache = {}


def setup(name):
    if name not in _cache:
        w = CASES[name]()
        ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
        ctx.classify_points()
        P = O.Problem(w.x, w.y, w.z, w.bodies, w.fluid_inside)
        otype = P.classify()
        _, _, oxyz = P.ibi()
        P.assemble()
        unk = np.flatnonzero((otype == O.REGULAR) | (otype == O.IRREGULAR))
        _cache[name] = (w, ctx, P, oxyz, unk)
    return _cache[name]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("sweeps", [1, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_ilu_preconditioner_matches_oracle(name, sweeps):
    w, ctx, P, oxyz, unk = setup(name)
    rng = np.random.default_rng(21 + sweeps)
    rho = np.zeros(w.N)
    rho[unk] = rng.standard_normal(unk.size)
    want = P.precond(rho, sweeps, kind=O.PRECOND_ILU)
    phi = torch.full((w.N,), 3.0, dtype=torch.float64, device="cuda")
    ctx.precondition_ex(dev(rho), phi, precond=cfp.PRECOND_ILU, sweeps=sweeps)
    got = phi.cpu().numpy()
    mask = np.ones(w.N, bool)
    mask[unk] = False
    assert np.all(got[mask] == 0.0)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 1e-12, err
    # the same map again: the work field's previous contents must not leak in
    phi2 = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    ctx.precondition_ex(dev(rho), phi2, precond=cfp.PRECOND_ILU, sweeps=sweeps)
    assert torch.equal(phi, phi2)


@pytest.mark.parametrize("name", ["c2-33", "ragged-torus", "interior-sphere"])
def test_solve_with_ilu_matches_oracle(name):
    w, ctx, P, oxyz, unk = setup(name)
    f, g = w.fields()
    gi = w.g_at(oxyz)
    # Different inner iterations stop at different iterates; at 1e-14 both
    # sides are within the 1e-10 bar of the exact discrete solution (at
    # 1e-13 the interior problem's conditioning leaves 1.3e-10 between them).
    P.set_precond(O.PRECOND_RBGS)
    uo, st, it, rel = P.solve(f, g, gi, tol=1e-14)
    assert st == 0
    sols = []
    for use_graph in (1, 0):
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        info = ctx.solve(dev(f), dev(g), dev(gi), u, tol=1e-14, precond=cfp.PRECOND_ILU, sweeps=2,
                         use_graph=use_graph)
        assert info.status == 0 and info.rel_residual <= 1e-14
        sols.append(u.cpu().numpy())
        assert np.max(np.abs(sols[-1] - uo)) <= 1e-10 * np.max(np.abs(uo))
    np.testing.assert_array_equal(sols[0], sols[1])  # graph and plain launches: the same arithmetic
    # mixed precision with FP32 ILU sweeps reaches the same solution
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    info = ctx.solve(dev(f), dev(g), dev(gi), u, tol=1e-14, precond=cfp.PRECOND_ILU, sweeps=2,
                     precision=cfp.PREC_MIXED)
    assert info.status == 0 and info.rel_residual <= 1e-14
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= 1e-10 * np.max(np.abs(uo))


def test_ilu_oracle_solve_matches_gpu_iteration_count_closely():
    # the same preconditioner on both sides: BiCGSTAB iteration counts agree
    # up to rounding-driven differences of a few iterations
    w, ctx, P, oxyz, unk = setup("c2-33")
    f, g = w.fields()
    gi = w.g_at(oxyz)
    P.set_precond(O.PRECOND_ILU)
    uo, st, it_o, rel = P.solve(f, g, gi, tol=1e-12, sweeps=2)
    P.set_precond(O.PRECOND_RBGS)
    assert st == 0
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    info = ctx.solve(dev(f), dev(g), dev(gi), u, tol=1e-12, precond=cfp.PRECOND_ILU, sweeps=2)
    assert info.status == 0
    assert abs(info.iterations - it_o) <= max(2, it_o // 10), (info.iterations, it_o)
