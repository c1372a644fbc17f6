"""Pins of the oracle's second inner iteration on K: ILU(0) of K in natural
node order, used as a Richardson iteration from phi = 0 (the
incomplete-factorisation class of the paper's inner solver, Sec. 3.3).

What fixes it independently of the oracle's recurrence:
  - ILU(0) is defined by M = (P + L) P^-1 (P + U) agreeing with K on K's
    sparsity pattern; the product is formed here with scipy from the
    exported pivots and K;
  - on a single grid line K is tridiagonal, ILU(0) is the exact LU, and one
    sweep returns K^-1 rho;
  - m Richardson sweeps from zero are the truncated series
    sum_{q<m} (I - M^-1 K)^q M^-1 rho (dense algebra on a small grid);
  - BiCGSTAB with either inner iteration reaches the direct solution."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import pyoracle as O
from paper_1901_08269_gb300 import workloads as W


def _grids(n):
    return (W.tanh_grid(-1, 1, n, 1.3), W.tanh_grid(-1, 1, n + 2, 0.8), W.uniform_grid(-1, 1, n - 2))


BODIES = {
    "none": [],
    "sphere": [W.sphere((0.05, -0.03, 0.02), 0.3)],
    "torus": [W.torus((0.02, 0.01, -0.03), 0.45, 0.18, W.rot_euler(0.1, 0.5, 0.3))],
}


def _problem(n, bodies):
    P = O.Problem(*_grids(n), bodies)
    P.classify()
    P.ibi()
    P.assemble()
    idx = P.unknowns()
    K = P.export(O.MAT_K)[idx][:, idx].tocsr()
    d = P.ilu_pivots()
    return P, idx, K, d


def _factor(K, dpiv):
    L = sp.tril(K, -1, format="csr")
    U = sp.triu(K, 1, format="csr")
    D = sp.diags(dpiv)
    return ((D + L) @ sp.diags(1.0 / dpiv) @ (D + U)).tocsr()


@pytest.mark.parametrize("case", list(BODIES))
def test_ilu0_factor_equals_K_on_its_pattern(case):
    P, idx, K, d = _problem(15, BODIES[case])
    assert np.all(d[idx] < 0.0)  # K is negative definite-like: pivots keep the sign of the diagonal
    M = _factor(K, d[idx])
    pattern = K.copy()
    pattern.data[:] = 1.0
    on = M.multiply(pattern)
    scale = np.max(np.abs(K.data))
    assert np.max(np.abs((on - K).data)) <= 1e-12 * scale
    off = M - on
    off.eliminate_zeros()
    assert off.nnz > 0  # the fill that ILU(0) drops is really there
    # non-unknowns carry no pivot
    mask = np.ones(P.N, bool)
    mask[idx] = False
    assert np.all(d[mask] == 0.0)


def test_ilu0_on_a_single_line_is_the_exact_inverse():
    x = W.tanh_grid(-1, 1, 23, 1.4)
    y = z = W.uniform_grid(-1, 1, 3)
    P = O.Problem(x, y, z, [])
    P.classify()
    P.assemble()
    idx = P.unknowns()
    K = P.export(O.MAT_K)[idx][:, idx].tocsc()
    rng = np.random.default_rng(4)
    rho = np.zeros(P.N)
    rho[idx] = rng.standard_normal(idx.size)
    phi = P.precond(rho, 1, kind=O.PRECOND_ILU)
    exact = spla.spsolve(K, rho[idx])
    assert np.max(np.abs(phi[idx] - exact)) <= 1e-13 * np.max(np.abs(exact))


@pytest.mark.parametrize("case", ["sphere", "torus"])
def test_ilu_richardson_is_the_truncated_series(case):
    P, idx, K, d = _problem(11, BODIES[case])
    Kd = K.toarray()
    Md = _factor(K, d[idx]).toarray()
    rng = np.random.default_rng(5)
    rho = np.zeros(P.N)
    rho[idx] = rng.standard_normal(idx.size)
    G = np.eye(idx.size) - np.linalg.solve(Md, Kd)
    base = np.linalg.solve(Md, rho[idx])
    want, term = np.zeros(idx.size), base.copy()
    for m in range(1, 4):
        want = want + term
        term = G @ term
        got = P.precond(rho, m, kind=O.PRECOND_ILU)[idx]
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want)), m
    # a linear map converging to K^-1
    exact = np.linalg.solve(Kd, rho[idx])
    e = [np.max(np.abs(P.precond(rho, m, kind=O.PRECOND_ILU)[idx] - exact)) for m in (1, 4, 16, 400)]
    assert e[0] > e[1] > e[2] > e[3] and e[3] < 1e-9 * np.max(np.abs(exact))
    np.testing.assert_array_equal(P.precond(rho, 0, kind=O.PRECOND_ILU)[idx], rho[idx])


@pytest.mark.parametrize("case,n", [("sphere", 17), ("torus", 19)])
def test_bicgstab_with_ilu_matches_direct_solve(case, n):
    w = W.Workload("ilu", *_grids(n), BODIES[case], W._c2_u, W._c2_f)
    P = O.Problem(w.x, w.y, w.z, w.bodies)
    P.classify()
    key, tt, xyz = P.ibi()
    f, g = w.fields()
    rhs = P.rhs(f, g, w.g_at(xyz))
    idx = P.unknowns()
    direct = spla.spsolve(P.export(O.MAT_B)[idx][:, idx].tocsc(), rhs[idx])
    its = {}
    for kind in (O.PRECOND_RBGS, O.PRECOND_ILU):
        P.set_precond(kind)
        xs, st, it, rel = P.bicgstab(rhs, tol=1e-14, sweeps=2)
        assert st == 0
        assert np.max(np.abs(xs[idx] - direct)) < 1e-11 * np.max(np.abs(direct))
        its[kind] = it
    P.set_precond(O.PRECOND_RBGS)
    assert its[O.PRECOND_ILU] > 0
