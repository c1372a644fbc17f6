"""Pins of the oracle's 1D and line operators against facts the paper and
the mathematics fix (closed forms, polynomial exactness, the printed moment
right-hand sides of Eqs. mat1-mat4)."""
import numpy as np
import pytest

from oracle import pyoracle as O


def test_compact_coefs_uniform_closed_form():
    # Eq. app_xxx with dx_f = dx_b = h: a = c = 1/10, ar = cr = 12/(10 h^2),
    # br = -12/(5 h^2) -- the classical (1, 10, 1)/12 Pade scheme scaled by 1.2.
    h = 0.125
    x = np.arange(9) * h
    a, c, ar, br, cr = O.compact_coefs(x)
    np.testing.assert_allclose(a[1:-1], 0.1, rtol=1e-14)
    np.testing.assert_allclose(c[1:-1], 0.1, rtol=1e-14)
    np.testing.assert_allclose(ar[1:-1], 1.2 / h ** 2, rtol=1e-14)
    np.testing.assert_allclose(cr[1:-1], 1.2 / h ** 2, rtol=1e-14)
    np.testing.assert_allclose(br[1:-1], -2.4 / h ** 2, rtol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_compact_coefs_nonuniform_exact_to_degree4(seed):
    # a u''_{i-1} + u''_i + c u''_{i+1} = ar u_{i-1} + br u_i + cr u_{i+1}
    # holds exactly for u = x^m, m <= 4, and not for m = 5 on a nonuniform grid.
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.uniform(0.5, 2.0, 12)) * 0.1
    a, c, ar, br, cr = O.compact_coefs(x)
    for m in range(7):
        u = x ** m
        upp = m * (m - 1) * x ** (m - 2) if m >= 2 else 0 * x
        lhs = a[1:-1] * upp[:-2] + upp[1:-1] + c[1:-1] * upp[2:]
        rhs = ar[1:-1] * u[:-2] + br[1:-1] * u[1:-1] + cr[1:-1] * u[2:]
        scale = np.abs(ar[1:-1] * u[:-2]) + np.abs(br[1:-1] * u[1:-1]) + np.abs(cr[1:-1] * u[2:]) + 1.0
        err = np.max(np.abs(lhs - rhs) / scale)
        if m <= 4:
            assert err < 1e-12, (m, err)
        elif m == 5:
            assert err > 1e-6, (m, err)


def test_second_order_coefs():
    rng = np.random.default_rng(4)
    x = np.cumsum(rng.uniform(0.5, 2.0, 10)) * 0.1
    a, b, c = O.second_coefs(x)
    for m in range(3):  # exact for quadratics (Eq. 2ndorder_coef)
        u = x ** m
        upp = m * (m - 1) * x ** (m - 2) if m >= 2 else 0 * x
        np.testing.assert_allclose(a[1:-1] * u[:-2] + b[1:-1] * u[1:-1] + c[1:-1] * u[2:], upp[1:-1],
                                   atol=1e-10 * np.max(np.abs(b)))
    h = 0.25
    a, b, c = O.second_coefs(np.arange(6) * h)
    np.testing.assert_allclose(a[1:-1], 1 / h ** 2)
    np.testing.assert_allclose(b[1:-1], -2 / h ** 2)
    np.testing.assert_allclose(c[1:-1], 1 / h ** 2)


def _paper_rhs_mat1(a, b, h0):
    # Eq. mat1 as printed: [0, 0, 2(a+b), 6 h0 a, 12 h0^2 a, 20 h0^3 a]
    return np.array([0.0, 0.0, 2 * (a + b), 6 * h0 * a, 12 * h0 ** 2 * a, 20 * h0 ** 3 * a])


@pytest.mark.parametrize("seed", range(5))
def test_line_operator_matches_printed_moments_mat1(seed):
    # +1 solid: expansion about x_i with nodes x_i, x_{i-1}..x_{i-4} and the IBI
    # in (x_i, x_{i+1}); the unknowns are ordered [br, ar, psi1, psi2, psi3, psi_b].
    rng = np.random.default_rng(seed)
    gaps = rng.uniform(0.5, 1.5, 5) * 0.01
    xi_nodes = np.array([0.0, -gaps[0], -gaps[:2].sum(), -gaps[:3].sum(), -gaps[:4].sum()])
    t = rng.uniform(0.05, 1.0)
    xb = t * 0.01
    a, bL = rng.uniform(0.05, 0.15), 1.0
    pts = np.concatenate([xi_nodes, [xb]])
    c = O.line_operator(pts, 0.0, [xi_nodes[1], 0.0], [a, bL])
    h = pts - 0.0
    moments = np.array([np.sum(c * h ** m) for m in range(6)])
    expect = _paper_rhs_mat1(a, bL, xi_nodes[1])
    np.testing.assert_allclose(moments, expect, rtol=1e-9, atol=1e-9 * np.max(np.abs(expect)))


@pytest.mark.parametrize("seed", range(5))
def test_line_operator_matches_printed_moments_mat2_mat3(seed):
    rng = np.random.default_rng(100 + seed)
    g = rng.uniform(0.5, 1.5, 6) * 0.01
    # Eq. mat2: expansion about the surviving node only -> [0, 0, 2a, 0, 0, 0]
    nodes = -np.cumsum(np.concatenate([[0.0], g[:4]]))
    xb = rng.uniform(0.0, 1.0) * g[5]
    a = 0.1
    c = O.line_operator(np.concatenate([nodes, [xb]]), 0.0, [0.0], [a])
    h = np.concatenate([nodes, [xb]])
    np.testing.assert_allclose([np.sum(c * h ** m) for m in range(6)], [0, 0, 2 * a, 0, 0, 0],
                               atol=1e-9 * 2 * a)
    # Eq. mat3: -1 solid, expansion about x_k with x_{k+1}..x_{k+4}:
    # [0, 0, 2(b+c), 6 h0 c, 12 h0^2 c, 20 h0^3 c], h0 = x_{k+1} - x_k
    nodes = np.cumsum(np.concatenate([[0.0], g[:4]]))
    xb = -rng.uniform(0.0, 1.0) * g[5]
    cc, bL = 0.11, 1.0
    c = O.line_operator(np.concatenate([nodes, [xb]]), 0.0, [0.0, nodes[1]], [bL, cc])
    h = np.concatenate([nodes, [xb]])
    h0 = nodes[1]
    expect = [0, 0, 2 * (bL + cc), 6 * h0 * cc, 12 * h0 ** 2 * cc, 20 * h0 ** 3 * cc]
    np.testing.assert_allclose([np.sum(c * h ** m) for m in range(6)], expect, rtol=1e-9,
                               atol=1e-9 * np.max(np.abs(expect)))


@pytest.mark.parametrize("M", [3, 4, 5, 6])
def test_line_operator_polynomial_exactness(M):
    # sum_n c_n p(x_n) = sum_s L_s p''(x_s) for every p of degree < M
    rng = np.random.default_rng(M)
    pts = np.sort(rng.uniform(-1, 1, M)) * 0.05
    xs = pts[:1]
    Ls = np.array([0.9])
    c = O.line_operator(pts, pts[0], xs, Ls)
    for deg in range(M + 1):
        p = np.polynomial.Polynomial(rng.standard_normal(deg + 1))
        lhs = np.sum(c * p(pts))
        rhs = np.sum(Ls * p.deriv(2)(xs))
        scale = np.sum(np.abs(c * p(pts))) + 1.0
        if deg < M:
            assert abs(lhs - rhs) < 1e-10 * scale, (deg, lhs, rhs)
