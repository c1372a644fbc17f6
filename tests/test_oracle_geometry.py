"""Pins of the oracle's point classification and IBI location (Sec. 2):
brute force on tiny grids, octant symmetry, closed-form roots along grid
lines: the sphere and rotated ellipsoid quadratics, the rotated torus quartic."""
import math

import numpy as np
import pytest

from oracle import pyoracle as O
from paper_1901_08269_gb300 import workloads as W


def _phi_np(bodies, X, Y, Z):
    """Level set evaluated with numpy (signs only are compared)."""
    out = np.full(X.shape, np.inf)
    for b in bodies:
        R = np.asarray(b["R"], float)
        d = np.stack([X - b["c"][0], Y - b["c"][1], Z - b["c"][2]], -1)
        q = d @ R  # q_a = sum_b R[b, a] d_b
        if b["kind"] == "sphere":
            v = (q ** 2).sum(-1) - b["p"][0] ** 2
        elif b["kind"] == "ellipsoid":
            v = ((q / np.asarray(b["p"])) ** 2).sum(-1) - 1.0
        else:
            rho = np.sqrt(q[..., 0] ** 2 + q[..., 1] ** 2)
            v = (rho - b["p"][0]) ** 2 + q[..., 2] ** 2 - b["p"][1] ** 2
        out = np.minimum(out, v)
    return out


def _brute_classify(x, y, z, bodies):
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    solid = _phi_np(bodies, X, Y, Z) <= 0
    nz, ny, nx = solid.shape
    t = np.ones(solid.shape, np.uint8)
    box = np.zeros_like(solid)
    box[0], box[-1], box[:, 0], box[:, -1], box[:, :, 0], box[:, :, -1] = True, True, True, True, True, True
    solid &= ~box
    t[solid] = O.SOLID
    for k in range(1, nz - 1):
        for j in range(1, ny - 1):
            for i in range(1, nx - 1):
                if not solid[k, j, i] and solid[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2].any():
                    t[k, j, i] = O.IRREGULAR
    t[box] = O.BOUNDARY
    return t.reshape(-1)


@pytest.mark.parametrize("case", ["sphere", "ellipsoid", "torus"])
def test_classification_brute_force(case):
    x = W.tanh_grid(-1, 1, 19, 0.9)
    y = W.tanh_grid(-1, 1, 17, 0.4)
    z = W.uniform_grid(-1, 1, 15)
    bodies = {"sphere": [W.sphere((0.03, -0.05, 0.02), 0.41)],
              "ellipsoid": [W.ellipsoid((0.02, 0.01, -0.03), (0.5, 0.3, 0.35), W.rot_euler(0.3, 0.5, 0.7))],
              "torus": [W.torus((0.01, 0.02, 0.03), 0.5, 0.17, W.rot_euler(0.2, 0.4, 0.1))]}[case]
    P = O.Problem(x, y, z, bodies)
    t = P.classify()
    np.testing.assert_array_equal(t, _brute_classify(x, y, z, bodies))
    assert P.n_irr == int(np.sum(t == O.IRREGULAR))


def test_classification_octant_symmetry():
    # A centred sphere on a grid symmetric about 0: the type field is invariant
    # under every axis reflection and axis permutation (equal axes).
    x = W.tanh_grid(-1, 1, 23, 1.1)
    P = O.Problem(x, x, x, [W.sphere((0, 0, 0), 0.47)])
    t = P.classify().reshape(23, 23, 23)
    for flip in [(0,), (1,), (2,)]:
        np.testing.assert_array_equal(t, np.flip(t, flip))
    np.testing.assert_array_equal(t, np.transpose(t, (1, 0, 2)))
    np.testing.assert_array_equal(t, np.transpose(t, (2, 1, 0)))


def test_ibi_sphere_closed_form():
    # Along an axis line the sphere gives a quadratic whose root is known in
    # closed form; the IBI must be that root (to bisection accuracy).
    c, r = (0.031, -0.017, 0.023), 0.43
    x = W.tanh_grid(-1, 1, 21, 0.7)
    P = O.Problem(x, x, x, [W.sphere(c, r)])
    t = P.classify()
    key, tt, xyz = P.ibi()
    assert len(key) > 0 and np.all((tt > 0) & (tt <= 1))
    n = x.size
    lin, d = key // 6, key % 6
    i, j, k = lin % n, (lin // n) % n, lin // (n * n)
    node = np.stack([x[i], x[j], x[k]], -1)
    for q in range(len(key)):
        ax, sgn = d[q] // 2, (1 if d[q] % 2 else -1)
        idx = (i[q], j[q], k[q])
        xa, xb = x[idx[ax]], x[idx[ax] + sgn]
        other = [a for a in range(3) if a != ax]
        rr = r ** 2 - sum((node[q, a] - c[a]) ** 2 for a in other)
        cand = [c[ax] + math.sqrt(rr), c[ax] - math.sqrt(rr)]
        lo, hi = min(xa, xb), max(xa, xb)
        inside = [v for v in cand if lo - 1e-15 <= v <= hi + 1e-15]
        assert len(inside) == 1, q
        assert abs(xyz[q, ax] - inside[0]) < 1e-13, (q, xyz[q, ax], inside)
        for a in other:
            assert xyz[q, a] == node[q, a]


def _line_roots(body, node, ax):
    """Roots t of the body's level set along node + t e_ax, from the closed
    form: a quadratic for the ellipsoid, the quartic
    (|q|^2 + R^2 - r^2)^2 = 4 R^2 (q_x^2 + q_y^2) for the torus, where
    q(t) = R^T (node + t e_ax - c) is linear in t (numpy's companion-matrix
    roots, then Newton steps on the same polynomial)."""
    Rm = np.asarray(body["R"], float)
    q0 = Rm.T @ (np.asarray(node, float) - np.asarray(body["c"], float))
    d = Rm.T[:, ax]
    if body["kind"] == "ellipsoid":
        a = np.asarray(body["p"], float)
        A, B, C = np.sum(d * d / a ** 2), 2 * np.sum(q0 * d / a ** 2), np.sum(q0 * q0 / a ** 2) - 1.0
        disc = B * B - 4 * A * C
        if disc < 0:
            return []
        sq = math.sqrt(disc)
        return [(-B + sq) / (2 * A), (-B - sq) / (2 * A)]
    Rmaj, rmin = body["p"][0], body["p"][1]
    quad = np.array([d @ d, 2 * (q0 @ d), q0 @ q0 + Rmaj ** 2 - rmin ** 2])
    rho2 = np.array([d[0] ** 2 + d[1] ** 2, 2 * (q0[0] * d[0] + q0[1] * d[1]), q0[0] ** 2 + q0[1] ** 2])
    poly = np.polysub(np.polymul(quad, quad), 4 * Rmaj ** 2 * np.concatenate([[0, 0], rho2]))
    dpoly = np.polyder(poly)
    out = []
    for t in np.roots(poly):
        if abs(t.imag) > 1e-6:
            continue
        t = t.real
        for _ in range(4):
            t -= np.polyval(poly, t) / np.polyval(dpoly, t)
        out.append(t)
    return out


@pytest.mark.parametrize("body", [
    W.ellipsoid((0.021, -0.013, 0.034), (0.52, 0.31, 0.4), W.rot_euler(0.4, -0.7, 0.2)),
    W.torus((0.02, 0.01, -0.03), 0.45, 0.16, W.rot_euler(0.1, 0.5, 0.3)),
])
def test_ibi_rotated_ellipsoid_and_torus_closed_forms(body):
    # every IBI coordinate the oracle's scan-and-bisection finds must be a root
    # of the body's own polynomial along that grid line, inside the segment
    x = W.tanh_grid(-1, 1, 25, 0.7)
    P = O.Problem(x, x, x, [body])
    P.classify()
    key, tt, xyz = P.ibi()
    assert len(key) > 100 and np.all((tt > 0) & (tt <= 1))
    n = x.size
    lin, d = key // 6, key % 6
    i, j, k = lin % n, (lin // n) % n, lin // (n * n)
    node = np.stack([x[i], x[j], x[k]], -1)
    for q in range(len(key)):
        ax, sgn = d[q] // 2, (1 if d[q] % 2 else -1)
        idx = (i[q], j[q], k[q])
        xa, xb = x[idx[ax]], x[idx[ax] + sgn]
        lo, hi = min(xa, xb), max(xa, xb)
        roots = [node[q, ax] + t for t in _line_roots(body, node[q], ax)]
        inside = [v for v in roots if lo - 1e-12 <= v <= hi + 1e-12]
        assert inside, q
        assert min(abs(xyz[q, ax] - v) for v in inside) < 1e-12, (q, xyz[q, ax], inside)
        for a in range(3):
            if a != ax:
                assert xyz[q, a] == node[q, a]


def test_irregular_count_growth():
    # N_irr of a fixed smooth body grows like n^2 (Tables p1, p2_flop: factor
    # 3.66-3.97 per doubling).
    counts = []
    for n in (33, 65, 129):
        x = W.uniform_grid(0, 1, n)
        P = O.Problem(x, x, x, [W.sphere((0.52, 0.49, 0.505), 0.27)])
        P.classify()
        counts.append(P.n_irr)
    r = np.array(counts[1:]) / np.array(counts[:-1])
    assert np.all((r > 3.5) & (r < 4.3)), counts
