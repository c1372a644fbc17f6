"""The rounding bounds behind the classification's FP32 fast path.

k_classify_solid and the IBI bisection take a body's level-set sign from an
FP32 evaluation wherever that value lies farther from zero than twice a bound
on its rounding error, and from the exact FP64 level set elsewhere.  The
bounds (stated with the kernel, u = 2^-24, A_j = |x_j| + |c_j|,
W_i = sum_j |R_ji| A_j, V_i = W_i / p_i):

  sphere     |phi32 - phi| <= 16.1 u sum W_i^2 + 4.01 u p^2
  ellipsoid  |phi32 - phi| <= 20.1 u sum V_i^2 + 1.01 u
  torus      E_rho = 14.05 u (W_0^2 + W_1^2) / rho32 + u rho32,
             E_s = E_rho + u (rho32 + 2 R), S = |s32| + E_s:
             |phi32 - phi| <= 2 E_s S + 3.01 u S^2 + 15.05 u W_2^2 + 4.01 u r^2

and the bounding-sphere test's threshold, |d2_32 - d2| <= 7.01 u sum A_j^2.
Here the same operations are carried out in numpy float32 (IEEE
round-to-nearest, as the kernel's __fadd_rn / __fmul_rn / __fsqrt_rn) and
float64 on rotated bodies and points drawn close to their surfaces, and the
error of each FP32 value is checked against its bound (not doubled)."""
import numpy as np

F = np.float32
U = 2.0 ** -24


def rotation(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return (rz @ ry @ rx).reshape(-1)


def phi64(kind, c, R, p, x):
    d = x - c
    q = [(R[i] * d[0] + R[3 + i] * d[1]) + R[6 + i] * d[2] for i in range(3)]
    if kind == 0:
        return (q[0] * q[0] + q[1] * q[1]) + q[2] * q[2] - p[0] * p[0]
    if kind == 1:
        e = [q[i] / p[i] for i in range(3)]
        return (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2] - 1.0
    s = np.sqrt(q[0] * q[0] + q[1] * q[1]) - p[0]
    return (s * s + q[2] * q[2]) - p[1] * p[1]


def phi32_and_bound(kind, c, R, p, x):
    cf, Rf, pf, xf = c.astype(F), R.astype(F), p.astype(F), x.astype(F)
    d = [F(xf[j] - cf[j]) for j in range(3)]
    a = [abs(float(xf[j])) + abs(float(cf[j])) for j in range(3)]
    q = [F(F(F(Rf[i] * d[0]) + F(Rf[3 + i] * d[1])) + F(Rf[6 + i] * d[2])) for i in range(3)]
    W = [abs(float(Rf[i])) * a[0] + abs(float(Rf[3 + i])) * a[1] + abs(float(Rf[6 + i])) * a[2] for i in range(3)]
    if kind == 0:
        s = F(F(F(q[0] * q[0]) + F(q[1] * q[1])) + F(q[2] * q[2]))
        pp = F(pf[0] * pf[0])
        return float(F(s - pp)), U * (16.1 * sum(w * w for w in W) + 4.01 * float(pp))
    if kind == 1:
        ip = [F(1.0 / p[i]) for i in range(3)]
        e = [F(q[i] * ip[i]) for i in range(3)]
        s = F(F(F(e[0] * e[0]) + F(e[1] * e[1])) + F(e[2] * e[2]))
        V = [W[i] * float(ip[i]) for i in range(3)]
        return float(F(s - F(1))), U * (20.1 * sum(v * v for v in V) + 1.01)
    t = F(F(q[0] * q[0]) + F(q[1] * q[1]))
    rho = np.sqrt(t, dtype=F)
    if not rho > 0:
        return None, None
    s = F(rho - pf[0])
    ph = F(F(F(s * s) + F(q[2] * q[2])) - F(pf[1] * pf[1]))
    rho = float(rho)
    er = 14.05 * U * (W[0] ** 2 + W[1] ** 2) / rho + U * rho
    es = er + U * (rho + 2 * float(pf[0]))
    S = abs(float(s)) + es
    return float(ph), 2 * es * S + U * (3.01 * S * S + 15.05 * W[2] ** 2 + 4.01 * float(pf[1]) ** 2)


def test_fp32_level_set_errors_stay_within_their_bounds():
    rng = np.random.default_rng(20261204)
    worst, certified, total = 0.0, 0, 0
    for trial in range(600):
        kind = trial % 3
        c = rng.uniform(-0.5, 0.5, 3)
        R = rotation(*rng.uniform(0, 6.3, 3))
        if kind == 0:
            p = np.array([rng.uniform(0.1, 0.5)] * 3)
        elif kind == 1:
            p = rng.uniform(0.1, 0.5, 3)
        else:
            p = np.array([rng.uniform(0.25, 0.45), rng.uniform(0.05, 0.2), 0.0])
        for k in range(20):
            x = rng.uniform(-1, 1, 3)
            if k % 2 == 0:  # close to the surface: bisect along c -> x, then jitter
                lo, hi = 0.0, 1.0
                for _ in range(50):
                    mid = 0.5 * (lo + hi)
                    if phi64(kind, c, R, p, c + mid * (x - c)) < 0:
                        lo = mid
                    else:
                        hi = mid
                x = c + hi * (x - c) + rng.normal(0, 10.0 ** rng.uniform(-9, -3), 3)
            ph, bound = phi32_and_bound(kind, c, R, p, x)
            if ph is None:
                continue
            exact = phi64(kind, c, R, p, x)
            total += 1
            assert abs(ph - exact) <= bound, (kind, ph, exact, bound)
            worst = max(worst, abs(ph - exact) / bound)
            if abs(ph) > 2 * bound:
                certified += 1
                assert (ph > 0) == (exact > 0) and exact != 0.0
    assert total > 10000 and certified > total // 3, (total, certified)
    assert worst < 1.0


def test_fp32_bounding_sphere_distance_error_stays_within_its_bound():
    rng = np.random.default_rng(7)
    for _ in range(20000):
        x = rng.uniform(-1, 1, 3)
        c = rng.uniform(-0.6, 0.6, 3)
        d64 = x - c
        d2 = float(np.dot(d64, d64))
        xf, cf = x.astype(F), c.astype(F)
        df = [F(xf[j] - cf[j]) for j in range(3)]
        d2f = F(F(F(df[0] * df[0]) + F(df[1] * df[1])) + F(df[2] * df[2]))
        A2 = sum((abs(x[j]) + abs(c[j])) ** 2 for j in range(3))
        assert abs(float(d2f) - d2) <= 7.01 * U * A2
