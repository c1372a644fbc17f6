"""Seeded synthetic inputs: grids, bodies and manufactured solutions.

This module holds none of the method's arithmetic.  It produces the inputs of
the solver (three 1D coordinate arrays, implicit body descriptions, the source
f and the Dirichlet data g as functions of position) for the workloads the
tests and the benchmark run.  Both the CUDA path and the CPU oracle receive
the same arrays from here.

Every function of position takes an array module ``xp`` (numpy or torch) so
that the same formula can be evaluated on the host or on the device.
"""
import math
from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np


# ---------------------------------------------------------------- grids
def uniform_grid(a: float, b: float, n: int) -> np.ndarray:
    x = a + (b - a) * np.arange(n, dtype=np.float64) / (n - 1)
    x[0], x[-1] = a, b
    return x


def tanh_grid(a: float, b: float, n: int, beta: float) -> np.ndarray:
    """Nodes clustered toward the centre of [a, b]: with xi uniform on
    [-1, 1], x = mid + half * artanh(xi * tanh(beta)) / beta.  The largest to
    smallest spacing ratio is about cosh(beta)**2; beta -> 0 is uniform."""
    if beta <= 0.0:
        return uniform_grid(a, b, n)
    xi = -1.0 + 2.0 * np.arange(n, dtype=np.float64) / (n - 1)
    s = np.arctanh(xi * math.tanh(beta)) / beta
    x = 0.5 * (a + b) + 0.5 * (b - a) * s
    x[0], x[-1] = a, b
    return x


def sinh_grid(n: int, beta: float, L: float, H: float, offset: float = 0.0) -> np.ndarray:
    """Sinh stretching of Sec. 4 (Eqs. p2_y, p2_s): x_j = offset + L (1 +
    sinh(beta (eta - s)) / sinh(beta s)), eta = j / (n - 1), with
    s = log((1 + (e^beta - 1) L / H) / (1 + (e^-beta - 1) L / H)) / (2 beta).
    Nodes cluster around offset + L; the interval is [offset, offset + H]."""
    eta = np.arange(n, dtype=np.float64) / (n - 1)
    s = math.log((1.0 + (math.exp(beta) - 1.0) * L / H) / (1.0 + (math.exp(-beta) - 1.0) * L / H)) / (2.0 * beta)
    return offset + L * (1.0 + np.sinh(beta * (eta - s)) / math.sinh(beta * s))


# ---------------------------------------------------------------- bodies
def rot_z(deg: float) -> np.ndarray:
    t = math.radians(deg)
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_euler(a: float, b: float, c: float) -> np.ndarray:
    """Body-to-world rotation Rz(a) Ry(b) Rx(c), angles in radians."""
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    Ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    Rx = np.array([[1.0, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


def sphere(c, r):
    return {"kind": "sphere", "c": tuple(map(float, c)), "R": np.eye(3), "p": (float(r), 0.0, 0.0)}


def ellipsoid(c, axes, R=None):
    return {"kind": "ellipsoid", "c": tuple(map(float, c)), "R": np.eye(3) if R is None else np.asarray(R, float),
            "p": tuple(map(float, axes))}


def torus(c, R_major, r_minor, R=None):
    return {"kind": "torus", "c": tuple(map(float, c)), "R": np.eye(3) if R is None else np.asarray(R, float),
            "p": (float(R_major), float(r_minor), 0.0)}


# ------------------------------------------------------- workload record
@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    bodies: List[dict]
    u: Callable          # u(X, Y, Z, xp) exact solution / Dirichlet data g
    f: Callable          # f(X, Y, Z, xp) source
    fluid_inside: bool = False
    tol: float = 1e-12
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.z.size, self.y.size, self.x.size)

    @property
    def N(self):
        return self.x.size * self.y.size * self.z.size

    def mesh(self, xp=np, device=None):
        """Full-grid coordinates as three arrays of shape (nz, ny, nx)."""
        if xp is np:
            Z, Y, X = np.meshgrid(self.z, self.y, self.x, indexing="ij")
            return X, Y, Z
        import torch
        x = torch.as_tensor(self.x, dtype=torch.float64, device=device)
        y = torch.as_tensor(self.y, dtype=torch.float64, device=device)
        z = torch.as_tensor(self.z, dtype=torch.float64, device=device)
        Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z

    def fields(self, xp=np, device=None):
        """(f, g) on every node, flattened in x-fastest order.  g is the exact
        solution, used by the solver only on the box boundary."""
        X, Y, Z = self.mesh(xp, device)
        f = self.f(X, Y, Z, xp).reshape(-1)
        g = self.u(X, Y, Z, xp).reshape(-1)
        if xp is np:
            return np.ascontiguousarray(f), np.ascontiguousarray(g)
        return f.contiguous(), g.contiguous()

    def g_at(self, xyz, xp=np):
        """Dirichlet data at IBI points given as an (n, 3) array."""
        if xyz.shape[0] == 0:
            return xp.zeros(0, dtype=xp.float64) if xp is np else xyz[:, 0].clone()
        return self.u(xyz[:, 0], xyz[:, 1], xyz[:, 2], xp)


# --------------------------------------------------- manufactured solutions
def _sinpi3(X, Y, Z, xp):
    return xp.sin(math.pi * X) * xp.sin(math.pi * Y) * xp.sin(math.pi * Z)


def _sinpi3_f(X, Y, Z, xp):
    return -3.0 * math.pi ** 2 * _sinpi3(X, Y, Z, xp)


def _c2_u(X, Y, Z, xp):
    return xp.exp(X) * xp.sin(Y) * xp.cos(2.0 * Z) + X * X * Y


def _c2_f(X, Y, Z, xp):
    return -4.0 * xp.exp(X) * xp.sin(Y) * xp.cos(2.0 * Z) + 2.0 * Y


def _c3_u(X, Y, Z, xp):
    return xp.sin(2.0 * X) * xp.cosh(Y) * xp.exp(-Z * Z)


def _c3_f(X, Y, Z, xp):
    return _c3_u(X, Y, Z, xp) * (4.0 * Z * Z - 5.0)


def _p1_u(X, Y, Z, xp, w=2.0 * math.pi):
    return xp.sin(w * X) * xp.cos(w * Y) * xp.cos(w * Z)


def _p1_f(X, Y, Z, xp, w=2.0 * math.pi):
    return -3.0 * w * w * _p1_u(X, Y, Z, xp, w)


def quartic(seed: int = 0):
    """A random polynomial of degree <= 4 in each variable (tensor Q4) and
    its Laplacian.  Returns (u, f) callables."""
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal((5, 5, 5)) / (1.0 + np.add.outer(np.add.outer(np.arange(5), np.arange(5)), np.arange(5)))

    def powers(V, xp):
        P = [V * 0.0 + 1.0]
        for _ in range(4):
            P.append(P[-1] * V)
        return P

    def u(X, Y, Z, xp):
        PX, PY, PZ = powers(X, xp), powers(Y, xp), powers(Z, xp)
        s = X * 0.0
        for a in range(5):
            for b in range(5):
                for c in range(5):
                    if coef[a, b, c] != 0.0:
                        s = s + coef[a, b, c] * PX[a] * PY[b] * PZ[c]
        return s

    def f(X, Y, Z, xp):
        PX, PY, PZ = powers(X, xp), powers(Y, xp), powers(Z, xp)
        s = X * 0.0
        for a in range(5):
            for b in range(5):
                for c in range(5):
                    k = coef[a, b, c]
                    if a >= 2:
                        s = s + k * a * (a - 1) * PX[a - 2] * PY[b] * PZ[c]
                    if b >= 2:
                        s = s + k * b * (b - 1) * PX[a] * PY[b - 2] * PZ[c]
                    if c >= 2:
                        s = s + k * c * (c - 1) * PX[a] * PY[b] * PZ[c - 2]
        return s

    return u, f


# ------------------------------------------------------------- workloads
def config1(n: int = 33) -> Workload:
    """Unit cube, uniform, no body, u = sin(pi x) sin(pi y) sin(pi z)."""
    x = uniform_grid(0.0, 1.0, n)
    return Workload("uniform-%d^3-nobody" % n, x, x.copy(), x.copy(), [], _sinpi3, _sinpi3_f, tol=1e-12)


def config2(n: int = 129, beta: float = 1.5) -> Workload:
    """[-1,1]^3, tanh-stretched toward the centre (factor 1.5 per axis),
    sphere r = 0.3 at (0.05, -0.03, 0.02); u = e^x sin y cos 2z + x^2 y."""
    x = tanh_grid(-1.0, 1.0, n, beta)
    return Workload("tanh%.1f-%d^3-sphere" % (beta, n), x, x.copy(), x.copy(),
                    [sphere((0.05, -0.03, 0.02), 0.3)], _c2_u, _c2_f, tol=1e-12)


def config3_bodies():
    return [ellipsoid((0.0, 0.0, 0.0), (0.4, 0.25, 0.2), rot_z(30.0)),
            torus((0.5, 0.4, -0.3), 0.3, 0.1)]


def config3(n: int = 513) -> Workload:
    """[-1,1]^3, tanh factors (2.0, 1.2, 1.2); an ellipsoid (0.4, 0.25, 0.2)
    rotated 30 degrees about z at the origin and a torus R = 0.3, r = 0.1 at
    (0.5, 0.4, -0.3) with its axis along z; u = sin 2x cosh y exp(-z^2)."""
    return Workload("tanh(2.0,1.2,1.2)-%d^3-ellipsoid+torus" % n,
                    tanh_grid(-1.0, 1.0, n, 2.0), tanh_grid(-1.0, 1.0, n, 1.2), tanh_grid(-1.0, 1.0, n, 1.2),
                    config3_bodies(), _c3_u, _c3_f, tol=1e-12)


def paper_problem1(n: int, bodies=()) -> Workload:
    """Problem 1 of Sec. 4: u = sin(2 pi x) cos(2 pi y) cos(2 pi z) on the
    uniform unit cube."""
    x = uniform_grid(0.0, 1.0, n)
    return Workload("p1-%d^3" % n, x, x.copy(), x.copy(), list(bodies), _p1_u, _p1_f)


def interior_sphere(n: int = 41) -> Workload:
    """Interior problem (fluid inside the body, as in Problem 4 of Sec. 4):
    a sphere of radius 0.72 centred near the middle of [-1,1]^3,
    u = exp(-(x^2 + y^2 + z^2)) on it and on Gamma."""
    x = tanh_grid(-1.0, 1.0, n, 0.8)

    def u(X, Y, Z, xp):
        return xp.exp(-(X * X + Y * Y + Z * Z))

    def f(X, Y, Z, xp):
        r2 = X * X + Y * Y + Z * Z
        return (4.0 * r2 - 6.0) * xp.exp(-r2)

    return Workload("interior-sphere-%d^3" % n, x, x.copy(), x.copy(), [sphere((0.02, -0.01, 0.03), 0.72)], u, f,
                    fluid_inside=True)


def quartic_workload(x, y, z, bodies=(), seed=0, fluid_inside=False) -> Workload:
    u, f = quartic(seed)
    return Workload("quartic", np.asarray(x, float), np.asarray(y, float), np.asarray(z, float),
                    list(bodies), u, f, fluid_inside=fluid_inside)


def _cells_inside(grid: np.ndarray, lo: float, hi: float, margin: int) -> bool:
    """True if [lo, hi] lies between grid nodes margin and n-1-margin."""
    return lo >= grid[margin] and hi <= grid[grid.size - 1 - margin]


def _local_h(grid: np.ndarray, lo: float, hi: float) -> float:
    """Largest spacing of the grid cells that meet [lo, hi]."""
    a = max(int(np.searchsorted(grid, lo)) - 1, 0)
    b = min(int(np.searchsorted(grid, hi)) + 1, grid.size - 1)
    return float(np.max(np.diff(grid[a:b + 1])))


BODY_CLEARANCE_CELLS = 3


def random_problem(seed: int, sizes=(33, 49, 65, 97, 129)) -> Workload:
    """One problem of the batched workload: n drawn from ``sizes`` (same on
    each axis), tanh factors U[1,2] per axis, 1-3 spheres/ellipsoids with
    radii in [0.1, 0.3] and random rotations, f = sum of 8 random Fourier
    modes with wavenumbers 1..6 and N(0,1) amplitudes, g = 0.

    Clearance is counted in cells of the stretched grid itself: the bounding
    box of every body (its centre +- its largest semi-axis) lies between the
    nodes 3 and n-4 of each axis (the batched workload's ">= 3 cells from the
    box"), and the surfaces of two bodies are at least 3 of the largest local
    cells apart (the cells of each axis over the interval the two bodies
    span).  A moment-matched stencil of Secs. 2.2-2.3 reaches five nodes past
    its irregular point, so near the box or another body some of them end
    early (the degenerate operators the library counts).  A candidate body that breaks a rule is
    redrawn (centre, radii, rotation); if the bodies still cannot be placed,
    the stretching factors are redrawn; a seed for which nothing fits raises
    ValueError instead of returning fewer bodies."""
    rng = np.random.default_rng(seed)
    n = int(rng.choice(sizes))
    nb = int(rng.integers(1, 4))
    m = BODY_CLEARANCE_CELLS
    for _attempt in range(50):
        betas = rng.uniform(1.0, 2.0, 3)
        x = tanh_grid(-1.0, 1.0, n, betas[0])
        y = tanh_grid(-1.0, 1.0, n, betas[1])
        z = tanh_grid(-1.0, 1.0, n, betas[2])
        axes = (x, y, z)
        placed = []  # (body, centre, bounding radius)
        for _ in range(400):
            if len(placed) == nb:
                break
            r = rng.uniform(0.1, 0.3, 3)
            kind = "sphere" if rng.random() < 0.5 else "ellipsoid"
            if kind == "sphere":
                r[:] = r[0]
            c = rng.uniform(-1.0, 1.0, 3)
            R = rot_euler(*rng.uniform(0, 2 * math.pi, 3))
            rad = float(np.max(r))
            if not all(_cells_inside(axes[d], c[d] - rad, c[d] + rad, m) for d in range(3)):
                continue
            ok = True
            for _b, c2, rad2 in placed:
                h = max(_local_h(axes[d], min(c[d] - rad, c2[d] - rad2), max(c[d] + rad, c2[d] + rad2))
                        for d in range(3))
                if np.linalg.norm(c - c2) - rad - rad2 < m * h:
                    ok = False
                    break
            if not ok:
                continue
            b = sphere(c, r[0]) if kind == "sphere" else ellipsoid(c, r, R)
            placed.append((b, c, rad))
        if len(placed) == nb:
            break
    else:
        raise ValueError("random_problem(seed=%d): could not place %d bodies on the %d^3 grid" % (seed, nb, n))
    bodies = [b for b, _c, _r in placed]
    k = rng.integers(1, 7, (8, 3)).astype(np.float64)
    amp = rng.standard_normal(8)
    ph = rng.uniform(0, 2 * math.pi, 8)

    def f(X, Y, Z, xp):
        s = X * 0.0
        for m in range(8):
            s = s + amp[m] * xp.sin(k[m, 0] * X + k[m, 1] * Y + k[m, 2] * Z + ph[m])
        return s

    def u(X, Y, Z, xp):
        return X * 0.0

    return Workload("random-%d-n%d" % (seed, n), x, y, z, bodies, u, f, tol=1e-10, meta={"seed": seed})
