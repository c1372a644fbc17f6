"""ctypes wrapper around the CPU oracle (``oracle/cfo.c``).

TEST INFRASTRUCTURE ONLY.  Every array is a host numpy array over the full
grid (node (i,j,k) at linear index i + nx*(j + ny*k), x fastest).
"""
import ctypes as C

import numpy as np

from . import build as _build

BOUNDARY, REGULAR, IRREGULAR, SOLID = 0, 1, 2, 3
MAT_B, MAT_BIBI, MAT_K, MAT_KIBI = 0, 1, 2, 3
PRECOND_RBGS, PRECOND_ILU = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 4: "EGEOM", 5: "ENOCONV", 6: "EBREAKDOWN", 7: "ENAN"}
KINDS = {"sphere": 0, "ellipsoid": 1, "torus": 2}


class _Body(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_double * 3), ("R", C.c_double * 9), ("p", C.c_double * 3)]


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.cfo_create.argtypes = [_D, C.c_int, _D, C.c_int, _D, C.c_int, C.POINTER(_Body), C.c_int,
                                 C.c_int, C.POINTER(C.c_void_p)]
        L.cfo_destroy.argtypes = [C.c_void_p]
        L.cfo_error.argtypes = [C.c_void_p]
        L.cfo_error.restype = C.c_char_p
        L.cfo_threads.restype = C.c_int
        L.cfo_compact_coefs.argtypes = [_D, C.c_int, _D, _D, _D, _D, _D]
        L.cfo_second_coefs.argtypes = [_D, C.c_int, _D, _D, _D]
        L.cfo_phi.argtypes = [C.POINTER(_Body), C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        L.cfo_phi.restype = C.c_double
        L.cfo_line_operator.argtypes = [C.c_int, _D, C.c_double, C.c_int, _D, _D, C.c_double, _D]
        L.cfo_classify.argtypes = [C.c_void_p, C.POINTER(C.c_uint8), _I64, _I64]
        L.cfo_ibi.argtypes = [C.c_void_p, _I64, _D, _D]
        L.cfo_assemble.argtypes = [C.c_void_p]
        L.cfo_nnz.argtypes = [C.c_void_p, C.c_int]
        L.cfo_nnz.restype = C.c_int64
        L.cfo_degenerate.argtypes = [C.c_void_p]
        L.cfo_degenerate.restype = C.c_int64
        L.cfo_export.argtypes = [C.c_void_p, C.c_int, _I64, C.POINTER(C.c_int32), _D]
        L.cfo_apply_B.argtypes = [C.c_void_p, _D, _D]
        L.cfo_apply_B_abs.argtypes = [C.c_void_p, _D, _D]
        L.cfo_rhs.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.cfo_rows.argtypes = [C.c_void_p, C.c_int64, _I64, _D, _D, _D, _D, _D, _D, _D, _I64]
        L.cfo_precond.argtypes = [C.c_void_p, C.c_int, _D, _D]
        L.cfo_precond_ilu.argtypes = [C.c_void_p, C.c_int, _D, _D]
        L.cfo_set_precond.argtypes = [C.c_void_p, C.c_int]
        L.cfo_ilu_pivots.argtypes = [C.c_void_p, _D]
        L.cfo_bicgstab.argtypes = [C.c_void_p, _D, _D, C.c_double, C.c_int, C.c_int,
                                   C.POINTER(C.c_int), _D]
        L.cfo_solve.argtypes = [C.c_void_p, _D, _D, _D, _D, C.c_double, C.c_int, C.c_int,
                                C.POINTER(C.c_int), _D]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_bodies(bodies):
    """bodies: sequence of dicts {kind, c, R (3x3 body->world), p}."""
    n = len(bodies)
    arr = (_Body * max(n, 1))()
    for m, b in enumerate(bodies):
        arr[m].kind = KINDS[b["kind"]] if isinstance(b["kind"], str) else int(b["kind"])
        for q in range(3):
            arr[m].c[q] = float(b["c"][q])
            arr[m].p[q] = float(b["p"][q]) if q < len(b["p"]) else 0.0
        R = np.asarray(b.get("R", np.eye(3)), dtype=np.float64).reshape(9)
        for q in range(9):
            arr[m].R[q] = float(R[q])
    return arr, n


class OracleError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def compact_coefs(x):
    x = _f64(x)
    n = x.size
    out = [np.zeros(n) for _ in range(5)]
    lib().cfo_compact_coefs(_dp(x), n, *[_dp(o) for o in out])
    return tuple(out)  # a, c, ar, br, cr


def second_coefs(x):
    x = _f64(x)
    n = x.size
    out = [np.zeros(n) for _ in range(3)]
    lib().cfo_second_coefs(_dp(x), n, *[_dp(o) for o in out])
    return tuple(out)  # a, b, c


def phi(bodies, x, y, z, fluid_inside=False):
    arr, n = make_bodies(bodies)
    return lib().cfo_phi(arr, n, int(fluid_inside), float(x), float(y), float(z))


def line_operator(xi, xe, xs, Ls, hs=None):
    xi = _f64(xi)
    xs = _f64(xs)
    Ls = _f64(Ls)
    M = xi.size
    if hs is None:
        hs = float(np.max(np.abs(xi - xe)))
    c = np.zeros(M)
    st = lib().cfo_line_operator(M, _dp(xi), float(xe), xs.size, _dp(xs), _dp(Ls), float(hs), _dp(c))
    if st:
        raise OracleError(st, "line operator")
    return c


class Problem:
    def __init__(self, x, y, z, bodies=(), fluid_inside=False):
        self.x, self.y, self.z = _f64(x), _f64(y), _f64(z)
        self.nx, self.ny, self.nz = self.x.size, self.y.size, self.z.size
        self.N = self.nx * self.ny * self.nz
        self.shape = (self.nz, self.ny, self.nx)
        arr, n = make_bodies(list(bodies))
        h = C.c_void_p()
        st = lib().cfo_create(_dp(self.x), self.nx, _dp(self.y), self.ny, _dp(self.z), self.nz,
                              arr, n, int(fluid_inside), C.byref(h))
        if st:
            raise OracleError(st, "create")
        self._h = h
        self.type = None
        self.n_irr = self.n_ibi = None
        self.assembled = False

    def __del__(self):
        if getattr(self, "_h", None):
            lib().cfo_destroy(self._h)
            self._h = None

    def _check(self, st, what):
        if st:
            raise OracleError(st, "%s: %s" % (what, lib().cfo_error(self._h).decode()))

    def classify(self):
        t = np.zeros(self.N, dtype=np.uint8)
        ni, nb = C.c_int64(), C.c_int64()
        self._check(lib().cfo_classify(self._h, t.ctypes.data_as(C.POINTER(C.c_uint8)),
                                       C.byref(ni), C.byref(nb)), "classify")
        self.type, self.n_irr, self.n_ibi = t, ni.value, nb.value
        return t

    def ibi(self):
        if self.type is None:
            self.classify()
        n = self.n_ibi
        key = np.zeros(n, dtype=np.int64)
        t = np.zeros(n)
        xyz = np.zeros((n, 3))
        self._check(lib().cfo_ibi(self._h, key.ctypes.data_as(_I64), _dp(t), _dp(xyz)), "ibi")
        return key, t, xyz

    def assemble(self):
        if self.type is None:
            self.classify()
        self._check(lib().cfo_assemble(self._h), "assemble")
        self.assembled = True

    def export(self, which=MAT_B):
        """The full-grid CSR (rows and columns over all N nodes; the IBI
        matrices have n_ibi columns) as a scipy.sparse.csr_matrix."""
        import scipy.sparse as sp
        if not self.assembled:
            self.assemble()
        nnz = lib().cfo_nnz(self._h, which)
        ptr = np.zeros(self.N + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1))
        self._check(lib().cfo_export(self._h, which, ptr.ctypes.data_as(_I64),
                                     col.ctypes.data_as(C.POINTER(C.c_int32)), _dp(val)), "export")
        ncol = self.N if which in (MAT_B, MAT_K) else max(self.n_ibi, 1)
        return sp.csr_matrix((val[:nnz], col[:nnz], ptr), shape=(self.N, ncol))

    def degenerate(self):
        return lib().cfo_degenerate(self._h)

    def unknowns(self):
        if self.type is None:
            self.classify()
        return np.flatnonzero((self.type == REGULAR) | (self.type == IRREGULAR))

    def apply_B(self, x, absval=False):
        if not self.assembled:
            self.assemble()
        x = _f64(x).reshape(-1)
        y = np.zeros(self.N)
        (lib().cfo_apply_B_abs if absval else lib().cfo_apply_B)(self._h, _dp(x), _dp(y))
        return y

    def rhs(self, f, g_nodes, g_ibi):
        if not self.assembled:
            self.assemble()
        f = _f64(f).reshape(-1)
        g = _f64(g_nodes).reshape(-1)
        gi = _f64(g_ibi).reshape(-1) if self.n_ibi else np.zeros(1)
        out = np.zeros(self.N)
        self._check(lib().cfo_rhs(self._h, _dp(f), _dp(g), _dp(gi), _dp(out)), "rhs")
        return out

    def rows(self, rows, x=None, f=None, g_nodes=None, g_ibi=None):
        """B x, sum |B||x| and the right-hand side at the nodes ``rows``
        (linear indices), each row built as the full assembly builds it but
        without assembling the system.  Returns (Bx, |B||x|, rhs,
        n_degenerate); an output whose inputs are None is None."""
        if self.type is None:
            self.classify()
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        n = rows.size
        want_b = x is not None
        want_r = f is not None
        xs = _f64(x).reshape(-1) if want_b else None
        fs = _f64(f).reshape(-1) if want_r else None
        gs = _f64(g_nodes).reshape(-1) if want_r else None
        gi = (_f64(g_ibi).reshape(-1) if self.n_ibi else np.zeros(1)) if want_r else None
        bx = np.zeros(n) if want_b else None
        ba = np.zeros(n) if want_b else None
        rh = np.zeros(n) if want_r else None
        ndeg = C.c_int64()
        nul = C.cast(None, _D)
        self._check(lib().cfo_rows(self._h, n, rows.ctypes.data_as(_I64), _dp(xs) if want_b else nul,
                                   _dp(fs) if want_r else nul, _dp(gs) if want_r else nul,
                                   _dp(gi) if want_r else nul, _dp(bx) if want_b else nul,
                                   _dp(ba) if want_b else nul, _dp(rh) if want_r else nul, C.byref(ndeg)),
                    "rows")
        return bx, ba, rh, ndeg.value

    def precond(self, rho, sweeps=8, kind=PRECOND_RBGS):
        """sweeps inner iterations on K from phi = 0 (red-black Gauss-Seidel
        or ILU(0)-Richardson)."""
        if not self.assembled:
            self.assemble()
        rho = _f64(rho).reshape(-1)
        out = np.zeros(self.N)
        fn = lib().cfo_precond_ilu if kind == PRECOND_ILU else lib().cfo_precond
        fn(self._h, int(sweeps), _dp(rho), _dp(out))
        return out

    def ilu_pivots(self):
        if not self.assembled:
            self.assemble()
        out = np.zeros(self.N)
        self._check(lib().cfo_ilu_pivots(self._h, _dp(out)), "ilu_pivots")
        return out

    def set_precond(self, kind):
        """inner iteration used by bicgstab / solve (PRECOND_RBGS or PRECOND_ILU)"""
        lib().cfo_set_precond(self._h, int(kind))

    def bicgstab(self, rhs, x0=None, tol=1e-12, maxit=10000, sweeps=8):
        if not self.assembled:
            self.assemble()
        rhs = _f64(rhs).reshape(-1)
        x = np.zeros(self.N) if x0 is None else _f64(x0).reshape(-1).copy()
        it, rel = C.c_int(), C.c_double()
        st = lib().cfo_bicgstab(self._h, _dp(rhs), _dp(x), float(tol), int(maxit), int(sweeps),
                                C.byref(it), C.byref(rel))
        return x, st, it.value, rel.value

    def solve(self, f, g_nodes, g_ibi, u0=None, tol=1e-12, maxit=10000, sweeps=8):
        """Full solve; returns (u, status, iterations, true relative residual)."""
        if self.type is None:
            self.classify()
        f = _f64(f).reshape(-1)
        g = _f64(g_nodes).reshape(-1)
        gi = _f64(g_ibi).reshape(-1) if self.n_ibi else np.zeros(1)
        u = np.zeros(self.N) if u0 is None else _f64(u0).reshape(-1).copy()
        it, rel = C.c_int(), C.c_double()
        st = lib().cfo_solve(self._h, _dp(f), _dp(g), _dp(gi), _dp(u), float(tol), int(maxit),
                             int(sweeps), C.byref(it), C.byref(rel))
        self.assembled = True
        return u, st, it.value, rel.value


def threads():
    return lib().cfo_threads()
