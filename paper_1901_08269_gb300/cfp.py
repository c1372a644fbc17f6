"""Thin ctypes binding of ``libcfp.so`` (C ABI in include/cfp.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Fields are torch CUDA tensors of dtype float64 with N = nx*ny*nz
elements in x-fastest order (any shape; they must be contiguous).  The
library fails loudly (ImportError / CfpError) when it cannot be loaded.
"""
import ctypes as C
import os

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, EGEOM, ENOCONV, EBREAKDOWN, ENAN, ESTATE = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EGEOM", "ENOCONV", "EBREAKDOWN", "ENAN", "ESTATE"]
BOUNDARY, REGULAR, IRREGULAR, SOLID = 0, 1, 2, 3
PREC_FP64, PREC_MIXED = 0, 1
PRECOND_RBGS, PRECOND_MG, PRECOND_ILU = 0, 1, 2
KINDS = {"sphere": 0, "ellipsoid": 1, "torus": 2}


class CfpError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s: %s" % (what, name, last_error()))


class Body(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_double * 3), ("R", C.c_double * 9), ("p", C.c_double * 3)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("sweeps", C.c_int), ("maxit", C.c_int), ("max_restarts", C.c_int),
                ("inner_tol", C.c_double), ("max_refine", C.c_int), ("use_graph", C.c_int),
                ("precond", C.c_int), ("mg_smooth", C.c_int), ("mg_post", C.c_int), ("mg_tma", C.c_int)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("restarts", C.c_int), ("refinements", C.c_int),
                ("rel_residual", C.c_double), ("n_irregular", C.c_int64), ("n_ibi", C.c_int64),
                ("n_degenerate", C.c_int64), ("ms_setup", C.c_double), ("ms_rhs", C.c_double),
                ("ms_solve", C.c_double), ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)

EXPORTS = ["cfp_default_opts", "cfp_last_error", "cfp_ctx_create", "cfp_ctx_destroy", "cfp_classify_points",
           "cfp_ibi_points", "cfp_assemble_rhs", "cfp_apply", "cfp_precondition", "cfp_solve", "cfp_solve_host",
           "cfp_time_kernel", "cfp_launch_count", "cfp_assemble_rhs_noalloc", "cfp_precondition_ex",
           "cfp_solve_batch", "cfp_autotune", "cfp_diag_bounded_wait", "cfp_nn_pack", "cfp_nn_conv3d",
           "cfp_nn_conv3d_dgrad", "cfp_nn_conv3d_wgrad", "cfp_nn_mse", "cfp_nn_adam", "cfp_nn_unpack",
           "cfp_vec_dot", "cfp_vec_axpby"]
KERNEL_APPLY, KERNEL_RBGS, KERNEL_UPDATE, KERNEL_MG_SWEEP = 0, 1, 2, 3


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libcfp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError("libcfp.so not found at %s (run __graft_entry__.build())" % path)
        L = C.CDLL(path)
        L.cfp_default_opts.argtypes = [C.POINTER(Opts)]
        L.cfp_last_error.restype = C.c_char_p
        L.cfp_ctx_create.argtypes = [_D, C.c_int, _D, C.c_int, _D, C.c_int, C.POINTER(Body), C.c_int, C.c_int,
                                     _P, C.POINTER(_P)]
        L.cfp_ctx_destroy.argtypes = [_P]
        L.cfp_classify_points.argtypes = [_P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.cfp_ibi_points.argtypes = [_P, _P, C.c_int]
        L.cfp_assemble_rhs.argtypes = [_P, _P, _P, _P, _P]
        L.cfp_apply.argtypes = [_P, _P, _P]
        L.cfp_precondition.argtypes = [_P, C.c_int, _P, _P]
        L.cfp_solve.argtypes = [_P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), C.POINTER(Info)]
        L.cfp_solve_host.argtypes = [_P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), C.POINTER(Info)]
        L.cfp_time_kernel.argtypes = [_P, C.c_int, C.c_int, C.c_int, _D, _D]
        L.cfp_assemble_rhs_noalloc.argtypes = [_P, _P, _P, _P, _P]
        L.cfp_precondition_ex.argtypes = [_P, C.POINTER(Opts), _P, _P]
        L.cfp_solve_batch.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                      C.POINTER(_P), C.c_double, C.POINTER(Opts), C.c_int, C.POINTER(Info)]
        L.cfp_autotune.argtypes = [_P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), _D]
        L.cfp_launch_count.argtypes = [_P]
        L.cfp_launch_count.restype = C.c_int64
        L.cfp_diag_bounded_wait.argtypes = [_P]
        L.cfp_nn_pack.argtypes = [_P, _P, _P, C.c_double, C.c_double, _P, _P, _P, _D]
        L.cfp_nn_conv3d.argtypes = [_P, _P, _P, _P, C.c_int, _P, _P]
        L.cfp_nn_conv3d_dgrad.argtypes = [_P, _P, _P, _P, _P]
        L.cfp_nn_conv3d_wgrad.argtypes = [_P, _P, _P, _P, _P]
        L.cfp_nn_mse.argtypes = [_P, _P, _P, _P, C.c_double, _P, _D]
        L.cfp_nn_adam.argtypes = [_P, C.c_int64, _P, _P, _P, _P, C.c_int, C.c_double, _P]
        L.cfp_nn_unpack.argtypes = [_P, _P, C.c_double, _P]
        L.cfp_vec_dot.argtypes = [_P, _P, _P, _D]
        L.cfp_vec_axpby.argtypes = [_P, C.c_double, _P, C.c_double, _P]
        for name in EXPORTS[2:]:
            if name not in ("cfp_ctx_destroy", "cfp_launch_count"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def last_error():
    return lib().cfp_last_error().decode() if _lib is not None else ""


def _check(st, what):
    if st != OK:
        raise CfpError(st, what)


def default_opts(**kw):
    o = Opts()
    lib().cfp_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_bodies(bodies):
    import numpy as np
    arr = (Body * max(len(bodies), 1))()
    for m, b in enumerate(bodies):
        arr[m].kind = KINDS[b["kind"]] if isinstance(b["kind"], str) else int(b["kind"])
        R = np.asarray(b.get("R", np.eye(3)), dtype=np.float64).reshape(9)
        for q in range(3):
            arr[m].c[q] = float(b["c"][q])
            arr[m].p[q] = float(b["p"][q]) if q < len(b["p"]) else 0.0
        for q in range(9):
            arr[m].R[q] = float(R[q])
    return arr, len(bodies)


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def solve_batch(ctxs, fs, gs, gis, us, tol=1e-12, opts=None, nthreads=0, check=True, **kw):
    """cfp_solve_batch over lists of contexts and CUDA float64 tensors."""
    n = len(ctxs)
    o = opts if opts is not None else default_opts(**kw)
    arr = lambda ts: (_P * max(n, 1))(*[_P(t.data_ptr()) if t is not None and t.numel() else None for t in ts])
    hs = (_P * max(n, 1))(*[c._h for c in ctxs])
    for c, f, g, u in zip(ctxs, fs, gs, us):
        c._field(f, "f"), c._field(g, "g_nodes"), c._field(u, "u")
    infos = (Info * max(n, 1))()
    st = lib().cfp_solve_batch(hs, n, arr(fs), arr(gs), arr(gis), arr(us), float(tol), C.byref(o), int(nthreads),
                               infos)
    if check:
        _check(st, "cfp_solve_batch")
    return [infos[m] for m in range(n)]


class Context:
    """One solver context (cfp_ctx) on the current CUDA device and stream."""

    def __init__(self, x, y, z, bodies=(), fluid_inside=False, stream=None):
        import numpy as np
        import torch
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        self.z = np.ascontiguousarray(z, dtype=np.float64)
        self.shape = (self.z.size, self.y.size, self.x.size)
        self.N = self.x.size * self.y.size * self.z.size
        arr, nb = make_bodies(list(bodies))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _P()
        st = lib().cfp_ctx_create(self.x.ctypes.data_as(_D), self.x.size, self.y.ctypes.data_as(_D), self.y.size,
                                  self.z.ctypes.data_as(_D), self.z.size, arr, nb, int(bool(fluid_inside)),
                                  _P(stream.cuda_stream), C.byref(h))
        _check(st, "cfp_ctx_create")
        self._h = h
        self.n_irregular = self.n_ibi = None

    # ---- the learned part (include/cfp_nn.h): activations are N x 16 bfloat16,
    # weights 16 x 27 x 16 bfloat16, all CUDA tensors; argument marshalling only
    def _nn(self, t, name, dtype, numel):
        if t is None or not t.is_cuda or t.dtype != dtype or t.numel() != numel:
            raise ValueError("%s must be a CUDA %s tensor with %d elements" % (name, dtype, numel))
        return _ptr(t)

    def nn_pack(self, r, e, scale, escale, x, target=None, mask=None):
        """Returns the scale used (scale <= 0: 1 / max |r| at the unknowns)."""
        import torch
        used = C.c_double()
        _check(lib().cfp_nn_pack(self._h, self._field(r, "r"), None if e is None else self._field(e, "e"),
                                 float(scale), float(escale), self._nn(x, "x", torch.bfloat16, 16 * self.N),
                                 None if target is None else self._nn(target, "target", torch.float32, self.N),
                                 None if mask is None else self._nn(mask, "mask", torch.float32, self.N),
                                 C.byref(used)), "cfp_nn_pack")
        return used.value

    def nn_conv3d(self, inp, w, bias, relu, out):
        import torch
        bf, f32 = (out, None) if out.dtype == torch.bfloat16 else (None, out)
        _check(lib().cfp_nn_conv3d(self._h, self._nn(inp, "in", torch.bfloat16, 16 * self.N),
                                   self._nn(w, "w", torch.bfloat16, 16 * 27 * 16),
                                   None if bias is None else self._nn(bias, "bias", torch.float32, 16), int(relu),
                                   None if bf is None else self._nn(bf, "out", torch.bfloat16, 16 * self.N),
                                   None if f32 is None else self._nn(f32, "out", torch.float32, 16 * self.N)),
               "cfp_nn_conv3d")
        return out

    def nn_dgrad(self, dout, w, act, din):
        import torch
        _check(lib().cfp_nn_conv3d_dgrad(self._h, self._nn(dout, "dout", torch.bfloat16, 16 * self.N),
                                         self._nn(w, "w", torch.bfloat16, 16 * 27 * 16),
                                         None if act is None else self._nn(act, "act", torch.bfloat16, 16 * self.N),
                                         self._nn(din, "din", torch.bfloat16, 16 * self.N)), "cfp_nn_conv3d_dgrad")
        return din

    def nn_wgrad(self, inp, dout, dw, db=None):
        import torch
        _check(lib().cfp_nn_conv3d_wgrad(self._h, self._nn(inp, "in", torch.bfloat16, 16 * self.N),
                                         self._nn(dout, "dout", torch.bfloat16, 16 * self.N),
                                         self._nn(dw, "dw", torch.float32, 16 * 27 * 16),
                                         None if db is None else self._nn(db, "db", torch.float32, 16)),
               "cfp_nn_conv3d_wgrad")

    def nn_mse(self, y, target, mask, inv_count, dout):
        import torch
        loss = C.c_double()
        _check(lib().cfp_nn_mse(self._h, self._nn(y, "y", torch.float32, 16 * self.N),
                                self._nn(target, "target", torch.float32, self.N),
                                self._nn(mask, "mask", torch.float32, self.N), float(inv_count),
                                self._nn(dout, "dout", torch.bfloat16, 16 * self.N), C.byref(loss)), "cfp_nn_mse")
        return loss.value

    def nn_adam(self, w, grad, m, v, step, lr, w_bf16=None):
        n = w.numel()
        for t in (grad, m, v):
            if t.numel() != n or not t.is_cuda:
                raise ValueError("Adam arrays must be CUDA tensors of equal size")
        _check(lib().cfp_nn_adam(self._h, n, _ptr(w), _ptr(grad), _ptr(m), _ptr(v), int(step), float(lr),
                                 _ptr(w_bf16)), "cfp_nn_adam")

    def nn_unpack(self, y, inv_scale, u):
        import torch
        _check(lib().cfp_nn_unpack(self._h, self._nn(y, "y", torch.float32, 16 * self.N), float(inv_scale),
                                   self._field(u, "u")), "cfp_nn_unpack")
        return u

    def vec_dot(self, a, b):
        out = C.c_double()
        _check(lib().cfp_vec_dot(self._h, self._field(a, "a"), self._field(b, "b"), C.byref(out)), "cfp_vec_dot")
        return out.value

    def vec_axpby(self, alpha, x, beta, y):
        _check(lib().cfp_vec_axpby(self._h, float(alpha), self._field(x, "x"), float(beta), self._field(y, "y")),
               "cfp_vec_axpby")
        return y

    def diag_bounded_wait(self):
        """(status, message) of cfp_diag_bounded_wait: CFP_ECUDA after about one
        second when the wait bound holds."""
        st = lib().cfp_diag_bounded_wait(self._h)
        return st, last_error()

    def close(self):
        if getattr(self, "_h", None):
            lib().cfp_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _field(self, t, name):
        import torch
        if t is None or not t.is_cuda or t.dtype != torch.float64 or t.numel() != self.N:
            raise ValueError("%s must be a CUDA float64 tensor with %d elements" % (name, self.N))
        return _ptr(t)

    def classify_points(self, type_out=None):
        ni, nb = C.c_int64(), C.c_int64()
        p = None
        if type_out is not None:
            import torch
            if not type_out.is_cuda or type_out.dtype != torch.uint8 or type_out.numel() != self.N:
                raise ValueError("type_out must be a CUDA uint8 tensor with N elements")
            p = _ptr(type_out)
        _check(lib().cfp_classify_points(self._h, p, C.byref(ni), C.byref(nb)), "cfp_classify_points")
        self.n_irregular, self.n_ibi = ni.value, nb.value
        return self.n_irregular, self.n_ibi

    def ibi_points(self, out=None):
        import torch
        if self.n_ibi is None:
            self.classify_points()
        if out is None:
            out = torch.empty((self.n_ibi, 3), dtype=torch.float64, device="cuda")
        on_host = 0 if out.is_cuda else 1
        _check(lib().cfp_ibi_points(self._h, _ptr(out), on_host), "cfp_ibi_points")
        return out

    def assemble_rhs(self, f, g_nodes, g_ibi, rhs):
        _check(lib().cfp_assemble_rhs(self._h, self._field(f, "f"), self._field(g_nodes, "g_nodes"),
                                      _ptr(g_ibi) if g_ibi is not None and g_ibi.numel() else None,
                                      self._field(rhs, "rhs")), "cfp_assemble_rhs")
        return rhs

    def assemble_rhs_noalloc(self, f, g_nodes, g_ibi, rhs):
        """cfp_assemble_rhs_noalloc: the right-hand side without any device
        allocation (grids of at most 2^22 nodes; see include/cfp.h)."""
        _check(lib().cfp_assemble_rhs_noalloc(self._h, self._field(f, "f"), self._field(g_nodes, "g_nodes"),
                                              _ptr(g_ibi) if g_ibi is not None and g_ibi.numel() else None,
                                              self._field(rhs, "rhs")), "cfp_assemble_rhs_noalloc")
        return rhs

    def apply(self, x, y):
        _check(lib().cfp_apply(self._h, self._field(x, "x"), self._field(y, "y")), "cfp_apply")
        return y

    def precondition(self, rho, phi, sweeps=8):
        _check(lib().cfp_precondition(self._h, int(sweeps), self._field(rho, "rho"), self._field(phi, "phi")),
               "cfp_precondition")
        return phi

    def precondition_ex(self, rho, phi, opts=None, **kw):
        o = opts if opts is not None else default_opts(**kw)
        _check(lib().cfp_precondition_ex(self._h, C.byref(o), self._field(rho, "rho"), self._field(phi, "phi")),
               "cfp_precondition_ex")
        return phi

    def solve(self, f, g_nodes, g_ibi, u, tol=1e-12, opts=None, check=True, **kw):
        o = opts if opts is not None else default_opts(**kw)
        info = Info()
        st = lib().cfp_solve(self._h, self._field(f, "f"), self._field(g_nodes, "g_nodes"),
                             _ptr(g_ibi) if g_ibi is not None and g_ibi.numel() else None,
                             self._field(u, "u"), float(tol), C.byref(o), C.byref(info))
        if check:
            _check(st, "cfp_solve")
        return info

    def launch_count(self):
        return lib().cfp_launch_count(self._h)

    def autotune(self, f, g_nodes, g_ibi, u, tol=1e-12, opts=None, **kw):
        """cfp_autotune: returns (best Opts, best time in ms)."""
        o = opts if opts is not None else default_opts(**kw)
        ms = C.c_double()
        _check(lib().cfp_autotune(self._h, self._field(f, "f"), self._field(g_nodes, "g_nodes"),
                                  _ptr(g_ibi) if g_ibi is not None and g_ibi.numel() else None,
                                  self._field(u, "u"), float(tol), C.byref(o), C.byref(ms)), "cfp_autotune")
        return o, ms.value

    def time_kernel(self, kernel, precision=PREC_FP64, reps=20):
        """Mean device time (ms) of one launch and its algorithmic bytes."""
        ms, by = C.c_double(), C.c_double()
        _check(lib().cfp_time_kernel(self._h, int(kernel), int(precision), int(reps), C.byref(ms), C.byref(by)),
               "cfp_time_kernel")
        return ms.value, by.value

    def solve_host(self, f, g_nodes, g_ibi, u, tol=1e-12, opts=None, check=True, **kw):
        """Host-buffer solve: f, g_nodes, g_ibi, u are CPU tensors (ideally
        pinned); copies in and out happen inside the library call."""
        o = opts if opts is not None else default_opts(**kw)
        info = Info()
        for t in (f, g_nodes, u):
            if t.is_cuda or t.numel() != self.N:
                raise ValueError("host tensors with N elements expected")
        st = lib().cfp_solve_host(self._h, _ptr(f), _ptr(g_nodes),
                                  _ptr(g_ibi) if g_ibi is not None and g_ibi.numel() else None,
                                  _ptr(u), float(tol), C.byref(o), C.byref(info))
        if check:
            _check(st, "cfp_solve_host")
        return info
