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
           "cfp_ibi_points", "cfp_assemble_rhs", "cfp_apply", "cfp_apply_f32", "cfp_precondition", "cfp_solve", "cfp_solve_host",
           "cfp_time_kernel", "cfp_launch_count", "cfp_assemble_rhs_noalloc", "cfp_precondition_ex",
           "cfp_solve_batch", "cfp_apply_shape", "cfp_batch_create", "cfp_batch_run", "cfp_batch_destroy", "cfp_autotune", "cfp_diag_bounded_wait", "cfp_vec_dot", "cfp_vec_axpby",
           "cfp_nn_conv3d", "cfp_nn_conv3d_wgrad", "cfp_nn_transfer", "cfp_unet_create", "cfp_unet_destroy",
           "cfp_unet_param_count", "cfp_unet_get_params", "cfp_unet_set_params", "cfp_unet_forward_raw",
           "cfp_unet_train_step", "cfp_unet_apply", "cfp_unet_check", "cfp_solve_fgmres", "cfp_tune_apply"]
NN_RELU, NN_MASK, NN_OUT_F32, NN_ACCUM, NN_DGRAD = 1, 2, 4, 8, 16
NN_INJECT, NN_PROLONG_ADD, NN_PROLONG_T, NN_SKIP_GRAD = 0, 1, 2, 3
KERNEL_APPLY, KERNEL_RBGS, KERNEL_UPDATE, KERNEL_MG_SWEEP, KERNEL_PROLONG, KERNEL_RESTRICT = 0, 1, 2, 3, 4, 5
KERNEL_MG_PAIR = 6
APPLY_STREAM, APPLY_RING = 1, 2


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
        L.cfp_apply_f32.argtypes = [_P, _P, _P]
        L.cfp_precondition.argtypes = [_P, C.c_int, _P, _P]
        L.cfp_solve.argtypes = [_P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), C.POINTER(Info)]
        L.cfp_solve_host.argtypes = [_P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), C.POINTER(Info)]
        L.cfp_time_kernel.argtypes = [_P, C.c_int, C.c_int, C.c_int, _D, _D]
        L.cfp_assemble_rhs_noalloc.argtypes = [_P, _P, _P, _P, _P]
        L.cfp_precondition_ex.argtypes = [_P, C.POINTER(Opts), _P, _P]
        L.cfp_solve_batch.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                      C.POINTER(_P), C.c_double, C.POINTER(Opts), C.c_int, C.POINTER(Info)]
        L.cfp_batch_create.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                       C.POINTER(_P), C.c_double, C.POINTER(Opts), C.POINTER(_P)]
        L.cfp_batch_run.argtypes = [_P, C.POINTER(Info)]
        L.cfp_batch_destroy.argtypes = [_P]
        L.cfp_batch_destroy.restype = None
        L.cfp_autotune.argtypes = [_P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), _D]
        L.cfp_launch_count.argtypes = [_P]
        L.cfp_launch_count.restype = C.c_int64
        L.cfp_diag_bounded_wait.argtypes = [_P]
        L.cfp_tune_apply.argtypes = [_P, C.c_int, C.c_int, C.c_int, C.c_int, _D]
        L.cfp_apply_shape.argtypes = [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.cfp_vec_dot.argtypes = [_P, _P, _P, _D]
        L.cfp_vec_axpby.argtypes = [_P, C.c_double, _P, C.c_double, _P]
        _I = C.c_int
        L.cfp_nn_conv3d.argtypes = [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P, _I, _P]
        L.cfp_nn_conv3d_wgrad.argtypes = [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P]
        L.cfp_nn_transfer.argtypes = [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P]
        L.cfp_unet_create.argtypes = [_P, C.c_uint64, C.POINTER(_P)]
        L.cfp_unet_destroy.argtypes = [_P]
        L.cfp_unet_destroy.restype = None
        L.cfp_unet_param_count.argtypes = []
        L.cfp_unet_param_count.restype = C.c_int64
        L.cfp_unet_get_params.argtypes = [_P, _P, _P]
        L.cfp_unet_set_params.argtypes = [_P, _P]
        L.cfp_unet_forward_raw.argtypes = [_P, _I, _I, _I, _P, _P, _P, _I, _P, _D]
        L.cfp_unet_train_step.argtypes = [_P, _P, _P, _P, C.c_double, _D]
        L.cfp_unet_apply.argtypes = [_P, _P, _P, _P]
        L.cfp_unet_check.argtypes = [_P]
        L.cfp_solve_fgmres.argtypes = [_P, _P, _P, _P, _P, _P, C.c_double, C.POINTER(Opts), _I, _I,
                                       C.POINTER(Info)]
        for name in EXPORTS[2:]:
            if name not in ("cfp_ctx_destroy", "cfp_launch_count", "cfp_unet_destroy", "cfp_unet_param_count"):
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


class Batch:
    """cfp_batch: the problems' mixed-precision solves as one graph launch.
    opts: None, one Opts for all problems or a list of one per problem.  The
    tensors must stay alive while the batch does."""

    def __init__(self, ctxs, fs, gs, gis, us, tol=1e-12, opts=None, **kw):
        n = len(ctxs)
        if opts is None:
            opts = default_opts(**kw)
        if isinstance(opts, Opts):
            opts = [opts] * n
        for c, f, g, u in zip(ctxs, fs, gs, us):
            c._field(f, "f"), c._field(g, "g_nodes"), c._field(u, "u")
        arr = lambda ts: (_P * n)(*[_P(t.data_ptr()) if t is not None and t.numel() else None for t in ts])
        self._keep = (list(ctxs), list(fs), list(gs), list(gis), list(us))
        self.n = n
        olist = (Opts * n)(*opts)
        h = _P()
        _check(lib().cfp_batch_create((_P * n)(*[c._h for c in ctxs]), n, arr(fs), arr(gs), arr(gis), arr(us),
                                      float(tol), olist, C.byref(h)), "cfp_batch_create")
        self._h = h

    def run(self, check=True):
        infos = (Info * self.n)()
        st = lib().cfp_batch_run(self._h, infos)
        if check:
            _check(st, "cfp_batch_run")
        return [infos[m] for m in range(self.n)]

    def close(self):
        if getattr(self, "_h", None):
            lib().cfp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


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

    # ---- the learned part's single kernels (include/cfp_nn.h): padded,
    # channels-last bfloat16 activations on an nx x ny x nz grid; argument
    # marshalling only
    @staticmethod
    def _bf(t, name, numel, dtype=None):
        import torch
        dtype = dtype or torch.bfloat16
        if t is None or not t.is_cuda or t.dtype != dtype or t.numel() != numel:
            raise ValueError("%s must be a CUDA %s tensor with %d elements" % (name, dtype, numel))
        return _ptr(t)

    def nn_conv3d(self, dims, cin, cout, inp, w, out, bias=None, act=None, flags=0):
        """out = epilogue(conv(inp, w) + bias) on the grid dims = (nx, ny, nz)."""
        import torch
        nx, ny, nz = dims
        npad = (nx + 2) * (ny + 2) * (nz + 2)
        f32 = bool(flags & NN_OUT_F32)
        _check(lib().cfp_nn_conv3d(self._h, nx, ny, nz, cin, cout, self._bf(inp, "in", npad * cin),
                                   self._bf(w, "w", cout * 27 * cin),
                                   None if bias is None else self._bf(bias, "bias", cout, torch.float32),
                                   None if act is None else self._bf(act, "act", npad * cout), int(flags),
                                   self._bf(out, "out", npad * cout, torch.float32 if f32 else torch.bfloat16)),
               "cfp_nn_conv3d")
        return out

    def nn_wgrad(self, dims, cin, cout, inp, gout, dw, db=None):
        import torch
        nx, ny, nz = dims
        npad = (nx + 2) * (ny + 2) * (nz + 2)
        _check(lib().cfp_nn_conv3d_wgrad(self._h, nx, ny, nz, cin, cout, self._bf(inp, "in", npad * cin),
                                         self._bf(gout, "gout", npad * cout),
                                         self._bf(dw, "dw", cout * 27 * cin, torch.float32),
                                         None if db is None else self._bf(db, "db", cout, torch.float32)),
               "cfp_nn_conv3d_wgrad")

    def nn_transfer(self, kind, dims, c, a, out, b=None, act=None):
        for t in (a, out, b, act):
            if t is not None and (not t.is_cuda or not t.is_contiguous()):
                raise ValueError("transfer operands must be contiguous CUDA tensors")
        nx, ny, nz = dims
        _check(lib().cfp_nn_transfer(self._h, int(kind), nx, ny, nz, c, _ptr(a), _ptr(b), _ptr(act), _ptr(out)),
               "cfp_nn_transfer")
        return out

    def solve_fgmres(self, f, g_nodes, g_ibi, u, tol=1e-10, net=None, m=20, net_guess=False, opts=None,
                     check=True, **kw):
        """cfp_solve_fgmres: flexible GMRES(m), with the network `net`
        (UNet or None) in its preconditioner."""
        o = opts if opts is not None else default_opts(**kw)
        info = Info()
        st = lib().cfp_solve_fgmres(self._h, None if net is None else net._h, self._field(f, "f"),
                                    self._field(g_nodes, "g_nodes"),
                                    None if g_ibi is None or g_ibi.numel() == 0 else _ptr(g_ibi),
                                    self._field(u, "u"), float(tol), C.byref(o), int(m), int(bool(net_guess)),
                                    C.byref(info))
        if check:
            _check(st, "cfp_solve_fgmres")
        return info

    def tune_apply(self, precision=PREC_MIXED, rows=0, planes=0, kernel=None):
        """cfp_tune_apply: the apply's kernel and tile shape (all 0:
        autotuned; kernel defaults to APPLY_STREAM when a shape is given);
        returns the chosen one's ms per launch."""
        if kernel is None:
            kernel = 0 if not (rows or planes) else APPLY_STREAM
        ms = C.c_double()
        _check(lib().cfp_tune_apply(self._h, int(precision), int(kernel), int(rows), int(planes), C.byref(ms)),
               "cfp_tune_apply")
        return ms.value

    def apply_shape(self, precision=PREC_MIXED):
        """cfp_apply_shape: (kernel, rows, planes) the apply runs with."""
        k, r, q = C.c_int(), C.c_int(), C.c_int()
        _check(lib().cfp_apply_shape(self._h, int(precision), C.byref(k), C.byref(r), C.byref(q)), "cfp_apply_shape")
        return k.value, r.value, q.value

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

    def _field(self, t, name, dtype=None):
        import torch
        dtype = torch.float64 if dtype is None else dtype
        if t is None or not t.is_cuda or t.dtype != dtype or t.numel() != self.N:
            raise ValueError("%s must be a CUDA %s tensor with %d elements" % (name, dtype, self.N))
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

    def apply_f32(self, x, y):
        """cfp_apply_f32: y = B x in FP32 (float32 tensors)."""
        import torch
        _check(lib().cfp_apply_f32(self._h, self._field(x, "x", torch.float32), self._field(y, "y", torch.float32)),
               "cfp_apply_f32")
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
        """Host-buffer solve: f, g_nodes, g_ibi, u are CPU tensors; pinned
        ones are read and written in place by the kernels, others are copied
        in and out inside the library call."""
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


class UNet:
    """The learned part's network (cfp_unet) on the device and stream of a
    context; its calls take FP64 fields of classified contexts."""

    def __init__(self, ctx, seed=0):
        h = _P()
        _check(lib().cfp_unet_create(ctx._h, int(seed), C.byref(h)), "cfp_unet_create")
        self._h = h
        self.ctx = ctx
        self.n_params = lib().cfp_unet_param_count()

    def params(self, grads=False):
        import numpy as np
        p = np.zeros(self.n_params, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32) if grads else None
        _check(lib().cfp_unet_get_params(self._h, p.ctypes.data_as(_P),
                                         None if g is None else g.ctypes.data_as(_P)), "cfp_unet_get_params")
        return (p, g) if grads else p

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.n_params:
            raise ValueError("expected %d parameters" % self.n_params)
        _check(lib().cfp_unet_set_params(self._h, p.ctypes.data_as(_P)), "cfp_unet_set_params")

    def forward_raw(self, dims, x, y=None, target=None, mask=None, count=0):
        """Forward (and, with target, mask, count, the loss and the backward
        pass into the gradient accumulators) on a packed input x."""
        nx, ny, nz = dims
        loss = C.c_double()
        _check(lib().cfp_unet_forward_raw(self._h, nx, ny, nz, _ptr(x), _ptr(target), _ptr(mask), int(count),
                                          _ptr(y), C.byref(loss)), "cfp_unet_forward_raw")
        return loss.value

    def train_step(self, ctx, r, e, lr, want_loss=False):
        loss = C.c_double()
        _check(lib().cfp_unet_train_step(self._h, ctx._h, ctx._field(r, "r"), ctx._field(e, "e"), float(lr),
                                         C.byref(loss) if want_loss else None), "cfp_unet_train_step")
        return loss.value if want_loss else None

    def apply(self, ctx, r, z):
        _check(lib().cfp_unet_apply(self._h, ctx._h, ctx._field(r, "r"), ctx._field(z, "z")), "cfp_unet_apply")
        return z

    def check(self):
        _check(lib().cfp_unet_check(self._h), "cfp_unet_check")

    def close(self):
        if getattr(self, "_h", None):
            lib().cfp_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
