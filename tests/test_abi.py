"""CPU checks of the boundary: the CUDA library builds and loads, exports
every entry point include/cfp.h declares, and the binding rejects bad
arguments before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1901_08269_gb300 import cfp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "cfp.h")).read() + open(os.path.join(ROOT, "include", "cfp_nn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cfp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["cfp_ctx_create", "cfp_classify_points", "cfp_ibi_points", "cfp_assemble_rhs", "cfp_solve",
              "cfp_ctx_destroy", "cfp_last_error", "cfp_apply", "cfp_precondition", "cfp_solve_host",
              "cfp_default_opts"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    L = cfp.lib()
    for n in declared():
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


def test_default_opts():
    o = cfp.default_opts()
    assert o.sweeps == 8 and o.precision == cfp.PREC_FP64 and o.use_graph == 1 and o.maxit > 0


def test_create_rejects_bad_grids_without_a_device():
    L = cfp.lib()
    D = ctypes.POINTER(ctypes.c_double)
    x = np.array([0.0, 0.5, 0.4, 1.0])  # not increasing
    h = ctypes.c_void_p()
    arr, nb = cfp.make_bodies([])
    st = L.cfp_ctx_create(x.ctypes.data_as(D), 4, x.ctypes.data_as(D), 4, x.ctypes.data_as(D), 4, arr, 0, 0,
                          None, ctypes.byref(h))
    assert st == cfp.EINVAL and "increasing" in cfp.last_error()
    y = np.array([0.0, 1.0])
    st = L.cfp_ctx_create(y.ctypes.data_as(D), 2, y.ctypes.data_as(D), 2, y.ctypes.data_as(D), 2, arr, 0, 0,
                          None, ctypes.byref(h))
    assert st == cfp.EINVAL
    st = L.cfp_ctx_create(None, 4, None, 4, None, 4, arr, 0, 0, None, None)
    assert st == cfp.EINVAL
    assert L.cfp_classify_points(None, None, None, None) == cfp.EINVAL


def test_learned_part_rejects_bad_arguments_without_a_device():
    L = cfp.lib()
    e = cfp.EINVAL
    assert L.cfp_nn_conv3d(None, 9, 9, 9, 16, 16, None, None, None, None, 0, None) == e
    assert L.cfp_nn_conv3d_wgrad(None, 9, 9, 9, 16, 16, None, None, None, None) == e
    assert L.cfp_nn_transfer(None, cfp.NN_INJECT, 9, 9, 9, 16, None, None, None, None) == e
    assert L.cfp_unet_create(None, 0, None) == e
    assert L.cfp_unet_get_params(None, None, None) == e
    assert L.cfp_unet_set_params(None, None) == e
    assert L.cfp_unet_forward_raw(None, 9, 9, 9, None, None, None, 0, None, None) == e
    assert L.cfp_unet_train_step(None, None, None, None, 1e-3, None) == e
    assert L.cfp_unet_apply(None, None, None, None) == e
    assert L.cfp_solve_fgmres(None, None, None, None, None, None, 1e-10, None, 20, 0, None) == e
    assert L.cfp_unet_param_count() == 1313968


def test_vec_axpby_accepts_aliased_operands_by_declaration():
    # x and y may be the same field (cfp.h); the kernel behind it declares
    # neither pointer __restrict__, checked here in its source
    src = open(os.path.join(ROOT, "paper_1901_08269_gb300", "csrc", "cfp_krylov.cu")).read()
    m = re.search(r"__global__ void k_axpby\(([^)]*)\)", src)
    assert m and "__restrict__" not in m.group(1)
