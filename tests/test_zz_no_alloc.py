"""cfp_assemble_rhs_noalloc against cfp_assemble_rhs, through the C ABI.

The no-allocation variant serves callers that cannot let the library call
cudaMalloc (device memory owned by a pooling allocator, fixed memory or
latency budgets).  Its scratch field lives in a static device array shared by
every call, so two consecutive calls with different inputs must each match
the allocating entry point.  This file is collected last so that a run that
stops at the first failure has already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1901_08269_gb300 import cfp  # noqa: E402
from paper_1901_08269_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _case(w):
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
    ctx.classify_points()
    xyz = ctx.ibi_points()
    return ctx, xyz


def _check_close(a, b, ref_scale):
    err = (a - b).abs()
    assert bool((err <= 1e-12 * ref_scale).all()), float((err / ref_scale).max())


def _row_bounds(w):
    """Per node, the sums of the absolute weights of its regular row: of the
    27-point operator (Rx Ly Lz + Lx Ry Lz + Lx Ly Rz, Eq. A27) and of the
    source operator Q = Lx Ly Lz (Eq. q), from the 1D coefficients of Eq.
    app_xxx.  Rounding of either assembly is bounded by 1e-12 times these
    sums times the data's magnitude (the test geometries keep the bodies away
    from the box, so the rows that see the box values are regular)."""
    from oracle import pyoracle as O
    sums = []
    for xs in (w.x, w.y, w.z):
        a, c, ar, br, cr = O.compact_coefs(xs)
        sums.append((np.abs(a) + 1.0 + np.abs(c), np.abs(ar) + np.abs(br) + np.abs(cr)))
    (Lx, Rx), (Ly, Ry), (Lz, Rz) = sums
    L3 = Lz[:, None, None] * Ly[None, :, None] * Lx[None, None, :]
    B3 = (Lz[:, None, None] * Ly[None, :, None] * Rx[None, None, :] +
          Lz[:, None, None] * Ry[None, :, None] * Lx[None, None, :] +
          Rz[:, None, None] * Ly[None, :, None] * Lx[None, None, :])
    return (torch.as_tensor(B3.reshape(-1), device="cuda"), torch.as_tensor(L3.reshape(-1), device="cuda"))


@pytest.mark.parametrize("make", [lambda: W.config2(33),
                                  lambda: W.Workload("ragged", W.tanh_grid(-1, 1, 37, 1.1),
                                                     W.tanh_grid(-1, 1, 49, 0.7), W.uniform_grid(-1, 1, 31),
                                                     [W.torus((0.02, 0.01, -0.03), 0.45, 0.16,
                                                              W.rot_euler(0.1, 0.5, 0.3))], W._c3_u, W._c3_f)])
def test_noalloc_rhs_matches_allocating_entry_point_twice(make):
    w = make()
    ctx, xyz = _case(w)
    f1, g1 = w.fields(torch, "cuda")
    gi1 = w.g_at(xyz, torch).contiguous()
    # second input set: other source, other Dirichlet data
    f2 = (0.5 * f1 + 1.0).contiguous()
    g2 = (g1 * g1 - 0.25).contiguous()
    gi2 = (gi1 * gi1 - 0.25).contiguous()
    outs = []
    for f, g, gi in ((f1, g1, gi1), (f2, g2, gi2)):
        ref = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        ctx.assemble_rhs(f, g, gi, ref)
        got = torch.full((w.N,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.assemble_rhs_noalloc(f, g, gi, got)
        torch.cuda.synchronize()
        Bsum, Lsum = _row_bounds(w)
        scale = ref.abs() + Bsum * g.abs().max() + Lsum * f.abs().max() + 1.0
        _check_close(got, ref, scale)
        outs.append(got)
    assert not torch.equal(outs[0], outs[1])


def test_noalloc_rejects_grids_beyond_its_scratch():
    x = W.uniform_grid(0, 1, 161)
    y = W.uniform_grid(0, 1, 163)  # 161 * 163 * 161 > 2^22 nodes
    ctx = cfp.Context(x, y, x)
    n = 161 * 163 * 161
    f = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(cfp.CfpError) as e:
        ctx.assemble_rhs_noalloc(f, f, None, f)
    assert e.value.status == cfp.EINVAL and "4194304" in str(e.value)
