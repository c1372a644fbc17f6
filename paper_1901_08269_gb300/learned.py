"""The learned part: a small 3x3x3 convolutional network that predicts the
error of an iterate from its residual, trained on pairs the solver produces.

Every computation runs in the library's kernels (include/cfp_nn.h); torch
tensors only hold the device memory.  Network: three layers of 16 -> 16
channels (input channels 0 and 1: the scaled residual and the unknowns'
mask; output channel 0: the scaled error), ReLU after the first two, BF16
activations and weights on the tensor cores, FP32 master weights trained
with Adam.  Here it supplies the initial guess of a solve: for x0 = 0 the
residual is the right-hand side, so u0 = net(rhs).
"""
import math

import torch

from . import cfp

NC, TAPS = 16, 27


class ConvNet:
    def __init__(self, seed=0, device="cuda", escale=1.0):
        """escale: the constant by which the scaled targets are multiplied (a
        property of the problem class, fixed before training)."""
        gen = torch.Generator().manual_seed(seed)
        self.escale = float(escale)
        self.device = device
        self.w32, self.b32 = [], []
        for layer, (cin, cout) in enumerate(((2, NC), (NC, NC), (NC, 1))):
            w = torch.zeros(NC, TAPS, NC, dtype=torch.float32)
            std = math.sqrt(2.0 / (cin * TAPS)) * (1.0 if layer < 2 else 0.1)
            w[:cout, :, :cin] = torch.randn(cout, TAPS, cin, generator=gen) * std
            self.w32.append(w.reshape(-1).to(device))
            self.b32.append(torch.zeros(NC, dtype=torch.float32, device=device))
        self.params = self.w32 + self.b32
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.wbf = [torch.empty(NC * TAPS * NC, dtype=torch.bfloat16, device=device) for _ in range(3)]
        self.steps = 0

    def sync_bf16(self, ctx):
        """BF16 copies of the master weights (an Adam step with lr 0)."""
        for i in range(3):
            ctx.nn_adam(self.w32[i], self.grads[i], self.m[i], self.v[i], max(1, self.steps), 0.0, self.wbf[i])

    def forward(self, ctx, x):
        n = ctx.N * NC
        a1 = torch.empty(n, dtype=torch.bfloat16, device=x.device)
        a2 = torch.empty(n, dtype=torch.bfloat16, device=x.device)
        y = torch.empty(n, dtype=torch.float32, device=x.device)
        ctx.nn_conv3d(x, self.wbf[0], self.b32[0], 1, a1)
        ctx.nn_conv3d(a1, self.wbf[1], self.b32[1], 1, a2)
        ctx.nn_conv3d(a2, self.wbf[2], self.b32[2], 0, y)
        return y, (x, a1, a2)

    def backward(self, ctx, acts, dy):
        """Accumulates the gradients of all layers for dL/dy (N x 16 BF16)."""
        x, a1, a2 = acts
        d2 = torch.empty_like(a2)
        d1 = torch.empty_like(a1)
        ctx.nn_wgrad(a2, dy, self.grads[2], self.grads[5])
        ctx.nn_dgrad(dy, self.wbf[2], a2, d2)
        ctx.nn_wgrad(a1, d2, self.grads[1], self.grads[4])
        ctx.nn_dgrad(d2, self.wbf[1], a1, d1)
        ctx.nn_wgrad(x, d1, self.grads[0], self.grads[3])

    def adam(self, ctx, lr):
        self.steps += 1
        for i, p in enumerate(self.params):
            ctx.nn_adam(p, self.grads[i], self.m[i], self.v[i], self.steps, lr, self.wbf[i] if i < 3 else None)

    def guess(self, ctx, rhs, u):
        """u = the network's prediction of the solution from the residual of x0 = 0."""
        x = torch.empty(ctx.N * NC, dtype=torch.bfloat16, device=rhs.device)
        scale = ctx.nn_pack(rhs, None, 0.0, self.escale, x)
        y, _ = self.forward(ctx, x)
        return ctx.nn_unpack(y, 1.0 / (scale * self.escale), u)


class Sample:
    """One training pair on its own context: input x (the residual of x0 = 0,
    i.e. the right-hand side), target (the error of x0 = 0, i.e. the solution
    at the unknowns) and the unknowns' mask.  pack() builds them once the
    target constant escale is chosen (ratio() gives this sample's
    max|rhs| / max|u|)."""

    def __init__(self, w, tol=1e-10, device="cuda"):
        self.w = w
        self.ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
        self.ctx.classify_points()
        f, g = w.fields(torch, device)
        gi = w.g_at(self.ctx.ibi_points(), torch) if self.ctx.n_ibi else None
        self.rhs = torch.empty(w.N, dtype=torch.float64, device=device)
        self.ctx.assemble_rhs(f, g, gi, self.rhs)
        u = torch.zeros(w.N, dtype=torch.float64, device=device)
        self.info = self.ctx.solve(f, g, gi, u, tol=tol, precision=cfp.PREC_MIXED, precond=cfp.PRECOND_MG)
        self.f, self.g, self.gi, self.u = f, g, gi, u
        n = self.ctx.N
        self.x = torch.empty(n * NC, dtype=torch.bfloat16, device=device)
        self.target = torch.empty(n, dtype=torch.float32, device=device)
        self.mask = torch.empty(n, dtype=torch.float32, device=device)
        self.inv_count = 1.0 / n
        self.scale_r = self.ctx.nn_pack(self.rhs, None, 0.0, 1.0, self.x)
        self.scale_u = self.ctx.nn_pack(u, None, 0.0, 1.0, self.x)

    def ratio(self):
        return self.scale_u / self.scale_r

    def pack(self, escale):
        self.scale = self.ctx.nn_pack(self.rhs, self.u, 0.0, escale, self.x, self.target, self.mask)
        return self


def make_samples(workloads, tol=1e-10, device="cuda"):
    """Solver-generated training pairs and the target constant (the median
    max|rhs| / max|u| of the problems)."""
    samples = [Sample(w, tol, device) for w in workloads]
    r = sorted(s.ratio() for s in samples)
    escale = r[len(r) // 2]
    return [s.pack(escale) for s in samples], escale


def train(net, samples, steps, lr=2e-3, log_every=0):
    """Adam on the masked MSE, cycling through the samples; returns the losses."""
    losses = []
    if net.steps == 0:
        net.sync_bf16(samples[0].ctx)
    for s in range(steps):
        smp = samples[s % len(samples)]
        ctx = smp.ctx
        y, acts = net.forward(ctx, smp.x)
        dy = torch.empty(ctx.N * NC, dtype=torch.bfloat16, device=y.device)
        loss = ctx.nn_mse(y, smp.target, smp.mask, smp.inv_count, dy)
        net.backward(ctx, acts, dy)
        net.adam(ctx, lr)
        losses.append(loss)
        if log_every and s % log_every == 0:
            print("step %d loss %.4e" % (s, loss))
    return losses


def mg_precond(ctx, opts):
    """z = one multigrid V-cycle on K applied to v (a fixed linear map)."""
    def apply(v, z):
        ctx.precondition_ex(v, z, opts=opts)
    return apply


def net_mg_precond(ctx, net, opts, net_steps=1):
    """For the first net_steps directions of a solve z = z1 + V(v - B z1), z1
    the network's prediction of B^-1 v (its guess corrected by one multigrid
    V-cycle on its residual); afterwards the V-cycle alone.  The network is
    trained on right-hand sides, which the first direction of a solve from
    x0 = 0 is; the later directions are oscillatory, where its output means
    nothing.  A preconditioner that changes between steps and is not linear:
    it needs a flexible Krylov method."""
    z1 = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    r = torch.empty(ctx.N, dtype=torch.float64, device="cuda")
    calls = [0]

    def apply(v, z):
        calls[0] += 1
        if calls[0] > net_steps:
            ctx.precondition_ex(v, z, opts=opts)
            return
        net.guess(ctx, v, z1)
        ctx.apply(z1, r)
        ctx.vec_axpby(1.0, v, -1.0, r)
        ctx.precondition_ex(r, z, opts=opts)
        ctx.vec_axpby(1.0, z1, 1.0, z)
    return apply


def fgmres(ctx, b, x, precond, m=30, tol=1e-10, maxit=300):
    """Right-preconditioned flexible GMRES(m) (Saad, SIAM J. Sci. Comput. 14,
    1993) for B x = b on the unknowns, x holding the initial guess (zero off
    the unknowns, as b is).  precond(v, z) may change between iterations; the
    search directions z_j are kept and x += Z y.  Vector work runs in the
    library's kernels (apply, dot, axpby), the (m+1) x m least-squares problem
    with Givens rotations on the host.  Returns (iterations, relative
    residual ||b - B x|| / ||b||, recomputed)."""
    import math

    import numpy as np
    n = ctx.N
    V = [torch.zeros(n, dtype=torch.float64, device=b.device) for _ in range(m + 1)]
    Z = [torch.zeros(n, dtype=torch.float64, device=b.device) for _ in range(m)]
    w = torch.zeros(n, dtype=torch.float64, device=b.device)
    bnorm = math.sqrt(ctx.vec_dot(b, b))
    its = 0

    def residual():
        ctx.apply(x, w)
        ctx.vec_axpby(1.0, b, -1.0, w)
        return math.sqrt(ctx.vec_dot(w, w))

    beta = residual()
    while beta > tol * bnorm and its < maxit:
        ctx.vec_axpby(1.0 / beta, w, 0.0, V[0])
        H = np.zeros((m + 1, m))
        cs, sn, g = np.zeros(m), np.zeros(m), np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            precond(V[j], Z[j])
            ctx.apply(Z[j], w)
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = ctx.vec_dot(w, V[i])
                ctx.vec_axpby(-H[i, j], V[i], 1.0, w)
            H[j + 1, j] = math.sqrt(ctx.vec_dot(w, w))
            if H[j + 1, j] > 0.0:
                ctx.vec_axpby(1.0 / H[j + 1, j], w, 0.0, V[j + 1])
            for i in range(j):  # the earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j], H[j + 1, j] = d, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            its += 1
            k = j + 1
            if abs(g[j + 1]) <= tol * bnorm or its >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):  # back substitution in the rotated Hessenberg matrix
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            ctx.vec_axpby(float(y[i]), Z[i], 1.0, x)
        beta = residual()
    return its, beta / bnorm
