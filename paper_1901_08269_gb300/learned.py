"""The learned part's driver: residual / error pairs the solver generates, the
U-Net's training on them, and its use inside the flexible GMRES.

Every computation runs in the library (include/cfp_nn.h, include/cfp.h):
the solves that generate the pairs, the operator applications that form the
residuals, the network's forward and backward passes and Adam steps, and the
flexible GMRES.  torch tensors hold device memory only.

Pairs.  For a random geometry (the batched workload's generator: 1-3
spheres / ellipsoids, stretched grid, random Fourier source), the converged
solution x* comes from the mixed-precision solve with the multigrid
preconditioner; the iterates x_k of the paper's method (BiCGSTAB with eight
red-black sweeps on K) stopped after k iterations give pairs
(r_k = rhs - B x_k, e_k = x* - x_k), k = 0 being (rhs, x*).  The network
learns e from r (both scaled by 1 / max |r|).
"""
import time

import torch

from . import cfp
from . import workloads as W

PAIR_ITERS = (0, 1, 2, 3, 5, 8, 12, 20)


class Problem:
    """A classified random problem with its right-hand side and its converged
    solution (unknowns only; g = 0 on the box)."""

    def __init__(self, seed, sizes=(65,), tol=1e-11):
        self.w = W.random_problem(seed, sizes=sizes)
        w = self.w
        self.ctx = cfp.Context(w.x, w.y, w.z, w.bodies, w.fluid_inside)
        self.ctx.classify_points()
        self.f, self.g = w.fields(torch, "cuda")
        xyz = self.ctx.ibi_points()
        self.gi = w.g_at(xyz, torch).contiguous() if self.ctx.n_ibi else None
        N = w.N
        self.rhs = torch.empty(N, dtype=torch.float64, device="cuda")
        self.ctx.assemble_rhs(self.f, self.g, self.gi, self.rhs)
        self.x = torch.zeros(N, dtype=torch.float64, device="cuda")
        self.ctx.solve(self.f, self.g, self.gi, self.x, tol=tol, precision=cfp.PREC_MIXED,
                       precond=cfp.PRECOND_MG)

    def pairs(self, iters=PAIR_ITERS, smoothed=True):
        """(r_k, e_k) for the paper's preconditioned BiCGSTAB stopped after k
        iterations, k in iters; smoothed: after one application of P."""
        c = self.ctx
        N = self.w.N
        xk = torch.zeros(N, dtype=torch.float64, device="cuda")
        for k in iters:
            xk.zero_()
            if k > 0:
                c.solve(self.f, self.g, self.gi, xk, tol=1e-300, maxit=k, max_restarts=0, precond=cfp.PRECOND_RBGS,
                        sweeps=8, check=False)
            r = torch.empty(N, dtype=torch.float64, device="cuda")
            c.apply(xk, r)
            c.vec_axpby(1.0, self.rhs, -1.0, r)     # r = rhs - B x_k
            e = self.x.clone()
            c.vec_axpby(-1.0, xk, 1.0, e)           # e = x* - x_k
            if smoothed:
                z = torch.empty_like(r)
                c.precondition_ex(r, z, precond=cfp.PRECOND_RBGS, sweeps=8)   # P r
                bz = torch.empty_like(r)
                c.apply(z, bz)
                c.vec_axpby(-1.0, bz, 1.0, r)       # r - B P r
                c.vec_axpby(-1.0, z, 1.0, e)        # e - P r
            yield r, e

    def close(self):
        self.ctx.close()


def train(net, seeds, sizes=(65,), lr=3e-4, lr_end=3e-5, log=None, max_pairs=None):
    """Train on the pairs of the problems `seeds` (one Adam step per pair,
    learning rate decaying geometrically from lr to lr_end).  Returns
    (pairs, wall seconds, the losses of the last 64 pairs)."""
    total = len(seeds) * len(PAIR_ITERS) if max_pairs is None else max_pairs
    n, tail = 0, []
    t0 = time.perf_counter()
    for s in seeds:
        p = Problem(s, sizes)
        for r, e in p.pairs():
            rate = lr * (lr_end / lr) ** (n / max(total - 1, 1))
            want = n >= total - 64 or (log and n % log == 0)
            loss = net.train_step(p.ctx, r, e, rate, want_loss=want)
            if loss is not None and n >= total - 64:
                tail.append(loss)
            if log and n % log == 0:
                print("pair %d loss %.4e lr %.2e" % (n, loss, rate), flush=True)
            n += 1
            if n >= total:
                break
        p.close()
        if n >= total:
            break
    torch.cuda.synchronize()
    net.check()
    return n, time.perf_counter() - t0, tail
