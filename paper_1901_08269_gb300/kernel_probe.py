"""Time single kernels of the solve through cfp_time_kernel.

Builds a context on the config-3 geometry at n^3, classifies it, and times
the red-black half-sweep on the fine level's red/black split arrays (the
kernel of both the multigrid smoother and the plain red-black inner
iterations), the apply (with its fused dot) and the x/r update in the
requested precision.  Small launch count, so it is the command used
for ncu captures of those kernels:

    python -m paper_1901_08269_gb300.kernel_probe --n 385 --precision mixed --reps 3
"""
import argparse
import json


def nn_time(ctx, name, reps):
    """One 16 -> 16 channel 3x3x3 layer of the learned part on the context's
    grid (random BF16 input and weights): event-timed mean of reps launches
    after two untimed ones; FLOP counted as 2 * 16 * 27 * 16 per node."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(0)
    n = ctx.N
    x = torch.randn(n * 16, generator=g, device="cuda").to(torch.bfloat16)
    dy = torch.randn(n * 16, generator=g, device="cuda").to(torch.bfloat16)
    w = (0.1 * torch.randn(16 * 27 * 16, generator=g, device="cuda")).to(torch.bfloat16)
    out = torch.empty(n * 16, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(16 * 27 * 16, dtype=torch.float32, device="cuda")

    def run():
        if name == "nn_conv":
            ctx.nn_conv3d(x, w, None, 1, out)
        else:
            ctx.nn_wgrad(x, dy, dw)

    for _ in range(2):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flop = 2.0 * 16 * 27 * 16 * n
    return {"ms": ms, "flop": flop, "TFLOPs": flop / ms / 1e9}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=385)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--kernels", default="mg_sweep,apply,update")
    a = ap.parse_args()
    import torch

    from . import cfp
    from . import workloads as W
    torch.cuda.set_device(0)
    w = W.config3(a.n)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
    ctx.classify_points()
    prec = cfp.PREC_MIXED if a.precision == "mixed" else cfp.PREC_FP64
    ids = {"rbgs": cfp.KERNEL_RBGS, "mg_sweep": cfp.KERNEL_MG_SWEEP, "apply": cfp.KERNEL_APPLY,
           "update": cfp.KERNEL_UPDATE}
    out = {"n": a.n, "precision": a.precision}
    for name in a.kernels.split(","):
        if name in ("nn_conv", "nn_wgrad"):
            out[name] = nn_time(ctx, name, a.reps)
            continue
        ms, by = ctx.time_kernel(ids[name], prec, reps=a.reps)
        out[name] = {"ms": ms, "bytes": by, "GBps": by / ms / 1e6}
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
