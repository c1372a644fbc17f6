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
        ms, by = ctx.time_kernel(ids[name], prec, reps=a.reps)
        out[name] = {"ms": ms, "bytes": by, "GBps": by / ms / 1e6}
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
