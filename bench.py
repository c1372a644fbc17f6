#!/usr/bin/env python3
"""Benchmark of the compact-stencil immersed-body Poisson solve on GB300.

Workload: the 513^3 stretched grid of [-1,1]^3 (tanh factors 2.0, 1.2, 1.2)
with an ellipsoid (0.4, 0.25, 0.2) rotated 30 degrees about z and a torus
(R 0.3, r 0.1) at (0.5, 0.4, -0.3); u = sin(2x) cosh(y) exp(-z^2).  One step
= the whole hot path: grid metrics, point classification, IBI location,
modified stencils, right-hand side, preconditioned BiCGSTAB to the
tolerance (mixed FP32/FP64 by default).  Inputs (f, g on the nodes, g at the
IBI points) are resident in HBM before the timed region; every field is
1.08 GB, far above the 129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
instead (bounded sample, extrapolated), see `reference_arm`.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s/solve at 513³ to equal max-norm error, plain FP64 vs mixed/learned; HBM GB/s"
UNIT = "s/solve"
FALLBACK_HBM_GBS = 6800.0
# BiCGSTAB iterations of the 513^3 workload in FP64 with the oracle's own
# preconditioner (8 red-black sweeps) to tol 1e-15, measured by the GPU path
# with the same preconditioner; the CPU baselines extrapolate with it since
# the oracle cannot run the 513^3 solve itself.
FP64_RBGS_ITERS_513 = 535


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=513)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-15)
    ap.add_argument("--inner-tol", type=float, default=3e-3)
    ap.add_argument("--batch-tol", type=float, default=1e-12,
                    help="tolerance of the batched workload (its random g = 0 problems reach a relative "
                         "residual of only 1e-14 .. 2e-13 in FP64, the oracle's included)")
    ap.add_argument("--sweeps", type=int, default=8)
    ap.add_argument("--precond", default="mg", choices=["mg", "rbgs"])
    ap.add_argument("--mg-smooth", type=int, default=5)
    ap.add_argument("--mg-post", type=int, default=3, help="post-smoothing sweeps (0: as --mg-smooth)")
    ap.add_argument("--no-graph", action="store_true",
                    help="plain launches instead of the CUDA graph (ncu cannot profile kernel nodes of graphs "
                         "with conditional nodes)")
    ap.add_argument("--no-fp64-check", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--fp64-steps", type=int, default=5,
                    help="timed steps of the FP64 comparison solve (at most --steps; about 3 s each at 513^3)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--oracle-n", type=int, default=129)
    ap.add_argument("--oracle-iters", type=int, default=10)
    ap.add_argument("--oracle-large", type=int, default=0,
                    help="nodes per axis of the larger oracle sample (0: 2 * --oracle-n - 1); config 3's "
                         "geometry needs at least 129")
    ap.add_argument("--workload", default="config3", choices=["config3", "batch", "learned"],
                    help="config3: the 513^3 two-body solve (default); batch: 64 random problems of uneven "
                         "size solved together; learned: the U-Net trained on solver-generated pairs, then "
                         "the paper's method, GMRES and the flexible GMRES with the network compared at "
                         "--learned-n^3 on held-out geometries")
    ap.add_argument("--learned-n", type=int, default=257)
    ap.add_argument("--learned-problems", type=int, default=300,
                    help="random geometries (65^3) whose solver-generated pairs train the network")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--kernels", default=None,
                    help="time single kernels instead of the solve: a comma list of mg_sweep, rbgs, apply, "
                         "update, prolong, restrict, nn_conv[C], nn_wgrad[C] (C -> C channels, default 16) on the "
                         "config-3 geometry "
                         "at --n^3 (--reps launches each); "
                         "few launches, so it is the command the ncu captures of those kernels run")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--apply-tile", default=None,
                    help="--kernels: the apply's kernel,rows,planes for cfp_tune_apply (1: streaming, 2: the "
                         "bulk-copy ring with rows 2), e.g. 2,2,64; default: the context's own choice")
    ap.add_argument("--seed", type=int, default=20261203)
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return {}, "fallback"


def hbm_peak():
    d, src = peaks()
    for k in ("hbm_gbs", "hbm_GBps", "hbm"):
        if k in d:
            v = d[k]
            if isinstance(v, dict):
                v = v.get("value", v.get("gbs"))
            try:
                return float(v), "measured"
            except (TypeError, ValueError):
                pass
    return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------- CPU baseline
def oracle_sample(n_sample, iters):
    """Time the CPU oracle on a bounded sample of the workload: the same
    geometry and solution on an n_sample^3 grid, set-up (classification, IBI,
    explicit CSR assembly, right-hand side) plus `iters` BiCGSTAB iterations
    with its 8-sweep red-black preconditioner."""
    from oracle import pyoracle as O
    from paper_1901_08269_gb300 import workloads as W
    w = W.config3(n_sample)
    f, g = w.fields()
    t0 = time.perf_counter()
    P = O.Problem(w.x, w.y, w.z, w.bodies)
    P.classify()
    key, tt, xyz = P.ibi()
    P.assemble()
    rhs = P.rhs(f, g, w.g_at(xyz))
    t1 = time.perf_counter()
    x, st, it, rel = P.bicgstab(rhs, tol=1e-30, maxit=iters, sweeps=8)
    t2 = time.perf_counter()
    return {"n": n_sample, "setup_s": t1 - t0, "iter_s": (t2 - t1) / max(it, 1), "iters": it,
            "cores": O.threads(), "wall_s": t2 - t0}


def oracle_extrapolate(small, large, n_full, iters_full):
    """A 513^3 solve of iters_full iterations from two measured samples: the
    set-up and the per-iteration time of the larger sample, scaled to n_full^3
    nodes with the exponents measured between the two samples (time ~
    nodes^p; p = 1 is linear)."""
    import math as m
    ratio = (small["n"] / large["n"]) ** 3
    p_it = m.log(small["iter_s"] / large["iter_s"]) / m.log(ratio)
    p_su = m.log(small["setup_s"] / large["setup_s"]) / m.log(ratio)
    scale = (n_full / large["n"]) ** 3
    it_full = large["iter_s"] * scale ** p_it
    su_full = large["setup_s"] * scale ** p_su
    return {"est_s_per_solve": su_full + iters_full * it_full, "iter_s_full": it_full, "setup_s_full": su_full,
            "p_iter": p_it, "p_setup": p_su}


def oracle_text(small, large, est, n_full, iters_full):
    return ("oracle (plain C, FP64, explicit CSR, OpenMP, %d threads) on the config-3 geometry, measured: "
            "%d^3 set-up %.2f s + %.3f s/iteration, %d^3 set-up %.2f s + %.3f s/iteration (%d BiCGSTAB "
            "iterations each, 8-sweep red-black preconditioner); time grows as nodes^%.2f per iteration and "
            "nodes^%.2f for the set-up between the two, so a %d^3 FP64 solve of %d iterations (the count the "
            "same preconditioner needs on the GPU) is estimated at %.0f s (set-up %.0f s, %.2f s/iteration)"
            % (large["cores"], small["n"], small["setup_s"], small["iter_s"], large["n"], large["setup_s"],
               large["iter_s"], large["iters"], est["p_iter"], est["p_setup"], n_full, iters_full,
               est["est_s_per_solve"], est["setup_s_full"], est["iter_s_full"]))


def reference_arm(args):
    """The oracle as it stands on the host cores.  Calibration (untimed): one
    sample at --oracle-large nodes per axis for the growth exponents; each
    step then times the --oracle-n sample and extrapolates it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n_large = args.oracle_large or 2 * args.oracle_n - 1
    large = oracle_sample(n_large, args.oracle_iters)
    vals, walls = [], []
    for s in range(args.warmup + args.steps):
        small = oracle_sample(args.oracle_n, args.oracle_iters)
        if s >= args.warmup:
            # this step's own small sample, scaled to the large one with the
            # calibration's exponents, then to the full size
            cal = oracle_extrapolate(small, large, args.n, FP64_RBGS_ITERS_513)
            vals.append(cal["est_s_per_solve"])
            walls.append(small["wall_s"])
    v = statistics.mean(vals)
    sample = oracle_text(small, large, cal, args.n, FP64_RBGS_ITERS_513)
    sample += "; each timed step is the %d^3 sample (%.2f s wall on average), extrapolated" % (
        args.oracle_n, statistics.mean(walls))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args, 1), precision="fp64", precond="rbgs", sweeps=8),
            "value_kind": "extrapolated from measured samples",
            "sample_wall_s_per_step": statistics.mean(walls),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": large["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ kernel mode
def nn_time(ctx, name, reps, cin=16, cout=16):
    """One cin -> cout 3x3x3 layer of the learned part on the context's grid
    (random BF16 activations and weights): event-timed mean of reps calls
    after two untimed ones (each call packs the weights, launches the
    tensor-core kernel and checks its wait word); FLOP = 2 * 27 * cin * cout
    per node."""
    import torch

    from paper_1901_08269_gb300 import cfp
    g = torch.Generator(device="cuda").manual_seed(0)
    dims = (ctx.x.size, ctx.y.size, ctx.z.size)
    npad = (dims[0] + 2) * (dims[1] + 2) * (dims[2] + 2)
    x = torch.randn(npad * cin, generator=g, device="cuda").to(torch.bfloat16)
    dy = torch.randn(npad * cout, generator=g, device="cuda").to(torch.bfloat16)
    w = (0.1 * torch.randn(cout * 27 * cin, generator=g, device="cuda")).to(torch.bfloat16)
    out = torch.empty(npad * cout, dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")

    def run():
        if name == "nn_conv":
            ctx.nn_conv3d(dims, cin, cout, x, w, out, flags=cfp.NN_RELU)
        else:
            ctx.nn_wgrad(dims, cin, cout, x, dy, dw)

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
    flop = 2.0 * 27 * cin * cout * dims[0] * dims[1] * dims[2]
    return {"ms": ms, "flop": flop, "TFLOPs": flop / ms / 1e9, "cin": cin, "cout": cout}


def kernel_arm(args):
    """Single kernels of the solve, event-timed through cfp_time_kernel on
    the config-3 geometry at n^3 (classification first): the red-black
    half-sweep on the fine level's split arrays (the multigrid smoother's and
    the plain inner iterations' kernel), the apply with its fused dot, the
    x/r update, and the learned part's convolution layers."""
    import torch

    from paper_1901_08269_gb300 import cfp
    from paper_1901_08269_gb300 import workloads as W
    torch.cuda.set_device(0)
    w = W.config3(args.n)
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
    ctx.classify_points()
    prec = cfp.PREC_MIXED if args.precision == "mixed" else cfp.PREC_FP64
    ids = {"rbgs": cfp.KERNEL_RBGS, "mg_sweep": cfp.KERNEL_MG_SWEEP, "apply": cfp.KERNEL_APPLY,
           "update": cfp.KERNEL_UPDATE, "prolong": cfp.KERNEL_PROLONG, "restrict": cfp.KERNEL_RESTRICT,
           "mg_pair": cfp.KERNEL_MG_PAIR}
    out = {"mode": "kernels", "n": args.n, "precision": args.precision, "reps": args.reps}
    if args.apply_tile:
        k, r, q = (int(v) for v in args.apply_tile.split(","))
        ctx.tune_apply(prec, r, q, kernel=k)
    for name in args.kernels.split(","):
        if name.startswith("nn_conv") or name.startswith("nn_wgrad"):
            # nn_conv / nn_wgrad: 16 -> 16 channels; nn_conv64 / nn_wgrad128: c -> c
            base = "nn_conv" if name.startswith("nn_conv") else "nn_wgrad"
            c = int(name[len(base):] or 16)
            out[name] = nn_time(ctx, base, args.reps, c, c)
            continue
        ms, by = ctx.time_kernel(ids[name], prec, reps=args.reps)
        out[name] = {"ms": ms, "bytes": by, "GBps": by / ms / 1e6}
    out["apply_tile"] = ctx.apply_shape(prec)  # after the timings, which set up the ring where it applies
    ctx.close()
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------- learned arm
def learned_arm(args):
    """The learned part as a workload: train the U-Net (tcgen05 kernels) on
    the pairs of --learned-problems random geometries at 65^3 (one Adam step
    per pair), then solve held-out random geometries with 1-3 bodies at
    --learned-n^3 to a relative residual of 1e-10 three ways: the paper's
    method (BiCGSTAB, eight red-black sweeps on K), GMRES(20) with the same
    sweeps, and the flexible GMRES(20) with the network in its
    preconditioner and initial guess.  Every solution is checked against a
    tight multigrid-preconditioned solve (max difference relative to its
    maximum); the line reports iterations and seconds per solve of each."""
    import torch

    from paper_1901_08269_gb300 import cfp, learned
    from paper_1901_08269_gb300 import workloads as W
    torch.cuda.set_device(0)
    host = cfp.Context(W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), W.uniform_grid(0, 1, 9), [])
    net = cfp.UNet(host, seed=5)
    pairs, train_s, tail = learned.train(net, seeds=list(range(2000, 2000 + args.learned_problems)), sizes=(65,))
    rows = []
    for seed in (9001, 9002, 9003):
        w = W.random_problem(seed, sizes=(args.learned_n,))
        ctx = cfp.Context(w.x, w.y, w.z, w.bodies)
        ctx.classify_points()
        xyz = ctx.ibi_points()
        f, g = w.fields(torch, "cuda")
        gi = w.g_at(xyz, torch).contiguous() if ctx.n_ibi else None
        ref = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        # random g = 0 problems reach a relative residual of about 1e-13 at best in FP64
        ctx.solve(f, g, gi, ref, tol=1e-12, precond=cfp.PRECOND_MG)
        row = {"seed": seed, "bodies": len(w.bodies), "n": args.learned_n}
        for name in ("bicgstab_rbgs8", "gmres_rbgs8", "fgmres_net_rbgs8"):
            for rep in range(2):  # the first run builds graphs and buffers
                u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if name == "bicgstab_rbgs8":
                    info = ctx.solve(f, g, gi, u, tol=1e-10, precond=cfp.PRECOND_RBGS, sweeps=8)
                else:
                    info = ctx.solve_fgmres(f, g, gi, u, tol=1e-10, net=net if "net" in name else None, m=20,
                                            net_guess="net" in name, precond=cfp.PRECOND_RBGS, sweeps=8)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
            row[name] = {"iterations": info.iterations, "s": dt, "rel_residual": info.rel_residual,
                         "max_diff_vs_ref": float((u - ref).abs().max() / ref.abs().max())}
            if "net" in name:
                row[name]["steps_with_network_direction"] = info.refinements
        rows.append(row)
        ctx.close()
    net.close()
    host.close()
    mean = lambda k, q: statistics.mean(r[k][q] for r in rows)
    line = {"metric": "s/solve at %d^3 to equal error: paper's method vs flexible GMRES with the learned network"
                      % args.learned_n, "value": mean("fgmres_net_rbgs8", "s"), "unit": "s/solve", "n_gpus": 1,
            "steps": len(rows), "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 network, f64 solve", "data": "synthetic",
            "config": {"workload": "config5-learned-%d^3" % args.learned_n, "train_problems": args.learned_problems,
                       "train_pairs": pairs, "train_s": train_s, "train_loss_tail": statistics.mean(tail),
                       "tol": 1e-10},
            "paper_method_s": mean("bicgstab_rbgs8", "s"), "gmres_s": mean("gmres_rbgs8", "s"),
            "iterations": {k: [r[k]["iterations"] for r in rows]
                           for k in ("bicgstab_rbgs8", "gmres_rbgs8", "fgmres_net_rbgs8")},
            "problems": rows}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------- batched arm
def batch_arm(args):
    """64 random problems (n in {33,49,65,97,129}, 1-3 spheres/ellipsoids,
    tanh factors in [1,2], 8-mode source, g = 0) solved together as one graph
    launch (cfp_batch: every problem's refinement and BiCGSTAB loops driven
    on the device), mixed precision, multigrid, the solver settings and the
    apply's tile autotuned per grid size; one step = classification of every
    problem + the batch (captured again, as the classification replaced the
    side data) + its launch.  The host-thread batch (cfp_solve_batch) is
    timed beside it."""
    import torch

    from paper_1901_08269_gb300 import cfp
    from paper_1901_08269_gb300 import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    probs = []
    for m in range(args.batch):
        w = W.random_problem(args.seed + m)
        ctx = cfp.Context(w.x, w.y, w.z, w.bodies, stream=torch.cuda.Stream())
        ctx.classify_points()
        xyz = ctx.ibi_points()
        f, g = w.fields(torch, "cuda")
        gi = w.g_at(xyz, torch).contiguous() if ctx.n_ibi else None
        u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
        probs.append((w, ctx, f, g, gi, u))
    torch.cuda.synchronize()
    prec = cfp.PREC_MIXED if args.precision == "mixed" else cfp.PREC_FP64
    opts = cfp.default_opts(precision=prec, precond=cfp.PRECOND_MG, mg_smooth=args.mg_smooth, mg_post=args.mg_post,
                            inner_tol=args.inner_tol)
    # autotune once per grid size (first problem of each size): the solver
    # settings and the FP32 apply's kernel and tile; the others of that size
    # take both
    tuned, shapes = {}, {}
    for w, ctx, f, g, gi, u in probs:
        n = w.x.size
        if n not in tuned:
            tuned[n] = ctx.autotune(f, g, gi, u, tol=args.batch_tol, opts=cfp.default_opts(
                precision=prec, precond=cfp.PRECOND_MG, inner_tol=args.inner_tol))[0]
            if prec == cfp.PREC_MIXED:
                ctx.tune_apply(cfp.PREC_MIXED)
                shapes[n] = ctx.apply_shape(cfp.PREC_MIXED)
        elif n in shapes:
            k, r, q = shapes[n]
            ctx.tune_apply(cfp.PREC_MIXED, r, q, kernel=k)
    by_n = {n: (o.mg_smooth, o.inner_tol) + tuple(shapes.get(n, ())) for n, o in tuned.items()}
    popts = [tuned[p[0].x.size] for p in probs]
    # the host-thread batch takes one opts: the setting tuned for the largest size
    opts = tuned[max(tuned)]

    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(16)  # contexts classify independently (the C calls release the GIL)
    graph = prec == cfp.PREC_MIXED
    batch = cfp.Batch([p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs], [p[4] for p in probs],
                      [p[5] for p in probs], tol=args.batch_tol, opts=popts) if graph else None

    def classify():
        list(pool.map(lambda p: p[1].classify_points(), probs))
        for w, ctx, f, g, gi, u in probs:
            u.zero_()
        torch.cuda.synchronize()

    def step_graph():
        classify()
        return batch.run()

    def step_threads():
        classify()
        return cfp.solve_batch([p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs],
                               [p[4] for p in probs], [p[5] for p in probs], tol=args.batch_tol, opts=opts)

    def timed(step, k):
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k):
            out = step()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / k, out

    dt, infos = timed(step_graph if graph else step_threads, args.steps)
    dt_threads = timed(step_threads, max(1, min(args.steps, 3)))[0] if graph else dt
    reuse = None
    if graph:
        # the same geometries again: no classification, the graph reused
        def step_reuse():
            for p in probs:
                p[5].zero_()
            torch.cuda.synchronize()
            return batch.run()
        reuse = timed(step_reuse, max(1, min(args.steps, 3)))[0]
    # the same problems one after another (no overlap), for comparison
    t1 = time.perf_counter()
    for w, ctx, f, g, gi, u in probs:
        ctx.classify_points()
        u.zero_()
        ctx.solve(f, g, gi, u, tol=args.batch_tol, opts=tuned[w.x.size])
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    nodes = sum(p[0].N for p in probs)
    launches = sum(i.launches for i in infos) if graph else None
    line = {"metric": "s per batch of %d random immersed-body problems (config 4)" % args.batch, "value": dt,
            "unit": "s/batch", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": 1000 * dt, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == cfp.PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": "config4-batch%d-seed%d" % (args.batch, args.seed), "total_nodes": nodes,
                       "sizes": sorted(set(p[0].x.size for p in probs)), "tuned": {str(k): v for k, v in by_n.items()},
                       "tol": args.batch_tol, "impl": "one graph launch per batch" if graph else "host threads"},
            "host_threads_s": dt_threads, "graph_reused_s": reuse, "sequential_s": seq, "iterations": [i.iterations for i in infos[:8]],
            "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    pool.shutdown()
    if batch is not None:
        batch.close()
    for p in probs:
        p[1].close()
    return 0


def workload_config(args, world):
    """The workload part of the JSON line's config, shared by both arms."""
    return {"workload": "config3-%d^3-ellipsoid+torus" % args.n, "n": args.n,
            "grid": "tanh (2.0, 1.2, 1.2) on [-1,1]^3", "tol": args.tol,
            "l2": "no flush: every field (%.2f GB at %d^3) exceeds the 129 MB L2" % (8e-9 * args.n ** 3, args.n),
            "parallelism": "replicas" if world > 1 else "single"}


def job_time(ms, steps, world, dist=None, device="cpu"):
    """Timed region of the whole job: the maximum over ranks of each rank's
    ms (every rank runs its own replica), ms per step, and the whole-job
    seconds per solve (all ranks' solves in that time)."""
    import torch
    if dist is not None and world > 1:
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ms / steps, ms / 1000.0 / (steps * world)


# --------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.kernels:
        return kernel_arm(args)
    if args.workload == "batch":
        return batch_arm(args)
    if args.workload == "learned":
        return learned_arm(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1901_08269_gb300 import cfp
    from paper_1901_08269_gb300 import workloads as W

    w = W.config3(args.n)
    stream = torch.cuda.current_stream()
    ctx = cfp.Context(w.x, w.y, w.z, w.bodies, stream=stream)
    t_type = torch.empty(w.N, dtype=torch.uint8, device="cuda")
    ctx.classify_points(t_type)
    xyz = ctx.ibi_points()
    f, g = w.fields(torch, "cuda")
    gi = w.g_at(xyz, torch).contiguous()
    u = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    prec = cfp.PREC_MIXED if args.precision == "mixed" else cfp.PREC_FP64
    pc = cfp.PRECOND_MG if args.precond == "mg" else cfp.PRECOND_RBGS
    opts = cfp.default_opts(precision=prec, sweeps=args.sweeps, inner_tol=args.inner_tol, precond=pc,
                            mg_smooth=args.mg_smooth, mg_post=args.mg_post, use_graph=0 if args.no_graph else 1)

    def step():
        ctx.classify_points()
        u.zero_()
        return ctx.solve(f, g, gi, u, tol=args.tol, opts=opts)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    # phase split of one step (outside the timed region)
    a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record(stream)
    ctx.classify_points()
    b.record(stream)
    u.zero_()
    ctx.solve(f, g, gi, u, tol=args.tol, opts=opts)
    c2.record(stream)
    torch.cuda.synchronize()
    phases = {"setup_ms": a.elapsed_time(b), "rhs_and_solve_ms": b.elapsed_time(c2)}
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    l0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    infos = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ctx.launch_count() - l0
    clk = clocks.stop()
    ms, ms_per_step, value = job_time(e0.elapsed_time(e1), args.steps, world, dist, "cuda")

    X, Y, Z = w.mesh(torch, "cuda")
    ue = w.u(X, Y, Z, torch).reshape(-1)
    fluid = t_type != cfp.SOLID
    err = float((u - ue).abs()[fluid].max())
    info = infos[-1]
    result = {"max_err": err, "iterations": info.iterations, "refinements": info.refinements,
              "rel_residual": info.rel_residual, "n_irregular": info.n_irregular, "n_ibi": info.n_ibi,
              "n_degenerate": info.n_degenerate}
    del X, Y, Z

    fp64 = None
    if not args.no_fp64_check:
        # the plain FP64 solve of the same step (classification + solve), one
        # untimed run (it builds the FP64 graph), then the mean of fp64_steps
        u64 = torch.zeros_like(u)
        k64 = max(1, min(args.steps, args.fp64_steps))

        def step64():
            ctx.classify_points()
            u64.zero_()
            return ctx.solve(f, g, gi, u64, tol=args.tol, precision=cfp.PREC_FP64, sweeps=args.sweeps,
                             precond=pc, mg_smooth=args.mg_smooth, mg_post=args.mg_post)

        step64()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k64):
            i64 = step64()
        b.record(stream)
        torch.cuda.synchronize()
        e64 = float((u64 - ue).abs()[fluid].max())
        fp64 = {"s_per_solve": a.elapsed_time(b) / 1000.0 / k64, "steps": k64, "max_err": e64,
                "iterations": i64.iterations, "err_ratio_vs_fp64": err / e64 if e64 > 0 else None,
                "equal_error": err <= 1.02 * e64, "max_diff_vs_fp64": float((u - u64).abs().max()),
                "speedup_mixed_vs_fp64": (a.elapsed_time(b) / 1000.0 / k64) / value}
        del u64

    # roofline of the dominant kernel: a red-black half-sweep of the
    # preconditioner (the multigrid smoother on the fine level, or the plain
    # inner iterations), in the precision of the inner solve
    kprec = prec
    kern = {}
    for name, kid in (("rb_half", cfp.KERNEL_MG_SWEEP), ("apply", cfp.KERNEL_APPLY), ("update", cfp.KERNEL_UPDATE)):
        kms, kbytes = ctx.time_kernel(kid, kprec, reps=20)
        kern[name] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6}
    peak, psrc = hbm_peak()
    tname = "float" if kprec == cfp.PREC_MIXED else "double"
    # both the multigrid smoother and the plain red-black inner iterations run
    # this half-sweep (red and black nodes in separate arrays); in FP32 on rows
    # of >= 192 nodes it is the TMA-fed kernel
    if kprec == cfp.PREC_MIXED and args.n // 2 >= 96:
        kname = "k_sweep_tma half-sweep"
    else:
        kname = "k_sweep_split<%s> half-sweep" % tname
    dom, src = kern["rb_half"], "cfp_mg.cu"
    roofline = {"bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": dom["gbs"] / peak, "traffic": None, "kernel": kname, "peak_source": psrc}
    tr = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr):
        try:
            d = json.load(open(tr)).get(kname)
            if d and d.get("source_sha") == _src_hash(src):
                roofline["traffic"] = d["bytes_per_interior_node"] * (args.n - 2) ** 3
        except Exception:
            pass

    e2e = None
    if not args.no_e2e:
        hf = f.cpu().pin_memory()
        hg = g.cpu().pin_memory()
        hgi = gi.cpu().pin_memory()
        hu = torch.zeros(w.N, dtype=torch.float64).pin_memory()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # one untimed call: the first allocates the context's device copies of the host buffers
        ctx.solve_host(hf, hg, hgi, hu, tol=args.tol, opts=opts)
        torch.cuda.synchronize()
        # each step: classification, the copies of f, g, g at the IBI points and
        # the initial guess in, the solve and the copy of u out, between two
        # events; the initial guess is zeroed in host memory before the span
        # (as f and g, it is the caller's input), and the spans of the same
        # steps as the headline are averaged
        es_sum = 0.0
        for _ in range(args.steps):
            hu.zero_()
            a.record(stream)
            ctx.classify_points()
            ctx.solve_host(hf, hg, hgi, hu, tol=args.tol, opts=opts)
            b.record(stream)
            torch.cuda.synchronize()
            es_sum += a.elapsed_time(b) / 1000.0
        es = es_sum / args.steps
        h2d = (hf.numel() + hg.numel() + hu.numel() + hgi.numel()) * 8
        e2e = {"value": es / world, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": hu.numel() * 8,
               "steps": args.steps}
        del hf, hg, hgi, hu

    cpu = None
    if rank == 0 and not args.no_cpu:
        iters_full = FP64_RBGS_ITERS_513
        small = oracle_sample(args.oracle_n, args.oracle_iters)
        large = oracle_sample(args.oracle_large or 2 * args.oracle_n - 1, args.oracle_iters)
        est = oracle_extrapolate(small, large, args.n, iters_full)
        cpu = {"value": est["est_s_per_solve"], "unit": UNIT, "cores": large["cores"], "kind": "oracle",
               "sample": oracle_text(small, large, est, args.n, iters_full),
               "measured": {"n%d" % small["n"]: small, "n%d" % large["n"]: large}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if prec == cfp.PREC_MIXED else "f64", "data": "synthetic",
                "config": dict(workload_config(args, world), precision=args.precision, inner_tol=args.inner_tol,
                               sweeps=args.sweeps, precond=args.precond, mg_smooth=args.mg_smooth,
                               mg_post=args.mg_post or args.mg_smooth, graph=not args.no_graph),
                "result": result, "phases": phases, "fp64": fp64, "kernels": kern, "roofline": roofline, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def _src_hash(name):
    import hashlib
    p = os.path.join(ROOT, "paper_1901_08269_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


if __name__ == "__main__":
    sys.exit(main())
