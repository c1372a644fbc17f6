// Batched solves and the solver-parameter autotuner.
//
// cfp_solve_batch runs many independent problems (for instance the random
// small geometries of the batched workload) at once: a pool of host threads
// takes problems from a shared counter and drives each one's solve on its
// own context.  Each context enqueues on its own stream and its iteration
// runs as one graph launch, so the problems overlap on the GPU; each result
// is bitwise the one a lone cfp_solve gives (same kernels, same order).
//
// cfp_autotune times a problem's solve under a small set of candidate
// settings (multigrid smoothing sweeps, inner tolerance of the mixed
// solve) and returns the fastest that converges.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "cfp_internal.cuh"

namespace cfp {
cfp_status solve_impl(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u, double tol,
                      const cfp_opts* opts, cfp_info* info);
}

using namespace cfp;

extern "C" cfp_status cfp_solve_batch(cfp_ctx* const* ctxs, int nprob, const double* const* f,
                                      const double* const* g, const double* const* gi, double* const* u,
                                      double tol, const cfp_opts* opts, int nthreads, cfp_info* infos) {
    if (!ctxs || !f || !g || !u || nprob < 0) return fail(CFP_EINVAL, "NULL batch array or negative count");
    for (int m = 0; m < nprob; ++m) {
        if (!ctxs[m] || !f[m] || !g[m] || !u[m]) return fail(CFP_EINVAL, "NULL entry in the batch");
        for (int q = 0; q < m; ++q)
            if (ctxs[q] == ctxs[m]) return fail(CFP_EINVAL, "a context appears twice in the batch");
    }
    int dev = 0;
    CFP_CUDA(cudaGetDevice(&dev));
    const int nt = std::max(1, std::min(nprob, nthreads > 0 ? nthreads : 16));
    std::vector<cfp_status> st(nprob, CFP_OK);
    std::vector<std::string> msg(nprob);
    std::atomic<int> next(0);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int m = next.fetch_add(1);
            if (m >= nprob) break;
            cfp_ctx* c = ctxs[m];
            cfp_info info = {};
            cfp_status s = CFP_OK;
            if (!c->classified) s = classify(c);
            if (s == CFP_OK) {
                const double* gim = gi ? gi[m] : nullptr;
                if (c->n_ibi > 0 && !gim) s = fail(CFP_EINVAL, "g_ibi missing for a problem with IBI points");
                else s = solve_impl(c, f[m], g[m], gim, u[m], tol, opts, &info);
            }
            st[m] = s;
            if (s != CFP_OK) msg[m] = cfp_last_error();
            if (infos) infos[m] = info;
            if (infos && s != CFP_OK) infos[m].status = s;
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (int m = 0; m < nprob; ++m)
        if (st[m] != CFP_OK) return fail(st[m], "problem " + std::to_string(m) + ": " + msg[m]);
    return CFP_OK;
}

extern "C" cfp_status cfp_autotune(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u,
                                   double tol, cfp_opts* opts, double* best_ms) {
    if (!c || !opts) return fail(CFP_EINVAL, "NULL context or opts");
    if (!c->classified) CFP_TRY(classify(c));
    const cfp_opts base = *opts;
    const int smooth[3] = {1, 2, 3};
    const double itol[3] = {1e-2, 1e-3, 1e-4};
    double best = -1.0;
    cfp_opts pick = base;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < (base.precision == CFP_PREC_MIXED ? 3 : 1); ++b) {
            cfp_opts o = base;
            o.precond = CFP_PRECOND_MG;
            o.mg_smooth = smooth[a];
            if (base.precision == CFP_PREC_MIXED) o.inner_tol = itol[b];
            double t = 1e300;
            for (int rep = 0; rep < 2; ++rep) {  // the first run also builds the graphs
                CFP_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * c->N, c->stream));
                const auto t0 = std::chrono::steady_clock::now();
                cfp_info info;
                const cfp_status s = solve_impl(c, f, g, gi, u, tol, &o, &info);
                const double ms =
                    std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
                if (s != CFP_OK) {
                    t = 1e300;
                    break;
                }
                t = std::min(t, ms);
            }
            if (t < 1e300 && (best < 0.0 || t < best)) {
                best = t;
                pick = o;
            }
        }
    if (best < 0.0) return fail(CFP_ENOCONV, "no candidate setting converged");
    *opts = pick;
    if (best_ms) *best_ms = best;
    return CFP_OK;
}

// ------------------------------------------------------- one-graph batches
// cfp_batch: every problem's whole mixed-precision solve, its refinement and
// BiCGSTAB loops as while nodes driven by device-side scalars
// (capture_device_solve), captured as the parallel branches of ONE graph.
// A run is one graph launch for the whole batch: no host round trip between
// refinement steps or problems; the GPU interleaves the problems' kernels.
// The graph holds the contexts' buffers and settings; a context whose
// buffers were replaced since (a new classification, a new multigrid
// hierarchy, another apply kernel: its generation counter moved) makes the
// next run capture the graph again.
namespace cfp {
cfp_status capture_device_solve(cfp_ctx* c, cudaStream_t s, const double* f, const double* g, const double* gi,
                                double* u, double tol, const cfp_opts& opts, int64_t counts[3]);
cfp_status prepare_device_solve(cfp_ctx* c, const cfp_opts& opts);
}  // namespace cfp

struct cfp_batch {
    std::vector<cfp_ctx*> ctxs;
    std::vector<const double*> f, g, gi;
    std::vector<double*> u;
    std::vector<cfp_opts> opts;
    double tol = 0.0;
    std::vector<int64_t> gens;            // the contexts' generations the graph was captured at
    std::vector<int64_t> pro, outer, inner;  // kernels per solve: outside the loops, per refinement body, per BiCGSTAB body
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

cfp_status batch_capture(cfp_batch* b) {
    const int n = (int)b->ctxs.size();
    for (int m = 0; m < n; ++m) {
        cfp_ctx* c = b->ctxs[m];
        CFP_TRY(prepare_device_solve(c, b->opts[m]));
        if (c->n_ibi > 0 && !b->gi[m]) return fail(CFP_EINVAL, "problem " + std::to_string(m) + ": g_ibi missing");
        CFP_CUDA(cudaStreamSynchronize(c->stream));
    }
    std::vector<cudaStream_t> ss(n, nullptr);
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    cfp_status st = CFP_OK;
    for (int m = 0; m < n && st == CFP_OK; ++m)
        if (cudaStreamCreateWithFlags(&ss[m], cudaStreamNonBlocking) != cudaSuccess) st = fail(CFP_ECUDA, "stream");
    for (int m = 0; m <= n && st == CFP_OK; ++m)
        if (cudaEventCreateWithFlags(&ev[m], cudaEventDisableTiming) != cudaSuccess) st = fail(CFP_ECUDA, "event");
    cudaGraph_t graph = nullptr;
    if (st == CFP_OK) {
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamBeginCapture");
        if (st == CFP_OK) {
            cudaEventRecord(ev[n], b->stream);
            for (int m = 0; m < n && st == CFP_OK; ++m) {
                cfp_ctx* c = b->ctxs[m];
                cudaStreamWaitEvent(ss[m], ev[n], 0);
                int64_t counts[3] = {0, 0, 0};
                st = capture_device_solve(c, ss[m], b->f[m], b->g[m], b->gi[m], b->u[m], b->tol, b->opts[m], counts);
                b->pro[m] = counts[0];
                b->outer[m] = counts[1];
                b->inner[m] = counts[2];
                cudaEventRecord(ev[m], ss[m]);
                cudaStreamWaitEvent(b->stream, ev[m], 0);
            }
            e = cudaStreamEndCapture(b->stream, &graph);
            if (st == CFP_OK && e != cudaSuccess) st = cuda_fail(e, "capturing the batch");
        }
    }
    if (st == CFP_OK && b->exec) {
        // the same topology (the usual case: the same problems reclassified)
        // updates the instantiated graph in place, cheaper than a new one
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(b->exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (st == CFP_OK && !b->exec) {
        const cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphInstantiate (batch)");
    }
    if (st != CFP_OK && b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
    for (cudaStream_t s : ss)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (st != CFP_OK) return st;
    for (int m = 0; m < n; ++m) b->gens[m] = b->ctxs[m]->generation;
    return CFP_OK;
}

}  // namespace

extern "C" cfp_status cfp_batch_create(cfp_ctx* const* ctxs, int nprob, const double* const* f,
                                       const double* const* g, const double* const* gi, double* const* u, double tol,
                                       const cfp_opts* opts, cfp_batch** out) {
    if (!out) return fail(CFP_EINVAL, "NULL output");
    *out = nullptr;
    if (!ctxs || !f || !g || !u || nprob < 1) return fail(CFP_EINVAL, "NULL batch array or no problem");
    if (!(tol > 0.0)) return fail(CFP_EINVAL, "bad tol");
    for (int m = 0; m < nprob; ++m) {
        if (!ctxs[m] || !f[m] || !g[m] || !u[m]) return fail(CFP_EINVAL, "NULL entry in the batch");
        for (int q = 0; q < m; ++q)
            if (ctxs[q] == ctxs[m]) return fail(CFP_EINVAL, "a context appears twice in the batch");
    }
    cfp_batch* b = new cfp_batch();
    b->ctxs.assign(ctxs, ctxs + nprob);
    b->f.assign(f, f + nprob);
    b->g.assign(g, g + nprob);
    b->gi.assign(nprob, nullptr);
    if (gi) b->gi.assign(gi, gi + nprob);
    b->u.assign(u, u + nprob);
    b->opts.resize(nprob);
    for (int m = 0; m < nprob; ++m) {
        if (opts) b->opts[m] = opts[m];
        else cfp_default_opts(&b->opts[m]);
    }
    b->tol = tol;
    b->gens.assign(nprob, -1);
    b->pro.assign(nprob, 0);
    b->outer.assign(nprob, 0);
    b->inner.assign(nprob, 0);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return fail(CFP_ECUDA, "cudaStreamCreateWithFlags");
    }
    const cfp_status st = batch_capture(b);
    if (st != CFP_OK) {
        cfp_batch_destroy(b);
        return st;
    }
    *out = b;
    return CFP_OK;
}

extern "C" cfp_status cfp_batch_run(cfp_batch* b, cfp_info* infos) {
    if (!b) return fail(CFP_EINVAL, "NULL batch");
    const int n = (int)b->ctxs.size();
    bool stale = !b->exec;
    for (int m = 0; m < n; ++m) stale = stale || b->gens[m] != b->ctxs[m]->generation || !b->ctxs[m]->classified;
    if (stale) CFP_TRY(batch_capture(b));
    for (int m = 0; m < n; ++m) CFP_CUDA(cudaStreamSynchronize(b->ctxs[m]->stream));  // the inputs are ready
    const auto t0 = std::chrono::steady_clock::now();
    CFP_CUDA(cudaGraphLaunch(b->exec, b->stream));
    CFP_CUDA(cudaStreamSynchronize(b->stream));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    cfp_status first = CFP_OK;
    std::string msg;
    for (int m = 0; m < n; ++m) {
        cfp_ctx* c = b->ctxs[m];
        CFP_CUDA(cudaMemcpy(c->hrst, c->rst, sizeof(RState), cudaMemcpyDeviceToHost));
        const RState& R = *c->hrst;
        cfp_status s = R.status == RSTATE_RUN ? CFP_ENOCONV : (cfp_status)R.status;
        const cfp_status w = check_waits(c);
        if (s == CFP_OK && w != CFP_OK) s = w;
        const int64_t launches = b->pro[m] + (int64_t)R.outer * b->outer[m] + R.inner_execs * b->inner[m];
        c->launches += launches;
        if (infos) {
            cfp_info& info = infos[m];
            info = cfp_info{};
            info.status = s;
            info.iterations = R.total;
            info.restarts = 0;
            info.refinements = R.refinements;
            info.rel_residual = R.rel;
            info.n_irregular = c->n_irr;
            info.n_ibi = c->n_ibi;
            info.n_degenerate = c->n_deg;
            info.ms_solve = ms;
            info.launches = launches;
        }
        if (s != CFP_OK && first == CFP_OK) {
            first = s;
            msg = "problem " + std::to_string(m) + ": " +
                  (s == CFP_ENAN ? "non-finite value in the solve"
                   : s == CFP_EBREAKDOWN ? "BiCGSTAB breakdown after restarts"
                   : s == CFP_ECUDA ? std::string(cfp_last_error())
                                    : "no convergence within the iteration cap");
        }
    }
    if (first != CFP_OK) return fail(first, msg);
    return CFP_OK;
}

extern "C" void cfp_batch_destroy(cfp_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}
