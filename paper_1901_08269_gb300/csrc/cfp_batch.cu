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
