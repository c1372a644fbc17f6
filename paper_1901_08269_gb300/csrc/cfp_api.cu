// C-ABI entry points of include/cfp.h: context life cycle, argument checks,
// error reporting, and the 1D grid metrics (Eq. app_xxx, Eq. 2ndorder_coef).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <mutex>

#include "cfp_internal.cuh"

namespace cfp {
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool
            cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}
}  // namespace cfp

namespace cfp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

cfp_status fail(cfp_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

cfp_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? CFP_ENOMEM : CFP_ECUDA;
}

cfp_status solve_impl(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u, double tol,
                      const cfp_opts* opts, cfp_info* info);

namespace {

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cfp_status need_classified(cfp_ctx* c) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (c->class_status != CFP_OK) return fail(c->class_status, "classification failed earlier");
    if (!c->classified) return fail(CFP_ESTATE, "call cfp_classify_points first");
    return CFP_OK;
}

cfp_status need_field(const void* p, const char* name) {
    if (!p) return fail(CFP_EINVAL, std::string(name) + " is NULL");
    if (!is_device_ptr(p)) return fail(CFP_EINVAL, std::string(name) + " is not a device pointer");
    return CFP_OK;
}

}  // namespace
}  // namespace cfp

using namespace cfp;

extern "C" {

void cfp_default_opts(cfp_opts* o) {
    if (!o) return;
    o->precision = CFP_PREC_FP64;
    o->sweeps = 8;
    o->maxit = 50000;
    o->max_restarts = 3;
    o->inner_tol = 1e-5;
    o->max_refine = 40;
    o->use_graph = 1;
    o->precond = CFP_PRECOND_RBGS;
    o->mg_smooth = 2;
    o->mg_post = 0;
    o->mg_tma = 1;
}

const char* cfp_last_error(void) { return g_last_error.c_str(); }

cfp_status cfp_ctx_create(const double* x, int nx, const double* y, int ny, const double* z, int nz,
                          const cfp_body* bodies, int nbodies, int fluid_inside, void* stream, cfp_ctx** out) {
    if (!out) return fail(CFP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!x || !y || !z) return fail(CFP_EINVAL, "coordinate array is NULL");
    if (nx < 3 || ny < 3 || nz < 3) return fail(CFP_EINVAL, "need at least 3 nodes per axis");
    if (nbodies < 0 || (nbodies > 0 && !bodies)) return fail(CFP_EINVAL, "bad body list");
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= ((int64_t)1 << 31)) return fail(CFP_EINVAL, "grid too large (N must be below 2^31)");
    const double* src[3] = {x, y, z};
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i + 1 < n[d]; ++i)
            if (!(src[d][i + 1] > src[d][i]) || !isfinite(src[d][i]) || !isfinite(src[d][i + 1]))
                return fail(CFP_EINVAL, "coordinates must be finite and strictly increasing");
    for (int m = 0; m < nbodies; ++m) {
        const cfp_body& b = bodies[m];
        if (b.kind < CFP_SPHERE || b.kind > CFP_TORUS) return fail(CFP_EINVAL, "unknown body kind");
        const int np = b.kind == CFP_SPHERE ? 1 : (b.kind == CFP_TORUS ? 2 : 3);
        for (int q = 0; q < np; ++q)
            if (!(b.p[q] > 0.0)) return fail(CFP_EINVAL, "body sizes must be positive");
        for (int r = 0; r < 3; ++r)       // R must be a rotation: R^T R = I
            for (int q = 0; q < 3; ++q) {
                double d = 0.0;
                for (int m2 = 0; m2 < 3; ++m2) d += b.R[3 * m2 + r] * b.R[3 * m2 + q];
                if (!(fabs(d - (r == q ? 1.0 : 0.0)) <= 1e-9)) return fail(CFP_EINVAL, "body R is not a rotation");
            }
    }
    cfp_ctx* c = new cfp_ctx();
    c->N = N;
    c->stream = (cudaStream_t)stream;
    c->fluid_inside = fluid_inside ? 1 : 0;
    c->bodies.assign(bodies, bodies + nbodies);
    cudaGetDevice(&c->device);
    cfp_status st = CFP_OK;
    auto chk = [&](cudaError_t e, const char* w) {
        if (e != cudaSuccess && st == CFP_OK) st = cuda_fail(e, w);
    };
    int64_t ncoef = 0;
    for (int d = 0; d < 3; ++d) {
        c->n[d] = n[d];
        c->X[d].assign(src[d], src[d] + n[d]);
        ncoef += 8 * (int64_t)n[d];
    }
    chk(cudaMalloc(&c->dcoef64, sizeof(double) * ncoef), "cudaMalloc");
    chk(cudaMalloc(&c->dcoef32, sizeof(float) * ncoef), "cudaMalloc");
    for (int d = 0; d < 3; ++d) chk(cudaMalloc(&c->dX[d], sizeof(double) * n[d]), "cudaMalloc");
    chk(cudaMalloc(&c->dbodies, sizeof(cfp_body) * std::max(nbodies, 1)), "cudaMalloc");
    chk(cudaMalloc(&c->dbody32, sizeof(Body32) * std::max(nbodies, 1)), "cudaMalloc");
    chk(cudaMalloc(&c->type, (size_t)N), "cudaMalloc");
    chk(cudaMalloc(&c->slot, sizeof(int32_t) * (size_t)N), "cudaMalloc");
    chk(cudaMalloc(&c->dtotal, sizeof(long long) * 8), "cudaMalloc");
    chk(cudaMalloc(&c->derr, sizeof(DevError)), "cudaMalloc");
    chk(cudaMalloc(&c->dwait, sizeof(int)), "cudaMalloc");
    if (c->dwait) chk(cudaMemsetAsync(c->dwait, 0, sizeof(int), c->stream), "cudaMemsetAsync");
    chk(cudaMalloc(&c->kst, sizeof(KState) * 2), "cudaMalloc");
    chk(cudaMallocHost(&c->hkst, sizeof(KState) * 2), "cudaMallocHost");
    chk(cudaMalloc(&c->rst, sizeof(RState)), "cudaMalloc");
    chk(cudaMallocHost(&c->hrst, sizeof(RState)), "cudaMallocHost");
    for (int q = 0; q < 3; ++q) {
        chk(cudaStreamCreateWithFlags(&c->auxs[q], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
        chk(cudaEventCreateWithFlags(&c->evfs[q], cudaEventDisableTiming), "cudaEventCreateWithFlags");
        chk(cudaEventCreateWithFlags(&c->evjs[q], cudaEventDisableTiming), "cudaEventCreateWithFlags");
    }
    use_aux(c, 0);
    if (st == CFP_OK) {
        for (int d = 0; d < 3; ++d)
            chk(cudaMemcpyAsync(c->dX[d], src[d], sizeof(double) * n[d], cudaMemcpyHostToDevice, c->stream),
                "cudaMemcpyAsync");
        launch_metrics(c);
        if (nbodies) {
            chk(cudaMemcpyAsync(c->dbodies, bodies, sizeof(cfp_body) * nbodies, cudaMemcpyHostToDevice, c->stream),
                "cudaMemcpyAsync");
            // bounding radius: sphere r, ellipsoid largest semi-axis, torus R + r;
            // the 1e-3 relative margin keeps phi far from zero outside it
            // (R is a rotation, so the body frame keeps distances).  The
            // device tests the squared distance in FP32, from the FP32
            // coordinates and centre: per axis its error is at most
            // 2.0001 u A (A = the largest |coordinate| + |centre|, u = 2^-24),
            // the squared distance's at most 7.01 u sum A^2; the threshold
            // adds 16 u sum A^2 and rounds up, so an FP32 distance above it
            // means an exact one above the bound.
            double amax[3];
            for (int d = 0; d < 3; ++d) {
                amax[d] = 0.0;
                for (int i = 0; i < n[d]; ++i) amax[d] = std::max(amax[d], fabs(src[d][i]));
            }
            static thread_local std::vector<Body32> sp;
            sp.assign(nbodies, Body32{});
            for (int m = 0; m < nbodies; ++m) {
                const cfp_body& b = bodies[m];
                const double r = b.kind == CFP_SPHERE ? b.p[0]
                               : b.kind == CFP_ELLIPSOID ? std::max(b.p[0], std::max(b.p[1], b.p[2]))
                                                         : b.p[0] + b.p[1];
                double a2 = 0.0;
                for (int d = 0; d < 3; ++d) a2 += (amax[d] + fabs(b.c[d])) * (amax[d] + fabs(b.c[d]));
                const double thr = (r * 1.001) * (r * 1.001) + 16.0 * ldexp(1.0, -24) * a2;
                float tf = (float)thr;
                if ((double)tf < thr) tf = nextafterf(tf, INFINITY);
                Body32& B = sp[m];
                B.kind = b.kind;
                for (int q = 0; q < 3; ++q) {
                    B.c[q] = (float)b.c[q];
                    B.p[q] = (float)b.p[q];
                    B.ip[q] = b.kind == CFP_ELLIPSOID ? (float)(1.0 / b.p[q]) : 0.f;
                }
                for (int q = 0; q < 9; ++q) B.R[q] = (float)b.R[q];
                B.thr = tf;
            }
            chk(cudaMemcpy(c->dbody32, sp.data(), sizeof(Body32) * nbodies, cudaMemcpyHostToDevice), "cudaMemcpy");
        }
        chk(cudaGetLastError(), "k_metrics");
        chk(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    }
    if (st != CFP_OK) {
        cfp_ctx_destroy(c);
        return st;
    }
    *out = c;
    return CFP_OK;
}

void cfp_ctx_destroy(cfp_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (int q = 0; q < 2; ++q)
        if (c->gexec[q]) cudaGraphExecDestroy(c->gexec[q]);
    free_mg(c);
    free_ilu(c);
    void* ptrs[] = {c->dcoef64, c->dcoef32, c->dX[0], c->dX[1], c->dX[2], c->dbodies, c->dbody32, c->type, c->slot, c->irr_lin,
                    c->ibi_off, c->ibi_xyz, c->corr_ptr, c->corr_off, c->corr_val, c->corr_val32, c->bib_ptr,
                    c->bib_idx, c->bib_val, c->krow, c->krow32, c->side_scratch, c->scan_bsum, c->dtotal, c->derr, c->dwait, c->nn_wflip, c->v64, c->v32,
                    c->partial, c->kst, c->rst, c->hs_f, c->hs_g, c->hs_u, c->hs_gi};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->hkst) cudaFreeHost(c->hkst);
    if (c->hrst) cudaFreeHost(c->hrst);
    for (int q = 0; q < 3; ++q) {
        if (c->auxs[q]) cudaStreamSynchronize(c->auxs[q]), cudaStreamDestroy(c->auxs[q]);
        if (c->evfs[q]) cudaEventDestroy(c->evfs[q]);
        if (c->evjs[q]) cudaEventDestroy(c->evjs[q]);
    }
    delete c;
}

cfp_status cfp_classify_points(cfp_ctx* c, uint8_t* type_dev, int64_t* n_irregular, int64_t* n_ibi) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (type_dev && !is_device_ptr(type_dev)) return fail(CFP_EINVAL, "type_dev is not a device pointer");
    CFP_TRY(classify(c));
    if (type_dev) CFP_CUDA(cudaMemcpyAsync(type_dev, c->type, (size_t)c->N, cudaMemcpyDeviceToDevice, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    if (n_irregular) *n_irregular = c->n_irr;
    if (n_ibi) *n_ibi = c->n_ibi;
    return CFP_OK;
}

cfp_status cfp_ibi_points(cfp_ctx* c, double* xyz, int on_host) {
    CFP_TRY(need_classified(c));
    if (c->n_ibi == 0) return CFP_OK;
    if (!xyz) return fail(CFP_EINVAL, "xyz is NULL");
    if (!on_host && !is_device_ptr(xyz)) return fail(CFP_EINVAL, "xyz is not a device pointer");
    CFP_CUDA(cudaMemcpyAsync(xyz, c->ibi_xyz, sizeof(double) * 3 * c->n_ibi,
                             on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    if (on_host) CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

cfp_status cfp_assemble_rhs(cfp_ctx* c, const double* f, const double* g, const double* gi, double* rhs) {
    CFP_TRY(need_classified(c));
    CFP_TRY(need_field(f, "f_dev"));
    CFP_TRY(need_field(g, "g_nodes_dev"));
    CFP_TRY(need_field(rhs, "rhs_dev"));
    if (c->n_ibi > 0) CFP_TRY(need_field(gi, "g_ibi_dev"));
    return assemble_rhs(c, f, g, gi, rhs);
}

}  // extern "C"

// the right-hand side after the checks (also of the solves, whose f, g and
// g_ibi may be page-locked host memory the kernels read in place)
cfp_status cfp::assemble_rhs(cfp_ctx* c, const double* f, const double* g, const double* gi, double* rhs) {
    CFP_TRY(ensure_work(c, false));
    double* gb = c->v64 + V_TMP * vstride(c);
    double* bg = c->v64 + V_TMP2 * vstride(c);
    double* qf = c->v64 + V_T * vstride(c);
    if (rhs == gb || rhs == bg || rhs == qf) return fail(CFP_EINVAL, "rhs aliases the context's work space");
    launch_boundary_lift(c, g, gb, c->stream);
    launch_apply_lift(c, gb, bg, c->stream);
    launch_qf(c, f, qf, c->stream);
    launch_rhs_finish(c, qf, bg, c->n_ibi ? gi : c->ibi_xyz, rhs, c->stream);
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

extern "C" {

cfp_status cfp_apply(cfp_ctx* c, const double* x, double* y) {
    CFP_TRY(need_classified(c));
    CFP_TRY(need_field(x, "x_dev"));
    CFP_TRY(need_field(y, "y_dev"));
    if (x == y) return fail(CFP_EINVAL, "x and y must not overlap");
    CFP_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * c->N, c->stream));
    launch_apply<double>(c, x, y, nullptr, 0, nullptr, c->stream, nullptr);
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_apply_f32(cfp_ctx* c, const float* x, float* y) {
    CFP_TRY(need_classified(c));
    CFP_TRY(need_field(x, "x_dev"));
    CFP_TRY(need_field(y, "y_dev"));
    if (x == y) return fail(CFP_EINVAL, "x and y must not overlap");
    setup_apply_ring(c);
    CFP_CUDA(cudaMemsetAsync(y, 0, sizeof(float) * c->N, c->stream));
    launch_apply<float>(c, x, y, nullptr, 0, nullptr, c->stream, nullptr);
    CFP_CUDA(cudaGetLastError());
    return check_waits(c);
}

cfp_status cfp_precondition(cfp_ctx* c, int sweeps, const double* rho, double* phi) {
    CFP_TRY(need_classified(c));
    CFP_TRY(need_field(rho, "rho_dev"));
    CFP_TRY(need_field(phi, "phi_dev"));
    if (sweeps < 0) return fail(CFP_EINVAL, "sweeps must be >= 0");
    if (rho == phi) return fail(CFP_EINVAL, "rho and phi must not overlap");
    CFP_TRY(ensure_work(c, false));
    if (phi == c->v64 + (int64_t)V_TMP2 * vstride(c)) return fail(CFP_EINVAL, "phi aliases the context's work space");
    if (sweeps > 0) CFP_TRY(ensure_mg(c, 0));
    CFP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * c->N, c->stream));
    c->precond_kind = CFP_PRECOND_RBGS;
    launch_precond<double>(c, sweeps, rho, phi, c->stream);
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_precondition_ex(cfp_ctx* c, const cfp_opts* o, const double* rho, double* phi) {
    cfp_opts opts;
    cfp_default_opts(&opts);
    if (o) opts = *o;
    CFP_TRY(need_classified(c));
    CFP_TRY(need_field(rho, "rho_dev"));
    CFP_TRY(need_field(phi, "phi_dev"));
    if (opts.sweeps < 0 ||
        (opts.precond != CFP_PRECOND_RBGS && opts.precond != CFP_PRECOND_MG && opts.precond != CFP_PRECOND_ILU))
        return fail(CFP_EINVAL, "bad sweeps or preconditioner");
    if (opts.precision != CFP_PREC_FP64 && opts.precision != CFP_PREC_MIXED) return fail(CFP_EINVAL, "bad precision");
    if (rho == phi) return fail(CFP_EINVAL, "rho and phi must not overlap");
    const int prec = opts.precision == CFP_PREC_MIXED ? 1 : 0;
    CFP_TRY(ensure_work(c, prec == 1));
    if (phi == c->v64 + (int64_t)V_TMP2 * vstride(c)) return fail(CFP_EINVAL, "phi aliases the context's work space");
    c->precond_kind = opts.precond;
    c->mg_smooth = std::max(1, opts.mg_smooth);
    c->mg_post = opts.mg_post > 0 ? opts.mg_post : c->mg_smooth;
    c->mg_tma = opts.mg_tma != 0;
    c->mg_fuse = opts.mg_tma == 2;
    cfp_status st = CFP_OK;
    if (c->precond_kind == CFP_PRECOND_MG || (c->precond_kind == CFP_PRECOND_RBGS && opts.sweeps > 0))
        st = ensure_mg(c, prec);
    if (st == CFP_OK && c->precond_kind == CFP_PRECOND_ILU) st = ensure_ilu(c, prec);
    if (st == CFP_OK) {
        if (prec == 1) {
            st = precondition32(c, opts.sweeps, rho, phi);
            if (st == CFP_OK) st = check_waits(c);
        } else {
            CFP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * c->N, c->stream));
            launch_precond<double>(c, opts.sweeps, rho, phi, c->stream);
            CFP_CUDA(cudaGetLastError());
        }
    }
    c->precond_kind = CFP_PRECOND_RBGS;
    return st;
}

cfp_status cfp_solve(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u, double tol,
                     const cfp_opts* opts, cfp_info* info) {
    if (!c) return fail(CFP_EINVAL, "null context");
    CFP_TRY(need_field(f, "f_dev"));
    CFP_TRY(need_field(g, "g_nodes_dev"));
    CFP_TRY(need_field(u, "u_dev"));
    if (!c->classified) CFP_TRY(classify(c));
    if (c->n_ibi > 0) CFP_TRY(need_field(gi, "g_ibi_dev"));
    return solve_impl(c, f, g, gi, u, tol, opts, info);
}

cfp_status cfp_solve_host(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u, double tol,
                          const cfp_opts* opts, cfp_info* info) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!f || !g || !u) return fail(CFP_EINVAL, "NULL host buffer");
    if (!c->classified) CFP_TRY(classify(c));
    if (c->n_ibi > 0 && !gi) return fail(CFP_EINVAL, "g_ibi_host is NULL");
    // page-locked host buffers are read and written by the kernels in place
    // (over the host link, once each: f by the source term, g at the box and
    // the initial guess at the start, u written by the last kernel), with no
    // staging copy; other host memory goes through the context's device buffers
    auto mapped = [](const void* p) -> void* {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
    };
    {
        const double* df = static_cast<const double*>(mapped(f));
        const double* dg = static_cast<const double*>(mapped(g));
        double* du = static_cast<double*>(mapped(u));
        const double* dgi = c->n_ibi ? static_cast<const double*>(mapped(gi)) : nullptr;
        if (df && dg && du && (dgi || !c->n_ibi)) {
            const cfp_status st = solve_impl(c, df, dg, dgi, du, tol, opts, info);
            const std::string msg = g_last_error;
            CFP_CUDA(cudaStreamSynchronize(c->stream));
            if (st != CFP_OK) g_last_error = msg;
            return st;
        }
    }
    const size_t bytes = sizeof(double) * (size_t)c->N;
    if (!c->hs_f) CFP_CUDA(cudaMalloc(&c->hs_f, bytes));
    if (!c->hs_g) CFP_CUDA(cudaMalloc(&c->hs_g, bytes));
    if (!c->hs_u) CFP_CUDA(cudaMalloc(&c->hs_u, bytes));
    if (c->hs_gi_cap < std::max<int64_t>(c->n_ibi, 1)) {
        if (c->hs_gi) cudaFree(c->hs_gi);
        c->hs_gi = nullptr;
        CFP_CUDA(cudaMalloc(&c->hs_gi, sizeof(double) * std::max<int64_t>(c->n_ibi, 1)));
        c->hs_gi_cap = std::max<int64_t>(c->n_ibi, 1);
    }
    CFP_CUDA(cudaMemcpyAsync(c->hs_f, f, bytes, cudaMemcpyHostToDevice, c->stream));
    CFP_CUDA(cudaMemcpyAsync(c->hs_g, g, bytes, cudaMemcpyHostToDevice, c->stream));
    CFP_CUDA(cudaMemcpyAsync(c->hs_u, u, bytes, cudaMemcpyHostToDevice, c->stream));
    if (c->n_ibi)
        CFP_CUDA(cudaMemcpyAsync(c->hs_gi, gi, sizeof(double) * c->n_ibi, cudaMemcpyHostToDevice, c->stream));
    const cfp_status st = solve_impl(c, c->hs_f, c->hs_g, c->hs_gi, c->hs_u, tol, opts, info);
    const std::string msg = g_last_error;
    CFP_CUDA(cudaMemcpyAsync(u, c->hs_u, bytes, cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    if (st != CFP_OK) g_last_error = msg;
    return st;
}

int64_t cfp_launch_count(const cfp_ctx* c) { return c ? c->launches : 0; }

cfp_status cfp_time_kernel(cfp_ctx* c, int kernel, int precision, int reps, double* ms, double* bytes) {
    CFP_TRY(need_classified(c));
    return time_kernel(c, kernel, precision, reps, ms, bytes);
}

cfp_status cfp_apply_shape(const cfp_ctx* c, int precision, int* kernel, int* rows, int* planes) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (precision != CFP_PREC_FP64 && precision != CFP_PREC_MIXED) return fail(CFP_EINVAL, "bad precision");
    const int q = precision == CFP_PREC_MIXED ? 1 : 0;
    int k = 0, r = 0, p = 0;
    apply_shape(c, q, &k, &r, &p);
    if (kernel) *kernel = k;
    if (rows) *rows = r;
    if (planes) *planes = p;
    return CFP_OK;
}

cfp_status cfp_tune_apply(cfp_ctx* c, int precision, int kernel, int rows, int planes, double* ms) {
    CFP_TRY(need_classified(c));
    if (precision != CFP_PREC_FP64 && precision != CFP_PREC_MIXED) return fail(CFP_EINVAL, "bad precision");
    return tune_apply(c, precision, kernel, rows, planes, 5, ms);
}

cfp_status cfp_vec_dot(cfp_ctx* c, const double* a, const double* b, double* out) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!out) return fail(CFP_EINVAL, "NULL output");
    CFP_TRY(need_field(a, "a_dev"));
    CFP_TRY(need_field(b, "b_dev"));
    return vec_dot(c, a, b, out);
}

cfp_status cfp_vec_axpby(cfp_ctx* c, double alpha, const double* x, double beta, double* y) {
    if (!c) return fail(CFP_EINVAL, "null context");
    CFP_TRY(need_field(x, "x_dev"));
    CFP_TRY(need_field(y, "y_dev"));
    return vec_axpby(c, alpha, x, beta, y);
}

cfp_status cfp_diag_bounded_wait(cfp_ctx* c) {
    if (!c) return fail(CFP_EINVAL, "null context");
    return diag_bounded_wait(c);
}

}  // extern "C"
