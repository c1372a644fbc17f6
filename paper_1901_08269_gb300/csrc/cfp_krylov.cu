// Preconditioned BiCGSTAB (Algorithm 1, Sec. 3.2), with the preconditioner
// of Sec. 3.3 applied on the right: p_hat = P p, s_hat = P s and the update
// u += alpha p_hat + omega s_hat.  All scalars live on the device; the
// iteration body is captured once per (precision, sweeps) into a CUDA graph
// whose while-node condition is set by the last scalar kernel, so a whole
// solve runs without returning to the host.  The iteration cap bounds the
// loop.
#include <math.h>

#include <algorithm>
#include <chrono>

#include "cfp_internal.cuh"

namespace cfp {
namespace {

__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double sa[32], sb[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
        for (int o = 16; o; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
    __syncthreads();
}

// fixed-order sum of nb pairs of block partials (one block of 256 threads)
__device__ void sum_partials(const double* partial, int nb, double& a, double& b) {
    a = 0.0;
    b = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        a += partial[2 * q];
        b += partial[2 * q + 1];
    }
    block_sum2(a, b);
}

#define GRID_STRIDE(l, N) \
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < (N); l += (int64_t)gridDim.x * blockDim.x)

// r = b - v (v = B x; NULL for x = 0: r = b), r_hat0 = r, p = r; partial (r, r)
template <class T>
__global__ void k_init_r(const T* __restrict__ b, const T* __restrict__ v, T* __restrict__ r, T* __restrict__ rh,
                         T* __restrict__ p, double* __restrict__ partial, int64_t N) {
    DotAcc<T> aa;
    GRID_STRIDE(l, N) {
        const T x = v ? b[l] - v[l] : b[l];
        r[l] = x;
        rh[l] = x;
        p[l] = x;
        aa.add(x, x);
    }
    double a = aa.total(), z = 0.0;
    block_sum2(a, z);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

// Algorithm 1, line 7: s = r - alpha v
template <class T>
__global__ void k_axpy_s(const T* __restrict__ r, const T* __restrict__ v, T* __restrict__ s,
                         const KState* __restrict__ st, int64_t N) {
    if (st->flag != FLAG_RUN) return;
    const T alpha = (T)st->alpha;
    GRID_STRIDE(l, N) s[l] = r[l] - alpha * v[l];
}

// Algorithm 1, lines 11-12 with the preconditioned directions:
// u += alpha p_hat + omega s_hat; r = s - omega t; partials (r_hat0, r), (r, r)
template <class T>
__global__ void k_update_xr(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ ph,
                            const T* __restrict__ sh, const T* __restrict__ s, const T* __restrict__ t,
                            const T* __restrict__ rh, const KState* __restrict__ st,
                            double* __restrict__ partial, int64_t N) {
    if (st->flag != FLAG_RUN) return;
    const T alpha = (T)st->alpha, omega = (T)st->omega;
    DotAcc<T> aa, bb;
    GRID_STRIDE(l, N) {
        x[l] += alpha * ph[l] + omega * sh[l];
        const T rn = s[l] - omega * t[l];
        r[l] = rn;
        aa.add(rh[l], rn);
        bb.add(rn, rn);
    }
    double a = aa.total(), b = bb.total();
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

// Algorithm 1, line 14: p = r + beta (p - omega v)
template <class T>
__global__ void k_update_p(T* __restrict__ p, const T* __restrict__ r, const T* __restrict__ v,
                           const KState* __restrict__ st, int64_t N) {
    if (st->flag != FLAG_RUN) return;
    const T beta = (T)st->beta, omega = (T)st->omega;
    GRID_STRIDE(l, N) p[l] = r[l] + beta * (p[l] - omega * v[l]);
}

__global__ void k_fin_init(KState* st, const double* partial, int nb) {
    double rr, z;
    sum_partials(partial, nb, rr, z);
    if (threadIdx.x == 0) {
        st->rr = rr;
        st->rho = rr;  // r_hat0 = r0
        st->iter = 0;
        st->flag = !isfinite(rr) ? FLAG_NAN : (rr <= st->stop2 ? FLAG_CONV : FLAG_RUN);
    }
}

// line 6: alpha = (r_hat0, r) / (r_hat0, v)
__global__ void k_fin_alpha(KState* st, const double* partial, int nb) {
    if (st->flag != FLAG_RUN) return;
    double sigma, z;
    sum_partials(partial, nb, sigma, z);
    if (threadIdx.x == 0) {
        st->sigma = sigma;
        if (!isfinite(sigma)) st->flag = FLAG_NAN;
        else if (sigma == 0.0) st->flag = FLAG_BREAK;
        else st->alpha = st->rho / sigma;
    }
}

// line 10: omega = (t, s) / (t, t)
__global__ void k_fin_omega(KState* st, const double* partial, int nb) {
    if (st->flag != FLAG_RUN) return;
    double ts, tt;
    sum_partials(partial, nb, ts, tt);
    if (threadIdx.x == 0) {
        st->ts = ts;
        st->tt = tt;
        if (!isfinite(tt) || !isfinite(ts)) st->flag = FLAG_NAN;
        else st->omega = tt > 0.0 ? ts / tt : 0.0;
    }
}

// line 13 and the stopping test; sets the graph's while condition
__global__ void k_fin_beta(KState* st, const double* partial, int nb, cudaGraphConditionalHandle h, int use_cond) {
    if (threadIdx.x == 0) st->execs += 1;
    if (st->flag == FLAG_RUN) {
        double rho_new, rr;
        sum_partials(partial, nb, rho_new, rr);
        if (threadIdx.x == 0) {
            st->iter += 1;
            st->rr = rr;
            st->rho_new = rho_new;
            if (!isfinite(rr)) st->flag = FLAG_NAN;
            else if (rr <= st->stop2) st->flag = FLAG_CONV;
            else if (st->omega == 0.0 || st->rho == 0.0) st->flag = FLAG_BREAK;
            else if (st->iter >= st->maxit) st->flag = FLAG_MAXIT;
            else {
                st->beta = (rho_new / st->rho) * (st->alpha / st->omega);
                st->rho = rho_new;
            }
        }
    }
    __syncthreads();
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(h, st->flag == FLAG_RUN ? 1u : 0u);
}

// out = b - y at every node; partial (out, out)
__global__ void k_resid(const double* __restrict__ b, const double* __restrict__ y, double* __restrict__ out,
                        double* __restrict__ partial, int64_t N) {
    double a = 0.0, z = 0.0;
    GRID_STRIDE(l, N) {
        const double v = b[l] - y[l];
        out[l] = v;
        a += v * v;
    }
    block_sum2(a, z);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ partial,
                      int64_t N) {
    double s = 0.0, z = 0.0;
    GRID_STRIDE(l, N) s += a[l] * b[l];
    block_sum2(s, z);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s;
        partial[2 * blockIdx.x + 1] = 0.0;
    }
}

__global__ void k_fin_store(const double* partial, int nb, double* out) {
    double a, b;
    sum_partials(partial, nb, a, b);
    if (threadIdx.x == 0) out[0] = a;
}

__global__ void k_to32(const double* __restrict__ in, float* __restrict__ out, double scale, int64_t N) {
    GRID_STRIDE(l, N) out[l] = (float)(in[l] * scale);
}

__global__ void k_add32(double* __restrict__ x, const float* __restrict__ e, double scale, int64_t N) {
    GRID_STRIDE(l, N) x[l] += (double)e[l] * scale;
}

template <class T>
__global__ void k_zero(T* __restrict__ x, int64_t N) {
    GRID_STRIDE(l, N) x[l] = T(0);
}

// --------------------------------------------------------------- host side
template <class T>
struct Vecs {
    T *x, *r, *rh, *p, *ph, *v, *s, *sh, *t;
};

Vecs<double> vecs64(cfp_ctx* c) {
    double* b = c->v64;
    const int64_t N = vstride(c);
    return Vecs<double>{b + V_X * N, b + V_R * N, b + V_RH * N, b + V_P * N, b + V_PH * N,
                        b + V_V * N, b + V_S * N, b + V_SH * N, b + V_T * N};
}
Vecs<float> vecs32(cfp_ctx* c) {
    float* b = c->v32;
    const int64_t N = vstride(c);
    return Vecs<float>{b + 0 * N, b + 1 * N, b + 2 * N, b + 3 * N, b + 4 * N, b + 5 * N, b + 6 * N, b + 7 * N, b + 8 * N};
}
template <class T>
Vecs<T> vecs(cfp_ctx* c);
template <>
Vecs<double> vecs<double>(cfp_ctx* c) { return vecs64(c); }
template <>
Vecs<float> vecs<float>(cfp_ctx* c) { return vecs32(c); }

// One iteration of Algorithm 1 (lines 4-14) on stream s.
template <class T>
void enqueue_body(cfp_ctx* c, int prec, int sweeps, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
    Vecs<T> V = vecs<T>(c);
    KState* st = c->kst + prec;
    const int64_t N = c->N;
    int nb = 0;
    launch_precond<T>(c, sweeps, V.p, V.ph, s);                       // line 4
    launch_apply<T>(c, V.ph, V.v, V.rh, 1, c->partial, s, &nb);        // line 5 (+ (r_hat0, v))
    k_fin_alpha<<<1, 256, 0, s>>>(st, c->partial, nb);                // line 6
    k_axpy_s<T><<<kUpdBlocks, kUpdThreads, 0, s>>>(V.r, V.v, V.s, st, N);  // line 7
    launch_precond<T>(c, sweeps, V.s, V.sh, s);                       // line 8
    launch_apply<T>(c, V.sh, V.t, V.s, 2, c->partial, s, &nb);         // line 9 (+ (t, s), (t, t))
    k_fin_omega<<<1, 256, 0, s>>>(st, c->partial, nb);                // line 10
    k_update_xr<T><<<kUpdBlocks, kUpdThreads, 0, s>>>(V.x, V.r, V.ph, V.sh, V.s, V.t, V.rh, st, c->partial, N);
    k_fin_beta<<<1, 256, 0, s>>>(st, c->partial, kUpdBlocks, h, use_cond);  // line 13 + stop test
    k_update_p<T><<<kUpdBlocks, kUpdThreads, 0, s>>>(V.p, V.r, V.v, st, N);  // line 14
    c->launches += 6;
}

int64_t body_launches(cfp_ctx* c);

// kernels of one iteration body, counted by enqueueing it on a dummy path
int64_t body_launches(cfp_ctx* c) { return c->body_launches; }

template <class T>
cfp_status build_graph(cfp_ctx* c, int prec, int sweeps) {
    if (c->gexec[prec] && c->gsweeps[prec] == sweeps && c->gprecond[prec] == c->precond_kind &&
        c->gmgs[prec] == mg_key(c) && c->ggen[prec] == c->generation)
        return CFP_OK;
    if (c->gexec[prec]) {
        cudaGraphExecDestroy(c->gexec[prec]);
        c->gexec[prec] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CFP_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    CFP_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CFP_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    CFP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        const int64_t saved = c->launches;
        enqueue_body<T>(c, prec, sweeps, cs, h, 1);
        c->body_launches = c->launches - saved;
        c->launches = saved;
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(cs, &out);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "capturing the BiCGSTAB body");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c->gexec[prec] = exec;
    c->ggen[prec] = c->generation;
    c->gsweeps[prec] = sweeps;
    c->gprecond[prec] = c->precond_kind;
    c->gmgs[prec] = mg_key(c);
    return CFP_OK;
}

// Solve B x = b (b and x zero off the unknowns) until ||r||^2 <= stop2 or
// maxit iterations; x holds the initial guess (x_zero: the caller knows it is
// zero, so r0 = b without applying B).  Returns the final flag.
template <class T>
cfp_status run_bicgstab(cfp_ctx* c, int prec, const T* b, double stop2, int maxit, int sweeps, bool use_graph,
                        bool x_zero, int* flag, int* used, double* rr) {
    Vecs<T> V = vecs<T>(c);
    KState* st = c->kst + prec;
    KState* hs = c->hkst + prec;
    const int64_t N = c->N;
    memset(hs, 0, sizeof(KState));
    hs->stop2 = stop2;
    hs->maxit = std::max(1, maxit);
    CFP_CUDA(cudaMemcpyAsync(st, hs, sizeof(KState), cudaMemcpyHostToDevice, c->stream));
    if (!x_zero) launch_apply<T>(c, V.x, V.v, nullptr, 0, nullptr, c->stream, nullptr);
    k_init_r<T><<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(b, x_zero ? nullptr : V.v, V.r, V.rh, V.p, c->partial, N);
    k_fin_init<<<1, 256, 0, c->stream>>>(st, c->partial, kUpdBlocks);
    c->launches += 2;
    CFP_CUDA(cudaGetLastError());
    if (use_graph) {
        CFP_TRY(build_graph<T>(c, prec, sweeps));
        CFP_CUDA(cudaGraphLaunch(c->gexec[prec], c->stream));
    } else {
        for (int it = 0; it < maxit;) {
            const int chunk = std::min(16, maxit - it);
            for (int q = 0; q < chunk; ++q) enqueue_body<T>(c, prec, sweeps, c->stream, 0, 0);
            it += chunk;
            CFP_CUDA(cudaGetLastError());
            CFP_CUDA(cudaMemcpyAsync(hs, st, sizeof(KState), cudaMemcpyDeviceToHost, c->stream));
            CFP_CUDA(cudaStreamSynchronize(c->stream));
            if (hs->flag != FLAG_RUN) break;
        }
    }
    CFP_CUDA(cudaMemcpyAsync(hs, st, sizeof(KState), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    if (use_graph) c->launches += (int64_t)hs->execs * c->body_launches;
    *flag = hs->flag == FLAG_RUN ? FLAG_MAXIT : hs->flag;
    *used = hs->iter;
    *rr = hs->rr;
    return CFP_OK;
}

double* scalar_slot(cfp_ctx* c, int q) { return reinterpret_cast<double*>(c->dtotal) + q; }

// ||b - B x||^2 with out = b - B x (FP64)
cfp_status true_residual(cfp_ctx* c, const double* b, const double* x, double* out, double* r2) {
    double* tmp = c->v64 + V_TMP2 * vstride(c);
    launch_apply<double>(c, x, tmp, nullptr, 0, nullptr, c->stream, nullptr);
    k_resid<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(b, tmp, out, c->partial, c->N);
    k_fin_store<<<1, 256, 0, c->stream>>>(c->partial, kUpdBlocks, scalar_slot(c, 6));
    c->launches += 2;
    CFP_CUDA(cudaGetLastError());
    CFP_CUDA(cudaMemcpyAsync(r2, scalar_slot(c, 6), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

cfp_status dot_host(cfp_ctx* c, const double* a, const double* b, double* out) {
    k_dot<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(a, b, c->partial, c->N);
    k_fin_store<<<1, 256, 0, c->stream>>>(c->partial, kUpdBlocks, scalar_slot(c, 7));
    c->launches += 2;
    CFP_CUDA(cudaGetLastError());
    CFP_CUDA(cudaMemcpyAsync(out, scalar_slot(c, 7), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

cfp_status status_of(int flag) {
    return flag == FLAG_NAN ? CFP_ENAN : flag == FLAG_BREAK ? CFP_EBREAKDOWN : CFP_ENOCONV;
}

}  // namespace

// y = alpha x + beta y over all nodes (FP64); x and y may be the same field,
// so neither pointer is declared __restrict__
__global__ void k_axpby(double alpha, const double* x, double beta, double* y, int64_t N) {
    GRID_STRIDE(l, N) y[l] = alpha * x[l] + beta * y[l];
}

cfp_status ensure_partial(cfp_ctx* c) {
    const int64_t need = 2 * (int64_t)std::max(apply_blocks(c), kUpdBlocks);
    if (c->partial_cap < need) {
        c->generation += 1;
        if (c->partial) cudaFree(c->partial);
        c->partial = nullptr;
        CFP_CUDA(cudaMalloc(&c->partial, sizeof(double) * need));
        c->partial_cap = need;
    }
    return CFP_OK;
}

cfp_status vec_dot(cfp_ctx* c, const double* a, const double* b, double* out) {
    CFP_TRY(ensure_partial(c));
    return dot_host(c, a, b, out);
}

cfp_status vec_axpby(cfp_ctx* c, double alpha, const double* x, double beta, double* y) {
    k_axpby<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(alpha, x, beta, y, c->N);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status ensure_work(cfp_ctx* c, bool need32) {
    const int64_t N = c->N;
    if (!c->v64) {
        CFP_CUDA(cudaMalloc(&c->v64, sizeof(double) * vstride(c) * kNV64));
        CFP_CUDA(cudaMemsetAsync(c->v64, 0, sizeof(double) * vstride(c) * kNV64, c->stream));
    }
    if (need32) setup_apply_ring(c);
    if (need32 && !c->v32) {
        CFP_CUDA(cudaMalloc(&c->v32, sizeof(float) * vstride(c) * (kNV32 + 1)));  // + the FP32 right-hand side
        CFP_CUDA(cudaMemsetAsync(c->v32, 0, sizeof(float) * vstride(c) * (kNV32 + 1), c->stream));
    }
    return ensure_partial(c);
}

namespace {
template <class T>
cfp_status time_kernel_t(cfp_ctx* c, int prec, int kernel, int reps, double* ms, double* bytes) {
    Vecs<T> V = vecs<T>(c);
    KState* st = c->kst + prec;
    KState* hs = c->hkst + prec;
    memset(hs, 0, sizeof(KState));
    hs->flag = FLAG_RUN;  // alpha = omega = 0: the update leaves x unchanged
    CFP_CUDA(cudaMemcpyAsync(st, hs, sizeof(KState), cudaMemcpyHostToDevice, c->stream));
    const int64_t nint = (int64_t)(c->n[0] - 2) * (c->n[1] - 2) * (c->n[2] - 2);
    auto launch = [&]() {
        if (kernel == CFP_KERNEL_APPLY) launch_apply<T>(c, V.ph, V.v, V.rh, 1, c->partial, c->stream, nullptr);
        else if (kernel == CFP_KERNEL_RBGS || kernel == CFP_KERNEL_MG_SWEEP) launch_mg_half_sweep<T>(c, c->stream);
        else if (kernel == CFP_KERNEL_PROLONG || kernel == CFP_KERNEL_RESTRICT)
            launch_mg_transfer<T>(c, kernel == CFP_KERNEL_PROLONG, c->stream);
        else if (kernel == CFP_KERNEL_MG_PAIR)
            launch_mg_pair<T>(c, c->stream);
        else
            k_update_xr<T><<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(V.x, V.r, V.ph, V.sh, V.s, V.t, V.rh, st,
                                                                      c->partial, c->N);
    };
    for (int q = 0; q < 2; ++q) launch();
    cudaEvent_t e0, e1;
    CFP_CUDA(cudaEventCreate(&e0));
    CFP_CUDA(cudaEventCreate(&e1));
    CFP_CUDA(cudaEventRecord(e0, c->stream));
    for (int q = 0; q < reps; ++q) launch();
    CFP_CUDA(cudaEventRecord(e1, c->stream));
    CFP_CUDA(cudaGetLastError());
    CFP_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    CFP_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / reps;
    const double w = (double)sizeof(T);
    if (bytes)
        *bytes = kernel == CFP_KERNEL_APPLY ? 3.0 * w * nint
               : kernel == CFP_KERNEL_RBGS || kernel == CFP_KERNEL_MG_SWEEP ? 1.5 * w * nint
               : kernel == CFP_KERNEL_PROLONG ? (0.5 * (1.0 + 2.0 * w) + w / 8.0) * nint
               : kernel == CFP_KERNEL_RESTRICT ? (0.5 * w + (1.0 + w) / 8.0) * nint
               : kernel == CFP_KERNEL_MG_PAIR ? 2.5 * w * nint
                                               : 8.0 * w * (double)c->N;
    return CFP_OK;
}
}  // namespace

// Autotuner of the apply: kernel (streaming with 2 or 4 rows per thread, or
// the FP32 ring with 2 rows per tile) x planes per z chunk, each candidate
// timed over `reps` launches (after two untimed) with the fused (r_hat0, v)
// dot, the fastest kept in the context.  kind, rows, planes > 0: that choice
// is set and timed only.
cfp_status tune_apply(cfp_ctx* c, int prec, int kind, int rows, int planes, int reps, double* best_ms) {
    const int q = prec == CFP_PREC_MIXED ? 1 : 0;
    struct Choice {
        int kind, ty, kc;
    };
    const bool ring = q == 1 && setup_apply_ring(c);
    std::vector<Choice> cand;
    if (kind > 0 || rows > 0 || planes > 0) {
        const bool shape = kind == CFP_APPLY_STREAM ? (rows == 2 || rows == 4) && (planes == 16 || planes == 32 || planes == 64)
                                                    : kind == CFP_APPLY_RING && rows == 2 && (planes == 32 || planes == 64);
        if (!shape)
            return fail(CFP_EINVAL, "apply: kernel 1 with rows 2 or 4 and planes 16, 32 or 64, or kernel 2 with "
                                    "rows 2 and planes 32 or 64");
        if (kind == CFP_APPLY_RING && !ring)
            return fail(CFP_EINVAL, "apply ring: FP32 only, and its launch could not be set up");
        cand.push_back({kind, rows, planes});
    } else {
        for (int r : {2, 4})
            for (int k : {16, 32, 64}) cand.push_back({CFP_APPLY_STREAM, r, k});
        if (ring)
            for (int k : {32, 64}) cand.push_back({CFP_APPLY_RING, 2, k});
    }
    double best = INFINITY;
    Choice bs{CFP_APPLY_STREAM, 0, 0};
    for (const Choice& ch : cand) {
        c->apply_kind[q] = ch.kind;
        c->apply_ty[q] = ch.ty;
        c->apply_kc[q] = ch.kc;
        double ms = 0.0;
        CFP_TRY(time_kernel(c, CFP_KERNEL_APPLY, prec, reps, &ms, nullptr));
        if (ms < best) {
            best = ms;
            bs = ch;
        }
    }
    c->apply_kind[q] = bs.kind;
    c->apply_ty[q] = bs.ty;
    c->apply_kc[q] = bs.kc;
    c->generation += 1;
    if (best_ms) *best_ms = best;
    return CFP_OK;
}

cfp_status time_kernel(cfp_ctx* c, int kernel, int prec, int reps, double* ms, double* bytes) {
    if (kernel < CFP_KERNEL_APPLY || kernel > CFP_KERNEL_MG_PAIR || reps < 1 || !ms)
        return fail(CFP_EINVAL, "bad kernel id, reps or output pointer");
    CFP_TRY(ensure_work(c, prec == CFP_PREC_MIXED));
    if (kernel != CFP_KERNEL_APPLY && kernel != CFP_KERNEL_UPDATE) CFP_TRY(ensure_mg(c, prec == CFP_PREC_MIXED ? 1 : 0));
    if ((kernel == CFP_KERNEL_PROLONG || kernel == CFP_KERNEL_RESTRICT) && c->mg.size() < 2)
        return fail(CFP_EINVAL, "the grid has a single multigrid level: no transfer to time");
    if (kernel == CFP_KERNEL_MG_PAIR) {
        if (prec != CFP_PREC_MIXED) return fail(CFP_EINVAL, "the fused pass is FP32 only");
        CFP_TRY(ensure_mg(c, 1));
        if (!c->mg[0].tma || !c->mg[0].pair)
            return fail(CFP_EINVAL, "the fine level has no fused pass (fewer than 192 nodes per row)");
    }
    CFP_TRY(prec == CFP_PREC_MIXED ? time_kernel_t<float>(c, 1, kernel, reps, ms, bytes)
                                   : time_kernel_t<double>(c, 0, kernel, reps, ms, bytes));
    return check_waits(c);
}

int mg_key(const cfp_ctx* c) {
    return c->mg_smooth * 1000 + c->mg_post + (c->mg_tma ? 1000000 : 0) + (c->mg_fuse ? 2000000 : 0);
}

cfp_status check_waits(cfp_ctx* c) {
    int w = 0;
    CFP_CUDA(cudaMemcpyAsync(&w, c->dwait, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    if (w == 0) return CFP_OK;
    CFP_CUDA(cudaMemsetAsync(c->dwait, 0, sizeof(int), c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return fail(CFP_ECUDA, "a shared-memory pipeline wait (multigrid smoother or apply ring) timed out (code " +
                               std::to_string(w) + "); the results of that call are not valid");
}

cfp_status precondition32(cfp_ctx* c, int sweeps, const double* rho, double* phi) {
    const int64_t N = c->N;
    float* rho32 = c->v32 + (int64_t)V_R * vstride(c);
    float* phi32 = c->v32 + (int64_t)V_PH * vstride(c);
    k_to32<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(rho, rho32, 1.0, N);
    k_zero<float><<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(phi32, N);
    launch_precond<float>(c, sweeps, rho32, phi32, c->stream);
    CFP_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * N, c->stream));
    k_add32<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(phi, phi32, 1.0, N);
    c->launches += 3;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status solve_impl(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u, double tol,
                      const cfp_opts* opts, cfp_info* info);

}  // namespace cfp

using namespace cfp;

// The FP64 and mixed-precision drivers.
cfp_status cfp::solve_impl(cfp_ctx* c, const double* f, const double* g, const double* gi, double* u, double tol,
                           const cfp_opts* o, cfp_info* info) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    cfp_opts opts;
    cfp_default_opts(&opts);
    if (o) opts = *o;
    if (!(tol > 0.0) || opts.maxit < 1 || opts.sweeps < 0) return fail(CFP_EINVAL, "bad tol, maxit or sweeps");
    const int64_t launches0 = c->launches;
    if (!c->classified) CFP_TRY(classify(c));
    if (opts.precond != CFP_PRECOND_RBGS && opts.precond != CFP_PRECOND_MG && opts.precond != CFP_PRECOND_ILU)
        return fail(CFP_EINVAL, "unknown preconditioner");
    c->precond_kind = opts.precond;
    c->mg_smooth = std::max(1, opts.mg_smooth);
    c->mg_post = opts.mg_post > 0 ? opts.mg_post : c->mg_smooth;
    c->mg_tma = opts.mg_tma != 0;
    c->mg_fuse = opts.mg_tma == 2;
    const bool mixed = opts.precision == CFP_PREC_MIXED;
    // the multigrid option and the red-black sweeps (on the fine level's split arrays)
    if (c->precond_kind == CFP_PRECOND_MG || (c->precond_kind == CFP_PRECOND_RBGS && opts.sweeps > 0))
        CFP_TRY(ensure_mg(c, mixed ? 1 : 0));
    if (c->precond_kind == CFP_PRECOND_ILU) CFP_TRY(ensure_ilu(c, mixed ? 1 : 0));
    CFP_TRY(ensure_work(c, mixed));
    const int64_t N = c->N;
    double* rhs = c->v64 + V_RHS * vstride(c);
    double* tmp = c->v64 + V_TMP * vstride(c);
    double* X = c->v64 + V_X * vstride(c);
    const auto t1 = clk::now();
    cfp_status st = assemble_rhs(c, f, g, gi, rhs);
    if (st) return st;
    launch_mask_unknowns(c, u, X, c->stream);
    double b2 = 0.0, x2 = 0.0;
    CFP_TRY(dot_host(c, rhs, rhs, &b2));
    CFP_TRY(dot_host(c, X, X, &x2));
    bool x_zero = x2 == 0.0;  // a zero initial guess: the first residual is rhs
    const auto t2 = clk::now();
    int total = 0, restarts = 0, refinements = 0;
    double rel = 0.0;
    cfp_status status = CFP_OK;
    if (!isfinite(b2)) {
        status = CFP_ENAN;
        rel = NAN;
    } else if (b2 == 0.0) {
        CFP_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * N, c->stream));
    } else if (!mixed) {
        for (;;) {
            int flag = 0, used = 0;
            double rr = 0.0;
            CFP_TRY(run_bicgstab<double>(c, 0, rhs, tol * tol * b2, opts.maxit - total, opts.sweeps,
                                         opts.use_graph != 0, x_zero, &flag, &used, &rr));
            x_zero = false;
            total += used;
            double r2 = 0.0;
            CFP_TRY(true_residual(c, rhs, X, tmp, &r2));
            rel = sqrt(r2 / b2);
            if (flag == FLAG_NAN || !isfinite(rel)) { status = CFP_ENAN; break; }
            if (rel <= tol) { status = CFP_OK; break; }
            if (total >= opts.maxit) { status = CFP_ENOCONV; break; }
            if (restarts >= opts.max_restarts) { status = status_of(flag); break; }
            ++restarts;
        }
    } else {
        // Iterative refinement: FP64 residual (with the FP64 irregular rows),
        // FP32 correction solve, FP64 update.
        float* b32 = c->v32 + kNV32 * vstride(c);
        float* e32 = c->v32;  // the x vector of the FP32 run
        double r2 = b2;
        const double* res = rhs;  // the current residual
        if (!x_zero) {
            CFP_TRY(true_residual(c, rhs, X, tmp, &r2));
            res = tmp;
        }
        rel = sqrt(r2 / b2);
        double prev = INFINITY;
        int stall = 0;
        while (rel > tol && isfinite(rel)) {
            if (refinements >= opts.max_refine || total >= opts.maxit) { status = CFP_ENOCONV; break; }
            const double scale = 1.0 / sqrt(r2);
            k_to32<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(res, b32, scale, N);
            k_zero<float><<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(e32, N);
            c->launches += 2;
            int flag = 0, used = 0;
            double rr = 0.0;
            // The inner solve's target reduction: inner_tol, tightened (down to
            // inner_tol / 8) to the reduction 0.3 tol / rel that would end the
            // solve in this step (a 3x margin) where inner_tol alone would
            // leave the residual just above tol and cost a whole further
            // refinement step.  Never looser than inner_tol.
            const double need = 0.3 * tol / rel;
            const double it = need < opts.inner_tol && need >= opts.inner_tol / 8 ? need : opts.inner_tol;
            CFP_TRY(run_bicgstab<float>(c, 1, b32, it * it, opts.maxit - total, opts.sweeps, opts.use_graph != 0, true,
                                        &flag, &used, &rr));
            total += used;
            ++refinements;
            if (flag == FLAG_NAN) { status = CFP_ENAN; break; }
            k_add32<<<kUpdBlocks, kUpdThreads, 0, c->stream>>>(X, e32, 1.0 / scale, N);
            c->launches += 1;
            CFP_TRY(true_residual(c, rhs, X, tmp, &r2));
            res = tmp;
            rel = sqrt(r2 / b2);
            if (!(rel < 0.9 * prev)) {
                if (++stall > opts.max_restarts) { status = status_of(flag); break; }
            }
            prev = std::min(prev, rel);
        }
        if (!isfinite(rel)) status = CFP_ENAN;
        restarts = 0;
    }
    launch_finish_solution(c, X, g, u, c->stream);
    CFP_CUDA(cudaGetLastError());
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    const auto t3 = clk::now();
    CFP_TRY(check_waits(c));
    if (info) {
        info->status = status;
        info->iterations = total;
        info->restarts = restarts;
        info->refinements = refinements;
        info->rel_residual = rel;
        info->n_irregular = c->n_irr;
        info->n_ibi = c->n_ibi;
        info->n_degenerate = c->n_deg;
        info->ms_setup = std::chrono::duration<double, std::milli>(t1 - t0).count();
        info->ms_rhs = std::chrono::duration<double, std::milli>(t2 - t1).count();
        info->ms_solve = std::chrono::duration<double, std::milli>(t3 - t2).count();
        info->launches = c->launches - launches0;
    }
    if (status != CFP_OK)
        return fail(status, status == CFP_ENAN ? "non-finite value in the solve"
                            : status == CFP_EBREAKDOWN ? "BiCGSTAB breakdown after restarts"
                                                       : "no convergence within the iteration cap");
    return CFP_OK;
}

// --------------------------------------------- the solve driven on the device
// The mixed-precision solve of solve_impl with its refinement loop moved onto
// the device: every decision the host loop takes (the FP32 right-hand side's
// scaling, the inner tolerance, the stopping and stall tests) is taken by a
// one-block kernel on the RState of the context, the refinement loop is a
// while node of a CUDA graph and the BiCGSTAB loop a while node inside its
// body.  The same kernels run in the same order on the same values, so the
// result is bitwise the one solve_impl gives; a whole solve is one graph
// launch.
namespace cfp {
namespace {

__device__ int status_of_flag(int flag) {
    return flag == FLAG_NAN ? CFP_ENAN : flag == FLAG_BREAK ? CFP_EBREAKDOWN : CFP_ENOCONV;
}

// before the loop: ||rhs||^2 and the first residual's ||r||^2 from their
// slots; the outcomes the host loop settles before its first step
__global__ void k_ref_setup(RState* R, const double* b2s, const double* r2s, double tol, double inner_tol, int maxit,
                            int max_refine, int max_restarts, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    const double b2 = *b2s;
    R->b2 = b2;
    R->tol = tol;
    R->inner_tol = inner_tol;
    R->maxit = maxit;
    R->max_refine = max_refine;
    R->max_restarts = max_restarts;
    R->refinements = R->total = R->stall = R->outer = 0;
    R->inner_execs = 0;
    R->prev = INFINITY;
    R->scale = 1.0;
    if (!isfinite(b2)) {
        R->status = CFP_ENAN;
        R->rel = NAN;
    } else if (b2 == 0.0) {
        R->status = CFP_OK;  // the solution is zero (k_zero_if)
        R->rel = 0.0;
        R->r2 = 0.0;
    } else {
        R->r2 = *r2s;
        R->rel = sqrt(R->r2 / b2);
        if (!(R->rel > tol && isfinite(R->rel))) R->status = isfinite(R->rel) ? CFP_OK : CFP_ENAN;
        else if (max_refine <= 0 || maxit <= 0) R->status = CFP_ENOCONV;
        else R->status = RSTATE_RUN;
    }
    cudaGraphSetConditional(h, R->status == RSTATE_RUN ? 1u : 0u);
}

// a refinement step's start: the scaling and the inner run's scalars
__global__ void k_ref_begin(RState* R, KState* st) {
    if (threadIdx.x != 0) return;
    R->scale = 1.0 / sqrt(R->r2);
    const double need = 0.3 * R->tol / R->rel;
    const double it = need < R->inner_tol && need >= R->inner_tol / 8 ? need : R->inner_tol;
    memset(st, 0, sizeof(KState));
    st->stop2 = it * it;
    st->maxit = max(1, R->maxit - R->total);
}

__global__ void k_to32_ref(const double* __restrict__ in, float* __restrict__ out, const RState* __restrict__ R,
                           int64_t N) {
    const double scale = R->scale;
    GRID_STRIDE(l, N) out[l] = (float)(in[l] * scale);
}

// k_fin_init, and the inner while node's condition
__global__ void k_fin_init_cond(KState* st, const double* partial, int nb, cudaGraphConditionalHandle h) {
    double rr, z;
    sum_partials(partial, nb, rr, z);
    if (threadIdx.x == 0) {
        st->rr = rr;
        st->rho = rr;
        st->iter = 0;
        st->flag = !isfinite(rr) ? FLAG_NAN : (rr <= st->stop2 ? FLAG_CONV : FLAG_RUN);
        cudaGraphSetConditional(h, st->flag == FLAG_RUN ? 1u : 0u);
    }
}

// after the inner run: its iterations, a non-finite inner result
__global__ void k_ref_mid(RState* R, const KState* st) {
    if (threadIdx.x != 0) return;
    R->total += st->iter;
    R->refinements += 1;
    R->inner_execs += st->execs;
    if (st->flag == FLAG_NAN) R->status = CFP_ENAN;
}

__global__ void k_add32_ref(double* __restrict__ x, const float* __restrict__ e, const RState* __restrict__ R,
                            int64_t N) {
    if (R->status != RSTATE_RUN) return;
    const double inv = 1.0 / R->scale;
    GRID_STRIDE(l, N) x[l] += (double)e[l] * inv;
}

// a step's end: the new residual, the stall and stopping tests, the outer
// while node's condition
__global__ void k_ref_end(RState* R, const KState* st, const double* r2s, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    R->outer += 1;
    if (R->status == RSTATE_RUN) {
        R->r2 = *r2s;
        R->rel = sqrt(R->r2 / R->b2);
        const int flag = st->flag == FLAG_RUN ? FLAG_MAXIT : st->flag;
        if (!(R->rel < 0.9 * R->prev) && ++R->stall > R->max_restarts) R->status = status_of_flag(flag);
        R->prev = fmin(R->prev, R->rel);
        if (R->status == RSTATE_RUN) {
            if (!(R->rel > R->tol && isfinite(R->rel))) R->status = isfinite(R->rel) ? CFP_OK : CFP_ENAN;
            else if (R->refinements >= R->max_refine || R->total >= R->maxit) R->status = CFP_ENOCONV;
        }
        if (!isfinite(R->rel)) R->status = CFP_ENAN;
    }
    cudaGraphSetConditional(h, R->status == RSTATE_RUN ? 1u : 0u);
}

__global__ void k_zero_if(const RState* __restrict__ R, double* __restrict__ x, int64_t N) {
    if (!(R->status == CFP_OK && R->b2 == 0.0)) return;
    GRID_STRIDE(l, N) x[l] = 0.0;
}

// ||b - B x||^2 into slot 6 and out = b - B x, enqueued on s
void enqueue_residual(cfp_ctx* c, const double* b, const double* x, double* out, cudaStream_t s) {
    double* tmp = c->v64 + V_TMP2 * vstride(c);
    launch_apply<double>(c, x, tmp, nullptr, 0, nullptr, s, nullptr);
    k_resid<<<kUpdBlocks, kUpdThreads, 0, s>>>(b, tmp, out, c->partial, c->N);
    k_fin_store<<<1, 256, 0, s>>>(c->partial, kUpdBlocks, scalar_slot(c, 6));
    c->launches += 2;
}

// a while node after the current capture dependencies of s, its body graph
// and the stream capturing into it; the node becomes s's dependency
cfp_status add_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    CFP_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, &edges, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(CFP_ECUDA, "stream is not capturing");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CFP_CUDA(cudaGraphAddNode(&node, graph, deps, edges, nd, &cp));
    CFP_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *body = cp.conditional.phGraph_out[0];
    return CFP_OK;
}

cfp_status capture_graph_of(cudaStream_t s, cudaGraph_t* g) {
    cudaStreamCaptureStatus cs;
    CFP_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return fail(CFP_ECUDA, "stream is not capturing");
    return CFP_OK;
}

// capture `fill` on a fresh stream into `body` (the body graph of a while node)
template <class F>
cfp_status capture_body(cudaGraph_t body, F&& fill) {
    cudaStream_t cs;
    CFP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    cfp_status st = e == cudaSuccess ? CFP_OK : cuda_fail(e, "cudaStreamBeginCaptureToGraph");
    if (st == CFP_OK) {
        st = fill(cs);
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(cs, &out);
        if (st == CFP_OK && e != cudaSuccess) st = cuda_fail(e, "capturing a loop body");
    }
    cudaStreamDestroy(cs);
    return st;
}

}  // namespace

// The whole mixed-precision solve of c (right-hand side, refinement loop,
// solution) enqueued on the capturing stream s.  The context must be
// classified with its work space, multigrid hierarchy and graphs' settings
// prepared for opts (prepare_device_solve).  counts: the kernels outside
// the loops, per refinement body (outside the BiCGSTAB loop), per BiCGSTAB
// body.
cfp_status capture_device_solve(cfp_ctx* c, cudaStream_t s, const double* f, const double* g, const double* gi,
                                double* u, double tol, const cfp_opts& opts, int64_t counts[3]) {
    const int64_t l0 = c->launches;
    int64_t l_body0 = 0, l_in0 = 0, l_in1 = 0, l_body1 = 0;
    const int64_t N = c->N;
    Vecs<float> V = vecs<float>(c);
    double* rhs = c->v64 + V_RHS * vstride(c);
    double* tmp = c->v64 + V_TMP * vstride(c);
    double* X = c->v64 + V_X * vstride(c);
    double* gb = c->v64 + V_TMP * vstride(c);
    double* bg = c->v64 + V_TMP2 * vstride(c);
    double* qf = c->v64 + V_T * vstride(c);
    float* b32 = c->v32 + kNV32 * vstride(c);
    float* e32 = c->v32;
    KState* st = c->kst + 1;
    use_aux(c, 0);
    // the right-hand side (cfp_assemble_rhs), the masked initial iterate, ||rhs||^2, the first residual
    launch_boundary_lift(c, g, gb, s);
    launch_apply_lift(c, gb, bg, s);
    launch_qf(c, f, qf, s);
    launch_rhs_finish(c, qf, bg, c->n_ibi ? gi : c->ibi_xyz, rhs, s);
    launch_mask_unknowns(c, u, X, s);
    k_dot<<<kUpdBlocks, kUpdThreads, 0, s>>>(rhs, rhs, c->partial, N);
    k_fin_store<<<1, 256, 0, s>>>(c->partial, kUpdBlocks, scalar_slot(c, 7));
    c->launches += 2;
    enqueue_residual(c, rhs, X, tmp, s);
    cudaGraph_t graph = nullptr;
    CFP_TRY(capture_graph_of(s, &graph));
    cudaGraphConditionalHandle h_out;
    CFP_CUDA(cudaGraphConditionalHandleCreate(&h_out, graph, 0, cudaGraphCondAssignDefault));
    k_ref_setup<<<1, 32, 0, s>>>(c->rst, scalar_slot(c, 7), scalar_slot(c, 6), tol, opts.inner_tol, opts.maxit,
                                 opts.max_refine, opts.max_restarts, h_out);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    cudaGraph_t outer = nullptr;
    CFP_TRY(add_while(s, h_out, &outer));
    // a refinement step; its streams fork the irregular rows onto aux[1] (and
    // aux[2] inside the BiCGSTAB body), streams of their own capture
    const int sweeps = opts.sweeps;
    cfp_status rs = capture_body(outer, [&](cudaStream_t cs) -> cfp_status {
        use_aux(c, 1);
        l_body0 = c->launches;
        k_ref_begin<<<1, 32, 0, cs>>>(c->rst, st);
        k_to32_ref<<<kUpdBlocks, kUpdThreads, 0, cs>>>(tmp, b32, c->rst, N);
        k_zero<float><<<kUpdBlocks, kUpdThreads, 0, cs>>>(e32, N);
        k_init_r<float><<<kUpdBlocks, kUpdThreads, 0, cs>>>(b32, nullptr, V.r, V.rh, V.p, c->partial, N);
        cudaGraphConditionalHandle h_in;
        CFP_CUDA(cudaGraphConditionalHandleCreate(&h_in, outer, 0, cudaGraphCondAssignDefault));
        k_fin_init_cond<<<1, 256, 0, cs>>>(st, c->partial, kUpdBlocks, h_in);
        c->launches += 5;
        CFP_CUDA(cudaGetLastError());
        cudaGraph_t inner = nullptr;
        CFP_TRY(add_while(cs, h_in, &inner));
        l_in0 = c->launches;
        CFP_TRY(capture_body(inner, [&](cudaStream_t cs2) -> cfp_status {
            use_aux(c, 2);
            enqueue_body<float>(c, 1, sweeps, cs2, h_in, 1);
            use_aux(c, 1);
            CFP_CUDA(cudaGetLastError());
            return CFP_OK;
        }));
        l_in1 = c->launches;
        k_ref_mid<<<1, 32, 0, cs>>>(c->rst, st);
        k_add32_ref<<<kUpdBlocks, kUpdThreads, 0, cs>>>(X, e32, c->rst, N);
        enqueue_residual(c, rhs, X, tmp, cs);
        k_ref_end<<<1, 32, 0, cs>>>(c->rst, st, scalar_slot(c, 6), h_out);
        c->launches += 3;
        l_body1 = c->launches;
        CFP_CUDA(cudaGetLastError());
        return CFP_OK;
    });
    use_aux(c, 0);
    CFP_TRY(rs);
    k_zero_if<<<kUpdBlocks, kUpdThreads, 0, s>>>(c->rst, X, N);
    c->launches += 1;
    launch_finish_solution(c, X, g, u, s);
    CFP_CUDA(cudaGetLastError());
    counts[2] = l_in1 - l_in0;
    counts[1] = (l_in0 - l_body0) + (l_body1 - l_in1);
    counts[0] = (c->launches - l0) - (l_body1 - l_body0);
    c->launches = l0;  // counted per executed body after a run
    return CFP_OK;
}

// What capture_device_solve needs in place before any capture: the
// classification, the work space, the preconditioner's data for opts and
// the settings solve_impl would take from opts.
cfp_status prepare_device_solve(cfp_ctx* c, const cfp_opts& opts) {
    if (opts.precision != CFP_PREC_MIXED) return fail(CFP_EINVAL, "the device-driven solve is mixed precision");
    if (opts.maxit < 1 || opts.sweeps < 0) return fail(CFP_EINVAL, "bad maxit or sweeps");
    if (opts.precond != CFP_PRECOND_RBGS && opts.precond != CFP_PRECOND_MG && opts.precond != CFP_PRECOND_ILU)
        return fail(CFP_EINVAL, "unknown preconditioner");
    if (!c->classified) CFP_TRY(classify(c));
    c->precond_kind = opts.precond;
    c->mg_smooth = std::max(1, opts.mg_smooth);
    c->mg_post = opts.mg_post > 0 ? opts.mg_post : c->mg_smooth;
    c->mg_tma = opts.mg_tma != 0;
    c->mg_fuse = opts.mg_tma == 2;
    if (c->precond_kind == CFP_PRECOND_MG || (c->precond_kind == CFP_PRECOND_RBGS && opts.sweeps > 0))
        CFP_TRY(ensure_mg(c, 1));
    if (c->precond_kind == CFP_PRECOND_ILU) CFP_TRY(ensure_ilu(c, 1));
    CFP_TRY(ensure_work(c, true));
    return CFP_OK;
}

}  // namespace cfp
