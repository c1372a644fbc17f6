// Flexible GMRES(m) for Eq. Bu=q (Saad, SIAM J. Sci. Comput. 14, 1993), the
// outer Krylov method of the learned part: right preconditioning by a map
// M_j that may change from step to step, with x = x0 + Z y built from the
// stored directions z_j = M_j(v_j).  With the network, each step forms the
// plain direction z1 = P v and a two-grid cycle whose coarse correction is
// the network:
//     r1 = v - B z1,  y = net(r1),  alpha = (y, r1) / (y, B y),
//     z2 = z1 + alpha y,  zn = z2 + P(v - B z2),
// P the inner preconditioner of K (pre- and post-smoothing), alpha the step
// along y in the energy norm (independent of the output's scale), and keeps
// zn only if ||v - B zn|| < ||v - B z1||: the plain preconditioner stays the
// fallback and the arbiter at every step.
//
// Everything stays on the device: the Krylov basis V (m + 1 fields) and the
// directions Z (m fields), the Hessenberg matrix, the Givens rotations, the
// right-hand side g of the small least-squares problem and the step index.
// Orthogonalisation: classical Gram-Schmidt applied twice (CGS2), each pass
// one multi-dot and one multi-axpy over all basis vectors so far.  One step
// is one CUDA graph launch (captured after one eager step, so that every
// buffer exists first); the host reads one flag per step.
#include <chrono>
#include <math.h>

#include "cfp_internal.cuh"
#include "../../include/cfp_nn.h"

namespace cfp {
namespace {

constexpr int kMaxM = 64;
constexpr int kDotBlocks = 304;
constexpr int kThreads = 256;

struct GmState {
    double H[(kMaxM + 1) * kMaxM];  // column-major: H[i + (m + 1) j]
    double cs[kMaxM], sn[kMaxM];
    double g[kMaxM + 1];
    double y[kMaxM];
    double h[kMaxM + 1];   // this step's Gram-Schmidt coefficients
    double h2[kMaxM + 1];  // the second pass's
    double beta, hnext, bnorm, tol;
    double alpha;   // the network correction's step (energy norm)
    double rplain;  // ||v - B z1||^2 of this step's plain direction z1 = P v
    int j, m, conv, its;
    int nnet;       // steps whose direction came from the network
};

struct GmFlags {
    int j, conv, its, pad;
    double est;
};

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    if (threadIdx.x < 32)
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// vin = V[j]
__global__ void k_gm_take(const double* __restrict__ V, const GmState* __restrict__ st, int64_t N,
                          double* __restrict__ vin) {
    const double* src = V + (int64_t)st->j * N;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        vin[l] = src[l];
}
// Z[j] = z
__global__ void k_gm_store(const double* __restrict__ z, const GmState* __restrict__ st, int64_t N,
                           double* __restrict__ Z) {
    double* dst = Z + (int64_t)st->j * N;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        dst[l] = z[l];
}
// partial[i][block] = sum over the block's nodes of V_i w, i = blockIdx.y <= j
__global__ void k_gm_mdot(const double* __restrict__ V, const double* __restrict__ w, const GmState* __restrict__ st,
                          int64_t N, double* __restrict__ partial) {
    const int i = blockIdx.y;
    if (i > st->j) return;
    const double* v = V + (int64_t)i * N;
    double s = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        s += v[l] * w[l];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[(int64_t)i * gridDim.x + blockIdx.x] = s;
}
// coefficients of the pass (fixed-order sums): pass 0 into h, pass 1 into h2
__global__ void k_gm_mdot_fin(const double* __restrict__ partial, int nb, GmState* __restrict__ st, int pass) {
    const int i = threadIdx.x;
    if (i > st->j) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[(int64_t)i * nb + b];
    if (pass == 0) st->h[i] = s;
    else st->h2[i] = s;
}
// w -= sum_{i <= j} c_i V_i, c = h (pass 0) or h2 (pass 1)
__global__ void k_gm_maxpy(const double* __restrict__ V, double* __restrict__ w, const GmState* __restrict__ st,
                           int64_t N, int pass) {
    __shared__ double c[kMaxM + 1];
    const int j = st->j;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) c[i] = pass == 0 ? st->h[i] : st->h2[i];
    __syncthreads();
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        double s = w[l];
        for (int i = 0; i <= j; ++i) s -= c[i] * V[(int64_t)i * N + l];
        w[l] = s;
    }
}
__global__ void k_gm_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t N,
                         double* __restrict__ partial) {
    double s = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        s += a[l] * b[l];
    s = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
// H column j from the two passes and ||w||; V[j+1] = w / ||w||
__global__ void k_gm_norm_fin(const double* __restrict__ partial, int nb, GmState* __restrict__ st) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    st->hnext = sqrt(s);
}
__global__ void k_gm_next(const double* __restrict__ w, const GmState* __restrict__ st, int64_t N,
                          double* __restrict__ V) {
    const double hn = st->hnext;
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    double* dst = V + (int64_t)(st->j + 1) * N;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        dst[l] = w[l] * inv;
}
// the new Hessenberg column, the earlier rotations on it, a new rotation,
// the least-squares residual estimate |g_{j+1}|, then j += 1
__global__ void k_gm_givens(GmState* __restrict__ st, GmFlags* __restrict__ fl) {
    if (threadIdx.x != 0) return;
    const int j = st->j, ld = st->m + 1;
    double* col = st->H + (int64_t)ld * j;
    for (int i = 0; i <= j; ++i) col[i] = st->h[i] + st->h2[i];
    col[j + 1] = st->hnext;
    for (int i = 0; i < j; ++i) {
        const double t = st->cs[i] * col[i] + st->sn[i] * col[i + 1];
        col[i + 1] = -st->sn[i] * col[i] + st->cs[i] * col[i + 1];
        col[i] = t;
    }
    const double d = hypot(col[j], col[j + 1]);
    const double c = d > 0.0 ? col[j] / d : 1.0, s = d > 0.0 ? col[j + 1] / d : 0.0;
    st->cs[j] = c;
    st->sn[j] = s;
    col[j] = d;
    col[j + 1] = 0.0;
    st->g[j + 1] = -s * st->g[j];
    st->g[j] = c * st->g[j];
    const double est = fabs(st->g[j + 1]);
    st->its += 1;
    st->j = j + 1;
    st->conv = !(est > st->tol * st->bnorm) || st->hnext == 0.0 || !isfinite(est);
    fl->j = st->j;
    fl->conv = st->conv;
    fl->its = st->its;
    fl->est = est;
}
// cycle start: beta = ||r|| (partials of (r, r)), g = beta e1, V0 = r / beta, j = 0
__global__ void k_gm_start_fin(const double* __restrict__ partial, int nb, GmState* __restrict__ st,
                               GmFlags* __restrict__ fl) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    st->beta = sqrt(s);
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = st->beta;
    st->j = 0;
    st->conv = 0;
    fl->j = 0;
    fl->conv = 0;
    fl->its = st->its;
    fl->est = st->beta;
}
__global__ void k_gm_scale(const double* __restrict__ r, const GmState* __restrict__ st, int64_t N,
                           double* __restrict__ V0) {
    const double b = st->beta;
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        V0[l] = r[l] * inv;
}
// y = R^-1 g over the j columns of the cycle (R: the rotated H)
__global__ void k_gm_backsolve(GmState* __restrict__ st) {
    if (threadIdx.x != 0) return;
    const int k = st->j, ld = st->m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double s = st->g[i];
        for (int q = i + 1; q < k; ++q) s -= st->H[i + (int64_t)ld * q] * st->y[q];
        const double d = st->H[i + (int64_t)ld * i];
        st->y[i] = d != 0.0 ? s / d : 0.0;
    }
}
// x += sum_{i < j} y_i Z_i
__global__ void k_gm_update(double* __restrict__ x, const double* __restrict__ Z, const GmState* __restrict__ st,
                            int64_t N) {
    __shared__ double y[kMaxM];
    const int k = st->j;
    for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] = st->y[i];
    __syncthreads();
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        double s = x[l];
        for (int i = 0; i < k; ++i) s += y[i] * Z[(int64_t)i * N + l];
        x[l] = s;
    }
}
// out = b - out (FP64)
__global__ void k_gm_resid(const double* __restrict__ b, double* __restrict__ out, int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        out[l] = b[l] - out[l];
}
// partials of (y, r) and (y, B y) in one pass
__global__ void k_gm_dot2(const double* __restrict__ r, const double* __restrict__ y, const double* __restrict__ By,
                          int64_t N, double* __restrict__ partial) {
    double s = 0.0, t = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const double yv = y[l];
        s += yv * r[l];
        t += yv * By[l];
    }
    s = block_sum(s);
    __syncthreads();
    t = block_sum(t);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s;
        partial[gridDim.x + blockIdx.x] = t;
    }
}
// alpha = (y, r) / (y, B y): the step along the network's correction y that
// would minimise the error in the energy norm of B if B were symmetric
// positive definite (-B nearly is: its symmetric part is, away from the
// bodies); unlike the residual-minimising step it does not let the
// high-frequency part of y, which B amplifies, decide the step.  0 when
// (y, B y) is not positive.
__global__ void k_gm_alpha(const double* __restrict__ partial, int nb, GmState* __restrict__ st) {
    if (threadIdx.x != 0) return;
    double s = 0.0, t = 0.0;
    for (int b = 0; b < nb; ++b) {
        s += partial[b];
        t += partial[nb + b];
    }
    // B is negative definite-like (the Laplacian): (y, B y) < 0 and (y, r) < 0 for a good y
    st->alpha = t < 0.0 && isfinite(s / t) ? s / t : 0.0;
}
// ||r1||^2 of the plain direction into the state
__global__ void k_gm_rplain(const double* __restrict__ partial, int nb, GmState* __restrict__ st) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    st->rplain = s;
}
// keep the network's direction zn in z only if it leaves a smaller residual
// than the plain one (the partials hold ||v - B zn||^2)
__global__ void k_gm_choose(const double* __restrict__ partial, int nb, GmState* __restrict__ st,
                            int* __restrict__ take) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    const int t = s < st->rplain && isfinite(s);
    *take = t;
    st->nnet += t;
}
__global__ void k_gm_take_net(const double* __restrict__ zn, const int* __restrict__ take, int64_t N,
                              double* __restrict__ z) {
    if (!*take) return;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        z[l] = zn[l];
}
// t -= alpha v (mode 0), t += alpha v (mode 1), alpha from the state
__global__ void k_gm_step(const double* __restrict__ v, double* __restrict__ t, const GmState* __restrict__ st,
                          int64_t N, int mode) {
    const double a = mode == 0 ? -st->alpha : st->alpha;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        t[l] += a * v[l];
}
__global__ void k_gm_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        y[l] = a * x[l] + b * y[l];
}

unsigned gblocks(int64_t N) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 152 * 8)); }

struct Fgm {
    cfp_ctx* c;
    cfp_unet* net;
    int64_t step_launches;
    int m, prec, sweeps;
    int64_t N;
    double *V, *Z, *w, *vin, *y1, *t, *zt, *z2, *partial;
    int* take;
    GmState* st;
    GmFlags* fl;
    GmFlags* hfl;
};

// z = M(vin) on stream c->stream
cfp_status precondition(Fgm& F, const double* rho, double* phi) {
    cfp_ctx* c = F.c;
    if (F.prec == CFP_PREC_MIXED) return precondition32(c, F.sweeps, rho, phi);
    launch_precond<double>(c, F.sweeps, rho, phi, c->stream);
    return CFP_OK;
}

cfp_status enqueue_step(Fgm& F) {
    cfp_ctx* c = F.c;
    cudaStream_t s = c->stream;
    const int64_t N = F.N;
    k_gm_take<<<gblocks(N), kThreads, 0, s>>>(F.V, F.st, N, F.vin);
    if (F.net) {
        // the plain direction z1 = P v and, from its residual, a two-grid
        // cycle with the network as the coarse correction; the step keeps
        // whichever leaves the smaller residual
        CFP_TRY(precondition(F, F.vin, F.zt));                                    // z1 = P v
        launch_apply<double>(c, F.zt, F.t, nullptr, 0, nullptr, s, nullptr);      // B z1
        k_gm_axpby<<<gblocks(N), kThreads, 0, s>>>(1.0, F.vin, -1.0, F.t, N);    // r1 = v - B z1
        k_gm_dot<<<kDotBlocks, kThreads, 0, s>>>(F.t, F.t, N, F.partial);
        k_gm_rplain<<<1, 32, 0, s>>>(F.partial, kDotBlocks, F.st);              // ||r1||^2
        CFP_TRY(cfp_unet_apply(F.net, c, F.t, F.y1));                             // y = net(r1)
        launch_apply<double>(c, F.y1, F.w, nullptr, 0, nullptr, s, nullptr);      // B y
        k_gm_dot2<<<kDotBlocks, kThreads, 0, s>>>(F.t, F.y1, F.w, N, F.partial);
        k_gm_alpha<<<1, 32, 0, s>>>(F.partial, kDotBlocks, F.st);                // alpha = (y, r1) / (y, B y)
        k_gm_axpby<<<gblocks(N), kThreads, 0, s>>>(1.0, F.zt, 0.0, F.z2, N);     // z2 = z1
        k_gm_step<<<gblocks(N), kThreads, 0, s>>>(F.y1, F.z2, F.st, N, 1);        //      + alpha y
        k_gm_step<<<gblocks(N), kThreads, 0, s>>>(F.w, F.t, F.st, N, 0);          // r2 = r1 - alpha B y
        CFP_TRY(precondition(F, F.t, F.y1));                                      // P r2
        k_gm_axpby<<<gblocks(N), kThreads, 0, s>>>(1.0, F.y1, 1.0, F.z2, N);     // zn = z2 + P r2
        launch_apply<double>(c, F.y1, F.w, nullptr, 0, nullptr, s, nullptr);      // B P r2
        k_gm_axpby<<<gblocks(N), kThreads, 0, s>>>(1.0, F.t, -1.0, F.w, N);      // v - B zn = r2 - B P r2
        k_gm_dot<<<kDotBlocks, kThreads, 0, s>>>(F.w, F.w, N, F.partial);
        k_gm_choose<<<1, 32, 0, s>>>(F.partial, kDotBlocks, F.st, F.take);
        k_gm_take_net<<<gblocks(N), kThreads, 0, s>>>(F.z2, F.take, N, F.zt);
        c->launches += 14;
    } else {
        CFP_TRY(precondition(F, F.vin, F.zt));
    }
    k_gm_store<<<gblocks(N), kThreads, 0, s>>>(F.zt, F.st, N, F.Z);
    launch_apply<double>(c, F.zt, F.w, nullptr, 0, nullptr, s, nullptr);  // w = B z_j
    for (int pass = 0; pass < 2; ++pass) {
        k_gm_mdot<<<dim3(kDotBlocks, F.m), kThreads, 0, s>>>(F.V, F.w, F.st, N, F.partial);
        k_gm_mdot_fin<<<1, kMaxM + 1, 0, s>>>(F.partial, kDotBlocks, F.st, pass);
        k_gm_maxpy<<<gblocks(N), kThreads, 0, s>>>(F.V, F.w, F.st, N, pass);
    }
    k_gm_dot<<<kDotBlocks, kThreads, 0, s>>>(F.w, F.w, N, F.partial);
    k_gm_norm_fin<<<1, 32, 0, s>>>(F.partial, kDotBlocks, F.st);
    k_gm_next<<<gblocks(N), kThreads, 0, s>>>(F.w, F.st, N, F.V);
    k_gm_givens<<<1, 32, 0, s>>>(F.st, F.fl);
    c->launches += 13;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

// out = rhs - B x and (out, out) partials; beta from them
cfp_status residual_start(Fgm& F, const double* rhs, const double* x) {
    cfp_ctx* c = F.c;
    cudaStream_t s = c->stream;
    launch_apply<double>(c, x, F.w, nullptr, 0, nullptr, s, nullptr);
    k_gm_resid<<<gblocks(F.N), kThreads, 0, s>>>(rhs, F.w, F.N);
    k_gm_dot<<<kDotBlocks, kThreads, 0, s>>>(F.w, F.w, F.N, F.partial);
    k_gm_start_fin<<<1, 32, 0, s>>>(F.partial, kDotBlocks, F.st, F.fl);
    k_gm_scale<<<gblocks(F.N), kThreads, 0, s>>>(F.w, F.st, F.N, F.V);
    c->launches += 4;
    CFP_CUDA(cudaMemcpyAsync(F.hfl, F.fl, sizeof(GmFlags), cudaMemcpyDeviceToHost, s));
    CFP_CUDA(cudaStreamSynchronize(s));
    return CFP_OK;
}

// one step as a CUDA graph: captured on a side stream that stands in for the
// context's (and the network's) stream during the capture
cfp_status capture_step(Fgm& F, cudaGraphExec_t* exec) {
    cfp_ctx* c = F.c;
    cudaStream_t cs;
    CFP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = c->stream;
    const int64_t l0 = c->launches, n0 = F.net ? unet_launches(F.net) : 0;
    c->stream = cs;
    if (F.net) unet_use_stream(F.net, cs);
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    cfp_status st = CFP_OK;
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) {
        st = enqueue_step(F);
        e = cudaStreamEndCapture(cs, &g);
    }
    c->stream = saved;
    if (F.net) unet_use_stream(F.net, saved);
    // kernels of one step: the solve's, plus the network's when they are
    // counted on another context
    F.step_launches = (c->launches - l0) + (F.net && unet_owner(F.net) != c ? unet_launches(F.net) - n0 : 0);
    c->launches = l0;
    cudaStreamDestroy(cs);
    if (st != CFP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "capturing a flexible GMRES step");
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (flexible GMRES step)");
    return CFP_OK;
}

}  // namespace
}  // namespace cfp

using namespace cfp;

extern "C" cfp_status cfp_solve_fgmres(cfp_ctx* c, cfp_unet* net, const double* f, const double* gn,
                                       const double* gi, double* u, double tol, const cfp_opts* o, int m,
                                       int net_guess, cfp_info* info) {
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    if (!c || !f || !gn || !u) return fail(CFP_EINVAL, "cfp_solve_fgmres: NULL argument");
    if (m < 1 || m > kMaxM || !(tol > 0.0)) return fail(CFP_EINVAL, "cfp_solve_fgmres: m in 1..64 and tol > 0");
    cfp_opts opts;
    cfp_default_opts(&opts);
    if (o) opts = *o;
    const int64_t launches0 = c->launches;
    if (!c->classified) CFP_TRY(classify(c));
    if (opts.precond != CFP_PRECOND_RBGS && opts.precond != CFP_PRECOND_MG)
        return fail(CFP_EINVAL, "cfp_solve_fgmres: the inner preconditioner is CFP_PRECOND_RBGS or CFP_PRECOND_MG");
    c->precond_kind = opts.precond;
    c->mg_smooth = std::max(1, opts.mg_smooth);
    c->mg_post = opts.mg_post > 0 ? opts.mg_post : c->mg_smooth;
    c->mg_tma = opts.mg_tma != 0;
    c->mg_fuse = opts.mg_tma == 2;
    const bool mixed = opts.precision == CFP_PREC_MIXED;
    if (c->precond_kind == CFP_PRECOND_MG || opts.sweeps > 0) CFP_TRY(ensure_mg(c, mixed ? 1 : 0));
    CFP_TRY(ensure_work(c, mixed));
    const int64_t N = c->N;
    Fgm F;
    F.c = c;
    F.net = net;
    F.m = m;
    F.prec = opts.precision;
    F.sweeps = opts.sweeps;
    F.N = N;
    const size_t vec_bytes = sizeof(double) * (size_t)N;
    void* work = nullptr;
    const size_t nvec = (size_t)(2 * m + 1) + 6;
    if (cudaMalloc(&work, vec_bytes * nvec + sizeof(double) * (kMaxM + 1) * kDotBlocks + sizeof(GmState) +
                              sizeof(GmFlags) + 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(CFP_ENOMEM, "device allocation failed for the flexible GMRES vectors");
    }
    double* p = (double*)work;
    F.V = p;
    p += (int64_t)(m + 1) * N;
    F.Z = p;
    p += (int64_t)m * N;
    F.w = p;
    p += N;
    F.vin = p;
    p += N;
    F.y1 = p;
    p += N;
    F.t = p;
    p += N;
    F.zt = p;
    p += N;
    F.z2 = p;
    p += N;
    F.partial = p;
    p += (kMaxM + 1) * kDotBlocks;
    F.st = (GmState*)p;
    F.fl = (GmFlags*)(F.st + 1);
    F.take = (int*)(F.fl + 1);
    GmFlags hfl_store;
    F.hfl = &hfl_store;
    F.step_launches = 0;
    cudaGraphExec_t exec = nullptr;
    // the network enqueues on this solve's stream while it runs
    cudaStream_t net_prev = net ? unet_use_stream(net, c->stream) : nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(c->stream);
        if (exec) cudaGraphExecDestroy(exec);
        cudaFree(work);
        if (net) unet_use_stream(net, net_prev);
    };

    double* rhs = c->v64 + V_RHS * vstride(c);
    double* X = c->v64 + V_X * vstride(c);
    const auto t1 = clk::now();
    cfp_status s = cfp_assemble_rhs(c, f, gn, gi, rhs);
    if (s) {
        cleanup();
        return s;
    }
    if (net && net_guess) {
        // x0 = alpha net(rhs), the energy-norm step as in the cycle
        s = cfp_unet_apply(net, c, rhs, F.y1);
        if (s) {
            cleanup();
            return s;
        }
        launch_apply<double>(c, F.y1, F.w, nullptr, 0, nullptr, c->stream, nullptr);
        k_gm_dot2<<<kDotBlocks, kThreads, 0, c->stream>>>(rhs, F.y1, F.w, N, F.partial);
        k_gm_alpha<<<1, 32, 0, c->stream>>>(F.partial, kDotBlocks, F.st);
        CFP_CUDA(cudaMemsetAsync(X, 0, vec_bytes, c->stream));
        k_gm_step<<<gblocks(N), kThreads, 0, c->stream>>>(F.y1, X, F.st, N, 1);
        c->launches += 4;
    } else {
        launch_mask_unknowns(c, u, X, c->stream);
    }
    // ||rhs||
    GmState hst;
    memset(&hst, 0, sizeof(hst));
    hst.m = m;
    hst.tol = tol;
    k_gm_dot<<<kDotBlocks, kThreads, 0, c->stream>>>(rhs, rhs, N, F.partial);
    k_gm_norm_fin<<<1, 32, 0, c->stream>>>(F.partial, kDotBlocks, F.st);
    c->launches += 2;
    double bn = 0.0;
    cudaMemcpyAsync(&bn, &F.st->hnext, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    hst.bnorm = bn;
    CFP_CUDA(cudaMemcpyAsync(F.st, &hst, sizeof(GmState), cudaMemcpyHostToDevice, c->stream));
    const auto t2 = clk::now();

    cfp_status status = CFP_OK;
    int cycles = 0, its = 0;
    double rel = 0.0;
    if (!isfinite(bn)) status = CFP_ENAN;
    else if (bn == 0.0) {
        CFP_CUDA(cudaMemsetAsync(X, 0, vec_bytes, c->stream));
    } else {
        for (;;) {
            s = residual_start(F, rhs, X);
            if (s) break;
            rel = F.hfl->est / bn;
            if (!isfinite(rel)) { status = CFP_ENAN; break; }
            if (rel <= tol) break;
            if (its >= opts.maxit) { status = CFP_ENOCONV; break; }
            for (int j = 0; j < m; ++j) {
                if (!exec && (cycles > 0 || j > 0)) {
                    s = capture_step(F, &exec);
                    if (s) break;
                }
                if (exec) {
                    const cudaError_t e = cudaGraphLaunch(exec, c->stream);
                    if (e != cudaSuccess) { s = cuda_fail(e, "launching a flexible GMRES step"); break; }
                    c->launches += F.step_launches;
                } else {
                    s = enqueue_step(F);
                    if (s) break;
                }
                cudaMemcpyAsync(F.hfl, F.fl, sizeof(GmFlags), cudaMemcpyDeviceToHost, c->stream);
                cudaStreamSynchronize(c->stream);
                its = F.hfl->its;
                if (F.hfl->conv || its >= opts.maxit) break;
            }
            if (s) break;
            k_gm_backsolve<<<1, 32, 0, c->stream>>>(F.st);
            k_gm_update<<<gblocks(N), kThreads, 0, c->stream>>>(X, F.Z, F.st, N);
            c->launches += 2;
            ++cycles;
        }
        if (s) {
            cleanup();
            return s;
        }
    }
    int nnet = 0;
    CFP_CUDA(cudaMemcpyAsync(&nnet, &F.st->nnet, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    launch_finish_solution(c, X, gn, u, c->stream);
    cleanup();
    CFP_CUDA(cudaGetLastError());
    const auto t3 = clk::now();
    CFP_TRY(check_waits(c));
    if (net) CFP_TRY(cfp_unet_check(net));
    if (info) {
        info->status = status;
        info->iterations = its;
        info->restarts = cycles;
        info->refinements = nnet;  // steps whose direction came from the network
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
        return fail(status, status == CFP_ENAN ? "non-finite value in the flexible GMRES solve"
                                               : "no convergence within the iteration cap");
    return CFP_OK;
}
