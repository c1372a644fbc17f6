// ILU(0) of K in natural node order as the inner iteration of the
// preconditioner (CFP_PRECOND_ILU): the incomplete-factorisation class of
// the paper's inner solver for K phi = rho (Sec. 3.3; K of Eq. A7 with the
// Shortley-Weller rows of Eq. A7_mod).
//
// On the unknowns K = L + D + U in natural order.  For a 7-point pattern
// ILU(0) is M = (P + L) P^-1 (P + U) with the pivots
//     P_l = K_ll - sum over unknown lower neighbours m of K_lm K_ml / P_m,
// and one Richardson sweep from phi is
//     w = rho - K phi;  (P + L) y = w;  (P + U) z = P y;  phi += z.
// Node l depends on its lower neighbours l - 1, l - n_x, l - n_x n_y only,
// so every node of the hyperplane i + j + k = h depends on hyperplane
// h - 1 alone: the pivots and the forward solve run one launch per
// hyperplane in ascending order, the backward solve in descending order.
// A triangular solve is therefore (n_x + n_y + n_z - 6) dependent launches;
// this option exists for fidelity to the paper's inner solver, not speed
// (the red-black and multigrid options are the fast ones).
//
// Storage: pivots (FP64, and an FP32 copy for mixed precision) and one work
// field w per precision, zero at every non-unknown node, so the triangular
// solves read neighbours without type tests.
#include <algorithm>

#include "cfp_internal.cuh"

namespace cfp {
namespace {

constexpr int kIluThreads = 128;

__device__ __forceinline__ bool ilu_unknown(uint8_t t) { return t == CFP_REGULAR || t == CFP_IRREGULAR; }

// K's row at (i, j, k): diagonal and the weights of x-, x+, y-, y+, z-, z+
template <class T>
__device__ __forceinline__ void row_of(const Grid<T>& G, const Side<T>& S, uint8_t t, int i, int j, int k,
                                       int64_t l, T c[7]) {
    if (t == CFP_IRREGULAR) {
        const T* kr = S.krow + 7 * (int64_t)S.slot[l];
        for (int q = 0; q < 7; ++q) c[q] = kr[q];
    } else {
        c[0] = G.ax[0].kb[i] + G.ax[1].kb[j] + G.ax[2].kb[k];
        c[1] = G.ax[0].ka[i];
        c[2] = G.ax[0].kc[i];
        c[3] = G.ax[1].ka[j];
        c[4] = G.ax[1].kc[j];
        c[5] = G.ax[2].ka[k];
        c[6] = G.ax[2].kc[k];
    }
}

// the weight of row m toward its upper neighbour in direction d (0 x, 1 y,
// 2 z), i.e. K_ml for l = m + stride_d
template <class T>
__device__ __forceinline__ T upper_weight(const Grid<T>& G, const Side<T>& S, uint8_t tm, int i, int j, int k,
                                          int64_t m, int d) {
    if (tm == CFP_IRREGULAR) return S.krow[7 * (int64_t)S.slot[m] + 2 + 2 * d];
    return d == 0 ? G.ax[0].kc[i] : d == 1 ? G.ax[1].kc[j] : G.ax[2].kc[k];
}

struct Plane {  // the nodes of hyperplane i + j + k = h with k in [k0, k0 + gridDim.y)
    int h, k0;
};

__device__ __forceinline__ bool plane_node(const Plane& H, int nx, int ny, int& i, int& j, int& k) {
    j = 1 + blockIdx.x * kIluThreads + threadIdx.x;
    k = H.k0 + blockIdx.y;
    i = H.h - j - k;
    return j <= ny - 2 && i >= 1 && i <= nx - 2;
}

// pivots on one hyperplane (FP64)
__global__ void k_ilu_pivots(Grid<double> G, Side<double> S, const uint8_t* __restrict__ type, Plane H,
                             double* __restrict__ d) {
    const int nx = G.nx, ny = G.ny;
    int i, j, k;
    if (!plane_node(H, nx, ny, i, j, k)) return;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t l = (int64_t)k * sz + (int64_t)j * sy + i;
    const uint8_t t = type[l];
    if (!ilu_unknown(t)) return;
    double c[7];
    row_of(G, S, t, i, j, k, l, c);
    double v = c[0];
    const int64_t ms[3] = {l - 1, l - sy, l - sz};
    const int mi[3] = {i - 1, i, i}, mj[3] = {j, j - 1, j}, mk[3] = {k, k, k - 1};
    for (int q = 0; q < 3; ++q) {
        const int64_t m = ms[q];
        const uint8_t tm = type[m];
        if (!ilu_unknown(tm)) continue;
        v -= c[1 + 2 * q] * upper_weight(G, S, tm, mi[q], mj[q], mk[q], m, q) / d[m];
    }
    d[l] = v;
}

__global__ void k_ilu_to32(const uint8_t* __restrict__ type, const double* __restrict__ d, float* __restrict__ d32,
                           int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        d32[l] = ilu_unknown(type[l]) ? (float)d[l] : 0.0f;
}

// w = rho - K phi at the unknowns (FIRST: phi = 0, w = rho); w is never
// written elsewhere
template <class T, bool FIRST>
__global__ void k_ilu_resid(Grid<T> G, Side<T> S, const uint8_t* __restrict__ type, const T* __restrict__ rho,
                            const T* __restrict__ phi, T* __restrict__ w) {
    const int nx = G.nx, ny = G.ny;
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y, k = 1 + blockIdx.z;
    if (i > nx - 2) return;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t l = (int64_t)k * sz + (int64_t)j * sy + i;
    const uint8_t t = type[l];
    if (!ilu_unknown(t)) return;
    if (FIRST) {
        w[l] = rho[l];
        return;
    }
    T c[7];
    row_of(G, S, t, i, j, k, l, c);
    w[l] = rho[l] - (c[0] * phi[l] + (c[1] * phi[l - 1] + c[2] * phi[l + 1]) +
                     (c[3] * phi[l - sy] + c[4] * phi[l + sy]) + (c[5] * phi[l - sz] + c[6] * phi[l + sz]));
}

// forward solve on one hyperplane: w_l = (w_l - sum_lower K_lm w_m) / P_l
template <class T>
__global__ void k_ilu_forward(Grid<T> G, Side<T> S, const uint8_t* __restrict__ type, const T* __restrict__ d,
                              Plane H, T* __restrict__ w) {
    const int nx = G.nx, ny = G.ny;
    int i, j, k;
    if (!plane_node(H, nx, ny, i, j, k)) return;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t l = (int64_t)k * sz + (int64_t)j * sy + i;
    const uint8_t t = type[l];
    if (!ilu_unknown(t)) return;
    T c[7];
    row_of(G, S, t, i, j, k, l, c);
    w[l] = (w[l] - (c[1] * w[l - 1] + c[3] * w[l - sy] + c[5] * w[l - sz])) / d[l];
}

// backward solve on one hyperplane: w_l -= (sum_upper K_lm w_m) / P_l, then
// phi_l (+)= w_l
template <class T, bool FIRST>
__global__ void k_ilu_backward(Grid<T> G, Side<T> S, const uint8_t* __restrict__ type, const T* __restrict__ d,
                               Plane H, T* __restrict__ w, T* __restrict__ phi) {
    const int nx = G.nx, ny = G.ny;
    int i, j, k;
    if (!plane_node(H, nx, ny, i, j, k)) return;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t l = (int64_t)k * sz + (int64_t)j * sy + i;
    const uint8_t t = type[l];
    if (!ilu_unknown(t)) return;
    T c[7];
    row_of(G, S, t, i, j, k, l, c);
    const T z = w[l] - (c[2] * w[l + 1] + c[4] * w[l + sy] + c[6] * w[l + sz]) / d[l];
    w[l] = z;
    phi[l] = FIRST ? z : phi[l] + z;
}

int plane_count(const int n[3]) { return (n[0] - 2) + (n[1] - 2) + (n[2] - 2) - 2; }  // h = 3 .. sum - 6 + 3

// launch shape of hyperplane h: threads over j, blocks over the k range
// whose i = h - j - k can be interior for some interior j
Plane plane(const int n[3], int h, dim3& grid) {
    const int nx = n[0], ny = n[1], nz = n[2];
    const int klo = std::max(1, h - (nx - 2) - (ny - 2));
    const int khi = std::min(nz - 2, h - 2);
    grid = dim3((unsigned)((ny - 2 + kIluThreads - 1) / kIluThreads), (unsigned)std::max(0, khi - klo + 1), 1);
    return Plane{h, klo};
}

template <class T>
T* ilu_pivots_of(cfp_ctx* c);
template <>
double* ilu_pivots_of<double>(cfp_ctx* c) { return c->ilu64; }
template <>
float* ilu_pivots_of<float>(cfp_ctx* c) { return c->ilu32; }

}  // namespace

void free_ilu(cfp_ctx* c) {
    if (c->ilu64 || c->ilu32) c->generation += 1;
    pool_free(c->ilu64, c->stream);
    pool_free(c->ilu32, c->stream);
    c->ilu64 = nullptr;
    c->ilu32 = nullptr;
}

// Pivots (and the work field) of precision `prec` (0 FP64, 1 FP32); the FP64
// pivots are always built first.
cfp_status ensure_ilu(cfp_ctx* c, int prec) {
    const int64_t N = c->N;
    if (!c->ilu64) {
        CFP_CUDA(pool_malloc(&c->ilu64, sizeof(double) * 2 * N, c->stream));  // [pivots | w]
        CFP_CUDA(cudaMemsetAsync(c->ilu64, 0, sizeof(double) * 2 * N, c->stream));
        const Grid<double> G = grid_view<double>(c);
        const Side<double> S = side_view<double>(c);
        const int nh = plane_count(c->n);
        for (int q = 0; q < nh; ++q) {
            dim3 g;
            const Plane H = plane(c->n, 3 + q, g);
            if (g.y == 0) continue;
            k_ilu_pivots<<<g, kIluThreads, 0, c->stream>>>(G, S, c->type, H, c->ilu64);
        }
        CFP_CUDA(cudaGetLastError());
        c->launches += nh;
    }
    if (prec == 1 && !c->ilu32) {
        CFP_CUDA(pool_malloc(&c->ilu32, sizeof(float) * 2 * N, c->stream));
        CFP_CUDA(cudaMemsetAsync(c->ilu32, 0, sizeof(float) * 2 * N, c->stream));
        const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 152 * 16));
        k_ilu_to32<<<nb, 256, 0, c->stream>>>(c->type, c->ilu64, c->ilu32, N);
        CFP_CUDA(cudaGetLastError());
        c->launches += 1;
    }
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

// `sweeps` >= 1 ILU(0)-Richardson sweeps from phi = 0, written at the unknowns
template <class T>
void launch_precond_ilu(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s) {
    const Grid<T> G = grid_view<T>(c);
    const Side<T> S = side_view<T>(c);
    const T* d = ilu_pivots_of<T>(c);
    T* w = ilu_pivots_of<T>(c) + c->N;
    const int nh = plane_count(c->n);
    const dim3 gr((unsigned)((c->n[0] - 2 + 127) / 128), (unsigned)(c->n[1] - 2), (unsigned)(c->n[2] - 2));
    for (int sw = 0; sw < sweeps; ++sw) {
        if (sw == 0) k_ilu_resid<T, true><<<gr, 128, 0, s>>>(G, S, c->type, rho, phi, w);
        else k_ilu_resid<T, false><<<gr, 128, 0, s>>>(G, S, c->type, rho, phi, w);
        c->launches += 1;
        for (int q = 0; q < nh; ++q) {
            dim3 g;
            const Plane H = plane(c->n, 3 + q, g);
            if (g.y == 0) continue;
            k_ilu_forward<T><<<g, kIluThreads, 0, s>>>(G, S, c->type, d, H, w);
            c->launches += 1;
        }
        for (int q = nh - 1; q >= 0; --q) {
            dim3 g;
            const Plane H = plane(c->n, 3 + q, g);
            if (g.y == 0) continue;
            if (sw == 0) k_ilu_backward<T, true><<<g, kIluThreads, 0, s>>>(G, S, c->type, d, H, w, phi);
            else k_ilu_backward<T, false><<<g, kIluThreads, 0, s>>>(G, S, c->type, d, H, w, phi);
            c->launches += 1;
        }
    }
}

template void launch_precond_ilu<double>(cfp_ctx*, int, const double*, double*, cudaStream_t);
template void launch_precond_ilu<float>(cfp_ctx*, int, const float*, float*, cudaStream_t);

}  // namespace cfp
