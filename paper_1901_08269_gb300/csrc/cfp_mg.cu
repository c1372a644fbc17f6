// Geometric multigrid V-cycle as the approximate solver of the
// preconditioner system K phi = rho (Sec. 3.3: K is the 7-point second-order
// operator of Eq. A7 with the Shortley-Weller rows of Eq. A7_mod; the paper
// solves it approximately with a fixed number of inner iterations).  This is
// an alternative to the red-black Gauss-Seidel inner iterations; it is a
// fixed linear map (fixed sweep counts, zero initial guesses), so BiCGSTAB
// stays valid, and its quality does not degrade with the grid size.
//
// Levels: vertex-centred coarsening per axis, coarse node I sits on fine node
// map(I) = min(2I, n-1), n_c = (n + 2) / 2, while every axis has >= 9 nodes.
// Coarse K is the 7-point operator rediscretised on the coarse coordinates
// (Eq. 2ndorder_coef); a coarse node is solid if its fine node is solid, and
// its solid neighbours enter with value zero (Dirichlet at the node, no
// Shortley-Weller distance).  Prolongation is trilinear in the coordinates;
// restriction is its transpose normalised by the weight sums (full
// weighting).  Smoother: red-black Gauss-Seidel half-sweeps (the same kernel
// as the plain inner iterations), mg_smooth sweeps before and after, 16 on
// the coarsest level.
#include <algorithm>
#include <vector>

#include "cfp_internal.cuh"

namespace cfp {
namespace {

template <class T>
struct Interp {       // per axis: fine node i = wlo * coarse[ilo] + whi * coarse[ilo + 1]
    const int* ilo;
    const T* wlo;
    const T* whi;
};

template <class T>
struct Transfer {
    Interp<T> ax[3];
    int nf[3], nc[3];
};

// r = b - K e at the unknowns of a level, 0 at its other interior nodes.
template <class T>
__global__ void k_resid7(Grid<T> G, Side<T> S, const uint8_t* __restrict__ type, const T* __restrict__ b,
                         const T* __restrict__ e, T* __restrict__ r) {
    const int nx = G.nx, ny = G.ny;
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y, k = 1 + blockIdx.z;
    if (i > nx - 2) return;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t l = (int64_t)k * sz + (int64_t)j * sy + i;
    // all loads in bounds for an interior node: issue them before the type test
    const uint8_t t = type[l];
    const T bl = b[l], e0 = e[l], exm = e[l - 1], exp_ = e[l + 1], eym = e[l - sy], eyp = e[l + sy];
    const T ezm = e[l - sz], ezp = e[l + sz];
    T dg = G.ax[0].kb[i] + G.ax[1].kb[j] + G.ax[2].kb[k];
    T cxm = G.ax[0].ka[i], cxp = G.ax[0].kc[i], cym = G.ax[1].ka[j], cyp = G.ax[1].kc[j];
    T czm = G.ax[2].ka[k], czp = G.ax[2].kc[k];
    if (t != CFP_REGULAR && t != CFP_IRREGULAR) {
        r[l] = T(0);
        return;
    }
    if (t == CFP_IRREGULAR) {
        const T* kr = S.krow + 7 * (int64_t)S.slot[l];
        dg = kr[0];
        cxm = kr[1];
        cxp = kr[2];
        cym = kr[3];
        cyp = kr[4];
        czm = kr[5];
        czp = kr[6];
    }
    const T ke = dg * e0 + (cxm * exm + cxp * exp_) + (cym * eym + cyp * eyp) + (czm * ezm + czp * ezp);
    r[l] = bl - ke;
}

__device__ __forceinline__ int fine_of(int I, int n) { return min(2 * I, n - 1); }

template <class T>
__device__ __forceinline__ T weight_to(const Interp<T>& A, int i, int I) {
    const int lo = A.ilo[i];
    return (lo == I ? A.wlo[i] : T(0)) + (lo + 1 == I ? A.whi[i] : T(0));
}

// b_c = (P^T r_f) / (P^T 1) at the coarse unknowns
template <class T>
__global__ void k_restrict(Transfer<T> X, const uint8_t* __restrict__ ctype, const T* __restrict__ rf,
                           T* __restrict__ bc) {
    const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int J = 1 + blockIdx.y, K = 1 + blockIdx.z;
    const int ncx = X.nc[0], ncy = X.nc[1];
    if (I > ncx - 2) return;
    const int64_t lc = (int64_t)K * ncx * ncy + (int64_t)J * ncx + I;
    const uint8_t t = ctype[lc];
    if (t != CFP_REGULAR && t != CFP_IRREGULAR) return;
    const int nfx = X.nf[0], nfy = X.nf[1], nfz = X.nf[2];
    const int fi = fine_of(I, nfx), fj = fine_of(J, nfy), fk = fine_of(K, X.nf[2]);
    T wx[3], wy[3], wz[3];
    for (int o = 0; o < 3; ++o) {
        const int i = fi - 1 + o, j = fj - 1 + o, k = fk - 1 + o;
        wx[o] = (i >= 0 && i < nfx) ? weight_to(X.ax[0], i, I) : T(0);
        wy[o] = (j >= 0 && j < nfy) ? weight_to(X.ax[1], j, J) : T(0);
        wz[o] = (k >= 0 && k < nfz) ? weight_to(X.ax[2], k, K) : T(0);
    }
    T s = 0, w = 0;
    const int64_t fsy = nfx, fsz = (int64_t)nfx * nfy;
    for (int c = 0; c < 3; ++c) {
        if (wz[c] == T(0)) continue;
        for (int b = 0; b < 3; ++b) {
            if (wy[b] == T(0)) continue;
            const T wyz = wy[b] * wz[c];
            const int64_t base = (int64_t)(fk - 1 + c) * fsz + (int64_t)(fj - 1 + b) * fsy + (fi - 1);
            for (int a = 0; a < 3; ++a) {
                if (wx[a] == T(0)) continue;
                const T ww = wx[a] * wyz;
                s += ww * rf[base + a];
                w += ww;
            }
        }
    }
    bc[lc] = s / w;
}

// e_f += P e_c at the fine unknowns (ilo + 1 is a valid coarse index for
// every fine node, with weight zero on coincident nodes)
template <class T>
__global__ void k_prolong_add(Transfer<T> X, const uint8_t* __restrict__ ftype, const T* __restrict__ ec,
                              T* __restrict__ ef) {
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y, k = 1 + blockIdx.z;
    const int nfx = X.nf[0], nfy = X.nf[1];
    if (i > nfx - 2) return;
    const int64_t l = (int64_t)k * nfx * nfy + (int64_t)j * nfx + i;
    const int ncx = X.nc[0], ncy = X.nc[1];
    const int I = X.ax[0].ilo[i], J = X.ax[1].ilo[j], K = X.ax[2].ilo[k];
    const T ax0 = X.ax[0].wlo[i], ax1 = X.ax[0].whi[i];
    const T ay0 = X.ax[1].wlo[j], ay1 = X.ax[1].whi[j];
    const T az0 = X.ax[2].wlo[k], az1 = X.ax[2].whi[k];
    const int64_t csy = ncx, csz = (int64_t)ncx * ncy;
    const int64_t c0 = (int64_t)K * csz + (int64_t)J * csy + I;
    const uint8_t t = ftype[l];
    const T f0 = ef[l];
    const T e000 = ec[c0], e001 = ec[c0 + 1], e010 = ec[c0 + csy], e011 = ec[c0 + csy + 1];
    const T e100 = ec[c0 + csz], e101 = ec[c0 + csz + 1], e110 = ec[c0 + csz + csy], e111 = ec[c0 + csz + csy + 1];
    if (t != CFP_REGULAR && t != CFP_IRREGULAR) return;
    const T v = az0 * (ay0 * (ax0 * e000 + ax1 * e001) + ay1 * (ax0 * e010 + ax1 * e011)) +
                az1 * (ay0 * (ax0 * e100 + ax1 * e101) + ay1 * (ax0 * e110 + ax1 * e111));
    ef[l] = f0 + v;
}

// coarse type by injection: box stays box, solid stays solid, fluid -> regular
__global__ void k_inject_type(const uint8_t* __restrict__ ft, int nfx, int nfy, int nfz, uint8_t* __restrict__ ct,
                              int ncx, int ncy, int ncz) {
    const int64_t nc = (int64_t)ncx * ncy * ncz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nc; q += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(q % ncx), J = (int)((q / ncx) % ncy), K = (int)(q / ((int64_t)ncx * ncy));
        const uint8_t t = ft[(int64_t)fine_of(K, nfz) * nfx * nfy + (int64_t)fine_of(J, nfy) * nfx + fine_of(I, nfx)];
        ct[q] = t == CFP_IRREGULAR ? (uint8_t)CFP_REGULAR : t;
    }
}

dim3 level_grid(int nx, int ny, int nz, int threads) {
    return dim3((unsigned)((nx - 2 + threads - 1) / threads), (unsigned)(ny - 2), (unsigned)(nz - 2));
}

template <class T>
Grid<T> level_grid_view(MgLevel& L);
template <>
Grid<double> level_grid_view<double>(MgLevel& L) {
    Grid<double> g;
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
        const int n = L.n[d];
        double* b = L.coef64 + off;
        g.ax[d] = Axis<double>{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n, b + 7 * n};
        off += 8 * (int64_t)n;
    }
    g.nx = L.n[0];
    g.ny = L.n[1];
    g.nz = L.n[2];
    return g;
}
template <>
Grid<float> level_grid_view<float>(MgLevel& L) {
    Grid<float> g;
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
        const int n = L.n[d];
        float* b = L.coef32 + off;
        g.ax[d] = Axis<float>{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n, b + 7 * n};
        off += 8 * (int64_t)n;
    }
    g.nx = L.n[0];
    g.ny = L.n[1];
    g.nz = L.n[2];
    return g;
}

template <class T>
T* lvec(MgLevel& L, int which);
template <>
double* lvec<double>(MgLevel& L, int which) { return L.v64 + which * L.N; }
template <>
float* lvec<float>(MgLevel& L, int which) { return L.v32 + which * L.N; }

template <class T>
Transfer<T> transfer(MgLevel& F, MgLevel& Cc);
template <>
Transfer<double> transfer<double>(MgLevel& F, MgLevel& Cc) {
    Transfer<double> X;
    for (int d = 0; d < 3; ++d) {
        X.ax[d] = Interp<double>{F.ilo[d], F.w64 + 2 * F.off[d], F.w64 + 2 * F.off[d] + F.n[d]};
        X.nf[d] = F.n[d];
        X.nc[d] = Cc.n[d];
    }
    return X;
}
template <>
Transfer<float> transfer<float>(MgLevel& F, MgLevel& Cc) {
    Transfer<float> X;
    for (int d = 0; d < 3; ++d) {
        X.ax[d] = Interp<float>{F.ilo[d], F.w32 + 2 * F.off[d], F.w32 + 2 * F.off[d] + F.n[d]};
        X.nf[d] = F.n[d];
        X.nc[d] = Cc.n[d];
    }
    return X;
}

template <class T>
void smooth(const Grid<T>& G, const Side<T>& S, const uint8_t* type, const T* b, T* e, int sweeps, bool from_zero,
            cudaStream_t s, int64_t& launches) {
    for (int q = 0; q < sweeps; ++q) {
        launch_half_sweep<T>(G, S, type, b, e, 0, from_zero && q == 0, s);
        launch_half_sweep<T>(G, S, type, b, e, 1, false, s);
    }
    launches += 2 * sweeps;
}

}  // namespace

void free_mg(cfp_ctx* c) {
    for (MgLevel& L : c->mg) {
        void* ptrs[] = {L.coef64, L.coef32, L.type, L.v64, L.v32, L.ilo[0], L.ilo[1], L.ilo[2], L.w64, L.w32};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    c->mg.clear();
}

// Build the level hierarchy below the fine grid (after classification).
cfp_status ensure_mg(cfp_ctx* c) {
    if (!c->mg.empty()) return CFP_OK;
    std::vector<MgLevel> levels(1);
    MgLevel& F0 = levels[0];
    for (int d = 0; d < 3; ++d) {
        F0.n[d] = c->n[d];
        F0.X[d] = c->X[d];
    }
    F0.N = c->N;
    while (std::min({levels.back().n[0], levels.back().n[1], levels.back().n[2]}) >= 9) {
        MgLevel Cn;
        const MgLevel& Fp = levels.back();
        for (int d = 0; d < 3; ++d) {
            const int n = Fp.n[d], nc = (n + 2) / 2;
            Cn.n[d] = nc;
            Cn.X[d].resize(nc);
            for (int I = 0; I < nc; ++I) Cn.X[d][I] = Fp.X[d][std::min(2 * I, n - 1)];
        }
        Cn.N = (int64_t)Cn.n[0] * Cn.n[1] * Cn.n[2];
        levels.push_back(Cn);
    }
    const int nl = (int)levels.size();
    for (int l = 0; l < nl; ++l) {
        MgLevel& L = levels[l];
        // interpolation tables from level l + 1 (per fine index of level l)
        if (l + 1 < nl) {
            const MgLevel& Cn = levels[l + 1];
            std::vector<double> w;
            int64_t tot = 0;
            for (int d = 0; d < 3; ++d) {
                L.off[d] = tot;
                tot += L.n[d];
            }
            std::vector<double> wv(2 * tot);
            for (int d = 0; d < 3; ++d) {
                const int n = L.n[d], nc = Cn.n[d];
                std::vector<int> lo(n);
                for (int i = 0; i < n; ++i) {
                    int I = std::min(i / 2, nc - 2);
                    while (I > 0 && std::min(2 * I, n - 1) > i) --I;
                    while (I + 1 < nc - 1 && std::min(2 * (I + 1), n - 1) <= i) ++I;
                    const int fa = std::min(2 * I, n - 1), fb = std::min(2 * (I + 1), n - 1);
                    double wl, wh;
                    if (i == fa) { wl = 1.0; wh = 0.0; }
                    else if (i == fb) { wl = 0.0; wh = 1.0; }
                    else {
                        const double xa = L.X[d][fa], xb = L.X[d][fb], xi = L.X[d][i];
                        wl = (xb - xi) / (xb - xa);
                        wh = (xi - xa) / (xb - xa);
                    }
                    lo[i] = I;
                    wv[2 * L.off[d] + i] = wl;
                    wv[2 * L.off[d] + n + i] = wh;
                }
                CFP_CUDA(cudaMalloc(&L.ilo[d], sizeof(int) * n));
                CFP_CUDA(cudaMemcpy(L.ilo[d], lo.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
            }
            // layout per axis d: [wlo (n_d) | whi (n_d)] starting at 2 * off[d]
            std::vector<float> wf(wv.begin(), wv.end());
            CFP_CUDA(cudaMalloc(&L.w64, sizeof(double) * wv.size()));
            CFP_CUDA(cudaMalloc(&L.w32, sizeof(float) * wf.size()));
            CFP_CUDA(cudaMemcpy(L.w64, wv.data(), sizeof(double) * wv.size(), cudaMemcpyHostToDevice));
            CFP_CUDA(cudaMemcpy(L.w32, wf.data(), sizeof(float) * wf.size(), cudaMemcpyHostToDevice));
        }
        if (l == 0) continue;  // the fine level uses the context's own arrays
        // metrics of the coarse coordinates
        int64_t nco = 0;
        for (int d = 0; d < 3; ++d) nco += 8 * (int64_t)L.n[d];
        std::vector<double> cf(nco, 0.0);
        int64_t off = 0;
        for (int d = 0; d < 3; ++d) {
            const int n = L.n[d];
            for (int i = 1; i < n - 1; ++i) {
                const double f = L.X[d][i + 1] - L.X[d][i], b = L.X[d][i] - L.X[d][i - 1];
                cf[off + 5 * n + i] = 2.0 / (b * (f + b));
                cf[off + 6 * n + i] = -2.0 / (b * f);
                cf[off + 7 * n + i] = 2.0 / (f * (f + b));
            }
            off += 8 * (int64_t)n;
        }
        std::vector<float> cf32(cf.begin(), cf.end());
        CFP_CUDA(cudaMalloc(&L.coef64, sizeof(double) * nco));
        CFP_CUDA(cudaMalloc(&L.coef32, sizeof(float) * nco));
        CFP_CUDA(cudaMemcpy(L.coef64, cf.data(), sizeof(double) * nco, cudaMemcpyHostToDevice));
        CFP_CUDA(cudaMemcpy(L.coef32, cf32.data(), sizeof(float) * nco, cudaMemcpyHostToDevice));
        CFP_CUDA(cudaMalloc(&L.type, (size_t)L.N));
        const MgLevel& Fp = levels[l - 1];
        const uint8_t* ft = l == 1 ? c->type : Fp.type;
        k_inject_type<<<(unsigned)std::min<int64_t>((L.N + 255) / 256, 152 * 16), 256, 0, c->stream>>>(
            ft, Fp.n[0], Fp.n[1], Fp.n[2], L.type, L.n[0], L.n[1], L.n[2]);
        CFP_CUDA(cudaGetLastError());
        // e, b, r per level in both precisions, zero-filled
        CFP_CUDA(cudaMalloc(&L.v64, sizeof(double) * 3 * L.N));
        CFP_CUDA(cudaMalloc(&L.v32, sizeof(float) * 3 * L.N));
        CFP_CUDA(cudaMemsetAsync(L.v64, 0, sizeof(double) * 3 * L.N, c->stream));
        CFP_CUDA(cudaMemsetAsync(L.v32, 0, sizeof(float) * 3 * L.N, c->stream));
    }
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    c->mg = levels;
    return CFP_OK;
}

// phi = V(rho): one V-cycle from zero on the level hierarchy.
template <class T>
void launch_precond_mg(cfp_ctx* c, const T* rho, T* phi, cudaStream_t s) {
    const int nl = (int)c->mg.size();
    const int nu = std::max(1, c->mg_smooth);
    const Side<T> S0 = side_view<T>(c);
    const Side<T> Sc = Side<T>{nullptr, nullptr, nullptr, nullptr, nullptr};
    T* r0 = precond_tmp<T>(c);
    // downward leg
    for (int l = 0; l < nl - 1; ++l) {
        MgLevel& L = c->mg[l];
        MgLevel& Cn = c->mg[l + 1];
        const Grid<T> G = l == 0 ? grid_view<T>(c) : level_grid_view<T>(L);
        const Side<T>& S = l == 0 ? S0 : Sc;
        const uint8_t* ty = l == 0 ? c->type : L.type;
        const T* b = l == 0 ? rho : lvec<T>(L, 1);
        T* e = l == 0 ? phi : lvec<T>(L, 0);
        T* r = l == 0 ? r0 : lvec<T>(L, 2);
        smooth<T>(G, S, ty, b, e, nu, true, s, c->launches);
        k_resid7<T><<<level_grid(L.n[0], L.n[1], L.n[2], 128), 128, 0, s>>>(G, S, ty, b, e, r);
        k_restrict<T><<<level_grid(Cn.n[0], Cn.n[1], Cn.n[2], 128), 128, 0, s>>>(transfer<T>(L, Cn), Cn.type, r,
                                                                                 lvec<T>(Cn, 1));
        c->launches += 2;
    }
    {  // coarsest level
        MgLevel& L = c->mg[nl - 1];
        const Grid<T> G = nl == 1 ? grid_view<T>(c) : level_grid_view<T>(L);
        smooth<T>(G, nl == 1 ? S0 : Sc, nl == 1 ? c->type : L.type, nl == 1 ? rho : lvec<T>(L, 1),
                  nl == 1 ? phi : lvec<T>(L, 0), 16, true, s, c->launches);
    }
    // upward leg
    for (int l = nl - 2; l >= 0; --l) {
        MgLevel& L = c->mg[l];
        MgLevel& Cn = c->mg[l + 1];
        const Grid<T> G = l == 0 ? grid_view<T>(c) : level_grid_view<T>(L);
        const Side<T>& S = l == 0 ? S0 : Sc;
        const uint8_t* ty = l == 0 ? c->type : L.type;
        const T* b = l == 0 ? rho : lvec<T>(L, 1);
        T* e = l == 0 ? phi : lvec<T>(L, 0);
        k_prolong_add<T><<<level_grid(L.n[0], L.n[1], L.n[2], 128), 128, 0, s>>>(transfer<T>(L, Cn), ty,
                                                                                 lvec<T>(Cn, 0), e);
        c->launches += 1;
        smooth<T>(G, S, ty, b, e, nu, false, s, c->launches);
    }
}

template void launch_precond_mg<double>(cfp_ctx*, const double*, double*, cudaStream_t);
template void launch_precond_mg<float>(cfp_ctx*, const float*, float*, cudaStream_t);

}  // namespace cfp
