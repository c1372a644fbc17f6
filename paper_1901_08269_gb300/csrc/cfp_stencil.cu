// Matrix-free operators on the grid:
//  - B x (Eq. Bdec): the regular 27-point compact stencil of Eqs. A27/As_qs
//    rebuilt on the fly from the 1D metrics, sum-factorised as
//      A x = sum_r Lz[r] (sum_q Ly[q] XR + Ry[q] XL) + Rz[r] (sum_q Ly[q] XL),
//      XR = sum_p Rx[p] x,  XL = sum_p Lx[p] x,
//    with the x-pass of each z-plane staged in shared memory and the y-pass
//    results of three planes kept in registers while a CTA marches in z;
//    rows of irregular points get their modified-stencil corrections from the
//    side list in the same pass; solid rows are zero.
//  - red-black Gauss-Seidel half-sweeps on K (Eqs. A7 / A7_mod, Sec. 3.3).
//  - the source term of Eq. q with solid weights dropped, and helpers of the
//    right-hand side of Eq. Bu=q.
#include <algorithm>

#include "cfp_internal.cuh"

namespace cfp {

template <>
Grid<double> grid_view<double>(cfp_ctx* c) {
    Grid<double> g;
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d];
        double* b = c->dcoef64 + off;
        g.ax[d] = Axis<double>{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n, b + 7 * n};
        off += 8 * (int64_t)n;
    }
    g.nx = c->n[0];
    g.ny = c->n[1];
    g.nz = c->n[2];
    return g;
}

template <>
Grid<float> grid_view<float>(cfp_ctx* c) {
    Grid<float> g;
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d];
        float* b = c->dcoef32 + off;
        g.ax[d] = Axis<float>{b, b + n, b + 2 * n, b + 3 * n, b + 4 * n, b + 5 * n, b + 6 * n, b + 7 * n};
        off += 8 * (int64_t)n;
    }
    g.nx = c->n[0];
    g.ny = c->n[1];
    g.nz = c->n[2];
    return g;
}

template <>
Side<double> side_view<double>(cfp_ctx* c) {
    return Side<double>{c->slot, c->corr_ptr, c->corr_off, c->corr_val, c->krow};
}

template <>
Side<float> side_view<float>(cfp_ctx* c) {
    return Side<float>{c->slot, c->corr_ptr, c->corr_off, c->corr_val32, c->krow32};
}

namespace {

__device__ __forceinline__ void block_reduce2(double& a, double& b) {
    __shared__ double sa[32], sb[32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, wid = tid >> 5;
    for (int o = 16; o; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    const int nw = (blockDim.x * blockDim.y) >> 5;
    if (wid == 0) {
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
        for (int o = 16; o; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
    }
}

// Regular part of B x at the unknowns.  One thread owns the column i of TY
// consecutive rows j and marches the planes k0 .. k1 - 1 of its z chunk (KC
// planes); TY x KC is the tile shape the autotuner picks per grid.  The z
// coefficients of the chunk are staged in shared memory once.
// Per plane it loads the values x(i-1..i+1, j) of the rows j0-1 .. j0+TY (the
// x and y neighbours come from L1/L2; the loads of the next plane are issued
// before the current one is used), forms the x-pass XR = Rx x, XL = Lx x of
// those rows (each shared by up to three output rows), the y-pass
// P = Ly XR + Ry XL, Q = Ly XL of its rows, and keeps P, Q of three planes in
// registers for the z-pass
//   out(k) = Lz (P(k-1), P(k), P(k+1)) + Rz (Q(k-1), Q(k), Q(k+1)).
// No shared memory and no barriers.  Solid rows are zero; the rows of
// irregular points get their side-list corrections from k_apply_corr, launched
// right after.  (Gathering the corrections inside this kernel, at each plane or
// from a per-warp list after the march, measured 1.57x slower at 513^3: the
// dependent side-list loads stall the streaming march, and the CTAs near the
// bodies become the tail.)
// DOT = 0: y only; 1: partial (d0, y); 2: partials (d0, y) and (y, y).
template <class T, int DOT, int TY, int KC>
__global__ void __launch_bounds__(kAX, TY == 2 ? (sizeof(T) == 4 ? 8 : 2) : (sizeof(T) == 4 ? 4 : 2))
    k_apply(Grid<T> G, const uint8_t* __restrict__ type, const T* __restrict__ x, T* __restrict__ y,
            const T* __restrict__ d0, double* __restrict__ partial) {
    constexpr int R = TY + 2;  // rows loaded per plane
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int i = 1 + blockIdx.x * kAX + threadIdx.x;
    const int j0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * KC;
    const int k1 = min(k0 + KC, nz - 1);
    // z coefficients of the chunk's output planes k0 .. k1 - 1
    __shared__ T zc[5][KC];
    for (int q = threadIdx.x; q < 5 * KC; q += kAX) {
        const int m = q / KC, kc = min(k0 + q % KC, nz - 2);
        const T* src = m == 0 ? G.ax[2].a : m == 1 ? G.ax[2].c : m == 2 ? G.ax[2].ar : m == 3 ? G.ax[2].br : G.ax[2].cr;
        zc[m][q % KC] = src[kc];
    }
    __syncthreads();
    const bool iin = i <= nx - 2;
    const int ic = iin ? i : 1;  // clamped: every load stays inside the grid
    // node offsets fit in 32 bits: contexts hold fewer than 2^31 nodes
    const unsigned sy = (unsigned)nx, sz = (unsigned)nx * (unsigned)ny;
    const T ax = G.ax[0].a[ic], cx = G.ax[0].c[ic];
    const T arx = G.ax[0].ar[ic], brx = G.ax[0].br[ic], crx = G.ax[0].cr[ic];
    T ay[TY], cy[TY], ary[TY], bry[TY], cry[TY];
    bool jin[TY];
    unsigned lout0[TY];
#pragma unroll
    for (int t = 0; t < TY; ++t) {
        jin[t] = j0 + t <= ny - 2;
        const int jc = jin[t] ? j0 + t : j0;
        ay[t] = G.ax[1].a[jc];
        cy[t] = G.ax[1].c[jc];
        ary[t] = G.ax[1].ar[jc];
        bry[t] = G.ax[1].br[jc];
        cry[t] = G.ax[1].cr[jc];
        lout0[t] = (unsigned)k0 * sz + (unsigned)jc * sy + (unsigned)ic;
    }
    unsigned roff[R];
#pragma unroll
    for (int r = 0; r < R; ++r) roff[r] = (unsigned)min(j0 - 1 + r, ny - 1) * sy;
    const T* p = x + ((unsigned)(k0 - 1) * sz + (unsigned)ic);
    T n[3 * R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const T* q = p + roff[r];
        n[3 * r] = q[-1];
        n[3 * r + 1] = q[0];
        n[3 * r + 2] = q[1];
    }
    // type byte and dot operand of the next output node of each row
    uint8_t t_next[TY];
    T d_next[TY];
#pragma unroll
    for (int t = 0; t < TY; ++t) {
        t_next[t] = type[lout0[t]];
        d_next[t] = DOT ? d0[lout0[t]] : T(0);
    }
    T Pm[TY], P0[TY], Pp[TY], Qm[TY], Q0[TY], Qp[TY];
#pragma unroll
    for (int t = 0; t < TY; ++t) Pm[t] = P0[t] = Pp[t] = Qm[t] = Q0[t] = Qp[t] = T(0);
    DotAcc<T> dacc0, dacc1;
#pragma unroll 3
    for (int kk = k0 - 1; kk <= k1; ++kk) {
        T c[3 * R];
#pragma unroll
        for (int q = 0; q < 3 * R; ++q) c[q] = n[q];
        if (kk < k1) {  // prefetch plane kk + 1
            p += sz;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T* q = p + roff[r];
                n[3 * r] = q[-1];
                n[3 * r + 1] = q[0];
                n[3 * r + 2] = q[1];
            }
        }
        // output of this step is plane kk - 1 (from step k0 + 1 on); its type
        // bytes and dot operands were fetched one step earlier
        uint8_t t_cur[TY];
        T d_cur[TY];
#pragma unroll
        for (int t = 0; t < TY; ++t) {
            t_cur[t] = t_next[t];
            d_cur[t] = d_next[t];
        }
        if (kk >= k0 + 1 && kk < k1) {
#pragma unroll
            for (int t = 0; t < TY; ++t) {
                const unsigned ln = lout0[t] + (unsigned)(kk - k0) * sz;
                t_next[t] = type[ln];
                if (DOT) d_next[t] = d0[ln];
            }
        }
        T XR[R], XL[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            XR[r] = arx * c[3 * r] + brx * c[3 * r + 1] + crx * c[3 * r + 2];
            XL[r] = ax * c[3 * r] + c[3 * r + 1] + cx * c[3 * r + 2];
        }
#pragma unroll
        for (int t = 0; t < TY; ++t) {
            Pm[t] = P0[t];
            P0[t] = Pp[t];
            Qm[t] = Q0[t];
            Q0[t] = Qp[t];
            Pp[t] = ay[t] * XR[t] + XR[t + 1] + cy[t] * XR[t + 2] + ary[t] * XL[t] + bry[t] * XL[t + 1] +
                    cry[t] * XL[t + 2];
            Qp[t] = ay[t] * XL[t] + XL[t + 1] + cy[t] * XL[t + 2];
        }
        if (kk >= k0 + 1 && iin) {
            const int k = kk - 1, kl = k - k0;
            const T az = zc[0][kl], cz = zc[1][kl];
            const T arz = zc[2][kl], brz = zc[3][kl], crz = zc[4][kl];
#pragma unroll
            for (int t = 0; t < TY; ++t) {
                if (!jin[t]) continue;
                T v = az * Pm[t] + P0[t] + cz * Pp[t] + (arz * Qm[t] + brz * Q0[t] + crz * Qp[t]);
                const unsigned l = (unsigned)k * sz + (unsigned)(j0 + t) * sy + (unsigned)i;
                if (t_cur[t] == CFP_SOLID) v = 0;  // irregular rows: k_apply_corr adds their corrections
                y[l] = v;
                if (DOT >= 1) dacc0.add(d_cur[t], v);
                if (DOT == 2) dacc1.add(v, v);
            }
        }
    }
    if (DOT) {
        double acc0 = dacc0.total(), acc1 = dacc1.total();
        block_reduce2(acc0, acc1);
        if (threadIdx.x == 0) {
            const int64_t b = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
            partial[2 * b] = acc0;
            partial[2 * b + 1] = acc1;
        }
    }
}
constexpr int kQfRows = 2;  // rows per thread of k_qf

// B gb for a field gb that is zero away from the box (the boundary lift of
// the right-hand side): its regular rows can be nonzero only on the shell of
// interior nodes next to the box, so only those rows are evaluated, with the
// 27 weights of Eq. A27 (Rx Ly Lz + Lx Ry Lz + Lx Ly Rz); every other
// interior row is zero (the caller clears y).  Solid rows are zero; the
// irregular rows get their corrections from k_apply_corr.  Thread q walks
// the shell as two z-planes, then two y-rows of each inner plane, then the
// two x-ends of each inner row.
__global__ void k_lift_shell(Grid<double> G, const uint8_t* __restrict__ type, const double* __restrict__ gb,
                             double* __restrict__ y) {
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int64_t ax = nx - 2, ay = ny - 2, az = nz - 2;
    const int64_t bz = az - 2 > 0 ? az - 2 : 0, by = ay - 2 > 0 ? ay - 2 : 0;
    const int64_t nA = 2 * ax * ay, nB = 2 * bz * ax, nC = 2 * bz * by;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nA + nB + nC;
         q += (int64_t)gridDim.x * blockDim.x) {
        int i, j, k;
        if (q < nA) {
            const int64_t r = q % (ax * ay);
            k = q < ax * ay ? 1 : nz - 2;
            i = 1 + (int)(r % ax);
            j = 1 + (int)(r / ax);
        } else if (q < nA + nB) {
            const int64_t r = (q - nA) % (bz * ax);
            j = q - nA < bz * ax ? 1 : ny - 2;
            i = 1 + (int)(r % ax);
            k = 2 + (int)(r / ax);
        } else {
            const int64_t r = (q - nA - nB) % (bz * by);
            i = q - nA - nB < bz * by ? 1 : nx - 2;
            j = 2 + (int)(r % by);
            k = 2 + (int)(r / by);
        }
        const int64_t l = (int64_t)k * sz + (int64_t)j * sy + i;
        if (type[l] == CFP_SOLID) {
            y[l] = 0.0;
            continue;
        }
        const double Lx[3] = {G.ax[0].a[i], 1.0, G.ax[0].c[i]}, Rx[3] = {G.ax[0].ar[i], G.ax[0].br[i], G.ax[0].cr[i]};
        const double Ly[3] = {G.ax[1].a[j], 1.0, G.ax[1].c[j]}, Ry[3] = {G.ax[1].ar[j], G.ax[1].br[j], G.ax[1].cr[j]};
        const double Lz[3] = {G.ax[2].a[k], 1.0, G.ax[2].c[k]}, Rz[3] = {G.ax[2].ar[k], G.ax[2].br[k], G.ax[2].cr[k]};
        double v = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int p = 0; p < 3; ++p)
                for (int o = 0; o < 3; ++o) {
                    const double w = Rx[o] * Ly[p] * Lz[r] + Lx[o] * Ry[p] * Lz[r] + Lx[o] * Ly[p] * Rz[r];
                    v += w * gb[l + (o - 1) + (p - 1) * sy + (r - 1) * sz];
                }
        y[l] = v;
    }
}

// Side-list corrections of the irregular rows (the modified stencils of
// Secs. 2.2-2.3, the C part of Eq. Bdec), one warp per irregular point: the
// lanes gather the merged entries in parallel, lane 0 adds the sum to y and
// updates the dot partials: (d0, y) gains d0 c, (y, y) gains 2 v c + c^2
// where v is the row's regular part.  Partials are written after those of
// k_apply, one pair per CTA.
template <class T, int DOT>
__global__ void __launch_bounds__(256)
    k_apply_corr(Side<T> S, const int32_t* __restrict__ irr_lin, int64_t n_irr, const T* __restrict__ x,
                 T* __restrict__ y, const T* __restrict__ d0, double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t s = warp; s < n_irr; s += nwarps) {
        const int64_t l = irr_lin[s];
        const int e0 = S.corr_ptr[s], e1 = S.corr_ptr[s + 1];
        T c = T(0);
        for (int e = e0 + lane; e < e1; e += 32) c += S.corr_val[e] * x[l + S.corr_off[e]];
        for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) {
            const T v = y[l];
            y[l] = v + c;
            if (DOT >= 1) acc0 += (double)d0[l] * (double)c;
            if (DOT == 2) acc1 += 2.0 * (double)v * (double)c + (double)c * (double)c;
        }
    }
    if (DOT) {
        block_reduce2(acc0, acc1);
        if (threadIdx.x == 0) {
            partial[2 * blockIdx.x] = acc0;
            partial[2 * blockIdx.x + 1] = acc1;
        }
    }
}


template <class T>
__global__ void k_mask_copy(const uint8_t* __restrict__ type, const T* __restrict__ in, T* __restrict__ out,
                            int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[l];
        out[l] = (t == CFP_REGULAR || t == CFP_IRREGULAR) ? in[l] : T(0);
    }
}

// Eq. q with the weights of solid points set to zero (Q-bar), i.e. the
// tensor product Q = Lx Ly Lz applied to f with its solid entries replaced
// by zero, sum-factorised like the apply: each thread owns the columns
// (i, j0) and (i, j0 + 1) and marches kApplyKC planes in z; per plane it
// loads rows j0-1 .. j0+2 of the masked f, forms the x-pass XL = Lx f of
// each row and the y-pass Q = Ly XL of its two rows, and keeps Q of three
// planes for the z-pass out = Lz Q.  Interior non-unknowns get 0.
__global__ void __launch_bounds__(kAX) k_qf(Grid<double> G, const uint8_t* __restrict__ type,
                                            const double* __restrict__ f, double* __restrict__ out) {
    constexpr int TY = kQfRows, R = TY + 2;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int i = 1 + blockIdx.x * kAX + threadIdx.x;
    const int j0 = 1 + blockIdx.y * TY;
    const int k0 = 1 + blockIdx.z * kApplyKC;
    const int k1 = min(k0 + kApplyKC, nz - 1);
    const bool iin = i <= nx - 2;
    const int ic = iin ? i : 1;  // clamped: every load stays inside the grid
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const double ax = G.ax[0].a[ic], cx = G.ax[0].c[ic];
    double ay[TY], cy[TY];
    bool jin[TY];
#pragma unroll
    for (int t = 0; t < TY; ++t) {
        jin[t] = j0 + t <= ny - 2;
        const int jc = jin[t] ? j0 + t : j0;
        ay[t] = G.ax[1].a[jc];
        cy[t] = G.ax[1].c[jc];
    }
    int64_t roff[R];
#pragma unroll
    for (int r = 0; r < R; ++r) roff[r] = (int64_t)min(j0 - 1 + r, ny - 1) * sy + ic;
    double Qm[TY], Q0[TY], Qp[TY];
#pragma unroll
    for (int t = 0; t < TY; ++t) Qm[t] = Q0[t] = Qp[t] = 0.0;
    for (int kk = k0 - 1; kk <= k1; ++kk) {
        const int64_t pz = (int64_t)kk * sz;
        double XL[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t q = pz + roff[r];
            const double fm = type[q - 1] == CFP_SOLID ? 0.0 : f[q - 1];
            const double f0 = type[q] == CFP_SOLID ? 0.0 : f[q];
            const double fp = type[q + 1] == CFP_SOLID ? 0.0 : f[q + 1];
            XL[r] = ax * fm + f0 + cx * fp;
        }
#pragma unroll
        for (int t = 0; t < TY; ++t) {
            Qm[t] = Q0[t];
            Q0[t] = Qp[t];
            Qp[t] = ay[t] * XL[t] + XL[t + 1] + cy[t] * XL[t + 2];
        }
        if (kk >= k0 + 1 && iin) {
            const int k = kk - 1;
            const double az = G.ax[2].a[k], cz = G.ax[2].c[k];
#pragma unroll
            for (int t = 0; t < TY; ++t) {
                if (!jin[t]) continue;
                const int64_t l = (int64_t)k * sz + (int64_t)(j0 + t) * sy + i;
                const uint8_t tl = type[l];
                out[l] = (tl == CFP_REGULAR || tl == CFP_IRREGULAR) ? az * Qm[t] + Q0[t] + cz * Qp[t] : 0.0;
            }
        }
    }
}

__global__ void k_rhs_finish(const uint8_t* __restrict__ type, const int32_t* __restrict__ slot,
                             const int32_t* __restrict__ bib_ptr, const int32_t* __restrict__ bib_idx,
                             const double* __restrict__ bib_val, const double* __restrict__ qf,
                             const double* __restrict__ bg, const double* __restrict__ g_ibi,
                             double* __restrict__ rhs, int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[l];
        double v = 0.0;
        if (t == CFP_REGULAR || t == CFP_IRREGULAR) {
            v = qf[l] - bg[l];
            if (t == CFP_IRREGULAR) {
                const int s = slot[l];
                for (int e = bib_ptr[s]; e < bib_ptr[s + 1]; ++e) v -= bib_val[e] * g_ibi[bib_idx[e]];
            }
        }
        rhs[l] = v;
    }
}

__global__ void k_boundary_lift(const uint8_t* __restrict__ type, const double* __restrict__ g,
                                double* __restrict__ gb, int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x)
        gb[l] = type[l] == CFP_BOUNDARY ? g[l] : 0.0;
}

__global__ void k_finish_solution(const uint8_t* __restrict__ type, const double* __restrict__ x,
                                  const double* __restrict__ g, double* __restrict__ u, int64_t N) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[l];
        u[l] = t == CFP_BOUNDARY ? g[l] : (t == CFP_SOLID ? 0.0 : x[l]);
    }
}

// Eq. app_xxx (compact, b = 1) and Eq. 2ndorder_coef at interior nodes;
// layout per axis: a, c, ar, br, cr, ka, kb, kc (n each), zero at the ends.
__global__ void k_metrics(const double* __restrict__ x, int n, double* __restrict__ out, float* __restrict__ out32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (i > 0 && i < n - 1) {
            const double f = x[i + 1] - x[i];
            const double b = x[i] - x[i - 1];
            const double D = f * f * f + 4.0 * f * f * b + 4.0 * f * b * b + b * b * b;
            v[0] = f * (b * b + b * f - f * f) / D;
            v[1] = b * (f * f + b * f - b * b) / D;
            v[2] = 12.0 * f / D;
            v[3] = -12.0 / (f * f + 3.0 * f * b + b * b);
            v[4] = 12.0 * b / D;
            v[5] = 2.0 / (b * (f + b));
            v[6] = -2.0 / (b * f);
            v[7] = 2.0 / (f * (f + b));
        }
        for (int q = 0; q < 8; ++q) {
            out[(int64_t)q * n + i] = v[q];
            out32[(int64_t)q * n + i] = (float)v[q];
        }
    }
}

unsigned flat_grid(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace


namespace {

dim3 rows_grid(const cfp_ctx* c, int rows, int kc = kApplyKC) {
    return dim3((unsigned)((c->n[0] - 2 + kAX - 1) / kAX), (unsigned)((c->n[1] - 2 + rows - 1) / rows),
                (unsigned)((c->n[2] - 2 + kc - 1) / kc));
}

// the apply's tile shape of precision q (0 FP64, 1 FP32): rows per thread
// and planes per z chunk, as set by the autotuner; otherwise 2 x 64 in FP32
// and 4 x 64 in FP64, the fastest of the six at 385^3 and 513^3 (measured)
int apply_rows(const cfp_ctx* c, int q) { return c->apply_ty[q] ? c->apply_ty[q] : (q ? 2 : 4); }
int apply_planes(const cfp_ctx* c, int q) { return c->apply_kc[q] ? c->apply_kc[q] : 64; }

}  // namespace

void launch_metrics(cfp_ctx* c) {
    int64_t off = 0;
    for (int d = 0; d < 3; ++d) {
        const int n = c->n[d];
        k_metrics<<<(n + 255) / 256, 256, 0, c->stream>>>(c->dX[d], n, c->dcoef64 + off, c->dcoef32 + off);
        off += 8 * (int64_t)n;
    }
    c->launches += 3;
}

// CTAs of the correction kernel (8 irregular points per CTA, at most 152 x 16)
int corr_blocks(const cfp_ctx* c) {
    if (c->n_irr <= 0) return 0;
    return (int)std::min<int64_t>((c->n_irr + 7) / 8, 152 * 16);
}

// the most CTAs any apply tile shape launches, with the correction kernel's
// (dot-product partials per launch)
int apply_blocks(cfp_ctx* c) {
    int64_t m = 0;
    for (int ty : {2, 4})
        for (int kc : {16, 32, 64}) {
            const dim3 g = rows_grid(c, ty, kc);
            m = std::max<int64_t>(m, (int64_t)g.x * g.y * g.z);
        }
    return (int)m + corr_blocks(c);
}

template <class T, int DOT, int TY, int KC>
void apply_launch(cfp_ctx* c, const T* x, T* y, const T* d0, double* partial, cudaStream_t s, int* nb) {
    const dim3 grid = rows_grid(c, TY, KC);
    k_apply<T, DOT, TY, KC><<<grid, kAX, 0, s>>>(grid_view<T>(c), c->type, x, y, d0, partial);
    const int nmain = (int)(grid.x * grid.y * grid.z);
    const int ncorr = corr_blocks(c);
    if (ncorr)
        k_apply_corr<T, DOT><<<ncorr, 256, 0, s>>>(side_view<T>(c), c->irr_lin, c->n_irr, x, y, d0,
                                                   partial ? partial + 2 * (int64_t)nmain : nullptr);
    c->launches += ncorr ? 1 : 0;
    if (nb) *nb = nmain + ncorr;
}

template <class T, int TY, int KC>
void apply_dot(cfp_ctx* c, const T* x, T* y, const T* d0, int dotmode, double* partial, cudaStream_t s, int* nb) {
    if (dotmode == 0) apply_launch<T, 0, TY, KC>(c, x, y, d0, partial, s, nb);
    else if (dotmode == 1) apply_launch<T, 1, TY, KC>(c, x, y, d0, partial, s, nb);
    else apply_launch<T, 2, TY, KC>(c, x, y, d0, partial, s, nb);
}

template <class T, int TY>
void apply_depth(cfp_ctx* c, int kc, const T* x, T* y, const T* d0, int dotmode, double* partial, cudaStream_t s,
                 int* nb) {
    if (kc == 16) apply_dot<T, TY, 16>(c, x, y, d0, dotmode, partial, s, nb);
    else if (kc == 64) apply_dot<T, TY, 64>(c, x, y, d0, dotmode, partial, s, nb);
    else apply_dot<T, TY, 32>(c, x, y, d0, dotmode, partial, s, nb);
}

template <class T>
void launch_apply(cfp_ctx* c, const T* x, T* y, const T* d0, int dotmode, double* partial, cudaStream_t s,
                  int* nblocks_out) {
    const int q = sizeof(T) == 4 ? 1 : 0;
    const int ty = apply_rows(c, q), kc = apply_planes(c, q);
    if (ty == 4) apply_depth<T, 4>(c, kc, x, y, d0, dotmode, partial, s, nblocks_out);
    else apply_depth<T, 2>(c, kc, x, y, d0, dotmode, partial, s, nblocks_out);
    c->launches += 1;
}

// `sweeps` red-black sweeps from phi = 0 (sweeps = 0: masked copy).  The
// sweeps run on the fine level's red/black split arrays of the multigrid
// hierarchy (the first red half-sweep reads rho, the last black one writes
// phi at every interior node), which ensure_mg provides.
template <class T>
void launch_precond_rbgs(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s) {
    if (sweeps <= 0) {
        c->launches += 1;
        k_mask_copy<T><<<flat_grid(c->N), 256, 0, s>>>(c->type, rho, phi, c->N);
        return;
    }
    launch_rbgs_split<T>(c, sweeps, rho, phi, s);
}

template <class T>
void launch_precond(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s) {
    if (c->precond_kind == CFP_PRECOND_MG) launch_precond_mg<T>(c, rho, phi, s);
    else if (c->precond_kind == CFP_PRECOND_ILU && sweeps > 0) launch_precond_ilu<T>(c, sweeps, rho, phi, s);
    else launch_precond_rbgs<T>(c, sweeps, rho, phi, s);
}

// y = B gb for the boundary lift gb (zero away from the box), FP64
void launch_apply_lift(cfp_ctx* c, const double* gb, double* y, cudaStream_t s) {
    cudaMemsetAsync(y, 0, sizeof(double) * c->N, s);
    k_lift_shell<<<flat_grid(c->N), 256, 0, s>>>(grid_view<double>(c), c->type, gb, y);
    c->launches += 1;
    if (corr_blocks(c)) {
        k_apply_corr<double, 0><<<corr_blocks(c), 256, 0, s>>>(side_view<double>(c), c->irr_lin, c->n_irr, gb, y,
                                                               nullptr, nullptr);
        c->launches += 1;
    }
}

template void launch_apply<double>(cfp_ctx*, const double*, double*, const double*, int, double*, cudaStream_t,
                                   int*);
template void launch_apply<float>(cfp_ctx*, const float*, float*, const float*, int, double*, cudaStream_t, int*);
template void launch_precond<double>(cfp_ctx*, int, const double*, double*, cudaStream_t);
template void launch_precond<float>(cfp_ctx*, int, const float*, float*, cudaStream_t);

void launch_qf(cfp_ctx* c, const double* f, double* out, cudaStream_t s) {
    c->launches += 1;
    k_qf<<<rows_grid(c, kQfRows), kAX, 0, s>>>(grid_view<double>(c), c->type, f, out);
}

void launch_rhs_finish(cfp_ctx* c, const double* qf, const double* bg, const double* g_ibi, double* rhs,
                       cudaStream_t s) {
    c->launches += 1;
    k_rhs_finish<<<flat_grid(c->N), 256, 0, s>>>(c->type, c->slot, c->bib_ptr, c->bib_idx, c->bib_val, qf, bg, g_ibi,
                                                 rhs, c->N);
}

void launch_boundary_lift(cfp_ctx* c, const double* g, double* gb, cudaStream_t s) {
    c->launches += 1;
    k_boundary_lift<<<flat_grid(c->N), 256, 0, s>>>(c->type, g, gb, c->N);
}

void launch_finish_solution(cfp_ctx* c, const double* x, const double* g, double* u, cudaStream_t s) {
    c->launches += 1;
    k_finish_solution<<<flat_grid(c->N), 256, 0, s>>>(c->type, x, g, u, c->N);
}

void launch_mask_unknowns(cfp_ctx* c, const double* in, double* out, cudaStream_t s) {
    c->launches += 1;
    k_mask_copy<double><<<flat_grid(c->N), 256, 0, s>>>(c->type, in, out, c->N);
}

}  // namespace cfp
