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
#include "cfp_tc.cuh"

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

// Fused multiply-add in either precision: the apply's sums are written as
// explicit chains so that every tile shape (and the packed FP32 kernel)
// rounds each row the same way.
__device__ __forceinline__ float fmat(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mult(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mult(double a, double b) { return __dmul_rn(a, b); }

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
// irregular points are left to k_apply_irr, which runs beside this kernel on
// a second stream.  (Gathering the corrections inside this kernel, at each plane or
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
            XR[r] = fmat(crx, c[3 * r + 2], fmat(brx, c[3 * r + 1], mult(arx, c[3 * r])));
            XL[r] = fmat(cx, c[3 * r + 2], fmat(ax, c[3 * r], c[3 * r + 1]));
        }
#pragma unroll
        for (int t = 0; t < TY; ++t) {
            Pm[t] = P0[t];
            P0[t] = Pp[t];
            Qm[t] = Q0[t];
            Q0[t] = Qp[t];
            Pp[t] = fmat(cry[t], XL[t + 2],
                         fmat(bry[t], XL[t + 1],
                              fmat(ary[t], XL[t], fmat(cy[t], XR[t + 2], fmat(ay[t], XR[t], XR[t + 1])))));
            Qp[t] = fmat(cy[t], XL[t + 2], fmat(ay[t], XL[t], XL[t + 1]));
        }
        if (kk >= k0 + 1 && iin) {
            const int k = kk - 1, kl = k - k0;
            const T az = zc[0][kl], cz = zc[1][kl];
            const T arz = zc[2][kl], brz = zc[3][kl], crz = zc[4][kl];
#pragma unroll
            for (int t = 0; t < TY; ++t) {
                if (!jin[t]) continue;
                T v = fmat(cz, Pp[t], fmat(az, Pm[t], P0[t])) + fmat(crz, Qp[t], fmat(brz, Q0[t], mult(arz, Qm[t])));
                const unsigned l = (unsigned)k * sz + (unsigned)(j0 + t) * sy + (unsigned)i;
                // solid rows are zero; irregular rows belong to k_apply_irr
                if (t_cur[t] != CFP_REGULAR) v = 0;
                if (t_cur[t] != CFP_IRREGULAR) y[l] = v;
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
// The FP32 apply fed by a ring of bulk copies (the TMA engine) through shared
// memory.  The streaming kernel above keeps one plane of loads in flight per
// thread, too few bytes per SM to cover the HBM latency.  Here a producer
// warp copies each plane of a tile several planes ahead of the consumers
// into one of kRingStages stages: the x rows j0-1 .. j0+2 with their halo
// columns, and for the output planes the dot operand and the type bytes of
// the rows j0, j0+1.  A tile is 512 columns x 2 rows x KC planes.  When it
// spans the whole row width (n_x <= 514), its rows are contiguous in the
// natural layout and each array's rows of a plane are one bulk copy; wider
// grids copy row by row.  Rows start at any 4-byte offset (n_x is odd in the
// benchmark grids), so each copy starts at the 16-byte boundary at or below
// its first element and the consumers add that offset.  A copy never passes
// the array's last 16-byte boundary; the elements after it (at the end of
// the array only) are stored into the stage by the producer lane itself.
// Tiles go to a persistent grid, rows fastest within a z chunk; 256 consumer
// threads own columns i0 + lx and i0 + 256 + lx of both rows and march the
// planes with the same sum-factorised arithmetic and fused multiply-add
// chains as k_apply<float>, so both give the same bits.  Solid rows are zero;
// irregular rows are left to k_apply_irr.
// A wait that runs out (1 s) records a code in *wait_err (31: producer, stage
// free; 32: producer, final drain; 33: consumer, stage filled).  A producer
// whose wait ran out issues no further copy and waits (bounded) for the
// copies it issued; a consumer whose wait ran out stops waiting (every index
// stays in bounds whatever a stage holds), so the launch still ends.
constexpr int kRingTX = 512;                // columns per tile
constexpr int kRingRows = 2;                // rows per tile
constexpr int kRingCons = 256;              // consumer threads: two columns each
constexpr int kRingThreads = kRingCons + 32;
constexpr int kRingStages = 6;
constexpr int kRingSpanNx = kRingTX + 2;    // widest grid copied as whole-plane spans
constexpr int kRingXRow = 520;              // floats per x row (row-by-row copies): 514 + alignment
constexpr int kRingDRow = 516;              // floats per dot-operand row: 512 + alignment
constexpr int kRingTRow = 528;              // bytes per type row: 512 + alignment
constexpr int kRingXBytes = 8320;           // >= 4 x-rows either way (span: 4 n_x + 6 floats)
constexpr int kRingDBytes = 4160;           // >= 2 dot rows either way (span: 2 n_x + 6 floats)
constexpr int kRingTBytes = 1088;           // >= 2 type rows either way (span: 2 n_x + 30 bytes)
constexpr int kRingDOff = kRingXBytes, kRingTOff = kRingDOff + kRingDBytes;
constexpr int kRingStage = kRingTOff + kRingTBytes;
constexpr int kRingSmem = kRingStages * kRingStage + 2 * kRingStages * 8;  // + barriers
static_assert(kRingXBytes >= (kRingRows + 2) * kRingXRow * 4 && kRingXBytes >= (4 * kRingSpanNx + 8) * 4 &&
                  kRingDBytes >= kRingRows * kRingDRow * 4 && kRingDBytes >= (2 * kRingSpanNx + 8) * 4 &&
                  kRingTBytes >= kRingRows * kRingTRow && kRingTBytes >= 2 * kRingSpanNx + 32,
              "stage regions hold either copy pattern");
static_assert(kRingStage % 128 == 0 && kRingDOff % 16 == 0 && kRingTOff % 16 == 0 && kRingXRow % 4 == 0 &&
                  kRingDRow % 4 == 0 && kRingTRow % 16 == 0,
              "bulk copies want 16-byte destinations");

// Elements e .. e + want - 1 of an array of n elements of esize bytes into
// the stage at dst, which receives the array from e0 = the 16-byte boundary
// at or below e onward.  The bulk copy stops at the array's last 16-byte
// boundary (and at the end of what is wanted, rounded up); the producer lane
// stores the remaining elements itself.  Returns the bytes the bulk copy
// delivers (0: none to issue) and its source in *src_out.
__device__ __forceinline__ unsigned ring_copy(unsigned char* dst, const unsigned char* base, int64_t e, int want,
                                              int esize, int64_t n, const unsigned char** src_out) {
    const int per16 = 16 / esize;
    const int64_t e0 = e & ~(int64_t)(per16 - 1);
    const int64_t end = e + want;                   // one past the last wanted element
    const int64_t nal = n & ~(int64_t)(per16 - 1);  // the array's last 16-byte boundary, in elements
    int64_t stop = (end + per16 - 1) & ~(int64_t)(per16 - 1);
    if (stop > nal) stop = nal;
    bool tail = false;
    for (int64_t q = max(stop, e0); q < min(end, n); ++q) {  // the tail after the last boundary
        for (int b = 0; b < esize; ++b) dst[(q - e0) * esize + b] = base[q * esize + b];
        tail = true;
    }
    // order these generic stores before later bulk (async-proxy) writes into
    // the stage; only the rare copies with a tail pay for the fence
    if (tail) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    *src_out = base + e0 * esize;
    return stop > e0 ? (unsigned)((stop - e0) * esize) : 0u;
}

// Packed FP32 pairs: the halves are the two columns a ring consumer thread
// owns, and one fma.rn.f32x2 instruction does the (IEEE, round-to-nearest)
// arithmetic of both, with the results of two scalar fmaf calls.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// DotAcc<float> on both halves at once: a running sum and its lost
// low-order part per column, the latter kept negated (cn = -c), so that no
// step needs a negation: v = x y - c = fma(x, y, cn); t = s + v; the new
// c = (t - s) - v, that is cn = (s - t) + v, with s - t formed exactly as
// fma(t, -1, s).  Round-to-nearest is symmetric, so every value is the
// negation of the plain form's, bit for bit.
struct DotAcc2 {
    float2 s = {0.f, 0.f}, cn = {0.f, 0.f};
    __device__ __forceinline__ void add(float2 x, float2 y) {
        const float2 v = fma2(x, y, cn);
        const float2 t = add2(s, v);
        cn = add2(fma2(t, make_float2(-1.f, -1.f), s), v);
        s = t;
    }
    __device__ __forceinline__ double total() const {
        return ((double)s.x + (double)cn.x) + ((double)s.y + (double)cn.y);
    }
};

template <int DOT, int KC, bool SPAN>
__global__ void __launch_bounds__(kRingThreads, 2)
    k_apply_ring(Grid<float> G, const uint8_t* __restrict__ type, const float* __restrict__ x, float* __restrict__ y,
                 const float* __restrict__ d0, double* __restrict__ partial, int ntx, int nty, int ntz,
                 int* __restrict__ wait_err) {
    using namespace tc;
    // indexed from the __shared__ array itself, so that every stage access
    // is a shared-memory load with a 32-bit address
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const float* sf = reinterpret_cast<const float*>(ring_smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(ring_smem + kRingStages * kRingStage);  // filled: 32 producer lanes
    uint64_t* empty = full + kRingStages;  // released by the consumer warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kRingStages; ++q) {
            mbar_init(&full[q], 32);
            mbar_init(&empty[q], kRingCons / 32);
        }
        mbar_fence_init();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const unsigned sy = (unsigned)nx, sz = (unsigned)nx * (unsigned)ny;
    const int64_t N = (int64_t)sz * nz;
    const int ntiles = ntx * nty * ntz;
    DotAcc2 dacc0, dacc1;
    if (warp == kRingCons / 32) {
        // producer warp.  SPAN (n_x <= 514, one tile column): lane 0 copies
        // x, lane 1 the dot operand, lane 2 the type bytes, each as one span
        // of whole rows.  Otherwise lanes 0-3 copy the x rows, 4-5 the dot
        // rows, 6-7 the type rows.  Every lane arrives on the stage's barrier
        // once per plane with the bytes its copy will deliver.
        constexpr int nxl = SPAN ? 1 : kRingRows + 2, per = SPAN ? 1 : kRingRows;
        const bool xl = lane < nxl, dl = !xl && lane < nxl + per, tl = !xl && !dl && lane < nxl + 2 * per;
        const int r = xl ? lane : dl ? lane - nxl : lane - nxl - per;  // row of a row copy
        const unsigned char* arr = xl ? (const unsigned char*)x : dl ? (const unsigned char*)d0 : type;
        const int esize = tl ? 1 : 4;
        const int dst_off = xl ? r * kRingXRow * 4 : dl ? kRingDOff + r * kRingDRow * 4 : kRingTOff + r * kRingTRow;
        unsigned g = 0;  // planes issued; plane g uses stage g % kRingStages
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int tyi = tile % nty, rest = tile / nty, tx = rest % ntx, tz = rest / ntx;
            const int i0 = 1 + tx * kRingTX, j0 = 1 + tyi * kRingRows, k0 = 1 + tz * KC;
            const int k1 = min(k0 + KC, nz - 1);
            int64_t rowe;  // the copy's first element within a plane
            int w;         // elements wanted
            if (SPAN) {
                rowe = (int64_t)(xl ? j0 - 1 : j0) * sy;
                w = xl ? min(4, ny - (j0 - 1)) * nx : 2 * nx;  // the rows that exist
            } else {
                rowe = xl ? (int64_t)min(j0 - 1 + r, ny - 1) * sy + (i0 - 1) : (int64_t)min(j0 + r, ny - 2) * sy + i0;
                w = xl ? kRingTX + 2 : kRingTX;
            }
            for (int k = k0 - 1; k <= k1; ++k, ++g) {
                const int st = g % kRingStages;
                if (g >= kRingStages) {  // refill only a stage every consumer warp released
                    bool okw = true;
                    if (lane == 0) okw = mbar_wait(&empty[st], ((g / kRingStages) - 1) & 1);
                    if (!__shfl_sync(0xffffffffu, okw, 0)) {
                        ok = false;
                        if (lane == 0) atomicExch(wait_err, 31);
                        break;
                    }
                }
                const bool outp = k >= k0 && k < k1;  // an output plane
                const bool act = xl || (outp && (tl || (dl && DOT)));
                unsigned bytes = 0;
                const unsigned char* src = nullptr;
                unsigned char* dst = ring_smem + st * kRingStage + dst_off;
                if (act) bytes = ring_copy(dst, arr, (int64_t)k * sz + rowe, w, esize, N, &src);
                mbar_arrive_expect_tx(&full[st], bytes);
                if (bytes) bulk_load(dst, src, bytes, &full[st]);
            }
        }
        // every copy issued has landed before the CTA may end (after a
        // timeout too): only the last kRingStages planes can be in flight
        if (lane == 0)
            for (unsigned q = g > (unsigned)kRingStages ? g - kRingStages : 0; q < g; ++q)
                if (!mbar_wait(&full[q % kRingStages], (q / kRingStages) & 1)) atomicExch(wait_err, 32);
        __syncwarp();
    } else {
        // consumer: columns i0 + lx (low half) and i0 + 256 + lx (high half)
        // of the rows j0, j0 + 1
        const int lx = threadIdx.x;
        unsigned g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int tyi = tile % nty, rest = tile / nty, tx = rest % ntx, tz = rest / ntx;
            const int i0 = 1 + tx * kRingTX, j0 = 1 + tyi * kRingRows, k0 = 1 + tz * KC;
            const int k1 = min(k0 + KC, nz - 1);
            const int c = i0 + lx;  // the low half's column; the high half's is c + 256
            const bool in0 = c <= nx - 2, in1 = c + kRingCons <= nx - 2;
            const int c0i = in0 ? c : nx - 2, c1i = in1 ? c + kRingCons : nx - 2;
            const float2 AX = f2(G.ax[0].a[c0i], G.ax[0].a[c1i]), CX = f2(G.ax[0].c[c0i], G.ax[0].c[c1i]);
            const float2 ARX = f2(G.ax[0].ar[c0i], G.ax[0].ar[c1i]), BRX = f2(G.ax[0].br[c0i], G.ax[0].br[c1i]);
            const float2 CRX = f2(G.ax[0].cr[c0i], G.ax[0].cr[c1i]);
            float2 AY[2], CY[2], ARY[2], BRY[2], CRY[2];
            bool jin[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                jin[t] = j0 + t <= ny - 2;
                const int jc = min(j0 + t, ny - 2);
                AY[t] = f2b(G.ax[1].a[jc]);
                CY[t] = f2b(G.ax[1].c[jc]);
                ARY[t] = f2b(G.ax[1].ar[jc]);
                BRY[t] = f2b(G.ax[1].br[jc]);
                CRY[t] = f2b(G.ax[1].cr[jc]);
            }
            // stage positions: element (row q, column col) of a plane at
            // xb[q] + ((kp + xa[q]) & 3) + col, kp = the plane's first element
            // (SPAN: one offset for all rows); likewise for the output rows
            int xb[4], db[2], tb[2];
            unsigned xa[4], da[2], ta[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xb[q] = SPAN ? q * nx : q * kRingXRow - (i0 - 1);
                xa[q] = SPAN ? ((unsigned)(j0 - 1) * sy) & 3u
                             : ((unsigned)min(j0 - 1 + q, ny - 1) * sy + (unsigned)(i0 - 1)) & 3u;
            }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const unsigned jr = SPAN ? (unsigned)j0 : (unsigned)min(j0 + t, ny - 2);
                db[t] = SPAN ? t * nx : t * kRingDRow - i0;
                tb[t] = SPAN ? t * nx : t * kRingTRow - i0;
                da[t] = (jr * sy + (SPAN ? 0u : (unsigned)i0)) & 3u;
                ta[t] = (jr * sy + (SPAN ? 0u : (unsigned)i0)) & 15u;
            }
            float2 Pm[2], P0[2], Pp[2], Qm[2], Q0[2], Qp[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) Pm[t] = P0[t] = Pp[t] = Qm[t] = Q0[t] = Qp[t] = f2b(0.f);
            // z coefficients of the plane the next step outputs, loaded a step ahead
            float zn[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            for (int kk = k0 - 1; kk <= k1; ++kk) {
                const float2 AZ = f2b(zn[0]), CZ = f2b(zn[1]), ARZ = f2b(zn[2]), BRZ = f2b(zn[3]), CRZ = f2b(zn[4]);
                if (kk < k1) {
                    const int kn = max(kk, 1);
                    zn[0] = G.ax[2].a[kn];
                    zn[1] = G.ax[2].c[kn];
                    zn[2] = G.ax[2].ar[kn];
                    zn[3] = G.ax[2].br[kn];
                    zn[4] = G.ax[2].cr[kn];
                }
                const unsigned gp = g + (unsigned)(kk - (k0 - 1));
                const unsigned st = gp % kRingStages;
                if (ok && !mbar_wait(&full[st], (gp / kRingStages) & 1)) {
                    ok = false;
                    atomicExch(wait_err, 33);
                }
                const unsigned kp = (unsigned)kk * sz;
                const float* xs = sf + st * (kRingStage / 4) + c;
                float2 XR[4], XL[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float* row = xs + xb[q] + (int)((kp + xa[SPAN ? 0 : q]) & 3u);
                    const float2 xm = f2(row[-1], row[kRingCons - 1]), x0 = f2(row[0], row[kRingCons]),
                                 xp = f2(row[1], row[kRingCons + 1]);
                    XR[q] = fma2(CRX, xp, fma2(BRX, x0, mul2(ARX, xm)));
                    XL[q] = fma2(CX, xp, fma2(AX, xm, x0));
                }
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    Pm[t] = P0[t];
                    P0[t] = Pp[t];
                    Qm[t] = Q0[t];
                    Q0[t] = Qp[t];
                    Pp[t] = fma2(CRY[t], XL[t + 2],
                                 fma2(BRY[t], XL[t + 1],
                                      fma2(ARY[t], XL[t], fma2(CY[t], XR[t + 2], fma2(AY[t], XR[t], XR[t + 1])))));
                    Qp[t] = fma2(CY[t], XL[t + 2], fma2(AY[t], XL[t], XL[t + 1]));
                }
                if (kk >= k0) {
                    const unsigned sq = (gp - 1) % kRingStages;  // plane kk - 1: output (from kk = k0 + 1 on), then released
                    if (kk >= k0 + 1 && in0) {
                        const unsigned kq = (unsigned)(kk - 1) * sz;
                        const unsigned char* ts = ring_smem + sq * kRingStage + kRingTOff + c;
                        const float* ds = sf + sq * (kRingStage / 4) + kRingDOff / 4 + c;
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            if (!jin[t]) continue;
                            float2 v = add2(fma2(CZ, Pp[t], fma2(AZ, Pm[t], P0[t])),
                                            fma2(CRZ, Qp[t], fma2(BRZ, Q0[t], mul2(ARZ, Qm[t]))));
                            const unsigned char* tr = ts + tb[t] + (int)((kq + ta[SPAN ? 0 : t]) & 15u);
                            // solid rows are zero; irregular rows belong to k_apply_irr
                            const uint8_t t0 = tr[0], t1 = in1 ? tr[kRingCons] : (uint8_t)CFP_SOLID;
                            if (t0 != CFP_REGULAR) v.x = 0.f;
                            if (t1 != CFP_REGULAR) v.y = 0.f;
                            float* yr = y + (kq + (unsigned)(j0 + t) * sy + (unsigned)c);
                            if (t0 != CFP_IRREGULAR) yr[0] = v.x;
                            if (in1 && t1 != CFP_IRREGULAR) yr[kRingCons] = v.y;
                            if (DOT >= 1) {
                                const float* dr = ds + db[t] + (int)((kq + da[SPAN ? 0 : t]) & 3u);
                                dacc0.add(f2(dr[0], in1 ? dr[kRingCons] : 0.f), v);
                            }
                            if (DOT == 2) dacc1.add(v, v);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[sq]);
                }
            }
            __syncwarp();
            g += (unsigned)(k1 - k0 + 2);
            if (lane == 0) mbar_arrive(&empty[(g - 1) % kRingStages]);  // the tile's last plane
        }
    }
    if (DOT) {
        double acc0 = dacc0.total(), acc1 = dacc1.total();
        block_reduce2(acc0, acc1);
        if (threadIdx.x == 0) {
            partial[2 * blockIdx.x] = acc0;
            partial[2 * blockIdx.x + 1] = acc1;
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

// The rows of the irregular points, whole (Eq. Bdec): the regular 27-point
// part with the arithmetic of the factorised kernels -- the same fused
// multiply-add chains on the same 27 values, so that part has the same bits
// as there -- plus the side-list corrections of the row's modified lines
// (Eqs. A27_mod, cor, cor_case2).  One thread per irregular point.  The
// regular rows' kernels leave these rows alone, so this kernel runs beside
// them on a second stream; its dot terms go to its own partials.
template <class T, int DOT>
__global__ void __launch_bounds__(128)
    k_apply_irr(Grid<T> G, Side<T> S, const int32_t* __restrict__ irr_lin, int64_t n_irr, const T* __restrict__ x,
                T* __restrict__ y, const T* __restrict__ d0, double* __restrict__ partial) {
    const int nx = G.nx, ny = G.ny;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    double acc0 = 0.0, acc1 = 0.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n_irr;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = irr_lin[s];
        const int k = (int)(l / sz), rem = (int)(l - k * sz), j = rem / nx, i = rem - j * nx;
        const T ax = G.ax[0].a[i], cx = G.ax[0].c[i], arx = G.ax[0].ar[i], brx = G.ax[0].br[i], crx = G.ax[0].cr[i];
        const T ay = G.ax[1].a[j], cy = G.ax[1].c[j], ary = G.ax[1].ar[j], bry = G.ax[1].br[j], cry = G.ax[1].cr[j];
        const T az = G.ax[2].a[k], cz = G.ax[2].c[k], arz = G.ax[2].ar[k], brz = G.ax[2].br[k], crz = G.ax[2].cr[k];
        T P[3], Q[3];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
            T XR[3], XL[3];
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const T* q = x + l + (dz - 1) * sz + (dy - 1) * sy;
                XR[dy] = fmat(crx, q[1], fmat(brx, q[0], mult(arx, q[-1])));
                XL[dy] = fmat(cx, q[1], fmat(ax, q[-1], q[0]));
            }
            P[dz] = fmat(cry, XL[2], fmat(bry, XL[1], fmat(ary, XL[0], fmat(cy, XR[2], fmat(ay, XR[0], XR[1])))));
            Q[dz] = fmat(cy, XL[2], fmat(ay, XL[0], XL[1]));
        }
        T v = fmat(cz, P[2], fmat(az, P[0], P[1])) + fmat(crz, Q[2], fmat(brz, Q[1], mult(arz, Q[0])));
        // the corrections, summed in entry order; the loads of four entries
        // are issued before their products are added (the gather is
        // latency-bound, and beside the ring kernel few of these CTAs fit)
        T cor = T(0);
        const int e1 = S.corr_ptr[s + 1];
        int e = S.corr_ptr[s];
        for (; e + 4 <= e1; e += 4) {
            const int o0 = S.corr_off[e], o1 = S.corr_off[e + 1], o2 = S.corr_off[e + 2], o3 = S.corr_off[e + 3];
            const T w0 = S.corr_val[e], w1 = S.corr_val[e + 1], w2 = S.corr_val[e + 2], w3 = S.corr_val[e + 3];
            const T x0 = x[l + o0], x1 = x[l + o1], x2 = x[l + o2], x3 = x[l + o3];
            cor = fmat(w3, x3, fmat(w2, x2, fmat(w1, x1, fmat(w0, x0, cor))));
        }
        for (; e < e1; ++e) cor = fmat(S.corr_val[e], x[l + S.corr_off[e]], cor);
        v = v + cor;
        y[l] = v;
        if (DOT >= 1) acc0 += (double)d0[l] * (double)v;
        if (DOT == 2) acc1 += (double)v * (double)v;
    }
    if (DOT) {
        block_reduce2(acc0, acc1);
        if (threadIdx.x == 0) {
            partial[2 * blockIdx.x] = acc0;
            partial[2 * blockIdx.x + 1] = acc1;
        }
    }
}

// Side-list corrections of the irregular rows (the modified stencils of
// Secs. 2.2-2.3, the C part of Eq. Bdec) added to a y that holds their
// regular part, one warp per irregular point: the lanes gather the merged
// entries in parallel, lane 0 adds the sum to y and updates the dot partials:
// (d0, y) gains d0 c, (y, y) gains 2 v c + c^2 where v is the row's regular
// part.  Used for the boundary lift (after k_lift_shell), one pair of
// partials per CTA.
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

// the apply's kernel and tile shape of precision q (0 FP64, 1 FP32), as set
// by the autotuner; otherwise in FP64 the streaming kernel with 4 x 64, in
// FP32 the ring (2 x 64) where its 512-column tiles are at least 85 % filled
// (n_x = 513: 511 of 512 columns) and else the streaming kernel with 2 x 64
// (at 385^3, 383 of 512 columns, it measured 0.285 ms against 0.256 ms)
int apply_kind(const cfp_ctx* c, int q) {
    if (c->apply_kind[q]) return c->apply_kind[q];
    if (q == 1 && c->ring_grid > 0) {
        const int cols = c->n[0] - 2, tiles = (cols + kRingTX - 1) / kRingTX;
        if (cols * 100 >= 85 * tiles * kRingTX) return CFP_APPLY_RING;
    }
    return CFP_APPLY_STREAM;
}
int apply_rows(const cfp_ctx* c, int q) { return c->apply_ty[q] ? c->apply_ty[q] : (q ? 2 : 4); }
int apply_planes(const cfp_ctx* c, int q) { return c->apply_kc[q] ? c->apply_kc[q] : 64; }

}  // namespace

// the kernel and tile shape the apply of precision q runs with
void apply_shape(const cfp_ctx* c, int q, int* kernel, int* rows, int* planes) {
    *kernel = apply_kind(c, q);
    *rows = *kernel == CFP_APPLY_RING ? 2 : apply_rows(c, q);
    *planes = apply_planes(c, q);
    if (*kernel == CFP_APPLY_RING && *planes < 32) *planes = 32;
}

namespace {

// the ring's tiles: 512 columns x 2 rows x kc planes
void ring_tiles(const cfp_ctx* c, int kc, int* ntx, int* nty, int* ntz) {
    *ntx = (c->n[0] - 2 + kRingTX - 1) / kRingTX;
    *nty = (c->n[1] - 2 + kRingRows - 1) / kRingRows;
    *ntz = (c->n[2] - 2 + kc - 1) / kc;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

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

// CTAs of k_apply_irr (128 threads, one irregular point each per pass; at
// most 152 x 8, never more than corr_blocks)
int irr_blocks(const cfp_ctx* c) {
    if (c->n_irr <= 0) return 0;
    return (int)std::min<int64_t>((c->n_irr + 127) / 128, 152 * 8);
}

// the most CTAs any apply tile shape launches, with the correction kernel's
// (dot-product partials per launch); the ring's persistent grid never has
// more CTAs than the streaming kernel with 2 rows x 16 planes
int apply_blocks(cfp_ctx* c) {
    int64_t m = 0;
    for (int ty : {2, 4})
        for (int kc : {16, 32, 64}) {
            const dim3 g = rows_grid(c, ty, kc);
            m = std::max<int64_t>(m, (int64_t)g.x * g.y * g.z);
        }
    return (int)m + corr_blocks(c);
}

// B x: the regular rows' kernel on s and, forked onto the context's second
// stream and joined back before anything later on s, the irregular rows'
// kernel; dot partials: the main kernel's CTAs, then k_apply_irr's.
template <class T, int DOT, int TY, int KC>
void apply_launch(cfp_ctx* c, const T* x, T* y, const T* d0, double* partial, cudaStream_t s, int* nb) {
    int nmain = 0;
    bool ring = false;
    constexpr int RKC = KC < 32 ? 32 : KC;  // the ring marches 32 or 64 planes
    int ntx = 0, nty = 0, ntz = 0;
    dim3 grid;
    if constexpr (sizeof(T) == 4)
        ring = apply_kind(c, 1) == CFP_APPLY_RING && c->ring_grid > 0 && aligned16(x) && (!DOT || aligned16(d0));
    if (ring) {
        ring_tiles(c, RKC, &ntx, &nty, &ntz);
        nmain = std::min(ntx * nty * ntz, c->ring_grid);
    } else {
        grid = rows_grid(c, TY, KC);
        nmain = (int)(grid.x * grid.y * grid.z);
    }
    const int nirr = irr_blocks(c);
    if (nirr) {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
        k_apply_irr<T, DOT><<<nirr, 128, 0, c->aux>>>(grid_view<T>(c), side_view<T>(c), c->irr_lin, c->n_irr, x, y,
                                                      d0, partial ? partial + 2 * (int64_t)nmain : nullptr);
    }
    if (ring) {
        if constexpr (sizeof(T) == 4) {
            if (c->n[0] <= kRingSpanNx)
                k_apply_ring<DOT, RKC, true><<<nmain, kRingThreads, kRingSmem, s>>>(
                    grid_view<float>(c), c->type, x, y, d0, partial, ntx, nty, ntz, c->dwait);
            else
                k_apply_ring<DOT, RKC, false><<<nmain, kRingThreads, kRingSmem, s>>>(
                    grid_view<float>(c), c->type, x, y, d0, partial, ntx, nty, ntz, c->dwait);
        }
    } else {
        k_apply<T, DOT, TY, KC><<<grid, kAX, 0, s>>>(grid_view<T>(c), c->type, x, y, d0, partial);
    }
    if (nirr) {
        cudaEventRecord(c->ev_join, c->aux);
        cudaStreamWaitEvent(s, c->ev_join, 0);
    }
    c->launches += nirr ? 1 : 0;
    if (nb) *nb = nmain + nirr;
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

namespace {
template <int DOT, int KC, bool SPAN>
bool ring_attr(int* per) {
    if (cudaFuncSetAttribute(k_apply_ring<DOT, KC, SPAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingSmem) !=
        cudaSuccess)
        return false;
    int p = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, k_apply_ring<DOT, KC, SPAN>, kRingThreads, kRingSmem) !=
        cudaSuccess)
        return false;
    *per = std::min(*per, p);
    return true;
}
template <int DOT>
bool ring_attr_kc(int* per) {
    return ring_attr<DOT, 32, true>(per) && ring_attr<DOT, 64, true>(per) && ring_attr<DOT, 32, false>(per) &&
           ring_attr<DOT, 64, false>(per);
}
}  // namespace

// The ring's launch attributes and persistent grid (CTAs resident on every
// SM at once), once per context before any capture.
bool setup_apply_ring(cfp_ctx* c) {
    if (c->ring_grid) return c->ring_grid > 0;
    int per = 1 << 20, nsm = 0;
    const bool ok = ring_attr_kc<0>(&per) && ring_attr_kc<1>(&per) && ring_attr_kc<2>(&per) &&
                    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess;
    cudaGetLastError();
    c->ring_grid = ok && per >= 1 ? per * nsm : -1;
    return c->ring_grid > 0;
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
