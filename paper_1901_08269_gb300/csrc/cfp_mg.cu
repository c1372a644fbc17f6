// Geometric multigrid V-cycle as the approximate solver of the
// preconditioner system K phi = rho (Sec. 3.3: K is the 7-point second-order
// operator of Eq. A7 with the Shortley-Weller rows of Eq. A7_mod; the paper
// solves it approximately with a fixed number of inner iterations).  This is
// an alternative to the red-black Gauss-Seidel inner iterations; it is a
// fixed linear map (fixed sweep counts, zero initial guesses), so BiCGSTAB
// stays valid, and its quality does not degrade with the grid size.
//
// Levels: vertex-centred coarsening per axis, coarse node I sits on fine node
// map(I) = min(2I, n-1), n_c = (n + 2) / 2, while every axis has >= 17 nodes
// (so the coarsest level has 9 to 16 nodes on its shortest axis: 10^3 below
// 513^3; one level more or less was slower there).
// Coarse K is the 7-point operator rediscretised on the coarse coordinates
// (Eq. 2ndorder_coef); a coarse node is solid if its fine node is solid, and
// its solid neighbours enter with value zero (Dirichlet at the node, no
// Shortley-Weller distance).  Prolongation is trilinear in the coordinates;
// restriction is its transpose normalised by the weight sums (full
// weighting).  Smoother: red-black Gauss-Seidel, mg_smooth sweeps (red then
// black) before the coarse correction and mg_post after it, 16 on the
// coarsest level.
//
// Storage: every level keeps its vectors in a red-black split layout (each
// colour in its own array, rows of (n_x + 1) / 2 entries padded to 16), so a
// half-sweep reads the other colour and writes its own without moving the
// unused half of each cache line.  On the large levels the FP32 half-sweeps
// stream tiles of the other colour (with a one-node halo) and of b through
// shared memory with TMA bulk-tensor copies (k_sweep_tma).  The fine level
// converts on the way in (the first red half-sweep reads rho in the natural
// layout and stores both colours of it) and on the way out (the last black
// half-sweep writes both colours of phi in the natural layout).
//
// Two exact shortcuts of red-black smoothing: after a sweep ends with the
// black half, the residual of every black row is zero (that half-sweep just
// solved those rows), so only red residuals are formed and restricted; and a
// red half-sweep overwrites every red value without reading it, so the
// coarse correction is only added to the black nodes.
#include <algorithm>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled

#include "cfp_internal.cuh"

namespace cfp {
namespace {

constexpr int kSplitThreads = 128;

// per fine index of an axis: fine node i = wlo * coarse[ilo] + whi * coarse[ilo + 1],
// one wide load
template <class T>
struct IpPk;
template <>
struct __align__(16) IpPk<float> {
    float wlo, whi;
    int ilo, pad;
};
template <>
struct __align__(32) IpPk<double> {
    double wlo, whi;
    int ilo, pad[3];
};
// per coarse index I of an axis: the interpolation weights of fine nodes
// 2I - 1, 2I, 2I + 1 to coarse node I (the rows of P^T)
template <class T>
struct __align__(4 * sizeof(T)) RwPk {
    T w[4];
};

template <class T>
struct Transfer {
    const IpPk<T>* ip[3];
    const RwPk<T>* rw[3];
};

// (ka, kb, kc) of one index of one axis, packed for a single wide load
template <class T>
struct Pk;
template <>
struct Pk<float> {
    using type = float4;
};
struct __align__(32) PkD {
    double x, y, z, w;
};
template <>
struct Pk<double> {
    using type = PkD;
};
template <class T>
using PkT = typename Pk<T>::type;

// one level in the split layout; entry offsets within a colour array are
// 32-bit (the level build rejects arrays of 2^31 entries or more)
template <class T>
struct SLev {
    int nx, ny, nz;
    int hp;                     // entries per row of one colour
    unsigned hs;                // hp * ny
    const PkT<T>* cx;           // packed K coefficients per axis index
    const PkT<T>* cy;
    const PkT<T>* cz;
    const uint8_t* ty[2];       // split type per colour
    T* e[2];                    // the iterate per colour
    T* b[2];                    // the right-hand side per colour
    T* r0;                      // the red residual
};

// the arrays one half-sweep of colour c touches (chosen on the host)
template <class T>
struct Half {
    const uint8_t* ty;   // type of colour c
    T* eown;             // e of colour c (written)
    const T* eoth;       // e of the other colour (read)
    T* bown;             // b of colour c
    T* both;             // b of the other colour (written in MODE 2)
    const uint8_t* tyo;  // type of the other colour (MODE 2)
};

// FP32 levels hold NaN in b at every entry that is not an unknown (the TMA
// passes tell the unknowns by b == b and need not load the type)
__device__ __forceinline__ float b_mark() { return __int_as_float(0x7fc00000); }

enum { kSplitVecs = 5 };  // e0 e1 b0 b1 r0

__device__ __forceinline__ bool is_unknown(uint8_t t) { return t == CFP_REGULAR || t == CFP_IRREGULAR; }

// x * (1 / d).  FP64: a correctly rounded reciprocal (two roundings instead
// of the division's one, several times cheaper than an IEEE division).  FP32:
// the hardware reciprocal approximation (rcp.approx.ftz.f32, within 1 ulp of
// 1 / d; the diagonal of K is a normal number), a single instruction where the
// correctly rounded one costs a short sequence: the FP32 smoother is the inner
// preconditioner of the mixed solve, whose FP64 refinement removes the error.
// The off-diagonal sum of a half-sweep node,
//   (cx_lo xm + cx_hi xp) + (cy_lo ym + cy_hi yp) + (cz_lo zm + cz_hi zp),
// each pair one product and one fused multiply-add in this order: written
// out so that every kernel that updates a node (one launch per half-sweep,
// the TMA pipeline, the single-CTA smoothing) rounds it the same way.
__device__ __forceinline__ float rb_pair(float a, float x, float b, float y) { return __fmaf_rn(b, y, __fmul_rn(a, x)); }
__device__ __forceinline__ double rb_pair(double a, double x, double b, double y) {
    return __fma_rn(b, y, __dmul_rn(a, x));
}
template <class T>
__device__ __forceinline__ T rb_sum(T cxl, T cxh, T cyl, T cyh, T czl, T czh, T xm, T xp, T ym, T yp, T zm, T zp) {
    return (rb_pair(cxl, xm, cxh, xp) + rb_pair(cyl, ym, cyh, yp)) + rb_pair(czl, zm, czh, zp);
}

__device__ __forceinline__ float times_rcp(float x, float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return x * r;
}
__device__ __forceinline__ double times_rcp(double x, double d) { return x * __drcp_rn(d); }

// One red-black half-sweep of colour `colour` on a split level, with K's
// regular coefficients at every node.  Thread (m, j, k0 + q), q <
// kSweepPlanes, owns the pair of nodes i = 2m, 2m + 1 of rows (j, k0 + q);
// its node of this colour is i = 2m + par.  Its x-neighbours (the other
// colour) sit at entries m - 1 + par and m + par of the other colour's row.
// Every load is in bounds for every thread that passes the first test (rows
// j, k and the pair are interior, entry m - 1 exists for m = 0 because the
// row is not the first; planes past the last interior one repeat plane k0
// and store nothing), so the loads of all kSweepPlanes nodes are issued
// before any value is stored: three independent nodes per thread keep more
// loads in flight.  The Shortley-Weller rows of the fine level's irregular
// nodes are applied afterwards by k_sweep_fix (no node reads another of its
// own colour, so the order within the half-sweep does not matter).
// MODE 0: plain; 1: from zero (the other colour is taken as zero);
// 2: from zero, and b of both colours is first read from the natural-layout
//    rho; 3: plain, and both nodes of the pair are written to the
//    natural-layout phi (the own node's new value is not stored).
constexpr int kSweepPlanes = 3;

template <class T, int MODE>
__global__ void __launch_bounds__(kSplitThreads)
    k_sweep_split(SLev<T> L, Half<T> H, int colour, const T* __restrict__ rho, T* __restrict__ phi) {
    const int nx = L.nx;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y, k0 = 1 + kSweepPlanes * blockIdx.z;
    if (2 * m > nx - 2 || j > L.ny - 2) return;
    const int hp = L.hp;
    const unsigned hs = L.hs;
    const T* __restrict__ eoth = H.eoth;
    T val[kSweepPlanes], bv[kSweepPlanes], bo[kSweepPlanes], xo[kSweepPlanes];
    bool inz[kSweepPlanes], live[kSweepPlanes];
    unsigned oo[kSweepPlanes];
#pragma unroll
    for (int q = 0; q < kSweepPlanes; ++q) {
        inz[q] = k0 + q <= L.nz - 2;
        const int k = inz[q] ? k0 + q : k0;
        const int par = (colour + j + k) & 1;
        const int i = 2 * m + par, io = 2 * m + 1 - par;
        const unsigned o = (unsigned)k * hs + (unsigned)(j * hp + m);
        const int64_t row = ((int64_t)k * L.ny + j) * nx;
        const uint8_t t = H.ty[o];
        bv[q] = MODE == 2 ? rho[row + i] : H.bown[o];
        if (MODE == 2) {
            bo[q] = rho[row + io];
            if (sizeof(T) == 4) {  // the NaN marks of the FP32 levels
                if (!is_unknown(t)) bv[q] = T(b_mark());
                if (!is_unknown(H.tyo[o])) bo[q] = T(b_mark());
            }
        }
        T xm = T(0), xp = T(0), ym = T(0), yp = T(0), zm = T(0), zp = T(0);
        if (MODE == 0 || MODE == 3) {
            xm = eoth[o - 1 + par];
            xp = eoth[o + par];
            ym = eoth[o - hp];
            yp = eoth[o + hp];
            zm = eoth[o - hs];
            zp = eoth[o + hs];
        }
        const PkT<T> ckx = L.cx[i], cky = L.cy[j], ckz = L.cz[k];
        const T dg = ckx.y + (cky.y + ckz.y);
        live[q] = inz[q] && i >= 1 && i <= nx - 2 && is_unknown(t);
        T v = bv[q];
        if (MODE == 0 || MODE == 3)
            v -= rb_sum(ckx.x, ckx.z, cky.x, cky.z, ckz.x, ckz.z, xm, xp, ym, yp, zm, zp);
        val[q] = times_rcp(v, dg);
        xo[q] = par ? xm : xp;  // MODE 3: the other node of the pair
        oo[q] = o;
    }
#pragma unroll
    for (int q = 0; q < kSweepPlanes; ++q) {
        if (!inz[q]) continue;
        const unsigned o = oo[q];
        if (MODE == 2) {
            H.bown[o] = bv[q];
            H.both[o] = bo[q];
        }
        if (MODE == 3) {
            const int k = k0 + q;
            const int par = (colour + j + k) & 1;
            const int i = 2 * m + par, io = 2 * m + 1 - par;
            const int64_t row = ((int64_t)k * L.ny + j) * nx;
            if (i >= 1 && i <= nx - 2) phi[row + i] = live[q] ? val[q] : T(0);
            if (io >= 1 && io <= nx - 2) phi[row + io] = xo[q];
        } else if (live[q]) {
            H.eown[o] = val[q];
        }
    }
}

// All the red-black sweeps of one smoothing of a small level (at most
// kCoarseMaxNodes nodes: the coarsest level's 16 sweeps, a 17^3 level's
// pre- or post-smoothing) in one CTA, with a CTA barrier between
// half-sweeps, where separate launches would cost a few microseconds each
// for a few thousand nodes.  The node update is k_sweep_split's (MODE 1 for
// a first red half-sweep from zero, MODE 0 otherwise) with the same rb_sum
// and reciprocal: the results are bitwise equal.
// CLUSTER: the same with the CTAs of one thread-block cluster (up to 16,
// one per SM) and a cluster barrier, whose release / acquire order the
// global writes of one half-sweep before the reads of the next, for levels
// of up to kClusterMaxNodes nodes (33^3; at 65^3, eight nodes per thread
// and half-sweep, separate launches on the whole GPU measured faster).
constexpr int kCoarseThreads = 512;
constexpr int64_t kCoarseMaxNodes = int64_t(1) << 15;
constexpr int kClusterThreads = 1024;
constexpr int64_t kClusterMaxNodes = int64_t(1) << 16;

template <class T, bool CLUSTER>
__global__ void __launch_bounds__(CLUSTER ? kClusterThreads : kCoarseThreads)
    k_smooth_cta(SLev<T> L, int sweeps, int first_red_zero) {
    const int nx = L.nx, ny = L.ny, nz = L.nz, hp = L.hp;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    const unsigned hs = L.hs;
    const int mp = (nx - 2) / 2 + 1;  // pairs m with 2 m <= nx - 2
    const int64_t items = (int64_t)mp * (ny - 2) * (nz - 2);
    for (int q = 0; q < 2 * sweeps; ++q) {
        const int colour = q & 1;
        const bool zero = q == 0 && first_red_zero;
        // plain pointers: the e arrays are written by this launch's earlier
        // half-sweeps, so their loads must not take the non-coherent
        // read-only path that a const __restrict__ pointer allows
        T* eown = colour ? L.e[1] : L.e[0];
        const T* eoth = colour ? L.e[0] : L.e[1];
        const T* bown = colour ? L.b[1] : L.b[0];
        const uint8_t* ty = colour ? L.ty[1] : L.ty[0];
        for (int64_t it = t0; it < items; it += nt) {
            const int m = (int)(it % mp);
            const int64_t rest = it / mp;
            const int j = 1 + (int)(rest % (ny - 2)), k = 1 + (int)(rest / (ny - 2));
            const int par = (colour + j + k) & 1;
            const int i = 2 * m + par;
            const unsigned o = (unsigned)k * hs + (unsigned)(j * hp + m);
            const uint8_t t = ty[o];
            T v = bown[o];
            T xm = T(0), xp = T(0), ym = T(0), yp = T(0), zm = T(0), zp = T(0);
            if (!zero) {
                xm = eoth[o - 1 + par];
                xp = eoth[o + par];
                ym = eoth[o - hp];
                yp = eoth[o + hp];
                zm = eoth[o - hs];
                zp = eoth[o + hs];
            }
            const PkT<T> ckx = L.cx[i], cky = L.cy[j], ckz = L.cz[k];
            const T dg = ckx.y + (cky.y + ckz.y);
            if (!zero) v -= rb_sum(ckx.x, ckx.z, cky.x, cky.z, ckz.x, ckz.z, xm, xp, ym, yp, zm, zp);
            const T val = times_rcp(v, dg);
            if (i >= 1 && i <= nx - 2 && is_unknown(t)) eown[o] = val;
        }
        if (CLUSTER) cooperative_groups::this_cluster().sync();
        else __syncthreads();
    }
}

// ---------------------------------------------------------------- TMA path
// Three FP32 passes of a large level with the access pattern of a half-sweep
// (a node of one colour reads its six neighbours of the other colour and its
// b, NaN where the node is not an unknown), run as a pipeline.  KIND 0: the plain half-sweep (MODE 0)
// into e of its colour; KIND 1: the red residual r0 = b0 - K e (k_resid_split;
// the stage also holds the red e of the tile); KIND 2: the fine level's last
// black half-sweep into the natural-layout phi, both nodes of each pair
// (MODE 3).  Per CTA
// one producer thread streams planes of a tile through a ring of shared-memory
// stages with cp.async.bulk.tensor (completion counted on an mbarrier per
// stage), and kTmaRows consumer warps update the tile's nodes from shared
// memory and release each plane through a second mbarrier.  A tile is
// kTmaTX pairs x kTmaRows rows x kTmaPlanes planes of colour `colour`; a
// stage holds, for one plane k, the other colour's pairs m0 - 4 .. m0 +
// kTmaTX + 3 of rows j0 - 1 .. j0 + kTmaRows (the one-node halo in x and y;
// the x start is a multiple of 4 entries, 16 bytes) and b of the tile's own
// rows; the output of plane k reads the stages of planes k - 1, k, k + 1.
// Copies outside the array (row j0 + kTmaRows past the last, pair -4 .. -1)
// fill zeros and feed only nodes that are not updated.  The CTAs
// are persistent: CTA q takes tiles q, q + grid, ... with the x tile varying
// fastest, then y, then the z chunk, so the CTAs at work at one time share
// their halo rows through L2.  Same arithmetic as k_sweep_split<float, 0>:
// the results are bitwise equal.
constexpr int kTmaTX = 128;     // pairs per tile row: one consumer thread each
constexpr int kTmaRows = 8;     // rows per tile: consumer warps 0-3 take rows 0-3, warps 4-7 rows 4-7
constexpr int kTmaPlanes = 32;  // output planes per tile
constexpr int kTmaMinPairs = 96;  // levels with fewer pairs per row use k_sweep_split
constexpr int kTmaOX = kTmaTX + 8;                                   // other-colour row in a stage
constexpr int kTmaOBytes = kTmaOX * (kTmaRows + 2) * 4;              // other-colour tile
constexpr int kTmaOPad = (kTmaOBytes + 127) / 128 * 128;
constexpr int kTmaBBytes = kTmaTX * kTmaRows * 4;                    // b of the tile
constexpr int kTmaThreads = 32 * (kTmaRows + 1);                     // + the producer warp
// a stage: [other colour with halo | b | (KIND 1) own e]; KIND 1 has a
// larger stage and one stage fewer, so three CTAs still fit an SM.  The type
// is not loaded: b is NaN exactly at the entries that are not unknowns.
__host__ __device__ constexpr int tma_stage(int kind) {
    return kTmaOPad + kTmaBBytes + (kind == 1 ? kTmaBBytes : 0);
}
__host__ __device__ constexpr int tma_stages(int kind) { return kind == 1 ? 5 : 6; }
__host__ __device__ constexpr int tma_smem(int kind) {
    return tma_stages(kind) * tma_stage(kind) + 2 * tma_stages(kind) * 8 + 128;  // + barriers, alignment
}
static_assert(tma_stage(0) % 128 == 0 && tma_stage(1) % 128 == 0 && kTmaBBytes % 128 == 0,
              "stage buffers stay 128-byte aligned");
static_assert(kTmaRows % 4 == 0, "rows come in groups of four per 128 consumer threads");

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` of barrier b to complete, for one
// second at most (a healthy wait takes microseconds); false if it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity) {
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int q = 0; q < 32; ++q)
            if (mbar_try_wait(b, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// A wait that runs out (1 s) records a code in *wait_err (1: producer, stage
// free; 2: producer, final drain; 3, 4: consumer, stage filled).  A producer
// whose wait ran out issues no further copy and then waits (bounded) for the
// copies it has issued, so no CTA ends with a bulk copy in flight into its
// shared memory; a consumer whose wait ran out stops waiting: every index
// stays in bounds whatever the stages hold, so the launch still ends, and
// the host reports the error.
// out: e of `colour` (KIND 0), r0 (KIND 1, colour 0), phi (KIND 2, colour 1).
template <int KIND>
__global__ void __launch_bounds__(kTmaThreads)
    k_sweep_tma(const __grid_constant__ CUtensorMap t_oth, const __grid_constant__ CUtensorMap t_b,
                const __grid_constant__ CUtensorMap t_own, SLev<float> L,
                float* __restrict__ out, int colour, int ntx, int nty, int ntz, int* __restrict__ wait_err) {
    constexpr int kTmaStages = tma_stages(KIND), kTmaStage = tma_stage(KIND);
    constexpr int kEOff = kTmaOPad + kTmaBBytes;  // KIND 1: own e of the tile
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t* full = (uint64_t*)(base + kTmaStages * kTmaStage);  // stage filled (tx bytes landed)
    uint64_t* empty = full + kTmaStages;                           // stage released by every consumer warp
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kTmaStages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kTmaRows);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int ntiles = ntx * nty * ntz;
    if (warp == kTmaRows) {  // producer
        if (lane != 0) return;
        unsigned g = 0;  // planes issued by this CTA; plane g uses stage g % kTmaStages
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int tx = tile % ntx, rest = tile / ntx, tyi = rest % nty, tz = rest / nty;
            const int m0 = tx * kTmaTX, j0 = 1 + tyi * kTmaRows, k0 = 1 + tz * kTmaPlanes;
            const int k1 = min(k0 + kTmaPlanes, nz - 1);
            for (int k = k0 - 1; k <= k1; ++k, ++g) {
                const int st = g % kTmaStages;
                // a stage is refilled only once every consumer warp released
                // it; if that wait runs out, nothing more is issued (the
                // consumers may still read the stage)
                if (g >= kTmaStages && !mbar_wait(&empty[st], ((g / kTmaStages) - 1) & 1)) {
                    ok = false;
                    atomicExch(wait_err, 1);
                    break;
                }
                unsigned char* buf = base + st * kTmaStage;
                mbar_arrive_expect_tx(&full[st], kTmaOBytes + kTmaBBytes + (KIND == 1 ? kTmaBBytes : 0));
                tma_load_3d(buf, &t_oth, &full[st], m0 - 4, j0 - 1, k);
                tma_load_3d(buf + kTmaOPad, &t_b, &full[st], m0, j0, k);
                if (KIND == 1) tma_load_3d(buf + kEOff, &t_own, &full[st], m0, j0, k);
            }
        }
        // Every copy issued has landed before the CTA may end, after a
        // timeout too: planes g - kTmaStages .. g - 1 are the only ones whose
        // stage was not released (an older plane's stage was waited free
        // before it was refilled), and each of their full phases is the
        // latest of its barrier.  Each wait is bounded again.
        for (unsigned q = g > (unsigned)kTmaStages ? g - kTmaStages : 0; q < g; ++q)
            if (!mbar_wait(&full[q % kTmaStages], (q / kTmaStages) & 1)) atomicExch(wait_err, 2);
        return;
    }
    // consumers: thread (lx, group) owns pair m0 + lx of the rows r0 .. r0 + 3
    const int lx = threadIdx.x & (kTmaTX - 1), r0 = 4 * (threadIdx.x / kTmaTX);
    const unsigned hs = L.hs;
    const int hp = L.hp;
    unsigned g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = tile % ntx, rest = tile / ntx, tyi = rest % nty, tz = rest / nty;
        const int m = tx * kTmaTX + lx, j0 = 1 + tyi * kTmaRows + r0, k0 = 1 + tz * kTmaPlanes;
        const int nk = min(k0 + kTmaPlanes, nz - 1) - k0;
        // the pair's two nodes: coefficients and whether each is an interior column
        const float4 c0 = L.cx[min(2 * m, nx - 1)], c1 = L.cx[min(2 * m + 1, nx - 1)];
        const bool in0 = 2 * m >= 1 && 2 * m <= nx - 2, in1 = 2 * m + 1 <= nx - 2;
        float cya[4], cyb[4], cyc[4];
        bool jin[4];
#pragma unroll
        for (int ly = 0; ly < 4; ++ly) {
            const float4 cy = L.cy[min(j0 + ly, ny - 1)];
            cya[ly] = cy.x;
            cyb[ly] = cy.y;
            cyc[ly] = cy.z;
            jin[ly] = j0 + ly <= ny - 2;
        }
        for (int q = 0; q < 2; ++q)
            if (ok && !mbar_wait(&full[(g + q) % kTmaStages], ((g + q) / kTmaStages) & 1)) {
                ok = false;
                atomicExch(wait_err, 3);
            }
        for (int kk = 0; kk < nk; ++kk) {
            const unsigned gp = g + kk;  // stage of plane k - 1
            if (ok && !mbar_wait(&full[(gp + 2) % kTmaStages], ((gp + 2) / kTmaStages) & 1)) {
                ok = false;
                atomicExch(wait_err, 4);
            }
            const int at = (r0 + 1) * kTmaOX + lx + 4;  // the thread's first row, centre entry
            const unsigned char* s0 = base + ((gp + 1) % kTmaStages) * kTmaStage;
            const float* Om = (const float*)(base + (gp % kTmaStages) * kTmaStage) + at;
            const float* O0 = (const float*)s0 + at;
            const float* Op = (const float*)(base + ((gp + 2) % kTmaStages) * kTmaStage) + at;
            const float* Bs = (const float*)(s0 + kTmaOPad) + r0 * kTmaTX + lx;
            const float* Es = (const float*)(s0 + kEOff) + r0 * kTmaTX + lx;  // KIND 1 only
            const int k = k0 + kk;
            const float4 cz = L.cz[k];
            const int p0 = (colour + j0 + k) & 1;  // parity of row r0; rows alternate
            const float4 ce = p0 ? c1 : c0, co = p0 ? c0 : c1;
            const bool ine = p0 ? in1 : in0, ino = p0 ? in0 : in1;
            float* ep = out + ((unsigned)k * hs + (unsigned)(j0 * hp + m));  // KIND 0, 1
            // KIND 2: natural-layout row of (j0, k) and the pair's first node
            float* pp = out + ((unsigned)k * (unsigned)ny + (unsigned)j0) * (unsigned)nx + 2u * (unsigned)m;
#pragma unroll
            for (int ly = 0; ly < 4; ++ly) {
                const int par = p0 ^ (ly & 1);
                const float4 cx = (ly & 1) ? co : ce;
                const int o = ly * kTmaOX;
                const float xm = O0[o - 1 + par], xp = O0[o + par], ym = O0[o - kTmaOX], yp = O0[o + kTmaOX];
                const float zm = Om[o], zp = Op[o];
                const float b = Bs[ly * kTmaTX];
                const bool unk = b == b;  // not NaN: an unknown
                const float dg = cx.y + (cyb[ly] + cz.y);
                const bool in = (ly & 1) ? ino : ine;  // the node of this colour is an interior column
                if (KIND == 1) {
                    const float e0 = Es[ly * kTmaTX];
                    const float ke =
                        dg * e0 + (cx.x * xm + cx.z * xp) + (cya[ly] * ym + cyc[ly] * yp) + (cz.x * zm + cz.z * zp);
                    if (in && jin[ly] && unk) ep[ly * hp] = b - ke;
                } else {
                    float v = b;
                    v -= rb_sum(cx.x, cx.z, cya[ly], cyc[ly], cz.x, cz.z, xm, xp, ym, yp, zm, zp);
                    if (KIND == 0) {
                        if (in && jin[ly] && unk) ep[ly * hp] = times_rcp(v, dg);
                    } else if (jin[ly]) {
                        // this colour's node i = 2m + par gets its new value (0 off
                        // the unknowns), the pair's other node keeps the other colour's
                        float* row = pp + (unsigned)ly * (unsigned)nx;
                        const bool ino2 = (ly & 1) ? ine : ino;  // the other node is an interior column
                        if (in) row[par] = unk ? times_rcp(v, dg) : 0.f;
                        if (ino2) row[1 - par] = par ? xm : xp;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[gp % kTmaStages]);
        }
        __syncwarp();
        if (lane == 0) {  // the tile's last two planes
            mbar_arrive(&empty[(g + nk) % kTmaStages]);
            mbar_arrive(&empty[(g + nk + 1) % kTmaStages]);
        }
        g += nk + 2;
    }
}

// The bounded wait on its own: one thread waits on the first phase of a
// barrier that expects one arrival that never comes; mbar_wait gives up after
// one second and the kernel records code 5.  No copy is in flight.
__global__ void k_wait_diag(int* __restrict__ wait_err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0)) atomicExch(wait_err, 5);
}

// An irregular node of the fine level, for the follow-up kernels: natural
// index, offset in its colour's split array, slot (its K row), parity of i.
struct __align__(16) FixPt {
    int lin;
    unsigned o;
    int slot;
    int par;
};

// The per-colour lists of FixPt in ascending natural index (irr_lin
// ascends): a stable split of the irregular nodes by colour.  k_fix_count
// counts the red nodes of each block of kFixBlock entries; k_fix_place ranks
// each node among the earlier nodes of its colour (the red counts of the
// earlier blocks, then a ballot count within the block) and stores it there.
constexpr int kFixBlock = 1024;

__device__ __forceinline__ int fix_colour(int64_t l, int nx, int ny) {
    const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
    return (i + j + k) & 1;
}

__global__ void __launch_bounds__(kFixBlock) k_fix_count(const int32_t* __restrict__ irr_lin, int64_t n_irr, int nx,
                                                         int ny, int* __restrict__ red_count) {
    __shared__ int wsum[kFixBlock / 32];
    const int64_t s = blockIdx.x * (int64_t)kFixBlock + threadIdx.x;
    const bool red = s < n_irr && fix_colour(irr_lin[s], nx, ny) == 0;
    const int w = __popc(__ballot_sync(0xffffffffu, red));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int q = 0; q < kFixBlock / 32; ++q) t += wsum[q];
        red_count[blockIdx.x] = t;
    }
}

// total[0], total[1]: the lengths of the red and the black list
__global__ void __launch_bounds__(kFixBlock)
    k_fix_place(const int32_t* __restrict__ irr_lin, int64_t n_irr, int nx, int ny, int hp, unsigned hs,
                const int* __restrict__ red_count, FixPt* __restrict__ out, int* __restrict__ total) {
    __shared__ int wsum[kFixBlock / 32];
    __shared__ int base;
    if (threadIdx.x < 32) {  // red nodes of the earlier blocks
        int t = 0;
        for (unsigned q = threadIdx.x; q < blockIdx.x; q += 32) t += red_count[q];
        for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
        if (threadIdx.x == 0) base = t;
    }
    const int64_t s = blockIdx.x * (int64_t)kFixBlock + threadIdx.x;
    const int64_t l = s < n_irr ? irr_lin[s] : 0;
    const bool red = s < n_irr && fix_colour(l, nx, ny) == 0;
    const unsigned bal = __ballot_sync(0xffffffffu, red);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int before = base;  // red nodes before node s
    for (int q = 0; q < warp; ++q) before += wsum[q];
    before += __popc(bal & ((1u << lane) - 1u));
    if (s < n_irr) {
        const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
        const FixPt p{(int)l, (unsigned)k * hs + (unsigned)(j * hp + (i >> 1)), (int)s, i & 1};
        if (red) out[before] = p;
        else out[n_irr + (s - before)] = p;  // the black nodes before s: s minus the red ones
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        int t = base;
        for (int q = 0; q < kFixBlock / 32; ++q) t += wsum[q];
        total[0] = t;
        total[1] = (int)(n_irr - t);
    }
}

// rows[r], r = 0 .. nrows: the first entry of `list` (n entries, ascending)
// whose row (k n_y + j = lin / n_x) is at least r
__global__ void k_fix_rows(const FixPt* __restrict__ list, int n, int nx, int64_t nrows, int32_t* __restrict__ rows) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= nrows; r += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (list[mid].lin / nx < r) lo = mid + 1;
            else hi = mid;
        }
        rows[r] = lo;
    }
}

// The half-sweep's update at the fine level's irregular nodes of colour
// `colour` (the list of that colour), with their Shortley-Weller rows
// (Eq. A7_mod); one thread per node.  Runs right after the half-sweep of the
// same colour and mode, overwriting what it stored there.
template <class T, int MODE>
__global__ void k_sweep_fix(SLev<T> L, Side<T> S, Half<T> H, const FixPt* __restrict__ list, int64_t n,
                            T* __restrict__ phi) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const FixPt p = list[q];
        const int par = p.par;
        const unsigned o = p.o;
        const T* kr = S.krow + 7 * (int64_t)p.slot;
        T v = H.bown[o];
        if (MODE == 0 || MODE == 3) {
            const T* __restrict__ eoth = H.eoth;
            v -= rb_sum(kr[1], kr[2], kr[3], kr[4], kr[5], kr[6], eoth[o - 1 + par], eoth[o + par], eoth[o - L.hp],
                        eoth[o + L.hp], eoth[o - L.hs], eoth[o + L.hs]);
        }
        v = times_rcp(v, kr[0]);
        if (MODE == 3) phi[p.lin] = v;
        else H.eown[o] = v;
    }
}

// ------------------------------------------------ fused black + red pass
// The black half-sweep of one red-black sweep and the red half-sweep of the
// next (both plain, MODE 0) in one TMA-fed pass over an FP32 level.  Per tile
// (kPairTX pairs x kTmaRows rows x up to kTmaPlanes planes) the CTA marches in
// z: at step k it forms the new black values of plane k on the tile and on a
// ring one pair (x) or one row (y) wide around it, from the old red values
// staged with a two-node halo, keeps them in a ring of kPairRing planes in
// shared memory, and then forms the new red values of plane k - 1 from them.
// A half-sweep reads no node of the colour it updates, so the black values
// are stored in place, while the red values go to the other red array: the
// neighbouring tiles still read the old red values for their rings.  On the
// fine level the Shortley-Weller rows (Eq. A7_mod) are applied in the pass,
// to the black ring as well, from per-row ranges of the sorted irregular
// lists.  Every node is formed by the arithmetic of k_sweep_tma<0> or
// k_sweep_fix<float, 0>, so the pass is bitwise the two half-sweeps.
constexpr int kPairTX = 64;                                       // pairs per tile row
constexpr int kPairOX = kPairTX + 8;                              // staged row: entries m0 - 4 .. m0 + kPairTX + 3
constexpr int kPairWarps = kPairTX * kTmaRows / (4 * 32);          // consumer warps: four rows per thread
constexpr int kPairThreads = 32 * (kPairWarps + 1);               // + the producer warp
constexpr int kPairYRows = kTmaRows + 4;                          // old red rows j0 - 2 .. j0 + rows + 1
constexpr int kPairXRows = kTmaRows + 2;                          // black rows j0 - 1 .. j0 + rows
constexpr int kPairYBytes = kPairOX * kPairYRows * 4;             // old red
constexpr int kPairBBytes = kPairOX * kPairXRows * 4;             // black b of the tile and its ring
constexpr int kPairBPad = (kPairBBytes + 127) / 128 * 128;
constexpr int kPairRBytes = kPairTX * kTmaRows * 4;               // red b of the tile
constexpr int kPairStage = kPairYBytes + kPairBPad + kPairRBytes;  // [old red | black b | red b]
constexpr int kPairStages = 5;
constexpr int kPairRing = 4;                                      // planes of new black values
constexpr int kPairPlane = kPairOX * kPairXRows;                  // floats per ring plane
constexpr int kPairSmem = kPairStages * kPairStage + kPairRing * kPairPlane * 4 + 2 * kPairStages * 8 + 128;
static_assert(kPairYBytes % 128 == 0 && kPairStage % 128 == 0, "stage buffers stay 128-byte aligned");
static_assert(kPairSmem <= 54 * 1024, "four CTAs per SM");

// the fine level's irregular nodes for the fused pass (list null elsewhere)
struct PairFix {
    const FixPt* list;     // colour c's nodes at list + c * n_irr, ascending natural index
    const int32_t* rows;   // colour c's row starts at rows + c * (nrows + 1)
    const float* krow;     // 7 K coefficients per slot
    int64_t n_irr;
    int64_t nrows;         // n_y n_z
};

__device__ __forceinline__ void pair_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kPairWarps * 32) : "memory"); }

// the new black value of one node from the staged values: c its centre in
// the old-red boxes (planes k - 1, k, k + 1 in Ym, Y0, Yp), b its right-hand
// side, par its parity, cx / cy / cz its coefficients; zero where it is not
// an unknown interior node (live false or b NaN), as the black array holds
__device__ __forceinline__ float pair_node(const float* Ym, const float* Y0, const float* Yp, float b, int c, int par,
                                           float4 cx, float4 cy, float4 cz, bool live) {
    const float v = b - rb_sum(cx.x, cx.z, cy.x, cy.z, cz.x, cz.z, Y0[c - 1 + par], Y0[c + par], Y0[c - kPairOX],
                               Y0[c + kPairOX], Ym[c], Yp[c]);
    const float dg = cx.y + (cy.y + cz.y);
    return live && b == b ? times_rcp(v, dg) : 0.f;
}

// Waits, codes and the drain as in k_sweep_tma (codes 1, 2 producer; 3, 4
// consumer).  t_red: the current red array (box kPairOX x kPairYRows); t_bb:
// black b (kPairOX x kPairXRows); t_br: red b (kPairTX x kTmaRows).  The new
// black values go to L.e[1], the new red values to red_out.
__global__ void __launch_bounds__(kPairThreads, 4)
    k_sweep_pair(const __grid_constant__ CUtensorMap t_red, const __grid_constant__ CUtensorMap t_bb,
                 const __grid_constant__ CUtensorMap t_br, SLev<float> L, float* __restrict__ red_out, PairFix F,
                 int ntx, int nty, int ntz, int* __restrict__ wait_err) {
    constexpr int S = kPairStages;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    float* ring = (float*)(base + S * kPairStage);
    uint64_t* full = (uint64_t*)(base + S * kPairStage + kPairRing * kPairPlane * 4);
    uint64_t* empty = full + S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], kPairWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int ntiles = ntx * nty * ntz;
    if (warp == kPairWarps) {  // producer: planes k0 - 2 .. k1 + 1 of each tile
        if (lane != 0) return;
        unsigned g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int tx = tile % ntx, rest = tile / ntx, tyi = rest % nty, tz = rest / nty;
            const int m0 = tx * kPairTX, j0 = 1 + tyi * kTmaRows, k0 = 1 + tz * kTmaPlanes;
            const int k1 = min(k0 + kTmaPlanes, nz - 1);
            for (int k = k0 - 2; k <= k1 + 1; ++k, ++g) {
                const int st = g % S;
                if (g >= (unsigned)S && !mbar_wait(&empty[st], ((g / S) - 1) & 1)) {
                    ok = false;
                    atomicExch(wait_err, 1);
                    break;
                }
                unsigned char* buf = base + st * kPairStage;
                mbar_arrive_expect_tx(&full[st], kPairYBytes + kPairBBytes + kPairRBytes);
                tma_load_3d(buf, &t_red, &full[st], m0 - 4, j0 - 2, k);
                tma_load_3d(buf + kPairYBytes, &t_bb, &full[st], m0 - 4, j0 - 1, k);
                tma_load_3d(buf + kPairYBytes + kPairBPad, &t_br, &full[st], m0, j0, k);
            }
        }
        for (unsigned q = g > (unsigned)S ? g - S : 0; q < g; ++q)
            if (!mbar_wait(&full[q % S], (q / S) & 1)) atomicExch(wait_err, 2);
        return;
    }
    // consumers: thread (lx, group) owns pair m0 + lx of the tile rows r0 ..
    // r0 + 3, the node of that pair in the ring row of its group (row -1 or
    // kTmaRows) and, for lx < kTmaRows, the ring node of row lx left (group
    // 0) or right (group 1) of the tile.  Per tile the z coefficients, the
    // ring's coefficients and the irregular lists' ranges of every plane are
    // first staged in shared memory: within the pass the CTA's warps meet at
    // a barrier every plane, so a global load in the loop would stall them all.
    __shared__ float4 czs[kTmaPlanes + 2];  // planes k0 - 1 .. k1
    __shared__ float4 cyt[kTmaRows + 2];    // rows j0 - 1 .. j0 + kTmaRows
    __shared__ float4 cxt[4];               // ring pairs m0 - 1, m0 + kPairTX: nodes 2m, 2m + 1
    __shared__ int2 xr[kTmaPlanes + 2];     // black irregular nodes of rows j0 - 1 .. j0 + kTmaRows, per plane
    __shared__ int2 yr[kTmaPlanes + 2];     // red irregular nodes of rows j0 .. j0 + kTmaRows - 1, per plane
    const int lx = threadIdx.x & (kPairTX - 1), grp = threadIdx.x / kPairTX, r0 = 4 * grp;
    const unsigned hs = L.hs;
    const int hp = L.hp;
    float* eb = L.e[1];
    unsigned g = 0, sx = 0;  // planes consumed; black planes formed (ring slot sx % kPairRing)
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tx = tile % ntx, rest = tile / ntx, tyi = rest % nty, tz = rest / nty;
        const int m0 = tx * kPairTX, m = m0 + lx, j0 = 1 + tyi * kTmaRows, k0 = 1 + tz * kTmaPlanes;
        const int nk = min(k0 + kTmaPlanes, nz - 1) - k0;
        pair_bar();  // the previous tile's tables are no longer read
        {
            const int t = threadIdx.x;
            if (t < nk + 2) {
                const int k = k0 - 1 + t;
                czs[t] = L.cz[k];
                if (F.list) {
                    const int64_t rb = (int64_t)k * ny;
                    const int32_t* rwb = F.rows + (F.nrows + 1);
                    xr[t] = make_int2(rwb[rb + j0 - 1], rwb[rb + min(j0 + kTmaRows, ny - 1) + 1]);
                    yr[t] = make_int2(F.rows[rb + j0], F.rows[rb + min(j0 + kTmaRows - 1, ny - 1) + 1]);
                }
            } else if (t >= 64 && t < 64 + kTmaRows + 2) {
                cyt[t - 64] = L.cy[min(j0 - 1 + (t - 64), ny - 1)];
            } else if (t >= 96 && t < 100) {
                const int mc = m0 + (t >= 98 ? kPairTX : -1);
                cxt[t - 96] = L.cx[min(max(2 * mc + (t & 1), 0), nx - 1)];
            }
        }
        const float4 c0 = L.cx[min(2 * m, nx - 1)], c1 = L.cx[min(2 * m + 1, nx - 1)];
        const bool in0 = 2 * m >= 1 && 2 * m <= nx - 2, in1 = 2 * m + 1 <= nx - 2;
        float4 cyo[4];
        bool jin[4];
#pragma unroll
        for (int ly = 0; ly < 4; ++ly) {
            cyo[ly] = L.cy[min(j0 + r0 + ly, ny - 1)];
            jin[ly] = j0 + r0 + ly <= ny - 2;
        }
        const int rr = grp ? kTmaRows : -1, jr = j0 + rr;  // the group's ring row
        const bool jrin = jr >= 1 && jr <= ny - 2;
        const int mc = grp ? kPairTX : -1, jc = j0 + lx;    // ring column node (lx < kTmaRows)
        const bool jcin = jc <= ny - 2;
        pair_bar();
        for (int q = 0; q < 2; ++q)
            if (ok && !mbar_wait(&full[(g + q) % S], ((g + q) / S) & 1)) {
                ok = false;
                atomicExch(wait_err, 3);
            }
        for (int q = 1; q <= nk + 2; ++q, ++sx) {
            const int k = k0 + q - 2;  // plane of the new black values; the red ones are of k - 1
            const unsigned gp = g + q;
            if (ok && !mbar_wait(&full[(gp + 1) % S], ((gp + 1) / S) & 1)) {
                ok = false;
                atomicExch(wait_err, 4);
            }
            const unsigned char* sM = base + ((gp - 1) % S) * kPairStage;
            const unsigned char* s0 = base + (gp % S) * kPairStage;
            const float* Ym = (const float*)sM;
            const float* Y0 = (const float*)s0;
            const float* Yp = (const float*)(base + ((gp + 1) % S) * kPairStage);
            const float* Bx = (const float*)(s0 + kPairYBytes);
            float* xb = ring + (sx % kPairRing) * kPairPlane;
            {  // black values of plane k
                const float4 cz = czs[q - 1];
                const bool kin = k >= 1 && k <= nz - 2;
                const int p0 = (1 + j0 + r0 + k) & 1;
#pragma unroll
                for (int ly = 0; ly < 4; ++ly) {
                    const int par = p0 ^ (ly & 1);
                    const int cb = (r0 + ly + 1) * kPairOX + lx + 4;
                    xb[cb] = pair_node(Ym, Y0, Yp, Bx[cb], cb + kPairOX, par, par ? c1 : c0, cyo[ly], cz,
                                       (par ? in1 : in0) && jin[ly] && kin);
                }
                {
                    const int par = (1 + jr + k) & 1;
                    const int cb = (rr + 1) * kPairOX + lx + 4;
                    xb[cb] = pair_node(Ym, Y0, Yp, Bx[cb], cb + kPairOX, par, par ? c1 : c0, cyt[rr + 1], cz,
                                       (par ? in1 : in0) && jrin && kin);
                }
                if (lx < kTmaRows) {
                    const int par = (1 + jc + k) & 1, i = 2 * (m0 + mc) + par;
                    const int cb = (lx + 1) * kPairOX + mc + 4;
                    xb[cb] = pair_node(Ym, Y0, Yp, Bx[cb], cb + kPairOX, par, cxt[2 * grp + par], cyt[lx + 1], cz,
                                       i >= 1 && i <= nx - 2 && jcin && kin);
                }
            }
            // the Shortley-Weller rows among the black nodes just formed
            if (F.list) {
                const int2 ra = xr[q - 1];
                if (ra.x < ra.y) {
                    pair_bar();
                    const FixPt* lst = F.list + F.n_irr;
                    for (int q2 = ra.x + (int)threadIdx.x; q2 < ra.y; q2 += kPairWarps * 32) {
                        const FixPt p = lst[q2];
                        const int i = p.lin % nx, j = (p.lin / nx) % ny;
                        const int mm = (i >> 1) - m0, r = j - j0;
                        if (mm < -1 || mm > kPairTX) continue;
                        const float* kr = F.krow + 7 * (int64_t)p.slot;
                        const int cb = (r + 1) * kPairOX + mm + 4, c = cb + kPairOX, par = p.par;
                        const float v = Bx[cb] - rb_sum(kr[1], kr[2], kr[3], kr[4], kr[5], kr[6], Y0[c - 1 + par],
                                                        Y0[c + par], Y0[c - kPairOX], Y0[c + kPairOX], Ym[c], Yp[c]);
                        xb[cb] = times_rcp(v, kr[0]);
                    }
                }
            }
            pair_bar();
            if (q >= 3) {  // red values of plane kr = k - 1 from the black planes kr - 1, kr, kr + 1
                const int kr = k - 1;
                const float* Xm = ring + ((sx - 2) % kPairRing) * kPairPlane;
                const float* X0 = ring + ((sx - 1) % kPairRing) * kPairPlane;
                const float* By = (const float*)(sM + kPairYBytes + kPairBPad);
                const float4 cz = czs[q - 2];
                const int p0 = (j0 + r0 + kr) & 1;
#pragma unroll
                for (int ly = 0; ly < 4; ++ly) {
                    const int par = p0 ^ (ly & 1);
                    const float4 cx = par ? c1 : c0;
                    const int c = (r0 + ly + 1) * kPairOX + lx + 4;
                    const float b = By[(r0 + ly) * kPairTX + lx];
                    const float v = b - rb_sum(cx.x, cx.z, cyo[ly].x, cyo[ly].z, cz.x, cz.z, X0[c - 1 + par],
                                               X0[c + par], X0[c - kPairOX], X0[c + kPairOX], Xm[c], xb[c]);
                    const float dg = cx.y + (cyo[ly].y + cz.y);
                    const unsigned o = (unsigned)kr * hs + (unsigned)((j0 + r0 + ly) * hp + m);
                    if ((par ? in1 : in0) && jin[ly] && b == b) red_out[o] = times_rcp(v, dg);
                    if ((par ? in0 : in1) && jin[ly]) eb[o] = X0[c];  // the pair's black node
                }
                if (F.list) {
                    const int2 ra = yr[q - 2];
                    if (ra.x < ra.y) {
                        pair_bar();
                        for (int q2 = ra.x + (int)threadIdx.x; q2 < ra.y; q2 += kPairWarps * 32) {
                            const FixPt p = F.list[q2];
                            const int i = p.lin % nx, j = (p.lin / nx) % ny;
                            const int mm = (i >> 1) - m0, r = j - j0;
                            if (mm < 0 || mm >= kPairTX) continue;
                            const float* kr7 = F.krow + 7 * (int64_t)p.slot;
                            const int c = (r + 1) * kPairOX + mm + 4, par = p.par;
                            const float v = By[r * kPairTX + mm] -
                                            rb_sum(kr7[1], kr7[2], kr7[3], kr7[4], kr7[5], kr7[6], X0[c - 1 + par],
                                                   X0[c + par], X0[c - kPairOX], X0[c + kPairOX], Xm[c], xb[c]);
                            red_out[p.o] = times_rcp(v, kr7[0]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[(gp - 1) % S]);
        }
        __syncwarp();
        if (lane == 0) {  // the tile's last two planes
            mbar_arrive(&empty[(g + nk + 2) % S]);
            mbar_arrive(&empty[(g + nk + 3) % S]);
        }
        g += nk + 4;
    }
}

// r0 = b0 - K e at the red unknowns with K's regular coefficients (black
// residuals are zero after a black half-sweep; r0 stays zero at the other
// red entries); three planes per thread with all loads first, as in the
// half-sweep.  k_resid_fix then redoes the fine level's irregular red nodes.
template <class T>
__global__ void __launch_bounds__(kSplitThreads) k_resid_split(SLev<T> L) {
    const int nx = L.nx;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y, k0 = 1 + kSweepPlanes * blockIdx.z;
    if (2 * m > nx - 2 || j > L.ny - 2) return;
    const int hp = L.hp;
    const unsigned hs = L.hs;
    const T* __restrict__ e1 = L.e[1];
    T rv[kSweepPlanes];
    bool live[kSweepPlanes];
    unsigned oo[kSweepPlanes];
#pragma unroll
    for (int q = 0; q < kSweepPlanes; ++q) {
        const bool inz = k0 + q <= L.nz - 2;
        const int k = inz ? k0 + q : k0;
        const int par = (j + k) & 1;
        const int i = 2 * m + par;
        const unsigned o = (unsigned)k * hs + (unsigned)(j * hp + m);
        const uint8_t t = L.ty[0][o];
        const T e0 = L.e[0][o], b0 = L.b[0][o];
        const T xm = e1[o - 1 + par], xp = e1[o + par], ym = e1[o - hp], yp = e1[o + hp], zm = e1[o - hs],
                zp = e1[o + hs];
        const PkT<T> ckx = L.cx[i], cky = L.cy[j], ckz = L.cz[k];
        const T dg = ckx.y + (cky.y + ckz.y);
        const T ke = dg * e0 + (ckx.x * xm + ckx.z * xp) + (cky.x * ym + cky.z * yp) + (ckz.x * zm + ckz.z * zp);
        rv[q] = b0 - ke;
        live[q] = inz && i >= 1 && i <= nx - 2 && is_unknown(t);
        oo[q] = o;
    }
#pragma unroll
    for (int q = 0; q < kSweepPlanes; ++q)
        if (live[q]) L.r0[oo[q]] = rv[q];
}

// the red residual at the fine level's irregular red nodes with their
// Shortley-Weller rows (after k_resid_split)
template <class T>
__global__ void k_resid_fix(SLev<T> L, Side<T> S, const FixPt* __restrict__ red, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const FixPt p = red[q];
        const int par = p.par;
        const unsigned o = p.o;
        const T* kr = S.krow + 7 * (int64_t)p.slot;
        const T* __restrict__ e1 = L.e[1];
        const T ke = kr[0] * L.e[0][o] + (kr[1] * e1[o - 1 + par] + kr[2] * e1[o + par]) +
                     (kr[3] * e1[o - L.hp] + kr[4] * e1[o + L.hp]) + (kr[5] * e1[o - L.hs] + kr[6] * e1[o + L.hs]);
        L.r0[o] = L.b[0][o] - ke;
    }
}

// b_c = (P^T r_f) / (P^T 1) at the coarse unknowns; r_f is the fine red
// residual (zero on black nodes).  One thread per coarse node (I, J, K);
// interior coarse nodes sit on fine node (2I, 2J, 2K).
template <class T>
__global__ void k_restrict_split(Transfer<T> X, SLev<T> F, SLev<T> C) {
    const int I = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int J = 1 + blockIdx.y, K = 1 + blockIdx.z;
    const int ncx = C.nx, ncy = C.ny;
    if (I > ncx - 2) return;
    const int cc = (I + J + K) & 1;
    const unsigned oc = (unsigned)(K * ncy + J) * (unsigned)C.hp + (unsigned)(I >> 1);
    // the type decides only the store, so the fine loads (in bounds for every
    // interior coarse node) are issued beside it
    const uint8_t tc = (cc ? C.ty[1] : C.ty[0])[oc];
    const int nfy = F.ny;
    const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
    const RwPk<T> rx = X.rw[0][I], ry = X.rw[1][J], rz = X.rw[2][K];
    const T* wx = rx.w;
    const T* wy = ry.w;
    const T* wz = rz.w;
    const T* __restrict__ r0 = F.r0;
    T s = 0;
    // fine node (2I - 1 + a, 2J - 1 + b, 2K - 1 + c) is red, (i + j + k) even,
    // exactly where a + b + c is odd: a pattern fixed at compile time, so
    // only those 13 of the 27 terms are formed
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int k = fk - 1 + c;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int j = fj - 1 + b;
            const T wyz = wy[b] * wz[c];
            const unsigned rowo = (unsigned)(k * nfy + j) * (unsigned)F.hp;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int i = fi - 1 + a;
                if ((a + b + c) & 1) s += (wx[a] * wyz) * r0[rowo + (unsigned)(i >> 1)];
            }
        }
    }
    // P^T 1 at the node: the sum of all 27 weights, separable per axis
    const T w = ((wx[0] + wx[1]) + wx[2]) * ((wy[0] + wy[1]) + wy[2]) * ((wz[0] + wz[1]) + wz[2]);
    if (is_unknown(tc)) (cc ? C.b[1] : C.b[0])[oc] = s / w;
}

// e1 += P e_c at the fine black unknowns (the red values are overwritten by
// the next red half-sweep without being read); three planes per thread.
template <class T>
__global__ void __launch_bounds__(kSplitThreads) k_prolong_split(Transfer<T> X, SLev<T> F, SLev<T> C) {
    const int nx = F.nx;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y, k0 = 1 + kSweepPlanes * blockIdx.z;
    if (2 * m > nx - 2 || j > F.ny - 2) return;
    const unsigned hc = (unsigned)C.hp;
    const IpPk<T> py = X.ip[1][j];
    const int J = py.ilo;
    const T ay0 = py.wlo, ay1 = py.whi;
    T* __restrict__ e1 = F.e[1];
    T val[kSweepPlanes];
    bool live[kSweepPlanes];
    unsigned oo[kSweepPlanes];
#pragma unroll
    for (int q = 0; q < kSweepPlanes; ++q) {
        const bool inz = k0 + q <= F.nz - 2;
        const int k = inz ? k0 + q : k0;
        const int i = 2 * m + ((1 + j + k) & 1);
        const int ic = i <= nx - 2 ? i : nx - 2;  // every load stays inside the tables and the level
        const unsigned o = (unsigned)k * F.hs + (unsigned)(j * F.hp + m);
        const uint8_t t = F.ty[1][o];
        const IpPk<T> px = X.ip[0][ic], pz = X.ip[2][k];
        const int I = px.ilo, K = pz.ilo;
        const T ax0 = px.wlo, ax1 = px.whi;
        const T az0 = pz.wlo, az1 = pz.whi;
        // coarse (I + a, J + b, K + c): colour (I + a + J + b + K + c) & 1,
        // entry ((K + c) * ncy + J + b) * hc + (I + a) >> 1
        const int p = (I + J + K) & 1;
        const unsigned r00 = (unsigned)(K * C.ny + J) * hc, r01 = r00 + hc, r10 = r00 + C.hs, r11 = r10 + hc;
        const unsigned x0 = (unsigned)(I >> 1), x1 = (unsigned)((I + 1) >> 1);
        const T* __restrict__ ea = p ? C.e[1] : C.e[0];  // colour p
        const T* __restrict__ eb = p ? C.e[0] : C.e[1];  // colour 1 - p
        const T e000 = ea[r00 + x0], e001 = eb[r00 + x1], e010 = eb[r01 + x0], e011 = ea[r01 + x1];
        const T e100 = eb[r10 + x0], e101 = ea[r10 + x1], e110 = ea[r11 + x0], e111 = eb[r11 + x1];
        const T f0 = e1[o];
        val[q] = f0 + (az0 * (ay0 * (ax0 * e000 + ax1 * e001) + ay1 * (ax0 * e010 + ax1 * e011)) +
                       az1 * (ay0 * (ax0 * e100 + ax1 * e101) + ay1 * (ax0 * e110 + ax1 * e111)));
        live[q] = inz && i >= 1 && i <= nx - 2 && is_unknown(t);
        oo[q] = o;
    }
#pragma unroll
    for (int q = 0; q < kSweepPlanes; ++q)
        if (live[q]) e1[oo[q]] = val[q];
}

// packed (ka, kb, kc) per index of each axis from a level's metric arrays
// The same e1 += P e_c with one thread per coarse cell (I, J, K): the fine
// nodes 2I .. 2I + 1 x 2J .. 2J + 1 x 2K .. 2K + 1 interpolate between the
// cell's eight corners (every interior fine node's lower table index is its
// cell's), so the four black nodes of a cell share eight coarse loads, and
// consecutive threads touch consecutive split entries.  Per node the
// expression is k_prolong_split's.
template <class T>
__global__ void __launch_bounds__(128) k_prolong_cell(Transfer<T> X, SLev<T> F, SLev<T> C) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I > C.nx - 2) return;
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const unsigned hc = (unsigned)C.hp;
    // the corners: colour (I + a + J + b + K + c) & 1, entry ((K + c) ncy + J + b) hc + (I + a) >> 1
    const int p = (I + J + K) & 1;
    const unsigned r00 = (unsigned)(K * C.ny + J) * hc, r01 = r00 + hc, r10 = r00 + C.hs, r11 = r10 + hc;
    const unsigned x0 = (unsigned)(I >> 1), x1 = (unsigned)((I + 1) >> 1);
    const T* __restrict__ ea = p ? C.e[1] : C.e[0];
    const T* __restrict__ eb = p ? C.e[0] : C.e[1];
    const T e000 = ea[r00 + x0], e001 = eb[r00 + x1], e010 = eb[r01 + x0], e011 = ea[r01 + x1];
    const T e100 = eb[r10 + x0], e101 = ea[r10 + x1], e110 = ea[r11 + x0], e111 = eb[r11 + x1];
    T* __restrict__ e1 = F.e[1];
    // every load of the four nodes first (indices clamped into the level, so
    // each is in bounds), the decisions after: the loads overlap
    const IpPk<T> px0 = X.ip[0][min(2 * I, nx - 1)], px1 = X.ip[0][min(2 * I + 1, nx - 1)];
    IpPk<T> pyv[2], pzv[2];
    unsigned o[2][2];
    uint8_t t[2][2];
    T f[2][2];
    bool live[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int k = 2 * K + c, kc = min(max(k, 1), nz - 2);
        pzv[c] = X.ip[2][kc];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int j = 2 * J + b, jc = min(max(j, 1), ny - 2);
            if (c == 0) pyv[b] = X.ip[1][jc];
            const int i = 2 * I + ((1 + j + k) & 1);  // the black node of this row in the cell
            o[c][b] = (unsigned)kc * F.hs + (unsigned)(jc * F.hp + I);  // pair m = I
            t[c][b] = F.ty[1][o[c][b]];
            f[c][b] = e1[o[c][b]];
            live[c][b] = k >= 1 && k <= nz - 2 && j >= 1 && j <= ny - 2 && i >= 1 && i <= nx - 2;
        }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const T az0 = pzv[c].wlo, az1 = pzv[c].whi;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (!live[c][b] || !is_unknown(t[c][b])) continue;
            const T ay0 = pyv[b].wlo, ay1 = pyv[b].whi;
            const IpPk<T>& px = ((1 + 2 * J + b + 2 * K + c) & 1) ? px1 : px0;
            const T ax0 = px.wlo, ax1 = px.whi;
            const T f0 = f[c][b];
            e1[o[c][b]] = f0 + (az0 * (ay0 * (ax0 * e000 + ax1 * e001) + ay1 * (ax0 * e010 + ax1 * e011)) +
                                az1 * (ay0 * (ax0 * e100 + ax1 * e101) + ay1 * (ax0 * e110 + ax1 * e111)));
        }
    }
}

template <class T>
__global__ void k_pack_coefs(Grid<T> G, PkT<T>* __restrict__ out) {
    const int n[3] = {G.nx, G.ny, G.nz};
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    for (int d = 0; d < 3; ++d) {
        if (q < n[d]) {
            PkT<T> v;
            v.x = G.ax[d].ka[q];
            v.y = G.ax[d].kb[q];
            v.z = G.ax[d].kc[q];
            v.w = T(0);
            out[q] = v;
            return;
        }
        q -= n[d];
        out += n[d];
    }
}

// coarse type by injection: box stays box, solid stays solid, fluid -> regular
__device__ __forceinline__ int fine_of(int I, int n) { return min(2 * I, n - 1); }

__global__ void k_inject_type(const uint8_t* __restrict__ ft, int nfx, int nfy, int nfz, uint8_t* __restrict__ ct,
                              int ncx, int ncy, int ncz) {
    const int64_t nc = (int64_t)ncx * ncy * ncz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nc; q += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(q % ncx), J = (int)((q / ncx) % ncy), K = (int)(q / ((int64_t)ncx * ncy));
        const uint8_t t = ft[(int64_t)fine_of(K, nfz) * nfx * nfy + (int64_t)fine_of(J, nfy) * nfx + fine_of(I, nfx)];
        ct[q] = t == CFP_IRREGULAR ? (uint8_t)CFP_REGULAR : t;
    }
}

// natural-layout type -> split type (padding entries are boundary)
__global__ void k_split_type(const uint8_t* __restrict__ nat, int nx, int ny, int nz, int hp,
                             uint8_t* __restrict__ st) {
    const int64_t Nh = (int64_t)hp * ny * nz;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 2 * Nh; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q / Nh);
        const int64_t e = q - c * Nh;
        const int m = (int)(e % hp);
        const int64_t rowi = e / hp;  // k * ny + j
        const int j = (int)(rowi % ny), k = (int)(rowi / ny);
        const int i = 2 * m + ((c + j + k) & 1);
        st[q] = i < nx ? nat[rowi * nx + i] : (uint8_t)CFP_BOUNDARY;
    }
}

// b of both colours (2 Nh entries from b): NaN where the split type is not an
// unknown (padding entries are typed boundary)
__global__ void k_mark_b(const uint8_t* __restrict__ st, float* __restrict__ b, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        if (!is_unknown(st[q])) b[q] = b_mark();
}

unsigned flat_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

// Threads over the pairs m = 0 .. (n_x - 2) / 2 (x) and the interior rows j
// (y), blocks over groups of kSweepPlanes interior planes (z).  A block is
// kSplitThreads threads: as many pairs as the row has, rounded up to a warp
// and at most kSplitThreads, times as many rows as fill it, so that the
// narrow coarse levels do not leave most lanes idle.
dim3 plane_block(const int n[3]) {
    const int bx = std::min(kSplitThreads, (n[0] / 2 + 31) / 32 * 32);
    return dim3((unsigned)bx, (unsigned)(kSplitThreads / bx));
}
dim3 plane_grid(const int n[3]) {
    const dim3 b = plane_block(n);
    return dim3((unsigned)((n[0] / 2 + b.x - 1) / b.x), (unsigned)((n[1] - 2 + b.y - 1) / b.y),
                (unsigned)((n[2] - 2 + kSweepPlanes - 1) / kSweepPlanes));
}

template <class T>
Grid<T> level_grid_view(cfp_ctx* c, MgLevel& L, int l);
template <>
Grid<double> level_grid_view<double>(cfp_ctx* c, MgLevel& L, int l) {
    if (l == 0) return grid_view<double>(c);
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
Grid<float> level_grid_view<float>(cfp_ctx* c, MgLevel& L, int l) {
    if (l == 0) return grid_view<float>(c);
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
T* svec(MgLevel& L);
template <>
double* svec<double>(MgLevel& L) { return L.s64; }
template <>
float* svec<float>(MgLevel& L) { return L.s32; }

template <class T>
const PkT<T>* packed(MgLevel& L);
template <>
const PkD* packed<double>(MgLevel& L) { return static_cast<const PkD*>(L.pk64); }
template <>
const float4* packed<float>(MgLevel& L) { return static_cast<const float4*>(L.pk32); }

template <class T>
SLev<T> slev(cfp_ctx* c, int l) {
    MgLevel& L = c->mg[l];
    SLev<T> v;
    v.nx = L.n[0];
    v.ny = L.n[1];
    v.nz = L.n[2];
    v.hp = L.hp;
    v.hs = (unsigned)((int64_t)L.hp * L.n[1]);
    v.cx = packed<T>(L);
    v.cy = v.cx + L.n[0];
    v.cz = v.cy + L.n[1];
    T* sv = svec<T>(L);
    for (int q = 0; q < 2; ++q) {
        v.ty[q] = L.stype + q * L.Nh;
        v.e[q] = sv + q * L.Nh;
        v.b[q] = sv + (2 + q) * L.Nh;
    }
    v.r0 = sv + 4 * L.Nh;
    if (std::is_same<T, float>::value && L.red_cur) v.e[0] = sv + 5 * L.Nh;  // after an odd number of fused passes
    return v;
}

template <class T>
Transfer<T> transfer(MgLevel& F);
template <>
Transfer<double> transfer<double>(MgLevel& F) {
    Transfer<double> X;
    for (int d = 0; d < 3; ++d) {
        X.ip[d] = static_cast<const IpPk<double>*>(F.ip64) + F.off[d];
        X.rw[d] = static_cast<const RwPk<double>*>(F.rw64) + F.coff[d];
    }
    return X;
}
template <>
Transfer<float> transfer<float>(MgLevel& F) {
    Transfer<float> X;
    for (int d = 0; d < 3; ++d) {
        X.ip[d] = static_cast<const IpPk<float>*>(F.ip32) + F.off[d];
        X.rw[d] = static_cast<const RwPk<float>*>(F.rw32) + F.coff[d];
    }
    return X;
}

// The TMA-fed pass where it applies (FP32, a level with maps): kind 0 the
// plain half-sweep of `colour`, kind 1 the red residual, kind 2 the last
// black half-sweep into phi (natural layout).  False: use the plain kernel.
bool sweep_tma(cfp_ctx*, int, const SLev<double>&, int, int, double*, cudaStream_t) { return false; }
bool sweep_tma(cfp_ctx* c, int l, const SLev<float>& L, int kind, int colour, float* phi, cudaStream_t s) {
    const MgLevel& M = c->mg[l];
    if (!M.tma || !c->mg_tma) return false;
    const int ntx = (M.n[0] / 2 + kTmaTX - 1) / kTmaTX, nty = (M.n[1] - 2 + kTmaRows - 1) / kTmaRows;
    const int ntz = (M.n[2] - 2 + kTmaPlanes - 1) / kTmaPlanes;
    // other colour's e (the red one from the array that holds it), b of `colour`
    const CUtensorMap& t_oth = colour == 1 && M.red_cur ? M.tmalt[0] : M.tm32[2 * colour];
    const CUtensorMap& t_b = M.tm32[2 * colour + 1];
    const unsigned grid = (unsigned)M.tma_grid[kind];
    if (kind == 0)
        k_sweep_tma<0><<<grid, kTmaThreads, tma_smem(0), s>>>(t_oth, t_b, t_oth, L, L.e[colour], colour, ntx, nty,
                                                               ntz, c->dwait);
    else if (kind == 1)
        k_sweep_tma<1><<<grid, kTmaThreads, tma_smem(1), s>>>(t_oth, t_b, M.red_cur ? M.tmalt[1] : M.tm32[4], L,
                                                               L.r0, 0, ntx, nty, ntz, c->dwait);
    else
        k_sweep_tma<2><<<grid, kTmaThreads, tma_smem(2), s>>>(t_oth, t_b, t_oth, L, phi, 1, ntx, nty, ntz,
                                                               c->dwait);
    return true;
}

// The fused black-then-red pass where it applies (FP32, a level with maps):
// the black half-sweep of one sweep and the red half-sweep of the next, both
// plain; the red values go to the other red array.  False: not issued.
// Issued when the context asks for it (mg_tma = 2) or `always` (timing).
bool sweep_pair(cfp_ctx*, int, const Side<double>&, cudaStream_t, bool = false) { return false; }
bool sweep_pair(cfp_ctx* c, int l, const Side<float>& S, cudaStream_t s, bool always = false) {
    MgLevel& M = c->mg[l];
    if (!M.tma || !M.pair || !(always || (c->mg_tma && c->mg_fuse))) return false;
    const SLev<float> L = slev<float>(c, l);
    const int ntx = (M.n[0] / 2 + kPairTX - 1) / kPairTX, nty = (M.n[1] - 2 + kTmaRows - 1) / kTmaRows;
    const int ntz = (M.n[2] - 2 + kTmaPlanes - 1) / kTmaPlanes;
    PairFix F{nullptr, nullptr, nullptr, 0, 0};
    if (l == 0 && M.fix && M.fixrows && S.krow)
        F = PairFix{static_cast<const FixPt*>(M.fix), M.fixrows, S.krow, c->n_irr, (int64_t)M.n[1] * M.n[2]};
    float* red_out = M.s32 + (M.red_cur ? 0 : 5 * M.Nh);
    k_sweep_pair<<<(unsigned)M.pair_grid, kPairThreads, kPairSmem, s>>>(M.tmp[M.red_cur], M.tmp[2], M.tmp[3], L,
                                                                         red_out, F, ntx, nty, ntz, c->dwait);
    M.red_cur ^= 1;
    c->launches += 1;
    return true;
}

// every level's red iterate back in its split array (the state each V-cycle
// and each smoothing call starts from)
void reset_red(cfp_ctx* c) {
    for (MgLevel& M : c->mg) M.red_cur = 0;
}

template <class T>
void half_sweep(cfp_ctx* c, int l, const SLev<T>& L, const Side<T>& S, int colour, int mode, const T* rho, T* phi,
                cudaStream_t s) {
    const dim3 g = plane_grid(c->mg[l].n), blk = plane_block(c->mg[l].n);
    const Half<T> H{L.ty[colour], L.e[colour], L.e[1 - colour], L.b[colour], L.b[1 - colour], L.ty[1 - colour]};
    switch (mode) {
        case 0:
            if (!sweep_tma(c, l, L, 0, colour, phi, s))
                k_sweep_split<T, 0><<<g, blk, 0, s>>>(L, H, colour, rho, phi);
            break;
        case 1: k_sweep_split<T, 1><<<g, blk, 0, s>>>(L, H, colour, rho, phi); break;
        case 2: k_sweep_split<T, 2><<<g, blk, 0, s>>>(L, H, colour, rho, phi); break;
        default:  // the last black half-sweep of the fine level
            if (colour != 1 || !sweep_tma(c, l, L, 2, colour, phi, s))
                k_sweep_split<T, 3><<<g, blk, 0, s>>>(L, H, colour, rho, phi);
            break;
    }
    c->launches += 1;
    const MgLevel& M0 = c->mg[0];
    if (l == 0 && M0.nfix[colour] > 0) {  // the Shortley-Weller rows of the irregular nodes
        const int64_t n = M0.nfix[colour];
        const FixPt* list = static_cast<const FixPt*>(M0.fix) + colour * c->n_irr;
        const unsigned nb = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8);
        switch (mode) {
            case 0: k_sweep_fix<T, 0><<<nb, 256, 0, s>>>(L, S, H, list, n, phi); break;
            case 1: k_sweep_fix<T, 1><<<nb, 256, 0, s>>>(L, S, H, list, n, phi); break;
            case 2: k_sweep_fix<T, 2><<<nb, 256, 0, s>>>(L, S, H, list, n, phi); break;
            default: k_sweep_fix<T, 3><<<nb, 256, 0, s>>>(L, S, H, list, n, phi); break;
        }
        c->launches += 1;
    }
}

// The cluster of k_smooth_cta<T, true>: 16 CTAs where the device schedules
// such a cluster (a non-portable size), else 8, else 0 (not used); found once.
template <class T>
int smooth_cluster_size() {
    static const int size = []() {
        cudaFuncSetAttribute(k_smooth_cta<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        for (int cl : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)cl);
            cfg.blockDim = dim3(kClusterThreads);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)cl;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_smooth_cta<T, true>, &cfg) == cudaSuccess && n >= 1) return cl;
            cudaGetLastError();
        }
        return 0;
    }();
    return size;
}

// `sweeps` red-black sweeps at level l.  first_red / last_black: the modes of
// the first red and the last black half-sweep.
template <class T>
void smooth(cfp_ctx* c, int l, const Side<T>& S, int sweeps, int first_red, int last_black, const T* rho, T* phi,
            cudaStream_t s) {
    const SLev<T> L = slev<T>(c, l);
    // a small coarse level (no irregular rows, plain or from-zero modes):
    // one CTA does every half-sweep
    if (c->mg_tma && l > 0 && c->mg[l].N <= kCoarseMaxNodes && (first_red == 0 || first_red == 1) &&
        last_black == 0) {
        k_smooth_cta<T, false><<<1, kCoarseThreads, 0, s>>>(L, sweeps, first_red);
        c->launches += 1;
        return;
    }
    // a mid-size coarse level: one thread-block cluster does every half-sweep
    const int cl = smooth_cluster_size<T>();
    if (cl > 0 && c->mg_tma && l > 0 && c->mg[l].N <= kClusterMaxNodes && (first_red == 0 || first_red == 1) &&
        last_black == 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cl);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, k_smooth_cta<T, true>, L, sweeps, first_red);
        c->launches += 1;
        return;
    }
    // red of sweep 0, then per sweep q its black half-sweep and the red one of
    // sweep q + 1: one fused pass where the level has one, else two launches
    half_sweep<T>(c, l, L, S, 0, first_red, rho, phi, s);
    for (int q = 0; q < sweeps; ++q) {
        const bool last = q == sweeps - 1;
        if (!last && sweep_pair(c, l, S, s)) continue;
        half_sweep<T>(c, l, slev<T>(c, l), S, 1, last ? last_black : 0, rho, phi, s);
        if (!last) half_sweep<T>(c, l, slev<T>(c, l), S, 0, 0, rho, phi, s);
    }
}

}  // namespace

void free_mg(cfp_ctx* c) {
    if (!c->mg.empty()) c->generation += 1;
    for (MgLevel& L : c->mg) {
        void* ptrs[] = {L.coef64, L.coef32, L.type, L.stype, L.s64, L.s32, L.pk64, L.pk32,
                        L.ip64, L.ip32, L.rw64, L.rw32, L.fix, L.fixrows};
        for (void* p : ptrs) pool_free(p, c->stream);
    }
    c->mg.clear();
}

namespace {

// The level hierarchy below the fine grid (after classification): sizes,
// coordinates, interpolation tables, coarse coefficients and types.
cfp_status build_levels(cfp_ctx* c) {
    std::vector<MgLevel> levels(1);
    MgLevel& F0 = levels[0];
    for (int d = 0; d < 3; ++d) {
        F0.n[d] = c->n[d];
        F0.X[d] = c->X[d];
    }
    F0.N = c->N;
    while (std::min({levels.back().n[0], levels.back().n[1], levels.back().n[2]}) >= 17) {
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
    // from here on every device pointer is owned by c->mg, so free_mg cleans
    // up after a failure
    c->mg = levels;
    for (int l = 0; l < nl; ++l) {
        MgLevel& L = c->mg[l];
        // interpolation tables from level l + 1 (per fine index of level l)
        if (l + 1 < nl) {
            const MgLevel& Cn = c->mg[l + 1];
            int64_t tot = 0, ctot = 0;
            for (int d = 0; d < 3; ++d) {
                L.off[d] = tot;
                tot += L.n[d];
                L.coff[d] = ctot;
                ctot += Cn.n[d];
            }
            std::vector<IpPk<double>> ipd(tot);
            std::vector<IpPk<float>> ipf(tot);
            std::vector<RwPk<double>> rwd(ctot);
            std::vector<RwPk<float>> rwf(ctot);
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
                    ipd[L.off[d] + i] = IpPk<double>{wl, wh, I, {0, 0, 0}};
                    ipf[L.off[d] + i] = IpPk<float>{(float)wl, (float)wh, I, 0};
                }
                // weight of fine node i to coarse node I: the interpolation
                // weight that names I (at most one of the two does), else 0
                for (int I = 0; I < nc; ++I)
                    for (int q = 0; q < 4; ++q) {
                        const int i = 2 * I - 1 + q;
                        double wd = 0.0;
                        float wfl = 0.f;
                        if (q < 3 && i >= 0 && i < n) {
                            const IpPk<double>& a = ipd[L.off[d] + i];
                            const IpPk<float>& b = ipf[L.off[d] + i];
                            wd = (a.ilo == I ? a.wlo : 0.0) + (a.ilo + 1 == I ? a.whi : 0.0);
                            wfl = (b.ilo == I ? b.wlo : 0.f) + (b.ilo + 1 == I ? b.whi : 0.f);
                        }
                        rwd[L.coff[d] + I].w[q] = wd;
                        rwf[L.coff[d] + I].w[q] = wfl;
                    }
            }
            CFP_CUDA(pool_malloc(&L.ip64, sizeof(IpPk<double>) * tot, c->stream));
            CFP_CUDA(pool_malloc(&L.ip32, sizeof(IpPk<float>) * tot, c->stream));
            CFP_CUDA(pool_malloc(&L.rw64, sizeof(RwPk<double>) * ctot, c->stream));
            CFP_CUDA(pool_malloc(&L.rw32, sizeof(RwPk<float>) * ctot, c->stream));
            CFP_CUDA(cudaMemcpyAsync(L.ip64, ipd.data(), sizeof(IpPk<double>) * tot, cudaMemcpyHostToDevice, c->stream));
            CFP_CUDA(cudaMemcpyAsync(L.ip32, ipf.data(), sizeof(IpPk<float>) * tot, cudaMemcpyHostToDevice, c->stream));
            CFP_CUDA(cudaMemcpyAsync(L.rw64, rwd.data(), sizeof(RwPk<double>) * ctot, cudaMemcpyHostToDevice, c->stream));
            CFP_CUDA(cudaMemcpyAsync(L.rw32, rwf.data(), sizeof(RwPk<float>) * ctot, cudaMemcpyHostToDevice, c->stream));
        }
        L.hp = ((L.n[0] + 1) / 2 + 15) / 16 * 16;
        L.Nh = (int64_t)L.hp * L.n[1] * L.n[2];
        if (L.Nh >= (int64_t(1) << 31))
            return fail(CFP_EINVAL, "grid too large for the multigrid preconditioner (2^31 entries per colour)");
        const uint8_t* nat = c->type;
        if (l > 0) {
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
            CFP_CUDA(pool_malloc(&L.coef64, sizeof(double) * nco, c->stream));
            CFP_CUDA(pool_malloc(&L.coef32, sizeof(float) * nco, c->stream));
            CFP_CUDA(cudaMemcpyAsync(L.coef64, cf.data(), sizeof(double) * nco, cudaMemcpyHostToDevice, c->stream));
            CFP_CUDA(cudaMemcpyAsync(L.coef32, cf32.data(), sizeof(float) * nco, cudaMemcpyHostToDevice, c->stream));
            CFP_CUDA(pool_malloc(&L.type, (size_t)L.N, c->stream));
            const MgLevel& Fp = c->mg[l - 1];
            const uint8_t* ft = l == 1 ? c->type : Fp.type;
            k_inject_type<<<flat_blocks(L.N), 256, 0, c->stream>>>(ft, Fp.n[0], Fp.n[1], Fp.n[2], L.type, L.n[0],
                                                                   L.n[1], L.n[2]);
            CFP_CUDA(cudaGetLastError());
            nat = L.type;
        }
        CFP_CUDA(pool_malloc(&L.stype, (size_t)(2 * L.Nh), c->stream));
        k_split_type<<<flat_blocks(2 * L.Nh), 256, 0, c->stream>>>(nat, L.n[0], L.n[1], L.n[2], L.hp, L.stype);
        CFP_CUDA(cudaGetLastError());
        // packed K coefficients of the level, both precisions
        const int ntot = L.n[0] + L.n[1] + L.n[2];
        CFP_CUDA(pool_malloc(&L.pk64, sizeof(PkD) * ntot, c->stream));
        CFP_CUDA(pool_malloc(&L.pk32, sizeof(float4) * ntot, c->stream));
        const unsigned pb = (unsigned)((ntot + 127) / 128);
        k_pack_coefs<double><<<pb, 128, 0, c->stream>>>(level_grid_view<double>(c, L, l), static_cast<PkD*>(L.pk64));
        k_pack_coefs<float><<<pb, 128, 0, c->stream>>>(level_grid_view<float>(c, L, l), static_cast<float4*>(L.pk32));
        CFP_CUDA(cudaGetLastError());
    }
    // the fine level's irregular nodes split by colour in ascending natural
    // index, with per-row starts, for the follow-ups and the fused pass
    MgLevel& L0 = c->mg[0];
    if (c->n_irr > 0) {
        const int64_t nrows = (int64_t)L0.n[1] * L0.n[2];
        const int nb = (int)((c->n_irr + kFixBlock - 1) / kFixBlock);
        const unsigned hs0 = (unsigned)((int64_t)L0.hp * L0.n[1]);
        int* red_count = nullptr;
        CFP_CUDA(pool_malloc(&L0.fix, sizeof(FixPt) * 2 * c->n_irr, c->stream));
        CFP_CUDA(pool_malloc(&L0.fixrows, sizeof(int32_t) * 2 * (nrows + 1), c->stream));
        CFP_CUDA(pool_malloc(&red_count, sizeof(int) * nb, c->stream));
        int* count = reinterpret_cast<int*>(c->dtotal + 5);  // scratch of the context
        k_fix_count<<<nb, kFixBlock, 0, c->stream>>>(c->irr_lin, c->n_irr, L0.n[0], L0.n[1], red_count);
        k_fix_place<<<nb, kFixBlock, 0, c->stream>>>(c->irr_lin, c->n_irr, L0.n[0], L0.n[1], L0.hp, hs0, red_count,
                                                     static_cast<FixPt*>(L0.fix), count);
        CFP_CUDA(cudaGetLastError());
        pool_free(red_count, c->stream);
        int hc[2] = {0, 0};
        CFP_CUDA(cudaMemcpyAsync(hc, count, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CFP_CUDA(cudaStreamSynchronize(c->stream));
        L0.nfix[0] = hc[0];
        L0.nfix[1] = hc[1];
        for (int col = 0; col < 2; ++col)
            k_fix_rows<<<flat_blocks(nrows + 1), 256, 0, c->stream>>>(
                static_cast<const FixPt*>(L0.fix) + col * c->n_irr, hc[col], L0.n[0], nrows,
                L0.fixrows + col * (nrows + 1));
        CFP_CUDA(cudaGetLastError());
    }
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

}  // namespace

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library does not link libcuda)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 3D map (x = entry in a row of hp, y = row, z = plane) of one colour array
// with a box of bx x by x 1 elements; out-of-array elements read as zero
cfp_status tile_map(CUtensorMap* m, CUtensorMapDataType dt, int esize, const void* base, const MgLevel& L, int bx,
                    int by) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(CFP_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t dims[3] = {(cuuint64_t)L.hp, (cuuint64_t)L.n[1], (cuuint64_t)L.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)L.hp * esize, (cuuint64_t)L.hp * L.n[1] * esize};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_64B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CFP_ECUDA, "cuTensorMapEncodeTiled failed for a multigrid level");
    return CFP_OK;
}

// maps and persistent grids of the TMA passes on the levels wide enough
cfp_status pair_occupancy(int* per) {
    CFP_CUDA(cudaFuncSetAttribute(k_sweep_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmem));
    CFP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_sweep_pair, kPairThreads, kPairSmem));
    return CFP_OK;
}

template <int KIND>
cfp_status tma_occupancy(int* per) {
    static_assert(tma_smem(KIND) <= 227 * 1024, "shared memory per CTA");
    CFP_CUDA(cudaFuncSetAttribute(k_sweep_tma<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, tma_smem(KIND)));
    CFP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, k_sweep_tma<KIND>, kTmaThreads, tma_smem(KIND)));
    return CFP_OK;
}

cfp_status setup_tma(cfp_ctx* c) {
    int per[3] = {0, 0, 0}, per_pair = 0, nsm = 0;
    CFP_TRY(pair_occupancy(&per_pair));
    CFP_TRY(tma_occupancy<0>(&per[0]));
    CFP_TRY(tma_occupancy<1>(&per[1]));
    CFP_TRY(tma_occupancy<2>(&per[2]));
    CFP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    for (MgLevel& L : c->mg) {
        L.tma = 0;
        if (L.n[0] / 2 < kTmaMinPairs || per[0] < 1 || per[1] < 1 || per[2] < 1) continue;
        for (int col = 0; col < 2; ++col) {
            const float* e_oth = L.s32 + (int64_t)(1 - col) * L.Nh;
            const float* b_own = L.s32 + (int64_t)(2 + col) * L.Nh;
            CFP_TRY(tile_map(&L.tm32[2 * col], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, e_oth, L, kTmaOX, kTmaRows + 2));
            CFP_TRY(tile_map(&L.tm32[2 * col + 1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b_own, L, kTmaTX, kTmaRows));
        }
        CFP_TRY(tile_map(&L.tm32[4], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.s32, L, kTmaTX, kTmaRows));  // red e
        const float* red2 = L.s32 + 5 * L.Nh;  // the second red array
        CFP_TRY(tile_map(&L.tmalt[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, red2, L, kTmaOX, kTmaRows + 2));
        CFP_TRY(tile_map(&L.tmalt[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, red2, L, kTmaTX, kTmaRows));
        CFP_TRY(tile_map(&L.tmp[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.s32, L, kPairOX, kPairYRows));
        CFP_TRY(tile_map(&L.tmp[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, red2, L, kPairOX, kPairYRows));
        CFP_TRY(tile_map(&L.tmp[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.s32 + 3 * L.Nh, L, kPairOX, kPairXRows));
        CFP_TRY(tile_map(&L.tmp[3], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L.s32 + 2 * L.Nh, L, kPairTX, kTmaRows));
        const int64_t tiles = (int64_t)((L.n[0] / 2 + kTmaTX - 1) / kTmaTX) * ((L.n[1] - 2 + kTmaRows - 1) / kTmaRows) *
                              ((L.n[2] - 2 + kTmaPlanes - 1) / kTmaPlanes);
        for (int q = 0; q < 3; ++q) L.tma_grid[q] = (int)std::min<int64_t>(tiles, (int64_t)per[q] * nsm);
        const int64_t ptiles = (int64_t)((L.n[0] / 2 + kPairTX - 1) / kPairTX) *
                               ((L.n[1] - 2 + kTmaRows - 1) / kTmaRows) * ((L.n[2] - 2 + kTmaPlanes - 1) / kTmaPlanes);
        L.pair_grid = (int)std::min<int64_t>(ptiles, (int64_t)per_pair * nsm);
        L.pair = per_pair >= 1;
        L.tma = 1;
    }
    return CFP_OK;
}

}  // namespace

// Build the hierarchy if needed and the split vectors of precision `prec`
// (0: FP64, 1: FP32), zero-filled: entries that are never written (the
// non-unknowns, the box, the black residuals) must read as zero.
cfp_status ensure_mg(cfp_ctx* c, int prec) {
    if (c->mg.empty()) {
        const cfp_status st = build_levels(c);
        if (st != CFP_OK) {
            free_mg(c);
            return st;
        }
    }
    bool fresh32 = false;
    for (MgLevel& L : c->mg) {
        const size_t n = (size_t)kSplitVecs * L.Nh;
        if (prec == 0 && !L.s64) {
            CFP_CUDA(pool_malloc(&L.s64, sizeof(double) * n, c->stream));
            CFP_CUDA(cudaMemsetAsync(L.s64, 0, sizeof(double) * n, c->stream));
        }
        if (prec == 1 && !L.s32) {  // + the second red array of the fused pass
            CFP_CUDA(pool_malloc(&L.s32, sizeof(float) * (n + L.Nh), c->stream));
            CFP_CUDA(cudaMemsetAsync(L.s32, 0, sizeof(float) * (n + L.Nh), c->stream));
            k_mark_b<<<flat_blocks(2 * L.Nh), 256, 0, c->stream>>>(L.stype, L.s32 + 2 * L.Nh, 2 * L.Nh);
            CFP_CUDA(cudaGetLastError());
            fresh32 = true;
        }
    }
    if (fresh32) CFP_TRY(setup_tma(c));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

// phi = V(rho): one V-cycle from zero on the level hierarchy.  phi is written
// at every interior node of the interior rows (zero at the non-unknowns).
// level l + 1's correction onto level l's black nodes: one thread per coarse
// cell (k_prolong_cell) with the fast kernels, else one per fine pair
template <class T>
void launch_prolong(cfp_ctx* c, int l, const SLev<T>& F, const SLev<T>& C, cudaStream_t s) {
    if (c->mg_tma) {
        const MgLevel& Cn = c->mg[l + 1];
        const dim3 g((unsigned)((Cn.n[0] - 1 + 127) / 128), (unsigned)(Cn.n[1] - 1), (unsigned)(Cn.n[2] - 1));
        k_prolong_cell<T><<<g, 128, 0, s>>>(transfer<T>(c->mg[l]), F, C);
    } else {
        k_prolong_split<T><<<plane_grid(c->mg[l].n), plane_block(c->mg[l].n), 0, s>>>(transfer<T>(c->mg[l]), F, C);
    }
}

template <class T>
void launch_precond_mg(cfp_ctx* c, const T* rho, T* phi, cudaStream_t s) {
    reset_red(c);
    const int nl = (int)c->mg.size();
    const int nu = std::max(1, c->mg_smooth);    // sweeps before the coarse correction
    const int npost = std::max(1, c->mg_post);   // and after it
    const Side<T> S0 = side_view<T>(c);
    const Side<T> Sc = Side<T>{nullptr, nullptr, nullptr, nullptr, nullptr};
    if (nl == 1) {
        smooth<T>(c, 0, S0, 16, 2, 3, rho, phi, s);
        return;
    }
    // downward leg: smooth from zero, red residual, restrict to b of l + 1
    for (int l = 0; l < nl - 1; ++l) {
        const Side<T>& S = l == 0 ? S0 : Sc;
        smooth<T>(c, l, S, nu, l == 0 ? 2 : 1, 0, rho, phi, s);
        const SLev<T> F = slev<T>(c, l), C = slev<T>(c, l + 1);
        if (!sweep_tma(c, l, F, 1, 0, phi, s)) k_resid_split<T><<<plane_grid(c->mg[l].n), plane_block(c->mg[l].n), 0, s>>>(F);
        if (l == 0 && c->mg[0].nfix[0] > 0) {
            const int64_t n = c->mg[0].nfix[0];
            k_resid_fix<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, s>>>(
                F, S, static_cast<const FixPt*>(c->mg[0].fix), n);
            c->launches += 1;
        }
        const MgLevel& Cn = c->mg[l + 1];
        const dim3 gr((unsigned)((Cn.n[0] - 2 + 127) / 128), (unsigned)(Cn.n[1] - 2), (unsigned)(Cn.n[2] - 2));
        k_restrict_split<T><<<gr, 128, 0, s>>>(transfer<T>(c->mg[l]), F, C);
        c->launches += 2;
    }
    smooth<T>(c, nl - 1, Sc, 16, 1, 0, rho, phi, s);  // coarsest level
    // upward leg: black coarse correction, smooth; the last half-sweep of the
    // fine level writes phi
    for (int l = nl - 2; l >= 0; --l) {
        const SLev<T> F = slev<T>(c, l), C = slev<T>(c, l + 1);
        launch_prolong<T>(c, l, F, C, s);
        c->launches += 1;
        smooth<T>(c, l, l == 0 ? S0 : Sc, npost, 0, l == 0 ? 3 : 0, rho, phi, s);
    }
}

template <class T>
void launch_rbgs_split(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s) {
    reset_red(c);
    smooth<T>(c, 0, side_view<T>(c), sweeps, 2, 3, rho, phi, s);
}

template <class T>
void launch_mg_half_sweep(cfp_ctx* c, cudaStream_t s) {
    reset_red(c);
    const SLev<T> L = slev<T>(c, 0);
    half_sweep<T>(c, 0, L, side_view<T>(c), 0, 0, (const T*)nullptr, (T*)nullptr, s);
}

// one transfer between the fine level and the next: restrict (the red
// residual to b of level 1) or prolong (level 1's correction to the fine
// black nodes), as in the V-cycle; false without a second level
template <class T>
bool launch_mg_transfer(cfp_ctx* c, bool prolong, cudaStream_t s) {
    if (c->mg.size() < 2) return false;
    reset_red(c);
    const SLev<T> F = slev<T>(c, 0), C = slev<T>(c, 1);
    if (prolong) {
        launch_prolong<T>(c, 0, F, C, s);
    } else {
        const MgLevel& Cn = c->mg[1];
        const dim3 gr((unsigned)((Cn.n[0] - 2 + 127) / 128), (unsigned)(Cn.n[1] - 2), (unsigned)(Cn.n[2] - 2));
        k_restrict_split<T><<<gr, 128, 0, s>>>(transfer<T>(c->mg[0]), F, C);
    }
    c->launches += 1;
    return true;
}

template <class T>
bool launch_mg_pair(cfp_ctx* c, cudaStream_t s) {
    reset_red(c);
    const bool ok = sweep_pair(c, 0, side_view<T>(c), s, true);
    reset_red(c);  // timing only: the next pass reads the split array again
    return ok;
}

cfp_status diag_bounded_wait(cfp_ctx* c) {
    k_wait_diag<<<1, 32, 0, c->stream>>>(c->dwait);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return check_waits(c);
}

template void launch_precond_mg<double>(cfp_ctx*, const double*, double*, cudaStream_t);
template void launch_precond_mg<float>(cfp_ctx*, const float*, float*, cudaStream_t);
template void launch_mg_half_sweep<double>(cfp_ctx*, cudaStream_t);
template void launch_rbgs_split<double>(cfp_ctx*, int, const double*, double*, cudaStream_t);
template void launch_rbgs_split<float>(cfp_ctx*, int, const float*, float*, cudaStream_t);
template void launch_mg_half_sweep<float>(cfp_ctx*, cudaStream_t);
template bool launch_mg_transfer<double>(cfp_ctx*, bool, cudaStream_t);
template bool launch_mg_transfer<float>(cfp_ctx*, bool, cudaStream_t);
template bool launch_mg_pair<double>(cfp_ctx*, cudaStream_t);
template bool launch_mg_pair<float>(cfp_ctx*, cudaStream_t);

}  // namespace cfp
