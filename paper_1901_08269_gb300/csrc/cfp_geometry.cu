// Point classification, IBI location and the irregular-point side list.
//
// Sec. 2: a node is solid if it lies inside a body (phi <= 0; box nodes are
// Dirichlet nodes whatever phi says), irregular if it is an interior fluid
// node with a solid node among its 26 neighbours, regular otherwise.  IBI
// points are where a grid line between a fluid node and a solid axis
// neighbour crosses Gamma.  Secs. 2.2-2.3 replace, at each irregular point,
// the RHS operator of every grid line of its 3x3x3 block that has a solid
// node by a moment-matched operator (Eqs. mod1-mat4, M, mod2_case2,
// mod2_case22); Sec. 3.3 gives the Shortley-Weller rows of K (Eqs.
// 2ndorder_xx, 2ndorder_coef_mod, A7_mod).
//
// The level set is evaluated with explicitly rounded operations (no
// contraction) so that the classification is reproducible bit for bit; an
// FP32 evaluation with a bound on its rounding decides the sign wherever the
// bound can tell, which gives the same bits with a fraction of the FP64 work.
#include <math.h>

#include <algorithm>

#include "cfp_internal.cuh"

namespace cfp {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t lin3(int i, int j, int k, int nx, int ny) {
    return (int64_t)i + (int64_t)nx * ((int64_t)j + (int64_t)ny * k);
}

// ---------------------------------------------------------------- level set
__device__ double body_phi(const cfp_body& b, double x, double y, double z) {
    const double d0 = __dsub_rn(x, b.c[0]);
    const double d1 = __dsub_rn(y, b.c[1]);
    const double d2 = __dsub_rn(z, b.c[2]);
    const double* R = b.R;
    const double q0 = __dadd_rn(__dadd_rn(__dmul_rn(R[0], d0), __dmul_rn(R[3], d1)), __dmul_rn(R[6], d2));
    const double q1 = __dadd_rn(__dadd_rn(__dmul_rn(R[1], d0), __dmul_rn(R[4], d1)), __dmul_rn(R[7], d2));
    const double q2 = __dadd_rn(__dadd_rn(__dmul_rn(R[2], d0), __dmul_rn(R[5], d1)), __dmul_rn(R[8], d2));
    if (b.kind == CFP_SPHERE) {
        const double s = __dadd_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)), __dmul_rn(q2, q2));
        return __dsub_rn(s, __dmul_rn(b.p[0], b.p[0]));
    }
    if (b.kind == CFP_ELLIPSOID) {
        const double e0 = __ddiv_rn(q0, b.p[0]);
        const double e1 = __ddiv_rn(q1, b.p[1]);
        const double e2 = __ddiv_rn(q2, b.p[2]);
        const double s = __dadd_rn(__dadd_rn(__dmul_rn(e0, e0), __dmul_rn(e1, e1)), __dmul_rn(e2, e2));
        return __dsub_rn(s, 1.0);
    }
    const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(q0, q0), __dmul_rn(q1, q1)));
    const double s = __dsub_rn(rho, b.p[0]);
    return __dsub_rn(__dadd_rn(__dmul_rn(s, s), __dmul_rn(q2, q2)), __dmul_rn(b.p[1], b.p[1]));
}

__device__ __forceinline__ double edge_pos(double xa, double xb, double t) {
    return __dadd_rn(__dmul_rn(__dsub_rn(1.0, t), xa), __dmul_rn(t, xb));
}

struct GeoArgs {
    const double* X[3];
    const cfp_body* bodies;
    const Body32* b32;     // per body: FP32 copy (certified sign, bounding-sphere threshold)
    int nb, inside;
    int n[3];
};

constexpr float kU32 = 5.9604645e-8f;  // 2^-24, the unit roundoff of FP32

// The sign of body b's level set at a point from an FP32 evaluation: -1 or
// +1 where the FP32 value lies farther from zero than twice a bound on its
// rounding error (the factor covers the bound's own FP32 rounding and
// body_phi's FP64 one, both far smaller), so that body_phi has that sign;
// 0 where only body_phi can tell.  With u = 2^-24, A_j = |x_j| + |c_j|
// and W_i = sum_j |R_ji| A_j (>= |q_i|; q_i's error is at most 6.01 u W_i):
//   sphere     |phi32 - phi| <= 16.1 u sum W_i^2 + 4.01 u p^2;
//   ellipsoid  with V_i = W_i / p_i: <= 20.1 u sum V_i^2 + 1.01 u;
//   torus      rho's error E_rho <= 14.05 u (W_0^2 + W_1^2) / rho32 + u rho32,
//              s = rho - R's E_s <= E_rho + u (rho32 + 2 R), S = |s32| + E_s:
//              <= 2 E_s S + 3.01 u S^2 + 15.05 u W_2^2 + 4.01 u r^2.
__device__ int body_sign32(const Body32& b, float x, float y, float z) {
    const float d0 = __fsub_rn(x, b.c[0]), d1 = __fsub_rn(y, b.c[1]), d2 = __fsub_rn(z, b.c[2]);
    const float a0 = fabsf(x) + fabsf(b.c[0]), a1 = fabsf(y) + fabsf(b.c[1]), a2 = fabsf(z) + fabsf(b.c[2]);
    const float* R = b.R;
    const float q0 = __fadd_rn(__fadd_rn(__fmul_rn(R[0], d0), __fmul_rn(R[3], d1)), __fmul_rn(R[6], d2));
    const float q1 = __fadd_rn(__fadd_rn(__fmul_rn(R[1], d0), __fmul_rn(R[4], d1)), __fmul_rn(R[7], d2));
    const float q2 = __fadd_rn(__fadd_rn(__fmul_rn(R[2], d0), __fmul_rn(R[5], d1)), __fmul_rn(R[8], d2));
    const float W0 = fabsf(R[0]) * a0 + fabsf(R[3]) * a1 + fabsf(R[6]) * a2;
    const float W1 = fabsf(R[1]) * a0 + fabsf(R[4]) * a1 + fabsf(R[7]) * a2;
    const float W2 = fabsf(R[2]) * a0 + fabsf(R[5]) * a1 + fabsf(R[8]) * a2;
    float phi, m;
    if (b.kind == CFP_SPHERE) {
        const float s = __fadd_rn(__fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1)), __fmul_rn(q2, q2));
        const float pp = __fmul_rn(b.p[0], b.p[0]);
        phi = __fsub_rn(s, pp);
        m = 2.f * kU32 * (16.1f * (W0 * W0 + W1 * W1 + W2 * W2) + 4.01f * pp);
    } else if (b.kind == CFP_ELLIPSOID) {
        const float e0 = __fmul_rn(q0, b.ip[0]), e1 = __fmul_rn(q1, b.ip[1]), e2 = __fmul_rn(q2, b.ip[2]);
        const float s = __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
        phi = __fsub_rn(s, 1.f);
        const float V0 = W0 * b.ip[0], V1 = W1 * b.ip[1], V2 = W2 * b.ip[2];
        m = 2.f * kU32 * (20.1f * (V0 * V0 + V1 * V1 + V2 * V2) + 1.01f);
    } else {
        const float t = __fadd_rn(__fmul_rn(q0, q0), __fmul_rn(q1, q1));
        const float rho = __fsqrt_rn(t);
        if (!(rho > 0.f)) return 0;  // on the torus axis: no bound on rho's error
        const float s = __fsub_rn(rho, b.p[0]);
        phi = __fsub_rn(__fadd_rn(__fmul_rn(s, s), __fmul_rn(q2, q2)), __fmul_rn(b.p[1], b.p[1]));
        const float er = 14.05f * kU32 * (W0 * W0 + W1 * W1) / rho + kU32 * rho;
        const float es = er + kU32 * (rho + 2.f * b.p[0]);
        const float S = fabsf(s) + es;
        m = 2.f * (2.f * es * S + kU32 * (3.01f * S * S + 15.05f * W2 * W2 + 4.01f * b.p[1] * b.p[1]));
    }
    return phi > m ? 1 : (phi < -m ? -1 : 0);
}

// Whether a point is solid (fluid outside the bodies: some body's level
// set <= 0; fluid inside: every body's >= 0).  Each body's sign comes from
// body_sign32 where it can tell, else from body_phi, so it is the sign
// body_phi gives.  Outside mode, a body is looked at only when the point may
// lie inside its bounding sphere (outside it phi > 0 holds with a margin far
// above rounding); that test runs in FP32 against a threshold above the
// FP32 squared distance of every point within the sphere (set on the host
// from a bound on the rounding), so it skips only points outside.
__device__ bool node_solid(const GeoArgs& g, double x, double y, double z) {
    const float xf = (float)x, yf = (float)y, zf = (float)z;
    for (int m = 0; m < g.nb; ++m) {
        const Body32& b = g.b32[m];
        if (!g.inside) {
            const float dx = __fsub_rn(xf, b.c[0]), dy = __fsub_rn(yf, b.c[1]), dz = __fsub_rn(zf, b.c[2]);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            if (d2 > b.thr) continue;
        }
        int sg = body_sign32(b, xf, yf, zf);
        if (sg == 0) {
            const double v = body_phi(g.bodies[m], x, y, z);
            sg = g.inside ? (v < 0.0 ? -1 : 1) : (v <= 0.0 ? -1 : 1);
        }
        if (sg < 0) return !g.inside;  // outside mode: solid; inside mode: fluid
    }
    return g.inside;
}

// ------------------------------------------------------------ classification
__global__ void k_classify_solid(GeoArgs g, uint8_t* type, int64_t N) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
         l += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(l % nx);
        const int j = (int)((l / nx) % ny);
        const int k = (int)(l / ((int64_t)nx * ny));
        uint8_t t;
        if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1) {
            t = CFP_BOUNDARY;
        } else {
            t = node_solid(g, g.X[0][i], g.X[1][j], g.X[2][k]) ? CFP_SOLID : CFP_REGULAR;
        }
        type[l] = t;
    }
}

// A regular interior node turns irregular if one of its 26 neighbours is
// solid.  Each thread owns node i of row j and marches the planes of one z
// chunk: per plane it loads the types of rows j - 1, j, j + 1 at i, and the
// warp ORs the solid flags with its x neighbours (lanes i - 1, i + 1) by
// shuffles, so the 3 x 3 (x, y) dilation of a plane costs three loads per
// node; three consecutive planes' dilations decide the plane between them.
// A warp covers nodes i0 .. i0 + 31 and marks i0 + 1 .. i0 + 30 (its edge
// lanes only feed their neighbours).  Only the solid flags are read, and a
// node turns irregular only from regular, so the in-place update does not
// race.
constexpr int kIrrPlanes = 16;  // planes per thread
constexpr int kIrrWarps = 8;    // warps per block

__global__ void __launch_bounds__(32 * kIrrWarps) k_classify_irregular(uint8_t* type, int nx, int ny, int nz) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * kIrrWarps + (threadIdx.x >> 5)) * 30 + lane;
    const int j = 1 + blockIdx.y;
    const int k0 = 1 + blockIdx.z * kIrrPlanes, k1 = min(k0 + kIrrPlanes, nz - 1);
    const bool inx = i < nx;
    const bool mine = lane >= 1 && lane <= 30 && i <= nx - 2;
    const int64_t row = (int64_t)nx;
    uint8_t* col = type + ((int64_t)j * nx + (inx ? i : 0));  // node (i, j) of plane 0
    const int64_t pl = (int64_t)nx * ny;
    // the dilated solid flag of plane k at (i, j), and the node's own type
    auto dil = [&](int k, uint8_t& own) -> bool {
        bool s = false;
        own = CFP_SOLID;
        if (inx) {
            const uint8_t* c = col + k * pl;
            own = c[0];
            s = c[-row] == CFP_SOLID || own == CFP_SOLID || c[row] == CFP_SOLID;
        }
        const unsigned b = s ? 1u : 0u;
        return (b | __shfl_up_sync(0xffffffffu, b, 1) | __shfl_down_sync(0xffffffffu, b, 1)) != 0u;
    };
    uint8_t tm, t0, tp;
    bool dm = dil(k0 - 1, tm), d0 = dil(k0, t0);
    for (int k = k0; k < k1; ++k) {
        const bool dp = dil(k + 1, tp);
        if (mine && t0 == CFP_REGULAR && (dm || d0 || dp)) col[k * pl] = CFP_IRREGULAR;
        dm = d0;
        d0 = dp;
        t0 = tp;
    }
}

// -------------------------------------------------------------------- scans
// Deterministic exclusive scan of per-item counts: per-chunk sums, a
// single-block scan of the chunk sums, then a per-chunk scan and scatter.
__device__ int block_excl_scan(int v, int* total) {
    __shared__ int warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        int t = lane < nw ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    const int before = wid ? warp_tot[wid - 1] : 0;
    if (total) *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

struct FlagIrregular {
    const uint8_t* type;
    __device__ int operator()(int64_t i) const { return type[i] == CFP_IRREGULAR; }
};
struct FetchInt {
    const int* a;
    __device__ int operator()(int64_t i) const { return a[i]; }
};
struct SinkSlots {
    int32_t* slot;
    int32_t* irr_lin;
    __device__ void operator()(int64_t i, int off, int v) const {
        slot[i] = v ? off : -1;
        if (v) irr_lin[off] = (int32_t)i;
    }
};
struct SinkOffsets {
    int32_t* out;
    __device__ void operator()(int64_t i, int off, int) const { out[i] = off; }
};

template <class F>
__global__ void k_scan_reduce(F f, int64_t n, int* bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    int s = 0;
    for (int q = threadIdx.x; q < kScanChunk; q += kScanThreads) {
        const int64_t i = base + q;
        if (i < n) s += f(i);
    }
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_blocks(int* bsum, int nb, long long* total) {
    __shared__ long long carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int tot;
        const int ex = block_excl_scan(v, &tot);
        const long long carry = carry_s;
        if (i < nb) bsum[i] = (int)(carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

template <class F, class S>
__global__ void k_scan_scatter(F f, S sink, int64_t n, const int* boff) {
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = (base + q < n) ? f(base + q) : 0;
        s += v[q];
    }
    int off = boff[blockIdx.x] + block_excl_scan(s, nullptr);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < n) {
            sink(base + q, off, v[q]);
            off += v[q];
        }
    }
}

template <class F, class S>
cfp_status scan(cfp_ctx* c, F f, S sink, int64_t n, long long* dtotal, long long* htotal) {
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (nb > c->scan_cap) {
        pool_free(c->scan_bsum, c->stream);
        c->scan_bsum = nullptr;
        CFP_CUDA(pool_malloc(&c->scan_bsum, sizeof(int) * std::max<int64_t>(nb, 1), c->stream));
        c->scan_cap = nb;
    }
    if (nb > 0) {
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(f, n, c->scan_bsum);
        k_scan_blocks<<<1, kScanThreads, 0, c->stream>>>(c->scan_bsum, (int)nb, dtotal);
        k_scan_scatter<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(f, sink, n, c->scan_bsum);
        c->launches += 3;
    } else {
        CFP_CUDA(cudaMemsetAsync(dtotal, 0, sizeof(long long), c->stream));
    }
    CFP_CUDA(cudaGetLastError());
    CFP_CUDA(cudaMemcpyAsync(htotal, dtotal, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    return CFP_OK;
}

// ------------------------------------------------------------------ IBIs
struct IrrArgs {
    const uint8_t* type;
    const int32_t* slot;
    const int32_t* irr_lin;
    int64_t n_irr;
    int n[3];
};

__device__ __forceinline__ int solid_axis_mask(const uint8_t* type, int64_t l, const int64_t st[3]) {
    int m = 0;
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int64_t nb = l + ((dir & 1) ? st[dir >> 1] : -st[dir >> 1]);
        if (type[nb] == CFP_SOLID) m |= 1 << dir;
    }
    return m;
}

__global__ void k_ibi_count(IrrArgs a, int* cnt) {
    const int64_t st[3] = {1, a.n[0], (int64_t)a.n[0] * a.n[1]};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < a.n_irr;
         s += (int64_t)gridDim.x * blockDim.x) {
        cnt[s] = __popc(solid_axis_mask(a.type, a.irr_lin[s], st));
    }
}

// Root of phi on the edge from fluid node A (t = 0) to solid node B (t = 1):
// scan t = 1/8 .. 7/8 for the first sign change seen from A, then 60
// bisection steps; the solid end of the last bracket is returned.  Only the
// sign of phi decides each step, so node_solid (which skips bodies whose
// bounding sphere excludes the point, those have phi > 0) gives the same
// decisions as the full union of the bodies.
__device__ double ibi_root(const GeoArgs& g, int d, const double pa[3], double xb) {
    double q[3] = {pa[0], pa[1], pa[2]};
    double lo = 0.0, hi = 1.0;
    for (int s = 1; s < 8; ++s) {
        const double ts = (double)s / 8.0;
        q[d] = edge_pos(pa[d], xb, ts);
        if (node_solid(g, q[0], q[1], q[2])) {
            hi = ts;
            break;
        }
        lo = ts;
    }
    for (int it = 0; it < 60; ++it) {
        const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
        q[d] = edge_pos(pa[d], xb, mid);
        if (!node_solid(g, q[0], q[1], q[2])) lo = mid;
        else hi = mid;
    }
    return hi;
}

// IBI m of the list comes from irregular slot src[m] >> 3 and direction
// src[m] & 7 (IBIs of a slot in direction order, from its offset ibi_off)
__global__ void k_ibi_map(IrrArgs a, const int32_t* ibi_off, int32_t* src) {
    const int64_t st[3] = {1, a.n[0], (int64_t)a.n[0] * a.n[1]};
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < a.n_irr;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int mask = solid_axis_mask(a.type, a.irr_lin[s], st);
        int m = ibi_off[s];
        for (int dir = 0; dir < 6; ++dir)
            if (mask & (1 << dir)) src[m++] = (int32_t)(s * 8 + dir);
    }
}

// one thread per IBI: its root and coordinates
__global__ void k_ibi_roots(IrrArgs a, GeoArgs g, const int32_t* src, int64_t n_ibi, double* xyz) {
    const int nx = a.n[0], ny = a.n[1];
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n_ibi;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int32_t code = src[m];
        const int64_t s = code >> 3;
        const int dir = code & 7;
        const int64_t l = a.irr_lin[s];
        const int idx[3] = {(int)(l % nx), (int)((l / nx) % ny), (int)(l / ((int64_t)nx * ny))};
        const double pa[3] = {g.X[0][idx[0]], g.X[1][idx[1]], g.X[2][idx[2]]};
        const int d = dir >> 1, sg = (dir & 1) ? 1 : -1;
        const double xb = g.X[d][idx[d] + sg];
        const double t = ibi_root(g, d, pa, xb);
        xyz[3 * m + 0] = pa[0];
        xyz[3 * m + 1] = pa[1];
        xyz[3 * m + 2] = pa[2];
        xyz[3 * m + d] = edge_pos(pa[d], xb, t);
    }
}

// ------------------------------------------------------------- side list
constexpr int kMaxRaw = 320;   // correction adds per row before merging (27 lines x <= 11)
constexpr int kMaxBib = 64;

// Correction adds of one row, appended in order to the row's slice of the
// global scratch (no merging here: k_side_merge merges them afterwards).
struct RawAcc {
    int n;
    int32_t* off;
    double* val;
    __device__ bool add(int o, double v) {
        if (n == kMaxRaw) return false;
        off[n] = o;
        val[n] = v;
        ++n;
        return true;
    }
};

// IBI weights of one row, appended to its scratch slice.
struct BibAcc {
    int n;
    int32_t* idx;
    double* val;
    __device__ bool add(int i, double v) {
        if (n == kMaxBib) return false;
        idx[n] = i;
        val[n] = v;
        ++n;
        return true;
    }
};

struct SideArgs {
    IrrArgs a;
    Axis<double> ax[3];
    const double* X[3];
    const int32_t* ibi_off;
    const double* ibi_xyz;
};

__device__ __forceinline__ double Lc(const Axis<double>& A, int m, int o) {
    return o < 0 ? A.a[m] : (o == 0 ? 1.0 : A.c[m]);
}
__device__ __forceinline__ double Rc(const Axis<double>& A, int m, int o) {
    return o < 0 ? A.ar[m] : (o == 0 ? A.br[m] : A.cr[m]);
}

// IBI index of the edge from interior fluid node l in direction dir
// (-x,+x,-y,+y,-z,+z), or -1 if that neighbour is not solid.
__device__ int ibi_index(const SideArgs& S, int64_t l, int dir) {
    const int64_t st[3] = {1, S.a.n[0], (int64_t)S.a.n[0] * S.a.n[1]};
    const int s = S.a.slot[l];
    if (s < 0) return -1;
    const int mask = solid_axis_mask(S.a.type, l, st);
    if (!(mask & (1 << dir))) return -1;
    return S.ibi_off[s] + __popc(mask & ((1 << dir) - 1));
}

// Moment matching of Eqs. mat1-mat4 (matrix M of Eq. M): c_n with
// sum_n c_n (xi_n - xe)^m = sum_s L_s m(m-1) (xs_s - xe)^(m-2), m < M,
// lengths scaled by hs, Gaussian elimination with partial pivoting.  The
// scaled distances are divided once per node and their powers built up
// row by row (FP64 division is costly on this GPU).  M is a template
// parameter and every loop is unrolled, so the matrix lives in registers
// (a runtime size or pivot index would put it in local memory); the pivot
// row is exchanged with predicated selects.
template <int M>
__device__ __forceinline__ bool moment_solve_m(const double* xi, double xe, int ns, const double* xs,
                                               const double* Ls, double hs, double* c) {
    double A[M][M + 1];
    double e[M], pw[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        e[q] = (xi[q] - xe) / hs;
        pw[q] = 1.0;
    }
    double es[3] = {0.0, 0.0, 0.0}, ps[3] = {1.0, 1.0, 1.0};
    for (int s = 0; s < ns; ++s) es[s] = (xs[s] - xe) / hs;
    const double ih2 = 1.0 / (hs * hs);
#pragma unroll
    for (int m = 0; m < M; ++m) {
#pragma unroll
        for (int q = 0; q < M; ++q) {
            A[m][q] = pw[q];
            pw[q] *= e[q];
        }
        double r = 0.0;
        if (m >= 2) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
                if (s < ns) {
                    r += Ls[s] * (double)(m * (m - 1)) * ps[s];
                    ps[s] *= es[s];
                }
        }
        A[m][M] = r * ih2;
    }
#pragma unroll
    for (int col = 0; col < M; ++col) {
        int piv = col;
        double best = fabs(A[col][col]);
#pragma unroll
        for (int r = col + 1; r < M; ++r)
            if (fabs(A[r][col]) > best) {
                best = fabs(A[r][col]);
                piv = r;
            }
        if (best == 0.0) return false;
#pragma unroll
        for (int r = col + 1; r < M; ++r)
            if (r == piv)
#pragma unroll
                for (int q = 0; q <= M; ++q) {
                    const double t = A[col][q];
                    A[col][q] = A[r][q];
                    A[r][q] = t;
                }
        const double ip = 1.0 / A[col][col];
#pragma unroll
        for (int r = col + 1; r < M; ++r) {
            const double f = A[r][col] * ip;
#pragma unroll
            for (int q = col; q <= M; ++q) A[r][q] -= f * A[col][q];
        }
    }
#pragma unroll
    for (int r = M - 1; r >= 0; --r) {
        double s = A[r][M];
#pragma unroll
        for (int q = r + 1; q < M; ++q) s -= A[r][q] * c[q];
        c[r] = s / A[r][r];
    }
    return true;
}

__device__ bool moment_solve(int M, const double* xi, double xe, int ns, const double* xs, const double* Ls,
                             double hs, double* c) {
    switch (M) {
        case 3: return moment_solve_m<3>(xi, xe, ns, xs, Ls, hs, c);
        case 4: return moment_solve_m<4>(xi, xe, ns, xs, Ls, hs, c);
        case 5: return moment_solve_m<5>(xi, xe, ns, xs, Ls, hs, c);
        case 6: return moment_solve_m<6>(xi, xe, ns, xs, Ls, hs, c);
        default: return false;
    }
}

// The modified operators of one line: the line's solid pattern `mask`
// (bit 2: node -1, bit 1: node 0, bit 0: node +1 solid) fixes each
// operator's expansion offset e, walk direction sg, walk length G (5 grid
// nodes for the six-point operators of Eqs. mod1-mod4, 4 for the five-point
// ones of Eqs. mod2_case2 / mod2_case22) and the surviving R nodes with their
// L weights (a, 1, c of the line's centre).
struct OpSpec {
    int e, sg, G, ns;
    int surv[2];
    double Ls[2];
};
__device__ __forceinline__ int line_nops(int mask) { return mask == 2 ? 2 : 1; }
__device__ __forceinline__ OpSpec op_spec(int mask, int k, double a, double c) {
    switch (mask) {
        case 1: return OpSpec{0, -1, 5, 2, {-1, 0}, {a, 1.0}};    // +1 solid (Eqs. mod1_top, mod1, mat1)
        case 4: return OpSpec{0, +1, 5, 2, {0, 1}, {1.0, c}};     // -1 solid (Eqs. mod3_top, mod3, mat3)
        case 3: return OpSpec{-1, -1, 5, 1, {-1, 0}, {a, 0.0}};   // 0 and +1 solid (Eqs. mod2_top, mod2, mat2)
        case 6: return OpSpec{1, +1, 5, 1, {1, 0}, {c, 0.0}};     // -1 and 0 solid (Eqs. mod4_top, mod4, mat4)
        case 2:                                                   // middle solid: Eqs. mod2_case2, mod2_case22
            return k == 0 ? OpSpec{-1, -1, 4, 1, {-1, 0}, {a, 0.0}} : OpSpec{1, +1, 4, 1, {1, 0}, {c, 0.0}};
        default: return OpSpec{0, -1, 5, 1, {0, 0}, {1.0, 0.0}};  // 5: fluid node between two solid nodes
    }
}

// One of the 27 lines of an irregular point's row (Eq. lhsrhs_xxyyzz_mod),
// L = 9 d + 3 (o1 + 1) + (o2 + 1): axis d, offsets o1, o2 along the two
// other axes; its weight w (the L coefficients across), its centre index
// vector `base`, the line centre's a and c, and its solid pattern.
struct Line {
    int d, m, mask;
    int base[3];
    int64_t bl;
    double w, a, c;
};
__device__ __forceinline__ void line_at(const SideArgs& S, const int idx[3], const int64_t st[3], int L, Line& ln) {
    const int d = L / 9, o1 = (L / 3) % 3 - 1, o2 = L % 3 - 1;
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    ln.d = d;
    ln.m = idx[d];
    ln.a = S.ax[d].a[ln.m];
    ln.c = S.ax[d].c[ln.m];
    ln.w = Lc(S.ax[t1], idx[t1], o1) * Lc(S.ax[t2], idx[t2], o2);
    ln.base[0] = idx[0];
    ln.base[1] = idx[1];
    ln.base[2] = idx[2];
    ln.base[t1] += o1;
    ln.base[t2] += o2;
    ln.bl = lin3(ln.base[0], ln.base[1], ln.base[2], S.a.n[0], S.a.n[1]);
    int mask = 0;
    for (int s = -1; s <= 1; ++s) mask = (mask << 1) | (S.a.type[ln.bl + s * st[d]] == CFP_SOLID);
    ln.mask = mask;
}

// The walk of one modified operator: from the expansion node e along sg over
// up to G grid nodes; a solid node met first closes the set with its edge's
// IBI; leaving the grid ends it at the box (fewer points, degenerate).  Its
// grid nodes (coordinates, offsets from the row's point) and IBIs, or an
// error detail.
struct OpWalk {
    int ng, nib, err;
    bool deg;
    double xi[7];
    int offs[6];
    int ib[2];
};
__device__ void op_walk(const SideArgs& S, const Line& ln, const OpSpec& o, int64_t lin, const int64_t st[3],
                        OpWalk& W) {
    const int d = ln.d, nd = S.a.n[d];
    W.ng = 0;
    W.nib = 0;
    W.err = 0;
    W.deg = false;
    int f[3] = {ln.base[0], ln.base[1], ln.base[2]};
    f[d] += o.e;
    const int64_t fl = lin3(f[0], f[1], f[2], S.a.n[0], S.a.n[1]);
    const uint8_t ft = S.a.type[fl];
    if (ft != CFP_REGULAR && ft != CFP_IRREGULAR) { W.err = DETAIL_BOXIBI; return; }
    W.ib[0] = ibi_index(S, fl, 2 * d + (o.sg > 0 ? 0 : 1));
    if (W.ib[0] < 0) { W.err = DETAIL_MISSINGIBI; return; }
    W.nib = 1;
    for (int q = 0; q < o.G; ++q) {
        int p[3] = {f[0], f[1], f[2]};
        p[d] += q * o.sg;
        if (p[d] < 0 || p[d] >= nd) break;
        const int64_t l = lin3(p[0], p[1], p[2], S.a.n[0], S.a.n[1]);
        if (S.a.type[l] == CFP_SOLID) {
            const int64_t pl = l - o.sg * st[d];
            const uint8_t pt = S.a.type[pl];
            if (pt != CFP_REGULAR && pt != CFP_IRREGULAR) { W.err = DETAIL_BOXIBI; return; }
            W.ib[W.nib] = ibi_index(S, pl, 2 * d + (o.sg > 0 ? 1 : 0));
            if (W.ib[W.nib] < 0) { W.err = DETAIL_MISSINGIBI; return; }
            ++W.nib;
            break;
        }
        W.xi[W.ng] = S.X[d][p[d]];
        W.offs[W.ng] = (int)(l - lin);
        ++W.ng;
    }
    if (W.ng + W.nib < 3) { W.err = DETAIL_FEWPOINTS; return; }
    W.deg = W.ng < o.G || W.nib > 1;
}

// An operator whose moments are still to be matched: the slot of its
// point, its line and operator index (code = 2 L + k), and where its
// correction adds and IBI weights go in the point's scratch slices.
struct SideTask {
    int slot, code, cpos, bpos;
};

// The first error of a row in the order of its lines, operators and steps:
// key (2 L + k) x 4 + step (0: the R subtraction overflows the slice; 1:
// the walk fails; 2: the moment matrix is singular; 3: the operator's adds
// overflow), times 16, plus the error detail.  The sequential order in which
// a row is built decides which error is reported.
__device__ __forceinline__ int side_err(int L, int k, int step, int detail) {
    return (((2 * L + k) * 4 + step) << 4) | detail;
}
constexpr int kSideNoErr = 0x7fffffff;

// Plans the row of every irregular point (one thread per point), walking its
// 27 lines in order up to its first error: the R subtraction of every line
// with a solid node (Eq. cor: minus the regular R operator at the line's
// fluid nodes) and the walk of its modified operator(s).  COUNT: only the
// number of operators; otherwise the R subtraction's adds are stored, each
// operator becomes a task at its place (task_off[s] onwards) with the
// positions of its adds, and the row's counts, first error and degenerate
// operators are kept for k_side_finish.
template <bool COUNT>
__global__ void __launch_bounds__(128) k_side_plan(SideArgs S, int* ntask, const int* task_off, SideTask* tasks,
                                                   int* ccount, int* bcount, int* ferr, int* ndegs, int32_t* toff,
                                                   double* tval) {
    const int nx = S.a.n[0], ny = S.a.n[1];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S.a.n_irr;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lin = S.a.irr_lin[s];
        const int idx[3] = {(int)(lin % nx), (int)((lin / nx) % ny), (int)(lin / ((int64_t)nx * ny))};
        const int64_t st[3] = {1, nx, (int64_t)nx * ny};
        int cn = 0, bn = 0, nt = 0, ndeg = 0, err = kSideNoErr;
        const int t0 = COUNT ? 0 : task_off[s];
        for (int L = 0; L < 27 && err == kSideNoErr; ++L) {
            Line ln;
            line_at(S, idx, st, L, ln);
            if (ln.mask == 0 || ln.mask == 7) continue;  // regular or dropped line
            for (int q = -1; q <= 1 && err == kSideNoErr; ++q)
                if (!((ln.mask >> (1 - q)) & 1)) {
                    if (cn == kMaxRaw) {
                        err = side_err(L, 0, 0, DETAIL_OVERFLOW);
                        break;
                    }
                    if (!COUNT) {
                        toff[s * kMaxRaw + cn] = (int32_t)(ln.bl + q * st[ln.d] - lin);
                        tval[s * kMaxRaw + cn] = -ln.w * Rc(S.ax[ln.d], ln.m, q);
                    }
                    ++cn;
                }
            for (int k = 0; k < line_nops(ln.mask) && err == kSideNoErr; ++k) {
                const OpSpec o = op_spec(ln.mask, k, ln.a, ln.c);
                OpWalk W;
                op_walk(S, ln, o, lin, st, W);
                if (W.err) {
                    err = side_err(L, k, 1, W.err);
                    break;
                }
                ndeg += W.deg ? 1 : 0;
                if (!COUNT) tasks[t0 + nt] = SideTask{(int)s, 2 * L + k, cn, bn};
                ++nt;
                cn += W.ng;
                bn += W.nib;
                // adds past the slice: the operator still runs, for a singular
                // matrix comes first, but stores nothing
                if (cn > kMaxRaw || bn > kMaxBib) err = side_err(L, k, 3, DETAIL_OVERFLOW);
            }
        }
        if (COUNT) {
            ntask[s] = nt;
        } else {
            ccount[s] = cn;
            bcount[s] = bn;
            ferr[s] = err;
            ndegs[s] = ndeg;
        }
    }
}

// One modified operator per thread: its walk again, the moment matching of
// Eqs. mat1-mat4 (matrix M of Eq. M), and its correction adds and IBI
// weights (script B of Eq. bc), scaled by the line's weight, at the places
// k_side_plan gave them.
__global__ void __launch_bounds__(64) k_side_solve(SideArgs S, const SideTask* tasks, int64_t ntasks, int* ferr,
                                                   int32_t* toff, double* tval, int32_t* tbidx, double* tbval) {
    const int nx = S.a.n[0], ny = S.a.n[1];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntasks;
         t += (int64_t)gridDim.x * blockDim.x) {
        const SideTask T = tasks[t];
        const int64_t s = T.slot;
        const int L = T.code >> 1, k = T.code & 1;
        const int64_t lin = S.a.irr_lin[s];
        const int idx[3] = {(int)(lin % nx), (int)((lin / nx) % ny), (int)(lin / ((int64_t)nx * ny))};
        const int64_t st[3] = {1, nx, (int64_t)nx * ny};
        Line ln;
        line_at(S, idx, st, L, ln);
        const OpSpec o = op_spec(ln.mask, k, ln.a, ln.c);
        OpWalk W;
        op_walk(S, ln, o, lin, st, W);
        const int d = ln.d, ng = W.ng, nib = W.nib, M = ng + nib;
        for (int q = 0; q < nib; ++q) W.xi[ng + q] = S.ibi_xyz[3 * (int64_t)W.ib[q] + d];
        const double xe = S.X[d][ln.base[d] + o.e];
        double xs[2];
        for (int q = 0; q < o.ns; ++q) xs[q] = S.X[d][ln.base[d] + o.surv[q]];
        double hs = 0.0;
        for (int q = 1; q < M; ++q) hs = fmax(hs, fabs(W.xi[q] - xe));
        double cc[7];
        if (!moment_solve(M, W.xi, xe, o.ns, xs, o.Ls, hs, cc)) {
            atomicMin(&ferr[s], side_err(L, k, 2, DETAIL_SINGULAR));
            continue;
        }
        if (T.cpos + ng > kMaxRaw || T.bpos + nib > kMaxBib) continue;
        for (int q = 0; q < ng; ++q) {
            toff[s * kMaxRaw + T.cpos + q] = W.offs[q];
            tval[s * kMaxRaw + T.cpos + q] = ln.w * cc[q];
        }
        for (int q = 0; q < nib; ++q) {
            tbidx[s * kMaxBib + T.bpos + q] = W.ib[q];
            tbval[s * kMaxBib + T.bpos + q] = ln.w * cc[ng + q];
        }
    }
}

__device__ void record_error(DevError* e, int code, int lin, int detail) {
    if (atomicCAS(&e->code, 0, code) == 0) {
        e->lin = lin;
        e->detail = detail;
    }
}

// Per irregular point: its first error (none: the counts stand and its
// degenerate operators are counted), and its Shortley-Weller row of K.
__global__ void k_side_finish(SideArgs S, int* ccount, int* bcount, const int* ferr, const int* ndegs,
                              double* krow, unsigned long long* ndeg, DevError* err) {
    const int nx = S.a.n[0], ny = S.a.n[1];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < S.a.n_irr;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lin = S.a.irr_lin[s];
        if (ferr[s] != kSideNoErr) {
            record_error(err, CFP_EGEOM, (int)lin, ferr[s] & 15);
            ccount[s] = 0;
            bcount[s] = 0;
            continue;
        }
        if (ndegs[s]) atomicAdd(ndeg, (unsigned long long)ndegs[s]);
        const int idx[3] = {(int)(lin % nx), (int)((lin / nx) % ny), (int)(lin / ((int64_t)nx * ny))};
        // Shortley-Weller row of K (Eqs. 2ndorder_coef_mod, A7_mod): the IBI
        // distance replaces the spacing on a solid side, whose term is dropped.
        double kr[7];
        kr[0] = 0.0;
        for (int d = 0; d < 3; ++d) {
            const int m = idx[d];
            const double xm = S.X[d][m];
            double fw = S.X[d][m + 1] - xm;
            double bw = xm - S.X[d][m - 1];
            const int im = ibi_index(S, lin, 2 * d);
            const int ip = ibi_index(S, lin, 2 * d + 1);
            if (im >= 0) bw = xm - S.ibi_xyz[3 * (int64_t)im + d];
            if (ip >= 0) fw = S.ibi_xyz[3 * (int64_t)ip + d] - xm;
            const double ca = 2.0 / (bw * (fw + bw));
            const double cb = -2.0 / (bw * fw);
            const double cc = 2.0 / (fw * (fw + bw));
            kr[0] += cb;
            kr[1 + 2 * d] = im >= 0 ? 0.0 : ca;
            kr[2 + 2 * d] = ip >= 0 ? 0.0 : cc;
        }
        for (int q = 0; q < 7; ++q) krow[7 * s + q] = kr[q];
    }
}

// Merges each row's correction adds in place, in their order: an offset
// seen before adds its value to that entry, a new offset opens the next
// entry (the order of first appearance).  One warp per row; lane 0 walks the
// adds through an open-addressing index in shared memory (kMergeSlots >
// kMaxRaw, so an empty slot always exists), then the warp writes the merged
// entries back to the front of the row's slice.
constexpr int kMergeWarps = 4;
constexpr int kMergeSlots = 512;

__global__ void __launch_bounds__(32 * kMergeWarps) k_side_merge(int64_t n_irr, int* ccount, int32_t* toff,
                                                                 double* tval) {
    __shared__ int32_t soff[kMergeWarps][kMaxRaw];
    __shared__ double sval[kMergeWarps][kMaxRaw];
    __shared__ int16_t sslot[kMergeWarps][kMergeSlots];
    __shared__ int smerged[kMergeWarps];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < n_irr; s += nwarps) {
        const int nraw = ccount[s];
        int32_t* off = toff + s * kMaxRaw;
        double* val = tval + s * kMaxRaw;
        for (int q = lane; q < kMergeSlots; q += 32) sslot[wl][q] = 0;
        __syncwarp();
        if (lane == 0) {
            int n = 0;
            for (int e = 0; e < nraw; ++e) {
                const int o = off[e];
                const double v = val[e];
                unsigned h = ((unsigned)o * 2654435761u) >> 23;  // 9 bits
                bool merged = false;
                for (int probe = 0; probe < kMergeSlots; ++probe) {
                    const int x = sslot[wl][h];
                    if (x == 0) break;
                    if (soff[wl][x - 1] == o) {
                        sval[wl][x - 1] += v;
                        merged = true;
                        break;
                    }
                    h = (h + 1) & (kMergeSlots - 1);
                }
                if (!merged) {
                    soff[wl][n] = o;
                    sval[wl][n] = v;
                    sslot[wl][h] = (int16_t)(n + 1);
                    ++n;
                }
            }
            smerged[wl] = n;
        }
        __syncwarp();
        const int n = smerged[wl];
        for (int q = lane; q < n; q += 32) {
            off[q] = soff[wl][q];
            val[q] = sval[wl][q];
        }
        if (lane == 0) ccount[s] = n;
        __syncwarp();
    }
}

// scratch -> CSR (one warp per irregular point), with the FP32 copies
__global__ void k_side_compact(int64_t n_irr, const int* ccount, const int* bcount, const int32_t* toff,
                               const double* tval, const int32_t* tbidx, const double* tbval,
                               const int32_t* corr_ptr, int32_t* corr_off, double* corr_val, float* corr_val32,
                               const int32_t* bib_ptr, int32_t* bib_idx, double* bib_val) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < n_irr; s += nwarps) {
        const int c0 = corr_ptr[s], nc = ccount[s];
        for (int q = lane; q < nc; q += 32) {
            const double v = tval[s * kMaxRaw + q];
            corr_off[c0 + q] = toff[s * kMaxRaw + q];
            corr_val[c0 + q] = v;
            corr_val32[c0 + q] = (float)v;
        }
        const int b0 = bib_ptr[s], nb = bcount[s];
        for (int q = lane; q < nb; q += 32) {
            bib_idx[b0 + q] = tbidx[s * kMaxBib + q];
            bib_val[b0 + q] = tbval[s * kMaxBib + q];
        }
    }
}

__global__ void k_to_float(const double* in, float* out, int64_t n) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

template <class T>
void free_ptr(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// a classification's buffer back to the pool, ordered on the context's stream
template <class T>
void pool_free_ptr(cfp_ctx* c, T*& p) {
    pool_free(p, c->stream);
    p = nullptr;
}

unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

cfp_status classify(cfp_ctx* c) {
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    const int64_t N = c->N;
    c->classified = false;
    c->generation += 1;
    pool_free_ptr(c, c->irr_lin);
    pool_free_ptr(c, c->ibi_off);
    pool_free_ptr(c, c->ibi_xyz);
    pool_free_ptr(c, c->corr_ptr);
    pool_free_ptr(c, c->corr_off);
    pool_free_ptr(c, c->corr_val);
    pool_free_ptr(c, c->corr_val32);
    pool_free_ptr(c, c->bib_ptr);
    pool_free_ptr(c, c->bib_idx);
    pool_free_ptr(c, c->bib_val);
    pool_free_ptr(c, c->krow);
    pool_free_ptr(c, c->krow32);
    c->gsweeps[0] = c->gsweeps[1] = -1;  // side data changes: rebuild graphs
    free_mg(c);
    free_ilu(c);

    GeoArgs g;
    for (int d = 0; d < 3; ++d) {
        g.X[d] = c->dX[d];
        g.n[d] = c->n[d];
    }
    g.bodies = c->dbodies;
    g.b32 = c->dbody32;
    g.nb = (int)c->bodies.size();
    g.inside = c->fluid_inside;

    launch_metrics(c);  // the 1D grid metrics are rebuilt with every classification
    k_classify_solid<<<grid_for(N, 256), 256, 0, c->stream>>>(g, c->type, N);
    c->launches += 2;
    {
        const int nw = (nx - 2 + 29) / 30;
        const dim3 gi((unsigned)((nw + kIrrWarps - 1) / kIrrWarps), (unsigned)(ny - 2),
                      (unsigned)((nz - 2 + kIrrPlanes - 1) / kIrrPlanes));
        k_classify_irregular<<<gi, 32 * kIrrWarps, 0, c->stream>>>(c->type, nx, ny, nz);
    }
    CFP_CUDA(cudaGetLastError());

    long long h = 0;
    // compaction of the irregular points (slot map and list), ascending index
    {
        // size the list first with a counting pass
        long long nirr = 0;
        const int64_t nb = (N + kScanChunk - 1) / kScanChunk;
        if (nb > c->scan_cap) {
            pool_free_ptr(c, c->scan_bsum);
            CFP_CUDA(pool_malloc(&c->scan_bsum, sizeof(int) * nb, c->stream));
            c->scan_cap = nb;
        }
        k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(FlagIrregular{c->type}, N, c->scan_bsum);
        k_scan_blocks<<<1, kScanThreads, 0, c->stream>>>(c->scan_bsum, (int)nb, c->dtotal);
        c->launches += 3;  // with the scatter below
        CFP_CUDA(cudaGetLastError());
        CFP_CUDA(cudaMemcpyAsync(&nirr, c->dtotal, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
        CFP_CUDA(cudaStreamSynchronize(c->stream));
        c->n_irr = nirr;
        CFP_CUDA(pool_malloc(&c->irr_lin, sizeof(int32_t) * std::max<long long>(nirr, 1), c->stream));
        k_scan_scatter<<<(unsigned)nb, kScanThreads, 0, c->stream>>>(FlagIrregular{c->type},
                                                                      SinkSlots{c->slot, c->irr_lin}, N,
                                                                      c->scan_bsum);
        CFP_CUDA(cudaGetLastError());
    }
    const int64_t nirr = c->n_irr;

    IrrArgs ia;
    ia.type = c->type;
    ia.slot = c->slot;
    ia.irr_lin = c->irr_lin;
    ia.n_irr = nirr;
    for (int d = 0; d < 3; ++d) ia.n[d] = c->n[d];

    // IBI list: per irregular point, one IBI per solid axis neighbour
    int* cnt = nullptr;
    int* cnt2 = nullptr;
    CFP_CUDA(pool_malloc(&cnt, sizeof(int) * (nirr + 1), c->stream));
    CFP_CUDA(pool_malloc(&cnt2, sizeof(int) * (nirr + 1), c->stream));
    CFP_CUDA(pool_malloc(&c->ibi_off, sizeof(int32_t) * (nirr + 1), c->stream));
    if (nirr) k_ibi_count<<<grid_for(nirr, 256), 256, 0, c->stream>>>(ia, cnt);
    if (nirr) c->launches += 1;
    CFP_TRY(scan(c, FetchInt{cnt}, SinkOffsets{c->ibi_off}, nirr, c->dtotal, &h));
    c->n_ibi = h;
    CFP_CUDA(cudaMemcpyAsync(c->ibi_off + nirr, c->dtotal, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
    CFP_CUDA(pool_malloc(&c->ibi_xyz, sizeof(double) * 3 * std::max<int64_t>(c->n_ibi, 1), c->stream));
    if (c->n_ibi > 0) {
        int32_t* isrc = nullptr;
        CFP_CUDA(pool_malloc(&isrc, sizeof(int32_t) * c->n_ibi, c->stream));
        k_ibi_map<<<grid_for(nirr, 256), 256, 0, c->stream>>>(ia, c->ibi_off, isrc);
        k_ibi_roots<<<grid_for(c->n_ibi, 128), 128, 0, c->stream>>>(ia, g, isrc, c->n_ibi, c->ibi_xyz);
        c->launches += 2;
        CFP_CUDA(cudaGetLastError());
        CFP_CUDA(cudaStreamSynchronize(c->stream));
        pool_free(isrc, c->stream);
    }
    CFP_CUDA(cudaGetLastError());

    // side list: count, scan, fill
    SideArgs S;
    S.a = ia;
    const Grid<double> gv = grid_view<double>(c);
    for (int d = 0; d < 3; ++d) {
        S.ax[d] = gv.ax[d];
        S.X[d] = c->dX[d];
    }
    S.ibi_off = c->ibi_off;
    S.ibi_xyz = c->ibi_xyz;
    CFP_CUDA(cudaMemsetAsync(c->derr, 0, sizeof(DevError), c->stream));
    CFP_CUDA(cudaMemsetAsync(c->dtotal + 4, 0, sizeof(long long), c->stream));
    unsigned long long* ndeg = reinterpret_cast<unsigned long long*>(c->dtotal + 4);
    // per-slot scratch slices, kept by the context across classifications
    const int64_t nsl = std::max<int64_t>(nirr, 1);
    const size_t need = (size_t)nsl * (kMaxRaw * (sizeof(int32_t) + sizeof(double)) +
                                       kMaxBib * (sizeof(int32_t) + sizeof(double)));
    if (c->side_scratch_bytes < need) {
        pool_free(c->side_scratch, c->stream);
        c->side_scratch = nullptr;
        c->side_scratch_bytes = 0;
        CFP_CUDA(pool_malloc(&c->side_scratch, need, c->stream));
        c->side_scratch_bytes = need;
    }
    double* tval = static_cast<double*>(c->side_scratch);
    double* tbval = tval + (size_t)nsl * kMaxRaw;
    int32_t* toff = reinterpret_cast<int32_t*>(tbval + (size_t)nsl * kMaxBib);
    int32_t* tbidx = toff + (size_t)nsl * kMaxRaw;
    CFP_CUDA(pool_malloc(&c->krow, sizeof(double) * 7 * std::max<int64_t>(nirr, 1), c->stream));
    CFP_CUDA(pool_malloc(&c->krow32, sizeof(float) * 7 * std::max<int64_t>(nirr, 1), c->stream));
    if (nirr) {
        // plan (count, then place), one thread per operator for the moment
        // matching, finish; the adds land in the order the row is built in
        int *ntask = nullptr, *task_off = nullptr, *ferr = nullptr, *ndegs = nullptr;
        SideTask* tasks = nullptr;
        CFP_CUDA(pool_malloc(&ntask, sizeof(int) * nirr, c->stream));
        CFP_CUDA(pool_malloc(&task_off, sizeof(int) * nirr, c->stream));
        CFP_CUDA(pool_malloc(&ferr, sizeof(int) * nirr, c->stream));
        CFP_CUDA(pool_malloc(&ndegs, sizeof(int) * nirr, c->stream));
        k_side_plan<true><<<grid_for(nirr, 128), 128, 0, c->stream>>>(S, ntask, nullptr, nullptr, nullptr, nullptr,
                                                                      nullptr, nullptr, nullptr, nullptr);
        c->launches += 1;
        CFP_CUDA(cudaGetLastError());
        long long ntasks = 0;
        CFP_TRY(scan(c, FetchInt{ntask}, SinkOffsets{task_off}, nirr, c->dtotal, &ntasks));
        CFP_CUDA(pool_malloc(&tasks, sizeof(SideTask) * std::max<long long>(ntasks, 1), c->stream));
        k_side_plan<false><<<grid_for(nirr, 128), 128, 0, c->stream>>>(S, ntask, task_off, tasks, cnt, cnt2, ferr,
                                                                       ndegs, toff, tval);
        if (ntasks)
            k_side_solve<<<grid_for(ntasks, 64), 64, 0, c->stream>>>(S, tasks, ntasks, ferr, toff, tval, tbidx,
                                                                    tbval);
        k_side_finish<<<grid_for(nirr, 128), 128, 0, c->stream>>>(S, cnt, cnt2, ferr, ndegs, c->krow, ndeg, c->derr);
        c->launches += ntasks ? 3 : 2;
        CFP_CUDA(cudaGetLastError());
        for (void* q : {(void*)ntask, (void*)task_off, (void*)ferr, (void*)ndegs, (void*)tasks}) pool_free(q, c->stream);
    }
    if (nirr) {
        k_side_merge<<<grid_for(32 * nirr, 32 * kMergeWarps), 32 * kMergeWarps, 0, c->stream>>>(nirr, cnt, toff, tval);
        c->launches += 1;
        CFP_CUDA(cudaGetLastError());
    }
    DevError he;
    long long hdeg = 0;
    CFP_CUDA(cudaMemcpyAsync(&he, c->derr, sizeof(DevError), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaMemcpyAsync(&hdeg, c->dtotal + 4, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    c->n_deg = hdeg;
    if (he.code) {
        pool_free(cnt, c->stream);
        pool_free(cnt2, c->stream);
        const int i = he.lin % nx, j = (he.lin / nx) % ny, k = he.lin / (nx * ny);
        const char* why = he.detail == DETAIL_BOXIBI ? "a modified stencil needs an IBI at a box node"
                        : he.detail == DETAIL_FEWPOINTS ? "fewer than three points for a modified operator"
                        : he.detail == DETAIL_SINGULAR ? "singular moment matrix"
                        : he.detail == DETAIL_OVERFLOW ? "too many stencil entries"
                        : "missing IBI";
        c->class_status = CFP_EGEOM;
        return fail(CFP_EGEOM, std::string("unsupported geometry at irregular point (") + std::to_string(i) + "," +
                                   std::to_string(j) + "," + std::to_string(k) + "): " + why);
    }
    CFP_CUDA(pool_malloc(&c->corr_ptr, sizeof(int32_t) * (nirr + 1), c->stream));
    CFP_CUDA(pool_malloc(&c->bib_ptr, sizeof(int32_t) * (nirr + 1), c->stream));
    CFP_TRY(scan(c, FetchInt{cnt}, SinkOffsets{c->corr_ptr}, nirr, c->dtotal, &h));
    c->n_corr = h;
    CFP_CUDA(cudaMemcpyAsync(c->corr_ptr + nirr, c->dtotal, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
    CFP_TRY(scan(c, FetchInt{cnt2}, SinkOffsets{c->bib_ptr}, nirr, c->dtotal, &h));
    c->n_bib = h;
    CFP_CUDA(cudaMemcpyAsync(c->bib_ptr + nirr, c->dtotal, sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
    CFP_CUDA(pool_malloc(&c->corr_off, sizeof(int32_t) * std::max<int64_t>(c->n_corr, 1), c->stream));
    CFP_CUDA(pool_malloc(&c->corr_val, sizeof(double) * std::max<int64_t>(c->n_corr, 1), c->stream));
    CFP_CUDA(pool_malloc(&c->corr_val32, sizeof(float) * std::max<int64_t>(c->n_corr, 1), c->stream));
    CFP_CUDA(pool_malloc(&c->bib_idx, sizeof(int32_t) * std::max<int64_t>(c->n_bib, 1), c->stream));
    CFP_CUDA(pool_malloc(&c->bib_val, sizeof(double) * std::max<int64_t>(c->n_bib, 1), c->stream));
    if (nirr)
        k_side_compact<<<grid_for(32 * nirr, 256), 256, 0, c->stream>>>(nirr, cnt, cnt2, toff, tval, tbidx, tbval,
                                                                        c->corr_ptr, c->corr_off, c->corr_val,
                                                                        c->corr_val32, c->bib_ptr, c->bib_idx,
                                                                        c->bib_val);
    if (nirr) k_to_float<<<grid_for(7 * nirr, 256), 256, 0, c->stream>>>(c->krow, c->krow32, 7 * nirr);
    c->launches += nirr ? 2 : 0;
    CFP_CUDA(cudaGetLastError());
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    pool_free(cnt, c->stream);
    pool_free(cnt2, c->stream);
    c->classified = true;
    c->class_status = CFP_OK;
    return CFP_OK;
}

}  // namespace cfp
