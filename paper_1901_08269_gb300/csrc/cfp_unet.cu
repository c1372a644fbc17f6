// The learned part (an extension of the method, not in the paper): a four-
// level 3D convolutional U-Net (16 / 32 / 64 / 128 channels, 3x3x3 kernels,
// BF16 weights and activations, FP32 accumulation) that maps a residual of
// the compact system to its error, trained on the GPU by the tcgen05 kernels
// of cfp_unet_kernels.cuh on residual / error pairs the solver generates.
//
// Network (level l holds the grid coarsened l times, n_{l+1} = (n_l + 1) / 2,
// coarse node I on fine node 2I; skips by addition):
//   a0 = relu(conv(x)), a1 = relu(conv(a0))                    16      level 0
//   a2 = relu(conv(R a1)), a3 = relu(conv(a2))                 16->32  level 1
//   a4 = relu(conv(R a3)), a5 = relu(conv(a4))                 32->64  level 2
//   a6 = relu(conv(R a5)), a7 = relu(conv(a6))                 64->128 level 3
//   c2 = conv(a7)        u2 = P c2 + a5,  a8 = relu(conv(u2))  128->64
//   c1 = conv(a8)        u1 = P c1 + a3,  a9 = relu(conv(u1))  64->32
//   c0 = conv(a9)                                               32->16  level 1
//   y = P c0 (channel 0)                                        level 0
// R: injection (coarse I = fine 2I); P: its linear interpolation in index
// space (fine 2I = coarse I, fine 2I + 1 = the mean of coarse I and I + 1).
// The output is a coarse-grid correction interpolated to the fine grid, so
// it carries no more high-frequency content than an interpolant (the
// network serves as the coarse correction of a two-grid cycle, where the
// smoother handles the rest).
// Input channels: 0 the scaled residual at the unknowns, 1 the unknowns'
// mask, 2 a signed distance to the bodies' surfaces (clamped, scaled), 3-5
// the logarithm of the local grid spacing over the mean spacing per axis.
#include <math.h>
#include <string.h>

#include <cudaTypedefs.h>

#include <random>
#include <vector>

#include "cfp_internal.cuh"
#include "cfp_unet_kernels.cuh"
#include "../../include/cfp_nn.h"

namespace cfp {
namespace nn {
namespace {

constexpr int kIn = 16;      // input channels (6 used)
// the network's output is the error times kOut / max |r|: with the residual
// scaled to max 1, errors of these problems are of order 1e-2, and the
// factor brings the targets to order 1 (a power of two: exact)
constexpr double kOut = 32.0;
constexpr int kLayers = 13;

struct LayerDef {
    int cin, cout, level, relu;
};
constexpr LayerDef kDef[kLayers] = {{16, 16, 0, 1},  {16, 16, 0, 1},  {16, 32, 1, 1},  {32, 32, 1, 1},
                                    {32, 64, 2, 1},  {64, 64, 2, 1},  {64, 128, 3, 1}, {128, 128, 3, 1},
                                    {128, 64, 3, 0}, {64, 64, 2, 1},  {64, 32, 2, 0},  {32, 32, 1, 1},
                                    {32, 16, 1, 0}};

int64_t wcount(int l) { return (int64_t)kDef[l].cout * 27 * kDef[l].cin; }
int64_t param_count() {
    int64_t n = 0;
    for (int l = 0; l < kLayers; ++l) n += wcount(l) + kDef[l].cout;
    return n;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
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

// Activation (Np x C BF16) as a 2D tensor (channels innermost) with a box of
// 8 channels x rows; rows outside [0, Np) read as zero.
cfp_status act_map(CUtensorMap* m, const void* base, int C, int Np, int rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return fail(CFP_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (((uintptr_t)base & 15) != 0) return fail(CFP_EINVAL, "activation arrays must be 16-byte aligned");
    const cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)Np};
    const cuuint64_t strides[1] = {(cuuint64_t)C * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CFP_ECUDA, "cuTensorMapEncodeTiled failed for an activation");
    return CFP_OK;
}

Pad make_pad(int nx, int ny, int nz) {
    Pad P;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.nxp = nx + 2;
    P.nyp = ny + 2;
    P.nzp = nz + 2;
    P.Np = P.nxp * P.nyp * P.nzp;
    return P;
}
Pad coarser(const Pad& f) { return make_pad((f.nx + 1) / 2, (f.ny + 1) / 2, (f.nz + 1) / 2); }

int num_sms() {
    static int n = []() {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

unsigned blocks(int64_t n, int per = 256) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 152 * 32));
}

// ------------------------------------------------------ launch dispatch
template <int CIN, int COUT>
cfp_status prep_conv() {
    using C = ConvCfg<CIN, COUT>;
    using W = WgCfg<CIN, COUT>;
    static cfp_status st = []() {
        if (cudaFuncSetAttribute(k_conv_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) !=
                cudaSuccess ||
            cudaFuncSetAttribute(k_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, W::SMEM) !=
                cudaSuccess)
            return CFP_ECUDA;
        return CFP_OK;
    }();
    if (st != CFP_OK) return fail(st, "cudaFuncSetAttribute failed for a convolution kernel");
    return CFP_OK;
}

template <int CIN, int COUT>
int conv_grid(const Pad& P) {
    using C = ConvCfg<CIN, COUT>;
    static int per = []() {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_conv_tc<CIN, COUT>, kConvThreads, C::SMEM);
        return v > 0 ? v : 1;
    }();
    const int ntiles = (P.Np + 127) / 128;
    return std::max(1, std::min(ntiles, per * num_sms()));
}

template <int CIN, int COUT>
cfp_status conv_t(cudaStream_t s, const uint16_t* in, const uint16_t* wsrc, bool flip, uint16_t* wpk,
                  const float* bias, const uint16_t* act, const Pad& P, int flags, void* out, int* err) {
    using C = ConvCfg<CIN, COUT>;
    { const cfp_status ps_ = prep_conv<CIN, COUT>(); if (ps_ != CFP_OK) return ps_; }
    CUtensorMap m;
    CFP_TRY(act_map(&m, in, CIN, P.Np, kWin));
    const int nw = COUT * 27 * CIN;
    if (flip) k_wpack<CIN, COUT, true><<<blocks(nw), 256, 0, s>>>(wsrc, wpk);
    else k_wpack<CIN, COUT, false><<<blocks(nw), 256, 0, s>>>(wsrc, wpk);
    k_conv_tc<CIN, COUT><<<conv_grid<CIN, COUT>(P), kConvThreads, C::SMEM, s>>>(
        m, wpk, bias, act, P, flags, (flags & F_OUT_F32) ? nullptr : (uint16_t*)out,
        (flags & F_OUT_F32) ? (float*)out : nullptr, err);
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

__global__ void k_wgrad_reduce(const float* __restrict__ part, int nchunks, int cin, int cout,
                               float* __restrict__ dw) {
    const int n = 27 * cin * cout;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int co = e % cout, r = e / cout, ci = r % cin, t = r / cin;
        float s = 0.f;
        for (int q = 0; q < nchunks; ++q) s += part[(size_t)q * n + e];
        dw[((size_t)co * 27 + t) * cin + ci] += s;
    }
}

// column sums of a (Np x C) BF16 matrix: per-block partials, then a fixed-order sum
__global__ void k_colsum_part(const uint16_t* __restrict__ g, int Np, int C, float* __restrict__ part) {
    const int c = threadIdx.x % C, lanes = blockDim.x / C, l = threadIdx.x / C;
    float s = 0.f;
    for (int r = blockIdx.x * lanes + l; r < Np; r += gridDim.x * lanes) s += bf2f(g[(size_t)r * C + c]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    if (l == 0) {
        for (int q = 1; q < lanes; ++q) s += red[q * C + c];
        part[blockIdx.x * C + c] = s;
    }
}
__global__ void k_colsum_final(const float* __restrict__ part, int nb, int C, float* __restrict__ db) {
    const int c = threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[b * C + c];
    db[c] += s;
}
constexpr int kColBlocks = 256;

template <int CIN, int COUT>
cfp_status wgrad_t(cudaStream_t s, const uint16_t* x, const uint16_t* g, const Pad& P, float* part, int64_t part_cap,
                   float* dw, float* db, float* bpart, int* err) {
    using W = WgCfg<CIN, COUT>;
    { const cfp_status ps_ = prep_conv<CIN, COUT>(); if (ps_ != CFP_OK) return ps_; }
    CUtensorMap mx, mg;
    CFP_TRY(act_map(&mx, x, CIN, P.Np, kWin));
    CFP_TRY(act_map(&mg, g, COUT, P.Np, 128));
    const int ntiles = (P.Np + 127) / 128;
    int nch = std::max(1, std::min(ntiles, num_sms() / W::NSETS));
    while ((int64_t)nch * 27 * CIN * COUT > part_cap && nch > 1) --nch;
    const int tpc = (ntiles + nch - 1) / nch;
    nch = (ntiles + tpc - 1) / tpc;
    k_wgrad_tc<CIN, COUT><<<dim3(W::NSETS, nch), kConvThreads, W::SMEM, s>>>(mx, mg, P, tpc, part, err);
    k_wgrad_reduce<<<blocks(27 * CIN * COUT), 256, 0, s>>>(part, nch, CIN, COUT, dw);
    if (db) {
        k_colsum_part<<<kColBlocks, 256 / COUT * COUT, 0, s>>>(g, P.Np, COUT, bpart);
        k_colsum_final<<<1, 128, 0, s>>>(bpart, kColBlocks, COUT, db);
    }
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

#define CFP_NN_PAIRS(X) X(16, 16) X(16, 32) X(32, 16) X(32, 32) X(32, 64) X(64, 32) X(64, 64) X(64, 128) X(128, 64) X(128, 128)

bool supported(int cin, int cout) {
#define X(a, b) if (cin == a && cout == b) return true;
    CFP_NN_PAIRS(X)
#undef X
    return false;
}

cfp_status conv_any(cudaStream_t s, int cin, int cout, const uint16_t* in, const uint16_t* w, bool flip,
                    uint16_t* wpk, const float* bias, const uint16_t* act, const Pad& P, int flags, void* out,
                    int* err) {
#define X(a, b) \
    if (cin == a && cout == b) return conv_t<a, b>(s, in, w, flip, wpk, bias, act, P, flags, out, err);
    CFP_NN_PAIRS(X)
#undef X
    return fail(CFP_EINVAL, "unsupported channel counts of a convolution");
}

cfp_status wgrad_any(cudaStream_t s, int cin, int cout, const uint16_t* x, const uint16_t* g, const Pad& P,
                     float* part, int64_t part_cap, float* dw, float* db, float* bpart, int* err) {
#define X(a, b) \
    if (cin == a && cout == b) return wgrad_t<a, b>(s, x, g, P, part, part_cap, dw, db, bpart, err);
    CFP_NN_PAIRS(X)
#undef X
    return fail(CFP_EINVAL, "unsupported channel counts of a weight gradient");
}

// ------------------------------------------------------ transfer kernels
// the network's output: y (level 0, 16 FP32 channels) = P c (channel 0 of the
// level-1 activation c), the other channels 0
__global__ void k_prolong_out(const uint16_t* __restrict__ c, Pad Cg, Pad F, float* __restrict__ y) {
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < F.Np; row += gridDim.x * blockDim.x) {
        float acc = 0.f;
        if (interior(F, row)) {
            const int ip = row % F.nxp, r = row / F.nxp, jp = r % F.nyp, kp = r / F.nyp;
            const int idx[3] = {ip - 1, jp - 1, kp - 1};
            int lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                lo[d] = idx[d] / 2;
                hi[d] = (idx[d] + 1) / 2;
            }
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int I = dx ? hi[0] : lo[0], J = dy ? hi[1] : lo[1], K = dz ? hi[2] : lo[2];
                        const int cr = ((K + 1) * Cg.nyp + (J + 1)) * Cg.nxp + (I + 1);
                        acc += 0.125f * bf2f(c[(size_t)cr * 16]);
                    }
        }
        float4* yp = reinterpret_cast<float4*>(y + (size_t)row * 16);
        yp[0] = make_float4(acc, 0.f, 0.f, 0.f);
        for (int q = 1; q < 4; ++q) yp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// injection: coarse interior node I = fine node 2I (padded: 2 I_p - 1), 8
// channels per thread; padding nodes 0
__global__ void k_inject(const uint16_t* __restrict__ f, Pad F, uint16_t* __restrict__ c, Pad Cg, int C) {
    const int c8 = C / 8;
    const int64_t n = (int64_t)Cg.Np * c8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / c8), q = (int)(e % c8);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (interior(Cg, row)) {
            const int i = row % Cg.nxp, r = row / Cg.nxp, j = r % Cg.nyp, k = r / Cg.nyp;
            const int fr = ((2 * k - 1) * F.nyp + (2 * j - 1)) * F.nxp + (2 * i - 1);
            v = reinterpret_cast<const uint4*>(f + (size_t)fr * C)[q];
        }
        reinterpret_cast<uint4*>(c + (size_t)row * C)[q] = v;
    }
}

// out = P c + s on the fine level (8 channels per thread), FP32 sums
__global__ void k_prolong_add(const uint16_t* __restrict__ c, Pad Cg, const uint16_t* __restrict__ s, Pad F,
                              uint16_t* __restrict__ out, int C) {
    const int c8 = C / 8;
    const int64_t n = (int64_t)F.Np * c8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / c8), q = (int)(e % c8);
        uint16_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (interior(F, row)) {
            const int ip = row % F.nxp, r = row / F.nxp, jp = r % F.nyp, kp = r / F.nyp;
            const int idx[3] = {ip - 1, jp - 1, kp - 1};
            int lo[3], hi[3];
            for (int d = 0; d < 3; ++d) {
                lo[d] = idx[d] / 2;
                hi[d] = (idx[d] + 1) / 2;  // = lo for even indices
            }
            float acc[8];
            const uint4 sv = reinterpret_cast<const uint4*>(s + (size_t)row * C)[q];
            const uint16_t* sh = reinterpret_cast<const uint16_t*>(&sv);
            for (int t = 0; t < 8; ++t) acc[t] = bf2f(sh[t]);
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx) {
                        const int I = dx ? hi[0] : lo[0], J = dy ? hi[1] : lo[1], K = dz ? hi[2] : lo[2];
                        // each axis: weight 1 split as 1/2 + 1/2 (even index: both halves the same node)
                        const float w = 0.125f;
                        const int cr = ((K + 1) * Cg.nyp + (J + 1)) * Cg.nxp + (I + 1);
                        const uint4 cv = reinterpret_cast<const uint4*>(c + (size_t)cr * C)[q];
                        const uint16_t* ch = reinterpret_cast<const uint16_t*>(&cv);
                        for (int t = 0; t < 8; ++t) acc[t] += w * bf2f(ch[t]);
                    }
            for (int t = 0; t < 8; ++t) h[t] = f2bf(acc[t]);
        }
        reinterpret_cast<uint4*>(out + (size_t)row * C)[q] = *reinterpret_cast<uint4*>(h);
    }
}

// out = P^T g on the coarse level: coarse I gathers fine 2I (weight 1) and
// 2I -+ 1 (weight 1/2) per axis, inside the fine grid
__global__ void k_prolong_t(const uint16_t* __restrict__ g, Pad F, uint16_t* __restrict__ out, Pad Cg, int C) {
    const int c8 = C / 8;
    const int64_t n = (int64_t)Cg.Np * c8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / c8), q = (int)(e % c8);
        uint16_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (interior(Cg, row)) {
            const int Ip = row % Cg.nxp, r = row / Cg.nxp, Jp = r % Cg.nyp, Kp = r / Cg.nyp;
            const int I = Ip - 1, J = Jp - 1, K = Kp - 1;
            float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int dz = -1; dz <= 1; ++dz) {
                const int k = 2 * K + dz;
                if (k < 0 || k > F.nz - 1) continue;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int j = 2 * J + dy;
                    if (j < 0 || j > F.ny - 1) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int i = 2 * I + dx;
                        if (i < 0 || i > F.nx - 1) continue;
                        const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
                        const int fr = ((k + 1) * F.nyp + (j + 1)) * F.nxp + (i + 1);
                        const uint4 gv = reinterpret_cast<const uint4*>(g + (size_t)fr * C)[q];
                        const uint16_t* gh = reinterpret_cast<const uint16_t*>(&gv);
                        for (int t = 0; t < 8; ++t) acc[t] += w * bf2f(gh[t]);
                    }
                }
            }
            for (int t = 0; t < 8; ++t) h[t] = f2bf(acc[t]);
        }
        reinterpret_cast<uint4*>(out + (size_t)row * C)[q] = *reinterpret_cast<uint4*>(h);
    }
}

// gradient at a skip source a (post-ReLU): out = (gu + R^T gb) * [a > 0]
// (gu NULL: 0); R^T puts coarse I on fine 2I
__global__ void k_skip_grad(const uint16_t* __restrict__ gu, const uint16_t* __restrict__ gb, Pad Cg,
                            const uint16_t* __restrict__ a, Pad F, uint16_t* __restrict__ out, int C) {
    const int c8 = C / 8;
    const int64_t n = (int64_t)F.Np * c8;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / c8), q = (int)(e % c8);
        uint16_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (interior(F, row)) {
            const int ip = row % F.nxp, r = row / F.nxp, jp = r % F.nyp, kp = r / F.nyp;
            const uint4 uv = gu ? reinterpret_cast<const uint4*>(gu + (size_t)row * C)[q] : make_uint4(0, 0, 0, 0);
            const uint4 av = reinterpret_cast<const uint4*>(a + (size_t)row * C)[q];
            const uint16_t* uh = reinterpret_cast<const uint16_t*>(&uv);
            const uint16_t* ah = reinterpret_cast<const uint16_t*>(&av);
            float acc[8];
            for (int t = 0; t < 8; ++t) acc[t] = bf2f(uh[t]);
            if ((ip - 1) % 2 == 0 && (jp - 1) % 2 == 0 && (kp - 1) % 2 == 0) {
                const int cr = (((kp - 1) / 2 + 1) * Cg.nyp + ((jp - 1) / 2 + 1)) * Cg.nxp + ((ip - 1) / 2 + 1);
                const uint4 bv = reinterpret_cast<const uint4*>(gb + (size_t)cr * C)[q];
                const uint16_t* bh = reinterpret_cast<const uint16_t*>(&bv);
                for (int t = 0; t < 8; ++t) acc[t] += bf2f(bh[t]);
            }
            for (int t = 0; t < 8; ++t) h[t] = bf_pos(ah[t]) ? f2bf(acc[t]) : (uint16_t)0;
        }
        reinterpret_cast<uint4*>(out + (size_t)row * C)[q] = *reinterpret_cast<uint4*>(h);
    }
}

// ------------------------------------------------- input, loss, optimiser
struct GridIn {
    const uint8_t* type;
    const double* X[3];
    const cfp_body* bodies;
    int nb, inside;
    int n[3];
    double hmean[3];
};

// approximate signed distance to the union of the bodies' surfaces
// (negative inside the solid): exact for spheres and tori, first order for
// ellipsoids
__device__ double body_dist(const cfp_body& b, double x, double y, double z) {
    const double d0 = x - b.c[0], d1 = y - b.c[1], d2 = z - b.c[2];
    const double* R = b.R;
    const double q0 = R[0] * d0 + R[3] * d1 + R[6] * d2;
    const double q1 = R[1] * d0 + R[4] * d1 + R[7] * d2;
    const double q2 = R[2] * d0 + R[5] * d1 + R[8] * d2;
    if (b.kind == CFP_SPHERE) return sqrt(q0 * q0 + q1 * q1 + q2 * q2) - b.p[0];
    if (b.kind == CFP_ELLIPSOID) {
        const double e0 = q0 / b.p[0], e1 = q1 / b.p[1], e2 = q2 / b.p[2];
        const double s = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        const double g0 = e0 / b.p[0], g1 = e1 / b.p[1], g2 = e2 / b.p[2];
        const double gn = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
        return gn > 0.0 ? (s - 1.0) * s / gn : -fmin(b.p[0], fmin(b.p[1], b.p[2]));
    }
    const double rho = sqrt(q0 * q0 + q1 * q1);
    return sqrt((rho - b.p[0]) * (rho - b.p[0]) + q2 * q2) - b.p[1];
}

// x0 (padded, 16 channels) from an FP64 field r on the solver grid, scaled by
// *scale; target = scale * e at the unknowns (e may be NULL: zero); mask = 1
// at the unknowns; *count += the unknowns (padding rows: all zero)
__global__ void k_unet_input(GridIn G, Pad P, const double* __restrict__ r, const double* __restrict__ e,
                             const double* __restrict__ scale, uint16_t* __restrict__ x0, float* __restrict__ target,
                             float* __restrict__ mask, int* __restrict__ count) {
    const double s = *scale;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < P.Np; row += gridDim.x * blockDim.x) {
        uint16_t h[16];
        for (int q = 0; q < 16; ++q) h[q] = 0;
        float t = 0.f, m = 0.f;
        if (interior(P, row)) {
            const int ip = row % P.nxp, rr = row / P.nxp, jp = rr % P.nyp, kp = rr / P.nyp;
            const int i = ip - 1, j = jp - 1, k = kp - 1;
            const int64_t l = i + (int64_t)G.n[0] * (j + (int64_t)G.n[1] * k);
            const uint8_t ty = G.type[l];
            const bool unk = ty == CFP_REGULAR || ty == CFP_IRREGULAR;
            const double px = G.X[0][i], py = G.X[1][j], pz = G.X[2][k];
            double dist = 1e30;
            for (int b = 0; b < G.nb; ++b) dist = fmin(dist, body_dist(G.bodies[b], px, py, pz));
            if (G.inside) dist = -dist;
            const double sd = G.nb ? fmax(-1.0, fmin(1.0, dist / 0.25)) : 1.0;
            const int idx[3] = {i, j, k};
            float hl[3];
            for (int d = 0; d < 3; ++d) {
                const int a = idx[d], n = G.n[d];
                const double h = 0.5 * (G.X[d][min(a + 1, n - 1)] - G.X[d][max(a - 1, 0)]) * (a == 0 || a == n - 1 ? 2.0 : 1.0);
                hl[d] = (float)log(h / G.hmean[d]);
            }
            h[0] = f2bf(unk ? (float)(s * r[l]) : 0.f);
            h[1] = f2bf(unk ? 1.f : 0.f);
            h[2] = f2bf((float)sd);
            h[3] = f2bf(hl[0]);
            h[4] = f2bf(hl[1]);
            h[5] = f2bf(hl[2]);
            if (unk) {
                m = 1.f;
                t = e ? (float)(kOut * s * e[l]) : 0.f;
                atomicAdd(count, 1);
            }
        }
        uint4* xp = reinterpret_cast<uint4*>(x0 + (size_t)row * 16);
        xp[0] = *reinterpret_cast<uint4*>(h);
        xp[1] = *reinterpret_cast<uint4*>(h + 8);
        if (target) target[row] = t;
        if (mask) mask[row] = m;
    }
}

// *scale = 1 / max |r| over the unknowns (1 if that maximum is 0): block
// maxima of |r| as ordered bits, then the reciprocal
__global__ void k_absmax(const uint8_t* __restrict__ type, const double* __restrict__ r, int64_t N,
                         unsigned long long* __restrict__ mx) {
    double m = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[l];
        if (t == CFP_REGULAR || t == CFP_IRREGULAR) m = fmax(m, fabs(r[l]));
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}
__global__ void k_scale_from_max(const unsigned long long* __restrict__ mx, double* __restrict__ scale,
                                 double* __restrict__ inv) {
    const double m = __longlong_as_double((long long)*mx);
    const double s = m > 0.0 && m < 1e300 ? 1.0 / m : 1.0;
    *scale = s;
    *inv = 1.0 / (s * kOut);
}

// Loss: the energy norm of the error of output channel 0 on the grid,
//     L = (1 / count) sum over the edges (p, q) of the padded grid of
//         (d_p - d_q)^2,   d = mask (y[.][0] - target)
// (d is 0 at the padding and at every node that is not an unknown: the
// error vanishes at Dirichlet nodes), the norm in which a preconditioner's
// error matters; unlike the mean squared error it weights the high-frequency
// part of the error the way the operator does.  Its gradient is
//     dL/dy_p[0] = (2 / count) mask_p (6 d_p - sum of d over the 6 neighbours),
// written as a 16-channel BF16 activation (channel 0 only); per-block loss
// partials over the edges to the +x, +y, +z neighbour of every padded node.
__device__ __forceinline__ float loss_d(const float* __restrict__ y, const float* __restrict__ target,
                                        const float* __restrict__ mask, int row) {
    return (y[(size_t)row * 16] - target[row]) * mask[row];
}
__global__ void k_unet_energy(const float* __restrict__ y, const float* __restrict__ target,
                              const float* __restrict__ mask, Pad P, const int* __restrict__ count,
                              uint16_t* __restrict__ gy, float* __restrict__ part) {
    const float inv = 1.f / (float)max(*count, 1);
    const int sy = P.nxp, sz = P.nxp * P.nyp;
    float acc = 0.f;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < P.Np; row += gridDim.x * blockDim.x) {
        const float d = loss_d(y, target, mask, row);
        const int i = row % P.nxp, r = row / P.nxp, j = r % P.nyp, k = r / P.nyp;
        float nb = 0.f;  // sum of the neighbours' d
        if (i + 1 < P.nxp) {
            const float q = loss_d(y, target, mask, row + 1);
            acc += (d - q) * (d - q);
            nb += q;
        }
        if (j + 1 < P.nyp) {
            const float q = loss_d(y, target, mask, row + sy);
            acc += (d - q) * (d - q);
            nb += q;
        }
        if (k + 1 < P.nzp) {
            const float q = loss_d(y, target, mask, row + sz);
            acc += (d - q) * (d - q);
            nb += q;
        }
        if (i > 0) nb += loss_d(y, target, mask, row - 1);
        if (j > 0) nb += loss_d(y, target, mask, row - sy);
        if (k > 0) nb += loss_d(y, target, mask, row - sz);
        uint16_t h[16];
        for (int q = 0; q < 16; ++q) h[q] = 0;
        h[0] = f2bf(2.f * inv * mask[row] * (6.f * d - nb));
        uint4* gp = reinterpret_cast<uint4*>(gy + (size_t)row * 16);
        gp[0] = *reinterpret_cast<uint4*>(h);
        gp[1] = *reinterpret_cast<uint4*>(h + 8);
    }
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0] * inv;
}
__global__ void k_sum_final(const float* __restrict__ part, int n, double* __restrict__ out) {
    double s = 0.0;
    for (int q = 0; q < n; ++q) s += part[q];
    *out = s;
}

// Adam (Kingma & Ba): first and second moments, bias corrections bc1 =
// 1 - beta1^step, bc2 = 1 - beta2^step; the gradient is cleared for the next
// accumulation; wbf (NULL: none) receives the BF16 weights
__global__ void k_adam(int64_t n, float* __restrict__ w, float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float bc1, float bc2, float eps) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gr = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gr;
        const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
        m[e] = mm;
        v[e] = vv;
        w[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
        g[e] = 0.f;
    }
}
__global__ void k_to_bf16(int64_t n, const float* __restrict__ w, uint16_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = f2bf(w[e]);
}

// u (FP64 field) = inv * y[.][0] at the unknowns, 0 elsewhere
__global__ void k_unet_output(const uint8_t* __restrict__ type, Pad P, int nx, int ny, int64_t N,
                              const float* __restrict__ y, const double* __restrict__ inv, double* __restrict__ u) {
    const double s = *inv;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[l];
        const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
        const int row = ((k + 1) * P.nyp + (j + 1)) * P.nxp + (i + 1);
        u[l] = (t == CFP_REGULAR || t == CFP_IRREGULAR) ? s * (double)y[(size_t)row * 16] : 0.0;
    }
}

}  // namespace
}  // namespace nn
}  // namespace cfp

using namespace cfp;
using namespace cfp::nn;

// ------------------------------------------------------------ the network
struct cfp_unet {
    cfp_ctx* owner = nullptr;
    cudaStream_t stream = nullptr;  // when set: the stream every call enqueues on (else the owner's)
    int64_t np = 0;  // parameters
    float* w32 = nullptr;  // FP32 master parameters: per layer W [cout][27][cin] then bias [cout]
    float* g32 = nullptr;  // gradients (accumulated)
    float* m32 = nullptr;
    float* v32 = nullptr;
    uint16_t* wbf = nullptr;  // BF16 weights (the layers' W only, same offsets as in w32)
    uint16_t* wpk = nullptr;  // packed operand weights of one convolution at a time
    int64_t woff[kLayers], boff[kLayers];
    int steps = 0;
    // work space
    float* part = nullptr;
    int64_t part_cap = 0;
    float* bpart = nullptr;
    float* lpart = nullptr;
    double* dscal = nullptr;  // [0] scale, [1] 1 / scale, [2] loss
    unsigned long long* dmax = nullptr;
    int* dcount = nullptr;
    int* derr = nullptr;
    // activations for the current grid
    Pad L[4];
    int64_t cap[4] = {0, 0, 0, 0};
    std::vector<void*> bufs;
    uint16_t *X = nullptr, *A0, *A1, *U0, *A10, *GY, *G1, *G2, *G3;
    float *Y = nullptr, *T, *M;
    uint16_t *B0, *A2, *A3, *U1, *A9, *C0, *GC0, *GB0, *H1, *H2, *H3;
    uint16_t *B1, *A4, *A5, *U2, *A8, *C1, *GC1, *GB1, *K1, *K2, *K3;
    uint16_t *B2, *A6, *A7, *C2, *GC2, *GB2, *M1, *M2;
    bool grads_ready = false;
};

namespace {

void free_bufs(cfp_unet* u) {
    for (void* p : u->bufs) cudaFree(p);
    u->bufs.clear();
    for (auto& c : u->cap) c = 0;
}

cfp_status alloc_into(cfp_unet* u, void** p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        return fail(CFP_ENOMEM, "device allocation failed for the network's activations");
    }
    u->bufs.push_back(*p);
    return CFP_OK;
}

// n = 4 m + 1 (m >= 2) nodes per axis: levels 0 to 2 have odd sizes, so
// injection and interpolation pair the nodes exactly (level 3 is only ever
// the coarse side)
bool unet_size_ok(int n) { return n >= 9 && (n - 1) % 4 == 0; }

// activation and gradient buffers for a level-0 grid of nx x ny x nz
cfp_status ensure_grid(cfp_unet* u, int nx, int ny, int nz, bool train) {
    if (!unet_size_ok(nx) || !unet_size_ok(ny) || !unet_size_ok(nz))
        return fail(CFP_EINVAL, "the network needs 4 m + 1 (>= 9) nodes per axis");
    Pad P[4];
    P[0] = make_pad(nx, ny, nz);
    for (int l = 1; l < 4; ++l) P[l] = coarser(P[l - 1]);
    bool fits = u->X != nullptr && (train ? u->GY != nullptr : true);
    for (int l = 0; l < 4; ++l) fits = fits && P[l].Np <= u->cap[l];
    for (int l = 0; l < 4; ++l) u->L[l] = P[l];
    if (fits) return CFP_OK;
    free_bufs(u);
    u->GY = nullptr;
    auto bf = [&](uint16_t** p, int l, int c) { return alloc_into(u, (void**)p, (size_t)P[l].Np * c * 2); };
    auto f32 = [&](float** p, int l, int c) { return alloc_into(u, (void**)p, (size_t)P[l].Np * c * 4); };
    CFP_TRY(bf(&u->X, 0, 16));
    CFP_TRY(bf(&u->A0, 0, 16));
    CFP_TRY(bf(&u->A1, 0, 16));
    CFP_TRY(bf(&u->U0, 0, 16));
    CFP_TRY(bf(&u->A10, 0, 16));
    CFP_TRY(f32(&u->Y, 0, 16));
    CFP_TRY(f32(&u->T, 0, 1));
    CFP_TRY(f32(&u->M, 0, 1));
    CFP_TRY(bf(&u->B0, 1, 16));
    CFP_TRY(bf(&u->A2, 1, 32));
    CFP_TRY(bf(&u->A3, 1, 32));
    CFP_TRY(bf(&u->U1, 1, 32));
    CFP_TRY(bf(&u->A9, 1, 32));
    CFP_TRY(bf(&u->C0, 1, 16));
    CFP_TRY(bf(&u->B1, 2, 32));
    CFP_TRY(bf(&u->A4, 2, 64));
    CFP_TRY(bf(&u->A5, 2, 64));
    CFP_TRY(bf(&u->U2, 2, 64));
    CFP_TRY(bf(&u->A8, 2, 64));
    CFP_TRY(bf(&u->C1, 2, 32));
    CFP_TRY(bf(&u->B2, 3, 64));
    CFP_TRY(bf(&u->A6, 3, 128));
    CFP_TRY(bf(&u->A7, 3, 128));
    CFP_TRY(bf(&u->C2, 3, 64));
    if (train) {
        CFP_TRY(bf(&u->GY, 0, 16));
        CFP_TRY(bf(&u->G1, 0, 16));
        CFP_TRY(bf(&u->G2, 0, 16));
        CFP_TRY(bf(&u->G3, 0, 16));
        CFP_TRY(bf(&u->GC0, 1, 16));
        CFP_TRY(bf(&u->GB0, 1, 16));
        CFP_TRY(bf(&u->H1, 1, 32));
        CFP_TRY(bf(&u->H2, 1, 32));
        CFP_TRY(bf(&u->H3, 1, 32));
        CFP_TRY(bf(&u->GC1, 2, 32));
        CFP_TRY(bf(&u->GB1, 2, 32));
        CFP_TRY(bf(&u->K1, 2, 64));
        CFP_TRY(bf(&u->K2, 2, 64));
        CFP_TRY(bf(&u->K3, 2, 64));
        CFP_TRY(bf(&u->GC2, 3, 64));
        CFP_TRY(bf(&u->GB2, 3, 64));
        CFP_TRY(bf(&u->M1, 3, 128));
        CFP_TRY(bf(&u->M2, 3, 128));
    }
    for (int l = 0; l < 4; ++l) u->cap[l] = P[l].Np;
    return CFP_OK;
}

cudaStream_t ustream(cfp_unet* u) { return u->stream ? u->stream : u->owner->stream; }

cfp_status conv_layer(cfp_unet* u, int l, const uint16_t* in, void* out, bool f32out) {
    const LayerDef& d = kDef[l];
    int flags = d.relu ? F_RELU : 0;
    if (f32out) flags |= F_OUT_F32;
    u->owner->launches += 2;
    return conv_any(ustream(u), d.cin, d.cout, in, u->wbf + u->woff[l], false, u->wpk, u->w32 + u->boff[l], nullptr,
                    u->L[d.level], flags, out, u->derr);
}

// input gradient of layer l: out = conv(g, W_l flipped), times [act > 0] if act
cfp_status dgrad_layer(cfp_unet* u, int l, const uint16_t* g, const uint16_t* act, uint16_t* out) {
    const LayerDef& d = kDef[l];
    u->owner->launches += 2;
    return conv_any(ustream(u), d.cout, d.cin, g, u->wbf + u->woff[l], true, u->wpk, nullptr, act, u->L[d.level],
                    act ? F_MASK : 0, out, u->derr);
}

cfp_status wgrad_layer(cfp_unet* u, int l, const uint16_t* x, const uint16_t* g) {
    const LayerDef& d = kDef[l];
    u->owner->launches += 4;
    return wgrad_any(ustream(u), d.cin, d.cout, x, g, u->L[d.level], u->part, u->part_cap, u->g32 + u->woff[l],
                     u->g32 + u->boff[l], u->bpart, u->derr);
}

void inject(cfp_unet* u, const uint16_t* f, int lf, uint16_t* c, int C) {
    k_inject<<<blocks((int64_t)u->L[lf + 1].Np * C / 8), 256, 0, ustream(u)>>>(f, u->L[lf], c, u->L[lf + 1], C);
    u->owner->launches += 1;
}
void prolong_add(cfp_unet* u, const uint16_t* c, int lf, const uint16_t* s, uint16_t* out, int C) {
    k_prolong_add<<<blocks((int64_t)u->L[lf].Np * C / 8), 256, 0, ustream(u)>>>(c, u->L[lf + 1], s, u->L[lf], out, C);
    u->owner->launches += 1;
}
void prolong_t(cfp_unet* u, const uint16_t* g, int lf, uint16_t* out, int C) {
    k_prolong_t<<<blocks((int64_t)u->L[lf + 1].Np * C / 8), 256, 0, ustream(u)>>>(g, u->L[lf], out, u->L[lf + 1], C);
    u->owner->launches += 1;
}
void skip_grad(cfp_unet* u, const uint16_t* gu, const uint16_t* gb, const uint16_t* a, int lf, uint16_t* out, int C) {
    k_skip_grad<<<blocks((int64_t)u->L[lf].Np * C / 8), 256, 0, ustream(u)>>>(gu, gb, u->L[lf + 1], a, u->L[lf], out,
                                                                                C);
    u->owner->launches += 1;
}

// forward pass from u->X; y (FP32, 16 channels) into u->Y
cfp_status forward(cfp_unet* u) {
    CFP_TRY(conv_layer(u, 0, u->X, u->A0, false));
    CFP_TRY(conv_layer(u, 1, u->A0, u->A1, false));
    inject(u, u->A1, 0, u->B0, 16);
    CFP_TRY(conv_layer(u, 2, u->B0, u->A2, false));
    CFP_TRY(conv_layer(u, 3, u->A2, u->A3, false));
    inject(u, u->A3, 1, u->B1, 32);
    CFP_TRY(conv_layer(u, 4, u->B1, u->A4, false));
    CFP_TRY(conv_layer(u, 5, u->A4, u->A5, false));
    inject(u, u->A5, 2, u->B2, 64);
    CFP_TRY(conv_layer(u, 6, u->B2, u->A6, false));
    CFP_TRY(conv_layer(u, 7, u->A6, u->A7, false));
    CFP_TRY(conv_layer(u, 8, u->A7, u->C2, false));
    prolong_add(u, u->C2, 2, u->A5, u->U2, 64);
    CFP_TRY(conv_layer(u, 9, u->U2, u->A8, false));
    CFP_TRY(conv_layer(u, 10, u->A8, u->C1, false));
    prolong_add(u, u->C1, 1, u->A3, u->U1, 32);
    CFP_TRY(conv_layer(u, 11, u->U1, u->A9, false));
    CFP_TRY(conv_layer(u, 12, u->A9, u->C0, false));
    k_prolong_out<<<blocks(u->L[0].Np), 256, 0, ustream(u)>>>(u->C0, u->L[1], u->L[0], u->Y);
    u->owner->launches += 1;
    return CFP_OK;
}

// backward pass for dL/dy in u->GY; gradients added to u->g32
cfp_status backward(cfp_unet* u) {
    prolong_t(u, u->GY, 0, u->GC0, 16);                   // g(c0) = P^T g(y)
    CFP_TRY(wgrad_layer(u, 12, u->A9, u->GC0));
    CFP_TRY(dgrad_layer(u, 12, u->GC0, u->A9, u->H1));
    CFP_TRY(wgrad_layer(u, 11, u->U1, u->H1));
    CFP_TRY(dgrad_layer(u, 11, u->H1, nullptr, u->H2));  // g(u1)
    prolong_t(u, u->H2, 1, u->GC1, 32);                   // g(c1)
    CFP_TRY(wgrad_layer(u, 10, u->A8, u->GC1));
    CFP_TRY(dgrad_layer(u, 10, u->GC1, u->A8, u->K1));
    CFP_TRY(wgrad_layer(u, 9, u->U2, u->K1));
    CFP_TRY(dgrad_layer(u, 9, u->K1, nullptr, u->K2));  // g(u2)
    prolong_t(u, u->K2, 2, u->GC2, 64);                  // g(c2)
    CFP_TRY(wgrad_layer(u, 8, u->A7, u->GC2));
    CFP_TRY(dgrad_layer(u, 8, u->GC2, u->A7, u->M1));
    CFP_TRY(wgrad_layer(u, 7, u->A6, u->M1));
    CFP_TRY(dgrad_layer(u, 7, u->M1, u->A6, u->M2));
    CFP_TRY(wgrad_layer(u, 6, u->B2, u->M2));
    CFP_TRY(dgrad_layer(u, 6, u->M2, nullptr, u->GB2));  // g(b2)
    skip_grad(u, u->K2, u->GB2, u->A5, 2, u->K3, 64);     // pre-activation gradient of a5
    CFP_TRY(wgrad_layer(u, 5, u->A4, u->K3));
    CFP_TRY(dgrad_layer(u, 5, u->K3, u->A4, u->K1));
    CFP_TRY(wgrad_layer(u, 4, u->B1, u->K1));
    CFP_TRY(dgrad_layer(u, 4, u->K1, nullptr, u->GB1));  // g(b1)
    skip_grad(u, u->H2, u->GB1, u->A3, 1, u->H3, 32);     // of a3
    CFP_TRY(wgrad_layer(u, 3, u->A2, u->H3));
    CFP_TRY(dgrad_layer(u, 3, u->H3, u->A2, u->H1));
    CFP_TRY(wgrad_layer(u, 2, u->B0, u->H1));
    CFP_TRY(dgrad_layer(u, 2, u->H1, nullptr, u->GB0));  // g(b0)
    skip_grad(u, nullptr, u->GB0, u->A1, 0, u->G3, 16);   // of a1 (no skip from the up path)
    CFP_TRY(wgrad_layer(u, 1, u->A0, u->G3));
    CFP_TRY(dgrad_layer(u, 1, u->G3, u->A0, u->G1));
    CFP_TRY(wgrad_layer(u, 0, u->X, u->G1));
    return CFP_OK;
}

cfp_status loss_grad(cfp_unet* u) {
    k_unet_energy<<<256, 256, 0, ustream(u)>>>(u->Y, u->T, u->M, u->L[0], u->dcount, u->GY, u->lpart);
    k_sum_final<<<1, 1, 0, ustream(u)>>>(u->lpart, 256, u->dscal + 2);
    u->owner->launches += 2;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status pack_input(cfp_unet* u, cfp_ctx* g, const double* r, const double* e) {
    cudaStream_t s = ustream(u);
    CFP_CUDA(cudaMemsetAsync(u->dmax, 0, sizeof(unsigned long long), s));
    CFP_CUDA(cudaMemsetAsync(u->dcount, 0, sizeof(int), s));
    k_absmax<<<blocks(g->N), 256, 0, s>>>(g->type, r, g->N, u->dmax);
    k_scale_from_max<<<1, 1, 0, s>>>(u->dmax, u->dscal, u->dscal + 1);
    GridIn G;
    G.type = g->type;
    for (int d = 0; d < 3; ++d) {
        G.X[d] = g->dX[d];
        G.n[d] = g->n[d];
        G.hmean[d] = (g->X[d].back() - g->X[d].front()) / (g->n[d] - 1);
    }
    G.bodies = g->dbodies;
    G.nb = (int)g->bodies.size();
    G.inside = g->fluid_inside;
    k_unet_input<<<blocks(u->L[0].Np), 256, 0, s>>>(G, u->L[0], r, e, u->dscal, u->X, u->T, u->M, u->dcount);
    u->owner->launches += 3;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status check_err(cfp_unet* u) {
    int h = 0;
    CFP_CUDA(cudaMemcpyAsync(&h, u->derr, sizeof(int), cudaMemcpyDeviceToHost, ustream(u)));
    CFP_CUDA(cudaStreamSynchronize(ustream(u)));
    if (h) {
        CFP_CUDA(cudaMemsetAsync(u->derr, 0, sizeof(int), ustream(u)));
        return fail(CFP_ECUDA, "a bounded pipeline wait of a tensor-core kernel timed out (code " + std::to_string(h) + ")");
    }
    return CFP_OK;
}

cfp_status adam_step(cfp_unet* u, double lr) {
    u->steps += 1;
    const double b1 = 0.9, b2 = 0.999;
    k_adam<<<blocks(u->np), 256, 0, ustream(u)>>>(u->np, u->w32, u->g32, u->m32, u->v32, (float)lr, (float)b1,
                                                  (float)b2, (float)(1.0 - pow(b1, u->steps)),
                                                  (float)(1.0 - pow(b2, u->steps)), 1e-8f);
    k_to_bf16<<<blocks(u->np), 256, 0, ustream(u)>>>(u->np, u->w32, u->wbf);
    u->owner->launches += 2;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

bool grid_ok(const cfp_ctx* g) { return g && g->classified && g->type; }

}  // namespace

// ------------------------------------------------------------------- C ABI
extern "C" {

int64_t cfp_unet_param_count(void) { return param_count(); }

cfp_status cfp_unet_create(cfp_ctx* ctx, uint64_t seed, cfp_unet** out) {
    if (!ctx || !out) return fail(CFP_EINVAL, "cfp_unet_create: NULL argument");
    cfp_unet* u = new cfp_unet();
    u->owner = ctx;
    u->np = param_count();
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        u->woff[l] = off;
        off += wcount(l);
        u->boff[l] = off;
        off += kDef[l].cout;
    }
    u->part_cap = 8 * 1024 * 1024;  // floats of weight-gradient partials
    bool ok = cudaMalloc(&u->w32, u->np * 4) == cudaSuccess && cudaMalloc(&u->g32, u->np * 4) == cudaSuccess &&
              cudaMalloc(&u->m32, u->np * 4) == cudaSuccess && cudaMalloc(&u->v32, u->np * 4) == cudaSuccess &&
              cudaMalloc(&u->wbf, u->np * 2) == cudaSuccess && cudaMalloc(&u->wpk, 27 * 128 * 128 * 2) == cudaSuccess &&
              cudaMalloc(&u->part, u->part_cap * 4) == cudaSuccess &&
              cudaMalloc(&u->bpart, kColBlocks * 128 * 4) == cudaSuccess &&
              cudaMalloc(&u->lpart, 256 * 4) == cudaSuccess && cudaMalloc(&u->dscal, 4 * 8) == cudaSuccess &&
              cudaMalloc(&u->dmax, 8) == cudaSuccess && cudaMalloc(&u->dcount, 4) == cudaSuccess &&
              cudaMalloc(&u->derr, 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cfp_unet_destroy(u);
        return fail(CFP_ENOMEM, "device allocation failed for the network");
    }
    // He initialisation from a seeded host generator; the linear layers
    // feeding the up path and the output start small
    std::vector<float> h(u->np, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    for (int l = 0; l < kLayers; ++l) {
        const float sd = sqrtf(2.f / (27.f * kDef[l].cin)) * (kDef[l].relu ? 1.f : 0.5f) * (l == kLayers - 1 ? 0.2f : 1.f);
        for (int64_t e = 0; e < wcount(l); ++e) h[u->woff[l] + e] = sd * nd(rng);
        if (l == kLayers - 1)  // only output channel 0 is used
            for (int64_t e = 27 * kDef[l].cin; e < wcount(l); ++e) h[u->woff[l] + e] = 0.f;
    }
    cudaStream_t s = ctx->stream;
    if (cudaMemcpyAsync(u->w32, h.data(), u->np * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(u->g32, 0, u->np * 4, s) != cudaSuccess || cudaMemsetAsync(u->m32, 0, u->np * 4, s) != cudaSuccess ||
        cudaMemsetAsync(u->v32, 0, u->np * 4, s) != cudaSuccess || cudaMemsetAsync(u->derr, 0, 4, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cfp_unet_destroy(u);
        return fail(CFP_ECUDA, "network initialisation failed");
    }
    k_to_bf16<<<blocks(u->np), 256, 0, s>>>(u->np, u->w32, u->wbf);
    ctx->launches += 1;
    *out = u;
    return CFP_OK;
}

void cfp_unet_destroy(cfp_unet* u) {
    if (!u) return;
    if (u->owner) cudaStreamSynchronize(u->owner->stream);
    free_bufs(u);
    for (void* p : {(void*)u->w32, (void*)u->g32, (void*)u->m32, (void*)u->v32, (void*)u->wbf, (void*)u->wpk,
                    (void*)u->part, (void*)u->bpart, (void*)u->lpart, (void*)u->dscal, (void*)u->dmax,
                    (void*)u->dcount, (void*)u->derr})
        if (p) cudaFree(p);
    delete u;
}

cfp_status cfp_unet_get_params(cfp_unet* u, float* host, float* grads_host) {
    if (!u) return fail(CFP_EINVAL, "cfp_unet_get_params: NULL network");
    if (host) CFP_CUDA(cudaMemcpyAsync(host, u->w32, u->np * 4, cudaMemcpyDeviceToHost, ustream(u)));
    if (grads_host) CFP_CUDA(cudaMemcpyAsync(grads_host, u->g32, u->np * 4, cudaMemcpyDeviceToHost, ustream(u)));
    CFP_CUDA(cudaStreamSynchronize(ustream(u)));
    return CFP_OK;
}

cfp_status cfp_unet_set_params(cfp_unet* u, const float* host) {
    if (!u || !host) return fail(CFP_EINVAL, "cfp_unet_set_params: NULL argument");
    CFP_CUDA(cudaMemcpyAsync(u->w32, host, u->np * 4, cudaMemcpyHostToDevice, ustream(u)));
    CFP_CUDA(cudaMemsetAsync(u->g32, 0, u->np * 4, ustream(u)));
    k_to_bf16<<<blocks(u->np), 256, 0, ustream(u)>>>(u->np, u->w32, u->wbf);
    u->owner->launches += 1;
    CFP_CUDA(cudaStreamSynchronize(ustream(u)));
    return CFP_OK;
}

cfp_status cfp_unet_forward_raw(cfp_unet* u, int nx, int ny, int nz, const uint16_t* x_dev, const float* target_dev,
                                const float* mask_dev, int count, float* y_dev, double* loss_host) {
    if (!u || !x_dev || nx < 3 || ny < 3 || nz < 3) return fail(CFP_EINVAL, "cfp_unet_forward_raw: bad argument");
    const bool train = target_dev != nullptr;
    if (train && (!mask_dev || count <= 0)) return fail(CFP_EINVAL, "cfp_unet_forward_raw: mask and count needed");
    CFP_TRY(ensure_grid(u, nx, ny, nz, train));
    cudaStream_t s = ustream(u);
    const Pad& P = u->L[0];
    CFP_CUDA(cudaMemcpyAsync(u->X, x_dev, (size_t)P.Np * 32, cudaMemcpyDeviceToDevice, s));
    CFP_TRY(forward(u));
    if (y_dev) CFP_CUDA(cudaMemcpyAsync(y_dev, u->Y, (size_t)P.Np * 64, cudaMemcpyDeviceToDevice, s));
    if (train) {
        CFP_CUDA(cudaMemcpyAsync(u->T, target_dev, (size_t)P.Np * 4, cudaMemcpyDeviceToDevice, s));
        CFP_CUDA(cudaMemcpyAsync(u->M, mask_dev, (size_t)P.Np * 4, cudaMemcpyDeviceToDevice, s));
        CFP_CUDA(cudaMemcpyAsync(u->dcount, &count, sizeof(int), cudaMemcpyHostToDevice, s));
        CFP_TRY(loss_grad(u));
        CFP_TRY(backward(u));
        if (loss_host) CFP_CUDA(cudaMemcpyAsync(loss_host, u->dscal + 2, 8, cudaMemcpyDeviceToHost, s));
    }
    return check_err(u);
}

cfp_status cfp_unet_train_step(cfp_unet* u, cfp_ctx* g, const double* r_dev, const double* e_dev, double lr,
                               double* loss_host) {
    if (!u || !r_dev || !e_dev) return fail(CFP_EINVAL, "cfp_unet_train_step: NULL argument");
    if (!grid_ok(g)) return fail(CFP_ESTATE, "cfp_unet_train_step: classify the grid's context first");
    CFP_TRY(ensure_grid(u, g->n[0], g->n[1], g->n[2], true));
    CFP_TRY(pack_input(u, g, r_dev, e_dev));
    CFP_TRY(forward(u));
    CFP_TRY(loss_grad(u));
    CFP_TRY(backward(u));
    CFP_TRY(adam_step(u, lr));
    if (loss_host) {
        CFP_CUDA(cudaMemcpyAsync(loss_host, u->dscal + 2, 8, cudaMemcpyDeviceToHost, ustream(u)));
        return check_err(u);
    }
    return CFP_OK;
}

cfp_status cfp_unet_apply(cfp_unet* u, cfp_ctx* g, const double* r_dev, double* z_dev) {
    if (!u || !r_dev || !z_dev) return fail(CFP_EINVAL, "cfp_unet_apply: NULL argument");
    if (!grid_ok(g)) return fail(CFP_ESTATE, "cfp_unet_apply: classify the grid's context first");
    CFP_TRY(ensure_grid(u, g->n[0], g->n[1], g->n[2], false));
    CFP_TRY(pack_input(u, g, r_dev, nullptr));
    CFP_TRY(forward(u));
    k_unet_output<<<blocks(g->N), 256, 0, ustream(u)>>>(g->type, u->L[0], g->n[0], g->n[1], g->N, u->Y, u->dscal + 1,
                                                      z_dev);
    u->owner->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

}  // extern "C"

namespace cfp {
// the stream a network's calls enqueue on (NULL: its context's); returns the previous one
cudaStream_t unet_use_stream(cfp_unet* u, cudaStream_t s) {
    cudaStream_t prev = u->stream;
    u->stream = s;
    return prev;
}
// kernels the network's calls launched so far (counted on its context)
int64_t unet_launches(const cfp_unet* u) { return u->owner->launches; }
cfp_ctx* unet_owner(const cfp_unet* u) { return u->owner; }
}  // namespace cfp

extern "C" {

cfp_status cfp_unet_check(cfp_unet* u) {
    if (!u) return fail(CFP_EINVAL, "cfp_unet_check: NULL network");
    return check_err(u);
}

// ---------------------------------------------- single kernels (parity tests)
cfp_status cfp_nn_conv3d(cfp_ctx* ctx, int nx, int ny, int nz, int cin, int cout, const uint16_t* in_dev,
                         const uint16_t* w_dev, const float* bias_dev, const uint16_t* act_dev, int flags,
                         void* out_dev) {
    if (!ctx || !in_dev || !w_dev || !out_dev || nx < 1 || ny < 1 || nz < 1)
        return fail(CFP_EINVAL, "cfp_nn_conv3d: bad argument");
    if (!supported(cin, cout)) return fail(CFP_EINVAL, "cfp_nn_conv3d: unsupported channel counts");
    if ((flags & CFP_NN_MASK) && !act_dev) return fail(CFP_EINVAL, "cfp_nn_conv3d: MASK needs act");
    const Pad P = make_pad(nx, ny, nz);
    if ((int64_t)(nx + 2) * (ny + 2) * (nz + 2) >= (int64_t)1 << 31) return fail(CFP_EINVAL, "cfp_nn_conv3d: grid too large");
    if (!ctx->dwait) {
        CFP_CUDA(cudaMalloc(&ctx->dwait, sizeof(int)));
        CFP_CUDA(cudaMemsetAsync(ctx->dwait, 0, sizeof(int), ctx->stream));
    }
    void* wpk = nullptr;
    CFP_CUDA(cudaMallocAsync(&wpk, (size_t)27 * cin * cout * 2, ctx->stream));
    const int f = (flags & CFP_NN_RELU ? F_RELU : 0) | (flags & CFP_NN_MASK ? F_MASK : 0) |
                  (flags & CFP_NN_OUT_F32 ? F_OUT_F32 : 0) | (flags & CFP_NN_ACCUM ? F_ACCUM : 0);
    cfp_status st = conv_any(ctx->stream, cin, cout, in_dev, w_dev, (flags & CFP_NN_DGRAD) != 0, (uint16_t*)wpk,
                             bias_dev, act_dev, P, f, out_dev, ctx->dwait);
    cudaFreeAsync(wpk, ctx->stream);
    ctx->launches += 2;
    if (st != CFP_OK) return st;
    return check_waits(ctx);
}

cfp_status cfp_nn_conv3d_wgrad(cfp_ctx* ctx, int nx, int ny, int nz, int cin, int cout, const uint16_t* in_dev,
                               const uint16_t* gout_dev, float* dw_dev, float* db_dev) {
    if (!ctx || !in_dev || !gout_dev || !dw_dev || nx < 1 || ny < 1 || nz < 1)
        return fail(CFP_EINVAL, "cfp_nn_conv3d_wgrad: bad argument");
    if (!supported(cin, cout)) return fail(CFP_EINVAL, "cfp_nn_conv3d_wgrad: unsupported channel counts");
    const Pad P = make_pad(nx, ny, nz);
    if (!ctx->dwait) {
        CFP_CUDA(cudaMalloc(&ctx->dwait, sizeof(int)));
        CFP_CUDA(cudaMemsetAsync(ctx->dwait, 0, sizeof(int), ctx->stream));
    }
    const int64_t cap = (int64_t)num_sms() * 27 * cin * cout;
    void *part = nullptr, *bpart = nullptr;
    CFP_CUDA(cudaMallocAsync(&part, cap * 4, ctx->stream));
    CFP_CUDA(cudaMallocAsync(&bpart, kColBlocks * 128 * 4, ctx->stream));
    cfp_status st = wgrad_any(ctx->stream, cin, cout, in_dev, gout_dev, P, (float*)part, cap, dw_dev, db_dev,
                              (float*)bpart, ctx->dwait);
    cudaFreeAsync(part, ctx->stream);
    cudaFreeAsync(bpart, ctx->stream);
    ctx->launches += db_dev ? 4 : 2;
    if (st != CFP_OK) return st;
    return check_waits(ctx);
}

cfp_status cfp_nn_transfer(cfp_ctx* ctx, int kind, int nx, int ny, int nz, int c, const uint16_t* a_dev,
                           const uint16_t* b_dev, const uint16_t* act_dev, uint16_t* out_dev) {
    if (!ctx || !a_dev || !out_dev || c % 8 != 0 || c <= 0 || nx < 3 || ny < 3 || nz < 3 || !(nx & 1) ||
        !(ny & 1) || !(nz & 1))
        return fail(CFP_EINVAL, "cfp_nn_transfer: bad argument (fine sizes must be odd)");
    const Pad F = make_pad(nx, ny, nz), C = coarser(F);
    cudaStream_t s = ctx->stream;
    switch (kind) {
    case CFP_NN_INJECT:
        k_inject<<<blocks((int64_t)C.Np * c / 8), 256, 0, s>>>(a_dev, F, out_dev, C, c);
        break;
    case CFP_NN_PROLONG_ADD:
        if (!b_dev) return fail(CFP_EINVAL, "cfp_nn_transfer: PROLONG_ADD needs the skip");
        k_prolong_add<<<blocks((int64_t)F.Np * c / 8), 256, 0, s>>>(a_dev, C, b_dev, F, out_dev, c);
        break;
    case CFP_NN_PROLONG_T:
        k_prolong_t<<<blocks((int64_t)C.Np * c / 8), 256, 0, s>>>(a_dev, F, out_dev, C, c);
        break;
    case CFP_NN_SKIP_GRAD:
        if (!b_dev || !act_dev) return fail(CFP_EINVAL, "cfp_nn_transfer: SKIP_GRAD needs gb and act");
        k_skip_grad<<<blocks((int64_t)F.Np * c / 8), 256, 0, s>>>(a_dev, b_dev, C, act_dev, F, out_dev, c);
        break;
    default:
        return fail(CFP_EINVAL, "cfp_nn_transfer: unknown kind");
    }
    ctx->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

}  // extern "C"
