// Kernels of the learned part (an extension of the method, not in the
// paper): a 3D convolutional U-Net on the solver's grid, BF16 activations
// and weights, FP32 accumulation in tensor memory (tcgen05).
//
// Layout.  A level of the network holds its activations on the level's grid
// padded by one node on every side (nxp = nx + 2, ...), channels last: channel
// c of padded voxel (i, j, k) at ((k nyp + j) nxp + i) C + c.  The padding
// nodes hold zeros, so a 3x3x3 convolution with zero padding reads, for the
// tap of offset (dx, dy, dz), the rows v + dx + nxp (dy + nyp dz) of the
// activation matrix: 128 consecutive output rows read 128 consecutive input
// rows.  Weights: [Cout][27][Cin], tap t for (dz, dy, dx) = (t/9 - 1,
// (t/3)%3 - 1, t%3 - 1):
//     out[v][co] = bias[co] + sum_t sum_ci W[co][t][ci] in[v + off(t)][ci].
//
// Forward convolution (k_conv_tc): the implicit GEMM D (128 voxels x Cout) =
// sum over taps of A_t (128 x Cin) B_t^T.  For each (dy, dz) pair one TMA
// window of 130 rows (the 128 outputs and one row either side) serves the
// three taps dx = -1, 0, 1, whose A operands start 0, 16 and 32 bytes into
// it (K-major, no swizzle).  The weights of the three taps come with it, in
// the operand layout (k_wpack).  The input gradient is the same kernel on
// flipped, transposed weights.  Weight gradient (k_wgrad_tc): D_t (Cin x
// Cout) = sum over voxels of X(v + off_t)^T G(v), both operands MN-major, the
// voxel shift again a start-address offset; per-chunk partials are summed in
// a fixed order (deterministic).
#pragma once

#include <cuda_bf16.h>

#include "cfp_tc.cuh"

namespace cfp {
namespace nn {

struct Pad {
    int nx, ny, nz;     // the level's grid
    int nxp, nyp, nzp;  // padded
    int Np;             // padded voxels (< 2^31)
};

enum { F_RELU = 1, F_MASK = 2, F_OUT_F32 = 4, F_ACCUM = 8 };

constexpr int kWin = 130;             // rows of a TMA window: 128 outputs + one either side
constexpr int kPlane = 136 * 16;      // bytes of one 8-channel plane of a window (128-byte multiple)
constexpr int kGPlane = 128 * 16;     // bytes of one 8-channel plane of a 128-voxel gradient tile
constexpr int kConvThreads = 192;     // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer

__host__ __device__ constexpr int pow2ceil(int v) {
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}
__host__ __device__ constexpr int rup(int v, int m) { return (v + m - 1) / m * m; }

__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) {
    const __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t*>(&b);
}
__device__ __forceinline__ bool bf_pos(uint16_t h) { return !(h & 0x8000u) && (h & 0x7fffu); }

__device__ __forceinline__ bool interior(const Pad& P, int row) {
    const int i = row % P.nxp, r = row / P.nxp, j = r % P.nyp, k = r / P.nyp;
    return i >= 1 && i <= P.nxp - 2 && j >= 1 && j <= P.nyp - 2 && k >= 1 && k <= P.nzp - 2;
}

// ------------------------------------------------------ forward convolution
template <int CIN, int COUT>
struct ConvCfg {
    static constexpr int KB = CIN < 64 ? CIN : 64;  // input channels per stage
    static constexpr int NKB = CIN / KB;
    static constexpr int NCH = KB / 8;              // 8-channel planes per stage
    static constexpr int A_BYTES = NCH * kPlane;
    static constexpr int W_TAP = NCH * COUT * 16;   // one tap's weights for the stage's channels
    static constexpr int W_BYTES = 3 * W_TAP;
    static constexpr int STAGE = rup(A_BYTES + W_BYTES, 128);
    static constexpr int S0 = (196 * 1024) / STAGE;
    static constexpr int STAGES = S0 < 2 ? 2 : (S0 > 8 ? 8 : S0);
    static constexpr int SPT = 9 * NKB;             // stages per 128-voxel tile
    static constexpr int TCOLS = pow2ceil(2 * COUT);  // two accumulators
    static constexpr int SMEM = 128 + STAGES * STAGE + (2 * STAGES + 5) * 8 + 16;
    static constexpr unsigned TX = NCH * kWin * 16 + W_BYTES;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 128, "channel counts");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Packed weights of a convolution for k_conv_tc: for stage (kb, g), g = 3
// (dz + 1) + (dy + 1), the taps dx = -1, 0, 1, each as NCH planes of COUT
// rows x 8 input channels (16 bytes): element (kb, g, dx, c, co, e) =
// W[co][3 g + dx + 1][kb KB + 8 c + e].  FLIP: the weights of the input
// gradient of a layer whose weights w are [CIN][27][COUT] (this kernel's
// COUT and CIN swapped): W'[co][t][ci] = w[ci][26 - t][co].
template <int CIN, int COUT, bool FLIP>
__global__ void k_wpack(const uint16_t* __restrict__ w, uint16_t* __restrict__ out) {
    using C = ConvCfg<CIN, COUT>;
    const int n = COUT * 27 * CIN;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        int r = e;
        const int el = r % 8;
        r /= 8;
        const int co = r % COUT;
        r /= COUT;
        const int c = r % C::NCH;
        r /= C::NCH;
        const int dx = r % 3;
        r /= 3;
        const int g = r % 9;
        const int kb = r / 9;
        const int t = 3 * g + dx;
        const int ci = kb * C::KB + 8 * c + el;
        out[e] = FLIP ? w[((int64_t)ci * 27 + (26 - t)) * COUT + co] : w[((int64_t)co * 27 + t) * CIN + ci];
    }
}

// out (Np x COUT) = epilogue(conv(in, W) + bias): RELU max(., 0); MASK times
// [act > 0]; ACCUM adds the values already in out (BF16); OUT_F32 FP32
// output.  Padding rows get 0.  Bounded waits: a wait that runs out records
// a code in *err and that role stops issuing; every issued copy and MMA is
// waited for (bounded) before the tensor memory is released.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap t_in, const uint16_t* __restrict__ wpk,
              const float* __restrict__ bias, const uint16_t* __restrict__ act, Pad P, int flags,
              uint16_t* __restrict__ out_bf, float* __restrict__ out_f, int* __restrict__ err) {
    using C = ConvCfg<CIN, COUT>;
    constexpr int S = C::STAGES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t* full = (uint64_t*)(base + S * C::STAGE);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;  // accumulator b filled
    uint64_t* acce = accf + 2;   // accumulator b read out by the four epilogue warps
    uint64_t* fin = acce + 2;    // every MMA of this CTA completed
    unsigned* tslot = (unsigned*)(fin + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&accf[q], 1);
            tc::mbar_init(&acce[q], 4);
        }
        tc::mbar_init(fin, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc<C::TCOLS>(tslot);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = *tslot;
    const int ntiles = (P.Np + 127) / 128;

    if (warp == 4 && lane == 0) {  // TMA producer
        unsigned g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int s = 0; s < C::SPT; ++s, ++g) {
                const int kb = s / 9, gi = s % 9, st = g % S;
                if (g >= S && !tc::mbar_wait(&empty[st], ((g / S) - 1) & 1)) {
                    ok = false;
                    atomicExch(err, 11);
                    break;
                }
                unsigned char* buf = base + st * C::STAGE;
                tc::mbar_arrive_expect_tx(&full[st], C::TX);
                const int row0 = tile * 128 + ((gi / 3 - 1) * P.nyp + (gi % 3 - 1)) * P.nxp - 1;
#pragma unroll
                for (int c = 0; c < C::NCH; ++c) tc::tma_load_2d(buf + c * kPlane, &t_in, &full[st], (kb * C::NCH + c) * 8, row0);
                tc::bulk_load(buf + C::A_BYTES, wpk + (size_t)(kb * 9 + gi) * (C::W_BYTES / 2), C::W_BYTES, &full[st]);
            }
        }
        for (unsigned q = g > (unsigned)S ? g - S : 0; q < g; ++q)
            if (!tc::mbar_wait(&full[q % S], (q / S) & 1)) atomicExch(err, 12);
    } else if (warp == 5 && lane == 0) {  // MMA issuer
        constexpr unsigned idesc = tc::idesc_bf16(128, COUT, 0, 0);
        unsigned g = 0, tl = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++tl) {
            const unsigned b = tl & 1;
            if (tl >= 2 && !tc::mbar_wait(&acce[b], ((tl / 2) - 1) & 1)) {
                ok = false;
                atomicExch(err, 13);
                break;
            }
            tc::fence_after();
            const unsigned d = tmem + b * COUT;
            for (int s = 0; s < C::SPT; ++s, ++g) {
                const int st = g % S;
                if (!tc::mbar_wait(&full[st], (g / S) & 1)) {
                    ok = false;
                    atomicExch(err, 14);
                    break;
                }
                tc::fence_after();
                const unsigned ab = tc::smem_u32(base + st * C::STAGE), wb = ab + C::A_BYTES;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int q = 0; q < C::NCH / 2; ++q) {
                        const uint64_t da = tc::sdesc(ab + dx * 16 + q * 2 * kPlane, kPlane, 128);
                        const uint64_t db = tc::sdesc(wb + dx * C::W_TAP + q * 2 * COUT * 16, COUT * 16, 128);
                        tc::mma_bf16(d, da, db, idesc, (s | dx | q) != 0);
                    }
                tc::mma_commit(&empty[st]);
            }
            if (!ok) break;
            tc::mma_commit(&accf[b]);
        }
        tc::mma_commit(fin);
        if (!tc::mbar_wait(fin, 0)) atomicExch(err, 15);
    } else if (warp < 4) {  // epilogue: warp w reads tensor-memory lanes 32w .. 32w + 31
        unsigned tl = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
            const unsigned b = tl & 1;
            int ok = 1;
            if (lane == 0 && !tc::mbar_wait(&accf[b], (tl / 2) & 1)) {
                ok = 0;
                atomicExch(err, 16);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc::fence_after();
            const int row = tile * 128 + 32 * warp + lane;
            const bool valid = row < P.Np;
            const bool in = valid && interior(P, row);
#pragma unroll 1
            for (int c16 = 0; c16 < COUT / 16; ++c16) {
                float v[16];
                tc::tmem_ld16(tmem + ((unsigned)(32 * warp) << 16) + b * COUT + 16 * c16, v);
                if (!valid) continue;
                const int c0 = 16 * c16;
                if (!in) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0.f;
                } else {
                    uint16_t am[16], ac[16];
                    if (flags & F_MASK) {
                        const uint4* ap = reinterpret_cast<const uint4*>(act + (size_t)row * COUT + c0);
                        *reinterpret_cast<uint4*>(am) = ap[0];
                        *reinterpret_cast<uint4*>(am + 8) = ap[1];
                    }
                    if ((flags & F_ACCUM) && !(flags & F_OUT_F32)) {
                        const uint4* op = reinterpret_cast<const uint4*>(out_bf + (size_t)row * COUT + c0);
                        *reinterpret_cast<uint4*>(ac) = op[0];
                        *reinterpret_cast<uint4*>(ac + 8) = op[1];
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        float x = v[q] + (bias ? __ldg(bias + c0 + q) : 0.f);
                        if (flags & F_RELU) x = fmaxf(x, 0.f);
                        if ((flags & F_MASK) && !bf_pos(am[q])) x = 0.f;
                        if ((flags & F_ACCUM) && !(flags & F_OUT_F32)) x += bf2f(ac[q]);
                        v[q] = x;
                    }
                }
                if (flags & F_OUT_F32) {
                    float4* op = reinterpret_cast<float4*>(out_f + (size_t)row * COUT + c0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        if (flags & F_ACCUM) {
                            const float4 p = op[q];
                            o.x += p.x;
                            o.y += p.y;
                            o.z += p.z;
                            o.w += p.w;
                        }
                        op[q] = o;
                    }
                } else {
                    uint16_t h[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) h[q] = f2bf(v[q]);
                    uint4* op = reinterpret_cast<uint4*>(out_bf + (size_t)row * COUT + c0);
                    op[0] = *reinterpret_cast<uint4*>(h);
                    op[1] = *reinterpret_cast<uint4*>(h + 8);
                }
            }
            tc::fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[b]);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free<C::TCOLS>(tmem);
    }
}

// ------------------------------------------------------- weight gradient
template <int CIN, int COUT>
struct WgCfg {
    static constexpr int NCA = CIN / 8;                    // planes of the X window
    static constexpr int NCB = COUT / 8;                   // planes of the gradient tile
    static constexpr int A_BYTES = NCA * kPlane;
    static constexpr int B_BYTES = NCB * kGPlane;
    static constexpr int STAGE = rup(A_BYTES + B_BYTES, 128);
    static constexpr int G0 = 512 / (3 * COUT);
    static constexpr int GMAX = G0 > 9 ? 9 : G0;           // (dy, dz) pairs per CTA
    static constexpr int NSETS = (9 + GMAX - 1) / GMAX;
    static constexpr int TCOLS = pow2ceil(3 * GMAX * COUT);
    // the MMA reads all 16 M planes of a window (128 rows; rows >= CIN are
    // discarded): the space after the last stage is reserved for them
    static constexpr int OVER = 16 * kPlane > STAGE ? 16 * kPlane - STAGE : 0;
    static constexpr int S0 = (190 * 1024 - OVER) / STAGE;
    static constexpr int STAGES = S0 < 2 ? 2 : (S0 > 8 ? 8 : S0);
    static constexpr int SMEM0 = 128 + STAGES * STAGE + OVER + (2 * STAGES + 3) * 8 + 16;
    // at least half an SM's shared memory: one CTA per SM, as it takes all
    // 512 tensor-memory columns
    static constexpr int SMEM = SMEM0 > 116 * 1024 ? SMEM0 : 116 * 1024;
    static constexpr unsigned TX = NCA * kWin * 16 + NCB * 128 * 16;
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(TCOLS <= 512, "tensor memory");
};

// Partial weight gradient of one voxel chunk and one set of (dy, dz) pairs:
// part[chunk][t][ci][co] = sum over the chunk's 128-voxel tiles of
// X[v + off(t)][ci] G[v][co].  Grid: (NSETS, nchunks); chunk q owns tiles
// [q * tpc, min((q + 1) * tpc, ntiles)).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap t_x, const __grid_constant__ CUtensorMap t_g, Pad P, int tpc,
               float* __restrict__ part, int* __restrict__ err) {
    using C = WgCfg<CIN, COUT>;
    constexpr int S = C::STAGES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t* full = (uint64_t*)(base + S * C::STAGE + C::OVER);
    uint64_t* empty = full + S;
    uint64_t* accf = empty + S;
    uint64_t* fin = accf + 1;
    unsigned* tslot = (unsigned*)(fin + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int set = blockIdx.x, chunk = blockIdx.y;
    const int g0 = set * C::GMAX, g1 = min(9, g0 + C::GMAX), ng = g1 - g0;
    const int ntiles = (P.Np + 127) / 128;
    const int t0 = chunk * tpc, t1 = min(ntiles, t0 + tpc);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        tc::mbar_init(accf, 1);
        tc::mbar_init(fin, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) tc::tmem_alloc<C::TCOLS>(tslot);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = *tslot;
    const int nst = (t1 > t0 ? t1 - t0 : 0) * ng;

    if (warp == 4 && lane == 0) {  // TMA producer
        unsigned g = 0;
        for (; (int)g < nst; ++g) {
            const int tile = t0 + (int)g / ng, gi = g0 + (int)g % ng, st = g % S;
            if (g >= (unsigned)S && !tc::mbar_wait(&empty[st], ((g / S) - 1) & 1)) {
                atomicExch(err, 21);
                break;
            }
            unsigned char* buf = base + st * C::STAGE;
            tc::mbar_arrive_expect_tx(&full[st], C::TX);
            const int row0 = tile * 128 + ((gi / 3 - 1) * P.nyp + (gi % 3 - 1)) * P.nxp - 1;
#pragma unroll
            for (int c = 0; c < C::NCA; ++c) tc::tma_load_2d(buf + c * kPlane, &t_x, &full[st], 8 * c, row0);
#pragma unroll
            for (int c = 0; c < C::NCB; ++c)
                tc::tma_load_2d(buf + C::A_BYTES + c * kGPlane, &t_g, &full[st], 8 * c, tile * 128);
        }
        for (unsigned q = g > (unsigned)S ? g - S : 0; q < g; ++q)
            if (!tc::mbar_wait(&full[q % S], (q / S) & 1)) atomicExch(err, 22);
    } else if (warp == 5 && lane == 0) {  // MMA issuer
        constexpr unsigned idesc = tc::idesc_bf16(128, COUT, 1, 1);
        for (int g = 0; g < nst; ++g) {
            const int st = g % S, first = g < ng;  // the chunk's first tile: the accumulators start
            const int gl = g % ng;
            if (!tc::mbar_wait(&full[st], (g / S) & 1)) {
                atomicExch(err, 23);
                break;
            }
            tc::fence_after();
            const unsigned ab = tc::smem_u32(base + st * C::STAGE), bb = ab + C::A_BYTES;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const unsigned d = tmem + (unsigned)((gl * 3 + dx) * COUT);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint64_t da = tc::sdesc(ab + dx * 16 + q * 256, 128, kPlane);
                    const uint64_t db = tc::sdesc(bb + q * 256, 128, kGPlane);
                    tc::mma_bf16(d, da, db, idesc, !(first && q == 0));
                }
            }
            tc::mma_commit(&empty[st]);
        }
        tc::mma_commit(accf);
        tc::mma_commit(fin);
        if (!tc::mbar_wait(fin, 0)) atomicExch(err, 24);
    } else if (warp < 4 && 32 * warp < CIN) {  // epilogue: lane = input channel
        int ok = 1;
        if (nst > 0) {
            if (lane == 0 && !tc::mbar_wait(accf, 0)) {
                ok = 0;
                atomicExch(err, 25);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (ok) {
            tc::fence_after();
            const int ci = 32 * warp + lane;
            for (int gl = 0; gl < ng; ++gl)
                for (int dx = 0; dx < 3; ++dx) {
                    const int t = 3 * (g0 + gl) + dx;
#pragma unroll 1
                    for (int c16 = 0; c16 < COUT / 16; ++c16) {
                        float v[16];
                        tc::tmem_ld16(tmem + ((unsigned)(32 * warp) << 16) + (unsigned)((gl * 3 + dx) * COUT + 16 * c16), v);
                        if (ci < CIN) {
                            float4* op = reinterpret_cast<float4*>(
                                part + (((size_t)chunk * 27 + t) * CIN + ci) * COUT + 16 * c16);
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                op[q] = nst > 0 ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3])
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free<C::TCOLS>(tmem);
    }
}

}  // namespace nn
}  // namespace cfp
