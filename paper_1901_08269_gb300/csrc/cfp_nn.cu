// The learned part: a small 3x3x3 convolutional network on the solver's grid,
// BF16 activations and weights with FP32 accumulation on the tensor cores
// (mma.sync m16n8k16), trained by its own forward and backward kernels.
//
// Layout: an activation is (N, 16) BF16, channels last, node (i, j, k) of the
// grid at row i + nx (j + ny k); weights are (16, 27, 16) BF16 as
// [co][tap][ci], tap t for the offset (dz, dy, dx) = (t/9 - 1, (t/3)%3 - 1,
// t%3 - 1), zero padding outside the grid:
//     out[v, co] = bias[co] + sum_t sum_ci W[co, t, ci] in[v + off(t), ci].
// Every layer is 16 -> 16 channels (unused channels hold zero weights), so one
// k-step of the implicit GEMM is one tap.
#include <cuda_bf16.h>
#include <string.h>

#include "cfp_internal.cuh"
#include "../../include/cfp_nn.h"

namespace cfp {
namespace {

constexpr int kC = 16;          // channels of every activation
constexpr int kTaps = 27;
constexpr int kWarps = 4;       // warps per CTA; a warp owns 16 consecutive x of one row

__device__ __forceinline__ uint32_t ld_pair(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) {
    const __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<const uint16_t*>(&b);
}

// D = A B + D for one m16n8k16 tile: A 16x16 BF16 row-major (4 registers of
// two values), B 16x8 BF16 column-major (2 registers), D 16x8 FP32.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Convolution of (N, 16) BF16 into (N, 16): the GEMM rows are the warp's 16
// voxels, the columns the 16 output channels (two n-tiles of 8), the k-steps
// the 27 taps of 16 input channels.  Lane (g = lane / 4, q = lane % 4) holds
// the voxel rows g and g + 8 and the channel pairs 2q and 2q + 8.  The
// layer's weights are staged in shared memory once per CTA; the tap loop is
// unrolled so the gathers of several taps are in flight together.
// Epilogue: + bias, ReLU, or (dgrad) multiplication by [act > 0].
template <bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(32 * kWarps)
    k_nn_conv(const uint16_t* __restrict__ in, const uint16_t* __restrict__ w, const float* __restrict__ bias,
              const uint16_t* __restrict__ act, int nx, int ny, int nz, uint16_t* __restrict__ out_bf,
              float* __restrict__ out_f) {
    // the layer's weights, staged once per CTA (16-byte copies)
    __shared__ __align__(16) uint16_t ws[kC * kTaps * kC];
    for (int e = threadIdx.x; e < kC * kTaps * kC / 8; e += blockDim.x)
        reinterpret_cast<uint4*>(ws)[e] = reinterpret_cast<const uint4*>(w)[e];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int ntx = (nx + 15) / 16;
    const int64_t tile = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (tile >= (int64_t)ntx * ny * nz) return;
    const int tx = (int)(tile % ntx), row = (int)(tile / ntx);
    const int y = row % ny, z = row / ny;
    const int g = lane >> 2, q = lane & 3;
    const int x0 = tx * 16;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 9
    for (int t = 0; t < kTaps; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const int ys = y + dy, zs = z + dz;
        const bool rowin = ys >= 0 && ys < ny && zs >= 0 && zs < nz;
        const int xa = x0 + g + dx, xb = x0 + g + 8 + dx;
        const bool va = rowin && xa >= 0 && xa < nx && x0 + g < nx;
        const bool vb = rowin && xb >= 0 && xb < nx && x0 + g + 8 < nx;
        const int64_t base = ((int64_t)zs * ny + ys) * nx;
        const uint16_t* pa = in + (base + xa) * kC + 2 * q;
        const uint16_t* pb = in + (base + xb) * kC + 2 * q;
        const uint32_t a0 = va ? ld_pair(pa) : 0u, a1 = vb ? ld_pair(pb) : 0u;
        const uint32_t a2 = va ? ld_pair(pa + 8) : 0u, a3 = vb ? ld_pair(pb + 8) : 0u;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const uint16_t* pw = ws + ((nt * 8 + g) * kTaps + t) * kC + 2 * q;
            mma_bf16(acc[nt], a0, a1, a2, a3, ld_pair(pw), ld_pair(pw + 8));
        }
    }
    const int64_t vrow = ((int64_t)z * ny + y) * nx;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int x = x0 + g + 8 * half;
        if (x >= nx) continue;
        const int64_t v = vrow + x;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int co = nt * 8 + 2 * q;
            float r0 = acc[nt][2 * half], r1 = acc[nt][2 * half + 1];
            if (bias) {
                r0 += bias[co];
                r1 += bias[co + 1];
            }
            if (RELU) {
                r0 = fmaxf(r0, 0.f);
                r1 = fmaxf(r1, 0.f);
            }
            if (act) {  // ReLU backward: the gradient passes where the activation is positive
                const uint32_t m = ld_pair(act + v * kC + co);
                if (!(bf2f((uint16_t)(m & 0xffffu)) > 0.f)) r0 = 0.f;
                if (!(bf2f((uint16_t)(m >> 16)) > 0.f)) r1 = 0.f;
            }
            if (OUT_F32) {
                out_f[v * kC + co] = r0;
                out_f[v * kC + co + 1] = r1;
            } else {
                *reinterpret_cast<uint32_t*>(out_bf + v * kC + co) = pack2(f2bf(r0), f2bf(r1));
            }
        }
    }
}

// wf[ci][26 - t][co] = w[co][t][ci]: the input gradient is the convolution
// of the output gradient with the mirrored, transposed weights
__global__ void k_nn_flip(const uint16_t* __restrict__ w, uint16_t* __restrict__ wf) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kC * kTaps * kC; e += gridDim.x * blockDim.x) {
        const int co = e / (kTaps * kC), t = (e / kC) % kTaps, ci = e % kC;
        wf[(ci * kTaps + (kTaps - 1 - t)) * kC + co] = w[e];
    }
}

// dW[co][t][ci] += sum_v dout[v, co] in[v + off(t), ci] for tap t =
// blockIdx.y: per warp a GEMM with rows co (A = dout^T, 16 x 16 voxels),
// columns ci (B = the tap's shifted input, 16 voxels x 8, two n-tiles) and
// k-steps over the row tiles of the forward kernel (16 consecutive x of one
// row); the warp's sums go to dW with atomics.
__global__ void __launch_bounds__(32 * kWarps)
    k_nn_wgrad(const uint16_t* __restrict__ in, const uint16_t* __restrict__ dout, int nx, int ny, int nz,
               float* __restrict__ dw) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const int t = blockIdx.y;
    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
    const int ntx = (nx + 15) / 16;
    const int64_t tiles = (int64_t)ntx * ny * nz;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int64_t s = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); s < tiles; s += (int64_t)gridDim.x * kWarps) {
        const int tx = (int)(s % ntx), row = (int)(s / ntx);
        const int y = row % ny, z = row / ny;
        const int ys = y + dy, zs = z + dz;
        const bool rowin = ys >= 0 && ys < ny && zs >= 0 && zs < nz;
        const int64_t vrow = ((int64_t)z * ny + y) * nx, srow = ((int64_t)zs * ny + ys) * nx;
        // the four voxels of this lane: x = 16 tx + 2q + {0, 1, 8, 9}
        uint16_t d[4][2];  // dout of channels g and g + 8
        int64_t src[4];    // v + off(t), or -1 outside the grid
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = 16 * tx + 2 * q + (u & 1) + 8 * (u >> 1);
            src[u] = -1;
            d[u][0] = d[u][1] = 0;
            if (x < nx) {
                const int64_t v = vrow + x;
                d[u][0] = dout[v * kC + g];
                d[u][1] = dout[v * kC + g + 8];
                if (rowin && x + dx >= 0 && x + dx < nx) src[u] = srow + x + dx;
            }
        }
        const uint32_t a0 = pack2(d[0][0], d[1][0]), a1 = pack2(d[0][1], d[1][1]);
        const uint32_t a2 = pack2(d[2][0], d[3][0]), a3 = pack2(d[2][1], d[3][1]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int ci = nt * 8 + g;
            uint16_t b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = src[u] >= 0 ? in[src[u] * kC + ci] : (uint16_t)0;
            mma_bf16(acc[nt], a0, a1, a2, a3, pack2(b[0], b[1]), pack2(b[2], b[3]));
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int co = g + 8 * (r >> 1), ci = nt * 8 + 2 * q + (r & 1);
            atomicAdd(&dw[(co * kTaps + t) * kC + ci], acc[nt][r]);
        }
}

// db[c] += sum_v dout[v, c]; the grid-stride step is a multiple of 16, so a
// thread always meets the same channel
__global__ void k_nn_bias_grad(const uint16_t* __restrict__ dout, int64_t n16, float* __restrict__ db) {
    float s = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n16; e += stride) s += bf2f(dout[e]);
    atomicAdd(&db[threadIdx.x % kC], s);
}

// max |r| over the unknowns, as the bit pattern of a non-negative float (the
// order of such patterns is the order of the values)
__global__ void k_nn_maxabs(const uint8_t* __restrict__ type, const double* __restrict__ r, int64_t n,
                            unsigned* __restrict__ out) {
    float m = 0.f;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (type[v] == CFP_REGULAR || type[v] == CFP_IRREGULAR) m = fmaxf(m, (float)fabs(r[v]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// network input: channel 0 = scale * r, channel 1 = 1 at the unknowns; target
// = escale * e at the unknowns (0 elsewhere) and the unknowns' mask
__global__ void k_nn_pack(const uint8_t* __restrict__ type, const double* __restrict__ r,
                          const double* __restrict__ e, double scale, double escale, int64_t n,
                          uint16_t* __restrict__ x, float* __restrict__ target, float* __restrict__ mask) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const bool unk = type[v] == CFP_REGULAR || type[v] == CFP_IRREGULAR;
        uint32_t* row = reinterpret_cast<uint32_t*>(x + v * kC);
        row[0] = pack2(f2bf(unk ? (float)(scale * r[v]) : 0.f), f2bf(unk ? 1.f : 0.f));
        for (int c = 1; c < kC / 2; ++c) row[c] = 0u;
        if (target) target[v] = unk && e ? (float)(escale * e[v]) : 0.f;
        if (mask) mask[v] = unk ? 1.f : 0.f;
    }
}

// masked MSE of channel 0: dout = 2 mask (y - target) / count in channel 0,
// 0 elsewhere; the loss sum (before the division) in *loss
__global__ void k_nn_mse(const float* __restrict__ y, const float* __restrict__ target, const float* __restrict__ mask,
                         int64_t n, float inv_count, uint16_t* __restrict__ dout, double* __restrict__ loss) {
    double s = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const float d = (y[v * kC] - target[v]) * mask[v];
        s += (double)d * d;
        uint32_t* row = reinterpret_cast<uint32_t*>(dout + v * kC);
        row[0] = pack2(f2bf(2.f * d * inv_count), 0);
        for (int c = 1; c < kC / 2; ++c) row[c] = 0u;
    }
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s);
}

// Adam (Kingma & Ba, Algorithm 1) on FP32 master weights; writes the BF16
// copy and clears the gradient for the next accumulation
__global__ void k_nn_adam(int64_t n, float* __restrict__ w, float* __restrict__ gr, float* __restrict__ m,
                          float* __restrict__ v2, float lr, float b1, float b2, float c1, float c2, float eps,
                          uint16_t* __restrict__ wbf) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = gr[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v2[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v2[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wbf) wbf[i] = f2bf(wi);
        gr[i] = 0.f;
    }
}

// u = inv_scale * y (channel 0) at the unknowns, 0 elsewhere
__global__ void k_nn_unpack(const uint8_t* __restrict__ type, const float* __restrict__ y, double inv_scale,
                            int64_t n, double* __restrict__ u) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const bool unk = type[v] == CFP_REGULAR || type[v] == CFP_IRREGULAR;
        u[v] = unk ? inv_scale * (double)y[v * kC] : 0.0;
    }
}

unsigned blocks_for(int64_t n, int threads) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 8));
}

unsigned conv_blocks(const cfp_ctx* c) {
    const int64_t tiles = (int64_t)((c->n[0] + 15) / 16) * c->n[1] * c->n[2];
    return (unsigned)((tiles + kWarps - 1) / kWarps);
}

cfp_status need_classified_nn(cfp_ctx* c) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!c->classified) return fail(CFP_ESTATE, "classify the points first (the network reads the unknowns)");
    return CFP_OK;
}

}  // namespace
}  // namespace cfp

using namespace cfp;

extern "C" {

cfp_status cfp_nn_pack(cfp_ctx* c, const double* r, const double* e, double scale, double escale, uint16_t* x,
                       float* target, float* mask, double* scale_used) {
    CFP_TRY(need_classified_nn(c));
    if (!r || !x) return fail(CFP_EINVAL, "r_dev and x_dev are required");
    if (!(scale > 0.0)) {  // 1 / max |r| at the unknowns
        unsigned* dm = reinterpret_cast<unsigned*>(c->dtotal + 2);  // a free slot of the context's device scalars
        CFP_CUDA(cudaMemsetAsync(dm, 0, sizeof(unsigned), c->stream));
        k_nn_maxabs<<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->type, r, c->N, dm);
        c->launches += 1;
        unsigned h = 0;
        CFP_CUDA(cudaMemcpyAsync(&h, dm, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
        CFP_CUDA(cudaStreamSynchronize(c->stream));
        float mx;
        memcpy(&mx, &h, sizeof(float));
        scale = mx > 0.f ? 1.0 / (double)mx : 1.0;
    }
    if (scale_used) *scale_used = scale;
    k_nn_pack<<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->type, r, e, scale, scale * escale, c->N, x, target,
                                                             mask);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_nn_conv3d(cfp_ctx* c, const uint16_t* in, const uint16_t* w, const float* bias, int relu,
                         uint16_t* out_bf16, float* out_f32) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!in || !w || (!out_bf16 == !out_f32)) return fail(CFP_EINVAL, "in, w and exactly one output are required");
    const unsigned nb = conv_blocks(c);
    const int nx = c->n[0], ny = c->n[1], nz = c->n[2];
    cudaStream_t s = c->stream;
    if (out_f32) {
        if (relu) k_nn_conv<true, true><<<nb, 32 * kWarps, 0, s>>>(in, w, bias, nullptr, nx, ny, nz, nullptr, out_f32);
        else k_nn_conv<false, true><<<nb, 32 * kWarps, 0, s>>>(in, w, bias, nullptr, nx, ny, nz, nullptr, out_f32);
    } else {
        if (relu)
            k_nn_conv<true, false><<<nb, 32 * kWarps, 0, s>>>(in, w, bias, nullptr, nx, ny, nz, out_bf16, nullptr);
        else k_nn_conv<false, false><<<nb, 32 * kWarps, 0, s>>>(in, w, bias, nullptr, nx, ny, nz, out_bf16, nullptr);
    }
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_nn_conv3d_dgrad(cfp_ctx* c, const uint16_t* dout, const uint16_t* w, const uint16_t* act,
                               uint16_t* din) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!dout || !w || !din) return fail(CFP_EINVAL, "dout, w and din are required");
    if (!c->nn_wflip) CFP_CUDA(cudaMalloc(&c->nn_wflip, sizeof(uint16_t) * kC * kTaps * kC));
    uint16_t* wf = static_cast<uint16_t*>(c->nn_wflip);
    k_nn_flip<<<(kC * kTaps * kC + 255) / 256, 256, 0, c->stream>>>(w, wf);
    k_nn_conv<false, false><<<conv_blocks(c), 32 * kWarps, 0, c->stream>>>(dout, wf, nullptr, act, c->n[0], c->n[1],
                                                                          c->n[2], din, nullptr);
    c->launches += 2;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_nn_conv3d_wgrad(cfp_ctx* c, const uint16_t* in, const uint16_t* dout, float* dw, float* db) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!in || !dout || !dw) return fail(CFP_EINVAL, "in, dout and dw are required");
    const int64_t tiles = (int64_t)((c->n[0] + 15) / 16) * c->n[1] * c->n[2];
    const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((tiles + kWarps - 1) / kWarps, 152 * 2)), kTaps);
    k_nn_wgrad<<<grid, 32 * kWarps, 0, c->stream>>>(in, dout, c->n[0], c->n[1], c->n[2], dw);
    c->launches += 1;
    if (db) {
        k_nn_bias_grad<<<blocks_for(c->N * kC, 256), 256, 0, c->stream>>>(dout, c->N * kC, db);
        c->launches += 1;
    }
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_nn_mse(cfp_ctx* c, const float* y, const float* target, const float* mask, double inv_count,
                      uint16_t* dout, double* loss) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (!y || !target || !mask || !dout || !loss) return fail(CFP_EINVAL, "NULL argument");
    double* dl = reinterpret_cast<double*>(c->dtotal) + 3;  // a free slot of the context's device scalars
    CFP_CUDA(cudaMemsetAsync(dl, 0, sizeof(double), c->stream));
    k_nn_mse<<<blocks_for(c->N, 256), 256, 0, c->stream>>>(y, target, mask, c->N, (float)inv_count, dout, dl);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    double h = 0.0;
    CFP_CUDA(cudaMemcpyAsync(&h, dl, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CFP_CUDA(cudaStreamSynchronize(c->stream));
    *loss = h * inv_count;
    return CFP_OK;
}

cfp_status cfp_nn_adam(cfp_ctx* c, int64_t n, float* w, float* grad, float* m, float* v, int step, double lr,
                       uint16_t* w_bf16) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (n < 1 || step < 1 || !w || !grad || !m || !v) return fail(CFP_EINVAL, "bad Adam arguments");
    const double b1 = 0.9, b2 = 0.999;
    k_nn_adam<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, w, grad, m, v, (float)lr, (float)b1, (float)b2,
                                                         (float)(1.0 - std::pow(b1, step)),
                                                         (float)(1.0 - std::pow(b2, step)), 1e-8f, w_bf16);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

cfp_status cfp_nn_unpack(cfp_ctx* c, const float* y, double inv_scale, double* u) {
    CFP_TRY(need_classified_nn(c));
    if (!y || !u) return fail(CFP_EINVAL, "y_dev and u_dev are required");
    k_nn_unpack<<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->type, y, inv_scale, c->N, u);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}

}  // extern "C"
