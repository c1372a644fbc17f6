// cfp_assemble_rhs_noalloc: the right-hand side assembly without any device
// allocation.
//
// Who needs it: callers that cannot let a library call cudaMalloc.  Examples
// are applications whose device memory is owned by a pooling or caching
// allocator (a cudaMalloc outside the pool can fail once the pool holds the
// memory, and it synchronises the device), and loops with a fixed memory or
// latency budget.  cfp_assemble_rhs itself allocates the context's whole
// solver work space on first use (twelve fields, about 13 GB at 513^3), which
// such a caller may not have room for when it only wants the right-hand side.
//
// The scratch field this assembly needs (the box Dirichlet values spread on
// the grid, zero elsewhere) lives instead in a file-scope device array of
// kNoAllocMaxNodes doubles (32 MiB).  Every GPU that loads this library
// holds that array until the process exits.  All calls share it: the lift
// kernel rewrites every entry the next kernel reads, so nothing from an
// earlier call is used, but calls whose work overlaps on the GPU (two streams
// or two host threads at once) race on it.
//
// Host code may not hand the array's name to a kernel (that is a host-side
// stand-in, not a device address).  The first call on each device therefore
// looks up the device address with cudaGetSymbolAddress, with that device
// current, and keeps it; make that first call before any stream capture.
#include <algorithm>
#include <mutex>
#include <string>

#include "cfp_internal.cuh"

namespace cfp {
namespace {

constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 22;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_lift_scratch[kNoAllocMaxNodes];

std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_lift_scratch on the current device (set-up once per
// device).
cfp_status scratch_address(double** out) {
    int dev = 0;
    CFP_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CFP_EINVAL, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_lift_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return CFP_OK;
}

bool device_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// rhs = Q-bar f - (B gb) - script-B g_ibi at the unknowns, 0 elsewhere; on
// entry rhs holds B gb at the interior rows (written by the apply kernel).
__global__ void k_rhs_finish_inplace(Grid<double> G, const uint8_t* __restrict__ type,
                                     const int32_t* __restrict__ slot, const int32_t* __restrict__ bib_ptr,
                                     const int32_t* __restrict__ bib_idx, const double* __restrict__ bib_val,
                                     const double* __restrict__ f, const double* __restrict__ g_ibi,
                                     double* __restrict__ rhs, int64_t N) {
    const int nx = G.nx, ny = G.ny;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N; l += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t t = type[l];
        if (t != CFP_REGULAR && t != CFP_IRREGULAR) {
            rhs[l] = 0.0;
            continue;
        }
        const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / sz);
        const double Lx[3] = {G.ax[0].a[i], 1.0, G.ax[0].c[i]};
        const double Ly[3] = {G.ax[1].a[j], 1.0, G.ax[1].c[j]};
        const double Lz[3] = {G.ax[2].a[k], 1.0, G.ax[2].c[k]};
        double q = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int p = 0; p < 3; ++p)
                for (int o = 0; o < 3; ++o) {
                    const int64_t c = l + (o - 1) + (p - 1) * sy + (r - 1) * sz;
                    if (type[c] == CFP_SOLID) continue;
                    q += Lx[o] * Ly[p] * Lz[r] * f[c];
                }
        double v = q - rhs[l];
        if (t == CFP_IRREGULAR) {
            const int s = slot[l];
            for (int e = bib_ptr[s]; e < bib_ptr[s + 1]; ++e) v -= bib_val[e] * g_ibi[bib_idx[e]];
        }
        rhs[l] = v;
    }
}

}  // namespace
}  // namespace cfp

using namespace cfp;

extern "C" cfp_status cfp_assemble_rhs_noalloc(cfp_ctx* c, const double* f, const double* g, const double* gi,
                                               double* rhs) {
    if (!c) return fail(CFP_EINVAL, "null context");
    if (c->N > kNoAllocMaxNodes)
        return fail(CFP_EINVAL, "cfp_assemble_rhs_noalloc supports at most " + std::to_string(kNoAllocMaxNodes) +
                                    " grid nodes; this grid has " + std::to_string(c->N) +
                                    " (use cfp_assemble_rhs)");
    if (c->class_status != CFP_OK) return fail(c->class_status, "classification failed earlier");
    if (!c->classified) return fail(CFP_ESTATE, "call cfp_classify_points first");
    if (!f || !g || !rhs || (c->n_ibi > 0 && !gi)) return fail(CFP_EINVAL, "NULL field pointer");
    if (!device_pointer(f) || !device_pointer(g) || !device_pointer(rhs) || (c->n_ibi > 0 && !device_pointer(gi)))
        return fail(CFP_EINVAL, "fields must be device pointers");
    double* scratch = nullptr;
    CFP_TRY(scratch_address(&scratch));
    if (rhs == scratch) return fail(CFP_EINVAL, "rhs aliases the scratch array");
    launch_boundary_lift(c, g, scratch, c->stream);                                   // gb, every entry
    launch_apply<double>(c, scratch, rhs, nullptr, 0, nullptr, c->stream, nullptr);   // B gb (interior rows)
    const int64_t blocks = std::min<int64_t>((c->N + 255) / 256, 152 * 16);
    k_rhs_finish_inplace<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, c->stream>>>(
        grid_view<double>(c), c->type, c->slot, c->bib_ptr, c->bib_idx, c->bib_val, f,
        c->n_ibi ? gi : c->ibi_xyz, rhs, c->N);
    c->launches += 1;
    CFP_CUDA(cudaGetLastError());
    return CFP_OK;
}
