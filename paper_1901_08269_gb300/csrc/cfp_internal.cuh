// Internal declarations of the CUDA library behind include/cfp.h.
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is fetched from the CUDA driver at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/cfp.h"
#include "../../include/cfp_nn.h"

namespace cfp {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
cfp_status fail(cfp_status st, const std::string& msg);
cfp_status cuda_fail(cudaError_t e, const char* what);

#define CFP_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ::cfp::cuda_fail(e_, #call); \
    } while (0)

#define CFP_TRY(call)                          \
    do {                                       \
        cfp_status s_ = (call);                \
        if (s_ != CFP_OK) return s_;           \
    } while (0)

// ------------------------------------------------------------ device types
// Per-axis 1D grid metrics.  Compact (Eq. app_xxx): a, c, ar, br, cr with
// b = 1; second order (Eq. 2ndorder_coef): ka, kb, kc.  Entries 0 and n-1
// are zero.
template <class T>
struct Axis {
    const T* a;
    const T* c;
    const T* ar;
    const T* br;
    const T* cr;
    const T* ka;
    const T* kb;
    const T* kc;
};

template <class T>
struct Grid {
    Axis<T> ax[3];
    int nx, ny, nz;
};

// Irregular-point side data, indexed by the slot of the irregular point
// (its rank in ascending linear index).
template <class T>
struct Side {
    const int32_t* slot;      // N: slot of an irregular node, -1 otherwise
    const int32_t* corr_ptr;  // n_irr + 1: correction entries per slot
    const int32_t* corr_off;  // linear-index offsets of the entries
    const T* corr_val;        // coefficients added to the regular row
    const T* krow;            // 7 per slot: K diag, -x, +x, -y, +y, -z, +z
};

// Per-thread accumulator of a dot product.  FP64 operands sum in FP64.  FP32
// operands sum in FP32 with a compensated (Kahan) sum, converted to FP64 once
// per thread: no FP64 arithmetic per term (GB300 issues FP64 at 1/58 of the
// FP32 rate, which made the FP64 pipe the limit of the FP32 kernels) and no
// branch in the loop, with an error of a few FP32 roundings of the sum
// instead of one per term.
template <class T>
struct DotAcc;
template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x, double y) { s += x * y; }
    __device__ __forceinline__ double total() const { return s; }
};
template <>
struct DotAcc<float> {
    float s = 0.0f, c = 0.0f;  // running sum and its lost low-order part (negated)
    __device__ __forceinline__ void add(float x, float y) {
        const float v = fmaf(x, y, -c);
        const float t = s + v;
        c = (t - s) - v;
        s = t;
    }
    __device__ __forceinline__ double total() const { return (double)s - (double)c; }
};

// Device-resident scalars of one BiCGSTAB run (Algorithm 1).
struct KState {
    double rho, alpha, omega, beta;
    double sigma, ts, tt, rr, rho_new;
    double bnorm2;     // ||b||^2 of the system being solved
    double stop2;      // stop when rr <= stop2
    int iter, maxit;
    int flag;          // FLAG_*
    int execs;         // executed iteration bodies
};

enum { FLAG_RUN = 0, FLAG_CONV = 1, FLAG_BREAK = 2, FLAG_NAN = 3, FLAG_MAXIT = 4 };

// Device-resident scalars of one mixed-precision solve driven on the device
// (the refinement loop of a captured solve graph): the same quantities and
// decisions as the host-driven refinement loop.
struct RState {
    double b2;          // ||rhs||^2
    double r2;          // ||rhs - B x||^2 of the current iterate
    double rel;         // sqrt(r2 / b2)
    double prev;        // smallest rel so far
    double scale;       // 1 / sqrt(r2): the FP32 right-hand side's scaling
    double tol, inner_tol;
    int refinements, total, maxit, max_refine, max_restarts, stall;
    int status;         // cfp_status; RSTATE_RUN while the loop goes on
    int outer;          // refinement bodies executed
    long long inner_execs;  // BiCGSTAB bodies executed over all steps
};
constexpr int RSTATE_RUN = -1;

// First device error of the set-up kernels.
struct DevError {
    int code;    // cfp_status, 0 = none
    int lin;     // node where it happened
    int detail;  // kernel-specific
    int pad;
};

enum { DETAIL_OFFGRID = 1, DETAIL_FEWPOINTS = 2, DETAIL_SINGULAR = 3, DETAIL_BOXIBI = 4,
       DETAIL_OVERFLOW = 5, DETAIL_MISSINGIBI = 6 };

constexpr int kAX = 128;           // apply CTA: columns (threads) along x
constexpr int kApplyKC = 32;       // planes per apply CTA
constexpr int kUpdBlocks = 152 * 8;   // grid of the vector-update kernels
constexpr int kUpdThreads = 256;

// One level of the multigrid hierarchy of the preconditioner (level 0 is the
// fine grid, whose arrays belong to the context).
struct MgLevel {
    int n[3] = {0, 0, 0};
    int64_t N = 0;
    std::vector<double> X[3];
    double* coef64 = nullptr;  // 8 arrays per axis (only ka, kb, kc used)
    float* coef32 = nullptr;
    uint8_t* type = nullptr;   // natural layout (levels >= 1; level 0 uses the context's)
    // red-black split layout: node (i, j, k) of colour (i + j + k) & 1 sits at
    // entry (k * n[1] + j) * hp + (i >> 1) of its colour's array
    int hp = 0;                // entries per row of one colour, padded to 16 (rows of 64 bytes
                               // in FP32: TMA tensor maps need 16-byte row strides)
    int64_t Nh = 0;            // entries per colour array: hp * n[1] * n[2]
    uint8_t* stype = nullptr;  // split type, colour c at stype + c * Nh
    double* s64 = nullptr;     // split e0 e1 b0 b1 r0 (Nh each), FP64
    float* s32 = nullptr;      // the same in FP32; b holds NaN at every entry that is not an unknown
    void* pk64 = nullptr;      // packed (ka, kb, kc, 0) per index, x then y then z, FP64
    void* pk32 = nullptr;      // the same in FP32
    // transfers with the next coarser level, FP64 and FP32 copies: per fine
    // index of each axis (entries from off[d]) the packed interpolation
    // (wlo, whi, ilo), per coarse index of each axis (entries from coff[d])
    // the restriction weights of fine nodes 2I - 1, 2I, 2I + 1
    int64_t off[3] = {0, 0, 0};
    int64_t coff[3] = {0, 0, 0};
    void* ip64 = nullptr;
    void* ip32 = nullptr;
    void* rw64 = nullptr;
    void* rw32 = nullptr;
    // TMA-fed FP32 passes (levels with at least kTmaMinPairs pairs per row):
    // per colour c, maps of the other colour's e and of b at tm32[2 c + 0, 1],
    // the red e at tm32[4]; per pass kind (half-sweep, red residual, last
    // black half-sweep) the persistent grid (resident CTAs x SMs)
    int tma = 0;
    int tma_grid[3] = {0, 0, 0};
    CUtensorMap tm32[5];
    // The fused black-then-red pass (FP32, TMA levels) writes the red iterate
    // into a second red array (entry 5 Nh of s32); red_cur (host, set while
    // launches are issued) names the array that holds the current red values:
    // 0 the split array, 1 the second one.  tmalt: the maps of tm32[2] and
    // tm32[4] on the second array; tmp: the fused pass's maps (red e of each
    // array, black b, red b, with the fused pass's boxes).
    int red_cur = 0;
    int pair = 0;
    int pair_grid = 0;
    CUtensorMap tmalt[2];
    CUtensorMap tmp[4];
    // level 0: the irregular nodes of each colour (natural index, split
    // offset, slot, parity) in ascending natural index, colour c at fix +
    // c * n_irr, nfix[c] of them; fixrows + c * (n[1] n[2] + 1): per row
    // (k n[1] + j) the first entry of that row in colour c's list
    void* fix = nullptr;
    int32_t* fixrows = nullptr;
    int64_t nfix[2] = {0, 0};
};

}  // namespace cfp

// ------------------------------------------------------------------ context
// FP32 copy of a body for the certified sign of its level set (the
// classification's fast path): centre, rotation, parameters, reciprocal
// semi-axes (ellipsoid), and the threshold of the FP32 bounding-sphere test.
struct Body32 {
    float c[3], R[9], p[3], ip[3];
    float thr;
    int kind;
};

struct cfp_ctx {
    int n[3] = {0, 0, 0};
    int64_t N = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    // a second stream and two events: the apply forks its irregular rows
    // onto `aux` to run beside the regular rows, and joins back.  Three sets,
    // one per capture level of a device-driven solve (the graph, the
    // refinement body, the BiCGSTAB body); aux / ev_* are the set in use.
    cudaStream_t auxs[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t evfs[3] = {nullptr, nullptr, nullptr}, evjs[3] = {nullptr, nullptr, nullptr};
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<double> X[3];
    std::vector<cfp_body> bodies;
    int fluid_inside = 0;

    // grid metrics (device)
    double* dX[3] = {nullptr, nullptr, nullptr};
    double* dcoef64 = nullptr;  // 8 arrays per axis, n[d] each
    float* dcoef32 = nullptr;
    cfp_body* dbodies = nullptr;
    Body32* dbody32 = nullptr;  // per body: its FP32 copy for the certified level-set sign

    // classification and side data
    bool classified = false;
    cfp_status class_status = CFP_OK;
    uint8_t* type = nullptr;
    int32_t* slot = nullptr;
    int32_t* irr_lin = nullptr;
    int64_t n_irr = 0, n_ibi = 0, n_deg = 0, n_corr = 0, n_bib = 0;
    int32_t* ibi_off = nullptr;
    double* ibi_xyz = nullptr;
    int32_t* corr_ptr = nullptr;
    int32_t* corr_off = nullptr;
    double* corr_val = nullptr;
    float* corr_val32 = nullptr;
    int32_t* bib_ptr = nullptr;
    int32_t* bib_idx = nullptr;
    double* bib_val = nullptr;
    double* krow = nullptr;
    float* krow32 = nullptr;

    // side-list build scratch (per-slot slices), kept across classifications
    void* side_scratch = nullptr;
    void* nn_wflip = nullptr;      // learned part: mirrored, transposed weights of a layer
    size_t side_scratch_bytes = 0;

    // scan scratch
    int* scan_bsum = nullptr;
    int64_t scan_cap = 0;
    long long* dtotal = nullptr;   // device counters (8)
    cfp::DevError* derr = nullptr;

    // Krylov work space
    double* v64 = nullptr;    // kNV64 fields
    float* v32 = nullptr;     // kNV32 fields
    double* partial = nullptr;
    int64_t partial_cap = 0;
    cfp::KState* kst = nullptr;   // [0]: FP64 run, [1]: FP32 run
    cfp::KState* hkst = nullptr;  // pinned host mirror
    cfp::RState* rst = nullptr;   // device-driven refinement loop
    cfp::RState* hrst = nullptr;  // pinned host mirror

    // host-buffer solve
    double* hs_f = nullptr;
    double* hs_g = nullptr;
    double* hs_u = nullptr;
    double* hs_gi = nullptr;
    int64_t hs_gi_cap = 0;

    // kernels enqueued since the context was created
    int64_t launches = 0;
    // moves whenever a buffer or kernel choice that captured graphs hold is
    // replaced (classification, multigrid / ILU data freed, the partials
    // reallocated, a new apply shape): graphs of other objects recapture
    int64_t generation = 0;

    // the apply's kernel and tile shape per precision (0 FP64, 1 FP32):
    // CFP_APPLY_STREAM (rows per thread 2 or 4) or CFP_APPLY_RING (FP32, 8
    // rows per tile), planes per z chunk (16, 32 or 64); 0: the defaults (set
    // by the autotuner)
    int apply_kind[2] = {0, 0};
    int apply_ty[2] = {0, 0};
    int apply_kc[2] = {0, 0};

    // preconditioner of the current solve and its multigrid hierarchy
    int precond_kind = CFP_PRECOND_RBGS;
    int mg_smooth = 2;
    int mg_post = 2;
    int mg_tma = 1;            // 1: TMA-fed FP32 half-sweeps where a level supports them
    int mg_fuse = 0;           // 1: and the fused black-then-red passes (opts.mg_tma == 2)
    int* dwait = nullptr;      // device word: nonzero once a bounded pipeline wait timed out
    int ring_grid = 0;         // CTAs of the apply ring's persistent grid (0: not set up)
    std::vector<cfp::MgLevel> mg;
    // ILU(0) of K (CFP_PRECOND_ILU): [pivots | work field], FP64 and FP32
    double* ilu64 = nullptr;
    float* ilu32 = nullptr;

    // graphs: [precision][sweeps-config]
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gsweeps[2] = {-1, -1};
    int64_t ggen[2] = {-1, -1};
    int gprecond[2] = {-1, -1};
    int64_t body_launches = 0;
    int gmgs[2] = {-1, -1};
};

namespace cfp {

constexpr int kNV64 = 12;  // x r rh p ph v s sh t rhs tmp tmp2
// distance between two work fields in v64 / v32: N rounded up to 64 entries,
// so that every field starts 256-byte aligned (bulk copies want 16)
inline int64_t vstride(const cfp_ctx* c) { return (c->N + 63) / 64 * 64; }
// Stream-ordered allocation from the library's memory pool of the current
// device (freed blocks stay in the pool for reuse), for the buffers that a
// classification and the preconditioners' set-up replace: unlike cudaMalloc
// and cudaFree, neither synchronises the device, so contexts classify in
// parallel beside running work.  The memory is ordered on stream s.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);
template <class T>
inline cudaError_t pool_malloc(T** p, size_t bytes, cudaStream_t s) {
    return pool_malloc(reinterpret_cast<void**>(p), bytes, s);
}
inline void pool_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}
// selects the stream and events the apply forks its irregular rows onto
inline void use_aux(cfp_ctx* c, int q) {
    c->aux = c->auxs[q];
    c->ev_fork = c->evfs[q];
    c->ev_join = c->evjs[q];
}
constexpr int kNV32 = 9;   // x r rh p ph v s sh t
enum { V_X = 0, V_R, V_RH, V_P, V_PH, V_V, V_S, V_SH, V_T, V_RHS, V_TMP, V_TMP2 };

// geometry (cfp_geometry.cu)
cfp_status classify(cfp_ctx* c);

// stencils (cfp_stencil.cu)
template <class T>
Grid<T> grid_view(cfp_ctx* c);
template <>
Grid<double> grid_view<double>(cfp_ctx* c);
template <>
Grid<float> grid_view<float>(cfp_ctx* c);
template <class T>
Side<T> side_view(cfp_ctx* c);
template <>
Side<double> side_view<double>(cfp_ctx* c);
template <>
Side<float> side_view<float>(cfp_ctx* c);
void launch_apply_lift(cfp_ctx* c, const double* gb, double* y, cudaStream_t s);
template <class T>
void launch_apply(cfp_ctx* c, const T* x, T* y, const T* d0, int dotmode, double* partial,
                  cudaStream_t s, int* nblocks_out);
template <class T>
void launch_precond(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s);

// multigrid (cfp_mg.cu)
cfp_status ensure_mg(cfp_ctx* c, int prec);  // prec: 0 FP64 vectors, 1 FP32 vectors
void free_mg(cfp_ctx* c);
template <class T>
void launch_precond_mg(cfp_ctx* c, const T* rho, T* phi, cudaStream_t s);
// ILU(0)-Richardson inner iteration (cfp_ilu.cu)
cfp_status ensure_ilu(cfp_ctx* c, int prec);  // prec: 0 FP64, 1 FP32 (and FP64 pivots)
void free_ilu(cfp_ctx* c);
template <class T>
void launch_precond_ilu(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s);
// red-black sweeps from zero on the fine level's split vectors (the inner
// iterations of CFP_PRECOND_RBGS)
template <class T>
void launch_rbgs_split(cfp_ctx* c, int sweeps, const T* rho, T* phi, cudaStream_t s);
// one plain red half-sweep on the fine level's split vectors (timing aid)
template <class T>
void launch_mg_half_sweep(cfp_ctx* c, cudaStream_t s);
// the V-cycle's restriction / prolongation between levels 0 and 1 (false: one level only)
template <class T>
bool launch_mg_transfer(cfp_ctx* c, bool prolong, cudaStream_t s);
// the fused black-then-red pass on the fine level; false where it does not apply
template <class T>
bool launch_mg_pair(cfp_ctx* c, cudaStream_t s);
void launch_qf(cfp_ctx* c, const double* f, double* out, cudaStream_t s);
void launch_rhs_finish(cfp_ctx* c, const double* qf, const double* bg, const double* g_ibi,
                       double* rhs, cudaStream_t s);
void launch_boundary_lift(cfp_ctx* c, const double* g, double* gb, cudaStream_t s);
void launch_finish_solution(cfp_ctx* c, const double* x, const double* g, double* u, cudaStream_t s);
void launch_mask_unknowns(cfp_ctx* c, const double* in, double* out, cudaStream_t s);
int apply_blocks(cfp_ctx* c);  // partial pairs written by one launch_apply
int corr_blocks(const cfp_ctx* c);
void launch_metrics(cfp_ctx* c);  // Eq. app_xxx and Eq. 2ndorder_coef per axis

// Krylov (cfp_krylov.cu)
cfp_status ensure_work(cfp_ctx* c, bool need32);
cfp_status time_kernel(cfp_ctx* c, int kernel, int prec, int reps, double* ms, double* bytes);
cfp_status tune_apply(cfp_ctx* c, int prec, int kind, int rows, int planes, int reps, double* best_ms);
// the right-hand side of Eq. Bu=q without the argument checks of cfp_assemble_rhs
cfp_status assemble_rhs(cfp_ctx* c, const double* f, const double* g, const double* gi, double* rhs);
// sets up the FP32 apply ring (shared-memory limit, persistent grid); false if unusable
bool setup_apply_ring(cfp_ctx* c);
// the kernel and tile shape the apply of precision q (0 FP64, 1 FP32) runs with
void apply_shape(const cfp_ctx* c, int q, int* kernel, int* rows, int* planes);
// phi = P(rho) in FP32 (the mixed solve's inner preconditioner) for FP64
// fields: rho rounded to FP32, phi widened back; phi zeroed first
cfp_status precondition32(cfp_ctx* c, int sweeps, const double* rho, double* phi);
// the graph-cache key of the multigrid settings
int mg_key(const cfp_ctx* c);
// CFP_ECUDA (and the device word cleared) if a bounded pipeline wait of a
// kernel timed out since the last check; synchronises the stream
cfp_status check_waits(cfp_ctx* c);
// one CTA whose bounded mbarrier wait runs out (code 5), then check_waits
cfp_status diag_bounded_wait(cfp_ctx* c);
// learned part (cfp_unet.cu): the stream a network enqueues on (NULL: its
// context's), returning the previous one; its context's launch counter
cudaStream_t unet_use_stream(cfp_unet* u, cudaStream_t s);
int64_t unet_launches(const cfp_unet* u);
cfp_ctx* unet_owner(const cfp_unet* u);
// FP64 vector helpers over all N nodes: dot (synchronises), y = alpha x + beta y
cfp_status vec_dot(cfp_ctx* c, const double* a, const double* b, double* out);
cfp_status vec_axpby(cfp_ctx* c, double alpha, const double* x, double beta, double* y);

}  // namespace cfp
