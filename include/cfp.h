/*
 * cfp.h -- C ABI of the GB300 (sm_103a) fourth-order compact Poisson solver
 * with immersed Dirichlet bodies (Hosseinverdi & Fasel, arXiv 1901.08269).
 *
 * Problem (Sec. 1, Eq. poisson): Laplace(u) = f in the fluid region of the
 * box [x_1,x_nx] x [y_1,y_ny] x [z_1,z_nz]; u = g on the box faces and on
 * the body surfaces Gamma; u = 0 inside the bodies.
 *
 * Conventions shared by every entry point:
 *  - Grid: three strictly increasing coordinate arrays (Sec. 2).  Node
 *    (i,j,k), 0-based, has linear index i + nx*(j + ny*k) (x fastest).
 *    A "field" is an FP64 array of N = nx*ny*nz values in that order.
 *  - Pointers named *_dev are CUDA device pointers on the context's device
 *    (for instance torch CUDA tensors); *_host are host pointers.
 *  - The caller owns every array it passes; the context owns its internal
 *    buffers and frees them in cfp_ctx_destroy.
 *  - Calls are ordered on the context's stream.  Calls that return host
 *    values (counts, cfp_info) synchronise that stream before returning.
 *  - Errors: every call returns a cfp_status; no call aborts, traps or
 *    exits.  cfp_last_error() returns a message for the calling thread.
 *  - One context may be used by one host thread at a time.
 */
#ifndef CFP_H
#define CFP_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CFP_OK = 0,
    CFP_EINVAL = 1,      /* bad argument (size, pointer, non-monotone grid) */
    CFP_ENOMEM = 2,      /* device allocation failed                       */
    CFP_ECUDA = 3,       /* a CUDA runtime call failed                      */
    CFP_EGEOM = 4,       /* geometry outside what the stencils support      */
    CFP_ENOCONV = 5,     /* iteration cap reached before the tolerance      */
    CFP_EBREAKDOWN = 6,  /* BiCGSTAB breakdown persisted after restarts     */
    CFP_ENAN = 7,        /* non-finite value met in the solve               */
    CFP_ESTATE = 8       /* call out of order (e.g. solve before classify)  */
} cfp_status;

/* point types of Sec. 2, as written by cfp_classify_points */
enum { CFP_BOUNDARY = 0, CFP_REGULAR = 1, CFP_IRREGULAR = 2, CFP_SOLID = 3 };

/* implicit bodies: phi < 0 inside; a union of bodies takes the minimum */
enum { CFP_SPHERE = 0, CFP_ELLIPSOID = 1, CFP_TORUS = 2 };

typedef struct {
    int kind;      /* CFP_SPHERE, CFP_ELLIPSOID or CFP_TORUS                */
    double c[3];   /* centre                                               */
    double R[9];   /* row-major body-to-world rotation (identity if none);
                      must be orthonormal to 1e-9 (else CFP_EINVAL)        */
    double p[3];   /* sphere: radius; ellipsoid: semi-axes; torus: major
                      radius, minor radius (torus axis = body z axis)      */
} cfp_body;

enum { CFP_PREC_FP64 = 0,   /* the whole solve in FP64                       */
       CFP_PREC_MIXED = 1   /* FP32 inner BiCGSTAB inside FP64 iterative
                               refinement; residuals, the irregular rows of
                               the residual and the right-hand side in FP64 */ };

enum { CFP_PRECOND_RBGS = 0, /* `sweeps` red-black Gauss-Seidel sweeps on K from
                                zero (the paper's fixed count of inner
                                iterations, Sec. 3.3)                         */
       CFP_PRECOND_MG = 1,   /* one multigrid V-cycle on K from zero: red-black
                                smoothing (mg_smooth sweeps before, mg_post
                                after the coarse correction),
                                rediscretised coarse levels; quality
                                independent of the grid size                  */
       CFP_PRECOND_ILU = 2   /* `sweeps` Richardson sweeps from zero with ILU(0)
                                of K in natural order (the incomplete-
                                factorisation class of the paper's inner
                                solver, Sec. 3.3); each triangular solve is
                                n_x + n_y + n_z - 8 dependent launches, one
                                per hyperplane i + j + k = const: slow by
                                construction, for fidelity, not speed       */ };

typedef struct {
    int precision;     /* CFP_PREC_FP64 (default) or CFP_PREC_MIXED            */
    int sweeps;        /* inner iterations of the preconditioner solve with
                          CFP_PRECOND_RBGS or CFP_PRECOND_ILU (Sec. 3.3 uses
                          8; default 8)                                      */
    int maxit;         /* cap on BiCGSTAB iterations (default 50000)           */
    int max_restarts;  /* restarts after a breakdown or a failed true-residual
                          check (default 3)                                  */
    double inner_tol;  /* CFP_PREC_MIXED: relative residual reduction of each
                          FP32 inner solve (default 1e-5); a step that can
                          end the solve aims at 0.3 tol / (its starting
                          relative residual) instead, where that lies
                          between inner_tol / 8 and inner_tol                */
    int max_refine;    /* CFP_PREC_MIXED: cap on refinement steps (default 40) */
    int use_graph;     /* 1 (default): the iteration runs as one CUDA graph
                          with a device-side while loop; 0: plain launches   */
    int precond;       /* CFP_PRECOND_RBGS (default), CFP_PRECOND_MG or
                          CFP_PRECOND_ILU                                    */
    int mg_smooth;     /* CFP_PRECOND_MG: sweeps before the coarse correction
                          on each level, and after it unless mg_post is set
                          (default 2)                                       */
    int mg_post;       /* CFP_PRECOND_MG: sweeps after the coarse correction;
                          0 (default): mg_smooth                            */
    int mg_tma;        /* 1 (default): the FP32 red-black half-sweeps of the
                          multigrid levels (and of the fine level's sweeps)
                          with at least 192 nodes per row stream their tiles
                          through shared memory with TMA bulk-tensor copies,
                          a coarse level of at most 2^15 nodes does all
                          sweeps of a smoothing in one single-CTA launch,
                          and the prolongation runs one thread per coarse
                          cell; 0: plain loads, one launch per half-sweep,
                          one prolongation thread per fine pair; 2: as 1,
                          and on those levels the black half-sweep of each
                          sweep and the red half-sweep of the next run as
                          one fused pass (10 instead of 12 bytes per node
                          in FP32; measured slower than the two passes at
                          513^3, hence not the default).  Same arithmetic,
                          bitwise equal results                           */
} cfp_opts;

typedef struct {
    int status;            /* cfp_status of the solve                        */
    int iterations;        /* BiCGSTAB iterations over all restarts and
                              refinement steps                               */
    int restarts;
    int refinements;       /* CFP_PREC_MIXED outer steps                      */
    double rel_residual;   /* ||rhs - B u||_2 / ||rhs||_2, recomputed in FP64 */
    int64_t n_irregular;
    int64_t n_ibi;
    int64_t n_degenerate;  /* modified operators built with fewer points than
                              the paper's six (five) because a body or the box
                              ended the stencil early                        */
    double ms_setup, ms_rhs, ms_solve;  /* host wall time of each phase       */
    int64_t launches;      /* kernels this call launched (graph bodies counted
                              once per executed iteration)                   */
} cfp_info;

typedef struct cfp_ctx cfp_ctx;

/* Fill opts with the defaults listed above. */
void cfp_default_opts(cfp_opts* opts);

/* Message of the last failed call on this host thread ("" if none). */
const char* cfp_last_error(void);

/*
 * Create a context on the current CUDA device (Sec. 2 grid).
 *   x, y, z  host arrays of nx, ny, nz >= 3 strictly increasing coordinates
 *            (a_1 = x_1 < x_2 < ... < x_nx = a_2); copied.  N = nx*ny*nz
 *            must be below 2^31 (larger grids do not fit the GPU anyway).
 *   bodies   host array of nbodies >= 0 bodies; copied.
 *   fluid_inside  0: the fluid is outside the bodies (Omega^+ of Sec. 1);
 *            1: the fluid is the inside (interior problems, Problem 4).
 *   stream   cudaStream_t to enqueue on (NULL: the legacy default stream).
 *   out      receives the context.
 * Builds the 1D grid metrics of Eq. app_xxx and Eq. 2ndorder_coef.
 * Errors: CFP_EINVAL, CFP_ENOMEM, CFP_ECUDA.
 */
cfp_status cfp_ctx_create(const double* x, int nx, const double* y, int ny,
                          const double* z, int nz, const cfp_body* bodies,
                          int nbodies, int fluid_inside, void* stream,
                          cfp_ctx** out);

/* Release the context and every buffer it owns.  NULL is ignored. */
void cfp_ctx_destroy(cfp_ctx* ctx);

/*
 * Point classification (Sec. 2) and the set-up that depends on it: solid
 * points (inside a body, u = 0 by Sec. 1), irregular points (fluid points
 * with a solid point among their 26 neighbours), IBI points (Gamma cut by
 * the grid line between a fluid point and a solid axis neighbour), the
 * modified stencils of Secs. 2.2-2.3 at every irregular point and the
 * modified preconditioner rows of Sec. 3.3.
 *   type_dev     NULL or a device array of N bytes; receives CFP_BOUNDARY,
 *                CFP_REGULAR, CFP_IRREGULAR or CFP_SOLID per node.  Box
 *                nodes are CFP_BOUNDARY whatever phi says.
 *   n_irregular, n_ibi  NULL or host pointers receiving the counts.
 * The IBI points are ordered by (linear index of the fluid point, direction
 * -x,+x,-y,+y,-z,+z).  Synchronises.  Errors: CFP_EGEOM (a stencil that
 * would need a node outside the grid or more than the supported points, a
 * body touching the box), CFP_ENOMEM, CFP_ECUDA.
 */
cfp_status cfp_classify_points(cfp_ctx* ctx, uint8_t* type_dev,
                               int64_t* n_irregular, int64_t* n_ibi);

/*
 * Coordinates of the IBI points, where the caller evaluates g on Gamma
 * (Eq. bc uses u at the IBI points).
 *   xyz      device (on_host = 0) or host (on_host = 1) array of 3*n_ibi
 *            doubles, (x, y, z) per point in the order of cfp_classify_points.
 * Errors: CFP_ESTATE before classification, CFP_EINVAL, CFP_ECUDA.
 */
cfp_status cfp_ibi_points(cfp_ctx* ctx, double* xyz, int on_host);

/*
 * Right-hand side of Eq. Bu=q for every unknown (interior fluid node): the
 * source term of Eq. q with the weights of solid points dropped (Q-bar of
 * Eq. A27_mod), minus the IBI term of Eqs. bc / qb_case2, minus the box
 * Dirichlet values times their matrix entries.  Zero at box and solid nodes.
 *   f_dev        field, source f (values at solid nodes are not read)
 *   g_nodes_dev  field, Dirichlet data (only box nodes are read)
 *   g_ibi_dev    n_ibi values of g at the IBI points (may be NULL if n_ibi=0)
 *   rhs_dev      field, output
 * Errors: CFP_ESTATE, CFP_EINVAL, CFP_ECUDA.
 */
cfp_status cfp_assemble_rhs(cfp_ctx* ctx, const double* f_dev,
                            const double* g_nodes_dev, const double* g_ibi_dev,
                            double* rhs_dev);

/*
 * y = B x at every unknown (Eq. Bdec: the 27-point compact stencil of Eq.
 * A27 matrix-free plus the modified rows of the irregular points); y = 0 at
 * box and solid nodes.  x is read at all nodes (box values included), so
 * callers that want the operator on unknowns only pass x = 0 there.
 * x_dev and y_dev: fields, must not overlap.  Errors: CFP_ESTATE, CFP_EINVAL.
 */
cfp_status cfp_apply(cfp_ctx* ctx, const double* x_dev, double* y_dev);

/*
 * The same y = B x in FP32: the operator the mixed-precision solve's inner
 * iterations use (the 1D metrics and the irregular rows' weights rounded
 * from their FP64 values, FP32 arithmetic), in the tile shape the context
 * holds for CFP_PREC_MIXED (cfp_tune_apply).  x_dev, y_dev: N floats on the
 * device, must not overlap.  Synchronises (a timed-out pipeline wait of the
 * ring kernel is reported).  Errors: CFP_ESTATE, CFP_EINVAL, CFP_ECUDA.
 */
cfp_status cfp_apply_f32(cfp_ctx* ctx, const float* x_dev, float* y_dev);

/*
 * phi = P(rho): `sweeps` red-black Gauss-Seidel sweeps on K phi = rho from
 * phi = 0 (K: the 7-point second-order operator of Eq. A7 with the
 * Shortley-Weller rows of Eq. A7_mod and zero Dirichlet data; Sec. 3.3),
 * red = (i+j+k) even first.  sweeps = 0 copies rho.  rho is read at the
 * unknowns only; phi is 0 at box and solid nodes.  Fields, no overlap.
 * Errors: CFP_ESTATE, CFP_EINVAL.
 */
cfp_status cfp_precondition(cfp_ctx* ctx, int sweeps, const double* rho_dev,
                            double* phi_dev);

/*
 * phi = P(rho) with the preconditioner chosen in opts (precond, sweeps,
 * mg_smooth, mg_post, mg_tma; NULL: defaults), as applied inside cfp_solve.
 * opts->precision CFP_PREC_FP64: in FP64; CFP_PREC_MIXED: in FP32, as the
 * mixed solve's inner iterations apply it (rho rounded to FP32, phi widened;
 * rho must lie within the FP32 range), and the call synchronises.  Fields,
 * no overlap; phi is 0 at box and solid nodes.  Errors as cfp_precondition,
 * and CFP_ECUDA if a bounded pipeline wait of a kernel timed out (one second;
 * the results are then not valid).
 */
cfp_status cfp_precondition_ex(cfp_ctx* ctx, const cfp_opts* opts,
                               const double* rho_dev, double* phi_dev);

/*
 * Solve Eq. Bu=q with BiCGSTAB (Algorithm 1, Sec. 3.2) right-preconditioned
 * by P (Sec. 3.3), the update being u += alpha*p_hat + omega*s_hat.
 *   f_dev, g_nodes_dev, g_ibi_dev  as for cfp_assemble_rhs
 *   u_dev   field; in: initial guess at the unknowns (other nodes ignored);
 *           out: the solution, g at box nodes, 0 at solid nodes.
 *   tol     stop when ||r||_2 <= tol ||rhs||_2; the true residual is then
 *           recomputed and the iteration restarted if it fails the test.
 *   opts    NULL for defaults.  info: NULL or receives the statistics.
 * Classifies first if cfp_classify_points has not run.  Synchronises.
 * Errors: CFP_ENOCONV, CFP_EBREAKDOWN, CFP_ENAN, CFP_EGEOM, CFP_EINVAL,
 * CFP_ENOMEM, CFP_ECUDA.  The iteration always ends (maxit bound).
 */
cfp_status cfp_solve(cfp_ctx* ctx, const double* f_dev, const double* g_nodes_dev,
                     const double* g_ibi_dev, double* u_dev, double tol,
                     const cfp_opts* opts, cfp_info* info);

/*
 * cfp_solve with host buffers.  Page-locked buffers (cudaHostAlloc,
 * cudaHostRegister) are used in place: the kernels read f, g (box values),
 * g_ibi and the initial guess from host memory and the last one writes u
 * there, each once, over the host link.  Other host memory is copied to
 * context-owned device buffers, solved on, and u copied back.  Same
 * arguments and errors.
 */
cfp_status cfp_solve_host(cfp_ctx* ctx, const double* f_host,
                          const double* g_nodes_host, const double* g_ibi_host,
                          double* u_host, double tol, const cfp_opts* opts,
                          cfp_info* info);

/*
 * Solve nprob independent problems at once (batched workload: many grids of
 * uneven size and geometry).  Problem m is cfp_solve(ctxs[m], f_dev[m],
 * g_nodes_dev[m], g_ibi_dev[m], u_dev[m], tol, opts, &infos[m]); nthreads
 * host threads (<= 0: up to 16) take problems from a shared counter, and
 * each context enqueues on its own stream, so the solves overlap on the
 * GPU.  Give every context its own stream (cfp_ctx_create's `stream`), or
 * the solves serialise.  The contexts must be distinct and on the current
 * device.  g_ibi_dev may be NULL when no problem has IBI points.  Each
 * result is bitwise the result of a lone cfp_solve.  infos: NULL or nprob
 * entries.  Returns the first failing problem's status (the others still
 * run).  Errors: as cfp_solve, plus CFP_EINVAL for NULL or repeated entries.
 */
cfp_status cfp_solve_batch(cfp_ctx* const* ctxs, int nprob,
                           const double* const* f_dev,
                           const double* const* g_nodes_dev,
                           const double* const* g_ibi_dev, double* const* u_dev,
                           double tol, const cfp_opts* opts, int nthreads,
                           cfp_info* infos);

/*
 * A batch of independent mixed-precision solves as ONE graph launch.  Each
 * problem's whole solve -- right-hand side, the refinement loop of
 * CFP_PREC_MIXED with its scaling, inner-tolerance, stall and stopping
 * decisions taken by one-block kernels on device-resident scalars, the
 * preconditioned BiCGSTAB loop inside each refinement step, the solution --
 * is captured with its two loops as nested while nodes of a CUDA graph, and
 * the problems are the parallel branches of one graph.  cfp_batch_run
 * launches it once: no host round trip between refinement steps or problems,
 * and the GPU interleaves the problems' kernels.  Each problem's result is
 * bitwise the one cfp_solve gives with the same settings (the same kernels
 * in the same order on the same values).
 *   cfp_batch_create: ctxs, f_dev, g_nodes_dev, g_ibi_dev (NULL allowed:
 *     every problem without IBI points), u_dev: nprob entries as cfp_solve
 *     (u_dev: initial guess in, solution out, of the next run); opts: NULL
 *     (defaults) or nprob settings, each with precision = CFP_PREC_MIXED;
 *     tol as cfp_solve.  Classifies the contexts that are not, prepares
 *     their work space and preconditioners, captures and instantiates the
 *     graph.  The batch holds the pointers: the buffers must live until
 *     cfp_batch_destroy; their contents may change between runs.
 *   cfp_batch_run: launches the graph and waits for it; infos (NULL
 *     allowed): nprob results, ms_solve = the whole batch's wall time.  A
 *     context reclassified (or whose multigrid / ILU data or apply kernel
 *     was replaced) since the capture makes the run capture the graph
 *     again first.  Returns the first failing problem's status (CFP_ENOCONV,
 *     CFP_ENAN, CFP_EBREAKDOWN) with its index in the message; infos holds
 *     every problem's.
 * A context must not be used by another call while its batch runs.
 * Errors: CFP_EINVAL (NULL or repeated entries, nprob < 1, a problem with
 * IBI points and no g_ibi_dev, another precision), CFP_ECUDA, CFP_ENOMEM,
 * CFP_EGEOM from the classification.
 */
typedef struct cfp_batch cfp_batch;
cfp_status cfp_batch_create(cfp_ctx* const* ctxs, int nprob, const double* const* f_dev,
                            const double* const* g_nodes_dev, const double* const* g_ibi_dev,
                            double* const* u_dev, double tol, const cfp_opts* opts, cfp_batch** out);
cfp_status cfp_batch_run(cfp_batch* batch, cfp_info* infos);
void cfp_batch_destroy(cfp_batch* batch);

/*
 * Autotuner of the solver settings for one problem: times the solve (best
 * of two runs each) with the multigrid preconditioner and mg_smooth in
 * {1, 2, 3} and, for CFP_PREC_MIXED, inner_tol in {1e-2, 1e-3, 1e-4}, and
 * writes the fastest converging setting into *opts (other fields kept) and
 * its time into *best_ms (NULL allowed).  u_dev is overwritten by the trial
 * solves.  Arguments otherwise as cfp_solve.  Synchronises.  Errors: as
 * cfp_solve; CFP_ENOCONV if no candidate converges.
 */
cfp_status cfp_autotune(cfp_ctx* ctx, const double* f_dev, const double* g_nodes_dev,
                        const double* g_ibi_dev, double* u_dev, double tol,
                        cfp_opts* opts, double* best_ms);

/*
 * cfp_assemble_rhs without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * call cudaMalloc -- for instance applications whose device memory belongs to
 * a pooling allocator (an allocation outside the pool may fail and it
 * synchronises the device) or loops with a fixed memory or latency budget.
 * cfp_assemble_rhs allocates the solver work space on first use; this
 * variant keeps its one scratch field in a static device array of 2^22
 * doubles (32 MiB) that every GPU loading the library holds until exit.
 *   Same arguments, output and errors as cfp_assemble_rhs, plus CFP_EINVAL
 *   when the grid has more than 2^22 = 4,194,304 nodes.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (two streams or threads at once) race.
 */
cfp_status cfp_assemble_rhs_noalloc(cfp_ctx* ctx, const double* f_dev,
                                    const double* g_nodes_dev,
                                    const double* g_ibi_dev, double* rhs_dev);

/* Kernels this context has launched since it was created (graph bodies
 * counted once per executed iteration).  0 for NULL. */
int64_t cfp_launch_count(const cfp_ctx* ctx);

enum { CFP_KERNEL_APPLY = 0,    /* B x with the fused (r_hat0, v) dot, as in
                                   Algorithm 1 line 5                        */
       CFP_KERNEL_RBGS = 1,     /* one red half-sweep of red-black Gauss-Seidel
                                   on K (Eq. A7), the inner iterations of
                                   Sec. 3.3; the same split-layout kernel as
                                   CFP_KERNEL_MG_SWEEP                       */
       CFP_KERNEL_UPDATE = 2,   /* the fused x/r update with two dots (lines
                                   11-12)                                    */
       CFP_KERNEL_MG_SWEEP = 3, /* one red half-sweep on the fine level of the
                                   multigrid preconditioner (CFP_PRECOND_MG),
                                   red and black nodes stored in separate
                                   arrays; includes the follow-up launch that
                                   applies the Shortley-Weller rows of the
                                   irregular nodes.  In FP32 on a fine level
                                   of >= 192 nodes per row, the TMA-fed
                                   kernel (unless the last solve or
                                   preconditioner call set mg_tma = 0)      */
       CFP_KERNEL_PROLONG = 4,  /* the multigrid prolongation of the second
                                   level's correction onto the fine level's
                                   black nodes (trilinear in the stretched
                                   coordinates)                              */
       CFP_KERNEL_RESTRICT = 5, /* the full-weighting restriction of the fine
                                   level's red residual to the second level */
       CFP_KERNEL_MG_PAIR = 6   /* the fused pass of a black half-sweep and
                                   the next red one on the fine level (FP32
                                   only, a fine level of >= 192 nodes per
                                   row, mg_tma on), with the Shortley-Weller
                                   rows of the irregular nodes; algorithmic
                                   bytes 2.5 x 4 per interior node (old red,
                                   both b, the new black and red values)    */ };

/*
 * Profiling aid: time `reps` >= 1 back-to-back launches of one kernel of the
 * solve (CFP_KERNEL_*) in FP64 (precision CFP_PREC_FP64) or FP32
 * (CFP_PREC_MIXED) with CUDA events on the context's stream, on the
 * context's own work vectors (their contents are overwritten).
 *   ms_per_launch     host pointer: mean device time of one launch
 *   bytes_per_launch  host pointer or NULL: algorithmic bytes of one launch
 *                     (minimum traffic: per interior node, apply 3 values
 *                     (x, y and the dot operand); a half-sweep 1.5 values
 *                     (rho and the new phi of its colour, phi of the other
 *                     colour); update 8 values over all nodes; prolongation
 *                     per fine interior node half of (type byte + e read +
 *                     e written) plus the coarse e once (1/8 value);
 *                     restriction half a value (the red residual) plus the
 *                     coarse type byte and b once (1/8 each))
 * Requires classification.  Synchronises.  Errors: CFP_ESTATE, CFP_EINVAL
 * (also for a transfer on a grid with a single multigrid level),
 * CFP_ECUDA.
 */
cfp_status cfp_time_kernel(cfp_ctx* ctx, int kernel, int precision, int reps,
                           double* ms_per_launch, double* bytes_per_launch);

/* The apply's kernels (cfp_tune_apply). */
enum { CFP_APPLY_STREAM = 1,  /* each thread streams its column of `rows`
                                 rows through the z planes of its chunk with
                                 plain loads, one plane ahead (FP64, FP32)  */
       CFP_APPLY_RING = 2     /* FP32: a producer warp copies the planes of a
                                 512-column x 2-row tile with bulk (TMA)
                                 copies into a ring of shared-memory stages
                                 ahead of 256 consumer threads; persistent
                                 grid.  Needs 16-byte aligned x and dot
                                 operand (otherwise the streaming kernel
                                 runs)                                       */
};

/*
 * Autotuner of the compact-stencil apply (B x: the regular rows of Eq. A27
 * matrix-free, then the corrections of the irregular rows of Eq. Bdec), per
 * precision (CFP_PREC_FP64, or CFP_PREC_MIXED for the FP32 apply of the
 * mixed solve's inner iterations): the kernel (CFP_APPLY_STREAM with 2 or 4
 * rows per thread and 16, 32 or 64 planes a CTA marches in z;
 * CFP_APPLY_RING, FP32 only, 2 rows per tile and 32 or 64 planes).
 * kernel = rows = planes = 0: every candidate (6 in FP64, 8 in FP32) is
 * timed (CUDA events, 5 launches after two untimed, on the context's work
 * vectors) and the fastest is kept by the context for its later solves;
 * otherwise that choice is set and timed.  The rows of B x do not depend on the choice (the same fused
 * multiply-add chain per row in every kernel); the dot products fused into
 * the apply are summed per CTA, so their rounding does.  Without a call the
 * context uses CFP_APPLY_STREAM with 4 rows x 64 planes in FP64; in FP32
 * CFP_APPLY_RING with 64 planes where its 512-column tiles are at least 85 %
 * filled by the n_x - 2 interior columns, else CFP_APPLY_STREAM with 2 x 64.
 *   ms  NULL or the chosen candidate's mean time per launch.
 * Requires classification.  Synchronises.  Errors: CFP_ESTATE, CFP_EINVAL
 * (a choice outside those values, or CFP_APPLY_RING with CFP_PREC_FP64 or
 * where the ring cannot be set up), CFP_ECUDA.
 */
cfp_status cfp_tune_apply(cfp_ctx* ctx, int precision, int kernel, int rows, int planes, double* ms);

/*
 * The apply's kernel and tile shape the context uses for `precision` (set
 * by cfp_tune_apply or the default), as cfp_tune_apply takes them: for
 * instance to give contexts of one grid size the shape tuned on one of them.
 * Outputs may be NULL.  Errors: CFP_EINVAL.
 */
cfp_status cfp_apply_shape(const cfp_ctx* ctx, int precision, int* kernel, int* rows, int* planes);

/*
 * FP64 vector helpers over all N nodes of two fields, for outer iterations
 * built on this interface (the learned part's flexible Krylov method):
 * *out_host = sum a[l] b[l] (synchronises); y = alpha x + beta y (x and y
 * may be the same field).  Errors: CFP_EINVAL.
 */
cfp_status cfp_vec_dot(cfp_ctx* ctx, const double* a_dev, const double* b_dev, double* out_host);
cfp_status cfp_vec_axpby(cfp_ctx* ctx, double alpha, const double* x_dev, double beta, double* y_dev);

/*
 * Diagnostic of the bounded waits of the TMA-fed smoother: launches one CTA
 * that waits on an mbarrier phase that nothing completes, with the same
 * one-second bound as the smoother's pipeline waits.  The wait gives up,
 * records code 5 in the context's wait word, and the call returns CFP_ECUDA
 * after about one second (cfp_last_error names the code), the status a
 * timed-out wait gives any call; no kernel is left running and the context
 * stays usable.  Synchronises.  Errors: CFP_EINVAL (NULL context),
 * CFP_ECUDA (the expected outcome).
 */
cfp_status cfp_diag_bounded_wait(cfp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
