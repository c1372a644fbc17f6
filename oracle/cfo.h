/*
 * cfo.h -- the CPU oracle's own interface.  TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 restatement of the fourth-order compact
 * finite-difference Poisson method with immersed Dirichlet bodies of
 * Hosseinverdi & Fasel (arXiv 1901.08269).  Only tests/, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code and
 * no header with the CUDA library.
 *
 * Index space: the full grid, node (i,j,k) (0-based) at linear index
 * i + nx*(j + ny*k).  Vectors are full-grid FP64 arrays of N = nx*ny*nz.
 */
#ifndef CFO_H
#define CFO_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum { CFO_OK = 0, CFO_EINVAL = 1, CFO_ENOMEM = 2, CFO_EGEOM = 4,
       CFO_ENOCONV = 5, CFO_EBREAKDOWN = 6, CFO_ENAN = 7 };

/* point types of Section 2 */
enum { CFO_BOUNDARY = 0, CFO_REGULAR = 1, CFO_IRREGULAR = 2, CFO_SOLID = 3 };

enum { CFO_SPHERE = 0, CFO_ELLIPSOID = 1, CFO_TORUS = 2 };

/* An implicit body: phi < 0 inside.  R is the row-major body-to-world
 * rotation, c the centre; p = radius (sphere), semi-axes (ellipsoid) or
 * (major radius, minor radius) of a torus whose axis is the body z axis. */
typedef struct {
    int kind;
    double c[3];
    double R[9];
    double p[3];
} cfo_body;

typedef struct cfo_problem cfo_problem;

/* which matrix cfo_export / cfo_nnz address */
enum { CFO_MAT_B = 0,   /* compact system rows, all grid columns          */
       CFO_MAT_BIBI = 1,/* IBI weights of each row (script B of Eq. bc)    */
       CFO_MAT_K = 2,   /* 7-point preconditioner matrix, all grid columns */
       CFO_MAT_KIBI = 3 /* IBI weights of the Shortley-Weller rows of K    */ };

int  cfo_create(const double* x, int nx, const double* y, int ny,
                const double* z, int nz, const cfo_body* bodies, int nbodies,
                int fluid_inside, cfo_problem** out);
void cfo_destroy(cfo_problem* p);
const char* cfo_error(const cfo_problem* p);
int  cfo_threads(void);

/* 1D grid metrics: Eq. app_xxx (compact) and Eq. 2ndorder_coef. Interior
 * nodes 1..n-2 are filled, the two end entries are set to zero. */
void cfo_compact_coefs(const double* x, int n, double* a, double* c,
                       double* ar, double* br, double* cr);
void cfo_second_coefs(const double* x, int n, double* a, double* b, double* c);

/* level-set value (union of bodies, sign flipped for interior problems) */
double cfo_phi(const cfo_body* b, int nb, int fluid_inside,
               double x, double y, double z);

/* moment-matching solve for a modified line operator (Eqs. mat1-mat4). */
int cfo_line_operator(int M, const double* xi, double xe, int ns,
                      const double* xs, const double* Ls, double hs, double* c);

int cfo_classify(cfo_problem* p, uint8_t* type_out, int64_t* n_irr, int64_t* n_ibi);
/* IBI list in canonical order (key = lin*6 + dir, dir = -x,+x,-y,+y,-z,+z) */
int cfo_ibi(cfo_problem* p, int64_t* key_out, double* t_out, double* xyz_out);
int cfo_assemble(cfo_problem* p);
int64_t cfo_nnz(cfo_problem* p, int which);
/* number of modified operators built with fewer points than the paper's */
int64_t cfo_degenerate(cfo_problem* p);
int cfo_export(cfo_problem* p, int which, int64_t* ptr, int32_t* col, double* val);

void cfo_apply_B(cfo_problem* p, const double* x, double* y);
void cfo_apply_B_abs(cfo_problem* p, const double* x, double* y);
int  cfo_rhs(cfo_problem* p, const double* f, const double* g_nodes,
             const double* g_ibi, double* rhs);
/* B x, sum_c |B_lc||x_c| and the right-hand side at the nodes rows[0..nrows)
 * (outputs indexed like rows; 0 at non-unknowns) without assembling the
 * system; needs cfo_classify only.  x, f, g_nodes: full-grid arrays, g_ibi:
 * n_ibi values; a NULL output skips its inputs.  n_degenerate: NULL or the
 * degenerate operators met in those rows. */
int cfo_rows(cfo_problem* p, int64_t nrows, const int64_t* rows, const double* x,
             const double* f, const double* g_nodes, const double* g_ibi,
             double* bx, double* bx_abs, double* rhs, int64_t* n_degenerate);
/* inner iterations on K from phi = 0: red-black Gauss-Seidel sweeps
 * (cfo_precond) or ILU(0)-Richardson sweeps (cfo_precond_ilu); the solve
 * uses the kind set by cfo_set_precond (red-black by default) */
enum { CFO_PRECOND_RBGS = 0, CFO_PRECOND_ILU = 1 };
void cfo_precond(cfo_problem* p, int sweeps, const double* rho, double* phi);
void cfo_precond_ilu(cfo_problem* p, int sweeps, const double* rho, double* phi);
void cfo_set_precond(cfo_problem* p, int kind);
/* ILU(0) pivots of K in natural order (N values, 0 at non-unknowns) */
int  cfo_ilu_pivots(cfo_problem* p, double* d_out);
int  cfo_bicgstab(cfo_problem* p, const double* rhs, double* x, double tol,
                  int maxit, int sweeps, int* iters, double* relres);
int  cfo_solve(cfo_problem* p, const double* f, const double* g_nodes,
               const double* g_ibi, double* u, double tol, int maxit,
               int sweeps, int* iters, double* relres);

#ifdef __cplusplus
}
#endif
#endif
