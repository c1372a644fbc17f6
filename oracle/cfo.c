/*
 * cfo.c -- CPU oracle.  TEST INFRASTRUCTURE ONLY: called by tests/, the
 * smoke check and the benchmark's CPU-baseline leg, never by the product
 * path.  Plain FP64, no fused multiply-add (built with -ffp-contract=off),
 * explicit CSR matrices, row by row, in the order and notation of
 * Hosseinverdi & Fasel, "A fourth-order accurate compact difference scheme
 * for solving the three-dimensional Poisson equation with arbitrary
 * boundaries" (arXiv 1901.08269).  Citations name the paper's sections and
 * equation labels.
 *
 * What each part follows:
 *   cfo_compact_coefs ........ Sec. 2.1, Eq. app_xxx
 *   regular rows ............. Sec. 2.1, Eqs. lhsrhs_xxyyzz, A27, q, As_qs
 *   cfo_classify ............. Sec. 2 (regular / irregular / solid points),
 *                              Sec. 1 (u = 0 in the solid)
 *   IBI roots ................ Sec. 2 (IBI points); root method not stated
 *                              by the paper: bracketed scan + bisection
 *   modified line operators .. Sec. 2.2 Eqs. mod1-mat4, M; Sec. 2.3
 *                              Eqs. mod2_case2, mod2_case22
 *   irregular rows ........... Sec. 2.2 Eqs. lhsrhs_xxyyzz_mod, A27_mod,
 *                              As_mod, bc, cor; Sec. 2.3 Eqs. A27_mod_case2,
 *                              cor_case2, qb_case2
 *   global system ............ Sec. 3, Eqs. Au=q, Bu=q, Bdec
 *   preconditioner matrix K .. Sec. 3.3, Eqs. 2ndorder, 2ndorder_coef, A7,
 *                              2ndorder_xx, 2ndorder_coef_mod, A7_mod
 *   inner solver of K ........ Sec. 3.3 names MSI, whose recurrences are not
 *                              in the paper; this oracle uses m sweeps of
 *                              red-black Gauss-Seidel from zero (a fixed
 *                              linear map), the same map the GPU path uses
 *   BiCGSTAB ................. Sec. 3.2, Algorithm 1, with the preconditioned
 *                              update u += alpha*p_hat + omega*s_hat
 *
 * Parity pins (tests/test_oracle_*.py): closed-form uniform coefficients,
 * polynomial exactness of every operator, exact reproduction of tensor
 * quartic solutions with bodies, 4th-order convergence, sparse direct
 * solves, spectra, brute-force classification.
 */
#include "cfo.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t* ptr;
    int32_t* col;
    double* val;
    int64_t nnz;
} csr_t;

struct cfo_problem {
    int n[3];
    int64_t N;
    double* X[3];          /* coordinates per axis */
    double* C[3][5];       /* compact coefs per axis: a, c, ar, br, cr */
    double* S[3][3];       /* second-order coefs per axis: a, b, c     */
    cfo_body* bodies;
    int nb, fluid_inside;
    uint8_t* type;
    int classified, assembled;
    int64_t n_irr, n_ibi, n_degenerate;
    int64_t* ibi_key;
    double* ibi_t;
    double* ibi_xyz;
    csr_t B, BI, K, KI;
    int precond_kind;      /* CFO_PRECOND_RBGS or CFO_PRECOND_ILU */
    double* ilu_d;         /* ILU(0) pivots of K, NULL until first needed */
    char err[256];
};

static void seterr(cfo_problem* p, const char* m) {
    snprintf(p->err, sizeof p->err, "%s", m);
}

const char* cfo_error(const cfo_problem* p) { return p ? p->err : "null problem"; }

int cfo_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1, Eq. app_xxx: 1D fourth-order compact coefficients for the  */
/* second derivative on a nonuniform grid, dx_f = x_{i+1}-x_i,          */
/* dx_b = x_i - x_{i-1}; the LHS centre coefficient b is 1.             */
/* ------------------------------------------------------------------ */
void cfo_compact_coefs(const double* x, int n, double* a, double* c,
                       double* ar, double* br, double* cr) {
    for (int i = 0; i < n; ++i) { a[i] = c[i] = ar[i] = br[i] = cr[i] = 0.0; }
    for (int i = 1; i < n - 1; ++i) {
        double f = x[i + 1] - x[i];
        double b = x[i] - x[i - 1];
        double D = f * f * f + 4.0 * f * f * b + 4.0 * f * b * b + b * b * b;
        a[i] = f * (b * b + b * f - f * f) / D;
        c[i] = b * (f * f + b * f - b * b) / D;
        ar[i] = 12.0 * f / D;
        br[i] = -12.0 / (f * f + 3.0 * f * b + b * b);
        cr[i] = 12.0 * b / D;
    }
}

/* Sec. 3.3, Eq. 2ndorder_coef: second-order 3-point coefficients. */
void cfo_second_coefs(const double* x, int n, double* a, double* b, double* c) {
    for (int i = 0; i < n; ++i) { a[i] = b[i] = c[i] = 0.0; }
    for (int i = 1; i < n - 1; ++i) {
        double f = x[i + 1] - x[i];
        double bk = x[i] - x[i - 1];
        a[i] = 2.0 / (bk * (f + bk));
        b[i] = -2.0 / (bk * f);
        c[i] = 2.0 / (f * (f + bk));
    }
}

/* ------------------------------------------------------------------ */
/* Level set of the immersed bodies (Sec. 1: Omega^- is the inside).    */
/* The body coordinates are q = R^T (p - c).  The sequence of roundings */
/* is fixed (no contraction) so that the sign is reproducible.          */
/* ------------------------------------------------------------------ */
static double body_phi(const cfo_body* b, double x, double y, double z) {
    double d0 = x - b->c[0], d1 = y - b->c[1], d2 = z - b->c[2];
    const double* R = b->R;
    double q0 = (R[0] * d0 + R[3] * d1) + R[6] * d2;
    double q1 = (R[1] * d0 + R[4] * d1) + R[7] * d2;
    double q2 = (R[2] * d0 + R[5] * d1) + R[8] * d2;
    if (b->kind == CFO_SPHERE) {
        return ((q0 * q0 + q1 * q1) + q2 * q2) - b->p[0] * b->p[0];
    } else if (b->kind == CFO_ELLIPSOID) {
        double e0 = q0 / b->p[0], e1 = q1 / b->p[1], e2 = q2 / b->p[2];
        return ((e0 * e0 + e1 * e1) + e2 * e2) - 1.0;
    } else {
        double rho = sqrt(q0 * q0 + q1 * q1);
        double s = rho - b->p[0];
        return (s * s + q2 * q2) - b->p[1] * b->p[1];
    }
}

double cfo_phi(const cfo_body* b, int nb, int fluid_inside, double x, double y, double z) {
    double phi = INFINITY;
    for (int m = 0; m < nb; ++m) {
        double v = body_phi(&b[m], x, y, z);
        if (v < phi) phi = v;
    }
    return fluid_inside ? -phi : phi;
}

/* ------------------------------------------------------------------ */
/* Problem set-up                                                      */
/* ------------------------------------------------------------------ */
int cfo_create(const double* x, int nx, const double* y, int ny,
               const double* z, int nz, const cfo_body* bodies, int nbodies,
               int fluid_inside, cfo_problem** out) {
    if (!out) return CFO_EINVAL;
    *out = NULL;
    if (nx < 3 || ny < 3 || nz < 3 || !x || !y || !z || nbodies < 0 ||
        (nbodies > 0 && !bodies))
        return CFO_EINVAL;
    const double* src[3] = {x, y, z};
    int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d)
        for (int i = 0; i + 1 < n[d]; ++i)
            if (!(src[d][i + 1] > src[d][i])) return CFO_EINVAL;
    cfo_problem* p = (cfo_problem*)calloc(1, sizeof *p);
    if (!p) return CFO_ENOMEM;
    p->N = (int64_t)nx * ny * nz;
    for (int d = 0; d < 3; ++d) {
        p->n[d] = n[d];
        p->X[d] = (double*)malloc(sizeof(double) * n[d]);
        memcpy(p->X[d], src[d], sizeof(double) * n[d]);
        for (int m = 0; m < 5; ++m) p->C[d][m] = (double*)malloc(sizeof(double) * n[d]);
        for (int m = 0; m < 3; ++m) p->S[d][m] = (double*)malloc(sizeof(double) * n[d]);
        cfo_compact_coefs(p->X[d], n[d], p->C[d][0], p->C[d][1], p->C[d][2],
                          p->C[d][3], p->C[d][4]);
        cfo_second_coefs(p->X[d], n[d], p->S[d][0], p->S[d][1], p->S[d][2]);
    }
    p->nb = nbodies;
    p->fluid_inside = fluid_inside ? 1 : 0;
    if (nbodies) {
        p->bodies = (cfo_body*)malloc(sizeof(cfo_body) * nbodies);
        memcpy(p->bodies, bodies, sizeof(cfo_body) * nbodies);
    }
    p->type = (uint8_t*)malloc((size_t)p->N);
    if (!p->type) { cfo_destroy(p); return CFO_ENOMEM; }
    *out = p;
    return CFO_OK;
}

static void csr_free(csr_t* m) {
    free(m->ptr); free(m->col); free(m->val);
    memset(m, 0, sizeof *m);
}

void cfo_destroy(cfo_problem* p) {
    if (!p) return;
    for (int d = 0; d < 3; ++d) {
        free(p->X[d]);
        for (int m = 0; m < 5; ++m) free(p->C[d][m]);
        for (int m = 0; m < 3; ++m) free(p->S[d][m]);
    }
    free(p->bodies); free(p->type);
    free(p->ibi_key); free(p->ibi_t); free(p->ibi_xyz);
    csr_free(&p->B); csr_free(&p->BI); csr_free(&p->K); csr_free(&p->KI);
    free(p->ilu_d);
    free(p);
}

static inline int64_t LIN(const cfo_problem* p, int i, int j, int k) {
    return (int64_t)i + (int64_t)p->n[0] * ((int64_t)j + (int64_t)p->n[1] * k);
}

static inline int is_unknown(uint8_t t) { return t == CFO_REGULAR || t == CFO_IRREGULAR; }

/* ------------------------------------------------------------------ */
/* Sec. 2: a point is solid if it lies inside a body (phi <= 0 here;    */
/* box nodes are Dirichlet nodes whatever phi says), irregular if it is */
/* an interior fluid point with a solid point among its 26 neighbours,  */
/* regular otherwise.  IBI points: intersections of grid lines with     */
/* Gamma between a fluid point and a solid axis neighbour.              */
/* ------------------------------------------------------------------ */
static double edge_pos(double xa, double xb, double t) { return (1.0 - t) * xa + t * xb; }

/* Root of phi on the edge from fluid node A (t=0) to solid node B (t=1):
 * scan t = 1/8..7/8 for the first sign change seen from the fluid side,
 * then 60 bisection steps; returns the solid end of the final bracket. */
static double ibi_root(const cfo_problem* p, int d, const double pa[3], double xb) {
    double q[3] = {pa[0], pa[1], pa[2]};
    double lo = 0.0, hi = 1.0;
    for (int s = 1; s < 8; ++s) {
        double ts = (double)s / 8.0;
        q[d] = edge_pos(pa[d], xb, ts);
        if (cfo_phi(p->bodies, p->nb, p->fluid_inside, q[0], q[1], q[2]) <= 0.0) { hi = ts; break; }
        lo = ts;
    }
    for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi);
        q[d] = edge_pos(pa[d], xb, mid);
        if (cfo_phi(p->bodies, p->nb, p->fluid_inside, q[0], q[1], q[2]) > 0.0) lo = mid;
        else hi = mid;
    }
    return hi;
}

int cfo_classify(cfo_problem* p, uint8_t* type_out, int64_t* n_irr, int64_t* n_ibi) {
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int64_t l = LIN(p, i, j, k);
                if (i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1) {
                    p->type[l] = CFO_BOUNDARY;
                } else {
                    double ph = cfo_phi(p->bodies, p->nb, p->fluid_inside,
                                        p->X[0][i], p->X[1][j], p->X[2][k]);
                    p->type[l] = (ph <= 0.0) ? CFO_SOLID : CFO_REGULAR;
                }
            }
    int64_t cnt = 0;
    #pragma omp parallel for schedule(static) reduction(+ : cnt)
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                int64_t l = LIN(p, i, j, k);
                if (p->type[l] != CFO_REGULAR) continue;
                int irr = 0;
                for (int r = -1; r <= 1 && !irr; ++r)
                    for (int q = -1; q <= 1 && !irr; ++q)
                        for (int o = -1; o <= 1; ++o)
                            if (p->type[LIN(p, i + o, j + q, k + r)] == CFO_SOLID) { irr = 1; break; }
                if (irr) { p->type[l] = CFO_IRREGULAR; cnt++; }
            }
    p->n_irr = cnt;
    /* IBI list in canonical order: ascending lin, then dir -x,+x,-y,+y,-z,+z */
    int64_t nibi = 0;
    for (int64_t l = 0; l < p->N; ++l) {
        if (p->type[l] != CFO_IRREGULAR) continue;
        int64_t st[3] = {1, nx, (int64_t)nx * ny};
        for (int dir = 0; dir < 6; ++dir) {
            int64_t nb = l + ((dir & 1) ? st[dir >> 1] : -st[dir >> 1]);
            if (p->type[nb] == CFO_SOLID) nibi++;
        }
    }
    free(p->ibi_key); free(p->ibi_t); free(p->ibi_xyz);
    p->ibi_key = (int64_t*)malloc(sizeof(int64_t) * (nibi + 1));
    p->ibi_t = (double*)malloc(sizeof(double) * (nibi + 1));
    p->ibi_xyz = (double*)malloc(sizeof(double) * 3 * (nibi + 1));
    int64_t m = 0;
    for (int k = 1; k < nz - 1; ++k)
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                int64_t l = LIN(p, i, j, k);
                if (p->type[l] != CFO_IRREGULAR) continue;
                int idx[3] = {i, j, k};
                for (int dir = 0; dir < 6; ++dir) {
                    int d = dir >> 1, sg = (dir & 1) ? 1 : -1;
                    int nidx[3] = {i, j, k};
                    nidx[d] += sg;
                    if (p->type[LIN(p, nidx[0], nidx[1], nidx[2])] != CFO_SOLID) continue;
                    double pa[3] = {p->X[0][i], p->X[1][j], p->X[2][k]};
                    double xb = p->X[d][idx[d] + sg];
                    double t = ibi_root(p, d, pa, xb);
                    p->ibi_key[m] = l * 6 + dir;
                    p->ibi_t[m] = t;
                    p->ibi_xyz[3 * m + 0] = pa[0];
                    p->ibi_xyz[3 * m + 1] = pa[1];
                    p->ibi_xyz[3 * m + 2] = pa[2];
                    p->ibi_xyz[3 * m + d] = edge_pos(pa[d], xb, t);
                    m++;
                }
            }
    p->n_ibi = nibi;
    p->classified = 1;
    p->assembled = 0;
    if (type_out) memcpy(type_out, p->type, (size_t)p->N);
    if (n_irr) *n_irr = p->n_irr;
    if (n_ibi) *n_ibi = p->n_ibi;
    return CFO_OK;
}

int cfo_ibi(cfo_problem* p, int64_t* key_out, double* t_out, double* xyz_out) {
    if (!p->classified) { seterr(p, "classify first"); return CFO_EINVAL; }
    if (key_out) memcpy(key_out, p->ibi_key, sizeof(int64_t) * p->n_ibi);
    if (t_out) memcpy(t_out, p->ibi_t, sizeof(double) * p->n_ibi);
    if (xyz_out) memcpy(xyz_out, p->ibi_xyz, sizeof(double) * 3 * p->n_ibi);
    return CFO_OK;
}

static int64_t ibi_find(const cfo_problem* p, int64_t key) {
    int64_t lo = 0, hi = p->n_ibi - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (p->ibi_key[mid] == key) return mid;
        if (p->ibi_key[mid] < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Eqs. mat1-mat4 with the matrix M of Eq. M: find c_n such that        */
/*   sum_n c_n (xi_n - xe)^m = sum_s L_s m(m-1) (xs_s - xe)^(m-2)       */
/* for m = 0..M-1, i.e. the modified RHS operator reproduces the kept   */
/* LHS terms for every polynomial of degree < M.  Lengths are divided   */
/* by hs (a diagonal scaling of the same system), then Gaussian         */
/* elimination with partial pivoting.                                   */
/* ------------------------------------------------------------------ */
int cfo_line_operator(int M, const double* xi, double xe, int ns,
                      const double* xs, const double* Ls, double hs, double* c) {
    double A[6][7];
    if (M < 1 || M > 6 || !(hs > 0.0)) return CFO_EINVAL;
    for (int m = 0; m < M; ++m) {
        for (int n = 0; n < M; ++n) A[m][n] = pow((xi[n] - xe) / hs, (double)m);
        double r = 0.0;
        if (m >= 2)
            for (int s = 0; s < ns; ++s)
                r += Ls[s] * (double)(m * (m - 1)) * pow((xs[s] - xe) / hs, (double)(m - 2));
        A[m][M] = r / (hs * hs);
    }
    for (int col = 0; col < M; ++col) {
        int piv = col;
        for (int r = col + 1; r < M; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return CFO_EGEOM;
        if (piv != col)
            for (int q = 0; q <= M; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        for (int r = col + 1; r < M; ++r) {
            double f = A[r][col] / A[col][col];
            for (int q = col; q <= M; ++q) A[r][q] -= f * A[col][q];
        }
    }
    for (int r = M - 1; r >= 0; --r) {
        double s = A[r][M];
        for (int q = r + 1; q < M; ++q) s -= A[r][q] * c[q];
        c[r] = s / A[r][r];
    }
    return CFO_OK;
}

/* ------------------------------------------------------------------ */
/* Row accumulator (column -> value, merged)                           */
/* ------------------------------------------------------------------ */
typedef struct { int64_t col[512]; double val[512]; int n; } rowacc_t;

static int acc_add(rowacc_t* r, int64_t col, double v) {
    for (int q = 0; q < r->n; ++q)
        if (r->col[q] == col) { r->val[q] += v; return 0; }
    if (r->n >= 512) return -1;
    r->col[r->n] = col; r->val[r->n] = v; r->n++;
    return 0;
}

typedef struct { int64_t cap, nnz; int64_t* ptr; int32_t* col; double* val; } builder_t;

static int bld_init(builder_t* b, int64_t N, int64_t cap) {
    b->cap = cap; b->nnz = 0;
    b->ptr = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    b->col = (int32_t*)malloc(sizeof(int32_t) * cap);
    b->val = (double*)malloc(sizeof(double) * cap);
    return (b->ptr && b->col && b->val) ? 0 : -1;
}
static int bld_push(builder_t* b, int64_t col, double v) {
    if (b->nnz == b->cap) {
        int64_t nc = b->cap * 2 + 16;
        int32_t* c2 = (int32_t*)realloc(b->col, sizeof(int32_t) * nc);
        double* v2 = (double*)realloc(b->val, sizeof(double) * nc);
        if (!c2 || !v2) return -1;
        b->col = c2; b->val = v2; b->cap = nc;
    }
    b->col[b->nnz] = (int32_t)col; b->val[b->nnz] = v; b->nnz++;
    return 0;
}
static void bld_finish(builder_t* b, csr_t* m) {
    m->ptr = b->ptr; m->col = b->col; m->val = b->val; m->nnz = b->nnz;
}

/* L coefficients of Eq. cfd_lhs_xxyyzz at index m of axis d: offset -1 -> a,
 * 0 -> b = 1, +1 -> c */
static double Lco(const cfo_problem* p, int d, int m, int o) {
    return o < 0 ? p->C[d][0][m] : (o == 0 ? 1.0 : p->C[d][1][m]);
}
/* R coefficients of Eq. cfd_rhs_xxyyzz: -1 -> ar, 0 -> br, +1 -> cr */
static double Rco(const cfo_problem* p, int d, int m, int o) {
    return o < 0 ? p->C[d][2][m] : (o == 0 ? p->C[d][3][m] : p->C[d][4][m]);
}

/* One modified operator along axis d of the line whose centre node has
 * index vector base[] (base[d] = the irregular point's own index along d).
 * e is the offset of the expansion node; the operator is bounded on the
 * side -sg by a solid node, whose IBI it uses, and takes grid nodes
 * e, e+sg, e+2sg, ... (G of them in the paper's stencils: 5 for the
 * six-point operators of Eqs. mod1-mod4, 4 for the five-point operators of
 * Eqs. mod2_case2 / mod2_case22).  survivors/Ls are the kept LHS offsets and
 * their L coefficients.  Adds w*c_n to the row and w*c_b to its IBI weights.
 *
 * Reading where the paper is silent: if the walk meets a solid node before
 * G grid nodes, the IBI on that edge closes the node set; if it leaves the
 * grid, the set ends at the box.  The operator then has fewer points (at
 * least 3, degree >= 2) and is counted as degenerate. */
static int modified_op(cfo_problem* p, const int base[3], int d, double w,
                       int e, int sg, int G, int ns, const int* surv, const double* Ls,
                       rowacc_t* row, rowacc_t* rib, int64_t* ndeg) {
    const int nd = p->n[d];
    double xi[7], xs[3], c[7];
    int64_t col[6], ib[2];
    int ng = 0, nib = 0;
    int fidx[3] = {base[0], base[1], base[2]};
    fidx[d] += e;
    int64_t fl = LIN(p, fidx[0], fidx[1], fidx[2]);
    if (!is_unknown(p->type[fl])) { seterr(p, "expansion node is not an interior fluid node"); return CFO_EGEOM; }
    /* the bounding IBI, on the edge from the expansion node towards -sg */
    ib[nib] = ibi_find(p, fl * 6 + 2 * d + (sg > 0 ? 0 : 1));
    if (ib[nib] < 0) { seterr(p, "missing IBI"); return CFO_EGEOM; }
    nib++;
    for (int q = 0; q < G; ++q) {
        int idx[3] = {fidx[0], fidx[1], fidx[2]};
        idx[d] += q * sg;
        if (idx[d] < 0 || idx[d] >= nd) break;            /* walked off the grid */
        int64_t l = LIN(p, idx[0], idx[1], idx[2]);
        if (p->type[l] == CFO_SOLID) {                    /* walked into a body */
            int prev[3] = {idx[0], idx[1], idx[2]};
            prev[d] -= sg;
            int64_t pl = LIN(p, prev[0], prev[1], prev[2]);
            if (!is_unknown(p->type[pl])) { seterr(p, "IBI at a box node"); return CFO_EGEOM; }
            ib[nib] = ibi_find(p, pl * 6 + 2 * d + (sg > 0 ? 1 : 0));
            if (ib[nib] < 0) { seterr(p, "missing IBI"); return CFO_EGEOM; }
            nib++;
            break;
        }
        xi[ng] = p->X[d][idx[d]];
        col[ng] = l;
        ng++;
    }
    const int M = ng + nib;
    if (M < 3) {
        snprintf(p->err, sizeof p->err, "only %d points for a modified operator on axis %d at (%d,%d,%d)",
                 M, d, fidx[0], fidx[1], fidx[2]);
        return CFO_EGEOM;
    }
    if (ng < G || nib > 1) (*ndeg)++;
    for (int q = 0; q < nib; ++q) xi[ng + q] = p->ibi_xyz[3 * ib[q] + d];
    const double xe = p->X[d][fidx[d]];
    for (int s = 0; s < ns; ++s) xs[s] = p->X[d][base[d] + surv[s]];
    double hs = 0.0;
    for (int q = 1; q < M; ++q) if (fabs(xi[q] - xe) > hs) hs = fabs(xi[q] - xe);
    int st = cfo_line_operator(M, xi, xe, ns, xs, Ls, hs, c);
    if (st) { seterr(p, "singular moment matrix"); return st; }
    for (int q = 0; q < ng; ++q)
        if (acc_add(row, col[q], w * c[q])) { seterr(p, "row overflow"); return CFO_EGEOM; }
    for (int q = 0; q < nib; ++q)
        if (acc_add(rib, ib[q], w * c[ng + q])) { seterr(p, "row overflow"); return CFO_EGEOM; }
    return CFO_OK;
}

/* Irregular row at (i,j,k): Eq. lhsrhs_xxyyzz_mod summed line by line.  For
 * each axis d and each of its 9 grid lines through the 3x3x3 block, the
 * weight is the product of the transverse L coefficients of the centre
 * point and the line operator is regular, dropped, or modified according to
 * which of its three block nodes are solid (Secs. 2.2 and 2.3). */
static int irregular_row(cfo_problem* p, int i, int j, int k, rowacc_t* row, rowacc_t* rib,
                         int64_t* ndeg) {
    const int idx[3] = {i, j, k};
    for (int d = 0; d < 3; ++d) {
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        const int m = idx[d];
        const double a = Lco(p, d, m, -1), c = Lco(p, d, m, 1);
        for (int o1 = -1; o1 <= 1; ++o1)
            for (int o2 = -1; o2 <= 1; ++o2) {
                const double w = Lco(p, t1, idx[t1], o1) * Lco(p, t2, idx[t2], o2);
                int base[3] = {i, j, k};
                base[t1] += o1;
                base[t2] += o2;
                int sol[3];
                int64_t sl[3];
                for (int s = -1; s <= 1; ++s) {
                    int q[3] = {base[0], base[1], base[2]};
                    q[d] += s;
                    sl[s + 1] = LIN(p, q[0], q[1], q[2]);
                    sol[s + 1] = p->type[sl[s + 1]] == CFO_SOLID;
                }
                const int mask = (sol[0] << 2) | (sol[1] << 1) | sol[2];
                int st = CFO_OK;
                switch (mask) {
                case 0: /* regular line: Eq. cfd_rhs_xxyyzz */
                    for (int s = -1; s <= 1; ++s)
                        if (acc_add(row, sl[s + 1], w * Rco(p, d, m, s))) { seterr(p, "row overflow"); return CFO_EGEOM; }
                    break;
                case 7: /* the whole segment is solid: the line is dropped */
                    break;
                case 1: { /* +1 solid: Eqs. mod1_top, mod1, mat1 */
                    const int surv[2] = {-1, 0};
                    const double Ls[2] = {a, 1.0};
                    st = modified_op(p, base, d, w, 0, -1, 5, 2, surv, Ls, row, rib, ndeg);
                } break;
                case 4: { /* -1 solid: Eqs. mod3_top, mod3, mat3 */
                    const int surv[2] = {0, 1};
                    const double Ls[2] = {1.0, c};
                    st = modified_op(p, base, d, w, 0, +1, 5, 2, surv, Ls, row, rib, ndeg);
                } break;
                case 3: { /* 0 and +1 solid: Eqs. mod2_top, mod2, mat2 */
                    const int surv[1] = {-1};
                    const double Ls[1] = {a};
                    st = modified_op(p, base, d, w, -1, -1, 5, 1, surv, Ls, row, rib, ndeg);
                } break;
                case 6: { /* -1 and 0 solid: Eqs. mod4_top, mod4, mat4 */
                    const int surv[1] = {1};
                    const double Ls[1] = {c};
                    st = modified_op(p, base, d, w, 1, +1, 5, 1, surv, Ls, row, rib, ndeg);
                } break;
                case 2: { /* only the middle node solid: two one-sided operators,
                             Eqs. mod2_top_case2 .. mod2_case22 (five points each) */
                    const int survm[1] = {-1};
                    const double Lsm[1] = {a};
                    st = modified_op(p, base, d, w, -1, -1, 4, 1, survm, Lsm, row, rib, ndeg);
                    if (st) break;
                    const int survp[1] = {1};
                    const double Lsp[1] = {c};
                    st = modified_op(p, base, d, w, 1, +1, 4, 1, survp, Lsp, row, rib, ndeg);
                } break;
                default: { /* 5: a fluid node between two solid ones.  Not covered by
                              the paper; read as the degenerate form of the rule above:
                              the centre node and the two IBIs (three points). */
                    const int surv[1] = {0};
                    const double Ls[1] = {1.0};
                    st = modified_op(p, base, d, w, 0, -1, 5, 1, surv, Ls, row, rib, ndeg);
                } break;
                }
                if (st) return st;
            }
    }
    return CFO_OK;
}

/* Sec. 3.3: row of K at an interior fluid point, Eq. A7; at points with a
 * solid axis neighbour the distance to the IBI replaces the grid spacing on
 * that side and the solid neighbour is dropped (phi_IBI = 0), Eqs.
 * 2ndorder_xx, 2ndorder_coef_mod, A7_mod.  Box neighbours keep their
 * column (their value is zero for the preconditioner). */
static int k_row(cfo_problem* p, int i, int j, int k, rowacc_t* row, rowacc_t* rib) {
    const int idx[3] = {i, j, k};
    const int64_t l = LIN(p, i, j, k);
    const int64_t st[3] = {1, p->n[0], (int64_t)p->n[0] * p->n[1]};
    double diag = 0.0;
    for (int d = 0; d < 3; ++d) {
        const int m = idx[d];
        const double xm = p->X[d][m];
        double f = p->X[d][m + 1] - xm;
        double b = xm - p->X[d][m - 1];
        const int64_t lm = l - st[d], lp = l + st[d];
        const int sm = p->type[lm] == CFO_SOLID, sp = p->type[lp] == CFO_SOLID;
        int64_t ibm = -1, ibp = -1;
        if (sm) {
            ibm = ibi_find(p, l * 6 + 2 * d);
            if (ibm < 0) { seterr(p, "missing IBI"); return CFO_EGEOM; }
            b = xm - p->ibi_xyz[3 * ibm + d];
        }
        if (sp) {
            ibp = ibi_find(p, l * 6 + 2 * d + 1);
            if (ibp < 0) { seterr(p, "missing IBI"); return CFO_EGEOM; }
            f = p->ibi_xyz[3 * ibp + d] - xm;
        }
        const double ca = 2.0 / (b * (f + b));
        const double cb = -2.0 / (b * f);
        const double cc = 2.0 / (f * (f + b));
        diag += cb;
        if (sm) acc_add(rib, ibm, ca); else acc_add(row, lm, ca);
        if (sp) acc_add(rib, ibp, cc); else acc_add(row, lp, cc);
    }
    acc_add(row, l, diag);
    return CFO_OK;
}

/* Regular row at (i,j,k), Eq. As_qs: the coefficient of u at offset
 * (o,q,r) is Rx Ly Lz + Lx Ry Lz + Lx Ly Rz of the centre's coefficients;
 * the 27 entries in the order r (z), q (y), o (x). */
static void regular_row(const cfo_problem* p, int i, int j, int k, rowacc_t* row) {
    for (int r = -1; r <= 1; ++r)
        for (int q = -1; q <= 1; ++q)
            for (int o = -1; o <= 1; ++o) {
                double v = Rco(p, 0, i, o) * Lco(p, 1, j, q) * Lco(p, 2, k, r) +
                           Lco(p, 0, i, o) * Rco(p, 1, j, q) * Lco(p, 2, k, r) +
                           Lco(p, 0, i, o) * Lco(p, 1, j, q) * Rco(p, 2, k, r);
                row->col[row->n] = LIN(p, i + o, j + q, k + r);
                row->val[row->n] = v;
                row->n++;
            }
}

int cfo_assemble(cfo_problem* p) {
    if (!p->classified) { seterr(p, "classify first"); return CFO_EINVAL; }
    csr_free(&p->B); csr_free(&p->BI); csr_free(&p->K); csr_free(&p->KI);
    free(p->ilu_d);
    p->ilu_d = NULL;
    const int nx = p->n[0], ny = p->n[1], nz = p->n[2];
    builder_t bB, bBI, bK, bKI;
    int64_t nun = (int64_t)(nx - 2) * (ny - 2) * (nz - 2);
    if (bld_init(&bB, p->N, nun * 27 + 64) || bld_init(&bBI, p->N, p->n_ibi * 4 + 64) ||
        bld_init(&bK, p->N, nun * 7 + 64) || bld_init(&bKI, p->N, p->n_ibi + 64)) {
        seterr(p, "out of memory"); return CFO_ENOMEM;
    }
    p->n_degenerate = 0;
    rowacc_t* row = (rowacc_t*)malloc(sizeof(rowacc_t));
    rowacc_t* rib = (rowacc_t*)malloc(sizeof(rowacc_t));
    int status = CFO_OK;
    for (int64_t l = 0; l < p->N && status == CFO_OK; ++l) {
        const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
        const uint8_t t = p->type[l];
        if (t == CFO_REGULAR) {
            row->n = 0;
            regular_row(p, i, j, k, row);
            for (int q = 0; q < row->n; ++q) bld_push(&bB, row->col[q], row->val[q]);
        } else if (t == CFO_IRREGULAR) {
            row->n = 0; rib->n = 0;
            status = irregular_row(p, i, j, k, row, rib, &p->n_degenerate);
            for (int q = 0; q < row->n; ++q) bld_push(&bB, row->col[q], row->val[q]);
            for (int q = 0; q < rib->n; ++q) bld_push(&bBI, rib->col[q], rib->val[q]);
        }
        if (is_unknown(t) && status == CFO_OK) {
            row->n = 0; rib->n = 0;
            status = k_row(p, i, j, k, row, rib);
            for (int q = 0; q < row->n; ++q) bld_push(&bK, row->col[q], row->val[q]);
            for (int q = 0; q < rib->n; ++q) bld_push(&bKI, rib->col[q], rib->val[q]);
        }
        bB.ptr[l + 1] = bB.nnz; bBI.ptr[l + 1] = bBI.nnz;
        bK.ptr[l + 1] = bK.nnz; bKI.ptr[l + 1] = bKI.nnz;
    }
    free(row); free(rib);
    bld_finish(&bB, &p->B); bld_finish(&bBI, &p->BI);
    bld_finish(&bK, &p->K); bld_finish(&bKI, &p->KI);
    if (status != CFO_OK) return status;
    p->assembled = 1;
    return CFO_OK;
}

static const csr_t* pick(const cfo_problem* p, int which) {
    switch (which) {
    case CFO_MAT_B: return &p->B;
    case CFO_MAT_BIBI: return &p->BI;
    case CFO_MAT_K: return &p->K;
    default: return &p->KI;
    }
}

int64_t cfo_degenerate(cfo_problem* p) { return p->assembled ? p->n_degenerate : -1; }

int64_t cfo_nnz(cfo_problem* p, int which) { return p->assembled ? pick(p, which)->nnz : -1; }

int cfo_export(cfo_problem* p, int which, int64_t* ptr, int32_t* col, double* val) {
    if (!p->assembled) { seterr(p, "assemble first"); return CFO_EINVAL; }
    const csr_t* m = pick(p, which);
    if (ptr) memcpy(ptr, m->ptr, sizeof(int64_t) * (p->N + 1));
    if (col) memcpy(col, m->col, sizeof(int32_t) * m->nnz);
    if (val) memcpy(val, m->val, sizeof(double) * m->nnz);
    return CFO_OK;
}

/* ------------------------------------------------------------------ */
/* Sparse products and vector helpers                                  */
/* ------------------------------------------------------------------ */
static void spmv(const csr_t* m, int64_t N, const double* x, double* y, int absval) {
    #pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < N; ++r) {
        double s = 0.0;
        for (int64_t e = m->ptr[r]; e < m->ptr[r + 1]; ++e)
            s += absval ? fabs(m->val[e]) * fabs(x[m->col[e]]) : m->val[e] * x[m->col[e]];
        y[r] = s;
    }
}

void cfo_apply_B(cfo_problem* p, const double* x, double* y) { spmv(&p->B, p->N, x, y, 0); }
void cfo_apply_B_abs(cfo_problem* p, const double* x, double* y) { spmv(&p->B, p->N, x, y, 1); }

static double dot(int64_t N, const double* a, const double* b) {
    double s = 0.0;
    #pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t q = 0; q < N; ++q) s += a[q] * b[q];
    return s;
}

/* Right-hand side of Eq. Bu=q for every unknown: the RHS of Eq. q with the
 * weights of solid points set to zero (Q-bar), minus the IBI term script B
 * of Eqs. bc / qb_case2, minus the known box-boundary values times their
 * matrix entries (Dirichlet data of Eq. poisson on the box). */
int cfo_rhs(cfo_problem* p, const double* f, const double* g_nodes,
            const double* g_ibi, double* rhs) {
    if (!p->assembled) { seterr(p, "assemble first"); return CFO_EINVAL; }
    const int nx = p->n[0], ny = p->n[1];
    #pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < p->N; ++l) {
        if (!is_unknown(p->type[l])) { rhs[l] = 0.0; continue; }
        const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
        double q = 0.0;
        for (int r = -1; r <= 1; ++r)
            for (int s = -1; s <= 1; ++s)
                for (int o = -1; o <= 1; ++o) {
                    int64_t c = LIN(p, i + o, j + s, k + r);
                    if (p->type[c] == CFO_SOLID) continue;
                    q += Lco(p, 0, i, o) * Lco(p, 1, j, s) * Lco(p, 2, k, r) * f[c];
                }
        for (int64_t e = p->BI.ptr[l]; e < p->BI.ptr[l + 1]; ++e) q -= p->BI.val[e] * g_ibi[p->BI.col[e]];
        for (int64_t e = p->B.ptr[l]; e < p->B.ptr[l + 1]; ++e)
            if (p->type[p->B.col[e]] == CFO_BOUNDARY) q -= p->B.val[e] * g_nodes[p->B.col[e]];
        rhs[l] = q;
    }
    return CFO_OK;
}

/* B x, sum |B||x| and the right-hand side of Eq. Bu=q at a list of nodes,
 * each row built as cfo_assemble builds it (regular_row, irregular_row)
 * and combined as cfo_apply_B and cfo_rhs combine the stored rows, in the
 * same order, without assembling the other rows: for grids whose explicit
 * CSR does not fit in host memory.  Rows are independent, so the list is
 * split over threads. */
int cfo_rows(cfo_problem* p, int64_t nrows, const int64_t* rows, const double* x,
             const double* f, const double* g_nodes, const double* g_ibi,
             double* bx, double* bx_abs, double* rhs, int64_t* n_degenerate) {
    if (!p->classified) { seterr(p, "classify first"); return CFO_EINVAL; }
    const int nx = p->n[0], ny = p->n[1];
    int status = CFO_OK;
    int64_t ndeg = 0;
    #pragma omp parallel reduction(+ : ndeg)
    {
        rowacc_t* row = (rowacc_t*)malloc(sizeof(rowacc_t));
        rowacc_t* rib = (rowacc_t*)malloc(sizeof(rowacc_t));
        #pragma omp for schedule(dynamic, 64)
        for (int64_t q = 0; q < nrows; ++q) {
            const int64_t l = rows[q];
            double y = 0.0, ya = 0.0, r = 0.0;
            int st = CFO_OK;
            if (!row || !rib) st = CFO_ENOMEM;
            else if (l < 0 || l >= p->N) st = CFO_EINVAL;
            const uint8_t t = st == CFO_OK ? p->type[l] : CFO_BOUNDARY;
            if (st == CFO_OK && is_unknown(t)) {
                const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
                row->n = 0; rib->n = 0;
                if (t == CFO_REGULAR) regular_row(p, i, j, k, row);
                else st = irregular_row(p, i, j, k, row, rib, &ndeg);
                if (st == CFO_OK) {
                    if (x)
                        for (int e = 0; e < row->n; ++e) {
                            y += row->val[e] * x[row->col[e]];
                            ya += fabs(row->val[e]) * fabs(x[row->col[e]]);
                        }
                    if (rhs) {
                        for (int rr = -1; rr <= 1; ++rr)
                            for (int ss = -1; ss <= 1; ++ss)
                                for (int o = -1; o <= 1; ++o) {
                                    int64_t c = LIN(p, i + o, j + ss, k + rr);
                                    if (p->type[c] == CFO_SOLID) continue;
                                    r += Lco(p, 0, i, o) * Lco(p, 1, j, ss) * Lco(p, 2, k, rr) * f[c];
                                }
                        for (int e = 0; e < rib->n; ++e) r -= rib->val[e] * g_ibi[rib->col[e]];
                        for (int e = 0; e < row->n; ++e)
                            if (p->type[row->col[e]] == CFO_BOUNDARY) r -= row->val[e] * g_nodes[row->col[e]];
                    }
                }
            }
            if (st != CFO_OK) {
                #pragma omp critical
                { if (status == CFO_OK) status = st; }
            }
            if (bx) bx[q] = y;
            if (bx_abs) bx_abs[q] = ya;
            if (rhs) rhs[q] = r;
        }
        free(row); free(rib);
    }
    if (n_degenerate) *n_degenerate = ndeg;
    if (status != CFO_OK && !p->err[0]) seterr(p, "row evaluation failed");
    return status;
}

/* Approximate solve of K phi = rho (Sec. 3.3): `sweeps` red-black
 * Gauss-Seidel sweeps from phi = 0, red = (i+j+k) even updated first.
 * sweeps = 0 gives phi = rho (no preconditioning). */
void cfo_precond(cfo_problem* p, int sweeps, const double* rho, double* phi) {
    const int nx = p->n[0], ny = p->n[1];
    if (sweeps <= 0) {
        for (int64_t l = 0; l < p->N; ++l) phi[l] = is_unknown(p->type[l]) ? rho[l] : 0.0;
        return;
    }
    memset(phi, 0, sizeof(double) * p->N);
    for (int sw = 0; sw < sweeps; ++sw)
        for (int colour = 0; colour < 2; ++colour) {
            #pragma omp parallel for schedule(static)
            for (int64_t l = 0; l < p->N; ++l) {
                if (!is_unknown(p->type[l])) continue;
                const int i = (int)(l % nx), j = (int)((l / nx) % ny), k = (int)(l / ((int64_t)nx * ny));
                if (((i + j + k) & 1) != colour) continue;
                double s = rho[l], dg = 0.0;
                for (int64_t e = p->K.ptr[l]; e < p->K.ptr[l + 1]; ++e) {
                    if (p->K.col[e] == l) dg = p->K.val[e];
                    else s -= p->K.val[e] * phi[p->K.col[e]];
                }
                phi[l] = s / dg;
            }
        }
}

/* ------------------------------------------------------------------ */
/* The second inner iteration on K (Sec. 3.3 solves K phi = rho with a  */
/* few iterations of an incomplete-factorisation method): ILU(0) of K   */
/* in natural node order, used as a Richardson iteration from phi = 0.  */
/*                                                                      */
/* Restricted to the unknowns, K = L + D + U (strictly lower, diagonal, */
/* strictly upper in natural order).  ILU(0) keeps the sparsity of K;   */
/* for a 7-point pattern the factorisation is M = (P + L) P^-1 (P + U)  */
/* with the pivots                                                      */
/*     P_l = K_ll - sum over unknown m < l in row l of K_lm K_ml / P_m, */
/* which makes M equal to K at every position of K's pattern (the       */
/* products L P^-1 U only add entries outside it).  One sweep:          */
/*     w = rho - K phi;  (P + L) y = w;  (P + U) z = P y;  phi += z.    */
/* ------------------------------------------------------------------ */
static double k_entry(const cfo_problem* p, int64_t row, int64_t col) {
    for (int64_t e = p->K.ptr[row]; e < p->K.ptr[row + 1]; ++e)
        if (p->K.col[e] == col) return p->K.val[e];
    return 0.0;
}

static int ilu_pivots(cfo_problem* p) {
    if (p->ilu_d) return CFO_OK;
    double* d = (double*)calloc((size_t)p->N, sizeof(double));
    if (!d) { seterr(p, "out of memory"); return CFO_ENOMEM; }
    for (int64_t l = 0; l < p->N; ++l) {       /* natural order: every m < l is final */
        if (!is_unknown(p->type[l])) continue;
        double v = k_entry(p, l, l);
        for (int64_t e = p->K.ptr[l]; e < p->K.ptr[l + 1]; ++e) {
            const int64_t m = p->K.col[e];
            if (m >= l || !is_unknown(p->type[m])) continue;
            v -= p->K.val[e] * k_entry(p, m, l) / d[m];
        }
        d[l] = v;
    }
    p->ilu_d = d;
    return CFO_OK;
}

int cfo_ilu_pivots(cfo_problem* p, double* d_out) {
    if (!p->assembled) { seterr(p, "assemble first"); return CFO_EINVAL; }
    int st = ilu_pivots(p);
    if (st) return st;
    memcpy(d_out, p->ilu_d, sizeof(double) * p->N);
    return CFO_OK;
}

void cfo_precond_ilu(cfo_problem* p, int sweeps, const double* rho, double* phi) {
    const int64_t N = p->N;
    memset(phi, 0, sizeof(double) * N);
    if (sweeps <= 0) {
        for (int64_t l = 0; l < N; ++l) phi[l] = is_unknown(p->type[l]) ? rho[l] : 0.0;
        return;
    }
    if (ilu_pivots(p)) return;
    const double* d = p->ilu_d;
    double* w = (double*)calloc((size_t)N, sizeof(double));
    if (!w) return;
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int64_t l = 0; l < N; ++l) {      /* w = rho - K phi at the unknowns */
            if (!is_unknown(p->type[l])) { w[l] = 0.0; continue; }
            double s = rho[l];
            for (int64_t e = p->K.ptr[l]; e < p->K.ptr[l + 1]; ++e) s -= p->K.val[e] * phi[p->K.col[e]];
            w[l] = s;
        }
        for (int64_t l = 0; l < N; ++l) {      /* forward: (P + L) y = w, y over w */
            if (!is_unknown(p->type[l])) continue;
            double s = w[l];
            for (int64_t e = p->K.ptr[l]; e < p->K.ptr[l + 1]; ++e) {
                const int64_t m = p->K.col[e];
                if (m < l && is_unknown(p->type[m])) s -= p->K.val[e] * w[m];
            }
            w[l] = s / d[l];
        }
        for (int64_t l = N - 1; l >= 0; --l) { /* backward: (P + U) z = P y, z over y */
            if (!is_unknown(p->type[l])) continue;
            double s = 0.0;
            for (int64_t e = p->K.ptr[l]; e < p->K.ptr[l + 1]; ++e) {
                const int64_t m = p->K.col[e];
                if (m > l && is_unknown(p->type[m])) s += p->K.val[e] * w[m];
            }
            w[l] -= s / d[l];
        }
        for (int64_t l = 0; l < N; ++l) phi[l] += w[l];
    }
    free(w);
}

void cfo_set_precond(cfo_problem* p, int kind) {
    p->precond_kind = kind == CFO_PRECOND_ILU ? CFO_PRECOND_ILU : CFO_PRECOND_RBGS;
}

static void precond_any(cfo_problem* p, int sweeps, const double* rho, double* phi) {
    if (p->precond_kind == CFO_PRECOND_ILU) cfo_precond_ilu(p, sweeps, rho, phi);
    else cfo_precond(p, sweeps, rho, phi);
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (Sec. 3.2), right preconditioned by K (Sec. 3.3).        */
/* ------------------------------------------------------------------ */
enum { RUN_CONV = 0, RUN_BREAK = 1, RUN_MAXIT = 2, RUN_NAN = 3 };

static int bicgstab_run(cfo_problem* p, const double* rhs, double* x, double tol,
                        double bnorm, int maxit, int sweeps, int* used, double** w) {
    const int64_t N = p->N;
    double *r = w[0], *rh = w[1], *pp = w[2], *ph = w[3], *v = w[4], *s = w[5], *sh = w[6], *t = w[7];
    cfo_apply_B(p, x, v);
    for (int64_t q = 0; q < N; ++q) { r[q] = rhs[q] - v[q]; rh[q] = r[q]; pp[q] = r[q]; }
    double rho = dot(N, rh, r);
    double rr = dot(N, r, r);
    *used = 0;
    if (!isfinite(rr)) return RUN_NAN;
    if (sqrt(rr) <= tol * bnorm) return RUN_CONV;
    for (int it = 1; it <= maxit; ++it) {
        precond_any(p, sweeps, pp, ph);                 /* line 4 */
        cfo_apply_B(p, ph, v);                          /* line 5 */
        const double sigma = dot(N, rh, v);
        *used = it;
        if (!isfinite(sigma)) return RUN_NAN;
        if (sigma == 0.0) return RUN_BREAK;
        const double alpha = rho / sigma;               /* line 6 */
        for (int64_t q = 0; q < N; ++q) s[q] = r[q] - alpha * v[q];   /* line 7 */
        precond_any(p, sweeps, s, sh);                  /* line 8 */
        cfo_apply_B(p, sh, t);                          /* line 9 */
        const double ts = dot(N, t, s), tt = dot(N, t, t);
        if (!isfinite(tt)) return RUN_NAN;
        const double omega = tt > 0.0 ? ts / tt : 0.0;  /* line 10 */
        for (int64_t q = 0; q < N; ++q) {
            x[q] += alpha * ph[q] + omega * sh[q];      /* line 11 */
            r[q] = s[q] - omega * t[q];                 /* line 12 */
        }
        const double rho_new = dot(N, rh, r);
        rr = dot(N, r, r);
        if (!isfinite(rr)) return RUN_NAN;
        if (sqrt(rr) <= tol * bnorm) return RUN_CONV;
        if (omega == 0.0 || rho == 0.0) return RUN_BREAK;
        const double beta = (rho_new / rho) * (alpha / omega);        /* line 13 */
        for (int64_t q = 0; q < N; ++q) pp[q] = r[q] + beta * (pp[q] - omega * v[q]); /* line 14 */
        rho = rho_new;
    }
    return RUN_MAXIT;
}

int cfo_bicgstab(cfo_problem* p, const double* rhs, double* x, double tol,
                 int maxit, int sweeps, int* iters, double* relres) {
    if (!p->assembled) { seterr(p, "assemble first"); return CFO_EINVAL; }
    const int64_t N = p->N;
    double* w[9];
    for (int q = 0; q < 9; ++q) {
        w[q] = (double*)calloc((size_t)N, sizeof(double));
        if (!w[q]) { for (int z = 0; z < q; ++z) free(w[z]); seterr(p, "out of memory"); return CFO_ENOMEM; }
    }
    for (int64_t q = 0; q < N; ++q) if (!is_unknown(p->type[q])) x[q] = 0.0;
    const double bnorm = sqrt(dot(N, rhs, rhs));
    int total = 0, restarts = 0, status = CFO_OK;
    double rel = 0.0;
    if (!isfinite(bnorm)) { status = CFO_ENAN; rel = NAN; goto done; }
    if (bnorm == 0.0) { memset(x, 0, sizeof(double) * N); goto done; }
    for (;;) {
        int used = 0;
        int run = bicgstab_run(p, rhs, x, tol, bnorm, maxit - total, sweeps, &used, w);
        total += used;
        cfo_apply_B(p, x, w[8]);
        for (int64_t q = 0; q < N; ++q) w[8][q] = rhs[q] - w[8][q];
        rel = sqrt(dot(N, w[8], w[8])) / bnorm;
        if (run == RUN_NAN || !isfinite(rel)) { status = CFO_ENAN; break; }
        if (rel <= tol) { status = CFO_OK; break; }
        if (total >= maxit) { status = CFO_ENOCONV; break; }
        if (restarts == 3) { status = run == RUN_BREAK ? CFO_EBREAKDOWN : CFO_ENOCONV; break; }
        restarts++;
    }
done:
    for (int q = 0; q < 9; ++q) free(w[q]);
    if (iters) *iters = total;
    if (relres) *relres = rel;
    if (status) seterr(p, status == CFO_ENAN ? "non-finite residual" :
                          status == CFO_EBREAKDOWN ? "BiCGSTAB breakdown" : "no convergence");
    return status;
}

int cfo_solve(cfo_problem* p, const double* f, const double* g_nodes,
              const double* g_ibi, double* u, double tol, int maxit,
              int sweeps, int* iters, double* relres) {
    int st;
    if (!p->classified && (st = cfo_classify(p, NULL, NULL, NULL))) return st;
    if (!p->assembled && (st = cfo_assemble(p))) return st;
    double* rhs = (double*)malloc(sizeof(double) * p->N);
    if (!rhs) return CFO_ENOMEM;
    cfo_rhs(p, f, g_nodes, g_ibi, rhs);
    st = cfo_bicgstab(p, rhs, u, tol, maxit, sweeps, iters, relres);
    for (int64_t l = 0; l < p->N; ++l) {
        if (p->type[l] == CFO_BOUNDARY) u[l] = g_nodes[l];
        else if (p->type[l] == CFO_SOLID) u[l] = 0.0;
    }
    free(rhs);
    return st;
}
