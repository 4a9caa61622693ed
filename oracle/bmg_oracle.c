/*
 * bmg_oracle.c -- the ORACLE.  Test infrastructure only.
 *
 * A plain, slow, single-threaded FP64 restatement of the structured
 * black-box multigrid (BoxMG) solve on the computational grid that the
 * paper builds in Sec. 2 (weak form pulled back through the map, eq.
 * "weak_computational"), Sec. 2.1 (Q1 discretisation; effective
 * coefficient D_c = J_T (D o T^-1) J_T^T |J_T^-1|) and Sec. 2.2 (factor-two
 * structured coarsening, operator-induced interpolation, Galerkin coarse
 * operators, V-cycle).  The paper does not spell out BoxMG's formulas (it
 * cites Dendy 1982); the readings used here are the textbook ones:
 *   - interpolation by collapsing the fine stencil onto lines (edge points)
 *     and solving the fine equation at interior points; where a collapsed
 *     denominator is not positive (the collapse assumption fails on
 *     operators with strong positive couplings, e.g. coarse Galerkin
 *     operators of a degenerate map), that point uses its own uncollapsed
 *     couplings instead (the diagonal of an SPD operator is positive);
 *   - restriction R = P^T (Sec. 2.3, the transpose relation derived through
 *     Riesz maps);
 *   - coarse operators A_{l+1} = P^T A_l P, formed here by the definition,
 *     scattering every product P(i,K) A(i,j) P(j,L) of the explicit sparse
 *     operators;
 *   - multicolour Gauss-Seidel, colour = parity pattern of the node,
 *     forward colour order before the coarse correction, reverse after;
 *   - a conjugate-gradient outer loop preconditioned by one V-cycle;
 *   - an FP32 arm of the V-cycle (float copies of every level's operator
 *     and interpolation, float arithmetic throughout, FP64 solve on the
 *     3-node grid) as the preconditioner of FP64 flexible CG, the
 *     mixed-precision form of the solve.
 * Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load this file.  It shares no code with the CUDA library.
 *
 * Layouts (all row-major, i fastest):
 *   node   (i,j[,k])       -> i + n*(j + n*k)
 *   cell   (ci,cj[,ck])    -> ci + (n-1)*(cj + (n-1)*ck), cell = lower corner
 *   coords                 -> coords[c*n^d + node], c = physical component
 *   full stencil           -> A[node*S + o], S = 3^d,
 *                             o = (dx+1) + 3(dy+1) + 9(dz+1)
 *   interpolation          -> pw[f*2^d + s]: weight of fine node f to the
 *                             coarse node (f_i>>1 + s_x, f_j>>1 + s_y, ...),
 *                             s = s_x + 2 s_y + 4 s_z.  Weights to coarse
 *                             boundary nodes are stored as zero.
 * Boundary nodes carry zero Dirichlet data and are eliminated: their rows
 * and every coupling to them are zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Built twice: plain, and with -fopenmp for the CPU-baseline timing on all
   cores.  Only loops whose iterations write disjoint entries and read
   nothing another iteration writes are shared out (operator application,
   the points of one colour, prolongation, elementwise vector updates), so
   the results are bitwise those of the plain build; scatter loops
   (restriction, Galerkin products, assembly) and dot products stay
   sequential. */
#ifdef _OPENMP
#include <omp.h>
#define OR_PARALLEL_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OR_PARALLEL_FOR
#endif

int or_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_FOLDED = 2, OR_ERR_BREAKDOWN = 3,
       OR_ERR_NOT_SPD = 4, OR_ERR_NOT_CONVERGED = 5, OR_ERR_RANGE = 6 };

/* ------------------------------------------------------------------ */
/* grid helpers                                                        */
/* ------------------------------------------------------------------ */
static long pw_int(int b, int e) { long r = 1; while (e-- > 0) r *= b; return r; }

static void node_coords(int dim, int n, long id, int c[3]) {
    c[0] = (int)(id % n); id /= n;
    c[1] = dim > 1 ? (int)(id % n) : 0; id /= n;
    c[2] = dim > 2 ? (int)id : 0;
}

static long node_id(int dim, int n, const int c[3]) {
    long id = c[0];
    if (dim > 1) id += (long)n * c[1];
    if (dim > 2) id += (long)n * n * c[2];
    return id;
}

static int is_interior(int dim, int n, const int c[3]) {
    for (int d = 0; d < dim; d++)
        if (c[d] < 1 || c[d] > n - 2) return 0;
    return 1;
}

static int in_range(int dim, int n, const int c[3]) {
    for (int d = 0; d < dim; d++)
        if (c[d] < 0 || c[d] > n - 1) return 0;
    return 1;
}

/* stencil slot of offset d (components in -1..1) */
static int slot_of(int dim, const int d[3]) {
    int o = d[0] + 1;
    if (dim > 1) o += 3 * (d[1] + 1);
    if (dim > 2) o += 9 * (d[2] + 1);
    return o;
}

static void offset_of(int dim, int o, int d[3]) {
    d[0] = o % 3 - 1;
    d[1] = dim > 1 ? (o / 3) % 3 - 1 : 0;
    d[2] = dim > 2 ? o / 9 - 1 : 0;
}

/* ------------------------------------------------------------------ */
/* Q1 element on the reference cell [0,1]^d, 2-point Gauss per axis   */
/* ------------------------------------------------------------------ */
static void gauss_rule(double g[2]) {
    g[0] = 0.5 - 0.5 / sqrt(3.0);
    g[1] = 0.5 + 0.5 / sqrt(3.0);
}

/* value and reference gradient of basis function a at xi */
static double basis(int dim, int a, const double xi[3], double grad[3]) {
    double f[3], df[3];
    for (int d = 0; d < dim; d++) {
        int bit = (a >> d) & 1;
        f[d] = bit ? xi[d] : 1.0 - xi[d];
        df[d] = bit ? 1.0 : -1.0;
    }
    double v = 1.0;
    for (int d = 0; d < dim; d++) v *= f[d];
    for (int m = 0; m < dim; m++) {
        double g = df[m];
        for (int d = 0; d < dim; d++) if (d != m) g *= f[d];
        grad[m] = g;
    }
    return v;
}

static void quad_point(int dim, int q, double xi[3]) {
    double g[2];
    gauss_rule(g);
    xi[0] = xi[1] = xi[2] = 0.0;
    for (int d = 0; d < dim; d++) xi[d] = g[(q >> d) & 1];
}

/* Jacobian J[r][m] = d x_r / d xi_m at xi from the cell's nodal coordinates
   xe[r*2^d + a]; returns det J. */
static double jacobian(int dim, const double* xe, const double xi[3], double J[3][3]) {
    int na = 1 << dim;
    for (int r = 0; r < dim; r++)
        for (int m = 0; m < dim; m++) J[r][m] = 0.0;
    for (int a = 0; a < na; a++) {
        double gr[3];
        basis(dim, a, xi, gr);
        for (int r = 0; r < dim; r++)
            for (int m = 0; m < dim; m++) J[r][m] += xe[r * na + a] * gr[m];
    }
    if (dim == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
    return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1])
         - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
         + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static void inverse(int dim, double J[3][3], double det, double Ji[3][3]) {
    if (dim == 2) {
        Ji[0][0] = J[1][1] / det;  Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
        return;
    }
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

/* Metric in reference coordinates at quadrature point q:
   G = kappa * det J * J^-1 J^-T, the effective coefficient of Sec. 2.1
   with F = T^-1 (so J_T = J^-1).  Returns det J. */
static double metric(int dim, const double* xe, double kappa, int q, double G[3][3]) {
    double xi[3], J[3][3], Ji[3][3];
    quad_point(dim, q, xi);
    double det = jacobian(dim, xe, xi, J);
    if (!(det > 0.0)) return det;
    inverse(dim, J, det, Ji);
    for (int m = 0; m < dim; m++)
        for (int p = 0; p < dim; p++) {
            double s = 0.0;
            for (int r = 0; r < dim; r++) s += Ji[m][r] * Ji[p][r];
            G[m][p] = kappa * det * s;
        }
    return det;
}

/* Element stiffness K[a*2^d + b] = sum_q w_q grad(phi_a)^T G_q grad(phi_b),
   w_q = 2^-d (Gauss weights on the unit reference cell). */
int or_element(int dim, const double* xe, double kappa, double* K) {
    if (dim != 2 && dim != 3) return OR_ERR_ARG;
    int na = 1 << dim, nq = 1 << dim;
    double w = 1.0 / (double)nq;
    for (int t = 0; t < na * na; t++) K[t] = 0.0;
    for (int q = 0; q < nq; q++) {
        double G[3][3], xi[3];
        double det = metric(dim, xe, kappa, q, G);
        if (!(det > 0.0)) return OR_ERR_FOLDED;
        quad_point(dim, q, xi);
        double gr[8][3];
        for (int a = 0; a < na; a++) basis(dim, a, xi, gr[a]);
        for (int a = 0; a < na; a++)
            for (int b = 0; b < na; b++) {
                double s = 0.0;
                for (int m = 0; m < dim; m++)
                    for (int p = 0; p < dim; p++) s += gr[a][m] * G[m][p] * gr[b][p];
                K[a * na + b] += w * s;
            }
    }
    return OR_OK;
}

/* Effective coefficient in computational coordinates s = h*xi + const at
   each quadrature point: D_c = G / h^(d-2), with det(dx/ds) = det J / h^d.
   Dc[q*9 + m*3 + p], detJs[q]. */
int or_metric(int dim, const double* xe, double kappa, double h, double* detJs, double* Dc) {
    if (dim != 2 && dim != 3) return OR_ERR_ARG;
    int nq = 1 << dim;
    for (int q = 0; q < nq; q++) {
        double G[3][3];
        double det = metric(dim, xe, kappa, q, G);
        if (!(det > 0.0)) return OR_ERR_FOLDED;
        detJs[q] = det / pow(h, dim);
        for (int m = 0; m < 3; m++)
            for (int p = 0; p < 3; p++)
                Dc[q * 9 + m * 3 + p] = (m < dim && p < dim) ? G[m][p] / pow(h, dim - 2) : 0.0;
    }
    return OR_OK;
}

static void gather_cell(int dim, int n, const double* coords, const int cc[3], double* xe) {
    int na = 1 << dim;
    long nn = pw_int(n, dim);
    for (int a = 0; a < na; a++) {
        int c[3] = {cc[0] + (a & 1), cc[1] + ((a >> 1) & 1), cc[2] + ((a >> 2) & 1)};
        long id = node_id(dim, n, c);
        for (int r = 0; r < dim; r++) xe[r * na + a] = coords[r * nn + id];
    }
}

static void cell_coords(int dim, int n, long e, int cc[3]) {
    int m = n - 1;
    cc[0] = (int)(e % m); e /= m;
    cc[1] = dim > 1 ? (int)(e % m) : 0; e /= m;
    cc[2] = dim > 2 ? (int)e : 0;
}

/* ------------------------------------------------------------------ */
/* Assembly (Sec. 2.1): element by element into full stencils          */
/* ------------------------------------------------------------------ */
int or_assemble(int dim, int n, const double* coords, const double* kappa, double* A) {
    if ((dim != 2 && dim != 3) || n < 3) return OR_ERR_ARG;
    int S = (int)pw_int(3, dim), na = 1 << dim;
    long nn = pw_int(n, dim), ne = pw_int(n - 1, dim);
    memset(A, 0, sizeof(double) * nn * S);
    for (long e = 0; e < ne; e++) {
        int cc[3];
        double xe[24], K[64];
        cell_coords(dim, n, e, cc);
        gather_cell(dim, n, coords, cc, xe);
        int st = or_element(dim, xe, kappa[e], K);
        if (st) return st;
        for (int a = 0; a < na; a++) {
            int ca[3] = {cc[0] + (a & 1), cc[1] + ((a >> 1) & 1), cc[2] + ((a >> 2) & 1)};
            if (!is_interior(dim, n, ca)) continue;
            for (int b = 0; b < na; b++) {
                int cb[3] = {cc[0] + (b & 1), cc[1] + ((b >> 1) & 1), cc[2] + ((b >> 2) & 1)};
                if (!is_interior(dim, n, cb)) continue;   /* Dirichlet: drop coupling */
                int d[3] = {cb[0] - ca[0], cb[1] - ca[1], cb[2] - ca[2]};
                A[node_id(dim, n, ca) * S + slot_of(dim, d)] += K[a * na + b];
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Tensor coefficient (Sec. 2, Eq. pde; Sec. 2.1): an SPD diffusion     */
/* tensor D per cell, effective coefficient det J J^-1 D J^-T            */
/* ------------------------------------------------------------------ */

/* Upper triangle of cell e's tensor from planes of ne values each:
   2-D: D11, D12, D22; 3-D: D11, D12, D13, D22, D23, D33. */
static void cell_tensor(int dim, long ne, long e, const double* Dt, double D[3][3]) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) D[r][c] = 0.0;
    if (dim == 2) {
        D[0][0] = Dt[0 * ne + e];
        D[0][1] = D[1][0] = Dt[1 * ne + e];
        D[1][1] = Dt[2 * ne + e];
        return;
    }
    D[0][0] = Dt[0 * ne + e];
    D[0][1] = D[1][0] = Dt[1 * ne + e];
    D[0][2] = D[2][0] = Dt[2 * ne + e];
    D[1][1] = Dt[3 * ne + e];
    D[1][2] = D[2][1] = Dt[4 * ne + e];
    D[2][2] = Dt[5 * ne + e];
}

/* G = det J * J^-1 D J^-T at quadrature point q; returns det J. */
static double metric_tensor(int dim, const double* xe, double D[3][3], int q, double G[3][3]) {
    double xi[3], J[3][3], Ji[3][3];
    quad_point(dim, q, xi);
    double det = jacobian(dim, xe, xi, J);
    if (!(det > 0.0)) return det;
    inverse(dim, J, det, Ji);
    for (int m = 0; m < dim; m++)
        for (int p = 0; p < dim; p++) {
            double s = 0.0;
            for (int r = 0; r < dim; r++)
                for (int c = 0; c < dim; c++) s += Ji[m][r] * D[r][c] * Ji[p][c];
            G[m][p] = det * s;
        }
    return det;
}

/* Element stiffness with a constant tensor D (row-major 3x3). */
int or_element_tensor(int dim, const double* xe, const double* Dm, double* K) {
    if (dim != 2 && dim != 3) return OR_ERR_ARG;
    int na = 1 << dim, nq = 1 << dim;
    double w = 1.0 / (double)nq, D[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) D[r][c] = Dm[r * 3 + c];
    for (int t = 0; t < na * na; t++) K[t] = 0.0;
    for (int q = 0; q < nq; q++) {
        double G[3][3], xi[3];
        double det = metric_tensor(dim, xe, D, q, G);
        if (!(det > 0.0)) return OR_ERR_FOLDED;
        quad_point(dim, q, xi);
        double gr[8][3];
        for (int a = 0; a < na; a++) basis(dim, a, xi, gr[a]);
        for (int a = 0; a < na; a++)
            for (int b = 0; b < na; b++) {
                double s = 0.0;
                for (int m = 0; m < dim; m++)
                    for (int p = 0; p < dim; p++) s += gr[a][m] * G[m][p] * gr[b][p];
                K[a * na + b] += w * s;
            }
    }
    return OR_OK;
}

/* Assembly with a tensor per cell (planes as in cell_tensor), otherwise as
   or_assemble. */
int or_assemble_tensor(int dim, int n, const double* coords, const double* Dt, double* A) {
    if ((dim != 2 && dim != 3) || n < 3) return OR_ERR_ARG;
    int S = (int)pw_int(3, dim), na = 1 << dim;
    long nn = pw_int(n, dim), ne = pw_int(n - 1, dim);
    memset(A, 0, sizeof(double) * nn * S);
    for (long e = 0; e < ne; e++) {
        int cc[3];
        double xe[24], K[64], D[3][3];
        cell_coords(dim, n, e, cc);
        gather_cell(dim, n, coords, cc, xe);
        cell_tensor(dim, ne, e, Dt, D);
        int st = or_element_tensor(dim, xe, &D[0][0], K);
        if (st) return st;
        for (int a = 0; a < na; a++) {
            int ca[3] = {cc[0] + (a & 1), cc[1] + ((a >> 1) & 1), cc[2] + ((a >> 2) & 1)};
            if (!is_interior(dim, n, ca)) continue;
            for (int b = 0; b < na; b++) {
                int cb[3] = {cc[0] + (b & 1), cc[1] + ((b >> 1) & 1), cc[2] + ((b >> 2) & 1)};
                if (!is_interior(dim, n, cb)) continue;
                int d[3] = {cb[0] - ca[0], cb[1] - ca[1], cb[2] - ca[2]};
                A[node_id(dim, n, ca) * S + slot_of(dim, d)] += K[a * na + b];
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Dirichlet data (Sec. 2, Eq. weak_computational, the lift g term):    */
/* out_i = -sum over boundary nodes j of A_ij g_j, for interior i        */
/* ------------------------------------------------------------------ */
int or_boundary_rhs(int dim, int n, const double* coords, const double* kappa, const double* g, double* out) {
    if ((dim != 2 && dim != 3) || n < 3) return OR_ERR_ARG;
    int na = 1 << dim;
    long nn = pw_int(n, dim), ne = pw_int(n - 1, dim);
    memset(out, 0, sizeof(double) * nn);
    for (long e = 0; e < ne; e++) {
        int cc[3];
        double xe[24], K[64];
        cell_coords(dim, n, e, cc);
        gather_cell(dim, n, coords, cc, xe);
        int st = or_element(dim, xe, kappa[e], K);
        if (st) return st;
        for (int a = 0; a < na; a++) {
            int ca[3] = {cc[0] + (a & 1), cc[1] + ((a >> 1) & 1), cc[2] + ((a >> 2) & 1)};
            if (!is_interior(dim, n, ca)) continue;
            for (int b = 0; b < na; b++) {
                int cb[3] = {cc[0] + (b & 1), cc[1] + ((b >> 1) & 1), cc[2] + ((b >> 2) & 1)};
                if (is_interior(dim, n, cb)) continue;
                out[node_id(dim, n, ca)] -= K[a * na + b] * g[node_id(dim, n, cb)];
            }
        }
    }
    return OR_OK;
}

/* Physical coordinates of every quadrature point: xq[(e*2^d + q)*dim + r] */
int or_gauss_points(int dim, int n, const double* coords, double* xq) {
    if ((dim != 2 && dim != 3) || n < 2) return OR_ERR_ARG;
    int na = 1 << dim;
    long ne = pw_int(n - 1, dim);
    for (long e = 0; e < ne; e++) {
        int cc[3];
        double xe[24];
        cell_coords(dim, n, e, cc);
        gather_cell(dim, n, coords, cc, xe);
        for (int q = 0; q < na; q++) {
            double xi[3], gr[3];
            quad_point(dim, q, xi);
            for (int r = 0; r < dim; r++) {
                double s = 0.0;
                for (int a = 0; a < na; a++) s += xe[r * na + a] * basis(dim, a, xi, gr);
                xq[(e * na + q) * dim + r] = s;
            }
        }
    }
    return OR_OK;
}

/* Consistent load vector b_i = sum_e sum_q w_q f(x_q) phi_i(x_q) det J,
   f given at the quadrature points: fq[e*2^d + q].  Interior nodes only. */
int or_load(int dim, int n, const double* coords, const double* fq, double* b) {
    if ((dim != 2 && dim != 3) || n < 3) return OR_ERR_ARG;
    int na = 1 << dim;
    long nn = pw_int(n, dim), ne = pw_int(n - 1, dim);
    memset(b, 0, sizeof(double) * nn);
    double w = 1.0 / (double)na;
    for (long e = 0; e < ne; e++) {
        int cc[3];
        double xe[24];
        cell_coords(dim, n, e, cc);
        gather_cell(dim, n, coords, cc, xe);
        for (int q = 0; q < na; q++) {
            double xi[3], J[3][3], gr[3];
            quad_point(dim, q, xi);
            double det = jacobian(dim, xe, xi, J);
            if (!(det > 0.0)) return OR_ERR_FOLDED;
            for (int a = 0; a < na; a++) {
                int ca[3] = {cc[0] + (a & 1), cc[1] + ((a >> 1) & 1), cc[2] + ((a >> 2) & 1)};
                if (!is_interior(dim, n, ca)) continue;
                b[node_id(dim, n, ca)] += w * fq[e * na + q] * basis(dim, a, xi, gr) * det;
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Operator application and multicolour Gauss-Seidel                   */
/* ------------------------------------------------------------------ */
void or_apply(int dim, int n, const double* A, const double* x, double* y) {
    int S = (int)pw_int(3, dim);
    long nn = pw_int(n, dim);
    OR_PARALLEL_FOR
    for (long id = 0; id < nn; id++) {
        int c[3];
        node_coords(dim, n, id, c);
        if (!is_interior(dim, n, c)) { y[id] = 0.0; continue; }
        double s = 0.0;
        for (int o = 0; o < S; o++) {
            int d[3];
            offset_of(dim, o, d);
            int cn[3] = {c[0] + d[0], c[1] + d[1], c[2] + d[2]};
            s += A[id * S + o] * x[node_id(dim, n, cn)];
        }
        y[id] = s;
    }
}

static int colour_of(int dim, const int c[3]) {
    int col = (c[0] & 1) + 2 * (c[1] & 1);
    if (dim > 2) col += 4 * (c[2] & 1);
    return col;
}

/* One multicolour Gauss-Seidel sweep; colours 0..C-1, or C-1..0 if reverse.
   x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii for all i of the colour. */
void or_smooth(int dim, int n, const double* A, const double* b, double* x, int reverse) {
    int S = (int)pw_int(3, dim), C = 1 << dim, ctr = (S - 1) / 2;
    long nn = pw_int(n, dim);
    for (int cc = 0; cc < C; cc++) {
        int col = reverse ? C - 1 - cc : cc;
        OR_PARALLEL_FOR
        for (long id = 0; id < nn; id++) {
            int c[3];
            node_coords(dim, n, id, c);
            if (!is_interior(dim, n, c) || colour_of(dim, c) != col) continue;
            double s = b[id];
            for (int o = 0; o < S; o++) {
                if (o == ctr) continue;
                int d[3];
                offset_of(dim, o, d);
                int cn[3] = {c[0] + d[0], c[1] + d[1], c[2] + d[2]};
                s -= A[id * S + o] * x[node_id(dim, n, cn)];
            }
            x[id] = s / A[id * S + ctr];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Operator-induced interpolation (Sec. 2.2; Dendy's collapse)          */
/* ------------------------------------------------------------------ */
typedef struct { int cnt; long idx[8]; double w[8]; } prow_t;

static void prow_add(prow_t* r, long idx, double w) {
    for (int t = 0; t < r->cnt; t++)
        if (r->idx[t] == idx) { r->w[t] += w; return; }
    r->idx[r->cnt] = idx;
    r->w[r->cnt] = w;
    r->cnt++;
}

/* row of fine node f read back from the slot storage, as global coarse ids */
static void prow_get(int dim, int nf, const double* pw, long f, prow_t* r) {
    int nc = (nf + 1) / 2, ns = 1 << dim;
    int c[3];
    node_coords(dim, nf, f, c);
    r->cnt = 0;
    for (int s = 0; s < ns; s++) {
        double w = pw[f * ns + s];
        if (w == 0.0) continue;
        int k[3] = {(c[0] >> 1) + (s & 1), (c[1] >> 1) + ((s >> 1) & 1), (c[2] >> 1) + ((s >> 2) & 1)};
        prow_add(r, node_id(dim, nc, k), w);
    }
}

static int prow_put(int dim, int nf, double* pw, long f, const prow_t* r) {
    int nc = (nf + 1) / 2, ns = 1 << dim;
    int c[3];
    node_coords(dim, nf, f, c);
    for (int s = 0; s < ns; s++) pw[f * ns + s] = 0.0;
    for (int t = 0; t < r->cnt; t++) {
        int k[3];
        node_coords(dim, nc, r->idx[t], k);
        int s = 0;
        for (int d = 0; d < dim; d++) {
            int sd = k[d] - (c[d] >> 1);
            if (sd < 0 || sd > 1) return OR_ERR_RANGE;
            s += sd << d;
        }
        if (is_interior(dim, nc, k)) pw[f * ns + s] = r->w[t];  /* boundary coarse values are 0 */
    }
    return OR_OK;
}

/* Sum of the stencil entries of node f over all offsets whose components
   along the axes in `keep` equal `kd`, summing over the other axes.  This
   is the "collapsed" stencil. */
static double collapsed(int dim, const double* A, long f, int keepmask, const int kd[3]) {
    int S = (int)pw_int(3, dim);
    double s = 0.0;
    for (int o = 0; o < S; o++) {
        int d[3], ok = 1;
        offset_of(dim, o, d);
        for (int a = 0; a < dim; a++)
            if (((keepmask >> a) & 1) && d[a] != kd[a]) ok = 0;
        if (ok) s += A[f * S + o];
    }
    return s;
}

int or_interp(int dim, int nf, const double* A, double* pw) {
    if ((dim != 2 && dim != 3) || nf < 5 || ((nf - 1) & (nf - 2))) return OR_ERR_ARG;
    int ns = 1 << dim;
    long nn = pw_int(nf, dim);
    memset(pw, 0, sizeof(double) * nn * ns);
    /* pass p handles fine nodes with exactly p odd coordinates */
    for (int p = 0; p <= dim; p++) {
        for (long f = 0; f < nn; f++) {
            int c[3];
            node_coords(dim, nf, f, c);
            if (!is_interior(dim, nf, c)) continue;
            int oddmask = 0, nodd = 0;
            for (int a = 0; a < dim; a++)
                if (c[a] & 1) { oddmask |= 1 << a; nodd++; }
            if (nodd != p) continue;
            prow_t row = {0};
            int nc = (nf + 1) / 2;
            if (p == 0) {
                int k[3] = {c[0] / 2, c[1] / 2, c[2] / 2};
                prow_add(&row, node_id(dim, nc, k), 1.0);
            } else if (p == 1) {
                /* line point: collapse onto the odd axis a */
                int a = 0;
                while (!((oddmask >> a) & 1)) a++;
                int km[3] = {0, 0, 0}, k0[3] = {0, 0, 0}, kp[3] = {0, 0, 0};
                km[a] = -1; kp[a] = 1;
                double AL = collapsed(dim, A, f, 1 << a, km);
                double A0 = collapsed(dim, A, f, 1 << a, k0);
                double AR = collapsed(dim, A, f, 1 << a, kp);
                if (!(A0 > 0.0)) {
                    /* collapse not usable: the point's own couplings along the axis */
                    int S = (int)pw_int(3, dim), ctr = (S - 1) / 2;
                    int dm[3] = {0, 0, 0}, dp[3] = {0, 0, 0};
                    dm[a] = -1; dp[a] = 1;
                    AL = A[f * S + slot_of(dim, dm)];
                    AR = A[f * S + slot_of(dim, dp)];
                    A0 = A[f * S + ctr];
                    if (!(A0 > 0.0)) return OR_ERR_BREAKDOWN;
                }
                int cl[3] = {c[0], c[1], c[2]}, cr[3] = {c[0], c[1], c[2]};
                cl[a] -= 1; cr[a] += 1;
                int kl[3] = {cl[0] / 2, cl[1] / 2, cl[2] / 2}, kr[3] = {cr[0] / 2, cr[1] / 2, cr[2] / 2};
                prow_add(&row, node_id(dim, nc, kl), -AL / A0);
                prow_add(&row, node_id(dim, nc, kr), -AR / A0);
            } else {
                /* p == 2 in 3D: collapse over the even axis, then solve the
                   collapsed plane equation; p == dim: solve the full fine
                   equation.  Neighbours are interpolated by their own rows. */
                int S = (int)pw_int(3, dim), ctr = (S - 1) / 2;
                int evenmask = ((1 << dim) - 1) & ~oddmask;
                double diag;
                double coef[27];
                for (int o = 0; o < S; o++) coef[o] = 0.0;
                /* coefficient per in-plane offset: sum over the even axes */
                for (int o = 0; o < S; o++) {
                    int d[3];
                    offset_of(dim, o, d);
                    int dp[3] = {d[0], d[1], d[2]};
                    for (int a = 0; a < dim; a++) if ((evenmask >> a) & 1) dp[a] = 0;
                    coef[slot_of(dim, dp)] += A[f * S + o];
                }
                diag = coef[ctr];
                if (!(diag > 0.0) && evenmask) {
                    /* collapse not usable: the point's own in-plane couplings */
                    for (int o = 0; o < S; o++) {
                        int d[3], inplane = 1;
                        offset_of(dim, o, d);
                        for (int a = 0; a < dim; a++)
                            if (((evenmask >> a) & 1) && d[a] != 0) inplane = 0;
                        coef[o] = inplane ? A[f * S + o] : 0.0;
                    }
                    diag = coef[ctr];
                }
                if (!(diag > 0.0)) return OR_ERR_BREAKDOWN;
                for (int o = 0; o < S; o++) {
                    if (o == ctr || coef[o] == 0.0) continue;
                    int d[3];
                    offset_of(dim, o, d);
                    int cn[3] = {c[0] + d[0], c[1] + d[1], c[2] + d[2]};
                    if (!is_interior(dim, nf, cn)) continue;  /* value 0 */
                    prow_t nb;
                    prow_get(dim, nf, pw, node_id(dim, nf, cn), &nb);
                    for (int t = 0; t < nb.cnt; t++) prow_add(&row, nb.idx[t], -coef[o] * nb.w[t] / diag);
                }
            }
            int st = prow_put(dim, nf, pw, f, &row);
            if (st) return st;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Galerkin coarse operator by definition: Ac = P^T A P                 */
/* ------------------------------------------------------------------ */
int or_rap(int dim, int nf, const double* Af, const double* pw, double* Ac) {
    if ((dim != 2 && dim != 3) || nf < 5) return OR_ERR_ARG;
    int S = (int)pw_int(3, dim), ns = 1 << dim, nc = (nf + 1) / 2;
    long nn = pw_int(nf, dim), ncn = pw_int(nc, dim);
    memset(Ac, 0, sizeof(double) * ncn * S);
    for (long i = 0; i < nn; i++) {
        int ci[3];
        node_coords(dim, nf, i, ci);
        if (!is_interior(dim, nf, ci)) continue;
        for (int o = 0; o < S; o++) {
            double a = Af[i * S + o];
            if (a == 0.0) continue;
            int d[3];
            offset_of(dim, o, d);
            int cj[3] = {ci[0] + d[0], ci[1] + d[1], ci[2] + d[2]};
            if (!in_range(dim, nf, cj)) return OR_ERR_RANGE;
            long j = node_id(dim, nf, cj);
            for (int s = 0; s < ns; s++) {
                double wi = pw[i * ns + s];
                if (wi == 0.0) continue;
                int K[3] = {(ci[0] >> 1) + (s & 1), (ci[1] >> 1) + ((s >> 1) & 1), (ci[2] >> 1) + ((s >> 2) & 1)};
                for (int t = 0; t < ns; t++) {
                    double wj = pw[j * ns + t];
                    if (wj == 0.0) continue;
                    int L[3] = {(cj[0] >> 1) + (t & 1), (cj[1] >> 1) + ((t >> 1) & 1), (cj[2] >> 1) + ((t >> 2) & 1)};
                    int dd[3] = {L[0] - K[0], L[1] - K[1], L[2] - K[2]};
                    for (int a = 0; a < dim; a++)
                        if (dd[a] < -1 || dd[a] > 1) return OR_ERR_RANGE;
                    Ac[node_id(dim, nc, K) * S + slot_of(dim, dd)] += wi * a * wj;
                }
            }
        }
    }
    return OR_OK;
}

/* restriction bc = P^T r  (R = P^T, Sec. 2.3) */
void or_restrict(int dim, int nf, const double* pw, const double* r, double* bc) {
    int ns = 1 << dim, nc = (nf + 1) / 2;
    long nn = pw_int(nf, dim), ncn = pw_int(nc, dim);
    memset(bc, 0, sizeof(double) * ncn);
    for (long i = 0; i < nn; i++) {
        int ci[3];
        node_coords(dim, nf, i, ci);
        if (!is_interior(dim, nf, ci)) continue;
        for (int s = 0; s < ns; s++) {
            double w = pw[i * ns + s];
            if (w == 0.0) continue;
            int K[3] = {(ci[0] >> 1) + (s & 1), (ci[1] >> 1) + ((s >> 1) & 1), (ci[2] >> 1) + ((s >> 2) & 1)};
            bc[node_id(dim, nc, K)] += w * r[i];
        }
    }
}

/* prolongation with correction x += P xc */
void or_prolong(int dim, int nf, const double* pw, const double* xc, double* x) {
    int ns = 1 << dim, nc = (nf + 1) / 2;
    long nn = pw_int(nf, dim);
    OR_PARALLEL_FOR
    for (long i = 0; i < nn; i++) {
        int ci[3];
        node_coords(dim, nf, i, ci);
        if (!is_interior(dim, nf, ci)) continue;
        double s = 0.0;
        for (int sl = 0; sl < ns; sl++) {
            double w = pw[i * ns + sl];
            if (w == 0.0) continue;
            int K[3] = {(ci[0] >> 1) + (sl & 1), (ci[1] >> 1) + ((sl >> 1) & 1), (ci[2] >> 1) + ((sl >> 2) & 1)};
            s += w * xc[node_id(dim, nc, K)];
        }
        x[i] += s;
    }
}

/* ------------------------------------------------------------------ */
/* Hierarchy, V-cycle and preconditioned CG                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int dim, nlev;
    int n[32];
    double* A[32];   /* full stencils per level */
    double* P[32];   /* interpolation from level l+1 to level l */
    double* b[32];
    double* x[32];
    double* r[32];
    /* FP32 arm: float copies of A and P and float level vectors, made on
       the first FP32 V-cycle */
    float* A32[32];
    float* P32[32];
    float* b32[32];
    float* x32[32];
    float* r32[32];
} or_hier;

static double dot(long nn, const double* a, const double* b) {
    double s = 0.0;
    for (long i = 0; i < nn; i++) s += a[i] * b[i];
    return s;
}

void or_hier_free(or_hier* h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; l++) {
        free(h->A[l]); free(h->P[l]); free(h->b[l]); free(h->x[l]); free(h->r[l]);
        free(h->A32[l]); free(h->P32[l]); free(h->b32[l]); free(h->x32[l]); free(h->r32[l]);
    }
    free(h);
}


/* Builds the hierarchy from the finest full stencil (copied).  Each level
   halves the cell count per axis (factor-two coarsening, Sec. 2.2) down to
   3 nodes per side, which leaves one unknown. */
int or_hier_create(int dim, int n, const double* A, or_hier** out) {
    *out = NULL;
    if ((dim != 2 && dim != 3) || n < 3 || ((n - 1) & (n - 2))) return OR_ERR_ARG;
    or_hier* h = (or_hier*)calloc(1, sizeof(or_hier));
    h->dim = dim;
    int S = (int)pw_int(3, dim), ns = 1 << dim;
    h->n[0] = n;
    h->A[0] = (double*)malloc(sizeof(double) * pw_int(n, dim) * S);
    memcpy(h->A[0], A, sizeof(double) * pw_int(n, dim) * S);
    for (int l = 0;; l++) {
        int nl = h->n[l];
        long nn = pw_int(nl, dim);
        h->b[l] = (double*)calloc(nn, sizeof(double));
        h->x[l] = (double*)calloc(nn, sizeof(double));
        h->r[l] = (double*)calloc(nn, sizeof(double));
        h->nlev = l + 1;
        if (nl == 3) break;
        h->P[l] = (double*)malloc(sizeof(double) * nn * ns);
        int st = or_interp(dim, nl, h->A[l], h->P[l]);
        if (st) { or_hier_free(h); return st; }
        int nc = (nl + 1) / 2;
        h->n[l + 1] = nc;
        h->A[l + 1] = (double*)malloc(sizeof(double) * pw_int(nc, dim) * S);
        st = or_rap(dim, nl, h->A[l], h->P[l], h->A[l + 1]);
        if (st) { h->nlev = l + 2; or_hier_free(h); return st; }
    }
    *out = h;
    return OR_OK;
}

int or_hier_levels(const or_hier* h) { return h->nlev; }
int or_hier_n(const or_hier* h, int l) { return h->n[l]; }
void or_hier_get_A(const or_hier* h, int l, double* out) {
    memcpy(out, h->A[l], sizeof(double) * pw_int(h->n[l], h->dim) * pw_int(3, h->dim));
}
void or_hier_get_P(const or_hier* h, int l, double* out) {
    memcpy(out, h->P[l], sizeof(double) * pw_int(h->n[l], h->dim) * (1 << h->dim));
}

/* V(1,1)-cycle on level l with zero initial guess: x_l = M_l b_l.
   Coarsest level (one unknown): exact scalar solve. */
static void vcycle_level(or_hier* h, int l) {
    int dim = h->dim, n = h->n[l], S = (int)pw_int(3, dim), ctr = (S - 1) / 2;
    long nn = pw_int(n, dim);
    memset(h->x[l], 0, sizeof(double) * nn);
    if (l == h->nlev - 1) {
        int c[3] = {1, 1, 1};
        long id = node_id(dim, n, c);
        h->x[l][id] = h->b[l][id] / h->A[l][id * S + ctr];
        return;
    }
    or_smooth(dim, n, h->A[l], h->b[l], h->x[l], 0);
    or_apply(dim, n, h->A[l], h->x[l], h->r[l]);
    OR_PARALLEL_FOR
    for (long i = 0; i < nn; i++) h->r[l][i] = h->b[l][i] - h->r[l][i];
    or_restrict(dim, n, h->P[l], h->r[l], h->b[l + 1]);
    vcycle_level(h, l + 1);
    or_prolong(dim, n, h->P[l], h->x[l + 1], h->x[l]);
    or_smooth(dim, n, h->A[l], h->b[l], h->x[l], 1);
}

/* z = M r: one V(1,1)-cycle from a zero initial guess.  Boundary entries
   of r are ignored; z is zero on the boundary. */
void or_vcycle(or_hier* h, const double* r, double* z) {
    int dim = h->dim, n = h->n[0];
    long nn = pw_int(n, dim);
    for (long i = 0; i < nn; i++) {
        int c[3];
        node_coords(dim, n, i, c);
        h->b[0][i] = is_interior(dim, n, c) ? r[i] : 0.0;
    }
    vcycle_level(h, 0);
    memcpy(z, h->x[0], sizeof(double) * nn);
}

/* ------------------------------------------------------------------ */
/* FP32 arm: the same V-cycle with single-precision arithmetic          */
/* ------------------------------------------------------------------ */
/* The FP32 preconditioner of the mixed-precision solve: every level's
   operator and interpolation rounded once to float (round to nearest),
   and every smoothing, residual, restriction and prolongation step
   evaluated in float variables, so each product and each partial sum is
   rounded to single precision.  The exact solve on the 3-node grid stays
   in FP64 (the one unknown's equation, float right-hand side widened,
   FP64 diagonal, result rounded to float).  The steps and their order are
   those of the FP64 functions above. */
static void apply32(int dim, int n, const float* A, const float* x, float* y) {
    int S = (int)pw_int(3, dim);
    long nn = pw_int(n, dim);
    for (long id = 0; id < nn; id++) {
        int c[3];
        node_coords(dim, n, id, c);
        if (!is_interior(dim, n, c)) { y[id] = 0.0f; continue; }
        float s = 0.0f;
        for (int o = 0; o < S; o++) {
            int d[3];
            offset_of(dim, o, d);
            int cn[3] = {c[0] + d[0], c[1] + d[1], c[2] + d[2]};
            float t = A[id * S + o] * x[node_id(dim, n, cn)];
            s = s + t;
        }
        y[id] = s;
    }
}

static void smooth32(int dim, int n, const float* A, const float* b, float* x, int reverse) {
    int S = (int)pw_int(3, dim), C = 1 << dim, ctr = (S - 1) / 2;
    long nn = pw_int(n, dim);
    for (int cc = 0; cc < C; cc++) {
        int col = reverse ? C - 1 - cc : cc;
        for (long id = 0; id < nn; id++) {
            int c[3];
            node_coords(dim, n, id, c);
            if (!is_interior(dim, n, c) || colour_of(dim, c) != col) continue;
            float s = b[id];
            for (int o = 0; o < S; o++) {
                if (o == ctr) continue;
                int d[3];
                offset_of(dim, o, d);
                int cn[3] = {c[0] + d[0], c[1] + d[1], c[2] + d[2]};
                float t = A[id * S + o] * x[node_id(dim, n, cn)];
                s = s - t;
            }
            x[id] = s / A[id * S + ctr];
        }
    }
}

static void restrict32(int dim, int nf, const float* pw, const float* r, float* bc) {
    int ns = 1 << dim, nc = (nf + 1) / 2;
    long nn = pw_int(nf, dim), ncn = pw_int(nc, dim);
    for (long k = 0; k < ncn; k++) bc[k] = 0.0f;
    for (long i = 0; i < nn; i++) {
        int ci[3];
        node_coords(dim, nf, i, ci);
        if (!is_interior(dim, nf, ci)) continue;
        for (int s = 0; s < ns; s++) {
            float w = pw[i * ns + s];
            if (w == 0.0f) continue;
            int K[3] = {(ci[0] >> 1) + (s & 1), (ci[1] >> 1) + ((s >> 1) & 1), (ci[2] >> 1) + ((s >> 2) & 1)};
            long k = node_id(dim, nc, K);
            float t = w * r[i];
            bc[k] = bc[k] + t;
        }
    }
}

static void prolong32(int dim, int nf, const float* pw, const float* xc, float* x) {
    int ns = 1 << dim, nc = (nf + 1) / 2;
    long nn = pw_int(nf, dim);
    for (long i = 0; i < nn; i++) {
        int ci[3];
        node_coords(dim, nf, i, ci);
        if (!is_interior(dim, nf, ci)) continue;
        float s = 0.0f;
        for (int sl = 0; sl < ns; sl++) {
            float w = pw[i * ns + sl];
            if (w == 0.0f) continue;
            int K[3] = {(ci[0] >> 1) + (sl & 1), (ci[1] >> 1) + ((sl >> 1) & 1), (ci[2] >> 1) + ((sl >> 2) & 1)};
            float t = w * xc[node_id(dim, nc, K)];
            s = s + t;
        }
        x[i] = x[i] + s;
    }
}

/* float copies of every level, rounded once from the FP64 hierarchy */
static void make32(or_hier* h) {
    if (h->A32[0]) return;
    int dim = h->dim, S = (int)pw_int(3, dim), ns = 1 << dim;
    for (int l = 0; l < h->nlev; l++) {
        long nn = pw_int(h->n[l], dim);
        h->A32[l] = (float*)malloc(sizeof(float) * nn * S);
        for (long k = 0; k < nn * S; k++) h->A32[l][k] = (float)h->A[l][k];
        if (l < h->nlev - 1) {
            h->P32[l] = (float*)malloc(sizeof(float) * nn * ns);
            for (long k = 0; k < nn * ns; k++) h->P32[l][k] = (float)h->P[l][k];
        }
        h->b32[l] = (float*)calloc(nn, sizeof(float));
        h->x32[l] = (float*)calloc(nn, sizeof(float));
        h->r32[l] = (float*)calloc(nn, sizeof(float));
    }
}

static void vcycle32_level(or_hier* h, int l) {
    int dim = h->dim, n = h->n[l], S = (int)pw_int(3, dim), ctr = (S - 1) / 2;
    long nn = pw_int(n, dim);
    for (long i = 0; i < nn; i++) h->x32[l][i] = 0.0f;
    if (l == h->nlev - 1) {
        int c[3] = {1, 1, 1};
        long id = node_id(dim, n, c);
        h->x32[l][id] = (float)((double)h->b32[l][id] / h->A[l][id * S + ctr]);
        return;
    }
    smooth32(dim, n, h->A32[l], h->b32[l], h->x32[l], 0);
    apply32(dim, n, h->A32[l], h->x32[l], h->r32[l]);
    for (long i = 0; i < nn; i++) h->r32[l][i] = h->b32[l][i] - h->r32[l][i];
    restrict32(dim, n, h->P32[l], h->r32[l], h->b32[l + 1]);
    vcycle32_level(h, l + 1);
    prolong32(dim, n, h->P32[l], h->x32[l + 1], h->x32[l]);
    smooth32(dim, n, h->A32[l], h->b32[l], h->x32[l], 1);
}

/* z = M32 r: one FP32 V(1,1)-cycle from a zero initial guess; r is rounded
   to float on entry and the result widened to double. */
void or_vcycle32(or_hier* h, const double* r, double* z) {
    make32(h);
    int dim = h->dim, n = h->n[0];
    long nn = pw_int(n, dim);
    for (long i = 0; i < nn; i++) {
        int c[3];
        node_coords(dim, n, i, c);
        h->b32[0][i] = is_interior(dim, n, c) ? (float)r[i] : 0.0f;
    }
    vcycle32_level(h, 0);
    for (long i = 0; i < nn; i++) z[i] = (double)h->x32[0][i];
}

/* Preconditioned conjugate gradients with M = one V-cycle.
   mode bit 0 clear: beta = r_{k+1}.z_{k+1} / r_k.z_k;
   mode bit 0 set (flexible): beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k;
   mode bit 1 set: M is the FP32 V-cycle (or_vcycle32), every vector, dot
   product and update of the CG itself staying FP64.
   Stops when ||r_k|| <= tol ||b|| for the recursive residual AND the true
   residual b - A x; when only the recursive one passes, r is replaced by
   the true residual and the iteration continues.  maxit caps the
   iterations; tol <= 0 runs exactly maxit iterations.
   hist[k] = ||r_k|| / ||b|| (recursive), k = 0..iters.  */
int or_pcg(or_hier* h, const double* b, double* x, double tol, int maxit, int mode,
           int* iters, double* hist, double* true_relres) {
    int dim = h->dim, n = h->n[0];
    int flexible = mode & 1;
    void (*precond)(or_hier*, const double*, double*) = (mode & 2) ? or_vcycle32 : or_vcycle;
    long nn = pw_int(n, dim);
    double* r = (double*)calloc(nn, sizeof(double));
    double* z = (double*)calloc(nn, sizeof(double));
    double* zo = (double*)calloc(nn, sizeof(double));
    double* p = (double*)calloc(nn, sizeof(double));
    double* q = (double*)calloc(nn, sizeof(double));
    double* bb = (double*)calloc(nn, sizeof(double));
    int st = OR_ERR_NOT_CONVERGED, k = 0;
    for (long i = 0; i < nn; i++) {
        int c[3];
        node_coords(dim, n, i, c);
        bb[i] = is_interior(dim, n, c) ? b[i] : 0.0;
        if (!is_interior(dim, n, c)) x[i] = 0.0;
    }
    double bnorm = sqrt(dot(nn, bb, bb));
    or_apply(dim, n, h->A[0], x, q);
    for (long i = 0; i < nn; i++) r[i] = bb[i] - q[i];
    double rn = sqrt(dot(nn, r, r));
    if (hist) hist[0] = bnorm > 0 ? rn / bnorm : 0.0;
    if (bnorm == 0.0) { st = OR_OK; goto done; }
    if (tol > 0 && rn <= tol * bnorm) { st = OR_OK; goto done; }
    precond(h, r, z);
    for (long i = 0; i < nn; i++) p[i] = z[i];
    double rz = dot(nn, r, z);
    for (k = 1; k <= maxit; k++) {
        or_apply(dim, n, h->A[0], p, q);
        double pq = dot(nn, p, q);
        if (!(pq > 0.0)) { st = OR_ERR_NOT_SPD; break; }
        double alpha = rz / pq;
        OR_PARALLEL_FOR
        for (long i = 0; i < nn; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rn = sqrt(dot(nn, r, r));
        if (hist) hist[k] = rn / bnorm;
        if (tol > 0 && rn <= tol * bnorm) {
            or_apply(dim, n, h->A[0], x, q);
            for (long i = 0; i < nn; i++) r[i] = bb[i] - q[i];
            rn = sqrt(dot(nn, r, r));
            if (rn <= tol * bnorm) { st = OR_OK; break; }
        }
        if (k == maxit) break;
        if (flexible) memcpy(zo, z, sizeof(double) * nn);
        precond(h, r, z);
        double rzn = dot(nn, r, z);
        double beta = flexible ? (rzn - dot(nn, r, zo)) / rz : rzn / rz;
        OR_PARALLEL_FOR
        for (long i = 0; i < nn; i++) p[i] = z[i] + beta * p[i];
        rz = rzn;
    }
    if (k > maxit) k = maxit;
    if (tol <= 0 && st == OR_ERR_NOT_CONVERGED) st = OR_OK;
done:
    if (iters) *iters = k;
    or_apply(dim, n, h->A[0], x, q);
    {
        double s = 0.0;
        for (long i = 0; i < nn; i++) { double d = bb[i] - q[i]; s += d * d; }
        if (true_relres) *true_relres = bnorm > 0 ? sqrt(s) / bnorm : 0.0;
    }
    free(r); free(z); free(zo); free(p); free(q); free(bb);
    return st;
}

/* ------------------------------------------------------------------ */
/* Adjoint gradient with respect to a per-cell coefficient              */
/* ------------------------------------------------------------------ */
/* For A(kappa) u = b and a loss L(u) with adjoint A lambda = dL/du, the
   derivative with respect to the cell coefficient kappa_e is
   dL/dkappa_e = -lambda_e^T K_e^0 u_e, K_e^0 the element matrix at
   kappa = 1 (A is linear in kappa_e).  Boundary values of u and lambda are
   zero, which removes the eliminated couplings. */
int or_adjoint_grad(int dim, int n, const double* coords, const double* u,
                    const double* lam, double* dLdkappa) {
    if ((dim != 2 && dim != 3) || n < 3) return OR_ERR_ARG;
    int na = 1 << dim;
    long ne = pw_int(n - 1, dim);
    for (long e = 0; e < ne; e++) {
        int cc[3];
        double xe[24], K[64], ue[8], le[8];
        cell_coords(dim, n, e, cc);
        gather_cell(dim, n, coords, cc, xe);
        int st = or_element(dim, xe, 1.0, K);
        if (st) return st;
        for (int a = 0; a < na; a++) {
            int ca[3] = {cc[0] + (a & 1), cc[1] + ((a >> 1) & 1), cc[2] + ((a >> 2) & 1)};
            long id = node_id(dim, n, ca);
            int in = is_interior(dim, n, ca);
            ue[a] = in ? u[id] : 0.0;
            le[a] = in ? lam[id] : 0.0;
        }
        double s = 0.0;
        for (int a = 0; a < na; a++)
            for (int b = 0; b < na; b++) s += le[a] * K[a * na + b] * ue[b];
        dLdkappa[e] = -s;
    }
    return OR_OK;
}
