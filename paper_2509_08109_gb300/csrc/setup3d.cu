// setup3d.cu -- 3-D setup kernels: trilinear Q1 assembly from the map
// (Sec. 2.1 in 3-D: 2x2x2 Gauss points, effective coefficient
// kappa det J J^-1 J^-T), operator-induced interpolation by hierarchical
// collapse (lines, then planes, then the cell centre) and Galerkin coarse
// operators P^T A P (Sec. 2.2), exports and the per-cell adjoint contraction.
#include "common.cuh"
#include "grid3.cuh"

namespace bmg {
namespace {

constexpr double kG0 = 0.21132486540518711775;
constexpr double kG1 = 0.78867513459481288225;

// Coefficient of a cell, as the metric it induces from adj(J) = det J J^-1
// (the 1/8 is the Gauss weight).  Scalar kappa: G = (kappa / det J) adj
// adj^T.  SPD tensor D (Sec. 2, Eq. pde): G = (1 / det J) adj D adj^T.
struct Scalar3 {
    double kap;
    __device__ __forceinline__ void metric(const double adj[3][3], double det, double G[3][3]) const {
        const double s = 0.125 * kap / det;
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
            for (int p = 0; p < 3; p++)
                G[m][p] = s * (adj[m][0] * adj[p][0] + adj[m][1] * adj[p][1] + adj[m][2] * adj[p][2]);
    }
};
struct Tensor3 {
    double d[3][3];
    __device__ __forceinline__ void metric(const double adj[3][3], double det, double G[3][3]) const {
        const double s = 0.125 / det;
        double t[3][3];   // adj D
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
            for (int c = 0; c < 3; c++) t[m][c] = adj[m][0] * d[0][c] + adj[m][1] * d[1][c] + adj[m][2] * d[2][c];
#pragma unroll
        for (int m = 0; m < 3; m++)
#pragma unroll
            for (int p = 0; p < 3; p++)
                G[m][p] = s * (t[m][0] * adj[p][0] + t[m][1] * adj[p][1] + t[m][2] * adj[p][2]);
    }
};

// Row `a` of the trilinear element matrix of cell (ci,cj,ck):
// Krow[b] = sum_q 1/8 grad(phi_a)^T G grad(phi_b), G from the cell's
// coefficient (above).  Corner b = bx + 2 by + 4 bz sits at node
// (ci+bx, cj+by, ck+bz).
template <class C>
__device__ bool element_row3d(const double* __restrict__ coords, int n, int ci, int cj, int ck, const C& coef, int a,
                              double Krow[8]) {
    const long long nn = (long long)n * n * n;
    double xa[3][8];
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const long long id = (long long)(ci + (b & 1)) + (long long)n * ((cj + ((b >> 1) & 1)) + (long long)n * (ck + (b >> 2)));
#pragma unroll
        for (int r = 0; r < 3; r++) xa[r][b] = coords[r * nn + id];
    }
#pragma unroll
    for (int b = 0; b < 8; b++) Krow[b] = 0.0;
    bool ok = true;
    for (int q = 0; q < 8; q++) {
        const double xi[3] = {(q & 1) ? kG1 : kG0, (q & 2) ? kG1 : kG0, (q & 4) ? kG1 : kG0};
        double g[8][3];
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const double f0 = (b & 1) ? xi[0] : 1.0 - xi[0];
            const double f1 = (b & 2) ? xi[1] : 1.0 - xi[1];
            const double f2 = (b & 4) ? xi[2] : 1.0 - xi[2];
            const double d0 = (b & 1) ? 1.0 : -1.0, d1 = (b & 2) ? 1.0 : -1.0, d2 = (b & 4) ? 1.0 : -1.0;
            g[b][0] = d0 * f1 * f2;
            g[b][1] = f0 * d1 * f2;
            g[b][2] = f0 * f1 * d2;
        }
        double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
        for (int b = 0; b < 8; b++)
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int m = 0; m < 3; m++) J[r][m] += xa[r][b] * g[b][m];
        // adjugate (transpose of the cofactor matrix): J^-1 = adj / det
        double adj[3][3];
        adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
        if (!(det > 0.0)) ok = false;
        double G[3][3];
        coef.metric(adj, det, G);
        const double ga0 = G[0][0] * g[a][0] + G[0][1] * g[a][1] + G[0][2] * g[a][2];
        const double ga1 = G[1][0] * g[a][0] + G[1][1] * g[a][1] + G[1][2] * g[a][2];
        const double ga2 = G[2][0] * g[a][0] + G[2][1] * g[a][1] + G[2][2] * g[a][2];
#pragma unroll
        for (int b = 0; b < 8; b++) Krow[b] += ga0 * g[b][0] + ga1 * g[b][1] + ga2 * g[b][2];
    }
    return ok;
}

__device__ __forceinline__ bool inner3(int n, int i, int j, int k) {
    return i >= 1 && j >= 1 && k >= 1 && i <= n - 2 && j <= n - 2 && k <= n - 2;
}

// Gather assembly: one thread per node, the 8 surrounding cells, the
// stored half of the 27-point row (14 planes).
// coefficient of cell e: kappa[e], or the tensor planes D11, D12, D13, D22,
// D23, D33 (ne cells each)
template <bool TENSOR>
__device__ __forceinline__ auto cell_coef3(const double* __restrict__ c, long long ne, long long e) {
    if constexpr (TENSOR) {
        const double d11 = c[e], d12 = c[ne + e], d13 = c[2 * ne + e], d22 = c[3 * ne + e], d23 = c[4 * ne + e],
                     d33 = c[5 * ne + e];
        return Tensor3{{{d11, d12, d13}, {d12, d22, d23}, {d13, d23, d33}}};
    } else {
        return Scalar3{c[e]};
    }
}

template <bool TENSOR>
__global__ void k_assemble3d(int n, int ld, long long pl, const double* __restrict__ coords,
                             const double* __restrict__ kappa, double* __restrict__ A, KState* st) {
    const long long ne = (long long)(n - 1) * (n - 1) * (n - 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= n) return;
    const long long o = (long long)i + (long long)ld * (j + (long long)n * k);
    double acc[14];
#pragma unroll
    for (int t = 0; t < 14; t++) acc[t] = 0.0;
    if (inner3(n, i, j, k)) {
        bool ok = true;
        for (int cz = 0; cz < 2; cz++)
            for (int cy = 0; cy < 2; cy++)
                for (int cx = 0; cx < 2; cx++) {
                    const int ci = i - 1 + cx, cj = j - 1 + cy, ck = k - 1 + cz;
                    const int a = (1 - cx) + 2 * (1 - cy) + 4 * (1 - cz);
                    const long long e = (long long)ci + (long long)(n - 1) * (cj + (long long)(n - 1) * ck);
                    double Kr[8];
                    ok &= element_row3d(coords, n, ci, cj, ck, cell_coef3<TENSOR>(kappa, ne, e), a, Kr);
                    for (int b = 0; b < 8; b++) {
                        const int dx = (b & 1) - (a & 1), dy = ((b >> 1) & 1) - ((a >> 1) & 1),
                                  dz = (b >> 2) - (a >> 2);
                        const int oo = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                        if (oo > 13) continue;
                        if (oo < 13 && !inner3(n, i + dx, j + dy, k + dz)) continue;
                        acc[oo] += Kr[b];
                    }
                }
        if (!ok) set_err(st, BMG_ERR_MAP_FOLDED);
    }
#pragma unroll
    for (int t = 0; t < 14; t++) A[(long long)t * pl + o] = acc[t];
}

__global__ void k_set_stencil3d(int n, int ld, long long pl, const double* __restrict__ full, double* __restrict__ A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= n) return;
    const long long o = (long long)i + (long long)ld * (j + (long long)n * k);
    const bool in = inner3(n, i, j, k);
    const double* row = full + ((long long)i + (long long)n * (j + (long long)n * k)) * 27;
    for (int t = 0; t < 14; t++) {
        double v = 0.0;
        if (in && (t == 13 || inner3(n, i + off_x(t), j + off_y(t), k + off_z(t)))) v = row[t];
        A[(long long)t * pl + o] = v;
    }
}

struct CoarseDims {
    int nf, nc, ldc;
    long long plc;
    __device__ __forceinline__ long long at(int I, int J, int K) const {
        return (long long)I + (long long)ldc * (J + (long long)nc * K);
    }
    __device__ __forceinline__ bool inner(int I, int J, int K) const {
        return I >= 1 && J >= 1 && K >= 1 && I <= nc - 2 && J <= nc - 2 && K <= nc - 2;
    }
};

// Line points (one odd coordinate): collapse the 27-point row over the plane
// perpendicular to the odd axis.  Where the collapsed denominator is not
// positive the point uses its own couplings along the axis (a_000 > 0).
__global__ void k_interp_lines3d(Sten3<double> F, CoarseDims D, double* __restrict__ P, KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I >= D.nc) return;
    const long long oc = D.at(I, J, K);
    for (int a = 0; a < 3; a++) {
        const int fi = 2 * I + (a == 0), fj = 2 * J + (a == 1), fk = 2 * K + (a == 2);
        double lo = 0.0, hi = 0.0;
        if (inner3(D.nf, fi, fj, fk)) {
            double S[3] = {0, 0, 0};
            for (int o = 0; o < 27; o++) {
                const int d = a == 0 ? off_x(o) : a == 1 ? off_y(o) : off_z(o);
                S[d + 1] += F.full(fi, fj, fk, o);
            }
            if (!(S[1] > 0.0)) {
                const int step = a == 0 ? 1 : a == 1 ? 3 : 9;   // offset of +e_a in the 27-numbering
                S[0] = F.full(fi, fj, fk, 13 - step);
                S[1] = F.full(fi, fj, fk, 13);
                S[2] = F.full(fi, fj, fk, 13 + step);
            }
            if (!(S[1] > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
            const int ax[3] = {I, J, K};
            lo = ax[a] >= 1 ? -S[0] / S[1] : 0.0;
            hi = ax[a] + 1 <= D.nc - 2 ? -S[2] / S[1] : 0.0;
        }
        const int base = kPBase(1 << a);
        P[(long long)base * D.plc + oc] = lo;
        P[(long long)(base + 1) * D.plc + oc] = hi;
    }
}

// Plane points (two odd coordinates): collapse over the even axis, then solve
// the collapsed plane equation with the in-plane neighbours interpolated.
// Where the collapsed diagonal is not positive the point uses its own
// in-plane couplings (no collapse; the diagonal a_000 > 0).
__global__ void k_interp_planes3d(Sten3<double> F, CoarseDims D, double* __restrict__ P, KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I >= D.nc) return;
    const long long oc = D.at(I, J, K);
    const int masks[3] = {3, 5, 6};
    for (int t = 0; t < 3; t++) {
        const int m = masks[t];
        const int e = m == 3 ? 2 : m == 5 ? 1 : 0;   // the even axis
        const int fi = 2 * I + (m & 1), fj = 2 * J + ((m >> 1) & 1), fk = 2 * K + ((m >> 2) & 1);
        double w[4] = {0, 0, 0, 0};
        if (inner3(D.nf, fi, fj, fk)) {
            double cf[27];
            for (int o = 0; o < 27; o++) cf[o] = 0.0;
            for (int o = 0; o < 27; o++) {
                int dx = off_x(o), dy = off_y(o), dz = off_z(o);
                if (e == 0) dx = 0;
                if (e == 1) dy = 0;
                if (e == 2) dz = 0;
                cf[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] += F.full(fi, fj, fk, o);
            }
            if (!(cf[13] > 0.0)) {
                for (int o = 0; o < 27; o++) {
                    const int de = e == 0 ? off_x(o) : e == 1 ? off_y(o) : off_z(o);
                    cf[o] = de == 0 ? F.full(fi, fj, fk, o) : 0.0;
                }
            }
            const double d0 = cf[13];
            if (!(d0 > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
            for (int c = 0; c < 4; c++) {
                // corner c of the (odd-axis) cell: bits over m's axes
                int s = 0, b = 0;
                for (int a = 0; a < 3; a++)
                    if ((m >> a) & 1) {
                        s |= ((c >> b) & 1) << a;
                        b++;
                    }
                const int KI = I + (s & 1), KJ = J + ((s >> 1) & 1), KK = K + ((s >> 2) & 1);
                double acc = 0.0;
                for (int o = 0; o < 27; o++) {
                    if (o == 13 || cf[o] == 0.0) continue;
                    acc += cf[o] * pweight3(P, D.ldc, D.nc, D.plc, D.nf, fi + off_x(o), fj + off_y(o), fk + off_z(o), KI,
                                            KJ, KK);
                }
                w[c] = D.inner(KI, KJ, KK) ? -acc / d0 : 0.0;
            }
        }
        for (int c = 0; c < 4; c++) P[(long long)(kPBase(m) + c) * D.plc + oc] = w[c];
    }
}

// Cell centre (three odd coordinates): solve the full fine equation with the
// 26 neighbours interpolated by their own rows.
__global__ void k_interp_centre3d(Sten3<double> F, CoarseDims D, double* __restrict__ P, KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I >= D.nc) return;
    const long long oc = D.at(I, J, K);
    const int fi = 2 * I + 1, fj = 2 * J + 1, fk = 2 * K + 1;
    double w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (inner3(D.nf, fi, fj, fk)) {
        const double d0 = F.full(fi, fj, fk, 13);
        if (!(d0 > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
        for (int s = 0; s < 8; s++) {
            const int KI = I + (s & 1), KJ = J + ((s >> 1) & 1), KK = K + (s >> 2);
            double acc = 0.0;
            for (int o = 0; o < 27; o++) {
                if (o == 13) continue;
                const double a = F.full(fi, fj, fk, o);
                if (a == 0.0) continue;
                acc += a * pweight3(P, D.ldc, D.nc, D.plc, D.nf, fi + off_x(o), fj + off_y(o), fk + off_z(o), KI, KJ, KK);
            }
            w[s] = D.inner(KI, KJ, KK) ? -acc / d0 : 0.0;
        }
    }
    for (int s = 0; s < 8; s++) P[(long long)(kPBase(7) + s) * D.plc + oc] = w[s];
}

// Galerkin coarse operator: A_c(K, K+d) for the 14 stored offsets d.
__global__ void k_rap3d(Sten3<double> F, CoarseDims D, const double* __restrict__ P, double* __restrict__ Ac,
                        KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I >= D.nc) return;
    const long long oc = D.at(I, J, K);
    double acc[14];
    for (int t = 0; t < 14; t++) acc[t] = 0.0;
    if (D.inner(I, J, K)) {
        for (int fz = 2 * K - 1; fz <= 2 * K + 1; fz++)
            for (int fy = 2 * J - 1; fy <= 2 * J + 1; fy++)
                for (int fx = 2 * I - 1; fx <= 2 * I + 1; fx++) {
                    const double wK = pweight3(P, D.ldc, D.nc, D.plc, D.nf, fx, fy, fz, I, J, K);
                    if (wK == 0.0) continue;
                    for (int o = 0; o < 27; o++) {
                        const double a = F.full(fx, fy, fz, o);
                        if (a == 0.0) continue;
                        const int jx = fx + off_x(o), jy = fy + off_y(o), jz = fz + off_z(o);
                        for (int s = 0; s < 8; s++) {
                            const int LI = (jx >> 1) + (s & 1), LJ = (jy >> 1) + ((s >> 1) & 1), LK = (jz >> 1) + (s >> 2);
                            const int dx = LI - I, dy = LJ - J, dz = LK - K;
                            if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) continue;
                            const int oo = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                            if (oo > 13) continue;
                            const double wL = pweight3(P, D.ldc, D.nc, D.plc, D.nf, jx, jy, jz, LI, LJ, LK);
                            if (wL == 0.0) continue;
                            acc[oo] += wK * a * wL;
                        }
                    }
                }
        if (!(acc[13] > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
    }
    for (int t = 0; t < 14; t++) Ac[(long long)t * D.plc + oc] = acc[t];
}

__global__ void k_export_stencil3d(Sten3<double> F, double* __restrict__ out) {
    const int n = F.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= n) return;
    double* row = out + ((long long)i + (long long)n * (j + (long long)n * k)) * 27;
    const bool in = inner3(n, i, j, k);
    for (int o = 0; o < 27; o++) row[o] = in ? F.full(i, j, k, o) : 0.0;
}

__global__ void k_export_interp3d(const double* __restrict__ P, CoarseDims D, double* __restrict__ out) {
    const int nf = D.nf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= nf) return;
    double* row = out + ((long long)i + (long long)nf * (j + (long long)nf * k)) * 8;
    for (int s = 0; s < 8; s++)
        row[s] = pweight3(P, D.ldc, D.nc, D.plc, nf, i, j, k, (i >> 1) + (s & 1), (j >> 1) + ((s >> 1) & 1),
                          (k >> 1) + (s >> 2));
}

// out_i = -sum over boundary nodes j of A_ij g_j at interior nodes i, as in 2-D.
__global__ void k_boundary_rhs3d(int n, const double* __restrict__ coords, const double* __restrict__ kappa,
                                 const double* __restrict__ g, double* __restrict__ out, KState* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= n) return;
    double acc = 0.0;
    if (inner3(n, i, j, k)) {
        bool ok = true;
        for (int cz = 0; cz < 2; cz++)
            for (int cy = 0; cy < 2; cy++)
                for (int cx = 0; cx < 2; cx++) {
                    const int ci = i - 1 + cx, cj = j - 1 + cy, ck = k - 1 + cz;
                    const int a = (1 - cx) + 2 * (1 - cy) + 4 * (1 - cz);
                    const double kap = kappa[(long long)ci + (long long)(n - 1) * (cj + (long long)(n - 1) * ck)];
                    double Kr[8];
                    ok &= element_row3d(coords, n, ci, cj, ck, Scalar3{kap}, a, Kr);
                    for (int b = 0; b < 8; b++) {
                        const int bi = ci + (b & 1), bj = cj + ((b >> 1) & 1), bk = ck + (b >> 2);
                        if (inner3(n, bi, bj, bk)) continue;
                        acc -= Kr[b] * g[(long long)bi + (long long)n * (bj + (long long)n * bk)];
                    }
                }
        if (!ok) set_err(st, BMG_ERR_MAP_FOLDED);
    }
    out[(long long)i + (long long)n * (j + (long long)n * k)] = acc;
}

__global__ void k_adjoint_cells3d(int n, const double* __restrict__ coords, const double* __restrict__ u,
                                  const double* __restrict__ lam, double* __restrict__ g, KState* st) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    const int cj = blockIdx.y, ck = blockIdx.z;
    if (ci >= n - 1) return;
    double ue[8], le[8];
    for (int b = 0; b < 8; b++) {
        const int i = ci + (b & 1), j = cj + ((b >> 1) & 1), k = ck + (b >> 2);
        const long long id = (long long)i + (long long)n * (j + (long long)n * k);
        const bool in = inner3(n, i, j, k);
        ue[b] = in ? u[id] : 0.0;
        le[b] = in ? lam[id] : 0.0;
    }
    double s = 0.0;
    bool ok = true;
    for (int a = 0; a < 8; a++) {
        if (le[a] == 0.0) continue;
        double Kr[8];
        ok &= element_row3d(coords, n, ci, cj, ck, Scalar3{1.0}, a, Kr);
        double t = 0.0;
        for (int b = 0; b < 8; b++) t += Kr[b] * ue[b];
        s += le[a] * t;
    }
    if (!ok) set_err(st, BMG_ERR_MAP_FOLDED);
    g[(long long)ci + (long long)(n - 1) * (cj + (long long)(n - 1) * ck)] = -s;
}

inline dim3 grid3(int ni, int nj, int nk) { return dim3(cdiv(ni, 64), nj, nk); }

}  // namespace

bmg_status assemble3d(Ctx& c, const double* coords, const double* kappa) {
    Level& L = c.lev[0];
    k_assemble3d<false><<<grid3(L.n, L.n, L.n), 64, 0, c.stream>>>(L.n, L.ld, L.plane, coords, kappa, L.A64, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// As assemble_export2d: assembly into caller-given half planes, then export.
bmg_status assemble_export3d(int n, int ld, long long pl, const double* coords, const double* kappa, double* A,
                             KState* st, double* out, cudaStream_t s) {
    k_assemble3d<false><<<grid3(n, n, n), 64, 0, s>>>(n, ld, pl, coords, kappa, A, st);
    BMG_CUDA(cudaGetLastError());
    k_export_stencil3d<<<grid3(n, n, n), 64, 0, s>>>(Sten3<double>{A, n, ld, pl}, out);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status assemble_tensor3d(Ctx& c, const double* coords, const double* D) {
    Level& L = c.lev[0];
    k_assemble3d<true><<<grid3(L.n, L.n, L.n), 64, 0, c.stream>>>(L.n, L.ld, L.plane, coords, D, L.A64, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status boundary_rhs3d(Ctx& c, const double* coords, const double* kappa, const double* g, double* out) {
    const int n = c.lev[0].n;
    k_boundary_rhs3d<<<grid3(n, n, n), 64, 0, c.stream>>>(n, coords, kappa, g, out, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status set_stencil3d(Ctx& c, const double* full) {
    Level& L = c.lev[0];
    k_set_stencil3d<<<grid3(L.n, L.n, L.n), 64, 0, c.stream>>>(L.n, L.ld, L.plane, full, L.A64);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status setup_level3d(Ctx& c, int l) {
    Level& F = c.lev[l];
    Level& K = c.lev[l + 1];
    Sten3<double> fs{F.A64, F.n, F.ld, F.plane};
    CoarseDims D{F.n, K.n, K.ld, K.plane};
    const dim3 g = grid3(K.n, K.n, K.n);
    k_interp_lines3d<<<g, 64, 0, c.stream>>>(fs, D, F.P64, c.st);
    k_interp_planes3d<<<g, 64, 0, c.stream>>>(fs, D, F.P64, c.st);
    k_interp_centre3d<<<g, 64, 0, c.stream>>>(fs, D, F.P64, c.st);
    k_rap3d<<<g, 64, 0, c.stream>>>(fs, D, F.P64, K.A64, c.st);
    c.launches += 4;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status export_stencil3d(Ctx& c, int l, double* out) {
    Level& L = c.lev[l];
    k_export_stencil3d<<<grid3(L.n, L.n, L.n), 64, 0, c.stream>>>(Sten3<double>{L.A64, L.n, L.ld, L.plane}, out);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status export_interp3d(Ctx& c, int l, double* out) {
    Level& F = c.lev[l];
    Level& K = c.lev[l + 1];
    k_export_interp3d<<<grid3(F.n, F.n, F.n), 64, 0, c.stream>>>(F.P64, CoarseDims{F.n, K.n, K.ld, K.plane}, out);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status adjoint_cells3d(Ctx& c, const double* coords, const double* u, const double* lam, double* g) {
    const int n = c.lev[0].n;
    k_adjoint_cells3d<<<grid3(n - 1, n - 1, n - 1), 64, 0, c.stream>>>(n, coords, u, lam, g, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
