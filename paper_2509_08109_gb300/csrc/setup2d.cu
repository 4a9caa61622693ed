// setup2d.cu -- 2-D setup kernels: Q1 assembly from the map (Sec. 2.1),
// operator-induced interpolation and Galerkin coarse operators (Sec. 2.2),
// exports for diagnostics, and the per-cell adjoint contraction.
#include "common.cuh"

namespace bmg {
namespace {

// 2-point Gauss nodes on [0,1]: 1/2 -+ 1/(2 sqrt 3)
constexpr double kG0 = 0.21132486540518711775;
constexpr double kG1 = 0.78867513459481288225;

// Coefficient of a cell, as the metric it induces from adj(J) = det J J^-1.
// Scalar kappa: G = (kappa / det J) adj adj^T.  SPD tensor D (Sec. 2, Eq.
// pde): G = (1 / det J) adj D adj^T, i.e. det J J^-1 D J^-T (Sec. 2.1).
struct Scalar2 {
    double kap;
    __device__ __forceinline__ void metric(double J11, double J12, double J21, double J22, double det, double& G11,
                                           double& G12, double& G22) const {
        const double s = 0.25 * kap / det;
        G11 = s * (J22 * J22 + J12 * J12);
        G12 = -s * (J22 * J21 + J12 * J11);
        G22 = s * (J21 * J21 + J11 * J11);
    }
};
struct Tensor2 {
    double d11, d12, d22;
    __device__ __forceinline__ void metric(double J11, double J12, double J21, double J22, double det, double& G11,
                                           double& G12, double& G22) const {
        const double a11 = J22, a12 = -J12, a21 = -J21, a22 = J11;   // adj(J)
        const double t11 = a11 * d11 + a12 * d12, t12 = a11 * d12 + a12 * d22;
        const double t21 = a21 * d11 + a22 * d12, t22 = a21 * d12 + a22 * d22;
        const double s = 0.25 / det;
        G11 = s * (t11 * a11 + t12 * a12);
        G12 = s * (t11 * a21 + t12 * a22);
        G22 = s * (t21 * a21 + t22 * a22);
    }
};

// Q1 element matrix of cell (ci,cj): K[a][b] = sum_q 1/4 grad(phi_a)^T G grad(phi_b),
// G from the cell's coefficient (above), J = dx/dxi on the reference cell
// (isoparametric map of the four nodal coordinates).  Corner a = ax + 2 ay
// sits at node (ci+ax, cj+ay).  Returns false if det J <= 0.
template <class C>
__device__ bool element2d(const double* __restrict__ X, const double* __restrict__ Y, int n, int ci, int cj,
                          const C& coef, double K[4][4]) {
    double xa[4], ya[4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        long long id = (long long)(cj + (a >> 1)) * n + (ci + (a & 1));
        xa[a] = X[id];
        ya[a] = Y[id];
    }
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) K[a][b] = 0.0;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const double xi = (q & 1) ? kG1 : kG0, eta = (q & 2) ? kG1 : kG0;
        const double dxi[4] = {-(1.0 - eta), 1.0 - eta, -eta, eta};
        const double det_[4] = {-(1.0 - xi), -xi, 1.0 - xi, xi};
        double J11 = 0, J12 = 0, J21 = 0, J22 = 0;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            J11 += xa[a] * dxi[a];
            J12 += xa[a] * det_[a];
            J21 += ya[a] * dxi[a];
            J22 += ya[a] * det_[a];
        }
        const double det = J11 * J22 - J12 * J21;
        if (!(det > 0.0)) ok = false;
        double G11, G12, G22;
        coef.metric(J11, J12, J21, J22, det, G11, G12, G22);
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const double ga = G11 * dxi[a] + G12 * det_[a];
            const double gb = G12 * dxi[a] + G22 * det_[a];
#pragma unroll
            for (int b = 0; b < 4; b++) K[a][b] += ga * dxi[b] + gb * det_[b];
        }
    }
    return ok;
}

// coefficient of cell e: kappa[e], or the tensor planes D11, D12, D22 (ne cells each)
template <bool TENSOR>
__device__ __forceinline__ auto cell_coef2(const double* __restrict__ c, long long ne, long long e) {
    if constexpr (TENSOR)
        return Tensor2{c[e], c[ne + e], c[2 * ne + e]};
    else
        return Scalar2{c[e]};
}

// Gather assembly (no atomics), tiled so that each cell's element matrix is
// formed once per tile rather than once per node of the cell: a CTA of 256
// threads owns kAsmTX x kAsmTY nodes, first forms the element matrices of
// the (kAsmTX+1) x (kAsmTY+1) cells around them (one cell per thread) into
// shared memory, then each node sums its four cells' entries in a fixed
// order.  Couplings to boundary nodes are dropped; boundary rows are zero.
constexpr int kAsmTX = 31, kAsmTY = 7;
constexpr int kAsmCX = kAsmTX + 1, kAsmCells = (kAsmTX + 1) * (kAsmTY + 1);   // 256
// the ten entries of a cell matrix the gather uses
enum AsmEntry { E00, E11, E22, E33, E10, E12, E20, E30, E31, E32, NE2 };

template <bool TENSOR>
__global__ void __launch_bounds__(kAsmCells) k_assemble2d(int n, int ld, long long pl,
                                                          const double* __restrict__ coords,
                                                          const double* __restrict__ kappa, double* __restrict__ A,
                                                          KState* st) {
    __shared__ double sK[NE2][kAsmCells];
    const long long ne = (long long)(n - 1) * (n - 1);
    const int i0 = blockIdx.x * kAsmTX, j0 = blockIdx.y * kAsmTY;    // first node of the tile
    const int t = threadIdx.x;
    {
        // cell (ci, cj) lies between nodes ci, ci+1 and cj, cj+1
        const int ci = i0 - 1 + t % kAsmCX, cj = j0 - 1 + t / kAsmCX;
        if (ci >= 0 && cj >= 0 && ci <= n - 2 && cj <= n - 2) {
            double K[4][4];
            const double* X = coords;
            const double* Y = coords + (long long)n * n;
            if (!element2d(X, Y, n, ci, cj, cell_coef2<TENSOR>(kappa, ne, (long long)cj * (n - 1) + ci), K))
                set_err(st, BMG_ERR_MAP_FOLDED);
            sK[E00][t] = K[0][0];
            sK[E11][t] = K[1][1];
            sK[E22][t] = K[2][2];
            sK[E33][t] = K[3][3];
            sK[E10][t] = K[1][0];
            sK[E12][t] = K[1][2];
            sK[E20][t] = K[2][0];
            sK[E30][t] = K[3][0];
            sK[E31][t] = K[3][1];
            sK[E32][t] = K[3][2];
        }
    }
    __syncthreads();
    if (t >= kAsmTX * kAsmTY) return;
    const int i = i0 + t % kAsmTX, j = j0 + t / kAsmTX;
    if (i >= n || j >= n) return;
    const long long o = (long long)j * ld + i;
    double C = 0, W = 0, S = 0, SW = 0, NW = 0;
    if (i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2) {
        // shared-memory slot of the cell whose lower-left node is (ci, cj)
        auto cell = [&](int ci, int cj) { return (ci - i0 + 1) + kAsmCX * (cj - j0 + 1); };
        // cell (i-1,j-1): node is corner 3
        int e = cell(i - 1, j - 1);
        C += sK[E33][e];
        if (i - 1 >= 1) W += sK[E32][e];
        if (j - 1 >= 1) S += sK[E31][e];
        if (i - 1 >= 1 && j - 1 >= 1) SW += sK[E30][e];
        // cell (i,j-1): node is corner 2
        e = cell(i, j - 1);
        C += sK[E22][e];
        if (j - 1 >= 1) S += sK[E20][e];
        // cell (i-1,j): node is corner 1
        e = cell(i - 1, j);
        C += sK[E11][e];
        if (i - 1 >= 1) W += sK[E10][e];
        if (i - 1 >= 1 && j + 1 <= n - 2) NW += sK[E12][e];
        // cell (i,j): node is corner 0
        e = cell(i, j);
        C += sK[E00][e];
    }
    A[C2 * pl + o] = C;
    A[W2 * pl + o] = W;
    A[S2 * pl + o] = S;
    A[SW2 * pl + o] = SW;
    A[NW2 * pl + o] = NW;
}

inline dim3 grid_asm(int n) { return dim3(cdiv(n, kAsmTX), cdiv(n, kAsmTY)); }

// Full 9-entry rows -> symmetric half planes; couplings to boundary nodes
// and boundary rows are forced to zero.
__global__ void k_set_stencil2d(int n, int ld, long long pl, const double* __restrict__ full,
                                double* __restrict__ A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    const long long o = (long long)j * ld + i;
    double C = 0, W = 0, S = 0, SW = 0, NW = 0;
    if (i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2) {
        const double* row = full + ((long long)j * n + i) * 9;
        C = row[4];
        W = i > 1 ? row[3] : 0.0;
        S = j > 1 ? row[1] : 0.0;
        SW = (i > 1 && j > 1) ? row[0] : 0.0;
        NW = (i > 1 && j < n - 2) ? row[6] : 0.0;
    }
    A[C2 * pl + o] = C;
    A[W2 * pl + o] = W;
    A[S2 * pl + o] = S;
    A[SW2 * pl + o] = SW;
    A[NW2 * pl + o] = NW;
}

// Edge points of the fine grid, owned by coarse node (I,J):
//   (2I+1, 2J): collapse the stencil over dy -> weights -A_L/A_0, -A_R/A_0
//   (2I, 2J+1): collapse over dx               -> weights -A_S/A_0, -A_N/A_0
// Where the collapsed denominator A_0 is not positive the point uses its own
// couplings along the line instead (A_0 = a_00 > 0 for an SPD operator).
// Weights to boundary coarse nodes and rows of boundary fine points are 0.
__global__ void k_interp_edges2d(Sten2<double> F, int nf, int nc, int ldc, long long plc,
                                 double* __restrict__ P, KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I >= nc) return;
    const long long o = (long long)J * ldc + I;
    double xl = 0, xr = 0, ys = 0, yn = 0;
    {   // x-edge point
        const int i = 2 * I + 1, j = 2 * J;
        if (i <= nf - 2 && j >= 1 && j <= nf - 2) {
            double AL = F.full(i, j, -1, -1) + F.full(i, j, -1, 0) + F.full(i, j, -1, 1);
            double A0 = F.full(i, j, 0, -1) + F.full(i, j, 0, 0) + F.full(i, j, 0, 1);
            double AR = F.full(i, j, 1, -1) + F.full(i, j, 1, 0) + F.full(i, j, 1, 1);
            if (!(A0 > 0.0)) {
                AL = F.full(i, j, -1, 0);
                AR = F.full(i, j, 1, 0);
                A0 = F.c(i, j);
            }
            if (!(A0 > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
            xl = (I >= 1) ? -AL / A0 : 0.0;
            xr = (I + 1 <= nc - 2) ? -AR / A0 : 0.0;
        }
    }
    {   // y-edge point
        const int i = 2 * I, j = 2 * J + 1;
        if (i >= 1 && i <= nf - 2 && j <= nf - 2) {
            double AS = F.full(i, j, -1, -1) + F.full(i, j, 0, -1) + F.full(i, j, 1, -1);
            double A0 = F.full(i, j, -1, 0) + F.full(i, j, 0, 0) + F.full(i, j, 1, 0);
            double AN = F.full(i, j, -1, 1) + F.full(i, j, 0, 1) + F.full(i, j, 1, 1);
            if (!(A0 > 0.0)) {
                AS = F.full(i, j, 0, -1);
                AN = F.full(i, j, 0, 1);
                A0 = F.c(i, j);
            }
            if (!(A0 > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
            ys = (J >= 1) ? -AS / A0 : 0.0;
            yn = (J + 1 <= nc - 2) ? -AN / A0 : 0.0;
        }
    }
    P[PXL * plc + o] = xl;
    P[PXR * plc + o] = xr;
    P[PYS * plc + o] = ys;
    P[PYN * plc + o] = yn;
}

// Interior point (2I+1, 2J+1): solve the fine equation with its four C
// neighbours (coarse values) and four edge neighbours (their edge
// interpolation):  v = -(1/a00) sum_{d != 0} a_d v(i+d).
__global__ void k_interp_interior2d(Sten2<double> F, int nf, int nc, int ldc, long long plc,
                                    double* __restrict__ P, KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I >= nc) return;
    const long long o = (long long)J * ldc + I;
    double sw = 0, se = 0, nw = 0, ne = 0;
    const int i = 2 * I + 1, j = 2 * J + 1;
    if (i <= nf - 2 && j <= nf - 2) {
        const double a00 = F.c(i, j);
        if (!(a00 > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
        auto Pv = [&](int p, int II, int JJ) { return P[p * plc + (long long)JJ * ldc + II]; };
        // edge neighbours: south (i,j-1) = x-edge of (I,J); north (i,j+1) = x-edge of (I,J+1);
        //                  west (i-1,j) = y-edge of (I,J);  east (i+1,j) = y-edge of (I+1,J)
        const double aS = F.full(i, j, 0, -1), aN = F.full(i, j, 0, 1);
        const double aW = F.full(i, j, -1, 0), aE = F.full(i, j, 1, 0);
        const double sxl = Pv(PXL, I, J), sxr = Pv(PXR, I, J);
        const double nxl = Pv(PXL, I, J + 1), nxr = Pv(PXR, I, J + 1);
        const double wys = Pv(PYS, I, J), wyn = Pv(PYN, I, J);
        const double eys = Pv(PYS, I + 1, J), eyn = Pv(PYN, I + 1, J);
        const double inv = -1.0 / a00;
        sw = (F.full(i, j, -1, -1) + aS * sxl + aW * wys) * inv;
        se = (F.full(i, j, 1, -1) + aS * sxr + aE * eys) * inv;
        nw = (F.full(i, j, -1, 1) + aN * nxl + aW * wyn) * inv;
        ne = (F.full(i, j, 1, 1) + aN * nxr + aE * eyn) * inv;
        if (I < 1 || J < 1) sw = 0.0;
        if (I + 1 > nc - 2 || J < 1) se = 0.0;
        if (I < 1 || J + 1 > nc - 2) nw = 0.0;
        if (I + 1 > nc - 2 || J + 1 > nc - 2) ne = 0.0;
    }
    P[PSW * plc + o] = sw;
    P[PSE * plc + o] = se;
    P[PNW * plc + o] = nw;
    P[PNE * plc + o] = ne;
}

// Weight of fine node (fi,fj) to coarse node (KI,KJ).
__device__ __forceinline__ double pweight2(const double* __restrict__ P, int ldc, long long plc, int nf,
                                           int fi, int fj, int KI, int KJ) {
    if (fi < 1 || fj < 1 || fi > nf - 2 || fj > nf - 2) return 0.0;
    const int oi = fi & 1, oj = fj & 1, I = fi >> 1, J = fj >> 1;
    const int dI = KI - I, dJ = KJ - J;
    if (dI < 0 || dJ < 0 || dI > oi || dJ > oj) return 0.0;
    const long long o = (long long)J * ldc + I;
    if (!oi && !oj) return 1.0;
    if (oi && !oj) return P[(dI ? PXR : PXL) * plc + o];
    if (!oi && oj) return P[(dJ ? PYN : PYS) * plc + o];
    const int p = dJ ? (dI ? PNE : PNW) : (dI ? PSE : PSW);
    return P[p * plc + o];
}

// Galerkin coarse operator A_c = P^T A P, one thread per coarse node, five
// stored entries: A_c(K, K+d) = sum_i P(i,K) sum_{j in N(i)} A(i,j) P(j,K+d).
__global__ void k_rap2d(Sten2<double> F, int nf, const double* __restrict__ P, int nc, int ldc,
                        long long plc, double* __restrict__ Ac, KState* st) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I >= nc) return;
    const long long o = (long long)J * ldc + I;
    double out[NS2] = {0, 0, 0, 0, 0};
    if (I >= 1 && J >= 1 && I <= nc - 2 && J <= nc - 2) {
        const int tdx[NS2] = {0, -1, 0, -1, -1};
        const int tdy[NS2] = {0, 0, -1, -1, 1};
#pragma unroll 1
        for (int t = 0; t < NS2; t++) {
            const int LI = I + tdx[t], LJ = J + tdy[t];
            if (LI < 1 || LJ < 1 || LI > nc - 2 || LJ > nc - 2) continue;
            double acc = 0.0;
            for (int fj = 2 * J - 1; fj <= 2 * J + 1; fj++)
                for (int fi = 2 * I - 1; fi <= 2 * I + 1; fi++) {
                    const double wK = pweight2(P, ldc, plc, nf, fi, fj, I, J);
                    if (wK == 0.0) continue;
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            const double a = F.full(fi, fj, dx, dy);
                            if (a == 0.0) continue;
                            const double wL = pweight2(P, ldc, plc, nf, fi + dx, fj + dy, LI, LJ);
                            acc += wK * a * wL;
                        }
                }
            out[t] = acc;
        }
        if (!(out[0] > 0.0)) set_err(st, BMG_ERR_SETUP_BREAKDOWN);
    }
#pragma unroll
    for (int t = 0; t < NS2; t++) Ac[t * plc + o] = out[t];
}

__global__ void k_export_stencil2d(Sten2<double> F, int n, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    double* row = out + ((long long)j * n + i) * 9;
    const bool in = i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2;
    for (int o = 0; o < 9; o++) row[o] = in ? F.full(i, j, o % 3 - 1, o / 3 - 1) : 0.0;
}

__global__ void k_export_interp2d(const double* __restrict__ P, int nf, int ldc, long long plc,
                                  double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= nf) return;
    double* row = out + ((long long)j * nf + i) * 4;
    for (int s = 0; s < 4; s++)
        row[s] = pweight2(P, ldc, plc, nf, i, j, (i >> 1) + (s & 1), (j >> 1) + (s >> 1));
}

// out_i = -sum over boundary nodes j of A_ij g_j at interior nodes i (the
// couplings the assembly drops, applied to Dirichlet data g; Sec. 2, the
// lift term of Eq. weak_computational); g and out in the caller's n^2
// layout, out zero on the boundary.
__global__ void k_boundary_rhs2d(int n, const double* __restrict__ coords, const double* __restrict__ kappa,
                                 const double* __restrict__ g, double* __restrict__ out, KState* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    double acc = 0.0;
    if (i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2) {
        const double* X = coords;
        const double* Y = coords + (long long)n * n;
        bool ok = true;
        for (int cy = 0; cy < 2; cy++)
            for (int cx = 0; cx < 2; cx++) {
                const int ci = i - 1 + cx, cj = j - 1 + cy;
                const int a = (1 - cx) + 2 * (1 - cy);      // the node's corner in the cell
                double K[4][4];
                ok &= element2d(X, Y, n, ci, cj, Scalar2{kappa[(long long)cj * (n - 1) + ci]}, K);
                for (int b = 0; b < 4; b++) {
                    const int bi = ci + (b & 1), bj = cj + (b >> 1);
                    if (bi >= 1 && bj >= 1 && bi <= n - 2 && bj <= n - 2) continue;
                    acc -= K[a][b] * g[(long long)bj * n + bi];
                }
            }
        if (!ok) set_err(st, BMG_ERR_MAP_FOLDED);
    }
    out[(long long)j * n + i] = acc;
}

// dL/dkappa_e = -lambda_e^T K_e^0 u_e (u, lambda in the caller's n^2 layout).
__global__ void k_adjoint_cells2d(int n, const double* __restrict__ coords, const double* __restrict__ u,
                                  const double* __restrict__ lam, double* __restrict__ g, KState* st) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    const int cj = blockIdx.y;
    if (ci >= n - 1) return;
    double K[4][4];
    if (!element2d(coords, coords + (long long)n * n, n, ci, cj, Scalar2{1.0}, K)) set_err(st, BMG_ERR_MAP_FOLDED);
    double ue[4], le[4];
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = ci + (a & 1), j = cj + (a >> 1);
        const bool in = i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2;
        const long long id = (long long)j * n + i;
        ue[a] = in ? u[id] : 0.0;
        le[a] = in ? lam[id] : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        double t = 0.0;
#pragma unroll
        for (int b = 0; b < 4; b++) t += K[a][b] * ue[b];
        s += le[a] * t;
    }
    g[(long long)cj * (n - 1) + ci] = -s;
}

inline dim3 grid_rows(int ni, int nj) { return dim3(cdiv(ni, 128), nj); }

}  // namespace

bmg_status assemble2d(Ctx& c, const double* coords, const double* kappa) {
    Level& L = c.lev[0];
    k_assemble2d<false><<<grid_asm(L.n), kAsmCells, 0, c.stream>>>(L.n, L.ld, L.plane, coords, kappa, L.A64, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// The two kernels of bmg_assemble and bmg_get_stencil(0) on caller-given
// storage: half planes A (row length ld, plane stride pl) and error word st.
bmg_status assemble_export2d(int n, int ld, long long pl, const double* coords, const double* kappa, double* A,
                             KState* st, double* out, cudaStream_t s) {
    k_assemble2d<false><<<grid_asm(n), kAsmCells, 0, s>>>(n, ld, pl, coords, kappa, A, st);
    BMG_CUDA(cudaGetLastError());
    k_export_stencil2d<<<grid_rows(n, n), 128, 0, s>>>(Sten2<double>{A, ld, pl}, n, out);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status assemble_tensor2d(Ctx& c, const double* coords, const double* D) {
    Level& L = c.lev[0];
    k_assemble2d<true><<<grid_asm(L.n), kAsmCells, 0, c.stream>>>(L.n, L.ld, L.plane, coords, D, L.A64, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status boundary_rhs2d(Ctx& c, const double* coords, const double* kappa, const double* g, double* out) {
    const int n = c.lev[0].n;
    k_boundary_rhs2d<<<grid_rows(n, n), 128, 0, c.stream>>>(n, coords, kappa, g, out, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status set_stencil2d(Ctx& c, const double* full) {
    Level& L = c.lev[0];
    k_set_stencil2d<<<grid_rows(L.n, L.n), 128, 0, c.stream>>>(L.n, L.ld, L.plane, full, L.A64);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status setup_level2d(Ctx& c, int l) {
    Level& F = c.lev[l];
    Level& K = c.lev[l + 1];
    Sten2<double> fs{F.A64, F.ld, F.plane};
    k_interp_edges2d<<<grid_rows(K.n, K.n), 128, 0, c.stream>>>(fs, F.n, K.n, K.ld, K.plane, F.P64, c.st);
    k_interp_interior2d<<<grid_rows(K.n, K.n), 128, 0, c.stream>>>(fs, F.n, K.n, K.ld, K.plane, F.P64, c.st);
    k_rap2d<<<grid_rows(K.n, K.n), 128, 0, c.stream>>>(fs, F.n, F.P64, K.n, K.ld, K.plane, K.A64, c.st);
    c.launches += 3;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status export_stencil2d(Ctx& c, int l, double* out) {
    Level& L = c.lev[l];
    k_export_stencil2d<<<grid_rows(L.n, L.n), 128, 0, c.stream>>>(Sten2<double>{L.A64, L.ld, L.plane}, L.n, out);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status export_interp2d(Ctx& c, int l, double* out) {
    Level& F = c.lev[l];
    Level& K = c.lev[l + 1];
    k_export_interp2d<<<grid_rows(F.n, F.n), 128, 0, c.stream>>>(F.P64, F.n, K.ld, K.plane, out);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status adjoint_cells2d(Ctx& c, const double* coords, const double* u, const double* lam, double* g) {
    const int n = c.lev[0].n;
    k_adjoint_cells2d<<<grid_rows(n - 1, n - 1), 128, 0, c.stream>>>(n, coords, u, lam, g, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
