// aux2d.cu -- the auxiliary-space two-grid method around the structured
// solve (Sec. 2.2 "Setup phase" and "Solution phase", Sec. 2.3, Sec. 2.4).
//
// The physical problem is the P1 system A_p u_p = f_p on a triangulation of
// the physical domain; the structured BoxMG hierarchy of a coarse context
// is its coarse level, reached through P = M_p^-1 C and R = P^T.
//
// Host side (bmg_aux_create): interior numbering of the vertices, the CSR
// patterns of A_p and M_p (rows and columns: interior vertices) with, for
// every stored entry, the list of the element contributions that sum to it
// (triangle order), the vertex-to-triangle incidence, and bounds (from the
// triangles' bounding boxes in computational space) that size the
// workspace of the coupled mass.
//
// Device side, setup: the rasterisation of the mapped triangles over the
// computational cells (Sec. 2.3.1's cell-wise evaluation): one thread per
// triangle counts the cells of its bounding box that no edge separates from
// it, a prefix sum numbers the (triangle, cell) pairs in triangle order and
// a second pass writes them; one thread per interior vertex then lists the
// contributions (pair, local vertex, cell corner) of its row of C in that
// order, sorts them by column (stably) and writes C's CSR pattern and the
// contribution list of every entry; C^T and the sliced-ELLPACK copies of C
// and C^T follow by counting and prefix sums.  Then per-triangle P1 element
// matrices and per-pair coupled-mass blocks are formed once (FP64) and every
// stored entry sums its contributions in list order -- deterministic, no
// atomics in any value.  A solve runs the cycle with CSR kernels (one thread
// per row), device-side CG scalars for the mass solves, and the coarse
// context's own V-cycle.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <new>
#include <vector>

#include "common.cuh"

using namespace bmg;

namespace {

constexpr int kAuxThreads = kThreads;     // 256, as block_sum expects
constexpr int kRedBlocks = 4 * 152;       // fixed grid of the reducing kernels

struct AuxState {
    double rr;          // ||f - A u||^2 (interior)
    double ff;          // ||f||^2
    double pq, rz, rzo; // the outer flexible CG's scalars
    double alpha_o, beta_o;
    double cg_rr, cg_pq, alpha, beta;
    int err;
    unsigned int counter[4];
};

__device__ __forceinline__ void aux_err(AuxState* st, int code) { atomicCAS(&st->err, 0, code); }

// ------------------------------------------------------------------ setup kernels
// P1 stiffness and consistent mass of every triangle (Sec. 2.1, V_p = P1):
// K_ab = kappa |T| grad l_a . grad l_b, M_ab = |T| (1 + delta_ab) / 12, the
// barycentric gradients from the edge opposite each vertex.
__global__ void k_tri_local(int ntri, const int* __restrict__ tri, const double* __restrict__ xy,
                            const double* __restrict__ kappa, double* __restrict__ lk, double* __restrict__ lm,
                            AuxState* st) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntri) return;
    double px[3], py[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int v = tri[3 * t + a];
        px[a] = xy[2 * v];
        py[a] = xy[2 * v + 1];
    }
    // edge opposite vertex a: from vertex a+1 to vertex a+2
    double ex[3], ey[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        ex[a] = px[(a + 2) % 3] - px[(a + 1) % 3];
        ey[a] = py[(a + 2) % 3] - py[(a + 1) % 3];
    }
    const double area = 0.5 * ((px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]));
    if (!(area > 0.0)) aux_err(st, BMG_ERR_MAP_FOLDED);
    const double s = kappa[t] / (4.0 * area);    // kappa |T| / (2|T|)^2
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            lk[9 * t + 3 * a + b] = s * (ex[a] * ex[b] + ey[a] * ey[b]);
            lm[9 * t + 3 * a + b] = area / 12.0 * (a == b ? 2.0 : 1.0);
        }
}

// The 3 x 4 coupled-mass block of one (triangle, cell) pair (Sec. 2.3, Eq.
// coupled_mass_comp): the mapped triangle (straight edges through the
// images of its vertices) is clipped to the cell (Sutherland-Hodgman, one
// half-plane at a time), the clipped polygon is split into a fan, and each
// fan triangle is integrated with a 3 x 3 Gauss rule in collapsed
// coordinates -- exact for the integrand, barycentric coordinate (degree 1)
// x bilinear basis (2) x |det J| of the Q1 cell (affine).
__device__ __forceinline__ int clip_half(const double* ix, const double* iy, int m, double* ox, double* oy, int ax,
                                         double bound, bool lower) {
    int k = 0;
    for (int e = 0; e < m; e++) {
        const int pe = e == 0 ? m - 1 : e - 1;
        const double ac = ax == 0 ? ix[pe] : iy[pe], bc = ax == 0 ? ix[e] : iy[e];
        const bool ka = lower ? ac >= bound : ac <= bound;
        const bool kb = lower ? bc >= bound : bc <= bound;
        if (ka != kb) {
            const double s = (bound - ac) / (bc - ac);
            double x = ix[pe] + s * (ix[e] - ix[pe]);
            double y = iy[pe] + s * (iy[e] - iy[pe]);
            if (ax == 0) x = bound; else y = bound;
            ox[k] = x;
            oy[k] = y;
            k++;
        }
        if (kb) {
            ox[k] = ix[e];
            oy[k] = iy[e];
            k++;
        }
    }
    return k;
}

__global__ void k_pair_local(int npairs, const int* __restrict__ pair_tri, const int* __restrict__ pair_cell,
                             const int* __restrict__ tri, const double* __restrict__ st,
                             const double* __restrict__ coords, int n, double* __restrict__ loc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npairs) return;
    const int t = pair_tri[p];
    const int cell = pair_cell[p];
    const int ci = cell % (n - 1), cj = cell / (n - 1);
    const double h = 1.0 / (n - 1);
    double Sx[3], Sy[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int v = tri[3 * t + a];
        Sx[a] = st[2 * v];
        Sy[a] = st[2 * v + 1];
    }
    const double d = (Sx[1] - Sx[0]) * (Sy[2] - Sy[0]) - (Sy[1] - Sy[0]) * (Sx[2] - Sx[0]);
    // corners of the cell in physical space (order 00, 10, 01, 11)
    const double* X = coords;
    const double* Y = coords + (long long)n * n;
    const long long o00 = (long long)cj * n + ci;
    const double Xc[4] = {X[o00], X[o00 + 1], X[o00 + n], X[o00 + n + 1]};
    const double Yc[4] = {Y[o00], Y[o00 + 1], Y[o00 + n], Y[o00 + n + 1]};
    double ax_[8], ay_[8], bx_[8], by_[8];
    int m = 3;
    for (int a = 0; a < 3; a++) {
        ax_[a] = Sx[a];
        ay_[a] = Sy[a];
    }
    m = clip_half(ax_, ay_, m, bx_, by_, 0, ci * h, true);
    m = clip_half(bx_, by_, m, ax_, ay_, 0, (ci + 1) * h, false);
    m = clip_half(ax_, ay_, m, bx_, by_, 1, cj * h, true);
    m = clip_half(bx_, by_, m, ax_, ay_, 1, (cj + 1) * h, false);
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = 0.0;
    // 3-point Gauss-Legendre on [0, 1]
    const double g[3] = {0.5 - 0.38729833462074168852, 0.5, 0.5 + 0.38729833462074168852};
    const double w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    const double inv_h2 = 1.0 / (h * h);
    for (int k = 1; k + 1 < m; k++) {
        const double v0x = ax_[0], v0y = ay_[0];
        const double v1x = ax_[k], v1y = ay_[k];
        const double v2x = ax_[k + 1], v2y = ay_[k + 1];
        const double area2 = fabs((v1x - v0x) * (v2y - v0y) - (v1y - v0y) * (v2x - v0x));
        for (int qa = 0; qa < 3; qa++)
            for (int qb = 0; qb < 3; qb++) {
                const double u = g[qa], v = g[qb];
                const double ps = v0x + u * ((v1x - v0x) + v * (v2x - v1x));
                const double pt = v0y + u * ((v1y - v0y) + v * (v2y - v1y));
                const double wt = w[qa] * w[qb] * u * area2 * inv_h2;
                const double l1 = ((ps - Sx[0]) * (Sy[2] - Sy[0]) - (pt - Sy[0]) * (Sx[2] - Sx[0])) / d;
                const double l2 = ((Sx[1] - Sx[0]) * (pt - Sy[0]) - (Sy[1] - Sy[0]) * (ps - Sx[0])) / d;
                const double lam[3] = {1.0 - l1 - l2, l1, l2};
                const double xi = ps * (n - 1) - ci, eta = pt * (n - 1) - cj;
                const double phi[4] = {(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta};
                const double dxi[4] = {-(1 - eta), 1 - eta, -eta, eta};
                const double deta[4] = {-(1 - xi), -xi, 1 - xi, xi};
                double J11 = 0, J12 = 0, J21 = 0, J22 = 0;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    J11 += dxi[c] * Xc[c];
                    J12 += deta[c] * Xc[c];
                    J21 += dxi[c] * Yc[c];
                    J22 += deta[c] * Yc[c];
                }
                const double dj = fabs(J11 * J22 - J12 * J21);
                const double f = wt * dj;
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++) acc[4 * a + b] += f * lam[a] * phi[b];
            }
    }
#pragma unroll
    for (int k = 0; k < 12; k++) loc[12LL * p + k] = acc[k];
}

// out[e] = sum of src[idx[k]] for k in [ptr[e], ptr[e+1]), in list order
__global__ void k_gather(int nout, const int* __restrict__ ptr, const int* __restrict__ idx,
                         const double* __restrict__ src, double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nout) return;
    double s = 0.0;
    for (int k = ptr[e]; k < ptr[e + 1]; k++) s += src[idx[k]];
    out[e] = s;
}

__global__ void k_diag_inv(int nr, const int* __restrict__ diag_pos, const double* __restrict__ va,
                           double* __restrict__ dinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) dinv[i] = 1.0 / va[diag_pos[i]];
}

__global__ void k_inv(int nr, double* __restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) v[i] = 1.0 / v[i];
}

// ------------------------------------------------------------------ solve kernels
// Row i of a matrix in sliced ELLPACK with slices of 32 rows: slice s
// holds its rows' entries column-major from so[s] (entry k of row 32 s + l
// at so[s] + 32 k + l), padded with zeros to the slice's longest row, so
// the 32 threads of a warp read consecutive words.  Entries keep their CSR
// order, so the sum is the CSR row's, plus zero terms.
__device__ __forceinline__ double csr_row(const int* __restrict__ so, const int* __restrict__ ci,
                                          const double* __restrict__ va, const double* __restrict__ x, int i) {
    const int sl = i >> 5;
    const int b = so[sl] + (i & 31), e = so[sl + 1];
    double s = 0.0;
    for (int k = b; k < e; k += 32) s += va[k] * x[ci[k]];
    return s;
}

// SELL values from CSR values: out[k] = src[map[k]], 0 for padding (map < 0)
__global__ void k_sell_fill(int n, const int* __restrict__ map, const double* __restrict__ src,
                            double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = map[k] >= 0 ? src[map[k]] : 0.0;
}

// interior entries of a vertex vector: out[i] = in[vtx[i]]
__global__ void k_compress(int nr, const int* __restrict__ vtx, const double* __restrict__ in, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) out[i] = in[vtx[i]];
}

// all vertices: out[v] = in[vid[v]] or 0 on Dirichlet vertices
__global__ void k_expand(int nv, const int* __restrict__ vid, const double* __restrict__ in, double* __restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) out[v] = vid[v] >= 0 ? in[vid[v]] : 0.0;
}

// damped Jacobi: uo = u + omega D^-1 (f - A u)
__global__ void k_jacobi(int nr, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ va,
                         const double* __restrict__ dinv, const double* __restrict__ f, const double* __restrict__ u,
                         double* __restrict__ uo, double omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) uo[i] = u[i] + omega * dinv[i] * (f[i] - csr_row(rp, ci, va, u, i));
}

// r = f - A u; with slot: *slot = ||r||^2 (deterministic grid reduction)
__global__ void k_residual_csr(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ va, const double* __restrict__ f,
                               const double* __restrict__ u, double* __restrict__ r, double* partials,
                               unsigned int* counter, double* slot) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const double v = f[i] - csr_row(rp, ci, va, u, i);
        if (r) r[i] = v;
        acc += v * v;
    }
    double t;
    if (slot && grid_sum(acc, partials, counter, &t)) *slot = t;
}

__global__ void k_dot_aux(int nr, const double* __restrict__ a, const double* __restrict__ b, double* partials,
                          unsigned int* counter, double* slot) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) acc += a[i] * b[i];
    double t;
    if (grid_sum(acc, partials, counter, &t)) *slot = t;
}

// restriction: rc[map[q]] = sum_k C^T[q,k] (y[col] * (w ? w[col] : 1)), C^T in SELL-32
__global__ void k_restrict_ct(int nq, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ va, const int* __restrict__ map, const double* __restrict__ y,
                              const double* __restrict__ w, double* __restrict__ rc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int sl = q >> 5;
    const int b = rp[sl] + (q & 31), e = rp[sl + 1];
    double s = 0.0;
    for (int k = b; k < e; k += 32) s += va[k] * (w ? y[ci[k]] * w[ci[k]] : y[ci[k]]);
    rc[map[q]] = s;
}

// prolongation: out[i] = (C z)_i * (w ? w[i] : 1), z in the padded coarse layout;
// with u: u[i] += gamma * out[i] instead
__global__ void k_prolong_c(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ va, const double* __restrict__ z, const double* __restrict__ w,
                            double* __restrict__ out, double* __restrict__ u, double gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    double s = csr_row(rp, ci, va, z, i);
    if (w) s *= w[i];
    if (u) u[i] += gamma * s;
    else out[i] = s;
}

// CG on M (the mass solves): x = 0, res = r, p = r, cg_rr = r.r
__global__ void k_cg_init(int nr, const double* __restrict__ r, double* __restrict__ x, double* __restrict__ res,
                          double* __restrict__ p, double* partials, AuxState* st) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const double v = r[i];
        x[i] = 0.0;
        res[i] = v;
        p[i] = v;
        acc += v * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[1], &t)) st->cg_rr = t;
}

// q = M p; alpha = cg_rr / p.q (0 when p.q is not positive: r was zero)
__global__ void k_cg_mp(int nr, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ va,
                        const double* __restrict__ p, double* __restrict__ q, double* partials, AuxState* st) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const double v = csr_row(rp, ci, va, p, i);
        q[i] = v;
        acc += p[i] * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[1], &t)) {
        st->cg_pq = t;
        st->alpha = t > 0.0 ? st->cg_rr / t : 0.0;
    }
}

// x += alpha p; res -= alpha q; beta = res.res / cg_rr; cg_rr = res.res
__global__ void k_cg_update(int nr, double* __restrict__ x, double* __restrict__ res, const double* __restrict__ p,
                            const double* __restrict__ q, double* partials, AuxState* st) {
    const double alpha = st->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double v = res[i] - alpha * q[i];
        res[i] = v;
        acc += v * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[1], &t)) {
        st->beta = st->cg_rr > 0.0 ? t / st->cg_rr : 0.0;
        st->cg_rr = t;
    }
}

__global__ void k_cg_p(int nr, const double* __restrict__ res, double* __restrict__ p, const AuxState* st) {
    const double beta = st->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x)
        p[i] = res[i] + beta * p[i];
}

// q = A p; alpha = rz / p.q (device-side, with a breakdown check)
__global__ void k_spmv_dot(int nr, const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ va,
                           const double* __restrict__ p, double* __restrict__ q, double* partials, AuxState* st) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        const double v = csr_row(rp, ci, va, p, i);
        q[i] = v;
        acc += p[i] * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[2], &t)) {
        st->pq = t;
        const bool ok = t > 0.0 && st->rz > 0.0;
        st->alpha_o = ok ? st->rz / t : 0.0;
        if (!ok) aux_err(st, BMG_ERR_NOT_SPD);
    }
}

// u += alpha p; r -= alpha q; ||r||^2 (alpha from the device state)
__global__ void k_update_ur(int nr, double* __restrict__ u, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, const AuxState* stc, double* partials, unsigned int* counter,
                            double* slot) {
    const double alpha = stc->alpha_o;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        u[i] += alpha * p[i];
        const double v = r[i] - alpha * q[i];
        r[i] = v;
        acc += v * v;
    }
    double t;
    if (grid_sum(acc, partials, counter, &t)) *slot = t;
}

// r.z and r.zo; beta = (r.z - r.zo) / rz_old and rz = r.z on the device
// (first: only rz)
__global__ void k_dot2_aux(int nr, const double* __restrict__ r, const double* __restrict__ z,
                           const double* __restrict__ zo, double* partials, AuxState* st, int first) {
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
        a += r[i] * z[i];
        b += r[i] * zo[i];
    }
    double t1, t2;
    if (grid_sum2(a, b, partials, &st->counter[3], &t1, &t2)) {
        st->rzo = t2;
        st->beta_o = first ? 0.0 : (st->rz > 0.0 ? (t1 - t2) / st->rz : 0.0);
        st->rz = t1;
    }
}

__global__ void k_p_update_aux(int nr, double* __restrict__ p, const double* __restrict__ z, const AuxState* st) {
    const double beta = st->beta_o;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) p[i] = z[i] + beta * p[i];
}

// ---- FP32 cycle (the flexible-CG preconditioner on an FP32 coarse context)
// A_p products in difference form, rs_i u_i + sum_j a_ij (u_j - u_i) with
// the row sums rs_i formed in FP64: a smooth u makes the plain FP32 product
// lose A u to cancellation (the diagonal entry contributes a_ii * 0).
__device__ __forceinline__ float sell_diff32(const int* __restrict__ so, const int* __restrict__ ci,
                                            const float* __restrict__ va, const float* __restrict__ rs,
                                            const float* __restrict__ x, int i) {
    const int sl = i >> 5;
    const int b = so[sl] + (i & 31), e = so[sl + 1];
    const float xi = x[i];
    float s = rs[i] * xi;
    for (int k = b; k < e; k += 32) s += va[k] * (x[ci[k]] - xi);
    return s;
}

__global__ void k_to64(int nr, const float* __restrict__ in, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) out[i] = (double)in[i];
}

// uo = u + omega D^-1 (f - A u); with u == nullptr, u = 0 (the first sweep)
__global__ void k_jacobi32(int nr, const int* __restrict__ so, const int* __restrict__ ci, const float* __restrict__ va,
                           const float* __restrict__ rs, const float* __restrict__ dinv, const float* __restrict__ f,
                           const float* __restrict__ u, float* __restrict__ uo, float omega) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    if (!u) {
        uo[i] = omega * dinv[i] * f[i];
        return;
    }
    uo[i] = u[i] + omega * dinv[i] * (f[i] - sell_diff32(so, ci, va, rs, u, i));
}

// r = f - A u (FP32, difference form)
__global__ void k_residual32(int nr, const int* __restrict__ so, const int* __restrict__ ci,
                             const float* __restrict__ va, const float* __restrict__ rs, const float* __restrict__ f,
                             const float* __restrict__ u, float* __restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) r[i] = f[i] - sell_diff32(so, ci, va, rs, u, i);
}

// rc[map[q]] = sum_k C^T[q,k] y[col] w[col] (FP32 products, FP64 out for the coarse solve)
__global__ void k_restrict_ct32(int nq, const int* __restrict__ so, const int* __restrict__ ci,
                                const float* __restrict__ va, const int* __restrict__ map, const float* __restrict__ y,
                                const float* __restrict__ w, double* __restrict__ rc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int sl = q >> 5;
    const int b = so[sl] + (q & 31), e = so[sl + 1];
    float s = 0.0f;
    for (int k = b; k < e; k += 32) s += va[k] * (y[ci[k]] * w[ci[k]]);
    rc[map[q]] = (double)s;
}

// u += gamma w (C z), z the coarse correction (FP64, padded layout)
__global__ void k_prolong_c32(int nr, const int* __restrict__ so, const int* __restrict__ ci,
                              const float* __restrict__ va, const double* __restrict__ z, const float* __restrict__ w,
                              float* __restrict__ u, float gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const int sl = i >> 5;
    const int b = so[sl] + (i & 31), e = so[sl + 1];
    float s = 0.0f;
    for (int k = b; k < e; k += 32) s += va[k] * (float)z[ci[k]];
    u[i] += gamma * (s * w[i]);
}

__global__ void k_row_sums_sell(int nr, const int* __restrict__ so, const double* __restrict__ va,
                                float* __restrict__ rs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const int sl = i >> 5;
    double s = 0.0;
    for (int k = so[sl] + (i & 31); k < so[sl + 1]; k += 32) s += va[k];
    rs[i] = (float)s;
}

__global__ void k_d2f(int n, const double* __restrict__ in, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

__global__ void k_axpy(int nr, double* __restrict__ u, const double* __restrict__ v, double gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) u[i] += gamma * v[i];
}

__global__ void k_spmv_csr(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ va, const double* __restrict__ x, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) y[i] = csr_row(rp, ci, va, x, i);
}

// natural n x n grid vector <-> the coarse context's padded layout (interior only)
__global__ void k_to_padded(int n, int ld, const double* __restrict__ src, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= ld) return;
    const bool in = i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2;
    dst[(long long)j * ld + i] = in ? src[(long long)j * n + i] : 0.0;
}

__global__ void k_from_padded(int n, int ld, const double* __restrict__ src, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= n) return;
    const bool in = i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2;
    dst[(long long)j * n + i] = in ? src[(long long)j * ld + i] : 0.0;
}

// Lanczos step: w -= alpha q + beta q_prev; v -= alpha b + beta b_prev
__global__ void k_lanczos_orth(int nr, double* __restrict__ w, const double* __restrict__ q,
                               const double* __restrict__ qp, double* __restrict__ v, const double* __restrict__ b,
                               const double* __restrict__ bp, double alpha, double beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    w[i] -= alpha * q[i] + beta * qp[i];
    v[i] -= alpha * b[i] + beta * bp[i];
}

// q_prev = q, q = w / beta; b_prev = b, b = v / beta
__global__ void k_lanczos_shift(int nr, double* __restrict__ q, double* __restrict__ qp, const double* __restrict__ w,
                                double* __restrict__ b, double* __restrict__ bp, const double* __restrict__ v,
                                double inv_beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    qp[i] = q[i];
    q[i] = w[i] * inv_beta;
    bp[i] = b[i];
    b[i] = v[i] * inv_beta;
}

inline int blocks(long long n) { return cdiv(n, kAuxThreads); }

// ------------------------------------------------------------------ rasterisation (device setup)
// Cell range of the bounding box of triangle t's image (s, t coordinates in
// [0,1]^2), clamped to the n-1 cells per side; the same arithmetic as the
// host bound.
__host__ __device__ inline int cell_of(double v, double h, int n) {
    long long k = (long long)floor(v / h);
    if (k < 0) k = 0;
    if (k > n - 2) k = n - 2;
    return (int)k;
}

// Separating-axis test of a triangle against an axis-aligned box (touching
// counts).  Products and sums rounded one by one (no fused multiply-add),
// as on the host.
__device__ bool tri_box_overlap_d(const double* sx, const double* sy, double x0, double y0, double x1, double y1) {
    const double mnx = fmin(sx[0], fmin(sx[1], sx[2])), mxx = fmax(sx[0], fmax(sx[1], sx[2]));
    const double mny = fmin(sy[0], fmin(sy[1], sy[2])), mxy = fmax(sy[0], fmax(sy[1], sy[2]));
    if (mxx < x0 || mnx > x1 || mxy < y0 || mny > y1) return false;
    for (int e = 0; e < 3; e++) {
        const int a = e, b = (e + 1) % 3, c = (e + 2) % 3;
        const double nx = __dsub_rn(sy[b], sy[a]), ny = __dsub_rn(sx[a], sx[b]);
        const double side = __dadd_rn(__dmul_rn(nx, __dsub_rn(sx[c], sx[a])), __dmul_rn(ny, __dsub_rn(sy[c], sy[a])));
        const double cx[4] = {x0, x1, x0, x1}, cy[4] = {y0, y0, y1, y1};
        bool all_out = true;
        for (int k = 0; k < 4 && all_out; k++) {
            const double v =
                __dadd_rn(__dmul_rn(nx, __dsub_rn(cx[k], sx[a])), __dmul_rn(ny, __dsub_rn(cy[k], sy[a])));
            if (side > 0 ? v >= 0 : v <= 0) all_out = false;
        }
        if (all_out) return false;
    }
    return true;
}

// Pairs of triangle t: the cells (ci, cj) of its bounding box, cj then ci
// ascending, that the separating-axis test keeps.  count only, or write
// them from pair index p0.
__device__ int tri_pairs(int t, const int* __restrict__ tri, const double* __restrict__ st, int n, int* pair_tri,
                         int* pair_cell, int p0) {
    const double h = 1.0 / (n - 1);
    double sx[3], sy[3];
    for (int a = 0; a < 3; a++) {
        sx[a] = st[2 * tri[3 * t + a]];
        sy[a] = st[2 * tri[3 * t + a] + 1];
    }
    const int i0 = cell_of(fmin(sx[0], fmin(sx[1], sx[2])), h, n), i1 = cell_of(fmax(sx[0], fmax(sx[1], sx[2])), h, n);
    const int j0 = cell_of(fmin(sy[0], fmin(sy[1], sy[2])), h, n), j1 = cell_of(fmax(sy[0], fmax(sy[1], sy[2])), h, n);
    int k = 0;
    for (int cj = j0; cj <= j1; cj++)
        for (int ci = i0; ci <= i1; ci++) {
            if (!tri_box_overlap_d(sx, sy, ci * h, cj * h, (ci + 1) * h, (cj + 1) * h)) continue;
            if (pair_tri) {
                pair_tri[p0 + k] = t;
                pair_cell[p0 + k] = cj * (n - 1) + ci;
            }
            k++;
        }
    return k;
}

__global__ void k_pair_count(int ntri, const int* __restrict__ tri, const double* __restrict__ st, int n,
                             int* __restrict__ cnt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntri) cnt[t] = tri_pairs(t, tri, st, n, nullptr, nullptr, 0);
}

__global__ void k_pair_fill(int ntri, const int* __restrict__ tri, const double* __restrict__ st, int n,
                            const int* __restrict__ poff, int* __restrict__ pair_tri, int* __restrict__ pair_cell) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntri) tri_pairs(t, tri, st, n, pair_tri, pair_cell, poff[t]);
}

// Row i of C: the contributions (12 p + 4 a + b: pair p, local vertex a of
// its triangle, cell corner b) of the pairs of the triangles incident to
// vertex i (triangle order, then pair order, then corner), to the interior
// coarse nodes (column j*ld + i), sorted stably by column in the row's
// scratch; counts the distinct columns.
__global__ void k_crow_records(int nvi, const int* __restrict__ vt_ptr, const int* __restrict__ vt_tri,
                               const int* __restrict__ vt_a, const int* __restrict__ poff,
                               const int* __restrict__ pair_cell, int n, int ld, const long long* __restrict__ rec_off,
                               int* __restrict__ rec_col, int* __restrict__ rec_src, int* __restrict__ rec_cnt,
                               int* __restrict__ uniq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvi) return;
    int* col = rec_col + rec_off[i];
    int* src = rec_src + rec_off[i];
    int m = 0;
    for (int e = vt_ptr[i]; e < vt_ptr[i + 1]; e++) {
        const int t = vt_tri[e], a = vt_a[e];
        for (int p = poff[t]; p < poff[t + 1]; p++) {
            const int cell = pair_cell[p];
            const int ci = cell % (n - 1), cj = cell / (n - 1);
            for (int b = 0; b < 4; b++) {
                const int ii = ci + (b & 1), jj = cj + (b >> 1);
                if (ii < 1 || jj < 1 || ii > n - 2 || jj > n - 2) continue;
                // stable insertion by column
                const int c = jj * ld + ii, v = 12 * p + 4 * a + b;
                int q = m;
                while (q > 0 && col[q - 1] > c) {
                    col[q] = col[q - 1];
                    src[q] = src[q - 1];
                    q--;
                }
                col[q] = c;
                src[q] = v;
                m++;
            }
        }
    }
    int u = 0;
    for (int q = 0; q < m; q++)
        if (q == 0 || col[q] != col[q - 1]) u++;
    rec_cnt[i] = m;
    uniq[i] = u;
}

// C's CSR pattern (columns, row of every entry) and the contribution lists:
// entry e of row i sums gidx[gptr[e] .. gptr[e+1]).
__global__ void k_crow_write(int nvi, const long long* __restrict__ rec_off, const int* __restrict__ rec_col,
                             const int* __restrict__ rec_src, const int* __restrict__ rec_cnt,
                             const int* __restrict__ c_ptr, const int* __restrict__ g_off, int* __restrict__ c_col,
                             int* __restrict__ c_row, int* __restrict__ c_gptr, int* __restrict__ c_gidx) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvi) return;
    const int* col = rec_col + rec_off[i];
    const int* src = rec_src + rec_off[i];
    const int m = rec_cnt[i];
    int e = c_ptr[i] - 1;
    const int g = g_off[i];
    for (int q = 0; q < m; q++) {
        if (q == 0 || col[q] != col[q - 1]) {
            e++;
            c_col[e] = col[q];
            c_row[e] = i;
            c_gptr[e] = g + q;
        }
        c_gidx[g + q] = src[q];
    }
}

// C^T: rows are the interior coarse nodes q = (j-1)(n-2) + (i-1); its
// entries are C's, in C order within a row (counted, placed, then each row
// sorted by C index, so the placement order does not matter).
__device__ __forceinline__ int q_of_col(int col, int ld, int n) { return (col / ld - 1) * (n - 2) + (col % ld - 1); }

__global__ void k_ct_count(int nnz, const int* __restrict__ c_col, int ld, int n, int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nnz) atomicAdd(&cnt[q_of_col(c_col[k], ld, n)], 1);
}

__global__ void k_ct_fill(int nnz, const int* __restrict__ c_col, const int* __restrict__ c_row, int ld, int n,
                          const int* __restrict__ ct_ptr, int* __restrict__ fill, int* __restrict__ ct_col,
                          int* __restrict__ ct_perm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    const int q = q_of_col(c_col[k], ld, n);
    const int pos = ct_ptr[q] + atomicAdd(&fill[q], 1);
    ct_col[pos] = c_row[k];
    ct_perm[pos] = k;
}

__global__ void k_ct_sort(int nq, const int* __restrict__ ct_ptr, int* __restrict__ ct_col, int* __restrict__ ct_perm) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    for (int e = ct_ptr[q] + 1; e < ct_ptr[q + 1]; e++) {
        const int k = ct_perm[e], c = ct_col[e];
        int f = e;
        while (f > ct_ptr[q] && ct_perm[f - 1] > k) {
            ct_perm[f] = ct_perm[f - 1];
            ct_col[f] = ct_col[f - 1];
            f--;
        }
        ct_perm[f] = k;
        ct_col[f] = c;
    }
}

// Sliced ELLPACK (32-row slices, entries column-major in a slice, rows
// padded with column 0 / map -1 to the slice's longest row): slot counts per
// slice, then the pattern; map[slot] = the CSR entry (through `through` if given).
__global__ void k_sell_width(int nr, const int* __restrict__ ptr, int* __restrict__ slots) {
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= (nr + 31) / 32) return;
    int w = 0;
    for (int i = sl * 32; i < min(nr, sl * 32 + 32); i++) w = max(w, ptr[i + 1] - ptr[i]);
    slots[sl] = 32 * w;
}

__global__ void k_sell_pattern(int nr, const int* __restrict__ ptr, const int* __restrict__ col,
                               const int* __restrict__ through, const int* __restrict__ off, int* __restrict__ scol,
                               int* __restrict__ smap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const int sl = i / 32, l = i % 32;
    for (int k = ptr[i]; k < ptr[i + 1]; k++) {
        const int slot = off[sl] + 32 * (k - ptr[i]) + l;
        scol[slot] = col[k];
        smap[slot] = through ? through[k] : k;
    }
}

// Exclusive prefix sum of n ints (out[n] = total), three passes over
// kScanB-element blocks; totals fit an int (the callers check the bounds).
constexpr int kScanB = 1024;

__global__ void k_scan_local(const int* __restrict__ in, int n, int* __restrict__ out, int* __restrict__ bsum) {
    __shared__ int sh[kScanB];
    const int base = blockIdx.x * kScanB;
    const int t = threadIdx.x;   // kScanB / 4 threads, four elements each
    int v[4], s = 0;
    for (int k = 0; k < 4; k++) {
        const int idx = base + 4 * t + k;
        v[k] = idx < n ? in[idx] : 0;
        s += v[k];
    }
    sh[t] = s;
    __syncthreads();
    for (int o = 1; o < kScanB / 4; o <<= 1) {   // inclusive scan of the per-thread sums (Hillis-Steele)
        const int add = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int run = sh[t] - s;
    for (int k = 0; k < 4; k++) {
        const int idx = base + 4 * t + k;
        if (idx < n) out[idx] = run;
        run += v[k];
    }
    if (t == kScanB / 4 - 1) bsum[blockIdx.x] = sh[t];
}

__global__ void k_scan_blocks(int* __restrict__ bsum, int nb, int* __restrict__ total) {
    if (threadIdx.x != 0) return;
    int run = 0;
    for (int b = 0; b < nb; b++) {
        const int v = bsum[b];
        bsum[b] = run;
        run += v;
    }
    *total = run;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ bsum) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += bsum[idx / kScanB];
}

// ------------------------------------------------------------------ host structure
struct Csr {
    std::vector<int> ptr, col;       // rows, columns
    std::vector<int> gptr, gidx;     // per entry: its contributions (indices into the local arrays)
};

// Builds a CSR from (row, col, contribution) records: entries sorted by
// column within a row, contributions of an entry in record order.
bool build_csr(int nrows, const std::vector<int>& rr, const std::vector<int>& cc, const std::vector<int>& src,
               Csr& out) {
    const size_t nrec = rr.size();
    std::vector<long long> cnt(nrows + 1, 0);
    for (size_t k = 0; k < nrec; k++) cnt[rr[k] + 1]++;
    for (int i = 0; i < nrows; i++) cnt[i + 1] += cnt[i];
    std::vector<int> order(nrec);
    {
        std::vector<long long> pos(cnt.begin(), cnt.end() - 1);
        for (size_t k = 0; k < nrec; k++) order[pos[rr[k]]++] = (int)k;
    }
    out.ptr.assign(nrows + 1, 0);
    out.col.clear();
    out.gptr.assign(1, 0);
    out.gidx.clear();
    out.gidx.reserve(nrec);
    std::vector<int> tmp;
    for (int i = 0; i < nrows; i++) {
        tmp.assign(order.begin() + cnt[i], order.begin() + cnt[i + 1]);
        std::stable_sort(tmp.begin(), tmp.end(), [&](int a, int b) { return cc[a] < cc[b]; });
        for (size_t k = 0; k < tmp.size(); k++) {
            if (k == 0 || cc[tmp[k]] != cc[tmp[k - 1]]) {
                out.col.push_back(cc[tmp[k]]);
                if (k > 0) out.gptr.push_back((int)out.gidx.size());
            }
            out.gidx.push_back(src[tmp[k]]);
        }
        if (!tmp.empty()) out.gptr.push_back((int)out.gidx.size());
        out.ptr[i + 1] = (int)out.col.size();
        if (out.gidx.size() > (size_t)0x7fffffff) return false;
    }
    return true;
}

struct Sell {
    std::vector<int> off, col, map;   // slice offsets, columns, CSR index of each slot (-1: padding)
};

// CSR (ptr, col) -> SELL-32; map[k] = CSR entry of slot k, composed with
// `through` if given.  False if the padded size exceeds 32-bit indices.
bool build_sell(const std::vector<int>& ptr, const std::vector<int>& col, const std::vector<int>* through,
                Sell& out) {
    const int nr = (int)ptr.size() - 1;
    const int ns = (nr + 31) / 32;
    out.off.assign(ns + 1, 0);
    long long total = 0;
    for (int sl = 0; sl < ns; sl++) {
        int w = 0;
        for (int i = sl * 32; i < std::min(nr, sl * 32 + 32); i++) w = std::max(w, ptr[i + 1] - ptr[i]);
        total += 32LL * w;
        if (total > 0x7fffffffLL) return false;
        out.off[sl + 1] = (int)total;
    }
    out.col.assign(out.off[ns], 0);
    out.map.assign(out.off[ns], -1);
    for (int i = 0; i < nr; i++) {
        const int sl = i / 32, l = i % 32;
        for (int k = ptr[i]; k < ptr[i + 1]; k++) {
            const int slot = out.off[sl] + 32 * (k - ptr[i]) + l;
            out.col[slot] = col[k];
            out.map[slot] = through ? (*through)[k] : k;
        }
    }
    return true;
}

}  // namespace

struct bmg_aux {
    bmg_ctx* coarse = nullptr;
    bmg_aux_opts opts{};
    int nv = 0, ntri = 0, nvi = 0, n = 0, ld = 0;
    std::vector<int> tri, vid, vtx;      // vertex -> interior id (-1), interior id -> vertex
    std::vector<double> xy, st;
    Csr am;                              // A_p and M_p pattern (contributions: 9 t + 3 a + b)
    std::vector<int> diag_pos;
    Csr lump;                            // lumped mass: one "entry" per interior row
    std::vector<int> ct_map;             // C^T rows (interior coarse nodes) -> padded coarse index
    Sell s_am;                           // the products run on SELL-32 copies
    // coupled mass, built on the device at setup: vertex-to-triangle
    // incidence (triangle order) and the workspace bounds
    std::vector<int> vt_ptr, vt_tri, vt_a;
    std::vector<long long> rec_off;      // per interior row: first slot of its record scratch
    long long cap_pairs = 0, cap_rec = 0, cap_sell_c = 0, cap_sell_ct = 0;
    int npairs = 0, nnz_c = 0, nrec_c = 0, nsell_c = 0, nsell_ct = 0;   // actual sizes (after setup)
    mutable std::vector<int> c_ptr_h, c_col_h;                          // C pattern, read back on export
    size_t ws_need = 0;
    bool ready = false;
    // device (carved from the workspace)
    int *d_tri = nullptr, *d_vid = nullptr, *d_vtx = nullptr, *d_pair_tri = nullptr, *d_pair_cell = nullptr;
    int *d_vt_ptr = nullptr, *d_vt_tri = nullptr, *d_vt_a = nullptr, *d_pcnt = nullptr, *d_poff = nullptr;
    long long* d_rec_off = nullptr;
    int *d_rec_col = nullptr, *d_rec_src = nullptr, *d_rec_cnt = nullptr, *d_uniq = nullptr, *d_c_ptr = nullptr,
        *d_g_off = nullptr, *d_c_col = nullptr, *d_c_row = nullptr;
    int *d_ct_ptr = nullptr, *d_ct_cnt = nullptr, *d_ct_col = nullptr, *d_ct_perm = nullptr, *d_sl = nullptr,
        *d_scan = nullptr, *d_total = nullptr;
    double *d_xy = nullptr, *d_st = nullptr;
    int *d_am_gptr = nullptr, *d_am_gidx = nullptr, *d_diag = nullptr;
    int *d_lp_gptr = nullptr, *d_lp_gidx = nullptr;
    int *d_c_gptr = nullptr, *d_c_gidx = nullptr;
    int* d_ct_map = nullptr;
    double *d_lk = nullptr, *d_lm = nullptr, *d_loc = nullptr;
    double *d_va = nullptr, *d_vm = nullptr, *d_vc = nullptr, *d_dinv = nullptr, *d_mlinv = nullptr;
    double *d_f = nullptr, *d_u = nullptr, *d_u2 = nullptr, *d_r = nullptr, *d_y = nullptr, *d_cres = nullptr,
           *d_cp = nullptr, *d_cq = nullptr, *d_w = nullptr;
    // outer flexible CG: residual, preconditioned residual (and its previous
    // value and the cycle's scratch), search direction, A p
    double *d_kr = nullptr, *d_kz = nullptr, *d_kzo = nullptr, *d_kz2 = nullptr, *d_kp = nullptr, *d_kq = nullptr;
    double* d_partials = nullptr;
    AuxState* d_st_aux = nullptr;
    int *d_sam_off = nullptr, *d_sam_col = nullptr, *d_sam_map = nullptr;
    int *d_sc_off = nullptr, *d_sc_col = nullptr, *d_sc_map = nullptr;
    int *d_sct_off = nullptr, *d_sct_col = nullptr, *d_sct_map = nullptr;
    double *d_sva = nullptr, *d_svm = nullptr, *d_svc = nullptr, *d_svct = nullptr;
    // FP32 preconditioner (flexible CG, lumped mass, FP32 coarse context)
    bool fp32 = false;
    float *d_sva32 = nullptr, *d_svc32 = nullptr, *d_svct32 = nullptr, *d_rs32 = nullptr, *d_dinv32 = nullptr,
          *d_mlinv32 = nullptr, *d_f32 = nullptr, *d_u32 = nullptr, *d_u32b = nullptr, *d_r32 = nullptr;
    // coarse-grid scaling (Lanczos): padded and natural coarse vectors
    double *d_cpad = nullptr, *d_cpad2 = nullptr;
    double *d_lq = nullptr, *d_lqp = nullptr, *d_lb = nullptr, *d_lbp = nullptr, *d_lv = nullptr, *d_lw = nullptr;
    // iteration graphs: flexible CG, one per parity of the z buffers (0, 1),
    // and the stationary cycle (2); valid for the coarse context's launch
    // shapes of epoch g_epoch
    cudaGraphExec_t g_exec[3] = {nullptr, nullptr, nullptr};
    long long g_kernels[3] = {0, 0, 0};
    unsigned long long g_epoch = 0;
    cudaStream_t g_stream = nullptr;
    ~bmg_aux() {
        for (int p = 0; p < 3; p++)
            if (g_exec[p]) cudaGraphExecDestroy(g_exec[p]);
        if (g_stream) cudaStreamDestroy(g_stream);
    }
};

namespace {

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

size_t carve_aux(bmg_aux& x, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = a256(off);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t I = sizeof(int), D = sizeof(double);
    const size_t npairs = (size_t)x.cap_pairs, nrec = (size_t)x.cap_rec;
    const size_t nq = x.ct_map.size();
    x.d_tri = (int*)take(I * x.tri.size());
    x.d_vid = (int*)take(I * x.nv);
    x.d_vtx = (int*)take(I * x.nvi);
    x.d_pair_tri = (int*)take(I * npairs);
    x.d_pair_cell = (int*)take(I * npairs);
    x.d_vt_ptr = (int*)take(I * x.vt_ptr.size());
    x.d_vt_tri = (int*)take(I * x.vt_tri.size());
    x.d_vt_a = (int*)take(I * x.vt_a.size());
    x.d_pcnt = (int*)take(I * (x.ntri + 1));
    x.d_poff = (int*)take(I * (x.ntri + 1));
    x.d_rec_off = (long long*)take(sizeof(long long) * x.rec_off.size());
    x.d_rec_col = (int*)take(I * nrec);
    x.d_rec_src = (int*)take(I * nrec);
    x.d_rec_cnt = (int*)take(I * (x.nvi + 1));
    x.d_uniq = (int*)take(I * (x.nvi + 1));
    x.d_c_ptr = (int*)take(I * (x.nvi + 1));
    x.d_g_off = (int*)take(I * (x.nvi + 1));
    x.d_c_col = (int*)take(I * nrec);
    x.d_c_row = (int*)take(I * nrec);
    x.d_ct_ptr = (int*)take(I * (nq + 1));
    x.d_ct_cnt = (int*)take(I * (nq + 1));
    x.d_ct_col = (int*)take(I * nrec);
    x.d_ct_perm = (int*)take(I * nrec);
    const size_t nsl = std::max<size_t>((size_t)(x.nvi + 31) / 32, (nq + 31) / 32) + 1;
    x.d_sl = (int*)take(I * nsl);
    x.d_scan = (int*)take(I * (std::max<size_t>({(size_t)x.ntri, (size_t)x.nvi, nq, nsl}) / kScanB + 2));
    x.d_total = (int*)take(I * 4);
    x.d_xy = (double*)take(D * x.xy.size());
    x.d_st = (double*)take(D * x.st.size());
    x.d_am_gptr = (int*)take(I * x.am.gptr.size());
    x.d_am_gidx = (int*)take(I * x.am.gidx.size());
    x.d_diag = (int*)take(I * x.diag_pos.size());
    x.d_lp_gptr = (int*)take(I * x.lump.gptr.size());
    x.d_lp_gidx = (int*)take(I * x.lump.gidx.size());
    x.d_c_gptr = (int*)take(I * (nrec + 1));
    x.d_c_gidx = (int*)take(I * nrec);
    x.d_ct_map = (int*)take(I * x.ct_map.size());
    x.d_lk = (double*)take(D * 9 * (size_t)x.ntri);
    x.d_lm = (double*)take(D * 9 * (size_t)x.ntri);
    x.d_loc = (double*)take(D * 12 * npairs);
    x.d_va = (double*)take(D * x.am.col.size());
    x.d_vm = (double*)take(D * x.am.col.size());
    x.d_vc = (double*)take(D * nrec);
    x.d_dinv = (double*)take(D * x.nvi);
    x.d_mlinv = (double*)take(D * x.nvi);
    double** vecs[] = {&x.d_f, &x.d_u, &x.d_u2, &x.d_r, &x.d_y, &x.d_cres, &x.d_cp, &x.d_cq, &x.d_w,
                       &x.d_kr, &x.d_kz, &x.d_kzo, &x.d_kz2, &x.d_kp, &x.d_kq};
    for (double** v : vecs) *v = (double*)take(D * std::max(x.nvi, 1));
    x.d_partials = (double*)take(D * 2 * kRedBlocks);   // two per block for the paired reductions
    x.d_st_aux = (AuxState*)take(sizeof(AuxState));
    x.d_sam_off = (int*)take(I * x.s_am.off.size());
    x.d_sam_col = (int*)take(I * x.s_am.col.size());
    x.d_sam_map = (int*)take(I * x.s_am.map.size());
    x.d_sc_off = (int*)take(I * ((x.nvi + 31) / 32 + 1));
    x.d_sc_col = (int*)take(I * (size_t)x.cap_sell_c);
    x.d_sc_map = (int*)take(I * (size_t)x.cap_sell_c);
    x.d_sct_off = (int*)take(I * ((nq + 31) / 32 + 1));
    x.d_sct_col = (int*)take(I * (size_t)x.cap_sell_ct);
    x.d_sct_map = (int*)take(I * (size_t)x.cap_sell_ct);
    x.d_sva = (double*)take(D * x.s_am.col.size());
    x.d_svm = (double*)take(D * x.s_am.col.size());
    x.d_svc = (double*)take(D * (size_t)x.cap_sell_c);
    x.d_svct = (double*)take(D * (size_t)x.cap_sell_ct);
    if (x.fp32) {
        const size_t F = sizeof(float);
        x.d_sva32 = (float*)take(F * x.s_am.col.size());
        x.d_svc32 = (float*)take(F * (size_t)x.cap_sell_c);
        x.d_svct32 = (float*)take(F * (size_t)x.cap_sell_ct);
        float** fv[] = {&x.d_rs32, &x.d_dinv32, &x.d_mlinv32, &x.d_f32, &x.d_u32, &x.d_u32b, &x.d_r32};
        for (float** v : fv) *v = (float*)take(F * std::max(x.nvi, 1));
    }
    const size_t plane = (size_t)x.ld * x.n, nn = (size_t)x.n * x.n;
    x.d_cpad = (double*)take(D * plane);
    x.d_cpad2 = (double*)take(D * plane);
    double** lv[] = {&x.d_lq, &x.d_lqp, &x.d_lb, &x.d_lbp, &x.d_lv, &x.d_lw};
    for (double** v : lv) *v = (double*)take(D * nn);
    return a256(off);
}

template <typename T>
bmg_status up(T* dst, const std::vector<T>& src, cudaStream_t s) {
    if (src.empty()) return BMG_OK;
    BMG_CUDA(cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
    return BMG_OK;
}

bmg_status aux_read(bmg_aux& x, AuxState& h) {
    cudaStream_t s = x.coarse->c.stream;
    BMG_CUDA(cudaMemcpyAsync(&h, x.d_st_aux, sizeof(AuxState), cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaStreamSynchronize(s));
    return BMG_OK;
}

// y = M^-1 r by x.opts.mass_steps CG iterations (mass_steps >= 1)
bmg_status mass_cg(bmg_aux& x, const double* r, double* y) {
    cudaStream_t s = x.coarse->c.stream;
    const int nr = x.nvi;
    k_cg_init<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, r, y, x.d_cres, x.d_cp, x.d_partials, x.d_st_aux);
    for (int k = 0; k < x.opts.mass_steps; k++) {
        if (k > 0) k_cg_p<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x.d_cres, x.d_cp, x.d_st_aux);
        k_cg_mp<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_svm, x.d_cp, x.d_cq, x.d_partials,
                                                   x.d_st_aux);
        k_cg_update<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, y, x.d_cres, x.d_cp, x.d_cq, x.d_partials, x.d_st_aux);
    }
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// one two-grid cycle (Sec. 2.2 "Solution phase") on interior vectors: u is
// updated in place for right-hand side f; u2 is scratch of the same length
bmg_status aux_cycle(bmg_aux& x, const double* f, double* u, double* u2) {
    Ctx& c = x.coarse->c;
    cudaStream_t s = c.stream;
    const int nr = x.nvi, nq = (int)x.ct_map.size();
    const bool lumped = x.opts.mass_steps == 0;
    // 1. pre-relaxation
    k_jacobi<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva, x.d_dinv, f, u, u2,
                                                x.opts.omega);
    std::swap(u, u2);
    // 2. restriction r_c = C^T M^-1 (f - A u)
    k_residual_csr<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva, f, u, x.d_r,
                                                      x.d_partials, &x.d_st_aux->counter[0], nullptr);
    const double* y = x.d_r;
    if (!lumped) {
        BMG_TRY(mass_cg(x, x.d_r, x.d_y));
        y = x.d_y;
    }
    BMG_CUDA(cudaMemsetAsync(c.r, 0, sizeof(double) * c.lev[0].plane, s));
    k_restrict_ct<<<blocks(nq), kAuxThreads, 0, s>>>(nq, x.d_sct_off, x.d_sct_col, x.d_svct, x.d_ct_map, y,
                                                     lumped ? x.d_mlinv : nullptr, c.r);
    // 3. BoxMG V-cycle on A_c e_c = r_c
    BMG_TRY(vcycle(c, c.r, c.z[0]));
    // 4. prolongation u += gamma M^-1 C e_c
    if (lumped) {
        k_prolong_c<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sc_off, x.d_sc_col, x.d_svc, c.z[0], x.d_mlinv, nullptr,
                                                       u, x.opts.gamma);
    } else {
        k_prolong_c<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sc_off, x.d_sc_col, x.d_svc, c.z[0], nullptr, x.d_w,
                                                       nullptr, 0.0);
        BMG_TRY(mass_cg(x, x.d_w, x.d_y));
        k_axpy<<<blocks(nr), kAuxThreads, 0, s>>>(nr, u, x.d_y, x.opts.gamma);
    }
    // 5. post-relaxation
    k_jacobi<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva, x.d_dinv, f, u, u2,
                                                x.opts.omega);
    std::swap(u, u2);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// One cycle from a zero guess as the preconditioner z = B r, with the
// physical level in FP32 (the coarse context's V-cycle is FP32 too): r, z
// are FP64 interior vectors.
bmg_status aux_precond32(bmg_aux& x, const double* r, double* z) {
    Ctx& c = x.coarse->c;
    cudaStream_t s = c.stream;
    const int nr = x.nvi, nq = (int)x.ct_map.size();
    const float om = (float)x.opts.omega;
    k_d2f<<<blocks(nr), kAuxThreads, 0, s>>>(nr, r, x.d_f32);
    k_jacobi32<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva32, x.d_rs32, x.d_dinv32,
                                                  x.d_f32, nullptr, x.d_u32, om);
    k_residual32<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva32, x.d_rs32, x.d_f32,
                                                    x.d_u32, x.d_r32);
    BMG_CUDA(cudaMemsetAsync(c.r, 0, sizeof(double) * c.lev[0].plane, s));
    k_restrict_ct32<<<blocks(nq), kAuxThreads, 0, s>>>(nq, x.d_sct_off, x.d_sct_col, x.d_svct32, x.d_ct_map, x.d_r32,
                                                       x.d_mlinv32, c.r);
    BMG_TRY(vcycle(c, c.r, c.z[0]));
    k_prolong_c32<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sc_off, x.d_sc_col, x.d_svc32, c.z[0], x.d_mlinv32,
                                                     x.d_u32, (float)x.opts.gamma);
    k_jacobi32<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva32, x.d_rs32, x.d_dinv32,
                                                  x.d_f32, x.d_u32, x.d_u32b, om);
    k_to64<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_u32b, z);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// z = B r: one cycle from a zero guess (FP64, or the FP32 form above)
bmg_status aux_precond(bmg_aux& x, const double* r, double* z) {
    if (x.fp32) return aux_precond32(x, r, z);
    BMG_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * x.nvi, x.coarse->c.stream));
    return aux_cycle(x, r, z, x.d_kz2);
}

// One flexible-CG iteration after the first (parity p: z_new in buffer p,
// z_old in buffer p^1): z = B r; beta; p = z + beta p; q = A p, alpha;
// u += alpha p, r -= alpha q, ||r||^2.  No host synchronisation inside.
bmg_status fcg_body(bmg_aux& x, int par) {
    cudaStream_t s = x.coarse->c.stream;
    const int nr = x.nvi;
    double* zb[2] = {x.d_kz, x.d_kzo};
    AuxState* dst = x.d_st_aux;
    BMG_TRY(aux_precond(x, x.d_kr, zb[par]));
    k_dot2_aux<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x.d_kr, zb[par], zb[par ^ 1], x.d_partials, dst, 0);
    k_p_update_aux<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_kp, zb[par], dst);
    k_spmv_dot<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva, x.d_kp, x.d_kq, x.d_partials,
                                                  dst);
    k_update_ur<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x.d_u, x.d_kr, x.d_kp, x.d_kq, dst, x.d_partials,
                                                   &dst->counter[0], &dst->rr);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// one stationary iteration: a cycle, then ||f - A u||^2
bmg_status stat_body(bmg_aux& x) {
    BMG_TRY(aux_cycle(x, x.d_f, x.d_u, x.d_u2));
    k_residual_csr<<<kRedBlocks, kAuxThreads, 0, x.coarse->c.stream>>>(x.nvi, x.d_sam_off, x.d_sam_col, x.d_sva,
                                                                       x.d_f, x.d_u, nullptr, x.d_partials,
                                                                       &x.d_st_aux->counter[0], &x.d_st_aux->rr);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

void drop_graphs(bmg_aux& x) {
    for (int p = 0; p < 3; p++)
        if (x.g_exec[p]) {
            cudaGraphExecDestroy(x.g_exec[p]);
            x.g_exec[p] = nullptr;
        }
}

bmg_status body(bmg_aux& x, int slot) { return slot < 2 ? fcg_body(x, slot) : stat_body(x); }

// Runs body(slot) as a replay of its captured graph (captured on first
// use, and again after the coarse context's launch shapes changed), or
// directly when graphs are off or the context is profiling.
bmg_status run_body(bmg_aux& x, int par) {
    Ctx& c = x.coarse->c;
    if (!c.use_graphs || c.prof_on) return body(x, par);
    if (x.g_epoch != c.shape_epoch) {
        drop_graphs(x);
        x.g_epoch = c.shape_epoch;
    }
    if (!x.g_exec[par]) {
        if (!x.g_stream) BMG_CUDA(cudaStreamCreateWithFlags(&x.g_stream, cudaStreamNonBlocking));
        cudaStream_t user = c.stream;
        c.stream = x.g_stream;
        cudaGraph_t g = nullptr;
        bmg_status st = cudaStreamBeginCapture(x.g_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess
                            ? BMG_OK
                            : BMG_ERR_DEVICE;
        const long long before = c.launches;
        if (st == BMG_OK) st = body(x, par);
        x.g_kernels[par] = c.launches - before;
        c.launches = before;
        const cudaError_t e = cudaStreamEndCapture(x.g_stream, &g);
        c.stream = user;
        if (st != BMG_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return st != BMG_OK ? st : BMG_ERR_DEVICE;
        }
        const cudaError_t ei = cudaGraphInstantiate(&x.g_exec[par], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            x.g_exec[par] = nullptr;
            return BMG_ERR_DEVICE;
        }
    }
    BMG_CUDA(cudaGraphLaunch(x.g_exec[par], c.stream));
    c.launches += x.g_kernels[par];
    return BMG_OK;
}

}  // namespace

extern "C" void bmg_aux_default_opts(bmg_aux_opts* o) {
    if (!o) return;
    o->omega = 2.0 / 3.0;
    o->mass_steps = 0;
    o->gamma = 1.0;
    o->krylov = 0;
}

namespace {
bmg_status aux_create(bmg_ctx* coarse, int nv, const double* xy, const double* st, const unsigned char* dirichlet,
                      int ntri, const int* tri, const bmg_aux_opts* opts, bmg_aux** out);
}  // namespace

// Host allocations of the build may fail for very large meshes; no C++
// exception crosses the C ABI.
extern "C" bmg_status bmg_aux_create(bmg_ctx* coarse, int nv, const double* xy, const double* st,
                                     const unsigned char* dirichlet, int ntri, const int* tri,
                                     const bmg_aux_opts* opts, bmg_aux** out) {
    try {
        return aux_create(coarse, nv, xy, st, dirichlet, ntri, tri, opts, out);
    } catch (...) {
        if (out) *out = nullptr;
        return BMG_ERR_SHAPE;
    }
}

namespace {
bmg_status aux_create(bmg_ctx* coarse, int nv, const double* xy, const double* st, const unsigned char* dirichlet,
                      int ntri, const int* tri, const bmg_aux_opts* opts, bmg_aux** out) {
    if (!out) return BMG_ERR_ARG;
    *out = nullptr;
    if (!coarse || !xy || !st || !dirichlet || !tri || nv < 3 || ntri < 1) return BMG_ERR_ARG;
    Ctx& c = coarse->c;
    if (c.dim != 2) return BMG_ERR_SHAPE;
    if (!c.attached || !c.have_setup) return BMG_ERR_STATE;
    bmg_aux_opts o;
    bmg_aux_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.omega > 0.0 && o.omega < 2.0) || o.mass_steps < 0 || o.mass_steps > 64 || !(o.gamma > 0.0) ||
        (o.krylov != 0 && o.krylov != 1))
        return BMG_ERR_ARG;
    for (long long k = 0; k < 3LL * ntri; k++)
        if (tri[k] < 0 || tri[k] >= nv) return BMG_ERR_ARG;
    if (9LL * ntri > 0x7fffffffLL) return BMG_ERR_SHAPE;
    std::unique_ptr<bmg_aux> x(new (std::nothrow) bmg_aux);
    if (!x) return BMG_ERR_ARG;
    x->coarse = coarse;
    x->opts = o;
    x->nv = nv;
    x->ntri = ntri;
    x->n = c.lev[0].n;
    x->ld = c.lev[0].ld;
    x->tri.assign(tri, tri + 3LL * ntri);
    x->xy.assign(xy, xy + 2LL * nv);
    x->st.assign(st, st + 2LL * nv);
    x->vid.assign(nv, -1);
    for (int v = 0; v < nv; v++)
        if (!dirichlet[v]) {
            x->vid[v] = (int)x->vtx.size();
            x->vtx.push_back(v);
        }
    x->nvi = (int)x->vtx.size();
    // A_p / M_p pattern and contributions (triangle order); lumped-mass rows
    {
        std::vector<int> rr, cc, src, lr, lc, ls;
        for (int t = 0; t < ntri; t++)
            for (int a = 0; a < 3; a++) {
                const int ia = x->vid[x->tri[3 * t + a]];
                if (ia < 0) continue;
                for (int b = 0; b < 3; b++) {
                    lr.push_back(ia);
                    lc.push_back(0);
                    ls.push_back(9 * t + 3 * a + b);
                    const int ib = x->vid[x->tri[3 * t + b]];
                    if (ib < 0) continue;
                    rr.push_back(ia);
                    cc.push_back(ib);
                    src.push_back(9 * t + 3 * a + b);
                }
            }
        if (!build_csr(x->nvi, rr, cc, src, x->am) || !build_csr(x->nvi, lr, lc, ls, x->lump)) {
            return BMG_ERR_SHAPE;
        }
        x->diag_pos.assign(x->nvi, -1);
        for (int i = 0; i < x->nvi; i++)
            for (int k = x->am.ptr[i]; k < x->am.ptr[i + 1]; k++)
                if (x->am.col[k] == i) x->diag_pos[i] = k;
        for (int i = 0; i < x->nvi; i++)
            if (x->diag_pos[i] < 0 || x->lump.ptr[i + 1] != i + 1) {   // an interior vertex in no triangle
                return BMG_ERR_ARG;
            }
    }
    // The coupled mass C is built on the device at setup.  Here: the
    // incidence lists (interior vertex -> (triangle, local vertex), triangle
    // order), the C^T row map, and bounds from the triangles' bounding boxes
    // in computational space for every array the device build fills.
    {
        const int n = x->n;
        const double h = 1.0 / (n - 1);
        std::vector<int> bcount(ntri);
        std::vector<int> cellcov((size_t)(n - 1) * (n - 1), 0);
        long long cap_pairs = 0;
        for (int t = 0; t < ntri; t++) {
            double sx[3], sy[3];
            for (int a = 0; a < 3; a++) {
                sx[a] = x->st[2 * x->tri[3 * t + a]];
                sy[a] = x->st[2 * x->tri[3 * t + a] + 1];
            }
            const int i0 = cell_of(std::min(sx[0], std::min(sx[1], sx[2])), h, n);
            const int i1 = cell_of(std::max(sx[0], std::max(sx[1], sx[2])), h, n);
            const int j0 = cell_of(std::min(sy[0], std::min(sy[1], sy[2])), h, n);
            const int j1 = cell_of(std::max(sy[0], std::max(sy[1], sy[2])), h, n);
            bcount[t] = (i1 - i0 + 1) * (j1 - j0 + 1);
            cap_pairs += bcount[t];
            for (int cj = j0; cj <= j1; cj++)
                for (int ci = i0; ci <= i1; ci++) cellcov[(size_t)cj * (n - 1) + ci]++;
        }
        if (12 * cap_pairs > 0x7fffffffLL) return BMG_ERR_SHAPE;
        x->cap_pairs = cap_pairs;
        // incidence, counting sort by vertex (triangles ascending within a vertex)
        x->vt_ptr.assign(x->nvi + 1, 0);
        for (int t = 0; t < ntri; t++)
            for (int a = 0; a < 3; a++) {
                const int ia = x->vid[x->tri[3 * t + a]];
                if (ia >= 0) x->vt_ptr[ia + 1]++;
            }
        for (int i = 0; i < x->nvi; i++) x->vt_ptr[i + 1] += x->vt_ptr[i];
        x->vt_tri.resize(x->vt_ptr[x->nvi]);
        x->vt_a.resize(x->vt_ptr[x->nvi]);
        {
            std::vector<int> pos(x->vt_ptr.begin(), x->vt_ptr.end() - 1);
            for (int t = 0; t < ntri; t++)
                for (int a = 0; a < 3; a++) {
                    const int ia = x->vid[x->tri[3 * t + a]];
                    if (ia < 0) continue;
                    x->vt_tri[pos[ia]] = t;
                    x->vt_a[pos[ia]] = a;
                    pos[ia]++;
                }
        }
        // records of row i: at most 4 per bounding-box cell of each incident triangle
        x->rec_off.assign(x->nvi + 1, 0);
        long long sell_c = 0;
        int slice_w = 0;
        for (int i = 0; i < x->nvi; i++) {
            long long rb = 0;
            for (int e = x->vt_ptr[i]; e < x->vt_ptr[i + 1]; e++) rb += 4LL * bcount[x->vt_tri[e]];
            x->rec_off[i + 1] = x->rec_off[i] + rb;
            if (rb > 0x7fffffffLL) return BMG_ERR_SHAPE;
            slice_w = std::max(slice_w, (int)rb);
            if (i % 32 == 31 || i == x->nvi - 1) {
                sell_c += 32LL * slice_w;
                slice_w = 0;
            }
        }
        x->cap_rec = x->rec_off[x->nvi];
        if (x->cap_rec > 0x7fffffffLL || sell_c > 0x7fffffffLL) return BMG_ERR_SHAPE;
        x->cap_sell_c = sell_c;
        // C^T rows: interior coarse nodes; entries at most 3 per triangle whose
        // bounding box covers one of the node's four cells
        const int nq = (n - 2) * (n - 2);
        x->ct_map.resize(nq);
        for (int j = 1; j <= n - 2; j++)
            for (int i = 1; i <= n - 2; i++) x->ct_map[(j - 1) * (n - 2) + (i - 1)] = j * x->ld + i;
        long long sell_ct = 0;
        long long w = 0;
        for (int q = 0; q < nq; q++) {
            const int I = q % (n - 2) + 1, J = q / (n - 2) + 1;
            long long rb = 0;
            for (int cj = J - 1; cj <= J; cj++)
                for (int ci = I - 1; ci <= I; ci++) rb += 3LL * cellcov[(size_t)cj * (n - 1) + ci];
            w = std::max(w, rb);
            if (q % 32 == 31 || q == nq - 1) {
                sell_ct += 32LL * w;
                w = 0;
            }
        }
        if (sell_ct > 0x7fffffffLL) return BMG_ERR_SHAPE;
        x->cap_sell_ct = sell_ct;
    }
    x->fp32 = o.krylov == 1 && o.mass_steps == 0 && c.opts.precision == BMG_PREC_FP32;
    if (!build_sell(x->am.ptr, x->am.col, nullptr, x->s_am)) return BMG_ERR_SHAPE;
    x->ws_need = carve_aux(*x, nullptr);
    *out = x.release();
    return BMG_OK;
}

}  // namespace

extern "C" bmg_status bmg_aux_workspace_bytes(const bmg_aux* x, size_t* bytes) {
    if (!x || !bytes) return BMG_ERR_ARG;
    *bytes = x->ws_need;
    return BMG_OK;
}

namespace {
// Exclusive prefix sum on the stream: out[0..n) and out[n] = total (also
// copied to *host_total, after a synchronisation).
bmg_status scan_ints(bmg_aux& x, const int* in, int n, int* out, int* host_total, cudaStream_t s) {
    const int nb = (n + kScanB - 1) / kScanB;
    if (nb > 0) {
        k_scan_local<<<nb, kScanB / 4, 0, s>>>(in, n, out, x.d_scan);
        k_scan_blocks<<<1, 32, 0, s>>>(x.d_scan, nb, x.d_total);
        k_scan_add<<<blocks(n), kAuxThreads, 0, s>>>(out, n, x.d_scan);
        BMG_CUDA(cudaMemcpyAsync(out + n, x.d_total, sizeof(int), cudaMemcpyDeviceToDevice, s));
    } else {
        BMG_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
    }
    if (host_total) {
        BMG_CUDA(cudaMemcpyAsync(host_total, out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
        BMG_CUDA(cudaStreamSynchronize(s));
    }
    return BMG_OK;
}

// The rasterisation and the coupled mass's sparsity on the device: (triangle,
// cell) pairs, C's CSR pattern with contribution lists, C^T, and the SELL
// patterns of C and C^T (see the kernels above).
bmg_status build_coupled_pattern(bmg_aux& x, cudaStream_t s) {
    const int ntri = x.ntri, nvi = x.nvi, n = x.n, ld = x.ld;
    const int nq = (int)x.ct_map.size();
    k_pair_count<<<blocks(ntri), kAuxThreads, 0, s>>>(ntri, x.d_tri, x.d_st, n, x.d_pcnt);
    BMG_TRY(scan_ints(x, x.d_pcnt, ntri, x.d_poff, &x.npairs, s));
    if (x.npairs > x.cap_pairs) return BMG_ERR_SHAPE;   // cannot happen: pairs lie in bounding boxes
    k_pair_fill<<<blocks(ntri), kAuxThreads, 0, s>>>(ntri, x.d_tri, x.d_st, n, x.d_poff, x.d_pair_tri, x.d_pair_cell);
    if (nvi > 0) {
        k_crow_records<<<blocks(nvi), kAuxThreads, 0, s>>>(nvi, x.d_vt_ptr, x.d_vt_tri, x.d_vt_a, x.d_poff,
                                                           x.d_pair_cell, n, ld, x.d_rec_off, x.d_rec_col,
                                                           x.d_rec_src, x.d_rec_cnt, x.d_uniq);
    }
    BMG_TRY(scan_ints(x, x.d_uniq, nvi, x.d_c_ptr, &x.nnz_c, s));
    BMG_TRY(scan_ints(x, x.d_rec_cnt, nvi, x.d_g_off, &x.nrec_c, s));
    if (nvi > 0) {
        k_crow_write<<<blocks(nvi), kAuxThreads, 0, s>>>(nvi, x.d_rec_off, x.d_rec_col, x.d_rec_src, x.d_rec_cnt,
                                                         x.d_c_ptr, x.d_g_off, x.d_c_col, x.d_c_row, x.d_c_gptr,
                                                         x.d_c_gidx);
    }
    BMG_CUDA(cudaMemcpyAsync(x.d_c_gptr + x.nnz_c, x.d_g_off + nvi, sizeof(int), cudaMemcpyDeviceToDevice, s));
    // C^T
    BMG_CUDA(cudaMemsetAsync(x.d_ct_cnt, 0, sizeof(int) * (nq + 1), s));
    if (x.nnz_c > 0) k_ct_count<<<blocks(x.nnz_c), kAuxThreads, 0, s>>>(x.nnz_c, x.d_c_col, ld, n, x.d_ct_cnt);
    BMG_TRY(scan_ints(x, x.d_ct_cnt, nq, x.d_ct_ptr, nullptr, s));
    BMG_CUDA(cudaMemsetAsync(x.d_ct_cnt, 0, sizeof(int) * (nq + 1), s));
    if (x.nnz_c > 0)
        k_ct_fill<<<blocks(x.nnz_c), kAuxThreads, 0, s>>>(x.nnz_c, x.d_c_col, x.d_c_row, ld, n, x.d_ct_ptr, x.d_ct_cnt,
                                                          x.d_ct_col, x.d_ct_perm);
    if (nq > 0) k_ct_sort<<<blocks(nq), kAuxThreads, 0, s>>>(nq, x.d_ct_ptr, x.d_ct_col, x.d_ct_perm);
    // SELL copies: slot counts per slice, offsets, then the patterns over a
    // cleared slot range (padding: column 0, map -1)
    const int ns_c = (nvi + 31) / 32, ns_t = (nq + 31) / 32;
    if (ns_c > 0) k_sell_width<<<blocks(ns_c), kAuxThreads, 0, s>>>(nvi, x.d_c_ptr, x.d_sl);
    BMG_TRY(scan_ints(x, x.d_sl, ns_c, x.d_sc_off, &x.nsell_c, s));
    if (x.nsell_c > x.cap_sell_c) return BMG_ERR_SHAPE;
    BMG_CUDA(cudaMemsetAsync(x.d_sc_col, 0, sizeof(int) * (size_t)x.nsell_c, s));
    BMG_CUDA(cudaMemsetAsync(x.d_sc_map, 0xff, sizeof(int) * (size_t)x.nsell_c, s));
    if (nvi > 0)
        k_sell_pattern<<<blocks(nvi), kAuxThreads, 0, s>>>(nvi, x.d_c_ptr, x.d_c_col, nullptr, x.d_sc_off,
                                                           x.d_sc_col, x.d_sc_map);
    if (ns_t > 0) k_sell_width<<<blocks(ns_t), kAuxThreads, 0, s>>>(nq, x.d_ct_ptr, x.d_sl);
    BMG_TRY(scan_ints(x, x.d_sl, ns_t, x.d_sct_off, &x.nsell_ct, s));
    if (x.nsell_ct > x.cap_sell_ct) return BMG_ERR_SHAPE;
    BMG_CUDA(cudaMemsetAsync(x.d_sct_col, 0, sizeof(int) * (size_t)x.nsell_ct, s));
    BMG_CUDA(cudaMemsetAsync(x.d_sct_map, 0xff, sizeof(int) * (size_t)x.nsell_ct, s));
    if (nq > 0)
        k_sell_pattern<<<blocks(nq), kAuxThreads, 0, s>>>(nq, x.d_ct_ptr, x.d_ct_col, x.d_ct_perm, x.d_sct_off,
                                                          x.d_sct_col, x.d_sct_map);
    BMG_CUDA(cudaGetLastError());
    x.c_ptr_h.clear();
    x.c_col_h.clear();
    return BMG_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" bmg_status bmg_aux_setup(bmg_aux* x, void* ws, size_t bytes, const double* kappa, const double* coords) {
    if (!x || !ws || !kappa || !coords) return BMG_ERR_ARG;
    if (!on_device(ws) || !on_device(kappa) || !on_device(coords)) return BMG_ERR_ARG;
    if (((uintptr_t)ws & 255) != 0) return BMG_ERR_ARG;
    if (bytes < x->ws_need) return BMG_ERR_WORKSPACE;
    Ctx& c = x->coarse->c;
    if (!c.attached || !c.have_setup) return BMG_ERR_STATE;
    cudaStream_t s = c.stream;
    carve_aux(*x, (char*)ws);
    BMG_CUDA(cudaMemsetAsync(x->d_st_aux, 0, sizeof(AuxState), s));
    BMG_TRY(up(x->d_tri, x->tri, s));
    BMG_TRY(up(x->d_vid, x->vid, s));
    BMG_TRY(up(x->d_vtx, x->vtx, s));
    BMG_TRY(up(x->d_xy, x->xy, s));
    BMG_TRY(up(x->d_st, x->st, s));
    BMG_TRY(up(x->d_am_gptr, x->am.gptr, s));
    BMG_TRY(up(x->d_am_gidx, x->am.gidx, s));
    BMG_TRY(up(x->d_diag, x->diag_pos, s));
    BMG_TRY(up(x->d_lp_gptr, x->lump.gptr, s));
    BMG_TRY(up(x->d_lp_gidx, x->lump.gidx, s));
    BMG_TRY(up(x->d_ct_map, x->ct_map, s));
    BMG_TRY(up(x->d_sam_off, x->s_am.off, s));
    BMG_TRY(up(x->d_sam_col, x->s_am.col, s));
    BMG_TRY(up(x->d_sam_map, x->s_am.map, s));
    BMG_TRY(up(x->d_vt_ptr, x->vt_ptr, s));
    BMG_TRY(up(x->d_vt_tri, x->vt_tri, s));
    BMG_TRY(up(x->d_vt_a, x->vt_a, s));
    BMG_TRY(up(x->d_rec_off, x->rec_off, s));
    BMG_TRY(build_coupled_pattern(*x, s));
    const int npairs = x->npairs;
    k_tri_local<<<blocks(x->ntri), kAuxThreads, 0, s>>>(x->ntri, x->d_tri, x->d_xy, kappa, x->d_lk, x->d_lm,
                                                        x->d_st_aux);
    if (npairs > 0)
        k_pair_local<<<cdiv(npairs, 128), 128, 0, s>>>(npairs, x->d_pair_tri, x->d_pair_cell, x->d_tri, x->d_st,
                                                       coords, x->n, x->d_loc);
    const int nnz = (int)x->am.col.size(), nnzc = x->nnz_c;
    if (nnz > 0) {
        k_gather<<<blocks(nnz), kAuxThreads, 0, s>>>(nnz, x->d_am_gptr, x->d_am_gidx, x->d_lk, x->d_va);
        k_gather<<<blocks(nnz), kAuxThreads, 0, s>>>(nnz, x->d_am_gptr, x->d_am_gidx, x->d_lm, x->d_vm);
    }
    if (x->nvi > 0) {
        k_diag_inv<<<blocks(x->nvi), kAuxThreads, 0, s>>>(x->nvi, x->d_diag, x->d_va, x->d_dinv);
        k_gather<<<blocks(x->nvi), kAuxThreads, 0, s>>>(x->nvi, x->d_lp_gptr, x->d_lp_gidx, x->d_lm, x->d_mlinv);
        k_inv<<<blocks(x->nvi), kAuxThreads, 0, s>>>(x->nvi, x->d_mlinv);
    }
    if (nnzc > 0) {
        k_gather<<<blocks(nnzc), kAuxThreads, 0, s>>>(nnzc, x->d_c_gptr, x->d_c_gidx, x->d_loc, x->d_vc);
    }
    const int na = (int)x->s_am.col.size(), nc = x->nsell_c, nt = x->nsell_ct;
    if (na > 0) {
        k_sell_fill<<<blocks(na), kAuxThreads, 0, s>>>(na, x->d_sam_map, x->d_va, x->d_sva);
        k_sell_fill<<<blocks(na), kAuxThreads, 0, s>>>(na, x->d_sam_map, x->d_vm, x->d_svm);
    }
    if (nc > 0) k_sell_fill<<<blocks(nc), kAuxThreads, 0, s>>>(nc, x->d_sc_map, x->d_vc, x->d_svc);
    if (nt > 0) k_sell_fill<<<blocks(nt), kAuxThreads, 0, s>>>(nt, x->d_sct_map, x->d_vc, x->d_svct);
    if (x->fp32) {
        k_d2f<<<blocks(na), kAuxThreads, 0, s>>>(na, x->d_sva, x->d_sva32);
        k_d2f<<<blocks(nc), kAuxThreads, 0, s>>>(nc, x->d_svc, x->d_svc32);
        k_d2f<<<blocks(nt), kAuxThreads, 0, s>>>(nt, x->d_svct, x->d_svct32);
        k_row_sums_sell<<<blocks(x->nvi), kAuxThreads, 0, s>>>(x->nvi, x->d_sam_off, x->d_sva, x->d_rs32);
        k_d2f<<<blocks(x->nvi), kAuxThreads, 0, s>>>(x->nvi, x->d_dinv, x->d_dinv32);
        k_d2f<<<blocks(x->nvi), kAuxThreads, 0, s>>>(x->nvi, x->d_mlinv, x->d_mlinv32);
    }
    BMG_CUDA(cudaGetLastError());
    AuxState h;
    BMG_TRY(aux_read(*x, h));
    if (h.err) return (bmg_status)h.err;
    x->ready = true;
    return BMG_OK;
}

extern "C" bmg_status bmg_aux_solve(bmg_aux* x, const double* f, double* u, double tol, int maxit, bmg_info* info) {
    if (!x || !f || !u || maxit < 0) return BMG_ERR_ARG;
    if (!on_device(f) || !on_device(u)) return BMG_ERR_ARG;
    if (!x->ready || !x->coarse->c.have_setup) return BMG_ERR_STATE;
    Ctx& c = x->coarse->c;
    cudaStream_t s = c.stream;
    const int nr = x->nvi;
    BMG_CUDA(cudaMemsetAsync(&x->d_st_aux->err, 0, sizeof(int), s));
    k_compress<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x->d_vtx, f, x->d_f);
    k_compress<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x->d_vtx, u, x->d_u);
    k_dot_aux<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_f, x->d_f, x->d_partials, &x->d_st_aux->counter[0],
                                                 &x->d_st_aux->ff);
    k_residual_csr<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_sam_off, x->d_sam_col, x->d_sva, x->d_f, x->d_u, nullptr,
                                                      x->d_partials, &x->d_st_aux->counter[0], &x->d_st_aux->rr);
    BMG_CUDA(cudaGetLastError());
    AuxState h;
    BMG_TRY(aux_read(*x, h));
    const double nf = sqrt(h.ff);
    double rel = nf > 0.0 ? sqrt(h.rr) / nf : 0.0;
    int it = 0;
    unsigned int* cnt = &x->d_st_aux->counter[0];
    if (x->opts.krylov == 0) {
        // the paper's stationary iteration
        while (it < maxit && rel > tol && nf > 0.0) {
            BMG_TRY(run_body(*x, 2));
            BMG_TRY(aux_read(*x, h));
            rel = sqrt(h.rr) / nf;
            it++;
            if (!(rel == rel)) break;   // NaN: diverged
        }
    } else if (rel > tol && nf > 0.0 && maxit > 0) {
        // flexible CG with one two-grid cycle (zero initial guess) as the
        // preconditioner z = B r; beta = r.(z - z_old) / (r_old.z_old).  The
        // scalars stay on the device; the host reads ||r|| once per
        // iteration.  Iterations after the first replay a captured graph.
        const size_t vb = sizeof(double) * nr;
        AuxState* dst = x->d_st_aux;
        k_residual_csr<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_sam_off, x->d_sam_col, x->d_sva, x->d_f, x->d_u,
                                                          x->d_kr, x->d_partials, cnt, &dst->rr);
        BMG_TRY(aux_precond(*x, x->d_kr, x->d_kz));
        BMG_CUDA(cudaMemsetAsync(x->d_kzo, 0, vb, s));
        k_dot2_aux<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_kr, x->d_kz, x->d_kzo, x->d_partials, dst, 1);
        BMG_CUDA(cudaMemcpyAsync(x->d_kp, x->d_kz, vb, cudaMemcpyDeviceToDevice, s));
        k_spmv_dot<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_sam_off, x->d_sam_col, x->d_sva, x->d_kp, x->d_kq,
                                                      x->d_partials, dst);
        k_update_ur<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_u, x->d_kr, x->d_kp, x->d_kq, dst, x->d_partials, cnt,
                                                       &dst->rr);
        BMG_CUDA(cudaGetLastError());
        while (true) {
            BMG_TRY(aux_read(*x, h));
            if (h.err) return (bmg_status)h.err;
            rel = sqrt(h.rr) / nf;
            it++;
            if (rel <= tol || !(rel == rel) || it >= maxit) break;
            BMG_TRY(run_body(*x, it & 1));
        }
        // the recursive residual drifts from f - A u: report the true one
        k_residual_csr<<<kRedBlocks, kAuxThreads, 0, s>>>(nr, x->d_sam_off, x->d_sam_col, x->d_sva, x->d_f, x->d_u,
                                                          nullptr, x->d_partials, cnt, &x->d_st_aux->rr);
        BMG_CUDA(cudaGetLastError());
        BMG_TRY(aux_read(*x, h));
        rel = sqrt(h.rr) / nf;
    }
    k_expand<<<blocks(x->nv), kAuxThreads, 0, s>>>(x->nv, x->d_vid, x->d_u, u);
    BMG_CUDA(cudaGetLastError());
    BMG_CUDA(cudaStreamSynchronize(s));
    const bmg_status st = rel <= tol || nf == 0.0 ? BMG_OK : BMG_ERR_NOT_CONVERGED;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iterations = it;
        info->levels = c.nlev + 1;
        info->relres = rel;
        info->true_relres = rel;
        info->rho = it > 0 && rel > 0.0 ? pow(rel, 1.0 / it) : 0.0;
        info->status = st;
    }
    return st;
}

namespace {

__global__ void k_scale2(int nr, double* __restrict__ a, double* __restrict__ b, double s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nr) {
        a[i] *= s;
        b[i] *= s;
    }
}

bmg_status dot_nat(bmg_aux& x, const double* a, const double* b, int len, double* out) {
    cudaStream_t s = x.coarse->c.stream;
    k_dot_aux<<<kRedBlocks, kAuxThreads, 0, s>>>(len, a, b, x.d_partials, &x.d_st_aux->counter[0], &x.d_st_aux->rr);
    BMG_CUDA(cudaGetLastError());
    AuxState h;
    BMG_TRY(aux_read(x, h));
    *out = h.rr;
    return BMG_OK;
}

// v = P^T A_p P q on the coarse grid's natural n x n layout (boundary zero),
// with the solver's own P = M_p^-1 C and P^T = C^T M_p^-1
bmg_status apply_ptap(bmg_aux& x, const double* q, double* v) {
    Ctx& c = x.coarse->c;
    cudaStream_t s = c.stream;
    const int nr = x.nvi, nq = (int)x.ct_map.size();
    const bool lumped = x.opts.mass_steps == 0;
    const dim3 gp(blocks(x.ld), x.n);
    k_to_padded<<<gp, kAuxThreads, 0, s>>>(x.n, x.ld, q, x.d_cpad);
    k_prolong_c<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sc_off, x.d_sc_col, x.d_svc, x.d_cpad,
                                                   lumped ? x.d_mlinv : nullptr, x.d_w, nullptr, 0.0);
    const double* y = x.d_w;
    if (!lumped) {
        BMG_TRY(mass_cg(x, x.d_w, x.d_y));
        y = x.d_y;
    }
    k_spmv_csr<<<blocks(nr), kAuxThreads, 0, s>>>(nr, x.d_sam_off, x.d_sam_col, x.d_sva, y, x.d_r);
    const double* z = x.d_r;
    if (!lumped) {
        BMG_TRY(mass_cg(x, x.d_r, x.d_y));
        z = x.d_y;
    }
    BMG_CUDA(cudaMemsetAsync(x.d_cpad2, 0, sizeof(double) * (size_t)x.ld * x.n, s));
    k_restrict_ct<<<blocks(nq), kAuxThreads, 0, s>>>(nq, x.d_sct_off, x.d_sct_col, x.d_svct, x.d_ct_map, z,
                                                     lumped ? x.d_mlinv : nullptr, x.d_cpad2);
    k_from_padded<<<gp, kAuxThreads, 0, s>>>(x.n, x.ld, x.d_cpad2, v);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status coarse_solve(bmg_aux& x, const double* b, double* w, double tol) {
    BMG_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * (size_t)x.n * x.n, x.coarse->c.stream));
    bmg_info info;
    return bmg_solve(x.coarse, 1, b, w, tol, 2000, &info);
}

}  // namespace

extern "C" bmg_status bmg_aux_estimate_gamma(bmg_aux* x, int k, const double* y0, double tol, double* gamma,
                                             double* alpha, double* beta, int* steps) {
    if (!x || !y0 || !gamma || k < 1 || k > 256 || !(tol > 0.0)) return BMG_ERR_ARG;
    if (!on_device(y0)) return BMG_ERR_ARG;
    if (!x->ready || !x->coarse->c.have_setup) return BMG_ERR_STATE;
    cudaStream_t s = x->coarse->c.stream;
    const int nn = x->n * x->n;
    const dim3 gp(blocks(x->ld), x->n);
    // b_0 = y0 on the interior nodes, q_0 = A_c^-1 b_0, both scaled to q_0^T A_c q_0 = 1
    k_to_padded<<<gp, kAuxThreads, 0, s>>>(x->n, x->ld, y0, x->d_cpad);
    k_from_padded<<<gp, kAuxThreads, 0, s>>>(x->n, x->ld, x->d_cpad, x->d_lb);
    BMG_CUDA(cudaGetLastError());
    BMG_TRY(coarse_solve(*x, x->d_lb, x->d_lq, tol));
    double qq = 0.0;
    BMG_TRY(dot_nat(*x, x->d_lq, x->d_lb, nn, &qq));
    if (!(qq > 0.0)) return BMG_ERR_ARG;
    k_scale2<<<blocks(nn), kAuxThreads, 0, s>>>(nn, x->d_lq, x->d_lb, 1.0 / sqrt(qq));
    BMG_CUDA(cudaMemsetAsync(x->d_lqp, 0, sizeof(double) * nn, s));
    BMG_CUDA(cudaMemsetAsync(x->d_lbp, 0, sizeof(double) * nn, s));
    double bprev = 0.0, sum = 0.0;
    int done = 0;
    for (int j = 0; j < k; j++) {
        // the vectors q_j (A_c-orthonormal) and their duals b_j = A_c q_j
        BMG_TRY(apply_ptap(*x, x->d_lq, x->d_lv));                 // v = B q_j
        double a = 0.0;
        BMG_TRY(dot_nat(*x, x->d_lq, x->d_lv, nn, &a));           // alpha_j = q_j^T B q_j
        BMG_TRY(coarse_solve(*x, x->d_lv, x->d_lw, tol));          // w = A_c^-1 B q_j
        k_lanczos_orth<<<blocks(nn), kAuxThreads, 0, s>>>(nn, x->d_lw, x->d_lq, x->d_lqp, x->d_lv, x->d_lb, x->d_lbp,
                                                          a, bprev);
        BMG_CUDA(cudaGetLastError());
        if (alpha) alpha[j] = a;
        sum += a;
        done = j + 1;
        if (j + 1 == k) break;
        double bb = 0.0;
        BMG_TRY(dot_nat(*x, x->d_lw, x->d_lv, nn, &bb));           // ||w'||_{A_c}^2 = w'^T A_c w'
        const double bj = sqrt(bb > 0.0 ? bb : 0.0);
        if (beta) beta[j] = bj;
        if (!(bj > 0.0)) break;                                     // invariant subspace
        k_lanczos_shift<<<blocks(nn), kAuxThreads, 0, s>>>(nn, x->d_lq, x->d_lqp, x->d_lw, x->d_lb, x->d_lbp,
                                                           x->d_lv, 1.0 / bj);
        BMG_CUDA(cudaGetLastError());
        bprev = bj;
    }
    BMG_CUDA(cudaStreamSynchronize(s));
    *gamma = sum / done;
    if (steps) *steps = done;
    return BMG_OK;
}

extern "C" bmg_status bmg_aux_set_gamma(bmg_aux* x, double gamma) {
    if (!x || !(gamma > 0.0)) return BMG_ERR_ARG;
    x->opts.gamma = gamma;
    drop_graphs(*x);   // gamma is a captured kernel argument
    return BMG_OK;
}

extern "C" bmg_status bmg_aux_export(const bmg_aux* x, int which, int* nrows, long long* nnz, long long* rowptr,
                                     int* col, double* val) {
    if (!x || !nrows || !nnz || which < 0 || which > 2) return BMG_ERR_ARG;
    const bool isc = which == 2;
    if (isc && !x->ready) return BMG_ERR_STATE;   // C's pattern is built on the device at setup
    if (isc && x->c_ptr_h.empty()) {
        x->c_ptr_h.resize(x->nvi + 1);
        x->c_col_h.resize(x->nnz_c);
        BMG_CUDA(cudaMemcpy(x->c_ptr_h.data(), x->d_c_ptr, sizeof(int) * (x->nvi + 1), cudaMemcpyDeviceToHost));
        if (x->nnz_c > 0)
            BMG_CUDA(cudaMemcpy(x->c_col_h.data(), x->d_c_col, sizeof(int) * x->nnz_c, cudaMemcpyDeviceToHost));
    }
    const std::vector<int>& ptr = isc ? x->c_ptr_h : x->am.ptr;
    const std::vector<int>& cl = isc ? x->c_col_h : x->am.col;
    *nrows = x->nvi;
    *nnz = (long long)cl.size();
    if (rowptr)
        for (size_t k = 0; k < ptr.size(); k++) rowptr[k] = ptr[k];
    if (col)
        for (size_t k = 0; k < cl.size(); k++) col[k] = isc ? (cl[k] / x->ld) * x->n + cl[k] % x->ld : cl[k];
    if (val) {
        if (!x->ready) return BMG_ERR_STATE;
        const double* src = which == 0 ? x->d_va : which == 1 ? x->d_vm : x->d_vc;
        if (!cl.empty()) {
            BMG_CUDA(cudaMemcpy(val, src, sizeof(double) * cl.size(), cudaMemcpyDeviceToHost));
        }
    }
    return BMG_OK;
}

extern "C" void bmg_aux_destroy(bmg_aux* x) { delete x; }
