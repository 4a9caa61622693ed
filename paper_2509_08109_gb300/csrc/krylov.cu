// krylov.cu -- vector kernels of the preconditioned conjugate-gradient outer
// loop (FP64) and of the FP32 inner CG of the refinement mode: operator
// application fused with its dot product, fused x/r updates with ||r||^2,
// r.z / r.z_old with the CG coefficient, p update, layout packing.  2-D
// (9-point) and 3-D (27-point) rows.  All reductions are deterministic:
// per-block partials summed in a fixed order by the last block (grid_sum);
// scalars stay on the device in KState.
#include "common.cuh"

namespace bmg {
namespace {

// Rows of the padded layout: r in [0, n^(DIM-1)), columns i in [0, ld).
template <int DIM>
struct RowGrid {
    int n, ld;
    __device__ __forceinline__ int rows() const { return DIM == 2 ? n : n * n; }
    __device__ __forceinline__ bool row_inner(int r) const {
        if (DIM == 2) return r >= 1 && r <= n - 2;
        const int j = r % n, k = r / n;
        return j >= 1 && j <= n - 2 && k >= 1 && k <= n - 2;
    }
};

// neighbour offset of stored plane t (t < 13) in 3-D
__device__ __forceinline__ long long d3(int t, int ld, int n) {
    return (long long)(t % 3 - 1) + (long long)ld * (((t / 3) % 3 - 1) + (long long)n * (t / 9 - 1));
}

// sum_j a_ij x_j of row o (symmetric-half storage)
template <int DIM, typename T>
__device__ __forceinline__ T apply_row(const T* __restrict__ A, long long pl, int ld, int n, const T* __restrict__ x,
                                       long long o) {
    if (DIM == 2) {
        T s = A[C2 * pl + o] * x[o];
        s += A[W2 * pl + o] * x[o - 1];
        s += A[W2 * pl + o + 1] * x[o + 1];
        s += A[S2 * pl + o] * x[o - ld];
        s += A[S2 * pl + o + ld] * x[o + ld];
        s += A[SW2 * pl + o] * x[o - ld - 1];
        s += A[SW2 * pl + o + ld + 1] * x[o + ld + 1];
        s += A[NW2 * pl + o] * x[o + ld - 1];
        s += A[NW2 * pl + o - ld + 1] * x[o - ld + 1];
        return s;
    } else {
        T s = A[13 * pl + o] * x[o];
#pragma unroll
        for (int t = 0; t < 13; t++) {
            const long long d = d3(t, ld, n);
            s += A[(long long)t * pl + o] * x[o + d];
            s += A[(long long)t * pl + o - d] * x[o - d];
        }
        return s;
    }
}

// True when every x_j row o couples to is +-0 (bit test, no FP64 op): then
// (A x)_o is zero and the FP64 products can be skipped, e.g. for a zero
// initial guess, where the residual is b itself.
template <int DIM, typename T>
__device__ __forceinline__ bool row_x_zero(const T* __restrict__ x, int ld, int n, long long o) {
    auto bits = [](T v) -> unsigned long long {
        return sizeof(T) == 8 ? (unsigned long long)__double_as_longlong((double)v) << 1
                              : (unsigned long long)__float_as_uint((float)v) << 1;
    };
    unsigned long long m = bits(x[o]);
    if (DIM == 2) {
        m |= bits(x[o - 1]) | bits(x[o + 1]) | bits(x[o - ld]) | bits(x[o + ld]);
        m |= bits(x[o - ld - 1]) | bits(x[o + ld + 1]) | bits(x[o + ld - 1]) | bits(x[o - ld + 1]);
    } else {
#pragma unroll
        for (int t = 0; t < 13; t++) {
            const long long d = d3(t, ld, n);
            m |= bits(x[o + d]) | bits(x[o - d]);
        }
    }
    return m == 0;
}

// (A x)_i in difference form: s_i x_i + sum_{j != i} a_ij (x_j - x_i), with
// the row sums s_i computed in FP64.  The operator's rows nearly sum to zero,
// so the plain FP32 product loses the smooth part of A x to cancellation; the
// differences keep FP32 relative accuracy on every mode.
template <int DIM>
__device__ __forceinline__ float apply_row_diff(const float* __restrict__ A, const float* __restrict__ rs, long long pl,
                                                int ld, int n, const float* __restrict__ x, long long o) {
    const float xo = x[o];
    float s = rs[o] * xo;
    if (DIM == 2) {
        s += A[W2 * pl + o] * (x[o - 1] - xo);
        s += A[W2 * pl + o + 1] * (x[o + 1] - xo);
        s += A[S2 * pl + o] * (x[o - ld] - xo);
        s += A[S2 * pl + o + ld] * (x[o + ld] - xo);
        s += A[SW2 * pl + o] * (x[o - ld - 1] - xo);
        s += A[SW2 * pl + o + ld + 1] * (x[o + ld + 1] - xo);
        s += A[NW2 * pl + o] * (x[o + ld - 1] - xo);
        s += A[NW2 * pl + o - ld + 1] * (x[o - ld + 1] - xo);
    } else {
#pragma unroll
        for (int t = 0; t < 13; t++) {
            const long long d = d3(t, ld, n);
            s += A[(long long)t * pl + o] * (x[o + d] - xo);
            s += A[(long long)t * pl + o - d] * (x[o - d] - xo);
        }
    }
    return s;
}

// Row sums s_i = sum_j a_ij of the FP64 operator (all stored couplings).
template <int DIM>
__device__ __forceinline__ double row_sum(const double* __restrict__ A, long long pl, int ld, int n, long long o) {
    if (DIM == 2)
        return A[C2 * pl + o] + A[W2 * pl + o] + A[W2 * pl + o + 1] + A[S2 * pl + o] + A[S2 * pl + o + ld] +
               A[SW2 * pl + o] + A[SW2 * pl + o + ld + 1] + A[NW2 * pl + o] + A[NW2 * pl + o - ld + 1];
    double s = A[13 * pl + o];
    for (int t = 0; t < 13; t++) s += A[(long long)t * pl + o] + A[(long long)t * pl + o - d3(t, ld, n)];
    return s;
}

// Compensated (Neumaier) FP32 accumulator for the inner CG's dot products.
struct Acc32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

#define FOR_ROWS(g)                                                       \
    for (int r_ = blockIdx.x; r_ < (g).rows(); r_ += gridDim.x)           \
        for (int i_ = threadIdx.x; i_ < (g).ld; i_ += blockDim.x)

// ---------------------------------------------------------------- layout
template <int DIM>
__global__ void k_pack_t(int n, int ld, const double* __restrict__ src, double* __restrict__ dst) {
    RowGrid<DIM> g{n, ld};
    FOR_ROWS(g) {
        const bool in = g.row_inner(r_) && i_ >= 1 && i_ <= n - 2;
        dst[(long long)r_ * ld + i_] = in ? src[(long long)r_ * n + i_] : 0.0;
    }
}

template <int DIM>
__global__ void k_unpack_t(int n, int ld, const double* __restrict__ src, double* __restrict__ dst) {
    RowGrid<DIM> g{n, ld};
    FOR_ROWS(g) {
        if (i_ < n) dst[(long long)r_ * n + i_] = src[(long long)r_ * ld + i_];
    }
}

// ---------------------------------------------------------------- FP64 outer CG
// r = b - A x ; st.rr = ||r||^2 (rows with a zero x neighbourhood: r = b)
template <int DIM>
__global__ void k_residual64(RowGrid<DIM> g, const double* __restrict__ A, long long pl, const double* __restrict__ b,
                             const double* __restrict__ x, double* __restrict__ r, double* partials, KState* st) {
    double acc = 0.0;
    FOR_ROWS(g) {
        const long long k = (long long)r_ * g.ld + i_;
        double v = 0.0;
        if (g.row_inner(r_) && i_ >= 1 && i_ <= g.n - 2)
            v = row_x_zero<DIM, double>(x, g.ld, g.n, k) ? b[k] : b[k] - apply_row<DIM, double>(A, pl, g.ld, g.n, x, k);
        r[k] = v;
        acc += v * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[0], &t)) st->rr = t;
}

__global__ void k_dot64(long long tot, const double* __restrict__ a, const double* __restrict__ b, double* partials,
                        KState* st, double* slot) {
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x)
        acc += a[k] * b[k];
    double t;
    if (grid_sum(acc, partials, &st->counter[1], &t)) *slot = t;
}

// q = A p; st.pq = p.q; alpha = rz / pq
template <int DIM>
__global__ void k_spmv_pq64(RowGrid<DIM> g, const double* __restrict__ A, long long pl, const double* __restrict__ p,
                            double* __restrict__ q, double* partials, KState* st) {
    double acc = 0.0;
    FOR_ROWS(g) {
        const long long k = (long long)r_ * g.ld + i_;
        double v = 0.0;
        if (g.row_inner(r_) && i_ >= 1 && i_ <= g.n - 2) v = apply_row<DIM, double>(A, pl, g.ld, g.n, p, k);
        q[k] = v;
        acc += p[k] * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[2], &t)) {
        st->pq = t;
        if (!(t > 0.0)) {
            set_err(st, BMG_ERR_NOT_SPD);
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / t;
        }
    }
}

// x += alpha p; r -= alpha q; st.rr = ||r||^2
__global__ void k_update_xr64(long long tot, double* __restrict__ x, double* __restrict__ r,
                              const double* __restrict__ p, const double* __restrict__ q, double* partials,
                              KState* st) {
    const double alpha = st->alpha;
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        x[k] += alpha * p[k];
        const double rv = r[k] - alpha * q[k];
        r[k] = rv;
        acc += rv * rv;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[3], &t)) st->rr = t;
}

// r.z and (flexible) r.z_old in one pass, then beta in the last block; the
// first iteration has no beta.
__global__ void k_rz_beta64(long long tot, const double* __restrict__ r, const double* __restrict__ z,
                            const double* __restrict__ zo, int flexible, double* partials, KState* st) {
    double a1 = 0.0, a2 = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        const double rv = r[k];
        a1 += rv * z[k];
        if (flexible) a2 += rv * zo[k];
    }
    double t1, t2;
    if (grid_sum2(a1, a2, partials, &st->counter[5], &t1, &t2)) {
        if (st->first) {
            st->beta = 0.0;
            st->first = 0;
        } else {
            st->beta = (flexible ? t1 - t2 : t1) / st->rz;
        }
        st->rz = t1;
    }
}

// p = z + beta p
__global__ void k_p_update64(long long tot, const double* __restrict__ z, double* __restrict__ p, KState* st) {
    const double beta = st->beta;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x)
        p[k] = z[k] + beta * p[k];
}

// ---------------------------------------------------------------- refinement (FP32 inner CG)
// r32 = (float)(b - A x), ||r||^2 in FP64; resets the inner CG to its first step.
// Rows whose x neighbourhood is zero take r = b without the FP64 products
// (the FP64 rate, not HBM, bounds this kernel otherwise).
template <int DIM>
__global__ void k_residual_to32_t(RowGrid<DIM> g, const double* __restrict__ A, long long pl,
                                  const double* __restrict__ b, const double* __restrict__ x,
                                  float* __restrict__ r32, double* partials, KState* st) {
    double acc = 0.0;
    FOR_ROWS(g) {
        const long long k = (long long)r_ * g.ld + i_;
        double v = 0.0;
        if (g.row_inner(r_) && i_ >= 1 && i_ <= g.n - 2)
            v = row_x_zero<DIM, double>(x, g.ld, g.n, k) ? b[k] : b[k] - apply_row<DIM, double>(A, pl, g.ld, g.n, x, k);
        r32[k] = (float)v;
        acc += v * v;
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[0], &t)) {
        st->rr = t;
        st->first = 1;
    }
}

template <int DIM>
__global__ void k_row_sums32_t(RowGrid<DIM> g, const double* __restrict__ A, long long pl, float* __restrict__ rs) {
    FOR_ROWS(g) {
        const long long k = (long long)r_ * g.ld + i_;
        double v = 0.0;
        if (g.row_inner(r_) && i_ >= 1 && i_ <= g.n - 2) v = row_sum<DIM>(A, pl, g.ld, g.n, k);
        rs[k] = (float)v;
    }
}

// p = z + beta p_old, then q = A p (difference form), alpha = rz / p.q, in one
// pass: each row forms p at its nine (27) neighbours on the fly from z and
// p_old, so p is written to a second buffer (p_old is still being read).
template <int DIM>
__global__ void k_pspmv32_t(RowGrid<DIM> g, const float* __restrict__ A, const float* __restrict__ rs, long long pl,
                            const float* __restrict__ z, const float* __restrict__ pold, float* __restrict__ p,
                            float* __restrict__ q, double* partials, KState* st) {
    const float beta = (float)st->beta;
    Acc32 acc;
    FOR_ROWS(g) {
        const long long k = (long long)r_ * g.ld + i_;
        float pv = 0.0f, v = 0.0f;
        if (g.row_inner(r_) && i_ >= 1 && i_ <= g.n - 2) {
            auto P = [&](long long o) { return z[o] + beta * pold[o]; };
            pv = P(k);
            float s = rs[k] * pv;
            if (DIM == 2) {
                const int ld = g.ld;
                s += A[W2 * pl + k] * (P(k - 1) - pv);
                s += A[W2 * pl + k + 1] * (P(k + 1) - pv);
                s += A[S2 * pl + k] * (P(k - ld) - pv);
                s += A[S2 * pl + k + ld] * (P(k + ld) - pv);
                s += A[SW2 * pl + k] * (P(k - ld - 1) - pv);
                s += A[SW2 * pl + k + ld + 1] * (P(k + ld + 1) - pv);
                s += A[NW2 * pl + k] * (P(k + ld - 1) - pv);
                s += A[NW2 * pl + k - ld + 1] * (P(k - ld + 1) - pv);
            } else {
#pragma unroll
                for (int t = 0; t < 13; t++) {
                    const long long d = d3(t, g.ld, g.n);
                    s += A[(long long)t * pl + k] * (P(k + d) - pv);
                    s += A[(long long)t * pl + k - d] * (P(k - d) - pv);
                }
            }
            v = s;
        }
        p[k] = pv;
        q[k] = v;
        acc.add(pv * v);
    }
    double t;
    if (grid_sum(acc.value(), partials, &st->counter[2], &t)) {
        st->pq = t;
        if (!(t > 0.0)) {
            set_err(st, BMG_ERR_NOT_SPD);
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / t;
        }
    }
}

// x += alpha p straight into the FP64 iterate (an FP32 correction would cap
// the true residual near eps_32 ||A|| ||d|| / ||A d||, far above 1e-10 for a
// smooth correction d); r -= alpha q in FP32.
__global__ void k_update_xr32(long long tot, double* __restrict__ x, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q, const KState* st) {
    const double alpha = st->alpha;
    const float a32 = (float)alpha;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        x[k] += alpha * (double)p[k];
        r[k] -= a32 * q[k];
    }
}

// r.z and r.z_old in one pass; the last block forms the flexible-CG beta
__global__ void k_rz_beta32_t(long long tot, const float* __restrict__ r, const float* __restrict__ z,
                              const float* __restrict__ zo, double* partials, KState* st) {
    Acc32 a1, a2;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        const float rv = r[k];
        a1.add(rv * z[k]);
        a2.add(rv * zo[k]);
    }
    double t1, t2;
    if (grid_sum2(a1.value(), a2.value(), partials, &st->counter[4], &t1, &t2)) {
        if (st->first) {
            st->beta = 0.0;
            st->first = 0;
        } else {
            st->beta = (t1 - t2) / st->rz;
        }
        st->rz = t1;
    }
}

inline double dofs0(const Ctx& c) {
    const double m = c.lev[0].n - 2;
    return c.dim == 2 ? m * m : m * m * m;
}

#define DISPATCH_DIM(c, KERNEL, ...)                                                                      \
    do {                                                                                                  \
        const Level& L_ = (c).lev[0];                                                                     \
        if ((c).dim == 2)                                                                                 \
            KERNEL<2><<<(c).red_blocks, kThreads, 0, (c).stream>>>(RowGrid<2>{L_.n, L_.ld}, __VA_ARGS__);  \
        else                                                                                              \
            KERNEL<3><<<(c).red_blocks, kThreads, 0, (c).stream>>>(RowGrid<3>{L_.n, L_.ld}, __VA_ARGS__);  \
        (c).launches++;                                                                                   \
    } while (0)

}  // namespace

bmg_status k_pack(Ctx& c, const double* src, double* dst) {
    const Level& L = c.lev[0];
    if (c.dim == 2)
        k_pack_t<2><<<c.red_blocks, kThreads, 0, c.stream>>>(L.n, L.ld, src, dst);
    else
        k_pack_t<3><<<c.red_blocks, kThreads, 0, c.stream>>>(L.n, L.ld, src, dst);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_unpack(Ctx& c, const double* src, double* dst) {
    const Level& L = c.lev[0];
    if (c.dim == 2)
        k_unpack_t<2><<<c.red_blocks, kThreads, 0, c.stream>>>(L.n, L.ld, src, dst);
    else
        k_unpack_t<3><<<c.red_blocks, kThreads, 0, c.stream>>>(L.n, L.ld, src, dst);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_residual(Ctx& c, const double* b, const double* x, double* r) {
    const Level& L = c.lev[0];
    DISPATCH_DIM(c, k_residual64, L.A64, L.plane, b, x, r, c.partials, c.st);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_dot(Ctx& c, const double* a, const double* b, double* slot) {
    const Level& L = c.lev[0];
    k_dot64<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, a, b, c.partials, c.st, slot);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_spmv_pq(Ctx& c, const double* p, double* q) {
    const Level& L = c.lev[0];
    prof_begin(c, BMG_PROF_SPMV, 0);
    DISPATCH_DIM(c, k_spmv_pq64, L.A64, L.plane, p, q, c.partials, c.st);
    prof_end(c, BMG_PROF_SPMV, 0, (c.ns + 2) * 8.0 * dofs0(c));
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_update_xr(Ctx& c) {
    const Level& L = c.lev[0];
    prof_begin(c, BMG_PROF_UPDATE, 0);
    k_update_xr64<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.x, c.r, c.p, c.q, c.partials, c.st);
    prof_end(c, BMG_PROF_UPDATE, 0, 6 * 8.0 * dofs0(c));
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_rz_beta(Ctx& c, const double* z, const double* zold, bool flexible) {
    const Level& L = c.lev[0];
    k_rz_beta64<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.r, z, zold, flexible ? 1 : 0, c.partials, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_p_update(Ctx& c, const double* z) {
    const Level& L = c.lev[0];
    k_p_update64<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, z, c.p, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_residual_to32(Ctx& c) {
    const Level& L = c.lev[0];
    DISPATCH_DIM(c, k_residual_to32_t, L.A64, L.plane, c.bvec, c.x, c.r32, c.partials, c.st);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// 2-D form of k_pspmv32_t: one CTA per tile of kThreads interior columns x H
// rows, marching up the rows.  Every value of z, p_old and of the stored
// planes is loaded once (plus a one-column, two-row halo) into a four-row
// ring in shared memory; the loads of row j+2 are in flight while row j is
// formed, with one barrier per row.  Same arithmetic, in the same order, as
// k_pspmv32_t<2>.
__global__ void __launch_bounds__(kThreads) k_pspmv2d_tiled(int n, int ld, long long pl, int H, int tiles_x,
                                                            const float* __restrict__ A,
                                                            const float* __restrict__ rs,
                                                            const float* __restrict__ z,
                                                            const float* __restrict__ pold, float* __restrict__ p,
                                                            float* __restrict__ q, double* partials, KState* st) {
    constexpr int TW = kThreads;
    __shared__ float sP[4][TW + 2];    // p at columns i0-1 .. i0+TW
    __shared__ float sW[4][TW + 1];    // stored planes at columns i0 .. i0+TW
    __shared__ float sSW[4][TW + 1];
    __shared__ float sNW[4][TW + 1];
    const float beta = (float)st->beta;
    const int t = threadIdx.x;
    const int i0 = 1 + (int)(blockIdx.x % tiles_x) * TW;
    const int j0 = 1 + (int)(blockIdx.x / tiles_x) * H;
    const int j1 = min(j0 + H, n - 1);
    const int i = i0 + t;
    const bool act = i <= n - 2;
    const int il = i0 - 1, ir = i0 + TW;    // halo columns (thread 0: left, thread 1: right)
    // raw loads only: p = z + beta p_old is formed when the row is stored,
    // a step later, so no instruction waits on these loads before the
    // current row has been computed
    struct Row {
        float z, po, w, sw, nw, s, r, hz, hpo, hw, hsw, hnw;
    };
    auto load = [&](int j, Row& v) {
        v = Row{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (j < 1 || j > n - 2) return;
        const long long kr = (long long)j * ld;
        if (act) {
            const long long k = kr + i;
            v.z = z[k];
            v.po = pold[k];
            v.w = A[W2 * pl + k];
            v.sw = A[SW2 * pl + k];
            v.nw = A[NW2 * pl + k];
            v.s = A[S2 * pl + k];
            v.r = rs[k];
        }
        if (t == 0 && il >= 1) {
            v.hz = z[kr + il];
            v.hpo = pold[kr + il];
        }
        if (t == 1 && ir <= n - 2) {
            const long long k = kr + ir;
            v.hz = z[k];
            v.hpo = pold[k];
            v.hw = A[W2 * pl + k];
            v.hsw = A[SW2 * pl + k];
            v.hnw = A[NW2 * pl + k];
        }
    };
    auto put = [&](int j, const Row& v) {
        const int sl = j & 3;
        sP[sl][t + 1] = v.z + beta * v.po;
        sW[sl][t] = v.w;
        sSW[sl][t] = v.sw;
        sNW[sl][t] = v.nw;
        if (t == 0) sP[sl][0] = v.hz + beta * v.hpo;
        if (t == 1) {
            sP[sl][TW + 1] = v.hz + beta * v.hpo;
            sW[sl][TW] = v.hw;
            sSW[sl][TW] = v.hsw;
            sNW[sl][TW] = v.hnw;
        }
    };
    Row nx;
    load(j0 - 1, nx);
    put(j0 - 1, nx);
    load(j0, nx);
    put(j0, nx);
    float rs_j = nx.r, s_j = nx.s;
    load(j0 + 1, nx);
    Acc32 acc;
    for (int j = j0; j < j1; j++) {
        put(j + 1, nx);
        const float s_n = nx.s, rs_n = nx.r;
        load(j + 2, nx);
        __syncthreads();
        if (act) {
            const int sm = (j - 1) & 3, s0 = j & 3, sp = (j + 1) & 3;
            const float pv = sP[s0][t + 1];
            float v = rs_j * pv;
            v += sW[s0][t] * (sP[s0][t] - pv);
            v += sW[s0][t + 1] * (sP[s0][t + 2] - pv);
            v += s_j * (sP[sm][t + 1] - pv);
            v += s_n * (sP[sp][t + 1] - pv);
            v += sSW[s0][t] * (sP[sm][t] - pv);
            v += sSW[sp][t + 1] * (sP[sp][t + 2] - pv);
            v += sNW[s0][t] * (sP[sp][t] - pv);
            v += sNW[sm][t + 1] * (sP[sm][t + 2] - pv);
            const long long k = (long long)j * ld + i;
            p[k] = pv;
            q[k] = v;
            acc.add(pv * v);
        }
        rs_j = rs_n;
        s_j = s_n;
    }
    double tot;
    if (grid_sum(acc.value(), partials, &st->counter[2], &tot)) {
        st->pq = tot;
        if (!(tot > 0.0)) {
            set_err(st, BMG_ERR_NOT_SPD);
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / tot;
        }
    }
}

bmg_status k_row_sums32(Ctx& c) {
    const Level& L = c.lev[0];
    DISPATCH_DIM(c, k_row_sums32_t, L.A64, L.plane, c.rs32);
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_rz_beta32(Ctx& c, const float* z, const float* zo) {
    const Level& L = c.lev[0];
    k_rz_beta32_t<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.r32, z, zo, c.partials, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// 3-D form of k_pspmv32_t: one CTA per tile of 32 x 8 (i, j) interior nodes
// and a band of k-planes, marching up k; p of the next k-plane, with a
// one-node halo in i and j, goes from registers (loaded a step ahead) into a
// shared ring of 4 slots, so one barrier per plane suffices.
constexpr int kP3I = 32, kP3J = 8;
constexpr int kP3W = kP3I + 2, kP3H = kP3J + 2, kP3A = kP3W * kP3H;   // halo tile
constexpr int kP3Per = (kP3A + kThreads - 1) / kThreads;              // halo positions per thread

// The stencil is read straight from global memory: each thread loads its
// node's 13 stored planes and the 13 mirrors a(-d) (stored at the node - d)
// into registers before the step's barrier, so the loads overlap the wait;
// the mirrors of the CTA's interior are its own threads' loads of a
// neighbouring row or of the next plane, served by L1 and L2.  Only p lives
// in shared memory, so the CTA's footprint is a few KB and occupancy is set
// by registers (64 per thread, 4 CTAs per SM).  A version that staged the 13
// planes in shared rings as well (58 KB per CTA, 3 CTAs per SM) took 349
// instead of 253 us per 257^3 product.  Same products in the same order as
// k_pspmv32_t<3>.
__global__ void __launch_bounds__(kThreads) k_pspmv3d_direct(int n, int ld, long long pl, int H, int tiles_i,
                                                             int tiles_j, const float* __restrict__ A,
                                                             const float* __restrict__ rs,
                                                             const float* __restrict__ z,
                                                             const float* __restrict__ pold, float* __restrict__ p,
                                                             float* __restrict__ q, double* partials, KState* st) {
    __shared__ float sP[4][kP3A];
    const float beta = (float)st->beta;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int ti = tile % tiles_i, tj = (tile / tiles_i) % tiles_j, tk = tile / (tiles_i * tiles_j);
    const int i0 = 1 + ti * kP3I, j0 = 1 + tj * kP3J, k0 = 1 + tk * H;
    const int k1 = min(k0 + H, n - 1);
    const long long sz = (long long)ld * n;
    float rz[kP3Per], rpo[kP3Per];
    auto load = [&](int k) {
#pragma unroll
        for (int u = 0; u < kP3Per; u++) {
            const int h = tid + u * kThreads;
            const int hi = h % kP3W, hj = h / kP3W;
            const int i = i0 - 1 + hi, j = j0 - 1 + hj;
            const bool in = h < kP3A && i <= n - 1 && j <= n - 1 && k >= 0 && k <= n - 1;
            const long long o = in ? (long long)i + (long long)ld * j + sz * k : 0;
            rz[u] = in ? z[o] : 0.f;
            rpo[u] = in ? pold[o] : 0.f;
        }
    };
    auto put = [&](int k) {
        float* pp = sP[k & 3];
#pragma unroll
        for (int u = 0; u < kP3Per; u++) {
            const int h = tid + u * kThreads;
            if (h < kP3A) pp[h] = rz[u] + beta * rpo[u];
        }
    };
    const int ti_ = tid % kP3I, tj_ = tid / kP3I;
    const int i = i0 + ti_, j = j0 + tj_;
    const bool act = i <= n - 2 && j <= n - 2;
    const int hc = (tj_ + 1) * kP3W + (ti_ + 1);
    load(k0 - 1);
    put(k0 - 1);
    load(k0);
    put(k0);
    load(k0 + 1);
    Acc32 acc;
    for (int k = k0; k < k1; k++) {
        put(k + 1);
        load(k + 2);
        const long long o = (long long)i + (long long)ld * j + sz * k;
        float a0[13], am[13], rsv = 0.f;
        if (act) {
#pragma unroll
            for (int t = 0; t < 13; t++) {
                const long long d = (t % 3 - 1) + (long long)ld * ((t / 3) % 3 - 1) + sz * (t / 9 - 1);
                a0[t] = __ldg(A + t * pl + o);
                am[t] = __ldg(A + t * pl + o - d);
            }
            rsv = __ldg(rs + o);
        }
        __syncthreads();
        if (act) {
            const float* pm = sP[(k + 3) & 3];   // p at k-1
            const float* p0 = sP[k & 3];         // p at k
            const float* pp = sP[(k + 1) & 3];   // p at k+1
            const float pv = p0[hc];
            float s = rsv * pv;
#pragma unroll
            for (int t = 0; t < 13; t++) {
                const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
                const int dh = dx + dy * kP3W;
                const float* pn = dz < 0 ? pm : p0;
                const float* pr = dz < 0 ? pp : p0;
                s += a0[t] * (pn[hc + dh] - pv);
                s += am[t] * (pr[hc - dh] - pv);
            }
            p[o] = pv;
            q[o] = s;
            acc.add(pv * s);
        }
    }
    double tot;
    if (grid_sum(acc.value(), partials, &st->counter[2], &tot)) {
        st->pq = tot;
        if (!(tot > 0.0)) {
            set_err(st, BMG_ERR_NOT_SPD);
            st->alpha = 0.0;
        } else {
            st->alpha = st->rz / tot;
        }
    }
}

// Rows per tile of k_pspmv2d_tiled: minimise waves x (rows + 2 halo rows)
// at the kernel's occupancy, with at most kMaxBlocks tiles.
bmg_status pspmv_prepare(Ctx& c) {
    if (!c.rs32) return BMG_OK;
    if (c.dim == 3) {
        // bands of k-planes: minimise waves x (planes + 2) with at most kMaxBlocks tiles
        int sms = 0, occ = 0;
        BMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
        BMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pspmv3d_direct, kThreads, 0));
        if (occ < 1) return BMG_ERR_DEVICE;
        const int m = c.lev[0].n - 2;
        const int ti = cdiv(m, kP3I), tj = cdiv(m, kP3J);
        const long long slots = (long long)sms * occ;
        long long best = -1;
        for (int h = 1; h <= m; h++) {
            const long long tiles = (long long)ti * tj * cdiv(m, h);
            if (tiles > kMaxBlocks) continue;
            const long long cost = cdiv(tiles, slots) * (h + 2LL);
            if (best < 0 || cost < best) {
                best = cost;
                c.spmv_h = h;
                c.spmv_tiles_x = ti;
                c.spmv_tiles = (int)tiles;
            }
        }
        return best < 0 ? BMG_ERR_SHAPE : BMG_OK;
    }
    int sms = 0, occ = 0;
    BMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    BMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pspmv2d_tiled, kThreads, 0));
    if (occ < 1) return BMG_ERR_DEVICE;
    const int m = c.lev[0].n - 2;
    const int tx = cdiv(m, kThreads);
    const long long slots = (long long)sms * occ;
    long long best = -1;
    for (int h = 1; h <= m; h++) {
        const long long tiles = (long long)tx * cdiv(m, h);
        if (tiles > kMaxBlocks) continue;
        const long long cost = cdiv(tiles, slots) * (h + 2LL);
        if (best < 0 || cost < best) {
            best = cost;
            c.spmv_h = h;
            c.spmv_tiles_x = tx;
            c.spmv_tiles = (int)tiles;
        }
    }
    return best < 0 ? BMG_ERR_SHAPE : BMG_OK;
}

bmg_status k_pspmv32(Ctx& c, const float* z, int parity) {
    const Level& L = c.lev[0];
    prof_begin(c, BMG_PROF_SPMV, 0);
    if (c.dim == 2 && c.spmv_h > 0) {
        k_pspmv2d_tiled<<<c.spmv_tiles, kThreads, 0, c.stream>>>(L.n, L.ld, L.plane, c.spmv_h, c.spmv_tiles_x,
                                                                 L.A32, c.rs32, z, c.p32s[parity ^ 1],
                                                                 c.p32s[parity], c.q32, c.partials, c.st);
        c.launches++;
    } else if (c.dim == 3 && c.spmv_h > 0) {
        const int tj = cdiv(L.n - 2, kP3J);
        k_pspmv3d_direct<<<c.spmv_tiles, kThreads, 0, c.stream>>>(L.n, L.ld, L.plane, c.spmv_h, c.spmv_tiles_x, tj,
                                                                 L.A32, c.rs32, z, c.p32s[parity ^ 1],
                                                                 c.p32s[parity], c.q32, c.partials, c.st);
        c.launches++;
    } else {
        DISPATCH_DIM(c, k_pspmv32_t, L.A32, c.rs32, L.plane, z, c.p32s[parity ^ 1], c.p32s[parity], c.q32,
                     c.partials, c.st);
    }
    prof_end(c, BMG_PROF_SPMV, 0, (c.ns + 4) * 4.0 * dofs0(c));
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_update_dr32(Ctx& c, int parity) {
    const Level& L = c.lev[0];
    prof_begin(c, BMG_PROF_UPDATE, 0);
    k_update_xr32<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.x, c.r32, c.p32s[parity], c.q32, c.st);
    prof_end(c, BMG_PROF_UPDATE, 0, (4 * 4.0 + 2 * 8.0) * dofs0(c));
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
