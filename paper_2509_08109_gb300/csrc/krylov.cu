// krylov.cu -- FP64 vector kernels of the preconditioned conjugate-gradient
// outer loop: operator application fused with its dot product, fused
// x/r updates with ||r||^2, r.z with the CG coefficient, p update, layout
// packing.  All reductions are deterministic: per-block partials summed in
// a fixed order by the last block (see grid_sum); scalars stay on the
// device in KState.
#include "common.cuh"

namespace bmg {
namespace {

__device__ __forceinline__ double apply_row2d(const double* __restrict__ A, long long pl, int ld,
                                              const double* __restrict__ x, long long o) {
    double s = A[C2 * pl + o] * x[o];
    s += A[W2 * pl + o] * x[o - 1];
    s += A[W2 * pl + o + 1] * x[o + 1];
    s += A[S2 * pl + o] * x[o - ld];
    s += A[S2 * pl + o + ld] * x[o + ld];
    s += A[SW2 * pl + o] * x[o - ld - 1];
    s += A[SW2 * pl + o + ld + 1] * x[o + ld + 1];
    s += A[NW2 * pl + o] * x[o + ld - 1];
    s += A[NW2 * pl + o - ld + 1] * x[o - ld + 1];
    return s;
}

// row-wise traversal of the padded layout (row j, column i)
struct Grid2 {
    int n, ld;
};

__global__ void k_pack2d(int n, int ld, const double* __restrict__ src, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= ld) return;
    const bool in = i >= 1 && j >= 1 && i <= n - 2 && j <= n - 2;
    dst[(long long)j * ld + i] = in ? src[(long long)j * n + i] : 0.0;
}

__global__ void k_unpack2d(int n, int ld, const double* __restrict__ src, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    dst[(long long)j * n + i] = src[(long long)j * ld + i];
}

// r = b - A x ; st.rr = ||r||^2
__global__ void k_residual64(Grid2 g, const double* __restrict__ A, long long pl, const double* __restrict__ b,
                             const double* __restrict__ x, double* __restrict__ r, double* partials, KState* st) {
    double acc = 0.0;
    for (int j = blockIdx.x; j < g.n; j += gridDim.x) {
        const bool rj = j >= 1 && j <= g.n - 2;
        for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
            const long long k = (long long)j * g.ld + i;
            double v = 0.0;
            if (rj && i >= 1 && i <= g.n - 2) v = b[k] - apply_row2d(A, pl, g.ld, x, k);
            r[k] = v;
            acc += v * v;
        }
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
__global__ void k_spmv_pq(Grid2 g, const double* __restrict__ A, long long pl, const double* __restrict__ p,
                          double* __restrict__ q, double* partials, KState* st) {
    double acc = 0.0;
    for (int j = blockIdx.x; j < g.n; j += gridDim.x) {
        const bool rj = j >= 1 && j <= g.n - 2;
        for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
            const long long k = (long long)j * g.ld + i;
            double v = 0.0;
            if (rj && i >= 1 && i <= g.n - 2) v = apply_row2d(A, pl, g.ld, p, k);
            q[k] = v;
            acc += p[k] * v;
        }
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
__global__ void k_update_xr(long long tot, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q, double* partials, KState* st) {
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
__global__ void k_p_update(long long tot, const double* __restrict__ z, double* __restrict__ p, KState* st) {
    const double beta = st->beta;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x)
        p[k] = z[k] + beta * p[k];
}

// ---------------------------------------------------------------- refinement (FP32 inner CG)
// Compensated (Neumaier) FP32 accumulator: the inner CG's dot products mix
// signs heavily, and a plain FP32 running sum loses the small total.
struct Acc32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// r32 = (float)(b - A x), ||r||^2 in FP64; resets the inner CG to its first step.
__global__ void k_residual_to32(Grid2 g, const double* __restrict__ A, long long pl, const double* __restrict__ b,
                                const double* __restrict__ x, float* __restrict__ r32, double* partials, KState* st) {
    double acc = 0.0;
    for (int j = blockIdx.x; j < g.n; j += gridDim.x) {
        const bool rj = j >= 1 && j <= g.n - 2;
        for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
            const long long k = (long long)j * g.ld + i;
            double v = 0.0;
            if (rj && i >= 1 && i <= g.n - 2) v = b[k] - apply_row2d(A, pl, g.ld, x, k);
            r32[k] = (float)v;
            acc += v * v;
        }
    }
    double t;
    if (grid_sum(acc, partials, &st->counter[0], &t)) {
        st->rr = t;
        st->first = 1;
    }
}

// x += d (FP64 += FP32), d = 0
__global__ void k_add_correction(long long tot, double* __restrict__ x, float* __restrict__ d) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        x[k] += (double)d[k];
        d[k] = 0.0f;
    }
}

// Row sums s_i = sum_j a_ij of the FP64 operator, stored in FP32.
__global__ void k_row_sums32(Grid2 g, const double* __restrict__ A, long long pl, float* __restrict__ rs) {
    for (int j = blockIdx.x; j < g.n; j += gridDim.x)
        for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
            const long long o = (long long)j * g.ld + i;
            double s = 0.0;
            if (j >= 1 && j <= g.n - 2 && i >= 1 && i <= g.n - 2) {
                s = A[C2 * pl + o] + A[W2 * pl + o] + A[W2 * pl + o + 1] + A[S2 * pl + o] + A[S2 * pl + o + g.ld] +
                    A[SW2 * pl + o] + A[SW2 * pl + o + g.ld + 1] + A[NW2 * pl + o] + A[NW2 * pl + o - g.ld + 1];
            }
            rs[o] = (float)s;
        }
}

// (A p)_i in difference form: s_i p_i + sum_{j != i} a_ij (p_j - p_i).  The
// operator's rows nearly sum to zero, so the plain FP32 product loses the
// smooth part of A p to cancellation; the differences keep FP32 relative
// accuracy on every mode.
__device__ __forceinline__ float apply_row2d_diff(const float* __restrict__ A, const float* __restrict__ rs,
                                                  long long pl, int ld, const float* __restrict__ x, long long o) {
    const float xo = x[o];
    float s = rs[o] * xo;
    s += A[W2 * pl + o] * (x[o - 1] - xo);
    s += A[W2 * pl + o + 1] * (x[o + 1] - xo);
    s += A[S2 * pl + o] * (x[o - ld] - xo);
    s += A[S2 * pl + o + ld] * (x[o + ld] - xo);
    s += A[SW2 * pl + o] * (x[o - ld - 1] - xo);
    s += A[SW2 * pl + o + ld + 1] * (x[o + ld + 1] - xo);
    s += A[NW2 * pl + o] * (x[o + ld - 1] - xo);
    s += A[NW2 * pl + o - ld + 1] * (x[o - ld + 1] - xo);
    return s;
}

// q = A p (FP32 operator, difference form), alpha = rz / p.q; per-thread sums
// in FP32, block and grid sums in FP64.
__global__ void k_spmv_pq32(Grid2 g, const float* __restrict__ A, const float* __restrict__ rs, long long pl,
                            const float* __restrict__ p, float* __restrict__ q, double* partials, KState* st) {
    Acc32 acc;
    for (int j = blockIdx.x; j < g.n; j += gridDim.x) {
        const bool rj = j >= 1 && j <= g.n - 2;
        for (int i = threadIdx.x; i < g.ld; i += blockDim.x) {
            const long long k = (long long)j * g.ld + i;
            float v = 0.0f;
            if (rj && i >= 1 && i <= g.n - 2) v = apply_row2d_diff(A, rs, pl, g.ld, p, k);
            q[k] = v;
            acc.add(p[k] * v);
        }
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

// d += alpha p; r -= alpha q
__global__ void k_update_dr32(long long tot, float* __restrict__ d, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q, const KState* st) {
    const float alpha = (float)st->alpha;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        d[k] += alpha * p[k];
        r[k] -= alpha * q[k];
    }
}

// r.z and r.z_old in one pass; the last block forms the flexible-CG beta
__global__ void k_rz_beta32(long long tot, const float* __restrict__ r, const float* __restrict__ z,
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

__global__ void k_p_update32(long long tot, const float* __restrict__ z, float* __restrict__ p, const KState* st) {
    const float beta = (float)st->beta;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x)
        p[k] = z[k] + beta * p[k];
}

}  // namespace

bmg_status k_residual_to32(Ctx& c) {
    const Level& L = c.lev[0];
    k_residual_to32<<<c.red_blocks, kThreads, 0, c.stream>>>(Grid2{L.n, L.ld}, L.A64, L.plane, c.bvec, c.x, c.r32,
                                                              c.partials, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_row_sums32(Ctx& c) {
    const Level& L = c.lev[0];
    k_row_sums32<<<c.red_blocks, kThreads, 0, c.stream>>>(Grid2{L.n, L.ld}, L.A64, L.plane, c.rs32);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_add_correction(Ctx& c) {
    const Level& L = c.lev[0];
    k_add_correction<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.x, c.d32);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_rz_beta32(Ctx& c, const float* z, const float* zo) {
    const Level& L = c.lev[0];
    k_rz_beta32<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.r32, z, zo, c.partials, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_p_update32(Ctx& c, const float* z) {
    const Level& L = c.lev[0];
    k_p_update32<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, z, c.p32, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_spmv_pq32(Ctx& c) {
    const Level& L = c.lev[0];
    const double N = (double)(L.n - 2) * (L.n - 2);
    prof_begin(c, BMG_PROF_SPMV, 0);
    k_spmv_pq32<<<c.red_blocks, kThreads, 0, c.stream>>>(Grid2{L.n, L.ld}, L.A32, c.rs32, L.plane, c.p32, c.q32,
                                                          c.partials, c.st);
    prof_end(c, BMG_PROF_SPMV, 0, (c.ns + 2) * 4.0 * N);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_update_dr32(Ctx& c) {
    const Level& L = c.lev[0];
    const double N = (double)(L.n - 2) * (L.n - 2);
    prof_begin(c, BMG_PROF_UPDATE, 0);
    k_update_dr32<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.d32, c.r32, c.p32, c.q32, c.st);
    prof_end(c, BMG_PROF_UPDATE, 0, 6 * 4.0 * N);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_pack(Ctx& c, const double* src, double* dst) {
    const Level& L = c.lev[0];
    k_pack2d<<<dim3(cdiv(L.ld, 128), L.n), 128, 0, c.stream>>>(L.n, L.ld, src, dst);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_unpack(Ctx& c, const double* src, double* dst) {
    const Level& L = c.lev[0];
    k_unpack2d<<<dim3(cdiv(L.n, 128), L.n), 128, 0, c.stream>>>(L.n, L.ld, src, dst);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_residual(Ctx& c, const double* b, const double* x, double* r) {
    const Level& L = c.lev[0];
    k_residual64<<<c.red_blocks, kThreads, 0, c.stream>>>(Grid2{L.n, L.ld}, L.A64, L.plane, b, x, r, c.partials,
                                                           c.st);
    c.launches++;
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
    const double N = (double)(L.n - 2) * (L.n - 2);
    prof_begin(c, BMG_PROF_SPMV, 0);
    k_spmv_pq<<<c.red_blocks, kThreads, 0, c.stream>>>(Grid2{L.n, L.ld}, L.A64, L.plane, p, q, c.partials, c.st);
    prof_end(c, BMG_PROF_SPMV, 0, (c.ns + 2) * 8.0 * N);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status k_update_xr(Ctx& c) {
    const Level& L = c.lev[0];
    const double N = (double)(L.n - 2) * (L.n - 2);
    prof_begin(c, BMG_PROF_UPDATE, 0);
    k_update_xr<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, c.x, c.r, c.p, c.q, c.partials, c.st);
    prof_end(c, BMG_PROF_UPDATE, 0, 6 * 8.0 * N);
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
    k_p_update<<<c.red_blocks, kThreads, 0, c.stream>>>(L.plane, z, c.p, c.st);
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
