// vcycle.cu -- the V(1,1)-cycle of Sec. 2.2 ("Solution phase" step 3) on the
// structured hierarchy: multicolour Gauss-Seidel pre-smoothing (colours in
// forward order), residual, restriction R = P^T, recursion, exact solve on
// the 3-node grid, prolongation with correction, post-smoothing in reverse
// colour order.  Templated on the V-cycle arithmetic (double or float).
#include "common.cuh"

namespace bmg {
namespace {

template <typename T>
struct LV {          // level view handed to kernels
    const T* A;
    int n, ld;
    long long pl;
};

template <typename T>
__device__ __forceinline__ T offdiag_sum2(const T* __restrict__ A, long long pl, int ld, const T* __restrict__ x,
                                          int i, int j) {
    const long long o = (long long)j * ld + i;
    const T* W = A + W2 * pl;
    const T* S = A + S2 * pl;
    const T* SW = A + SW2 * pl;
    const T* NW = A + NW2 * pl;
    T s = W[o] * x[o - 1];
    s += W[o + 1] * x[o + 1];
    s += S[o] * x[o - ld];
    s += S[o + ld] * x[o + ld];
    s += SW[o] * x[o - ld - 1];
    s += SW[o + ld + 1] * x[o + ld + 1];
    s += NW[o] * x[o + ld - 1];
    s += NW[o - ld + 1] * x[o - ld + 1];
    return s;
}

// One colour of Gauss-Seidel: nodes (2u+ci, 2v+cj);
// x_i <- (f_i - sum_{j != i} a_ij x_j) / a_ii.
template <typename T>
__global__ void k_gs_colour2d(LV<T> L, const T* __restrict__ f, T* __restrict__ x, int ci, int cj) {
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ci;
    const int j = 2 * blockIdx.y + cj;
    if (i < 1 || i > L.n - 2 || j < 1 || j > L.n - 2) return;
    const long long o = (long long)j * L.ld + i;
    const T s = f[o] - offdiag_sum2(L.A, L.pl, L.ld, x, i, j);
    x[o] = s / L.A[o];
}

template <typename T>
__global__ void k_residual2d(LV<T> L, const T* __restrict__ f, const T* __restrict__ x, T* __restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < 1 || i > L.n - 2 || j < 1 || j > L.n - 2) return;
    const long long o = (long long)j * L.ld + i;
    r[o] = f[o] - (L.A[o] * x[o] + offdiag_sum2(L.A, L.pl, L.ld, x, i, j));
}

// b_c(I,J) = sum_i P(i,(I,J)) r_i over the 3x3 fine neighbourhood of (2I,2J).
template <typename T>
__global__ void k_restrict2d(int nf, int ldf, const T* __restrict__ r, const T* __restrict__ P, int nc, int ldc,
                             long long plc, T* __restrict__ bc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    if (I < 1 || I > nc - 2 || J < 1 || J > nc - 2) return;
    const long long oc = (long long)J * ldc + I;
    const long long of = (long long)(2 * J) * ldf + 2 * I;
    auto p = [&](int pp, int dI, int dJ) { return P[pp * plc + oc + (long long)dJ * ldc + dI]; };
    T s = r[of];
    s += p(PXR, -1, 0) * r[of - 1];
    s += p(PXL, 0, 0) * r[of + 1];
    s += p(PYN, 0, -1) * r[of - ldf];
    s += p(PYS, 0, 0) * r[of + ldf];
    s += p(PNE, -1, -1) * r[of - ldf - 1];
    s += p(PNW, 0, -1) * r[of - ldf + 1];
    s += p(PSE, -1, 0) * r[of + ldf - 1];
    s += p(PSW, 0, 0) * r[of + ldf + 1];
    bc[oc] = s;
}

// x_f += P x_c.
template <typename T>
__global__ void k_prolong2d(int nf, int ldf, T* __restrict__ x, const T* __restrict__ P, int ldc, long long plc,
                            const T* __restrict__ xc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < 1 || i > nf - 2 || j < 1 || j > nf - 2) return;
    const int I = i >> 1, J = j >> 1;
    const long long oc = (long long)J * ldc + I;
    const long long of = (long long)j * ldf + i;
    T v;
    if (!(i & 1) && !(j & 1)) {
        v = xc[oc];
    } else if ((i & 1) && !(j & 1)) {
        v = P[PXL * plc + oc] * xc[oc] + P[PXR * plc + oc] * xc[oc + 1];
    } else if (!(i & 1) && (j & 1)) {
        v = P[PYS * plc + oc] * xc[oc] + P[PYN * plc + oc] * xc[oc + ldc];
    } else {
        v = P[PSW * plc + oc] * xc[oc] + P[PSE * plc + oc] * xc[oc + 1] + P[PNW * plc + oc] * xc[oc + ldc] +
            P[PNE * plc + oc] * xc[oc + ldc + 1];
    }
    x[of] += v;
}

// 3x3 grid, one unknown: x = b / a, in FP64.
template <typename T>
__global__ void k_coarsest2d(LV<T> L, const double* __restrict__ A64, const T* __restrict__ b, T* __restrict__ x) {
    const long long o = (long long)L.ld + 1;
    x[o] = (T)((double)b[o] / A64[o]);
}

template <typename S, typename D>
__global__ void k_convert(long long count, const S* __restrict__ src, D* __restrict__ dst) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = (D)src[k];
}

inline dim3 rows(int ni, int nj) { return dim3(cdiv(ni, 128), nj); }

template <typename T>
const T* Aof(const Level& L);
template <>
const double* Aof<double>(const Level& L) { return L.A64; }
template <>
const float* Aof<float>(const Level& L) { return L.A32; }
template <typename T>
const T* Pof(const Level& L);
template <>
const double* Pof<double>(const Level& L) { return L.P64; }
template <>
const float* Pof<float>(const Level& L) { return L.P32; }

// Interior unknowns of a level (the unit of the algorithmic byte counts).
inline double dofs(const Ctx& c, int l) {
    const double m = c.lev[l].n - 2;
    return c.dim == 2 ? m * m : m * m * m;
}

template <typename T>
bmg_status vcycle2d_impl(Ctx& c, const T* b0, T* x0) {
    cudaStream_t s = c.stream;
    const int L = c.nlev;
    const double sz = sizeof(T);
    auto bl = [&](int l) { return l == 0 ? b0 : (const T*)c.lev[l].b; };
    auto xl = [&](int l) { return l == 0 ? x0 : (T*)c.lev[l].x; };
    for (int l = 0; l < L - 1; l++) {
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        LV<T> v{Aof<T>(F), F.n, F.ld, F.plane};
        BMG_CUDA(cudaMemsetAsync(xl(l), 0, sizeof(T) * F.plane, s));
        const dim3 gc(cdiv((F.n + 1) / 2, 128), (F.n + 1) / 2);
        const double N = dofs(c, l);
        for (int col = 0; col < 4; col++) {
            prof_begin(c, BMG_PROF_SMOOTH, l);
            k_gs_colour2d<T><<<gc, 128, 0, s>>>(v, bl(l), xl(l), col & 1, col >> 1);
            prof_end(c, BMG_PROF_SMOOTH, l, (c.ns + 3) * sz * N / 4);
        }
        prof_begin(c, BMG_PROF_RESIDUAL, l);
        k_residual2d<T><<<rows(F.n, F.n), 128, 0, s>>>(v, bl(l), xl(l), (T*)F.r);
        prof_end(c, BMG_PROF_RESIDUAL, l, (c.ns + 3) * sz * N);
        prof_begin(c, BMG_PROF_RESTRICT, l);
        k_restrict2d<T><<<rows(K.n, K.n), 128, 0, s>>>(F.n, F.ld, (const T*)F.r, Pof<T>(F), K.n, K.ld, K.plane,
                                                      (T*)K.b);
        prof_end(c, BMG_PROF_RESTRICT, l, (1.0 + c.np / 4.0 + 0.25) * sz * N);
        c.launches += 6;
    }
    {
        const Level& C = c.lev[L - 1];
        LV<T> v{Aof<T>(C), C.n, C.ld, C.plane};
        BMG_CUDA(cudaMemsetAsync(xl(L - 1), 0, sizeof(T) * C.plane, s));
        k_coarsest2d<T><<<1, 1, 0, s>>>(v, C.A64, bl(L - 1), xl(L - 1));
        c.launches++;
    }
    for (int l = L - 2; l >= 0; l--) {
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        LV<T> v{Aof<T>(F), F.n, F.ld, F.plane};
        const double N = dofs(c, l);
        prof_begin(c, BMG_PROF_PROLONG, l);
        k_prolong2d<T><<<rows(F.n, F.n), 128, 0, s>>>(F.n, F.ld, xl(l), Pof<T>(F), K.ld, K.plane, xl(l + 1));
        prof_end(c, BMG_PROF_PROLONG, l, (2.0 + c.np / 4.0 + 0.25) * sz * N);
        const dim3 gc(cdiv((F.n + 1) / 2, 128), (F.n + 1) / 2);
        for (int col = 3; col >= 0; col--) {
            prof_begin(c, BMG_PROF_SMOOTH, l);
            k_gs_colour2d<T><<<gc, 128, 0, s>>>(v, bl(l), xl(l), col & 1, col >> 1);
            prof_end(c, BMG_PROF_SMOOTH, l, (c.ns + 3) * sz * N / 4);
        }
        c.launches += 5;
    }
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// Streaming path: one down kernel and one up kernel per level pair above
// the tail, and one single-CTA kernel for the tail levels.
template <typename T>
bmg_status vcycle2d_fused(Ctx& c, void* z, bool ir = false, const float* zold = nullptr) {
    const double sz = sizeof(T);
    // levels t.. (n <= kTailMaxN) run in one single-CTA launch
    const int t = tail_first_level(c);
    for (int l = 0; l < t; l++) {
        const double N = dofs(c, l);
        const double szf = (l == 0 && !ir) ? 8.0 : sz;
        prof_begin(c, BMG_PROF_VDOWN, l);
        BMG_TRY(fused_down(c, l, ir));
        // restriction reads the four edge weights of each coarse node (the
        // odd-odd fine points carry no residual after the last colour)
        prof_end(c, BMG_PROF_VDOWN, l, N * (c.ns * sz + szf + sz + (c.np / 2) / 4.0 * sz + sz / 4));
    }
    BMG_TRY(tail_vcycle(c, t));
    for (int l = t - 1; l >= 0; l--) {
        const double N = dofs(c, l);
        const double szf = (l == 0 && !ir) ? 8.0 : sz;
        const double szo = (l == 0 && !ir) ? 8.0 : sz;
        prof_begin(c, BMG_PROF_VUP, l);
        BMG_TRY(fused_up(c, l, l == 0 ? z : c.lev[l].r, ir, zold));
        const double szz = (l == 0 && ir && zold) ? 4.0 : 0.0;   // z_old read for the fused beta
        prof_end(c, BMG_PROF_VUP, l, N * (c.ns * sz + szf + sz + c.np / 4.0 * sz + sz / 4 + szo + szz));
    }
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace

bmg_status demote_levels(Ctx& c) {
    if (c.opts.precision != BMG_PREC_FP32) return BMG_OK;
    for (int l = 0; l < c.nlev; l++) {
        Level& L = c.lev[l];
        k_convert<double, float><<<1216, 256, 0, c.stream>>>((long long)c.ns * L.plane, L.A64, L.A32);
        c.launches++;
        if (l < c.nlev - 1) {
            const Level& K = c.lev[l + 1];
            k_convert<double, float><<<1216, 256, 0, c.stream>>>((long long)c.np * K.plane, L.P64, L.P32);
            c.launches++;
        }
    }
    BMG_CUDA(cudaGetLastError());
    if (c.dim == 3) BMG_TRY(colour_blocks3d(c));
    return BMG_OK;
}

bool vcycle_forms_beta(const Ctx& c) { return c.dim == 2 && c.use_fused && c.nlev >= 2; }

bmg_status vcycle_f32(Ctx& c, float* z32, const float* zold) {
    if (c.opts.precision != BMG_PREC_FP32) return BMG_ERR_STATE;
    if (c.dim == 3) return vcycle3d_impl<float>(c, c.r32, z32, nullptr);
    if (c.use_fused && c.nlev >= 2) return vcycle2d_fused<float>(c, z32, true, zold);
    return vcycle2d_impl<float>(c, c.r32, z32);
}

bmg_status vcycle(Ctx& c, const double* r, double* z) {
    if (c.dim == 3) {
        if (c.opts.precision == BMG_PREC_FP64) return vcycle3d_impl<double>(c, r, z, nullptr);
        Level& F = c.lev[0];
        k_convert<double, float><<<1216, 256, 0, c.stream>>>(F.plane, r, (float*)F.b);
        BMG_TRY(vcycle3d_impl<float>(c, (const float*)F.b, (float*)F.x, nullptr));
        k_convert<float, double><<<1216, 256, 0, c.stream>>>(F.plane, (const float*)F.x, z);
        c.launches += 2;
        BMG_CUDA(cudaGetLastError());
        return BMG_OK;
    }
    if (c.use_fused && c.nlev >= 2) {
        if (r != c.r) return BMG_ERR_ARG;   // the level-0 tensor map streams c.r
        if (c.opts.precision == BMG_PREC_FP64) return vcycle2d_fused<double>(c, z);
        return vcycle2d_fused<float>(c, z);
    }
    if (c.opts.precision == BMG_PREC_FP64) return vcycle2d_impl<double>(c, r, z);
    Level& F = c.lev[0];
    k_convert<double, float><<<1216, 256, 0, c.stream>>>(F.plane, r, (float*)F.b);
    BMG_TRY(vcycle2d_impl<float>(c, (const float*)F.b, (float*)F.x));
    k_convert<float, double><<<1216, 256, 0, c.stream>>>(F.plane, (const float*)F.x, z);
    c.launches += 2;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
