// vcycle3d.cu -- the V(1,1)-cycle on 3-D levels (27-point operators,
// 8-colour Gauss-Seidel with colour (i&1) + 2(j&1) + 4(k&1), forward colour
// order before the coarse correction and reverse after; residual;
// restriction P^T; prolongation with correction; exact solve on 3^3).
#include "common.cuh"
#include "grid3.cuh"

namespace bmg {
namespace {

template <typename T>
struct L3 {
    const T* A;
    int n, ld;
    long long pl;
    __device__ __forceinline__ long long idx(int i, int j, int k) const {
        return (long long)i + (long long)ld * (j + (long long)n * k);
    }
};

// sum over the 26 off-diagonal couplings of row (i,j,k) applied to x
template <typename T>
__device__ __forceinline__ T offdiag3(const L3<T>& L, const T* __restrict__ x, int i, int j, int k) {
    const long long o = L.idx(i, j, k);
    const long long sy = L.ld, sz = (long long)L.ld * L.n;
    T s = 0;
#pragma unroll
    for (int t = 0; t < 13; t++) {
        const long long d = off_x(t) + sy * off_y(t) + sz * off_z(t);
        s += L.A[(long long)t * L.pl + o] * x[o + d];          // a(d) at the node
        s += L.A[(long long)t * L.pl + o - d] * x[o - d];      // a(-d) stored at the node - d
    }
    return s;
}

template <typename T>
__global__ void k_gs_colour3d(L3<T> L, const T* __restrict__ f, T* __restrict__ x, int ci, int cj, int ck) {
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ci;
    const int j = 2 * blockIdx.y + cj, k = 2 * blockIdx.z + ck;
    if (i < 1 || j < 1 || k < 1 || i > L.n - 2 || j > L.n - 2 || k > L.n - 2) return;
    const long long o = L.idx(i, j, k);
    x[o] = (f[o] - offdiag3(L, x, i, j, k)) / L.A[13 * L.pl + o];
}

template <typename T>
__global__ void k_residual3d(L3<T> L, const T* __restrict__ f, const T* __restrict__ x, T* __restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > L.n - 2 || j > L.n - 2 || k > L.n - 2) return;
    const long long o = L.idx(i, j, k);
    r[o] = f[o] - (L.A[13 * L.pl + o] * x[o] + offdiag3(L, x, i, j, k));
}

// b_c(K) = sum over the 27 fine neighbours of 2K of P(f, K) r_f
template <typename T>
__global__ void k_restrict3d(int nf, int ldf, const T* __restrict__ r, const T* __restrict__ P, int nc, int ldc,
                             long long plc, T* __restrict__ bc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I < 1 || J < 1 || K < 1 || I > nc - 2 || J > nc - 2 || K > nc - 2) return;
    T s = 0;
    for (int o = 0; o < 27; o++) {
        const int fi = 2 * I + off_x(o), fj = 2 * J + off_y(o), fk = 2 * K + off_z(o);
        const T w = pweight3<T>(P, ldc, nc, plc, nf, fi, fj, fk, I, J, K);
        if (w != (T)0) s += w * r[(long long)fi + (long long)ldf * (fj + (long long)nf * fk)];
    }
    bc[(long long)I + (long long)ldc * (J + (long long)nc * K)] = s;
}

// x_f += P x_c
template <typename T>
__global__ void k_prolong3d(int nf, int ldf, T* __restrict__ x, const T* __restrict__ P, int nc, int ldc,
                            long long plc, const T* __restrict__ xc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > nf - 2 || j > nf - 2 || k > nf - 2) return;
    T v = 0;
    for (int s = 0; s < 8; s++) {
        const int KI = (i >> 1) + (s & 1), KJ = (j >> 1) + ((s >> 1) & 1), KK = (k >> 1) + (s >> 2);
        const T w = pweight3<T>(P, ldc, nc, plc, nf, i, j, k, KI, KJ, KK);
        if (w != (T)0) v += w * xc[(long long)KI + (long long)ldc * (KJ + (long long)nc * KK)];
    }
    x[(long long)i + (long long)ldf * (j + (long long)nf * k)] += v;
}

template <typename T>
__global__ void k_coarsest3d(L3<T> L, const double* __restrict__ A64, const T* __restrict__ b, T* __restrict__ x) {
    const long long o = L.idx(1, 1, 1);
    x[o] = (T)((double)b[o] / A64[13 * L.pl + o]);
}

inline dim3 g3(int ni, int nj, int nk) { return dim3(cdiv(ni, 64), nj, nk); }

inline double dofs3(const Ctx& c, int l) {
    const double m = c.lev[l].n - 2;
    return m * m * m;
}

template <typename T>
const T* A_of(const Level& L) { return (const T*)(sizeof(T) == 4 ? (const void*)L.A32 : (const void*)L.A64); }
template <typename T>
const T* P_of(const Level& L) { return (const T*)(sizeof(T) == 4 ? (const void*)L.P32 : (const void*)L.P64); }

}  // namespace

template <typename T>
bmg_status vcycle3d_impl(Ctx& c, const T* b0, T* x0, T* xout) {
    cudaStream_t s = c.stream;
    const int L = c.nlev;
    const double sz = sizeof(T);
    auto bl = [&](int l) { return l == 0 ? b0 : (const T*)c.lev[l].b; };
    auto xl = [&](int l) { return l == 0 ? x0 : (T*)c.lev[l].x; };
    for (int l = 0; l < L - 1; l++) {
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        L3<T> v{A_of<T>(F), F.n, F.ld, F.plane};
        BMG_CUDA(cudaMemsetAsync(xl(l), 0, sizeof(T) * F.plane, s));
        const int h = (F.n + 1) / 2;
        const double N = dofs3(c, l);
        for (int col = 0; col < 8; col++) {
            prof_begin(c, BMG_PROF_SMOOTH, l);
            k_gs_colour3d<T><<<g3(h, h, h), 64, 0, s>>>(v, bl(l), xl(l), col & 1, (col >> 1) & 1, col >> 2);
            prof_end(c, BMG_PROF_SMOOTH, l, (c.ns + 3) * sz * N / 8);
        }
        prof_begin(c, BMG_PROF_RESIDUAL, l);
        k_residual3d<T><<<g3(F.n, F.n, F.n), 64, 0, s>>>(v, bl(l), xl(l), (T*)F.r);
        prof_end(c, BMG_PROF_RESIDUAL, l, (c.ns + 3) * sz * N);
        prof_begin(c, BMG_PROF_RESTRICT, l);
        k_restrict3d<T><<<g3(K.n, K.n, K.n), 64, 0, s>>>(F.n, F.ld, (const T*)F.r, P_of<T>(F), K.n, K.ld, K.plane,
                                                        (T*)K.b);
        prof_end(c, BMG_PROF_RESTRICT, l, (1.0 + c.np / 8.0 + 0.125) * sz * N);
        c.launches += 10;
    }
    {
        const Level& C = c.lev[L - 1];
        L3<T> v{A_of<T>(C), C.n, C.ld, C.plane};
        BMG_CUDA(cudaMemsetAsync(xl(L - 1), 0, sizeof(T) * C.plane, s));
        k_coarsest3d<T><<<1, 1, 0, s>>>(v, C.A64, bl(L - 1), xl(L - 1));
        c.launches++;
    }
    for (int l = L - 2; l >= 0; l--) {
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        L3<T> v{A_of<T>(F), F.n, F.ld, F.plane};
        const double N = dofs3(c, l);
        prof_begin(c, BMG_PROF_PROLONG, l);
        k_prolong3d<T><<<g3(F.n, F.n, F.n), 64, 0, s>>>(F.n, F.ld, xl(l), P_of<T>(F), K.n, K.ld, K.plane, xl(l + 1));
        prof_end(c, BMG_PROF_PROLONG, l, (2.0 + c.np / 8.0 + 0.125) * sz * N);
        const int h = (F.n + 1) / 2;
        for (int col = 7; col >= 0; col--) {
            prof_begin(c, BMG_PROF_SMOOTH, l);
            k_gs_colour3d<T><<<g3(h, h, h), 64, 0, s>>>(v, bl(l), xl(l), col & 1, (col >> 1) & 1, col >> 2);
            prof_end(c, BMG_PROF_SMOOTH, l, (c.ns + 3) * sz * N / 8);
        }
        c.launches += 9;
    }
    (void)xout;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

template bmg_status vcycle3d_impl<double>(Ctx&, const double*, double*, double*);
template bmg_status vcycle3d_impl<float>(Ctx&, const float*, float*, float*);

}  // namespace bmg
