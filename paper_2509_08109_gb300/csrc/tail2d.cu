// tail2d.cu -- the coarse end of the 2-D V(1,1)-cycle (Sec. 2.2, "Solution
// phase" step 3) in a single CTA.
//
// Below about 33 nodes per side a level holds a few thousand values, and the
// streaming kernels spend their time on launch and pipeline latency rather
// than on data.  This kernel runs every level from the first one with
// n <= kTailMaxN down to the 3-node grid and back up in one launch: it copies
// the operators and interpolation weights of those levels into shared memory
// (compact rows, row length n), then performs the same steps in the same
// order as the streaming kernels (zero guess, forward colours 0..3, residual,
// restriction of the five fine points per coarse node that carry a residual,
// exact coarsest solve in FP64, correction, reverse colours 3..0), with one
// block barrier between dependent phases, and writes the finished iterate of
// its first level back for the up kernel of the level above.
#include "common.cuh"

namespace bmg {
namespace {

constexpr int kTailThreads = 1024;

struct TailLevel {
    int n, ld;
    long long pl;       // plane stride of A (and of b, r) in global memory
    const void* A;      // 5 symmetric-half planes
    const void* P;      // interpolation from the next level: 8 planes on its grid
    int ldc;
    long long plc;
};

struct TailArgs {
    int nlev;                     // levels in the tail (the last one has 3 nodes)
    TailLevel lv[kMaxLevels];
    const void* b0;               // right-hand side of the first tail level
    void* x0;                     // finished iterate of the first tail level
    const double* a64c;           // FP64 centre entry of the coarsest operator
};

template <typename T>
__device__ __forceinline__ T tdiv(T s, T d) { return s / d; }
template <>
__device__ __forceinline__ float tdiv<float>(float s, float d) { return __fdividef(s, d); }

// shared-memory footprint (elements of T) of level l of the tail
__host__ __device__ inline long long tail_elems(const int* n, int nlev, int l) {
    const long long m2 = (long long)n[l] * n[l];
    const long long mc2 = l + 1 < nlev ? (long long)n[l + 1] * n[l + 1] : 0;
    return (NS2 + 3) * m2 + NP2 * mc2;
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_vtail2d(TailArgs a) {
    extern __shared__ unsigned char smem_raw[];
    T* base = (T*)(((uintptr_t)smem_raw + 15) & ~(uintptr_t)15);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int L = a.nlev;
    int ns[kMaxLevels];
    for (int l = 0; l < L; l++) ns[l] = a.lv[l].n;
    // per level: A (5 planes), b, x (pre-smoothed), r (residual, then the
    // finished iterate), P (8 planes on the next level's grid)
    T *sA[kMaxLevels], *sB[kMaxLevels], *sX[kMaxLevels], *sR[kMaxLevels], *sP[kMaxLevels];
    {
        T* q = base;
        for (int l = 0; l < L; l++) {
            const long long m2 = (long long)ns[l] * ns[l];
            sA[l] = q;
            sB[l] = sA[l] + NS2 * m2;
            sX[l] = sB[l] + m2;
            sR[l] = sX[l] + m2;
            sP[l] = sR[l] + m2;
            q += tail_elems(ns, L, l);
        }
    }
    // load operators and weights; zero the vectors; right-hand side of level 0
    for (int l = 0; l < L; l++) {
        const TailLevel& g = a.lv[l];
        const int m = g.n;
        const long long m2 = (long long)m * m;
        const T* Ag = (const T*)g.A;
        for (long long k = tid; k < NS2 * m2; k += nth) {
            const int p = (int)(k / m2);
            const int r = (int)(k - p * m2);
            const int j = r / m, i = r - j * m;
            sA[l][k] = Ag[p * g.pl + (long long)j * g.ld + i];
        }
        for (long long k = tid; k < 3 * m2; k += nth) sB[l][k] = (T)0;
        if (l + 1 < L) {
            const int mc = ns[l + 1];
            const long long mc2 = (long long)mc * mc;
            const T* Pg = (const T*)g.P;
            for (long long k = tid; k < NP2 * mc2; k += nth) {
                const int p = (int)(k / mc2);
                const int r = (int)(k - p * mc2);
                const int j = r / mc, i = r - j * mc;
                sP[l][k] = Pg[p * g.plc + (long long)j * g.ldc + i];
            }
        }
    }
    __syncthreads();
    {
        const TailLevel& g = a.lv[0];
        const T* bg = (const T*)a.b0;
        for (int k = tid; k < g.n * g.n; k += nth) {
            const int j = k / g.n, i = k - j * g.n;
            sB[0][k] = bg[(long long)j * g.ld + i];
        }
    }
    __syncthreads();

    // off-diagonal part of row (i, j) of the level with operator A (row
    // length m, plane stride m2) on iterate x, in the order of the streaming
    // kernels (W, E, S, N, SW, NE, NW, SE)
    auto offdiag = [&](const T* A, int m, int m2, const T* x, int i, int j) {
        const int o = j * m + i;
        T s = A[W2 * m2 + o] * x[o - 1];
        s += A[W2 * m2 + o + 1] * x[o + 1];
        s += A[S2 * m2 + o] * x[o - m];
        s += A[S2 * m2 + o + m] * x[o + m];
        s += A[SW2 * m2 + o] * x[o - m - 1];
        s += A[SW2 * m2 + o + m + 1] * x[o + m + 1];
        s += A[NW2 * m2 + o] * x[o + m - 1];
        s += A[NW2 * m2 + o - m + 1] * x[o - m + 1];
        return s;
    };
    // every interior node of colour c of level l
    auto colour = [&](const T* A, int m, T* x, const T* f, int c) {
        const int m2 = m * m;
        // colour c has i parity (c & 1) and j parity (c >> 1): first interior
        // index of that parity i0, j0, and ni x nj such nodes
        const int i0 = 1 + ((c & 1) ^ 1), j0 = 1 + (((c >> 1) & 1) ^ 1);
        const int ni = (m - i0) / 2, nj = (m - j0) / 2;
        for (int k = tid; k < ni * nj; k += nth) {
            const int jj = k / ni, ii = k - jj * ni;
            const int i = i0 + 2 * ii, j = j0 + 2 * jj;
            const int o = j * m + i;
            x[o] = tdiv<T>(f[o] - offdiag(A, m, m2, x, i, j), A[C2 * m2 + o]);
        }
    };

    // ---- down: pre-smooth, residual, restriction
    for (int l = 0; l + 1 < L; l++) {
        const int m = ns[l], mc = ns[l + 1];
        const int m2 = m * m, mc2 = mc * mc;
        const T* A = sA[l];
        T* x = sX[l];
        const T* f = sB[l];
        T* r = sR[l];
        for (int c = 0; c < 4; c++) {
            colour(A, m, x, f, c);
            __syncthreads();
        }
        // residual at the interior points of colours 0, 1, 2 (colour 3 was
        // solved last and has none)
        for (int k = tid; k < (m - 2) * (m - 2); k += nth) {
            const int j = 1 + k / (m - 2), i = 1 + k % (m - 2);
            const int o = j * m + i;
            r[o] = ((i & 1) && (j & 1)) ? (T)0 : f[o] - A[C2 * m2 + o] * x[o] - offdiag(A, m, m2, x, i, j);
        }
        __syncthreads();
        const T* P = sP[l];
        T* bc = sB[l + 1];
        for (int k = tid; k < (mc - 2) * (mc - 2); k += nth) {
            const int J = 1 + k / (mc - 2), I = 1 + k % (mc - 2);
            const int O = J * mc + I, o = 2 * J * m + 2 * I;
            T b = r[o];
            b += P[PXR * mc2 + O - 1] * r[o - 1];
            b += P[PXL * mc2 + O] * r[o + 1];
            b += P[PYN * mc2 + O - mc] * r[o - m];
            b += P[PYS * mc2 + O] * r[o + m];
            bc[O] = b;
        }
        __syncthreads();
    }
    // ---- coarsest: one unknown, exact in FP64
    if (tid == 0) {
        const int o = ns[L - 1] + 1;
        sR[L - 1][o] = (T)((double)sB[L - 1][o] / *a.a64c);
    }
    __syncthreads();
    // ---- up: correction x_pre + P x_c, reverse colours 3..0
    for (int l = L - 2; l >= 0; l--) {
        const int m = ns[l], mc = ns[l + 1];
        const int mc2 = mc * mc;
        const T* P = sP[l];
        const T* xc = sR[l + 1];
        const T* xpre = sX[l];
        T* x = sR[l];
        for (int k = tid; k < (m - 2) * (m - 2); k += nth) {
            const int j = 1 + k / (m - 2), i = 1 + k % (m - 2);
            const int o = j * m + i;
            const int I = i >> 1, J = j >> 1, O = J * mc + I;
            const T xp = xpre[o];
            T v;
            if (!(i & 1) && !(j & 1)) {
                v = xp + xc[O];
            } else if (!(j & 1)) {      // (2I+1, 2J)
                v = xp + P[PXL * mc2 + O] * xc[O] + P[PXR * mc2 + O] * xc[O + 1];
            } else if (!(i & 1)) {      // (2I, 2J+1)
                v = xp + P[PYS * mc2 + O] * xc[O] + P[PYN * mc2 + O] * xc[O + mc];
            } else {                    // (2I+1, 2J+1)
                v = xp + P[PSW * mc2 + O] * xc[O] + P[PSE * mc2 + O] * xc[O + 1] + P[PNW * mc2 + O] * xc[O + mc] +
                    P[PNE * mc2 + O] * xc[O + mc + 1];
            }
            x[o] = v;
        }
        __syncthreads();
        for (int c = 3; c >= 0; c--) {
            colour(sA[l], m, x, sB[l], c);
            __syncthreads();
        }
    }
    {
        const TailLevel& g = a.lv[0];
        T* xg = (T*)a.x0;
        for (int k = tid; k < (g.n - 2) * (g.n - 2); k += nth) {
            const int j = 1 + k / (g.n - 2), i = 1 + k % (g.n - 2);
            xg[(long long)j * g.ld + i] = sR[0][j * g.n + i];
        }
    }
}

}  // namespace

int tail_first_level(const Ctx& c) {
    int t = c.nlev - 1;
    while (t > 1 && c.lev[t - 1].n <= kTailMaxN) t--;
    return t;
}

size_t tail_smem_bytes(const Ctx& c, int t) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    int ns[kMaxLevels];
    const int L = c.nlev - t;
    for (int l = 0; l < L; l++) ns[l] = c.lev[t + l].n;
    long long e = 0;
    for (int l = 0; l < L; l++) e += tail_elems(ns, L, l);
    return 16 + (size_t)e * (f32 ? 4 : 8);
}

// Levels t .. nlev-1 in one launch: reads lev[t].b, writes lev[t].r.
bmg_status tail_vcycle(Ctx& c, int t) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    TailArgs a{};
    a.nlev = c.nlev - t;
    for (int l = 0; l < a.nlev; l++) {
        const Level& Lv = c.lev[t + l];
        TailLevel& g = a.lv[l];
        g.n = Lv.n;
        g.ld = Lv.ld;
        g.pl = Lv.plane;
        g.A = f32 ? (const void*)Lv.A32 : (const void*)Lv.A64;
        g.P = f32 ? (const void*)Lv.P32 : (const void*)Lv.P64;
        if (l + 1 < a.nlev) {
            g.ldc = c.lev[t + l + 1].ld;
            g.plc = c.lev[t + l + 1].plane;
        }
    }
    a.b0 = c.lev[t].b;
    a.x0 = c.lev[t].r;
    const Level& C = c.lev[c.nlev - 1];
    a.a64c = C.A64 + (long long)C2 * C.plane + C.ld + 1;
    const size_t smem = tail_smem_bytes(c, t);
    if (f32) {
        if (cudaFuncSetAttribute(k_vtail2d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return BMG_ERR_DEVICE;
        k_vtail2d<float><<<1, kTailThreads, smem, c.stream>>>(a);
    } else {
        if (cudaFuncSetAttribute(k_vtail2d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return BMG_ERR_DEVICE;
        k_vtail2d<double><<<1, kTailThreads, smem, c.stream>>>(a);
    }
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
