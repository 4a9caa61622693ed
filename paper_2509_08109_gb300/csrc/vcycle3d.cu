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

// Colour-blocked rows: node t of colour col (t runs i fastest over that
// colour's interior nodes) keeps its 27 full-row entries at
// cb[cb_offset(col) + e * count(col) + t], so a colour sweep reads them
// coalesced instead of at stride 2 from the symmetric-half planes.
__global__ void k_cblocks3d(Sten3<float> S, float* __restrict__ cb) {
    const int n = S.n;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > n - 2 || j > n - 2 || k > n - 2) return;
    const int col = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    const int ni = cb_side(n, i & 1), nj = cb_side(n, j & 1);
    // first interior index of parity p is 2 - p
    const long long t = (long long)((i - (2 - (i & 1))) >> 1) +
                        (long long)ni * (((j - (2 - (j & 1))) >> 1) + (long long)nj * ((k - (2 - (k & 1))) >> 1));
    const long long nc = cb_count(n, col);
    float* b = cb + cb_offset(n, col) + t;
    for (int e = 0; e < 27; e++) b[e * nc] = S.full(i, j, k, e);
}

// One colour of the FP32 smoother from the colour blocks: the same products
// summed in the same order as k_gs_colour3d (offset t, then its mirror).
__global__ void k_gs_colour3d_cb(const float* __restrict__ blk, long long nc, int ni, int nj, int i0, int j0,
                                 int k0, int n, int ld, const float* __restrict__ f, float* __restrict__ x) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int a = (int)(t % ni);
    const long long r = t / ni;
    const int b = (int)(r % nj), cz = (int)(r / nj);
    const int i = i0 + 2 * a, j = j0 + 2 * b, k = k0 + 2 * cz;
    const long long o = (long long)i + (long long)ld * (j + (long long)n * k);
    const long long sy = ld, sz = (long long)ld * n;
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < 13; e++) {
        const long long d = off_x(e) + sy * off_y(e) + sz * off_z(e);
        s += __ldcs(&blk[e * nc + t]) * x[o + d];
        s += __ldcs(&blk[(26 - e) * nc + t]) * x[o - d];
    }
    x[o] = (__ldcs(&f[o]) - s) / __ldcs(&blk[13 * nc + t]);
}

// Residual after the forward 8-colour sweep from a zero guess: a point's own
// update zeroed its residual while the neighbours of later colours were
// still zero, so r = - sum over the neighbours of a later colour of a x.
// The neighbour at offset d has colour col ^ m(d), m(d) the mask of the
// non-zero components of d; same order of terms as offdiag3.
template <typename T>
__global__ void k_residual3d_sweep(L3<T> L, const T* __restrict__ x, T* __restrict__ r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i < 1 || j < 1 || k < 1 || i > L.n - 2 || j > L.n - 2 || k > L.n - 2) return;
    const int col = (i & 1) | ((j & 1) << 1) | ((k & 1) << 2);
    const long long o = L.idx(i, j, k);
    const long long sy = L.ld, sz = (long long)L.ld * L.n;
    T s = 0;
#pragma unroll
    for (int t = 0; t < 13; t++) {
        const int m = (off_x(t) != 0) | ((off_y(t) != 0) << 1) | ((off_z(t) != 0) << 2);
        if ((col ^ m) > col) {
            const long long d = off_x(t) + sy * off_y(t) + sz * off_z(t);
            s += L.A[(long long)t * L.pl + o] * x[o + d];
            s += L.A[(long long)t * L.pl + o - d] * x[o - d];
        }
    }
    r[o] = -s;
}

// b_c(K) = sum over the 27 fine neighbours f = 2K + d of P(f, K) r_f, in the
// order of d.  For an interior coarse node every such f is an interior fine
// node; its weight to K sits at the coarse node owning f (K - 1 in each
// direction where d = -1), in the plane of f's parity mask m and of the
// corner K - owner.  All of that is fixed by d, so the loop unrolls to plain
// loads.
// ldv: row length of the coarse vector bc (ldc, that of the weight planes,
// unless the coarse level lives in another layout).
template <typename T>
__device__ __forceinline__ void restrict_node3d(int nf, int ldf, const T* __restrict__ r, const T* __restrict__ P,
                                                int nc, int ldc, long long plc, T* __restrict__ bc, int ldv, int I,
                                                int J, int K) {
    const long long oc = (long long)I + (long long)ldc * (J + (long long)nc * K);
    const long long of = 2LL * I + (long long)ldf * (2 * J + (long long)nf * 2 * K);
    T s = 0;
#pragma unroll
    for (int o = 0; o < 27; o++) {
        const int dx = off_x(o), dy = off_y(o), dz = off_z(o);
        const int m = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
        T w = (T)1;
        if (m) {
            const int sb = (dx < 0) | ((dy < 0) << 1) | ((dz < 0) << 2);
            const long long own = oc - (dx < 0) - (long long)ldc * ((dy < 0) + (long long)nc * (dz < 0));
            w = P[(long long)(kPBase(m) + compress3(sb, m)) * plc + own];
        }
        s += w * r[of + dx + (long long)ldf * (dy + (long long)nf * dz)];
    }
    bc[(long long)I + (long long)ldv * (J + (long long)nc * K)] = s;
}

template <typename T>
__global__ void k_restrict3d(int nf, int ldf, const T* __restrict__ r, const T* __restrict__ P, int nc, int ldc,
                             long long plc, T* __restrict__ bc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I < 1 || J < 1 || K < 1 || I > nc - 2 || J > nc - 2 || K > nc - 2) return;
    restrict_node3d<T>(nf, ldf, r, P, nc, ldc, plc, bc, ldc, I, J, K);
}

// x_f += sum over s subset of m of P(f, (I,J,K) + s) x_c((I,J,K) + s) for the
// eight fine points f = 2(I,J,K) + b (parity mask m = b) that coarse node
// (I,J,K) owns: one thread per coarse node, the 26 weights of its cell read
// once and contiguously across the warp.  Summation over s ascending, as the
// weights' own numbering.
// ldv: row length of the coarse vector xc (as in restrict_node3d).
template <typename T>
__device__ __forceinline__ void prolong_node3d(int nf, int ldf, T* __restrict__ x, const T* __restrict__ P, int nc,
                                               int ldc, long long plc, const T* __restrict__ xc, int ldv, int I,
                                               int J, int K) {
    const long long oc = (long long)I + (long long)ldc * (J + (long long)nc * K);
    const long long ov = (long long)I + (long long)ldv * (J + (long long)nc * K);
    const long long sy = ldv, sz = (long long)ldv * nc;
    T c8[8];
#pragma unroll
    for (int q = 0; q < 8; q++) c8[q] = xc[ov + (q & 1) + sy * ((q >> 1) & 1) + sz * (q >> 2)];
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const int fi = 2 * I + (b & 1), fj = 2 * J + ((b >> 1) & 1), fk = 2 * K + (b >> 2);
        if (fi < 1 || fj < 1 || fk < 1 || fi > nf - 2 || fj > nf - 2 || fk > nf - 2) continue;
        T v = 0;
        if (b == 0) {
            v = c8[0];
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++)
                if ((q & ~b) == 0) v += P[(long long)(kPBase(b) + compress3(q, b)) * plc + oc] * c8[q];
        }
        x[(long long)fi + (long long)ldf * (fj + (long long)nf * fk)] += v;
    }
}

template <typename T>
__global__ void k_prolong3d(int nf, int ldf, T* __restrict__ x, const T* __restrict__ P, int nc, int ldc,
                            long long plc, const T* __restrict__ xc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I > nc - 2 || J > nc - 2 || K > nc - 2) return;
    prolong_node3d<T>(nf, ldf, x, P, nc, ldc, plc, xc, ldc, I, J, K);
}

template <typename T>
__global__ void k_coarsest3d(L3<T> L, const double* __restrict__ A64, const T* __restrict__ b, T* __restrict__ x) {
    const long long o = L.idx(1, 1, 1);
    x[o] = (T)((double)b[o] / A64[13 * L.pl + o]);
}

inline dim3 g3(int ni, int nj, int nk) { return dim3(cdiv(ni, 64), nj, nk); }

// ---------------------------------------------------------------- tail
// The coarse end of the 3-D V-cycle (levels with n <= tail3_max_n down to the
// 3^3 grid and back) in one launch of one CTA: the same per-node steps as the
// kernels above, each phase a block-strided loop followed by a block barrier.
// Each phase waits on its loads, so the tail's time is about its number of
// phases times the latency of the memory it reads.  In FP32 the tail starts
// at 9^3 and all its levels (9^3, 5^3, 3^3: about 76 KB in a compact layout,
// n in place of the padded row length) live in shared memory for the launch:
// operators and weights copied from their arrays at the start, the first
// level's right-hand side copied in and its iterate copied out; the 17^3
// level runs the half-sweep kernels instead.  In FP64 the tail starts at
// 17^3 (its operator alone is 550 KB) and works on the levels' arrays in
// global memory (L2-resident).  Measured on the 257^3 shell (FP32
// refinement solve): 1.052 s with a 17^3 tail in global memory, 1.045 s with
// its lower levels staged.
constexpr int kTail3Threads = 1024;
template <typename T>
constexpr int tail3_max_n() { return sizeof(T) == 4 ? 9 : 17; }   // first tail level: n <= this
constexpr int kTail3Lev = 4;     // levels of a tail: 17, 9, 5, 3 at most

template <typename T>
struct Tail3Level {
    L3<T> A;
    const T* P;        // interpolation from the next level (its grid: ldc, plane plc)
    int ldc;
    long long plc;
    const T* b;
    T* x;
    T* r;
};

template <typename T>
struct Tail3Args {
    int nlev;
    Tail3Level<T> lv[kTail3Lev];
    const double* a64c;    // FP64 centre entry of the coarsest operator at (1,1,1)
};

// Elements of shared memory for the staged levels (all of them, FP32 only).
template <typename T>
__host__ __device__ constexpr bool tail3_stages() { return sizeof(T) == 4; }
inline size_t tail3_smem_elems(const int* ns, int nlev) {
    size_t e = 0;
    for (int q = 0; q < nlev; q++) {
        const size_t n3 = (size_t)ns[q] * ns[q] * ns[q];
        e += (NS3 + 3) * n3;
        if (q + 1 < nlev) e += (size_t)NP3 * ns[q + 1] * ns[q + 1] * ns[q + 1];
    }
    return e;
}

template <typename T>
__global__ void __launch_bounds__(kTail3Threads) k_vtail3d(Tail3Args<T> a) {
    extern __shared__ __align__(16) unsigned char t3_raw[];
    __shared__ Tail3Level<T> lv[kTail3Lev];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int L = a.nlev;
    if (tid == 0) {
        T* sp = reinterpret_cast<T*>(t3_raw);
        for (int q = 0; q < L; q++) {
            lv[q] = a.lv[q];
            if (tail3_stages<T>()) {
                const int n = a.lv[q].A.n;
                const long long n3 = (long long)n * n * n;
                lv[q].A = L3<T>{sp, n, n, n3};
                sp += NS3 * n3;
                if (q + 1 < L) {
                    const int nc = a.lv[q + 1].A.n;
                    lv[q].P = sp;
                    lv[q].ldc = nc;
                    lv[q].plc = (long long)nc * nc * nc;
                    sp += NP3 * lv[q].plc;
                }
                lv[q].b = sp;
                lv[q].x = sp + n3;
                lv[q].r = sp + 2 * n3;
                sp += 3 * n3;
            }
        }
    }
    __syncthreads();
    if (tail3_stages<T>()) {
        // operators (NS3 planes) and weights (NP3 planes on the next grid),
        // from the padded layout into the compact one; the first level's
        // right-hand side
        {
            const Tail3Level<T>& g = a.lv[0];
            const int n = g.A.n, n3 = n * n * n;
            T* db = const_cast<T*>(lv[0].b);
            for (int u = tid; u < n3; u += nth) {
                const int i = u % n, j = (u / n) % n, k = u / (n * n);
                db[u] = g.b[g.A.idx(i, j, k)];
            }
        }
        for (int q = 0; q < L; q++) {
            const Tail3Level<T>& g = a.lv[q];
            const int n = g.A.n;
            const int n3 = n * n * n;
            T* dA = const_cast<T*>(lv[q].A.A);
            for (int e = tid; e < NS3 * n3; e += nth) {
                const int t = e / n3, u = e - t * n3;
                const int i = u % n, j = (u / n) % n, k = u / (n * n);
                dA[e] = g.A.A[t * g.A.pl + g.A.idx(i, j, k)];
            }
            if (q + 1 < L) {
                const int nc = a.lv[q + 1].A.n, nc3 = nc * nc * nc;
                T* dP = const_cast<T*>(lv[q].P);
                for (int e = tid; e < NP3 * nc3; e += nth) {
                    const int t = e / nc3, u = e - t * nc3;
                    const int i = u % nc, j = (u / nc) % nc, k = u / (nc * nc);
                    dP[e] = g.P[t * g.plc + (long long)i + (long long)g.ldc * (j + (long long)nc * k)];
                }
            }
        }
        __syncthreads();
    }
    auto colour = [&](const Tail3Level<T>& v, int col) {
        const int n = v.A.n;
        const int pi = col & 1, pj = (col >> 1) & 1, pk = col >> 2;
        const int ni = cb_side(n, pi), nj = cb_side(n, pj), nk = cb_side(n, pk);
        for (int t = tid; t < ni * nj * nk; t += nth) {
            const int i = 2 - pi + 2 * (t % ni), j = 2 - pj + 2 * ((t / ni) % nj), k = 2 - pk + 2 * (t / (ni * nj));
            const long long o = v.A.idx(i, j, k);
            v.x[o] = (v.b[o] - offdiag3(v.A, v.x, i, j, k)) / v.A.A[13 * v.A.pl + o];
        }
    };
    for (int l = 0; l + 1 < L; l++) {
        const Tail3Level<T>& v = lv[l];
        const Tail3Level<T>& w = lv[l + 1];
        const int n = v.A.n, m = n - 2;
        for (long long q = tid; q < (long long)v.A.ld * n * n; q += nth) v.x[q] = (T)0;
        __syncthreads();
        for (int col = 0; col < 8; col++) {
            colour(v, col);
            __syncthreads();
        }
        for (int q = tid; q < m * m * m; q += nth) {
            const int i = 1 + q % m, j = 1 + (q / m) % m, k = 1 + q / (m * m);
            const long long o = v.A.idx(i, j, k);
            v.r[o] = v.b[o] - (v.A.A[13 * v.A.pl + o] * v.x[o] + offdiag3(v.A, v.x, i, j, k));
        }
        __syncthreads();
        const int nc = w.A.n, mc = nc - 2;
        for (int q = tid; q < mc * mc * mc; q += nth) {
            const int I = 1 + q % mc, J = 1 + (q / mc) % mc, K = 1 + q / (mc * mc);
            restrict_node3d<T>(n, v.A.ld, v.r, v.P, nc, v.ldc, v.plc, (T*)w.b, w.A.ld, I, J, K);
        }
        __syncthreads();
    }
    {   // coarsest: one unknown, exact in FP64; the rest of its iterate is zero
        const Tail3Level<T>& v = lv[L - 1];
        const int n = v.A.n;
        for (long long q = tid; q < (long long)v.A.ld * n * n; q += nth) v.x[q] = (T)0;
        __syncthreads();
        if (tid == 0) {
            const long long o = v.A.idx(1, 1, 1);
            v.x[o] = (T)((double)v.b[o] / *a.a64c);
        }
        __syncthreads();
    }
    for (int l = L - 2; l >= 0; l--) {
        const Tail3Level<T>& v = lv[l];
        const Tail3Level<T>& w = lv[l + 1];
        const int n = v.A.n, nc = w.A.n, mc = nc - 1;
        for (int q = tid; q < mc * mc * mc; q += nth) {
            const int I = q % mc, J = (q / mc) % mc, K = q / (mc * mc);
            prolong_node3d<T>(n, v.A.ld, v.x, v.P, nc, v.ldc, v.plc, w.x, w.A.ld, I, J, K);
        }
        __syncthreads();
        for (int col = 7; col >= 0; col--) {
            colour(v, col);
            __syncthreads();
        }
    }
    if (tail3_stages<T>()) {   // the first level's iterate back to its array
        const Tail3Level<T>& g = a.lv[0];
        const int n = g.A.n, n3 = n * n * n;
        for (int u = tid; u < n3; u += nth) {
            const int i = u % n, j = (u / n) % n, k = u / (n * n);
            g.x[g.A.idx(i, j, k)] = lv[0].x[u];
        }
    }
}

// ---------------------------------------------------------------- half sweeps
// The 8-colour order visits all colours of the even k-planes (0..3) before
// those of the odd planes (4..7), and the only couplings between planes are
// the 18 z-couplings of a point, which all join planes of opposite parity.
// So each half of a sweep is, plane by plane, an independent 4-colour sweep
// of the plane with the couplings to its two neighbouring planes (whose
// values do not change during that half) taken as they stand:
//   forward (pre-smoothing, zero guess): the even planes first, whose odd
//     neighbours are still zero (in-plane couplings only), then the odd
//     planes against the finished even planes;
//   reverse (post-smoothing): the odd planes against the corrected even
//     planes, then the even planes against the finished odd planes.
// k_hsweep3d runs one such half for every plane of one parity at once: a
// CTA per (tile, plane) holds the plane's iterate over its tile and a halo
// in shared memory, with the two neighbouring planes' iterates beside it.
// Within a plane, colour (i&1) + 2(j&1) of the last phase depends on the
// first through a chain of at most three column steps and one row step, so
// a tile of kHsTI x TJ owned points computes (kHsTI + 6) x (TJ + 2) points
// and neighbouring tiles recompute each other's halo.  Each point's update
// is the per-colour kernels' update: the same 26 products summed in the
// same order (offset t, then its mirror), the same division.
//
// Threads.  Lane p of a warp owns the column pair (ib + 2p, ib + 2p + 1) of
// a row; the two points of a pair have consecutive colours, so a thread
// loads both points' stencils with 2-wide vector loads when it updates the
// first and keeps the second one's in registers for the next phase.  The
// iterate rows in shared memory keep even and odd columns apart, so the
// neighbour reads of a phase (stride 2 in the natural layout) hit distinct
// banks.
//
// Inputs and outputs are separate arrays (xout is never read), so a CTA
// never sees a neighbour's finished values in place of the initial ones.
constexpr int kHsPairs = 32;                 // column pairs per row: one per lane
constexpr int kHsWarps = 8;
constexpr int kHsThreads = 32 * kHsWarps;
constexpr int kHsTI = 2 * kHsPairs - 6;      // owned columns of a tile (58)
constexpr int kHsHalf = kHsPairs + 2;        // one parity's columns in a shared row
constexpr int kHsCols = 2 * kHsHalf;         // shared row: columns ib-2 .. ib+65
__host__ __device__ constexpr int hs_tj(int rows) { return 2 * kHsWarps * rows - 2; }   // owned rows
__host__ __device__ constexpr int hs_srows(int rows) { return hs_tj(rows) + 4; }        // shared rows
// Rows per warp and phase: one (58 x 14 owned points, 80 registers, 3 CTAs
// per SM) measured faster than two (58 x 30, 128 registers, 2 CTAs per SM):
// 0.66 against 0.76 ms per 257^3 V-cycle's finest-level half sweeps.
template <typename T>
constexpr int hs_rows() { return 1; }
template <typename T>
constexpr size_t hs_smem() { return sizeof(T) * 3 * (size_t)hs_srows(hs_rows<T>()) * kHsCols; }

template <typename T>
struct HS3Args {
    const T* A;          // symmetric-half planes (NS3)
    int n, ld;
    long long pl;
    const T* f;          // right-hand side
    const T* xcur;       // initial iterate of the swept planes (mode 2)
    const T* xz;         // iterate of the neighbouring planes (modes 1, 2)
    T* xout;             // swept planes' result (owned points)
    int parity;          // planes k with k & 1 == parity
};

template <typename T>
struct V2 {
    T x, y;
};
template <typename T>
__device__ __forceinline__ V2<T> ld2(const T* p) {
    if constexpr (sizeof(T) == 4) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return {v.x, v.y};
    } else {
        const double2 v = __ldg(reinterpret_cast<const double2*>(p));
        return {v.x, v.y};
    }
}

// One pair's stencil: the 14 stored planes at both points (own) and, for
// each stored offset d, the mirror a(q, q - d) stored at q - d.
template <typename T, int MODE>
struct HsPair {
    T own0[NS3], own1[NS3];   // first (even column) / second point
    T mir0[13], mir1[13];
    T f0, f1;
    __device__ __forceinline__ void load(const HS3Args<T>& a, long long o0, bool first_ok) {
        const long long sz = (long long)a.ld * a.n;
#pragma unroll
        for (int t = 0; t < NS3; t++) {
            if (MODE == 0 && t < 9) continue;   // z-couplings: the odd planes are still zero
            const V2<T> v = ld2(a.A + t * a.pl + o0);
            own0[t] = v.x;
            own1[t] = v.y;
        }
#pragma unroll
        for (int t = 0; t < 13; t++) {
            if (MODE == 0 && t < 9) continue;
            const int dx = off_x(t), dy = off_y(t), dz = off_z(t);
            const long long m = o0 - (long long)dy * a.ld - dz * sz;   // node (i, j - dy, k - dz)
            const T* b = a.A + t * a.pl + m;
            const V2<T> v = ld2(b);
            if (dx == 0) {
                mir0[t] = v.x;
                mir1[t] = v.y;
            } else if (dx < 0) {             // mirrors at columns i + 1 and i + 2
                mir0[t] = v.y;
                mir1[t] = __ldg(b + 2);
            } else {                         // mirrors at columns i - 1 and i
                mir0[t] = first_ok ? __ldg(b - 1) : (T)0;
                mir1[t] = v.x;
            }
        }
        const V2<T> v = ld2(a.f + o0);
        f0 = v.x;
        f1 = v.y;
    }
};

// Gauss-Seidel update of one point from its stencil and the shared
// iterates.  ODD: the point is the pair's second (odd) column.  s: index of
// the point's row in the shared arrays (row start), p: the pair.
template <typename T, int MODE, bool ODD>
__device__ __forceinline__ T hs_update(const T* own, const T* mir, T f, const T* xc, const T* xb, const T* xa,
                                       int rs, int p) {
    // shared index of the neighbour at column offset dx, row offset dy
    auto at = [&](int dx, int dy) {
        const int c = ODD ? (dx == 0 ? kHsHalf + p + 1 : (dx < 0 ? p + 1 : p + 2))
                          : (dx == 0 ? p + 1 : (dx < 0 ? kHsHalf + p : kHsHalf + p + 1));
        return rs + dy * kHsCols + c;
    };
    T s = 0;
#pragma unroll
    for (int t = 0; t < 13; t++) {
        if (MODE == 0 && t < 9) continue;
        const int dx = off_x(t), dy = off_y(t), dz = off_z(t);
        const T* xp = dz < 0 ? xb : xc;   // plane of q + d
        const T* xm = dz < 0 ? xa : xc;   // plane of q - d
        s += own[t] * xp[at(dx, dy)];
        s += mir[t] * xm[at(-dx, -dy)];
    }
    return (f - s) / own[13];
}

// MODE 0: zero initial iterate, no z-couplings (forward sweep of the even
// planes); MODE 1: zero initial iterate, z-couplings to xz (forward sweep of
// the odd planes); MODE 2: initial iterate xcur, z-couplings to xz (reverse
// sweeps).  FWD: colours of the plane ascending, else descending.
template <typename T, int MODE, bool FWD>
__global__ void __launch_bounds__(kHsThreads) k_hsweep3d(HS3Args<T> a) {
    constexpr int ROWS = hs_rows<T>();
    constexpr int TJ = hs_tj(ROWS);
    constexpr int SR = hs_srows(ROWS);
    constexpr int PLANE = SR * kHsCols;
    extern __shared__ __align__(16) unsigned char hs_raw[];
    T* xc = reinterpret_cast<T*>(hs_raw);   // swept plane k
    T* xb = xc + PLANE;                      // plane k - 1
    T* xa = xb + PLANE;                      // plane k + 1
    const int n = a.n, ld = a.ld;
    const long long sz = (long long)ld * n;
    const int k = 2 - a.parity + 2 * (int)blockIdx.z;
    const int i0 = 1 + (int)blockIdx.x * kHsTI, j0 = 1 + (int)blockIdx.y * TJ;
    const int ib = i0 - 3;                   // first computed column (even)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // shared position (lr, lc) holds node (ib - 2 + lc, j0 - 2 + lr)
    for (int q = tid; q < PLANE; q += kHsThreads) {
        const int lr = q / kHsCols, lc = q - lr * kHsCols;
        const int i = ib - 2 + lc, j = j0 - 2 + lr;
        const bool in = i >= 1 && i <= n - 2 && j >= 1 && j <= n - 2;
        const int s = lr * kHsCols + (lc & 1) * kHsHalf + (lc >> 1);
        const long long o = (long long)i + (long long)ld * j + sz * k;
        xc[s] = (MODE == 2 && in) ? a.xcur[o] : (T)0;
        if (MODE >= 1) {
            xb[s] = (in && k >= 2) ? a.xz[o - sz] : (T)0;
            xa[s] = (in && k <= n - 3) ? a.xz[o + sz] : (T)0;
        }
    }
    __syncthreads();
    const int p = lane;
    const int i = ib + 2 * p;                // the pair's first column
    HsPair<T, MODE> hold[ROWS];
    bool ok0[ROWS], ok1[ROWS];
    // one row parity: PH = 0 loads and updates the pair's earlier colour,
    // PH = 1 updates the later one from the registers
    auto phase = [&](int jpar, bool second) {
#pragma unroll
        for (int r = 0; r < ROWS; r++) {
            const int lrow = 2 * (warp + kHsWarps * r) + jpar;   // region row, j = j0 - 1 + lrow
            const int j = j0 - 1 + lrow;
            const int rs = (lrow + 1) * kHsCols;
            const bool pv = j >= 1 && j <= n - 2 && i >= 0 && i <= n - 2;
            if (!second) {
                ok0[r] = pv && i >= 1;
                ok1[r] = pv && i + 1 <= n - 2;
                if (pv) hold[r].load(a, (long long)i + (long long)ld * j + sz * k, ok0[r]);
            }
            // FWD: even column first; reverse: odd column first
            const bool do_odd = FWD ? second : !second;
            if (do_odd) {
                if (ok1[r]) xc[rs + kHsHalf + p + 1] =
                    hs_update<T, MODE, true>(hold[r].own1, hold[r].mir1, hold[r].f1, xc, xb, xa, rs, p);
            } else {
                if (ok0[r]) xc[rs + p + 1] =
                    hs_update<T, MODE, false>(hold[r].own0, hold[r].mir0, hold[r].f0, xc, xb, xa, rs, p);
            }
        }
        __syncthreads();
    };
    if (FWD) {
        phase(0, false);
        phase(0, true);
        phase(1, false);
        phase(1, true);
    } else {
        phase(1, false);
        phase(1, true);
        phase(0, false);
        phase(0, true);
    }
    for (int q = tid; q < kHsTI * TJ; q += kHsThreads) {
        const int lj = q / kHsTI, li = q - lj * kHsTI;
        const int ii = i0 + li, jj = j0 + lj;
        if (ii > n - 2 || jj > n - 2) continue;
        const int lc = ii - ib + 2, lr = jj - j0 + 2;
        a.xout[(long long)ii + (long long)ld * jj + sz * k] = xc[lr * kHsCols + (lc & 1) * kHsHalf + (lc >> 1)];
    }
}

// x_out = x_in + P x_c at every interior fine point (out of place; the
// same sum as prolong_node3d).
template <typename T>
__global__ void k_prolong3d_to(int nf, int ldf, const T* __restrict__ xin, T* __restrict__ xout,
                               const T* __restrict__ P, int nc, int ldc, long long plc, const T* __restrict__ xc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y, K = blockIdx.z;
    if (I > nc - 2 || J > nc - 2 || K > nc - 2) return;
    const long long oc = (long long)I + (long long)ldc * (J + (long long)nc * K);
    const long long sy = ldc, szc = (long long)ldc * nc;
    T c8[8];
#pragma unroll
    for (int q = 0; q < 8; q++) c8[q] = xc[oc + (q & 1) + sy * ((q >> 1) & 1) + szc * (q >> 2)];
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const int fi = 2 * I + (b & 1), fj = 2 * J + ((b >> 1) & 1), fk = 2 * K + (b >> 2);
        if (fi < 1 || fj < 1 || fk < 1 || fi > nf - 2 || fj > nf - 2 || fk > nf - 2) continue;
        T v = 0;
        if (b == 0) {
            v = c8[0];
        } else {
#pragma unroll
            for (int q = 0; q < 8; q++)
                if ((q & ~b) == 0) v += P[(long long)(kPBase(b) + compress3(q, b)) * plc + oc] * c8[q];
        }
        const long long o = (long long)fi + (long long)ldf * (fj + (long long)nf * fk);
        xout[o] = xin[o] + v;
    }
}

inline double dofs3(const Ctx& c, int l) {
    const double m = c.lev[l].n - 2;
    return m * m * m;
}

template <typename T>
const T* A_of(const Level& L) { return (const T*)(sizeof(T) == 4 ? (const void*)L.A32 : (const void*)L.A64); }
template <typename T>
const T* P_of(const Level& L) { return (const T*)(sizeof(T) == 4 ? (const void*)L.P32 : (const void*)L.P64); }

// one colour of the smoother on level l: colour blocks when the level has
// them (FP32), otherwise the symmetric-half planes
template <typename T>
bmg_status colour_sweep(Ctx& c, int l, const L3<T>& v, const T* f, T* x, int col, int h) {
    const Level& F = c.lev[l];
    const double N = dofs3(c, l);
    prof_begin(c, BMG_PROF_SMOOTH, l);
    if constexpr (sizeof(T) == 4) {
        if (F.cb) {
            const int pi = col & 1, pj = (col >> 1) & 1, pk = col >> 2;
            const long long nc = cb_count(F.n, col);
            const unsigned blocks = (unsigned)((nc + 255) / 256);
            k_gs_colour3d_cb<<<blocks, 256, 0, c.stream>>>(F.cb + cb_offset(F.n, col), nc, cb_side(F.n, pi),
                                                           cb_side(F.n, pj), 2 - pi, 2 - pj, 2 - pk, F.n, F.ld, f, x);
            c.launches++;
            prof_end(c, BMG_PROF_SMOOTH, l, (27.0 + 3.0) * sizeof(T) * N / 8);
            return BMG_OK;
        }
    }
    k_gs_colour3d<T><<<g3(h, h, h), 64, 0, c.stream>>>(v, f, x, col & 1, (col >> 1) & 1, col >> 2);
    c.launches++;
    prof_end(c, BMG_PROF_SMOOTH, l, (c.ns + 3) * sizeof(T) * N / 8);
    return BMG_OK;
}

}  // namespace

bmg_status colour_blocks3d(Ctx& c) {
    if (c.opts.precision != BMG_PREC_FP32 || c.dim != 3) return BMG_OK;
    for (int l = 0; l + 1 < c.nlev; l++) {
        const Level& L = c.lev[l];
        if (!L.cb) continue;
        k_cblocks3d<<<g3(L.n, L.n, L.n), 64, 0, c.stream>>>(Sten3<float>{L.A32, L.n, L.ld, L.plane}, L.cb);
        c.launches++;
    }
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

// One half sweep on level l (all planes of one parity); bytes for the
// profiler: per point of the parity its stored planes (in-plane ones only in
// mode 0), the mirrored z-planes of the plane above, the neighbouring
// planes' iterate, the right-hand side, the output and (mode 2) the input.
template <typename T, int MODE, bool FWD>
bmg_status hsweep3d(Ctx& c, int l, const T* f, const T* xcur, const T* xz, T* xout, int parity) {
    const Level& F = c.lev[l];
    constexpr int TJ = hs_tj(hs_rows<T>());
    const int planes = parity ? (F.n - 1) / 2 : (F.n - 3) / 2;
    if (planes < 1) return BMG_OK;
    HS3Args<T> a{A_of<T>(F), F.n, F.ld, F.plane, f, xcur, xz, xout, parity};
    const dim3 grid(cdiv(F.n - 2, kHsTI), cdiv(F.n - 2, TJ), planes);
    prof_begin(c, BMG_PROF_SMOOTH, l);
    k_hsweep3d<T, MODE, FWD><<<grid, kHsThreads, hs_smem<T>(), c.stream>>>(a);
    c.launches++;
    const double per = MODE == 0 ? 5.0 + 2.0 : (MODE == 1 ? 14.0 + 9.0 + 2.0 + 2.0 : 14.0 + 9.0 + 2.0 + 3.0);
    prof_end(c, BMG_PROF_SMOOTH, l, per * sizeof(T) * dofs3(c, l) / 2);
    return BMG_OK;
}

// The half-sweep legs of a level (FP32 only: see use_hs3).
template <typename T>
bool hs3_on(const Ctx& c) { return sizeof(T) == 4 && c.use_hs3; }

template <typename T>
bmg_status hs3_down(Ctx& c, int l, const T* f, T* x) {
    if constexpr (sizeof(T) == 4) {
        // even planes (their odd neighbours still zero), then odd planes
        BMG_TRY((hsweep3d<T, 0, true>(c, l, f, nullptr, nullptr, x, 0)));
        return hsweep3d<T, 1, true>(c, l, f, nullptr, x, x, 1);
    } else {
        return BMG_ERR_STATE;
    }
}

template <typename T>
bmg_status hs3_up(Ctx& c, int l, const T* f, T* x, const T* xc) {
    if constexpr (sizeof(T) == 4) {
        // x + P x_c into the residual buffer (free until the next down leg),
        // then the odd planes against the corrected even planes, then the
        // even planes against the finished odd planes
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        T* xcor = (T*)F.r;
        prof_begin(c, BMG_PROF_PROLONG, l);
        k_prolong3d_to<T><<<g3(K.n - 1, K.n - 1, K.n - 1), 64, 0, c.stream>>>(F.n, F.ld, x, xcor, P_of<T>(F), K.n,
                                                                               K.ld, K.plane, xc);
        prof_end(c, BMG_PROF_PROLONG, l, (2.0 + c.np / 8.0 + 0.125) * sizeof(T) * dofs3(c, l));
        c.launches += 1;
        BMG_TRY((hsweep3d<T, 2, false>(c, l, f, xcor, xcor, x, 1)));
        return hsweep3d<T, 2, false>(c, l, f, xcor, x, x, 0);
    } else {
        return BMG_ERR_STATE;
    }
}

template <typename T>
bmg_status vcycle3d_impl(Ctx& c, const T* b0, T* x0, T* xout) {
    cudaStream_t s = c.stream;
    const int L = c.nlev;
    const double sz = sizeof(T);
    auto bl = [&](int l) { return l == 0 ? b0 : (const T*)c.lev[l].b; };
    auto xl = [&](int l) { return l == 0 ? x0 : (T*)c.lev[l].x; };
    // levels t .. L-1 (n <= tail3_max_n) run in the single-CTA tail
    int t = L - 1;
    while (t > 0 && c.lev[t - 1].n <= tail3_max_n<T>()) t--;
    for (int l = 0; l < t; l++) {
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        L3<T> v{A_of<T>(F), F.n, F.ld, F.plane};
        BMG_CUDA(cudaMemsetAsync(xl(l), 0, sizeof(T) * F.plane, s));
        const int h = (F.n + 1) / 2;
        const double N = dofs3(c, l);
        if (hs3_on<T>(c)) {
            BMG_TRY(hs3_down(c, l, bl(l), xl(l)));
        } else {
            for (int col = 0; col < 8; col++) BMG_TRY(colour_sweep<T>(c, l, v, bl(l), xl(l), col, h));
        }
        prof_begin(c, BMG_PROF_RESIDUAL, l);
        k_residual3d_sweep<T><<<g3(F.n, F.n, F.n), 64, 0, s>>>(v, xl(l), (T*)F.r);
        prof_end(c, BMG_PROF_RESIDUAL, l, (c.ns + 3) * sz * N);
        prof_begin(c, BMG_PROF_RESTRICT, l);
        k_restrict3d<T><<<g3(K.n, K.n, K.n), 64, 0, s>>>(F.n, F.ld, (const T*)F.r, P_of<T>(F), K.n, K.ld, K.plane,
                                                        (T*)K.b);
        prof_end(c, BMG_PROF_RESTRICT, l, (1.0 + c.np / 8.0 + 0.125) * sz * N);
        c.launches += 2;   // residual, restriction (the colours count themselves)
    }
    {
        Tail3Args<T> a{};
        a.nlev = L - t;
        if (a.nlev > kTail3Lev) return BMG_ERR_STATE;   // n <= 17 has at most kTail3Lev levels
        for (int q = 0; q < a.nlev; q++) {
            const int l = t + q;
            const Level& F = c.lev[l];
            Tail3Level<T>& g = a.lv[q];
            g.A = L3<T>{A_of<T>(F), F.n, F.ld, F.plane};
            g.P = l + 1 < L ? P_of<T>(F) : nullptr;
            g.ldc = l + 1 < L ? c.lev[l + 1].ld : 0;
            g.plc = l + 1 < L ? c.lev[l + 1].plane : 0;
            g.b = bl(l);
            g.x = xl(l);
            g.r = (T*)F.r;
        }
        const Level& C = c.lev[L - 1];
        a.a64c = C.A64 + 13 * C.plane + (long long)C.ld * (1 + (long long)C.n) + 1;
        size_t smem = 0;
        if (tail3_stages<T>()) {
            int ns[kTail3Lev];
            for (int q = 0; q < a.nlev; q++) ns[q] = c.lev[t + q].n;
            smem = sizeof(T) * tail3_smem_elems(ns, a.nlev);
            BMG_CUDA(cudaFuncSetAttribute(k_vtail3d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
        k_vtail3d<T><<<1, kTail3Threads, smem, s>>>(a);
        c.launches++;
    }
    for (int l = t - 1; l >= 0; l--) {
        const Level& F = c.lev[l];
        const Level& K = c.lev[l + 1];
        L3<T> v{A_of<T>(F), F.n, F.ld, F.plane};
        const double N = dofs3(c, l);
        if (hs3_on<T>(c)) {
            BMG_TRY(hs3_up(c, l, bl(l), xl(l), xl(l + 1)));
            continue;
        }
        prof_begin(c, BMG_PROF_PROLONG, l);
        k_prolong3d<T><<<g3(K.n - 1, K.n - 1, K.n - 1), 64, 0, s>>>(F.n, F.ld, xl(l), P_of<T>(F), K.n, K.ld,
                                                                     K.plane, xl(l + 1));
        prof_end(c, BMG_PROF_PROLONG, l, (2.0 + c.np / 8.0 + 0.125) * sz * N);
        const int h = (F.n + 1) / 2;
        for (int col = 7; col >= 0; col--) BMG_TRY(colour_sweep<T>(c, l, v, bl(l), xl(l), col, h));
        c.launches += 1;   // prolongation
    }
    (void)xout;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

template bmg_status vcycle3d_impl<double>(Ctx&, const double*, double*, double*);
template bmg_status vcycle3d_impl<float>(Ctx&, const float*, float*, float*);

}  // namespace bmg
