// tail2d.cu -- the coarse end of the 2-D V(1,1)-cycle (Sec. 2.2, "Solution
// phase" step 3) in a single CTA.
//
// Below about 33 nodes per side a level holds a few thousand values, and the
// streaming kernels spend their time on launch and pipeline latency rather
// than on data.  This kernel runs every level from the first one with
// n <= kTailMaxN down to the 3-node grid and back up in one launch: it copies
// the operators and interpolation weights of those levels into shared memory
// (compact rows, row length n), then performs the steps of the streaming
// kernels (zero guess, forward colours 0..3, the residual from the couplings
// to later colours, restriction of the five fine points per coarse node that
// carry a residual, exact coarsest solve in FP64, correction, reverse
// colours 3..0) in seven barrier-separated phases per level, and writes the
// finished iterate of its first level back for the up kernel of the level
// above.
//
// The operators and weights of the tail levels do not change between
// V-cycles, so bmg_setup packs them once (tail_pack) into a contiguous
// buffer that is already the kernel's shared-memory image; each launch then
// stages it with a few bulk asynchronous copies completed on one mbarrier
// (bounded wait), while the threads clear the vectors and load the
// right-hand side.
#include <type_traits>

#include "common.cuh"
#include "mbar.cuh"

namespace bmg {
namespace {

constexpr int kTailThreads = 256;      // one thread per node of a colour at n = 33
constexpr unsigned kTailChunk = 16384;    // bytes per bulk copy

template <typename T>
__device__ __forceinline__ T tdiv(T s, T d) { return s / d; }
template <>
__device__ __forceinline__ float tdiv<float>(float s, float d) { return __fdividef(s, d); }

// Packed image, per level l: A (5 planes of n_l^2, compact rows of length
// n_l), then P (8 planes of n_{l+1}^2) unless l is the last level.  The
// vectors (b, x, r per level) follow the image in shared memory.
__host__ __device__ inline long long tail_pack_elems(const int* n, int nlev) {
    long long e = 0;
    for (int l = 0; l < nlev; l++) {
        e += (long long)NS2 * n[l] * n[l];
        if (l + 1 < nlev) e += (long long)NP2 * n[l + 1] * n[l + 1];
    }
    return e;
}

__host__ __device__ inline long long tail_vec_elems(const int* n, int nlev) {
    long long e = 0;
    for (int l = 0; l < nlev; l++) e += 3LL * n[l] * n[l];
    return e;
}

template <typename T>
__host__ __device__ inline unsigned tail_pack_bytes_of(const int* n, int nlev) {
    return (unsigned)((tail_pack_elems(n, nlev) * sizeof(T) + 15) & ~15LL);
}

// Copies plane-strided planes (row length ld, plane stride pl) of an m x m
// grid into compact planes (row length m).
template <typename T>
__global__ void k_tail_pack(const T* __restrict__ src, int planes, int m, int ld, long long pl, T* __restrict__ dst) {
    const int total = planes * m * m;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int p = k / (m * m);
        const int r = k - p * m * m;
        const int j = r / m, i = r - j * m;
        dst[k] = src[p * pl + (long long)j * ld + i];
    }
}

// NR right-hand sides: vectors interleaved, NR values per node, operators
// and weights shared.  BATCH: one CTA per problem, arguments from targs.
template <typename T, int NR = 1, bool BATCH = false>
__global__ void __launch_bounds__(kTailThreads) k_vtail2d(TailArgs a0, const TailArgs* __restrict__ targs) {
    const TailArgs& a = BATCH ? targs[blockIdx.x] : a0;
    if (BATCH && a.sys && batch_frozen(a.sys, 0)) return;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t bar;
    // per level: nodes per side and element offsets (from base) of A, P and
    // of the vectors b, x = b + n^2, r = b + 2 n^2.  Kept in shared memory:
    // per-thread arrays indexed by the level would live in local memory.
    __shared__ int s_n[kMaxLevels], s_oA[kMaxLevels], s_oP[kMaxLevels], s_oB[kMaxLevels];
    __shared__ int s_nvec;
    T* base = (T*)(((uintptr_t)smem_raw + 15) & ~(uintptr_t)15);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int L = a.nlev;
    if (tid == 0) {
        // stage the packed image (A_0, P_0, A_1, P_1, ..., A_{L-1})
        mbar::init(&bar, 1);
        mbar::fence_init();
        mbar::expect_tx(&bar, a.pack_bytes);
        const unsigned char* src = (const unsigned char*)a.pack;
        for (unsigned off = 0; off < a.pack_bytes; off += kTailChunk) {
            const unsigned len = a.pack_bytes - off < kTailChunk ? a.pack_bytes - off : kTailChunk;
            mbar::bulk_g2s((unsigned char*)base + off, src + off, len, &bar);
        }
        int q = 0;
        for (int l = 0; l < L; l++) {
            const int m = a.ns[l];
            s_n[l] = m;
            s_oA[l] = q;
            q += NS2 * m * m;
            s_oP[l] = q;
            if (l + 1 < L) q += NP2 * a.ns[l + 1] * a.ns[l + 1];
        }
        q = (int)(a.pack_bytes / sizeof(T));
        const int v0 = q;
        for (int l = 0; l < L; l++) {
            s_oB[l] = q;
            q += 3 * s_n[l] * s_n[l] * NR;
        }
        s_nvec = q - v0;
    }
    __syncthreads();
    // meanwhile: clear the vectors, load the right-hand side of level 0
    {
        T* v = base + s_oB[0];
        const int nv = s_nvec;
        for (int k = tid; k < nv; k += nth) v[k] = (T)0;
    }
    __syncthreads();
    {
        const int m = s_n[0];
        T* b = base + s_oB[0];
        const T* bg = (const T*)a.b0;
        for (int k = tid; k < m * m * NR; k += nth) {
            const int kn = k / NR, rh = k - kn * NR;
            const int j = kn / m, i = kn - j * m;
            b[k] = bg[((long long)j * a.ld0 + i) * NR + rh];
        }
    }
    const bool staged = mbar::wait(&bar, 0);
    if (!staged) {
        // record the expiry, give the copies in flight one more bounded wait
        // (the shared memory must outlive them) and leave
        if (tid == 0) set_err(a.st, BMG_ERR_TIMEOUT);
        mbar::wait(&bar, 0);
        return;
    }
    __syncthreads();

    // off-diagonal part of row (i, j) of the level with operator A (row
    // length m, plane stride m2) on iterate x (NR values per node, right-hand
    // side rh), in the order of the streaming kernels (W, E, S, N, SW, NE, NW, SE)
    auto offdiag = [&](const T* A, int m, int m2, const T* x, int i, int j, int rh) {
        const int o = j * m + i;
        auto X = [&](int q) { return x[q * NR + rh]; };
        T s = A[W2 * m2 + o] * X(o - 1);
        s += A[W2 * m2 + o + 1] * X(o + 1);
        s += A[S2 * m2 + o] * X(o - m);
        s += A[S2 * m2 + o + m] * X(o + m);
        s += A[SW2 * m2 + o] * X(o - m - 1);
        s += A[SW2 * m2 + o + m + 1] * X(o + m + 1);
        s += A[NW2 * m2 + o] * X(o + m - 1);
        s += A[NW2 * m2 + o - m + 1] * X(o - m + 1);
        return s;
    };
    // every interior node of colour c of level l
    auto colour = [&](const T* A, int m, T* x, const T* f, int c) {
        const int m2 = m * m;
        // colour c has i parity (c & 1) and j parity (c >> 1): first interior
        // index of that parity i0, j0, and ni x nj such nodes
        const int i0 = 1 + ((c & 1) ^ 1), j0 = 1 + (((c >> 1) & 1) ^ 1);
        const int ni = (m - i0) / 2, nj = (m - j0) / 2;
        for (int kk = tid; kk < ni * nj * NR; kk += nth) {
            const int k = kk / NR, rh = kk - k * NR;
            const int jj = k / ni, ii = k - jj * ni;
            const int i = i0 + 2 * ii, j = j0 + 2 * jj;
            const int o = j * m + i;
            x[o * NR + rh] = tdiv<T>(f[o * NR + rh] - offdiag(A, m, m2, x, i, j, rh), A[C2 * m2 + o]);
        }
    };

    // Fine points are grouped in 2x2 blocks {2I, 2I+1} x {2J, 2J+1} around
    // each odd-odd (colour-3) point (2I+1, 2J+1), I, J in [0, nb), nb =
    // (m-1)/2; every interior point lies in exactly one block.  Phases that
    // need values of a colour being written in the same phase form those
    // values in registers (same expression, same order, so the same bits as
    // the thread that stores them) instead of waiting at a barrier.

    // ---- down: forward sweep from a zero guess, residual, restriction
    for (int l = 0; l + 1 < L; l++) {
        const int m = s_n[l], mc = s_n[l + 1];
        const int m2 = m * m, mc2 = mc * mc, nb = (m - 1) >> 1;
        const T* A = base + s_oA[l];
        const T* f = base + s_oB[l];
        T* x = base + s_oB[l] + m2 * NR;
        // colours 0 and 1, one thread per colour-1 point (2I+1, 2J), J >= 1:
        // a colour-0 point sees only zero neighbours, x = f / a_c; the
        // thread stores the colour-0 point (2I, 2J) of its block
        for (int kk = tid; kk < nb * (nb - 1) * NR; kk += nth) {
            const int k = kk / NR, rh = kk - k * NR;
            const int J = 1 + k / nb, I = k - (J - 1) * nb;
            const int o = 2 * J * m + 2 * I + 1;
            const T xl = I >= 1 ? tdiv<T>(f[(o - 1) * NR + rh], A[C2 * m2 + o - 1]) : (T)0;
            const T xr = I + 1 < nb ? tdiv<T>(f[(o + 1) * NR + rh], A[C2 * m2 + o + 1]) : (T)0;
            T sum = A[W2 * m2 + o] * xl;
            sum += A[W2 * m2 + o + 1] * xr;
            if (I >= 1) x[(o - 1) * NR + rh] = xl;
            x[o * NR + rh] = tdiv<T>(f[o * NR + rh] - sum, A[C2 * m2 + o]);
        }
        __syncthreads();
        // colours 2 and 3, one thread per colour-3 point: the colour-2 row
        // neighbours (whose own row neighbours, colour 3, are still zero)
        // are formed in registers; the thread stores the left one and itself
        auto c2val = [&](int o, int rh) {
            auto X = [&](int q) { return x[q * NR + rh]; };
            T sum = A[W2 * m2 + o] * (T)0;
            sum += A[W2 * m2 + o + 1] * (T)0;
            sum += A[S2 * m2 + o] * X(o - m);
            sum += A[S2 * m2 + o + m] * X(o + m);
            sum += A[SW2 * m2 + o] * X(o - m - 1);
            sum += A[SW2 * m2 + o + m + 1] * X(o + m + 1);
            sum += A[NW2 * m2 + o] * X(o + m - 1);
            sum += A[NW2 * m2 + o - m + 1] * X(o - m + 1);
            return tdiv<T>(f[o * NR + rh] - sum, A[C2 * m2 + o]);
        };
        for (int kk = tid; kk < nb * nb * NR; kk += nth) {
            const int k = kk / NR, rh = kk - k * NR;
            auto X = [&](int q) { return x[q * NR + rh]; };
            const int J = k / nb, I = k - J * nb;
            const int o = (2 * J + 1) * m + 2 * I + 1;
            const T xl = I >= 1 ? c2val(o - 1, rh) : (T)0;
            const T xr = I + 1 < nb ? c2val(o + 1, rh) : (T)0;
            T sum = A[W2 * m2 + o] * xl;
            sum += A[W2 * m2 + o + 1] * xr;
            sum += A[S2 * m2 + o] * X(o - m);
            sum += A[S2 * m2 + o + m] * X(o + m);
            sum += A[SW2 * m2 + o] * X(o - m - 1);
            sum += A[SW2 * m2 + o + m + 1] * X(o + m + 1);
            sum += A[NW2 * m2 + o] * X(o + m - 1);
            sum += A[NW2 * m2 + o - m + 1] * X(o - m + 1);
            if (I >= 1) x[(o - 1) * NR + rh] = xl;
            x[o * NR + rh] = tdiv<T>(f[o * NR + rh] - sum, A[C2 * m2 + o]);
        }
        __syncthreads();
        // residual and restriction, one thread per interior coarse node.
        // Each point's update zeroed its residual when its later-colour
        // neighbours were still zero, so the residual is minus those
        // couplings times their new values: colour 0 all eight neighbours,
        // colour 1 the six off its row, colour 2 its two row neighbours,
        // colour 3 none (so its weights are not needed)
        const T* P = base + s_oP[l];
        T* bc = base + s_oB[l + 1];
        auto r1 = [&](int o, int rh) {   // colour 1 (odd i, even j)
            auto X = [&](int q) { return x[q * NR + rh]; };
            T sum = A[S2 * m2 + o] * X(o - m);
            sum += A[S2 * m2 + o + m] * X(o + m);
            sum += A[SW2 * m2 + o] * X(o - m - 1);
            sum += A[SW2 * m2 + o + m + 1] * X(o + m + 1);
            sum += A[NW2 * m2 + o] * X(o + m - 1);
            sum += A[NW2 * m2 + o - m + 1] * X(o - m + 1);
            return -sum;
        };
        auto r2 = [&](int o, int rh) {   // colour 2 (even i, odd j)
            return -(A[W2 * m2 + o] * x[(o - 1) * NR + rh] + A[W2 * m2 + o + 1] * x[(o + 1) * NR + rh]);
        };
        for (int kk = tid; kk < (mc - 2) * (mc - 2) * NR; kk += nth) {
            const int k = kk / NR, rh = kk - k * NR;
            const int J = 1 + k / (mc - 2), I = 1 + k % (mc - 2);
            const int O = J * mc + I, o = 2 * J * m + 2 * I;
            T b = -offdiag(A, m, m2, x, 2 * I, 2 * J, rh);
            b += P[PXR * mc2 + O - 1] * r1(o - 1, rh);
            b += P[PXL * mc2 + O] * r1(o + 1, rh);
            b += P[PYN * mc2 + O - mc] * r2(o - m, rh);
            b += P[PYS * mc2 + O] * r2(o + m, rh);
            bc[O * NR + rh] = b;
        }
        __syncthreads();
    }
    // ---- coarsest: one unknown, exact in FP64
    if (tid < NR) {
        const int m = s_n[L - 1];
        const int o = m + 1;
        base[s_oB[L - 1] + (2 * m * m + o) * NR + tid] = (T)((double)base[s_oB[L - 1] + o * NR + tid] / *a.a64c);
    }
    __syncthreads();
    // ---- up: correction x_pre + P x_c, reverse colours 3..0
    for (int l = L - 2; l >= 0; l--) {
        const int m = s_n[l], mc = s_n[l + 1];
        const int m2 = m * m, mc2 = mc * mc, nb = (m - 1) >> 1;
        const T* P = base + s_oP[l];
        const T* xc = base + s_oB[l + 1] + 2 * mc2 * NR;
        const T* xpre = base + s_oB[l] + m2 * NR;
        const T* A = base + s_oA[l];
        const T* f = base + s_oB[l];
        T* x = base + s_oB[l] + 2 * m2 * NR;
        // corrected value of interior point (i, j); zero on the boundary
        auto corr = [&](int i, int j, int rh) -> T {
            if (i < 1 || j < 1 || i > m - 2 || j > m - 2) return (T)0;
            const int o = j * m + i;
            const int I = i >> 1, J = j >> 1, O = J * mc + I;
            auto XC = [&](int q) { return xc[q * NR + rh]; };
            const T xp = xpre[o * NR + rh];
            if (!(i & 1) && !(j & 1)) return xp + XC(O);
            if (!(j & 1)) return xp + P[PXL * mc2 + O] * XC(O) + P[PXR * mc2 + O] * XC(O + 1);   // (2I+1, 2J)
            return xp + P[PYS * mc2 + O] * XC(O) + P[PYN * mc2 + O] * XC(O + mc);              // (2I, 2J+1)
        };
        // correction and colour 3, one thread per colour-3 point: its eight
        // corrected neighbours in registers; stores the corrected points of
        // its block and its own new value
        for (int kk = tid; kk < nb * nb * NR; kk += nth) {
            const int k = kk / NR, rh = kk - k * NR;
            const int J = k / nb, I = k - J * nb;
            const int i = 2 * I + 1, j = 2 * J + 1, o = j * m + i;
            const T w = corr(i - 1, j, rh), e = corr(i + 1, j, rh);
            const T so = corr(i, j - 1, rh), no = corr(i, j + 1, rh);
            const T sw = corr(i - 1, j - 1, rh), ne = corr(i + 1, j + 1, rh);
            const T nw = corr(i - 1, j + 1, rh), se = corr(i + 1, j - 1, rh);
            T sum = A[W2 * m2 + o] * w;
            sum += A[W2 * m2 + o + 1] * e;
            sum += A[S2 * m2 + o] * so;
            sum += A[S2 * m2 + o + m] * no;
            sum += A[SW2 * m2 + o] * sw;
            sum += A[SW2 * m2 + o + m + 1] * ne;
            sum += A[NW2 * m2 + o] * nw;
            sum += A[NW2 * m2 + o - m + 1] * se;
            if (I >= 1 && J >= 1) x[(o - m - 1) * NR + rh] = sw;
            if (J >= 1) x[(o - m) * NR + rh] = so;
            if (I >= 1) x[(o - 1) * NR + rh] = w;
            x[o * NR + rh] = tdiv<T>(f[o * NR + rh] - sum, A[C2 * m2 + o]);
        }
        __syncthreads();
        for (int c = 2; c >= 0; c--) {
            colour(A, m, x, f, c);
            __syncthreads();
        }
    }
    {
        const int m = s_n[0];
        const T* x = base + s_oB[0] + 2 * m * m * NR;
        T* xg = (T*)a.x0;
        for (int kk = tid; kk < (m - 2) * (m - 2) * NR; kk += nth) {
            const int k = kk / NR, rh = kk - k * NR;
            const int j = 1 + k / (m - 2), i = 1 + k % (m - 2);
            xg[((long long)j * a.ld0 + i) * NR + rh] = x[(j * m + i) * NR + rh];
        }
    }
}

}  // namespace

int tail_first_level(const Ctx& c) {
    int t = c.nlev - 1;
    while (t > 1 && c.lev[t - 1].n <= kTailMaxN) t--;
    return t;
}

namespace {

int tail_sizes(const Ctx& c, int t, int* ns) {
    const int L = c.nlev - t;
    for (int l = 0; l < L; l++) ns[l] = c.lev[t + l].n;
    return L;
}

}  // namespace

size_t tail_pack_bytes(const Ctx& c) {
    if (c.dim != 2 || c.nlev < 2) return 0;
    int ns[kMaxLevels];
    const int L = tail_sizes(c, tail_first_level(c), ns);
    return c.opts.precision == BMG_PREC_FP32 ? tail_pack_bytes_of<float>(ns, L) : tail_pack_bytes_of<double>(ns, L);
}

size_t tail_smem_bytes(const Ctx& c, int t) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    int ns[kMaxLevels];
    const int L = tail_sizes(c, t, ns);
    const size_t pack = f32 ? tail_pack_bytes_of<float>(ns, L) : tail_pack_bytes_of<double>(ns, L);
    return 16 + pack + (size_t)tail_vec_elems(ns, L) * (f32 ? 4 : 8);
}

// Packs the operators and weights of the tail levels into c.tail_pack (the
// kernel's shared-memory image); called by bmg_setup after the FP32 copies
// are made.
template <typename T>
bmg_status tail_pack_impl(Ctx& c) {
    const int t = tail_first_level(c);
    const int L = c.nlev - t;
    T* q = (T*)c.tail_pack;
    for (int l = 0; l < L; l++) {
        const Level& Lv = c.lev[t + l];
        const T* A = std::is_same<T, float>::value ? (const T*)Lv.A32 : (const T*)Lv.A64;
        k_tail_pack<T><<<cdiv(NS2 * Lv.n * Lv.n, 256), 256, 0, c.stream>>>(A, NS2, Lv.n, Lv.ld, Lv.plane, q);
        c.launches++;
        q += (long long)NS2 * Lv.n * Lv.n;
        if (l + 1 < L) {
            const Level& K = c.lev[t + l + 1];
            const T* P = std::is_same<T, float>::value ? (const T*)Lv.P32 : (const T*)Lv.P64;
            k_tail_pack<T><<<cdiv(NP2 * K.n * K.n, 256), 256, 0, c.stream>>>(P, NP2, K.n, K.ld, K.plane, q);
            c.launches++;
            q += (long long)NP2 * K.n * K.n;
        }
    }
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status tail_pack(Ctx& c) {
    if (!c.tail_pack) return BMG_OK;
    return c.opts.precision == BMG_PREC_FP32 ? tail_pack_impl<float>(c) : tail_pack_impl<double>(c);
}

// Arguments of the tail kernel of an FP32 context whose first tail level
// reads its right-hand side from b0 and writes its iterate to x0 (row
// length ld0, nr values per node).
bmg_status tail_args(const Ctx& c, const void* b0, void* x0, int ld0, KState* st, TailArgs* a) {
    if (!c.tail_pack || c.opts.precision != BMG_PREC_FP32) return BMG_ERR_STATE;
    const int t = tail_first_level(c);
    *a = TailArgs{};
    a->nlev = tail_sizes(c, t, a->ns);
    a->pack = c.tail_pack;
    a->pack_bytes = (unsigned)tail_pack_bytes(c);
    a->b0 = b0;
    a->x0 = x0;
    a->ld0 = ld0;
    const Level& C = c.lev[c.nlev - 1];
    a->a64c = C.A64 + (long long)C2 * C.plane + C.ld + 1;
    a->st = st;
    return BMG_OK;
}

// Shared memory of the batched tail kernel for tail levels ns[0..L).
size_t batch_tail_smem(const int* ns, int L) {
    return 16 + tail_pack_bytes_of<float>(ns, L) + (size_t)tail_vec_elems(ns, L) * kBatchR * sizeof(float);
}

// One CTA per problem, kBatchR right-hand sides; args: device array of count
// entries whose tails all have the sizes the smem bound was computed for.
bmg_status batch_tail(const TailArgs* args, int count, size_t smem, cudaStream_t s) {
    auto kern = k_vtail2d<float, kBatchR, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BMG_ERR_DEVICE;
    kern<<<count, kTailThreads, smem, s>>>(TailArgs{}, args);
    return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
}

// Levels t .. nlev-1 in one launch: reads lev[t].b, writes lev[t].r.
bmg_status tail_vcycle(Ctx& c, int t) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    if (!c.tail_pack || t != tail_first_level(c)) return BMG_ERR_STATE;
    TailArgs a{};
    a.nlev = tail_sizes(c, t, a.ns);
    a.pack = c.tail_pack;
    a.pack_bytes = (unsigned)tail_pack_bytes(c);
    a.b0 = c.lev[t].b;
    a.x0 = c.lev[t].r;
    a.ld0 = c.lev[t].ld;
    const Level& C = c.lev[c.nlev - 1];
    a.a64c = C.A64 + (long long)C2 * C.plane + C.ld + 1;
    a.st = c.st;
    const size_t smem = tail_smem_bytes(c, t);
    if (f32) {
        if (cudaFuncSetAttribute(k_vtail2d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return BMG_ERR_DEVICE;
        k_vtail2d<float><<<1, kTailThreads, smem, c.stream>>>(a, nullptr);
    } else {
        if (cudaFuncSetAttribute(k_vtail2d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return BMG_ERR_DEVICE;
        k_vtail2d<double><<<1, kTailThreads, smem, c.stream>>>(a, nullptr);
    }
    c.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

}  // namespace bmg
