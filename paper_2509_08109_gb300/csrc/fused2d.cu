// fused2d.cu -- streaming V-cycle kernels for one 2-D level pair.
//
// vdown: zero initial guess -> one forward multicolour Gauss-Seidel sweep
//        (colours 0,1,2,3) -> residual -> restriction b_c = P^T r.
// vup:   x += P x_c -> one reverse sweep (colours 3,2,1,0).
// Both are the per-level steps of the V(1,1)-cycle (Sec. 2.2, "Solution
// phase" step 3); the fine residual and the corrected iterate never touch
// HBM.
//
// Design.  A CTA owns a strip of coarse columns [I0, I0+wc) and a chunk of
// coarse rows [J0, J0+hc) and streams through the fine rows of that strip
// in pairs (2J+1, 2J+2).  Colour dependencies of the 4-colour sweep are
// local in j: in the forward sweep an even row needs only itself (colour 0
// sees only untouched zero neighbours, colour 1 only its colour-0 row
// neighbours), an odd row needs its two even neighbour rows; in the reverse
// sweep an odd row needs the corrected (not yet smoothed) even rows and an
// even row needs its two finished odd rows.  So one pass over the rows, with
// a window of a few rows in shared memory, finishes every row; a column halo
// of 8-9 fine points (recomputed by both neighbours) covers the horizontal
// dependencies.  A step handles K row pairs at once: thread (x, y) owns
// the column pair (2x, 2x+1) of row pair y, so every colour phase keeps all
// threads busy and a step costs six block barriers for 2K fine rows (K = 2).  Rows
// arrive by TMA (cp.async.bulk.tensor) into a ring of RP = K+1+D row-pair
// slots, each completed by an mbarrier with an expected byte count; the
// next D = K pairs are in flight while a step computes; one thread issues all
// copies.  Interpolation weights go straight from global memory into
// registers (each is used by one thread).  Every mbarrier wait is bounded
// by the global timer; on expiry the CTA records BMG_ERR_TIMEOUT, drains its
// outstanding copies (bounded) and returns.
//
// Several right-hand sides (NR = 4).  Vectors are interleaved, NR values per
// node, and a thread handles one column pair for all right-hand sides, its
// values as a float4: every stencil and interpolation value is read once
// per sweep (from global memory and from shared memory) for all of them.
// Batched form (BATCH).  All (problem, level) members of one size class
// keep their arrays in class-contiguous storage with one more tensor
// dimension (the member); a persistent grid walks the class's work-list of
// (member, tile) items, carrying its ring's mbarrier phases from item to
// item.  Per-member output pointers and interpolation weights come from a
// device table (BatchMember).
#include <cuda.h>

#include <type_traits>

#include "common.cuh"
#include "fused2d.cuh"
#include "mbar.cuh"

namespace bmg {
namespace {

using mbar::smem_u32;

__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((unsigned long long)m), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma3d(void* dst, const CUtensorMap* m, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma4d(void* dst, const CUtensorMap* m, uint64_t* bar, int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)m), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// The values of a node's NR right-hand sides: T itself for one, a float4
// for four (FP32); vectors are interleaved in memory, so a row of them is
// an array of these.
template <typename T, int NR>
struct VecOf {
    using type = T;
};
template <>
struct VecOf<float, 4> {
    using type = float4;
};

__device__ __forceinline__ float4 operator+(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 operator-(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 operator-(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 operator*(float s, float4 b) { return make_float4(s * b.x, s * b.y, s * b.z, s * b.w); }
__device__ __forceinline__ float4& operator+=(float4& a, float4 b) {
    a = a + b;
    return a;
}

template <typename V>
__device__ __forceinline__ V vzero() { return (V)0; }
template <>
__device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// conversions between the value types (precision casts for one right-hand side)
template <typename D, typename S>
__device__ __forceinline__ D vcast(S s) { return (D)s; }
template <>
__device__ __forceinline__ float4 vcast<float4, float4>(float4 s) { return s; }

// a row of values: element c is p[c]
template <typename V>
struct RowV {
    V* p;
    __device__ __forceinline__ V& operator[](int c) const { return p[c]; }
};

// A row of the iterate and residual rings, which the threads write
// themselves: the even columns first, then the odd ones (HALF of each), so
// that the column pairs the threads of a warp own map to consecutive words
// (no bank conflicts on the neighbour reads).
template <typename V, int HALF>
struct SRow {
    V* p;
    __device__ __forceinline__ V& operator[](int c) const { return p[(c & 1) * HALF + (c >> 1)]; }
};

// NR compensated FP32 accumulators (one per right-hand side); add(f, x)
// accumulates f * x per right-hand side.
struct Acc32f;
template <int NR>
struct AccN;

// ------------------------------------------------------------------ layout
__host__ __device__ constexpr int r128(int b) { return (b + 127) & ~127; }

template <typename T>
__device__ __forceinline__ T divide(T s, T d) { return s / d; }
template <>
__device__ __forceinline__ float divide<float>(float s, float d) { return __fdividef(s, d); }
__device__ __forceinline__ float4 divide(float4 s, float d) {
    return make_float4(__fdividef(s.x, d), __fdividef(s.y, d), __fdividef(s.z, d), __fdividef(s.w, d));
}

// Shared-memory layout: RP ring slots of one row pair each (stencil planes,
// right-hand side, and for the up kernel the pre-smoothed iterate and one
// coarse row of the coarse iterate), then a (2K+4)-row ring of the iterate X
// and (down) an equal ring of the residual R, then the mbarriers.
template <typename T, typename TF, int K, bool UP, int NR = 1>
struct Lay {
    // ring slots: the K pairs of the current step, the pair below it (halo
    // rows), and D = K pairs in flight (one step ahead; two steps ahead
    // measured no faster on the 4097^2 refinement solve, with the wider ring
    // costing strip width or occupancy).  The one-right-hand-side up kernel
    // keeps one more slot, which it fills one pair further ahead: measured
    // on the 4097^2 refinement solve it runs faster that way at 4 CTAs per
    // SM (3.46 ms per solve) than with the smaller ring at 5 (3.52 ms), while
    // the down kernel gains from the fifth CTA (2.36 ms against 2.51 ms).
    static constexpr int D = K;
    static constexpr int RP = K + 1 + D + (UP && NR == 1 ? 1 : 0);
    // rows of the X / R rings: a step reads and writes fine rows 2J-1 .. 2J+2K
    // (2K+2 rows); consecutive steps are separated by a block barrier
    // (rounded up to a power of two in the down kernel, whose rings have the
    // shared memory to spare, so that the row index wraps with a mask)
    static constexpr int XR = UP ? 2 * K + 4 : (2 * K + 4 <= 8 ? 8 : 16);
    int WW, WWc, sA, sF, sXp, sC;
    __host__ __device__ Lay(int wc) {
        WW = 2 * wc + 16;
        WWc = wc + 8;
        sA = r128(10 * WW * (int)sizeof(T));
        sF = r128(2 * WW * NR * (int)sizeof(TF));
        sXp = UP ? r128(2 * WW * NR * (int)sizeof(T)) : 0;
        sC = UP ? r128(WWc * NR * (int)sizeof(T)) : 0;
    }
    __host__ __device__ int slot() const { return sA + sF + sXp + sC; }
    __host__ __device__ int bytes() const {
        return 128 + RP * slot() + (UP ? 1 : 2) * XR * WW * NR * (int)sizeof(T) + RP * 8;
    }
    __host__ __device__ uint32_t tx() const {
        return (uint32_t)(10 * WW * sizeof(T) + 2 * WW * NR * sizeof(TF) +
                          (UP ? 2 * WW * NR * sizeof(T) + WWc * NR * sizeof(T) : 0));
    }
};

// Row-pair ring shared by both kernels.  Pair q (local index, q >= 0) is
// the fine rows 2(q0+q)+1 and 2(q0+q)+2 and, for the up kernel, coarse row
// q0+q+1 of the coarse iterate.
// qb: pairs this CTA issued before the current item (the persistent batched
// kernels carry the ring's slots and mbarrier phases from item to item).
template <typename T, typename TF, int K, bool UP, int NR = 1>
struct Ring {
    using V = typename VecOf<T, NR>::type;
    using VF = typename VecOf<TF, NR>::type;
    static constexpr unsigned RPu = (unsigned)Lay<T, TF, K, UP, NR>::RP;
    unsigned char *pA, *pF, *pXp, *pC;
    uint64_t* bars;
    int q0, WW, sA, sF, sXp, sC;
    unsigned qb;
    __device__ __forceinline__ int slot_of_row(int j) const {
        return (int)((qb + (unsigned)(((j - 1) >> 1) - q0)) % RPu);
    }
    __device__ __forceinline__ const T* A(int j) const {      // plane 0 of fine row j
        return (const T*)(pA + slot_of_row(j) * sA) + ((j - 1) & 1) * WW;
    }
    __device__ __forceinline__ RowV<const VF> F(int j) const {
        return {(const VF*)(pF + slot_of_row(j) * sF) + ((j - 1) & 1) * WW};
    }
    __device__ __forceinline__ RowV<const V> Xp(int j) const {
        return {(const V*)(pXp + slot_of_row(j) * sXp) + ((j - 1) & 1) * WW};
    }
    __device__ __forceinline__ RowV<const V> C(int J) const {      // coarse row J (carried by pair J-1)
        return {(const V*)(pC + (int)((qb + (unsigned)(J - 1 - q0)) % RPu) * sC)};
    }
};

// bounded wait for the pairs with ring indices [qa, qb); returns false (in
// every thread) on expiry
template <int RP>
__device__ __forceinline__ bool wait_pairs(uint64_t* bars, unsigned qa, unsigned qb) {
    bool mine = true;
    for (unsigned q = qa; q < qb; q++) mine = mine && mbar::wait(bars + (q % RP), (q / RP) & 1u);
    return __syncthreads_and(mine) != 0;
}

// Compensated (Neumaier) FP32 accumulator for the fused dot products.
struct Acc32f {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <>
struct AccN<1> {
    Acc32f a[1];
    __device__ __forceinline__ void add(float f, float x) { a[0].add(f * x); }
};
template <>
struct AccN<4> {
    Acc32f a[4];
    __device__ __forceinline__ void add(float4 f, float4 x) {
        a[0].add(f.x * x.x);
        a[1].add(f.y * x.y);
        a[2].add(f.z * x.z);
        a[3].add(f.w * x.w);
    }
};

// ------------------------------------------------------------------ node updates
// Symmetric-half stencil rows: plane p of row j is A(j) + p * 2 * WW.
// Offsets: W(c) couples (c-1), W(c+1) couples (c+1) of the row; S(j) couples
// row j-1, S(j+1) row j+1; SW(j,c) couples (c-1, j-1), SW(j+1,c+1) (c+1, j+1);
// NW(j,c) couples (c-1, j+1), NW(j-1,c+1) (c+1, j-1).
template <typename T, typename V, typename XA>
struct Rows {
    const T *a, *an, *as;          // stencil rows j, j+1, j-1 (plane 0)
    XA x, xn, xs;                  // iterate rows j, j+1, j-1
    int PL;                        // plane stride
    __device__ __forceinline__ V offdiag(int c) const {
        V s = a[W2 * PL + c] * x[c - 1];
        s += a[W2 * PL + c + 1] * x[c + 1];
        s += a[S2 * PL + c] * xs[c];
        s += an[S2 * PL + c] * xn[c];
        s += a[SW2 * PL + c] * xs[c - 1];
        s += an[SW2 * PL + c + 1] * xn[c + 1];
        s += a[NW2 * PL + c] * xn[c - 1];
        s += as[NW2 * PL + c + 1] * xs[c + 1];
        return s;
    }
    // forward sweep, colour 2: the (c +- 1, j) neighbours are still zero
    __device__ __forceinline__ V offdiag_no_row(int c) const {
        V s = a[S2 * PL + c] * xs[c];
        s += an[S2 * PL + c] * xn[c];
        s += a[SW2 * PL + c] * xs[c - 1];
        s += an[SW2 * PL + c + 1] * xn[c + 1];
        s += a[NW2 * PL + c] * xn[c - 1];
        s += as[NW2 * PL + c + 1] * xs[c + 1];
        return s;
    }
    __device__ __forceinline__ T diag(int c) const { return a[C2 * PL + c]; }
};

// ------------------------------------------------------------------ down kernel
template <typename T, typename TF, int K, int WC, int NR = 1, bool BATCH = false>
__global__ void __launch_bounds__((WC + 8) * K, sizeof(T) == 4 ? 3 : 1)
    k_vdown2d(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmF, FusedArgs p) {
    using LY = Lay<T, TF, K, false, NR>;
    using V = typename VecOf<T, NR>::type;       // a node's values, all right-hand sides
    constexpr int RP = LY::RP;
    extern __shared__ unsigned char smem_raw[];
    const LY L(WC);   // strip width fixed at compile time: every shared-memory stride is a constant
    const int WW = L.WW, PL = 2 * WW;
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    Ring<T, TF, K, false, NR> rg;
    rg.pA = base;
    rg.pF = base + RP * L.sA;
    rg.pXp = rg.pC = nullptr;
    constexpr int XR = LY::XR;
    V* sX = (V*)(base + RP * L.slot());
    V* sR = sX + XR * WW;
    rg.bars = (uint64_t*)(sR + XR * WW);
    rg.WW = WW;
    rg.sA = L.sA;
    rg.sF = L.sF;
    rg.sXp = rg.sC = 0;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool lead = tx == 0 && ty == 0;
    const int nf = p.nf, nc = p.nc;
    const uint32_t txb = L.tx();
    if (lead) {
        for (int s = 0; s < RP; s++) mbar::init(rg.bars + s, 1);
        mbar::fence_init();
    }
    __syncthreads();
    const int nitems = BATCH ? p.nmem * p.tiles_x * p.tiles_y : 1;
    unsigned qb = 0;
    for (int item = BATCH ? (int)blockIdx.x : 0; item < nitems; item += BATCH ? (int)gridDim.x : 1) {
    int bx, by, mi = 0;
    if (BATCH) {
        const int tpm = p.tiles_x * p.tiles_y;
        mi = item / tpm;
        const int t = item - mi * tpm;
        by = t / p.tiles_x;
        bx = t - by * p.tiles_x;
        // a problem none of whose systems takes this iteration: no copies,
        // no stores, no arrival (the same decision in every CTA)
        if (p.sys && batch_frozen(p.sys, p.mem[mi].prob)) continue;
    } else {
        bx = blockIdx.x;
        by = blockIdx.y;
    }
    const int I0 = 1 + bx * WC, J0 = 1 + by * p.hc;
    const int x0 = 2 * I0 - 10, xc0 = I0 - 5;
    rg.q0 = J0 - 2;
    rg.qb = qb;
    const int npairs = p.hc + 2;
    auto issue = [&](int q) {
        const int s = (int)((qb + (unsigned)q) % (unsigned)RP), Jp = rg.q0 + q;
        uint64_t* bar = rg.bars + s;
        mbar::expect_tx(bar, txb);
        if constexpr (BATCH) {
            // vector maps group 8 nodes x NR values into their innermost
            // dimension (x0 is a multiple of 8)
            tma4d(rg.pA + s * L.sA, &tmA, bar, x0, 2 * Jp + 1, 0, mi);
            tma4d(rg.pF + s * L.sF, &tmF, bar, 0, x0 / 8, 2 * Jp + 1, mi);
        } else {
            tma3d(rg.pA + s * L.sA, &tmA, bar, x0, 2 * Jp + 1, 0);
            tma2d(rg.pF + s * L.sF, &tmF, bar, x0, 2 * Jp + 1);
        }
    };
    int issued = npairs < RP ? npairs : RP, waited = 0;
    if (lead)
        for (int q = 0; q < issued; q++) issue(q);

    // per-thread columns: the even/odd pair (2 tx, 2 tx + 1) of the window
    const int ce = 2 * tx, co = ce + 1;
    const int ie = x0 + ce;
    const bool ve = ce >= 1 && ce <= WW - 2 && ie >= 1 && ie <= nf - 2;
    const bool vo = co <= WW - 2 && ie + 1 >= 1 && ie + 1 <= nf - 2;
    const bool own_e = ve && ce >= 9 && ce < 9 + 2 * WC;
    const bool own_o = vo && co >= 9 && co < 9 + 2 * WC;
    const int I = xc0 + tx;
    const bool vres = tx >= 5 && tx < 5 + WC && I >= 1 && I <= nc - 2;
    auto inrow = [&](int j) { return j >= 1 && j <= nf - 2; };
    using XA = SRow<V, WC + 8>;
    auto X = [&](int j) { return XA{sX + (int)((unsigned)j % XR) * WW}; };
    auto RR = [&](int j) { return XA{sR + (int)((unsigned)j % XR) * WW}; };
    auto rows = [&](int j) {
        return Rows<T, V, XA>{rg.A(j), rg.A(j + 1), rg.A(j - 1), X(j), X(j + 1), X(j - 1), PL};
    };
    const BatchMember* M = BATCH ? p.mem + mi : nullptr;
    const T* Pg = BATCH ? (const T*)M->P : (const T*)p.P;
    V* xg = (V*)(BATCH ? M->x[0] : p.x);
    V* bcg = (V*)(BATCH ? M->bc : p.bc);
    const V z0 = vzero<V>();

    // colour 0 / 1 of even row j, colour 2 / 3 of odd row j, residual of row j
    auto c0 = [&](int j) {
        const Rows<T, V, XA> r = rows(j);
        X(j)[ce] = (ve && inrow(j)) ? divide(vcast<V>(rg.F(j)[ce]), r.diag(ce)) : z0;
    };
    auto c1 = [&](int j) {
        const Rows<T, V, XA> r = rows(j);
        V v = z0;
        if (vo && inrow(j)) {
            const V s = vcast<V>(rg.F(j)[co]) - r.a[W2 * PL + co] * r.x[co - 1] - r.a[W2 * PL + co + 1] * r.x[co + 1];
            v = divide(s, r.diag(co));
        }
        X(j)[co] = v;
    };
    auto c2 = [&](int j) {
        const Rows<T, V, XA> r = rows(j);
        X(j)[ce] = (ve && inrow(j)) ? divide(vcast<V>(rg.F(j)[ce]) - r.offdiag_no_row(ce), r.diag(ce)) : z0;
    };
    auto c3 = [&](int j) {
        const Rows<T, V, XA> r = rows(j);
        X(j)[co] = (vo && inrow(j)) ? divide(vcast<V>(rg.F(j)[co]) - r.offdiag(co), r.diag(co)) : z0;
    };
    // Residual after the forward sweep from a zero guess.  A point's own
    // update zeroed its residual given the values of that moment, and the
    // neighbours of later colours were still zero then, so what remains is
    // minus their couplings times their new values:
    //   colour 0 (even row, even column): all eight neighbours;
    //   colour 1 (even row, odd column): the six on the odd rows above and below;
    //   colour 2 (odd row, even column): the two colour-3 row neighbours;
    //   colour 3 (odd row, odd column): none.
    auto resid = [&](int j) {
        const Rows<T, V, XA> r = rows(j);
        const XA Rj = RR(j);
        const bool rj = inrow(j);
        if (!(j & 1)) {
            Rj[ce] = (ve && rj) ? -r.offdiag(ce) : z0;
            Rj[co] = (vo && rj) ? -r.offdiag_no_row(co) : z0;
        } else {
            Rj[ce] = (ve && rj) ? -(r.a[W2 * PL + ce] * r.x[ce - 1] + r.a[W2 * PL + ce + 1] * r.x[ce + 1]) : z0;
            Rj[co] = z0;
        }
    };

    bool ok = wait_pairs<RP>(rg.bars, qb, qb + 2);
    waited = ok ? 2 : 0;
    if (ok) {   // pre-roll: rows 2J0-2 .. 2J0 final, residual of row 2J0-1
        if (ty == 0) { c0(2 * J0 - 2); c0(2 * J0); }
        __syncthreads();
        if (ty == 0) { c1(2 * J0 - 2); c1(2 * J0); }
        __syncthreads();
        if (ty == 0) c2(2 * J0 - 1);
        __syncthreads();
        if (ty == 0) c3(2 * J0 - 1);
        __syncthreads();
        if (ty == 0) resid(2 * J0 - 1);
        __syncthreads();
    }
    // interpolation weights of the thread's coarse node for the restriction,
    // loaded one step ahead.  After colour 3 the odd-odd fine points have
    // zero residual, so their four weights are not needed.
    T w[4];
    auto load_w = [&](int Jp) {
        const bool d = vres && Jp <= nc - 2;
        const long long o = (long long)Jp * p.ldc + I;
        w[0] = d ? Pg[PXR * p.plc + o - 1] : (T)0;
        w[1] = d ? Pg[PXL * p.plc + o] : (T)0;
        w[2] = d ? Pg[PYN * p.plc + o - p.ldc] : (T)0;
        w[3] = d ? Pg[PYS * p.plc + o] : (T)0;
    };
    load_w(J0 + ty);
    for (int J = J0; ok && J < J0 + p.hc; J += K) {
        const int qa = J - rg.q0;
        ok = wait_pairs<RP>(rg.bars, qb + qa, qb + qa + K);
        if (!ok) break;
        waited = qa + K;
        // every thread is past the previous step: refill the freed slots
        // (a step reads pairs qa - 1 .. qa + K - 1, so pairs up to qa - 2 are
        // done) with the pairs D ahead
        const int lim = min(npairs, qa - 1 + RP);
        if (lead)
            for (int q = issued; q < lim; q++) issue(q);
        issued = max(issued, lim);
        const int Jp = J + ty, jm = 2 * Jp, jo = jm + 1, je = jm + 2;
        const bool do_res = vres && Jp <= nc - 2;
        c0(je);
        __syncthreads();
        c1(je);
        __syncthreads();
        c2(jo);
        __syncthreads();
        c3(jo);
        __syncthreads();
        resid(jm);
        resid(jo);
        __syncthreads();
        if (do_res) {
            const XA Rm = RR(jm);
            const XA Rs = RR(jm - 1);
            const XA Rn = RR(jo);
            const int c = ce;
            V b = Rm[c];
            b += w[0] * Rm[c - 1];
            b += w[1] * Rm[c + 1];
            b += w[2] * Rs[c];
            b += w[3] * Rn[c];
            bcg[(long long)Jp * p.ldc + I] = b;
        }
        load_w(Jp + K);
        // finished rows 2Jp-1 and 2Jp of the owned columns
        if (inrow(jm - 1)) {
            const XA Xr = X(jm - 1);
            if (own_e) xg[(long long)(jm - 1) * p.ldf + ie] = Xr[ce];
            if (own_o) xg[(long long)(jm - 1) * p.ldf + ie + 1] = Xr[co];
        }
        if (inrow(jm)) {
            const XA Xr = X(jm);
            if (own_e) xg[(long long)jm * p.ldf + ie] = Xr[ce];
            if (own_o) xg[(long long)jm * p.ldf + ie + 1] = Xr[co];
        }
        // no barrier here: the next step's writes (rows 2Jp+2K+1.. of the X and R
        // rings) do not alias rows read above, and slots are refilled only after
        // the next step's first barrier
    }
    if (!ok) {
        if (lead) {
            set_err(p.st, BMG_ERR_TIMEOUT);
            for (int q = waited; q < issued; q++) {
                const unsigned g = qb + (unsigned)q;
                mbar::wait(rg.bars + (g % RP), (g / RP) & 1u);
            }
        }
        __syncthreads();
        return;
    }
    qb += (unsigned)npairs;
    if (BATCH) __syncthreads();   // the next item's copies reuse the ring and the rows
    }
}

// ------------------------------------------------------------------ up kernel
template <typename T, typename TF, typename TO, int K, int WC, int NR = 1, bool BATCH = false>
__global__ void __launch_bounds__((WC + 8) * K, sizeof(T) == 4 ? 3 : 1)
    k_vup2d(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmF,
            const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmC, FusedArgs p) {
    using LY = Lay<T, TF, K, true, NR>;
    using V = typename VecOf<T, NR>::type;        // a node's values, all right-hand sides
    using VO = typename VecOf<TO, NR>::type;
    using VZ = typename VecOf<float, NR>::type;   // FP32 values of the fused dot products
    constexpr int RP = LY::RP;
    extern __shared__ unsigned char smem_raw[];
    const LY L(WC);   // strip width fixed at compile time: every shared-memory stride is a constant
    const int WW = L.WW, PL = 2 * WW;
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    Ring<T, TF, K, true, NR> rg;
    rg.pA = base;
    rg.pF = rg.pA + RP * L.sA;
    rg.pXp = rg.pF + RP * L.sF;
    rg.pC = rg.pXp + RP * L.sXp;
    constexpr int XR = LY::XR;
    V* sX = (V*)(base + RP * L.slot());
    rg.bars = (uint64_t*)(sX + XR * WW);
    rg.WW = WW;
    rg.sA = L.sA;
    rg.sF = L.sF;
    rg.sXp = L.sXp;
    rg.sC = L.sC;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool lead = tx == 0 && ty == 0;
    const int nf = p.nf, nc = p.nc;
    const uint32_t txb = L.tx();
    const int tid = ty * blockDim.x + tx, nthr = blockDim.x * blockDim.y;
    if (lead) {
        for (int s = 0; s < RP; s++) mbar::init(rg.bars + s, 1);
        mbar::fence_init();
    }
    __syncthreads();
    const int nitems = BATCH ? p.nmem * p.tiles_x * p.tiles_y : 1;
    unsigned qb = 0;
    for (int item = BATCH ? (int)blockIdx.x : 0; item < nitems; item += BATCH ? (int)gridDim.x : 1) {
    int bx, by, mi = 0;
    if (BATCH) {
        const int tpm = p.tiles_x * p.tiles_y;
        mi = item / tpm;
        const int t = item - mi * tpm;
        by = t / p.tiles_x;
        bx = t - by * p.tiles_x;
        // a problem none of whose systems takes this iteration: no copies,
        // no stores, no arrival (the same decision in every CTA)
        if (p.sys && batch_frozen(p.sys, p.mem[mi].prob)) continue;
    } else {
        bx = blockIdx.x;
        by = blockIdx.y;
    }
    const BatchMember* M = BATCH ? p.mem + mi : nullptr;
    const int cmi = BATCH ? M->cmem : 0;
    const int I0 = 1 + bx * WC, J0 = 1 + by * p.hc;
    const int x0 = 2 * I0 - 10, xc0 = I0 - 5;
    rg.q0 = J0 - 2;
    rg.qb = qb;
    const int npairs = p.hc + 2;
    auto issue = [&](int q) {
        const int s = (int)((qb + (unsigned)q) % (unsigned)RP), Jp = rg.q0 + q;
        uint64_t* bar = rg.bars + s;
        mbar::expect_tx(bar, txb);
        if constexpr (BATCH) {
            // vector maps group 8 nodes x NR values (fine rows; x0 is a
            // multiple of 8) or 4 nodes (the coarse row; xc0 a multiple of 4)
            // into their innermost dimension
            tma4d(rg.pA + s * L.sA, &tmA, bar, x0, 2 * Jp + 1, 0, mi);
            tma4d(rg.pF + s * L.sF, &tmF, bar, 0, x0 / 8, 2 * Jp + 1, mi);
            tma4d(rg.pXp + s * L.sXp, &tmX, bar, 0, x0 / 8, 2 * Jp + 1, mi);
            tma4d(rg.pC + s * L.sC, &tmC, bar, 0, xc0 / 4, Jp + 1, cmi);
        } else {
            tma3d(rg.pA + s * L.sA, &tmA, bar, x0, 2 * Jp + 1, 0);
            tma2d(rg.pF + s * L.sF, &tmF, bar, x0, 2 * Jp + 1);
            tma2d(rg.pXp + s * L.sXp, &tmX, bar, x0, 2 * Jp + 1);
            tma2d(rg.pC + s * L.sC, &tmC, bar, xc0, Jp + 1);
        }
    };
    int issued = npairs < RP ? npairs : RP, waited = 0;
    if (lead)
        for (int q = 0; q < issued; q++) issue(q);

    const int ce = 2 * tx, co = ce + 1;
    const int ie = x0 + ce;
    const bool ve = ce >= 1 && ce <= WW - 2 && ie >= 1 && ie <= nf - 2;
    const bool vo = co <= WW - 2 && ie + 1 >= 1 && ie + 1 <= nf - 2;
    const bool own_e = ve && ce >= 9 && ce < 9 + 2 * WC;
    const bool own_o = vo && co >= 9 && co < 9 + 2 * WC;
    const int I = xc0 + tx;                      // coarse column of the thread's column pair
    const bool vI = I >= 0 && I <= nc - 1;
    auto inrow = [&](int j) { return j >= 1 && j <= nf - 2; };
    using XA = SRow<V, WC + 8>;
    auto X = [&](int j) { return XA{sX + (int)((unsigned)j % XR) * WW}; };
    auto rows = [&](int j) {
        return Rows<T, V, XA>{rg.A(j), rg.A(j + 1), rg.A(j - 1), X(j), X(j + 1), X(j - 1), PL};
    };
    const T* Pg = BATCH ? (const T*)M->P : (const T*)p.P;
    VO* out = (VO*)(BATCH ? M->x[p.parity] : p.x);
    // finest level of the refinement mode only
    const VZ* zold = (const VZ*)(BATCH ? M->zold[p.parity] : p.zold);
    AccN<NR> rz, rzo;
    const V z0 = vzero<V>();
    auto pw = [&](int plane, int Jc) -> T {
        return (vI && Jc >= 0 && Jc <= nc - 1) ? Pg[plane * p.plc + (long long)Jc * p.ldc + I] : (T)0;
    };

    // corrected iterate x_pre + P x_c of the thread's two columns of row j,
    // weights w (even row: PXL, PXR of coarse row j/2; odd row: PYS, PYN,
    // PSW, PSE, PNW, PNE of coarse row (j-1)/2)
    auto corr_even = [&](int j, T wxl, T wxr) {
        const bool rj = inrow(j);
        const RowV<const V> C0 = rg.C(j >> 1);
        const RowV<const V> xp = rg.Xp(j);
        const XA x = X(j);
        x[ce] = (ve && rj) ? xp[ce] + C0[tx] : z0;
        x[co] = (vo && rj) ? xp[co] + wxl * C0[tx] + wxr * C0[tx + 1] : z0;
    };
    auto corr_odd = [&](int j, const T* wy) {
        const bool rj = inrow(j);
        const RowV<const V> C0 = rg.C(j >> 1);
        const RowV<const V> C1 = rg.C((j >> 1) + 1);
        const RowV<const V> xp = rg.Xp(j);
        const XA x = X(j);
        x[ce] = (ve && rj) ? xp[ce] + wy[0] * C0[tx] + wy[1] * C1[tx] : z0;
        x[co] = (vo && rj) ? xp[co] + wy[2] * C0[tx] + wy[3] * C0[tx + 1] + wy[4] * C1[tx] + wy[5] * C1[tx + 1]
                           : z0;
    };
    auto gs = [&](int j, int c, bool v) {      // one Gauss-Seidel update
        if (!(v && inrow(j))) return;
        const Rows<T, V, XA> r = rows(j);
        X(j)[c] = divide(vcast<V>(rg.F(j)[c]) - r.offdiag(c), r.diag(c));
    };

    bool ok = wait_pairs<RP>(rg.bars, qb, qb + 2);
    waited = ok ? 2 : 0;
    if (ok) {   // pre-roll: corrected rows 2J0-2 .. 2J0, odd row 2J0-1 smoothed
        if (ty == 0) {
            const int Jm = J0 - 1;
            const T wy[6] = {pw(PYS, Jm), pw(PYN, Jm), pw(PSW, Jm), pw(PSE, Jm), pw(PNW, Jm), pw(PNE, Jm)};
            corr_even(2 * J0 - 2, pw(PXL, Jm), pw(PXR, Jm));
            corr_odd(2 * J0 - 1, wy);
            corr_even(2 * J0, pw(PXL, J0), pw(PXR, J0));
        }
        __syncthreads();
        if (ty == 0) gs(2 * J0 - 1, co, vo);     // colour 3
        __syncthreads();
        if (ty == 0) gs(2 * J0 - 1, ce, ve);     // colour 2
        __syncthreads();
    }
    // weights for the corrected values of this thread's rows, loaded one step ahead
    T wy[6], wxl, wxr;
    auto load_w = [&](int Jp) {
        wy[0] = pw(PYS, Jp);
        wy[1] = pw(PYN, Jp);
        wy[2] = pw(PSW, Jp);
        wy[3] = pw(PSE, Jp);
        wy[4] = pw(PNW, Jp);
        wy[5] = pw(PNE, Jp);
        wxl = pw(PXL, Jp + 1);
        wxr = pw(PXR, Jp + 1);
    };
    load_w(J0 + ty);
    // previous preconditioned residual at this thread's stored nodes of the
    // rows 2Jp-1, 2Jp, also loaded one step ahead (refinement mode only)
    const VZ zz = vzero<VZ>();
    VZ zo_nx[2][2] = {{zz, zz}, {zz, zz}};
    auto load_zo = [&](int Jp) {
        for (int rr = 0; rr < 2; rr++) {
            const int j = 2 * Jp - 1 + rr;
            const long long o = (long long)j * p.ldf + ie;
            const bool rj = inrow(j);
            zo_nx[rr][0] = (rj && own_e) ? zold[o] : zz;
            zo_nx[rr][1] = (rj && own_o) ? zold[o + 1] : zz;
        }
    };
    if (zold) load_zo(J0 + ty);
    for (int J = J0; ok && J < J0 + p.hc; J += K) {
        const int qa = J - rg.q0;
        const int Jp = J + ty, jm = 2 * Jp, jo = jm + 1, je = jm + 2;
        ok = wait_pairs<RP>(rg.bars, qb + qa, qb + qa + K);
        if (!ok) break;
        waited = qa + K;
        // every thread is past the previous step: refill the freed slots
        // (a step reads pairs qa - 1 .. qa + K - 1, so pairs up to qa - 2 are
        // done) with the pairs D ahead
        const int lim = min(npairs, qa - 1 + RP);
        if (lead)
            for (int q = issued; q < lim; q++) issue(q);
        issued = max(issued, lim);
        corr_odd(jo, wy);
        corr_even(je, wxl, wxr);
        load_w(Jp + K);
        VZ zo_now[2][2] = {{zo_nx[0][0], zo_nx[0][1]}, {zo_nx[1][0], zo_nx[1][1]}};
        if (zold) load_zo(Jp + K);
        __syncthreads();
        gs(jo, co, vo);      // colour 3
        __syncthreads();
        gs(jo, ce, ve);      // colour 2
        __syncthreads();
        gs(jm, co, vo);      // colour 1
        __syncthreads();
        gs(jm, ce, ve);      // colour 0
        // right-hand side of the stored rows, read while their ring slots
        // cannot yet be refilled (the next refill follows the next barrier)
        VZ fr[2][2] = {{zz, zz}, {zz, zz}};
        if (zold)
            for (int rr = 0; rr < 2; rr++) {
                const RowV<const typename Ring<T, TF, K, true, NR>::VF> Fr = rg.F(jm - 1 + rr);
                fr[rr][0] = vcast<VZ>(Fr[ce]);
                fr[rr][1] = vcast<VZ>(Fr[co]);
            }
        __syncthreads();
        for (int rr = 0; rr < 2; rr++) {
            const int j = jm - 1 + rr;
            if (!inrow(j)) continue;
            const XA Xr = X(j);
            const long long o = (long long)j * p.ldf + ie;
            if (own_e) out[o] = vcast<VO>(Xr[ce]);
            if (own_o) out[o + 1] = vcast<VO>(Xr[co]);
            if (zold) {
                if (own_e) {
                    rz.add(fr[rr][0], vcast<VZ>(Xr[ce]));
                    rzo.add(fr[rr][0], zo_now[rr][0]);
                }
                if (own_o) {
                    rz.add(fr[rr][1], vcast<VZ>(Xr[co]));
                    rzo.add(fr[rr][1], zo_now[rr][1]);
                }
            }
        }
    }
    if (!ok) {
        if (lead) {
            set_err(p.st, BMG_ERR_TIMEOUT);
            for (int q = waited; q < issued; q++) {
                const unsigned g = qb + (unsigned)q;
                mbar::wait(rg.bars + (g % RP), (g / RP) & 1u);
            }
        }
        __syncthreads();
        return;
    }
    qb += (unsigned)npairs;
    if (zold) {
        // Deterministic reduction of (r.z, r.z_old) per right-hand side; the
        // last CTA (of the grid, or of the problem's tiles when batched)
        // forms the flexible-CG beta.  Every copy into the rings has
        // completed, so after the barrier the A ring is free to hold the
        // per-thread sums.
        double* red = (double*)rg.pA;
        int* last = (int*)(red + 2 * nthr);
        // sums of v1 / v2 over the CTA's threads in a fixed order; valid in thread 0
        auto block_sum2 = [&](double v1, double v2, double& s1, double& s2) {
            __syncthreads();
            red[tid] = v1;
            red[nthr + tid] = v2;
            __syncthreads();
            if (tid < 32) {     // warp 0: strided partial sums, then a fixed shuffle tree
                double a1 = 0.0, a2 = 0.0;
                for (int k = tid; k < nthr; k += 32) {
                    a1 += red[k];
                    a2 += red[nthr + k];
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a1 += __shfl_down_sync(0xffffffffu, a1, o);
                    a2 += __shfl_down_sync(0xffffffffu, a2, o);
                }
                s1 = a1;
                s2 = a2;
            }
        };
        double b1[NR], b2[NR];
        for (int r = 0; r < NR; r++) block_sum2(rz.a[r].value(), rzo.a[r].value(), b1[r], b2[r]);
        if constexpr (!BATCH) {
            const int nb = gridDim.x * gridDim.y;
            if (tid == 0) {
                const int bid = blockIdx.y * gridDim.x + blockIdx.x;
                p.partials[2 * bid] = b1[0];
                p.partials[2 * bid + 1] = b2[0];
                __threadfence();
                *last = atomicAdd(&p.st->counter[6], 1u) == (unsigned)nb - 1;
            }
            __syncthreads();
            if (*last) {
                __threadfence();
                double v1 = 0.0, v2 = 0.0;
                for (int k = tid; k < nb; k += nthr) {
                    v1 += ((volatile double*)p.partials)[2 * k];
                    v2 += ((volatile double*)p.partials)[2 * k + 1];
                }
                double t1 = 0.0, t2 = 0.0;
                block_sum2(v1, v2, t1, t2);
                if (tid == 0) {
                    p.st->counter[6] = 0u;
                    KState* st = p.st;
                    if (st->first) {
                        st->beta = 0.0;
                        st->first = 0;
                    } else {
                        st->beta = (t1 - t2) / st->rz;
                    }
                    st->rz = t1;
                }
            }
        } else {
            const int tpm = p.tiles_x * p.tiles_y;
            double* part = p.partials + (M->part + (by * p.tiles_x + bx)) * 2 * NR;
            if (tid == 0) {
                for (int r = 0; r < NR; r++) {
                    part[2 * r] = b1[r];
                    part[2 * r + 1] = b2[r];
                }
                __threadfence();
                *last = atomicAdd(&p.counters[M->prob], 1u) == (unsigned)tpm - 1;
            }
            __syncthreads();
            if (*last) {
                __threadfence();
                // fixed-order sums over the problem's tiles, per right-hand side
                const double* base_p = p.partials + M->part * 2 * NR;
                double v1[NR], v2[NR];
                for (int r = 0; r < NR; r++) v1[r] = v2[r] = 0.0;
                for (int k = tid; k < tpm; k += nthr)
                    for (int r = 0; r < NR; r++) {
                        v1[r] += ((volatile const double*)base_p)[(long long)k * 2 * NR + 2 * r];
                        v2[r] += ((volatile const double*)base_p)[(long long)k * 2 * NR + 2 * r + 1];
                    }
                double t1[NR], t2[NR];
                for (int r = 0; r < NR; r++) block_sum2(v1[r], v2[r], t1[r], t2[r]);
                if (tid == 0) {
                    for (int r = 0; r < NR; r++) {
                        SysState& sy = p.sys[(long long)M->prob * NR + r];
                        const bool live = sy.active && sy.left > 0;
                        if (live && sy.first) {
                            sy.beta = 0.0;
                            sy.first = 0;
                            sy.rz0 = t1[r];
                        } else if (!live || !(sy.rz != 0.0)) {
                            sy.beta = 0.0;
                        } else {
                            sy.beta = (t1[r] - t2[r]) / sy.rz;
                        }
                        if (live) {
                            sy.rz = t1[r];
                            // the run's goal reached (r.z fell by the factor
                            // the host set): the system stops before this
                            // iteration's update and waits for the refinement
                            if (sy.stop > 0.0 && !(t1[r] > sy.stop * sy.rz0)) sy.left = 0;
                        }
                    }
                    p.counters[M->prob] = 0u;
                }
            }
        }
    }
    if (BATCH) __syncthreads();   // the next item's copies reuse the ring and the rows
    }
}

// ------------------------------------------------------------------ host side
template <typename T>
// Row pairs per step, 2 in both precisions.  Measured on the 4097^2
// refinement-mode solve (autotuned strips): FP32 with 2 pairs (rings of 6
// slots, 4 CTAs per SM) took 3.52 / 2.61 ms per solve in the up / down
// kernels, against 3.69 / 2.75 with 3 pairs (3 CTAs per SM), 4.20 / 2.97
// with 4 and 3.83 / 2.79 with 1.
constexpr int k_of() { return sizeof(T) == 4 ? 2 : 2; }

template <typename T, typename TF>
int down_smem(int wc) { return Lay<T, TF, k_of<T>(), false>(wc).bytes(); }
template <typename T, typename TF>
int up_smem(int wc) { return Lay<T, TF, k_of<T>(), true>(wc).bytes(); }

// The strip widths the kernels are built for (multiples of 8 up to 64, so
// that the TMA x coordinates stay 16-byte aligned); f(integral_constant<W>).
template <class F>
bmg_status with_wc(int wc, F&& f) {
    switch (wc) {
        case 8: return f(std::integral_constant<int, 8>{});
        case 16: return f(std::integral_constant<int, 16>{});
        case 24: return f(std::integral_constant<int, 24>{});
        case 32: return f(std::integral_constant<int, 32>{});
        case 40: return f(std::integral_constant<int, 40>{});
        case 48: return f(std::integral_constant<int, 48>{});
        case 56: return f(std::integral_constant<int, 56>{});
        case 64: return f(std::integral_constant<int, 64>{});
        default: return BMG_ERR_ARG;
    }
}

template <typename T, typename TF>
bmg_status launch_down(Ctx& c, const FusedLevel& F, cudaStream_t s) {
    return with_wc(F.wc, [&](auto W) {
        auto kern = k_vdown2d<T, TF, k_of<T>(), decltype(W)::value>;
        const int smem = down_smem<T, TF>(F.wc);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return BMG_ERR_DEVICE;
        kern<<<dim3(F.tiles_x, F.tiles_y), dim3(F.wc + 8, k_of<T>()), smem, s>>>(F.mA, F.mF, F.down);
        c.launches++;
        return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
    });
}

template <typename T, typename TF, typename TO>
bmg_status launch_up(Ctx& c, const FusedLevel& F, cudaStream_t s, void* out, const void* zold = nullptr) {
    return with_wc(F.wc, [&](auto W) {
        auto kern = k_vup2d<T, TF, TO, k_of<T>(), decltype(W)::value>;
        const int smem = up_smem<T, TF>(F.wc);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return BMG_ERR_DEVICE;
        FusedArgs a = F.up;
        a.x = out;
        a.zold = zold;
        a.partials = zold ? c.partials : nullptr;
        kern<<<dim3(F.tiles_x, F.tiles_y_up), dim3(F.wc + 8, k_of<T>()), smem, s>>>(F.mA, F.mF, F.mXp, F.mXc, a);
        c.launches++;
        return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
    });
}

template <typename T, typename TF, typename TO>
bmg_status occupancy(int wc, int* down_blocks, int* up_blocks) {
    return with_wc(wc, [&](auto W) {
        constexpr int w = decltype(W)::value;
        auto kd = k_vdown2d<T, TF, k_of<T>(), w>;
        auto ku = k_vup2d<T, TF, TO, k_of<T>(), w>;
        const int sd = down_smem<T, TF>(wc), su = up_smem<T, TF>(wc);
        const int nt = (wc + 8) * k_of<T>();
        if (cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, sd) != cudaSuccess ||
            cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, su) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(down_blocks, kd, nt, sd) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(up_blocks, ku, nt, su) != cudaSuccess)
            return BMG_ERR_DEVICE;
        return BMG_OK;
    });
}

// Batched kernels: FP32, kBatchR right-hand sides, kBatchK row pairs per
// step, strip widths 16 or 32 coarse columns.
template <class F>
bmg_status with_batch_wc(int wc, F&& f) {
    switch (wc) {
        case 16: return f(std::integral_constant<int, 16>{});
        case 32: return f(std::integral_constant<int, 32>{});
        default: return BMG_ERR_ARG;
    }
}

}  // namespace

int batch_down_smem(int wc) { return Lay<float, float, kBatchK, false, kBatchR>(wc).bytes(); }
int batch_up_smem(int wc) { return Lay<float, float, kBatchK, true, kBatchR>(wc).bytes(); }

bmg_status batch_occupancy(int wc, int* down_blocks, int* up_blocks) {
    return with_batch_wc(wc, [&](auto W) {
        constexpr int w = decltype(W)::value;
        auto kd = k_vdown2d<float, float, kBatchK, w, kBatchR, true>;
        auto ku = k_vup2d<float, float, float, kBatchK, w, kBatchR, true>;
        const int sd = batch_down_smem(wc), su = batch_up_smem(wc);
        const int nt = (wc + 8) * kBatchK;
        if (cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, sd) != cudaSuccess ||
            cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, su) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(down_blocks, kd, nt, sd) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(up_blocks, ku, nt, su) != cudaSuccess)
            return BMG_ERR_DEVICE;
        return BMG_OK;
    });
}

// One persistent launch over the work-list of a size class (grid CTAs).
bmg_status batch_down(const CUtensorMap& mA, const CUtensorMap& mF, const FusedArgs& a, int grid,
                      cudaStream_t s) {
    return with_batch_wc(a.wc, [&](auto W) {
        auto kern = k_vdown2d<float, float, kBatchK, decltype(W)::value, kBatchR, true>;
        const int smem = batch_down_smem(a.wc);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return BMG_ERR_DEVICE;
        kern<<<grid, dim3(a.wc + 8, kBatchK), smem, s>>>(mA, mF, a);
        return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
    });
}

bmg_status batch_up(const CUtensorMap& mA, const CUtensorMap& mF, const CUtensorMap& mXp, const CUtensorMap& mXc,
                    const FusedArgs& a, int grid, cudaStream_t s) {
    return with_batch_wc(a.wc, [&](auto W) {
        auto kern = k_vup2d<float, float, float, kBatchK, decltype(W)::value, kBatchR, true>;
        const int smem = batch_up_smem(a.wc);
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return BMG_ERR_DEVICE;
        kern<<<grid, dim3(a.wc + 8, kBatchK), smem, s>>>(mA, mF, mXp, mXc, a);
        return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
    });
}

int fused_rows_per_step(bool f32) { return f32 ? k_of<float>() : k_of<double>(); }

int fused_down_smem(bool f32, bool f64in, int wc) {
    if (!f32) return down_smem<double, double>(wc);
    return f64in ? down_smem<float, double>(wc) : down_smem<float, float>(wc);
}

int fused_up_smem(bool f32, bool f64in, int wc) {
    if (!f32) return up_smem<double, double>(wc);
    return f64in ? up_smem<float, double>(wc) : up_smem<float, float>(wc);
}

bmg_status fused_occupancy(bool f32, bool f64in, int wc, int* down_blocks, int* up_blocks) {
    if (!f32) return occupancy<double, double, double>(wc, down_blocks, up_blocks);
    if (f64in) return occupancy<float, double, double>(wc, down_blocks, up_blocks);
    return occupancy<float, float, float>(wc, down_blocks, up_blocks);
}

bmg_status fused_down(Ctx& c, int l, bool ir) {
    const FusedLevel& F = (ir && l == 0) ? c.fused_ir0 : c.fused[l];
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    if (!f32) return launch_down<double, double>(c, F, c.stream);
    if (l == 0 && !ir) return launch_down<float, double>(c, F, c.stream);
    return launch_down<float, float>(c, F, c.stream);
}

bmg_status fused_up(Ctx& c, int l, void* out, bool ir, const float* zold) {
    const FusedLevel& F = (ir && l == 0) ? c.fused_ir0 : c.fused[l];
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    if (!f32) return launch_up<double, double, double>(c, F, c.stream, out);
    if (l == 0 && !ir) return launch_up<float, double, double>(c, F, c.stream, out);
    return launch_up<float, float, float>(c, F, c.stream, out, (ir && l == 0) ? zold : nullptr);
}

}  // namespace bmg
