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
// dependencies.  Rows arrive by TMA (cp.async.bulk.tensor) into a ring of
// RP row-pair slots, each completed by an mbarrier with an expected byte
// count, prefetched RP-3 pairs ahead; one thread issues all copies.  Every
// mbarrier wait is bounded by the global timer; on expiry the CTA records
// BMG_ERR_TIMEOUT, drains its outstanding copies (bounded) and returns.
#include <cuda.h>

#include "common.cuh"
#include "fused2d.cuh"

namespace bmg {
namespace {

constexpr int kNT = 128;                      // threads per CTA
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try(b, parity))
        if (gtimer() - t0 > kWaitNs) return false;
    return true;
}

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


// ------------------------------------------------------------------ down
template <typename T, typename TF, int RP>
struct DownSmem {
    int WW, WWc, sA, sF, sP;   // slot strides in bytes
    __host__ __device__ DownSmem(int wc) {
        WW = 2 * wc + 16;
        WWc = wc + 8;
        sA = (10 * WW * (int)sizeof(T) + 127) & ~127;
        sF = (2 * WW * (int)sizeof(TF) + 127) & ~127;
        sP = (8 * WWc * (int)sizeof(T) + 127) & ~127;
    }
    __host__ __device__ int bytes() const {
        return RP * (sA + sF + sP) + 8 * WW * (int)sizeof(T) + 4 * WW * (int)sizeof(T) + RP * 8 + 128;
    }
};

template <typename T, typename TF, int RP>
__global__ void __launch_bounds__(kNT) k_vdown2d(const __grid_constant__ CUtensorMap tmA,
                                                 const __grid_constant__ CUtensorMap tmF,
                                                 const __grid_constant__ CUtensorMap tmP, FusedArgs p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const DownSmem<T, TF, RP> L(p.wc);
    const int WW = L.WW, WWc = L.WWc;
    unsigned char* base = (unsigned char*)(((uintptr_t)smem + 127) & ~(uintptr_t)127);
    unsigned char* pA = base;
    unsigned char* pF = pA + RP * L.sA;
    unsigned char* pP = pF + RP * L.sF;
    T* sX = (T*)(pP + RP * L.sP);
    T* sR = sX + 8 * WW;
    uint64_t* bars = (uint64_t*)(((uintptr_t)(sR + 4 * WW) + 7) & ~(uintptr_t)7);
    const int tid = threadIdx.x;
    const int I0 = 1 + blockIdx.x * p.wc, J0 = 1 + blockIdx.y * p.hc;
    const int x0 = 2 * I0 - 10, xc0 = I0 - 5;
    const int q0 = J0 - 2, npairs = p.hc + 2;
    const int nf = p.nf, nc = p.nc;
    const uint32_t tx_bytes = (uint32_t)(10 * WW * sizeof(T) + 2 * WW * sizeof(TF) + 8 * WWc * sizeof(T));

    auto issue = [&](int q) {
        const int s = q % RP, Jp = q0 + q;
        uint64_t* bar = bars + s;
        mbar_expect_tx(bar, tx_bytes);
        tma3d(pA + s * L.sA, &tmA, bar, x0, 2 * Jp + 1, 0);
        tma2d(pF + s * L.sF, &tmF, bar, x0, 2 * Jp + 1);
        tma3d(pP + s * L.sP, &tmP, bar, xc0, Jp + 1, 0);
    };
    if (tid == 0) {
        for (int s = 0; s < RP; s++) mbar_init(bars + s, 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = 0, waited = 0;
    if (tid == 0)
        for (; issued < RP && issued < npairs; issued++) issue(issued);
    issued = min(RP, npairs);

    // accessors -------------------------------------------------------
    auto slotA = [&](int j) -> const T* {       // fine row j -> its stencil row (plane 0)
        const int q = ((j - 1) >> 1) - q0;
        return (const T*)(pA + (q % RP) * L.sA) + ((j - 1) & 1) * WW;
    };
    auto Fr = [&](int j) -> const TF* {
        const int q = ((j - 1) >> 1) - q0;
        return (const TF*)(pF + (q % RP) * L.sF) + ((j - 1) & 1) * WW;
    };
    auto Pr = [&](int J) -> const T* {          // coarse row J of P (plane 0)
        const int q = J - 1 - q0;
        return (const T*)(pP + (q % RP) * L.sP);
    };
    auto Xr = [&](int j) -> T* { return sX + (j & 7) * WW; };
    auto Rr = [&](int j) -> T* { return sR + (j & 3) * WW; };
    const int PL = 2 * WW;  // plane stride inside a stencil slot
    auto inrow = [&](int j) { return j >= 1 && j <= nf - 2; };
    auto incol = [&](int c) { const int i = x0 + c; return c >= 1 && c <= WW - 2 && i >= 1 && i <= nf - 2; };

    bool ok = true;
    auto wait_pair = [&](int q) {
        bool mine = mbar_wait(bars + (q % RP), (uint32_t)((q / RP) & 1));
        ok = __syncthreads_and(mine) != 0;
        waited = q + 1;
    };

    // even row j: colour 0 (even c) then colour 1 (odd c); zero initial guess
    auto even_row = [&](int j) {
        const T* A = slotA(j);
        const TF* F = Fr(j);
        T* X = Xr(j);
        const bool rj = inrow(j);
        for (int c = 2 * tid; c < WW; c += 2 * kNT)
            X[c] = (rj && incol(c)) ? (T)F[c] / A[C2 * PL + c] : (T)0;
        __syncthreads();
        for (int c = 2 * tid + 1; c < WW; c += 2 * kNT) {
            T v = 0;
            if (rj && incol(c)) {
                const T s = (T)F[c] - A[W2 * PL + c] * X[c - 1] - A[W2 * PL + c + 1] * X[c + 1];
                v = s / A[C2 * PL + c];
            }
            X[c] = v;
        }
    };
    // odd row j: colour 2 (even c) then colour 3 (odd c)
    auto odd_row = [&](int j) {
        const T* A = slotA(j);
        const T* An = slotA(j + 1);
        const T* As = slotA(j - 1);
        const TF* F = Fr(j);
        T* X = Xr(j);
        const T* Xs = Xr(j - 1);
        const T* Xn = Xr(j + 1);
        const bool rj = inrow(j);
        for (int c = 2 * tid; c < WW; c += 2 * kNT) {
            T v = 0;
            if (rj && incol(c)) {
                T s = (T)F[c];
                s -= A[S2 * PL + c] * Xs[c];
                s -= An[S2 * PL + c] * Xn[c];
                s -= A[SW2 * PL + c] * Xs[c - 1];
                s -= An[SW2 * PL + c + 1] * Xn[c + 1];
                s -= A[NW2 * PL + c] * Xn[c - 1];
                s -= As[NW2 * PL + c + 1] * Xs[c + 1];
                v = s / A[C2 * PL + c];
            }
            X[c] = v;
        }
        __syncthreads();
        for (int c = 2 * tid + 1; c < WW; c += 2 * kNT) {
            T v = 0;
            if (rj && incol(c)) {
                T s = (T)F[c];
                s -= A[W2 * PL + c] * X[c - 1];
                s -= A[W2 * PL + c + 1] * X[c + 1];
                s -= A[S2 * PL + c] * Xs[c];
                s -= An[S2 * PL + c] * Xn[c];
                s -= A[SW2 * PL + c] * Xs[c - 1];
                s -= An[SW2 * PL + c + 1] * Xn[c + 1];
                s -= A[NW2 * PL + c] * Xn[c - 1];
                s -= As[NW2 * PL + c + 1] * Xs[c + 1];
                v = s / A[C2 * PL + c];
            }
            X[c] = v;
        }
    };
    // residual of row j; the last colour (odd, odd) has zero residual by construction
    auto resid_row = [&](int j) {
        const T* A = slotA(j);
        const T* An = slotA(j + 1);
        const T* As = slotA(j - 1);
        const TF* F = Fr(j);
        const T* X = Xr(j);
        const T* Xs = Xr(j - 1);
        const T* Xn = Xr(j + 1);
        T* R = Rr(j);
        const bool rj = inrow(j);
        const bool oddj = j & 1;
        for (int c = tid; c < WW; c += kNT) {
            T v = 0;
            if (rj && incol(c) && !(oddj && (c & 1))) {
                T s = (T)F[c] - A[C2 * PL + c] * X[c];
                s -= A[W2 * PL + c] * X[c - 1];
                s -= A[W2 * PL + c + 1] * X[c + 1];
                s -= A[S2 * PL + c] * Xs[c];
                s -= An[S2 * PL + c] * Xn[c];
                s -= A[SW2 * PL + c] * Xs[c - 1];
                s -= An[SW2 * PL + c + 1] * Xn[c + 1];
                s -= A[NW2 * PL + c] * Xn[c - 1];
                s -= As[NW2 * PL + c + 1] * Xs[c + 1];
                v = s;
            }
            R[c] = v;
        }
    };

    T* xg = (T*)p.x;
    T* bcg = (T*)p.bc;
    const int cown0 = 9, cown1 = 9 + 2 * p.wc;

    // pre-roll: rows 2J0-2 .. 2J0 final, residual of row 2J0-1
    wait_pair(0);
    if (ok) wait_pair(1);
    if (ok) {
        even_row(2 * J0 - 2);
        __syncthreads();
        even_row(2 * J0);
        __syncthreads();
        odd_row(2 * J0 - 1);
        __syncthreads();
        resid_row(2 * J0 - 1);
        __syncthreads();
    }
    for (int J = J0; ok && J < J0 + p.hc; J++) {
        wait_pair(J - q0);
        if (!ok) break;
        even_row(2 * J + 2);
        __syncthreads();
        odd_row(2 * J + 1);
        __syncthreads();
        resid_row(2 * J);
        resid_row(2 * J + 1);
        __syncthreads();
        // restriction b_c(I, J) = sum_i P(i,(I,J)) r_i
        if (J <= nc - 2) {
            const T* Pj = Pr(J);
            const T* Pm = Pr(J - 1);
            const T* R0 = Rr(2 * J);
            const T* Rs = Rr(2 * J - 1);
            const T* Rn = Rr(2 * J + 1);
            for (int cc = 5 + tid; cc < 5 + p.wc; cc += kNT) {
                const int I = xc0 + cc;
                if (I < 1 || I > nc - 2) continue;
                const int c = 2 * cc;
                T b = R0[c];
                b += Pj[PXR * WWc + cc - 1] * R0[c - 1];
                b += Pj[PXL * WWc + cc] * R0[c + 1];
                b += Pm[PYN * WWc + cc] * Rs[c];
                b += Pj[PYS * WWc + cc] * Rn[c];
                b += Pm[PNE * WWc + cc - 1] * Rs[c - 1];
                b += Pm[PNW * WWc + cc] * Rs[c + 1];
                b += Pj[PSE * WWc + cc - 1] * Rn[c - 1];
                b += Pj[PSW * WWc + cc] * Rn[c + 1];
                bcg[(long long)J * p.ldc + I] = b;
            }
        }
        // finished rows 2J-1, 2J of the owned columns
        for (int r = 0; r < 2; r++) {
            const int j = 2 * J - 1 + r;
            if (!inrow(j)) continue;
            const T* X = Xr(j);
            for (int c = cown0 + tid; c < cown1; c += kNT) {
                const int i = x0 + c;
                if (i >= 1 && i <= nf - 2) xg[(long long)j * p.ldf + i] = X[c];
            }
        }
        __syncthreads();
        if (tid == 0 && J - J0 + RP < npairs) issue(J - J0 + RP);
        issued = min(npairs, J - J0 + RP + 1) > issued ? min(npairs, J - J0 + RP + 1) : issued;
    }
    if (!ok) {
        if (tid == 0) {
            set_err(p.st, BMG_ERR_TIMEOUT);
            for (int q = waited; q < issued; q++) mbar_wait(bars + (q % RP), (uint32_t)((q / RP) & 1));
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ up
template <typename T, typename TF, int RP>
struct UpSmem {
    int WW, WWc, sA, sF, sX, sP, sC;
    __host__ __device__ UpSmem(int wc) {
        WW = 2 * wc + 16;
        WWc = wc + 8;
        sA = (10 * WW * (int)sizeof(T) + 127) & ~127;
        sF = (2 * WW * (int)sizeof(TF) + 127) & ~127;
        sX = (2 * WW * (int)sizeof(T) + 127) & ~127;
        sP = (8 * WWc * (int)sizeof(T) + 127) & ~127;
        sC = (WWc * (int)sizeof(T) + 127) & ~127;
    }
    __host__ __device__ int bytes() const {
        return RP * (sA + sF + sX + sP + sC) + 8 * WW * (int)sizeof(T) + RP * 8 + 128;
    }
};

template <typename T, typename TF, typename TO, int RP>
__global__ void __launch_bounds__(kNT) k_vup2d(const __grid_constant__ CUtensorMap tmA,
                                               const __grid_constant__ CUtensorMap tmF,
                                               const __grid_constant__ CUtensorMap tmX,
                                               const __grid_constant__ CUtensorMap tmP,
                                               const __grid_constant__ CUtensorMap tmC, FusedArgs p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const UpSmem<T, TF, RP> L(p.wc);
    const int WW = L.WW, WWc = L.WWc;
    unsigned char* pA = (unsigned char*)(((uintptr_t)smem + 127) & ~(uintptr_t)127);
    unsigned char* pF = pA + RP * L.sA;
    unsigned char* pXp = pF + RP * L.sF;
    unsigned char* pP = pXp + RP * L.sX;
    unsigned char* pC = pP + RP * L.sP;
    T* sX = (T*)(pC + RP * L.sC);
    uint64_t* bars = (uint64_t*)(((uintptr_t)(sX + 8 * WW) + 7) & ~(uintptr_t)7);
    const int tid = threadIdx.x;
    const int I0 = 1 + blockIdx.x * p.wc, J0 = 1 + blockIdx.y * p.hc;
    const int x0 = 2 * I0 - 10, xc0 = I0 - 5;
    const int q0 = J0 - 2, npairs = p.hc + 2;
    const int nf = p.nf;
    const uint32_t tx_bytes =
        (uint32_t)(10 * WW * sizeof(T) + 2 * WW * sizeof(TF) + 2 * WW * sizeof(T) + 8 * WWc * sizeof(T) +
                   WWc * sizeof(T));

    auto issue = [&](int q) {
        const int s = q % RP, Jp = q0 + q;
        uint64_t* bar = bars + s;
        mbar_expect_tx(bar, tx_bytes);
        tma3d(pA + s * L.sA, &tmA, bar, x0, 2 * Jp + 1, 0);
        tma2d(pF + s * L.sF, &tmF, bar, x0, 2 * Jp + 1);
        tma2d(pXp + s * L.sX, &tmX, bar, x0, 2 * Jp + 1);
        tma3d(pP + s * L.sP, &tmP, bar, xc0, Jp + 1, 0);
        tma2d(pC + s * L.sC, &tmC, bar, xc0, Jp + 1);
    };
    if (tid == 0) {
        for (int s = 0; s < RP; s++) mbar_init(bars + s, 1);
        fence_mbar_init();
    }
    __syncthreads();
    int issued = min(RP, npairs), waited = 0;
    if (tid == 0)
        for (int q = 0; q < issued; q++) issue(q);

    auto slotA = [&](int j) -> const T* {
        const int q = ((j - 1) >> 1) - q0;
        return (const T*)(pA + (q % RP) * L.sA) + ((j - 1) & 1) * WW;
    };
    auto Fr = [&](int j) -> const TF* {
        const int q = ((j - 1) >> 1) - q0;
        return (const TF*)(pF + (q % RP) * L.sF) + ((j - 1) & 1) * WW;
    };
    auto XPr = [&](int j) -> const T* {
        const int q = ((j - 1) >> 1) - q0;
        return (const T*)(pXp + (q % RP) * L.sX) + ((j - 1) & 1) * WW;
    };
    auto Pr = [&](int J) -> const T* { return (const T*)(pP + ((J - 1 - q0) % RP) * L.sP); };
    auto Cr = [&](int J) -> const T* { return (const T*)(pC + ((J - 1 - q0) % RP) * L.sC); };
    auto Xr = [&](int j) -> T* { return sX + (j & 7) * WW; };
    const int PL = 2 * WW;
    auto inrow = [&](int j) { return j >= 1 && j <= nf - 2; };
    auto incol = [&](int c) { const int i = x0 + c; return c >= 1 && c <= WW - 2 && i >= 1 && i <= nf - 2; };

    bool ok = true;
    auto wait_pair = [&](int q) {
        bool mine = mbar_wait(bars + (q % RP), (uint32_t)((q / RP) & 1));
        ok = __syncthreads_and(mine) != 0;
        waited = q + 1;
    };

    // corrected iterate of row j: x_pre + P x_c
    auto corrected = [&](int j) {
        const T* Xp = XPr(j);
        T* X = Xr(j);
        const bool rj = inrow(j);
        const int Jc = j >> 1;
        const T* P0 = Pr(Jc);
        const T* C0 = Cr(Jc);
        const T* C1 = Cr(Jc + 1);
        const bool oddj = j & 1;
        for (int c = tid; c < WW; c += kNT) {
            T v = 0;
            if (rj && incol(c)) {
                const int cc = c >> 1;
                T pv;
                if (!(c & 1) && !oddj) {
                    pv = C0[cc];
                } else if ((c & 1) && !oddj) {
                    pv = P0[PXL * WWc + cc] * C0[cc] + P0[PXR * WWc + cc] * C0[cc + 1];
                } else if (!(c & 1) && oddj) {
                    pv = P0[PYS * WWc + cc] * C0[cc] + P0[PYN * WWc + cc] * C1[cc];
                } else {
                    pv = P0[PSW * WWc + cc] * C0[cc] + P0[PSE * WWc + cc] * C0[cc + 1] + P0[PNW * WWc + cc] * C1[cc] +
                         P0[PNE * WWc + cc] * C1[cc + 1];
                }
                v = Xp[c] + pv;
            }
            X[c] = v;
        }
    };
    // Gauss-Seidel update of the nodes of row j with column parity par
    auto gs = [&](int j, int par) {
        const T* A = slotA(j);
        const T* An = slotA(j + 1);
        const T* As = slotA(j - 1);
        const TF* F = Fr(j);
        T* X = Xr(j);
        const T* Xs = Xr(j - 1);
        const T* Xn = Xr(j + 1);
        const bool rj = inrow(j);
        for (int c = 2 * tid + par; c < WW; c += 2 * kNT) {
            if (!(rj && incol(c))) continue;
            T s = (T)F[c];
            s -= A[W2 * PL + c] * X[c - 1];
            s -= A[W2 * PL + c + 1] * X[c + 1];
            s -= A[S2 * PL + c] * Xs[c];
            s -= An[S2 * PL + c] * Xn[c];
            s -= A[SW2 * PL + c] * Xs[c - 1];
            s -= An[SW2 * PL + c + 1] * Xn[c + 1];
            s -= A[NW2 * PL + c] * Xn[c - 1];
            s -= As[NW2 * PL + c + 1] * Xs[c + 1];
            X[c] = s / A[C2 * PL + c];
        }
    };

    TO* out = (TO*)p.x;
    const int cown0 = 9, cown1 = 9 + 2 * p.wc;

    wait_pair(0);
    if (ok) wait_pair(1);
    if (ok) {
        corrected(2 * J0 - 2);
        corrected(2 * J0 - 1);
        corrected(2 * J0);
        __syncthreads();
        gs(2 * J0 - 1, 1);   // colour 3
        __syncthreads();
        gs(2 * J0 - 1, 0);   // colour 2
        __syncthreads();
    }
    for (int J = J0; ok && J < J0 + p.hc; J++) {
        wait_pair(J - q0);
        if (!ok) break;
        corrected(2 * J + 1);
        corrected(2 * J + 2);
        __syncthreads();
        gs(2 * J + 1, 1);    // colour 3
        __syncthreads();
        gs(2 * J + 1, 0);    // colour 2
        __syncthreads();
        gs(2 * J, 1);        // colour 1
        __syncthreads();
        gs(2 * J, 0);        // colour 0
        __syncthreads();
        for (int r = 0; r < 2; r++) {
            const int j = 2 * J - 1 + r;
            if (!inrow(j)) continue;
            const T* X = Xr(j);
            for (int c = cown0 + tid; c < cown1; c += kNT) {
                const int i = x0 + c;
                if (i >= 1 && i <= nf - 2) out[(long long)j * p.ldf + i] = (TO)X[c];
            }
        }
        __syncthreads();
        if (tid == 0 && J - J0 + RP < npairs) issue(J - J0 + RP);
        issued = max(issued, min(npairs, J - J0 + RP + 1));
    }
    if (!ok) {
        if (tid == 0) {
            set_err(p.st, BMG_ERR_TIMEOUT);
            for (int q = waited; q < issued; q++) mbar_wait(bars + (q % RP), (uint32_t)((q / RP) & 1));
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
template <typename T>
constexpr int rp_of() { return sizeof(T) == 4 ? 8 : 6; }

template <typename T, typename TF>
int down_smem(int wc) { return DownSmem<T, TF, rp_of<T>()>(wc).bytes(); }
template <typename T, typename TF>
int up_smem(int wc) { return UpSmem<T, TF, rp_of<T>()>(wc).bytes(); }

template <typename T, typename TF>
bmg_status launch_down(Ctx& c, const FusedLevel& F, cudaStream_t s) {
    auto kern = k_vdown2d<T, TF, rp_of<T>()>;
    const int smem = down_smem<T, TF>(F.wc);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return BMG_ERR_DEVICE;
    dim3 grid(F.tiles_x, F.tiles_y);
    kern<<<grid, kNT, smem, s>>>(F.mA, F.mF, F.mP, F.down);
    c.launches++;
    return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
}

template <typename T, typename TF, typename TO>
bmg_status launch_up(Ctx& c, const FusedLevel& F, cudaStream_t s, void* out) {
    auto kern = k_vup2d<T, TF, TO, rp_of<T>()>;
    const int smem = up_smem<T, TF>(F.wc);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return BMG_ERR_DEVICE;
    dim3 grid(F.tiles_x, F.tiles_y);
    FusedArgs a = F.up;
    a.x = out;
    kern<<<grid, kNT, smem, s>>>(F.mA, F.mF, F.mXp, F.mP, F.mXc, a);
    c.launches++;
    return cudaGetLastError() == cudaSuccess ? BMG_OK : BMG_ERR_DEVICE;
}

}  // namespace

int fused_down_smem(bool f32, bool f64in, int wc) {
    if (!f32) return down_smem<double, double>(wc);
    return f64in ? down_smem<float, double>(wc) : down_smem<float, float>(wc);
}

int fused_up_smem(bool f32, bool f64in, int wc) {
    if (!f32) return up_smem<double, double>(wc);
    return f64in ? up_smem<float, double>(wc) : up_smem<float, float>(wc);
}

bmg_status fused_occupancy(bool f32, bool f64in, int wc, int* down_blocks, int* up_blocks) {
    const int sd = fused_down_smem(f32, f64in, wc), su = fused_up_smem(f32, f64in, wc);
    cudaError_t e1, e2, e3, e4;
    if (!f32) {
        auto kd = k_vdown2d<double, double, rp_of<double>()>;
        auto ku = k_vup2d<double, double, double, rp_of<double>()>;
        e1 = cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, sd);
        e2 = cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, su);
        e3 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(down_blocks, kd, kNT, sd);
        e4 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(up_blocks, ku, kNT, su);
    } else if (f64in) {
        auto kd = k_vdown2d<float, double, rp_of<float>()>;
        auto ku = k_vup2d<float, double, double, rp_of<float>()>;
        e1 = cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, sd);
        e2 = cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, su);
        e3 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(down_blocks, kd, kNT, sd);
        e4 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(up_blocks, ku, kNT, su);
    } else {
        auto kd = k_vdown2d<float, float, rp_of<float>()>;
        auto ku = k_vup2d<float, float, float, rp_of<float>()>;
        e1 = cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, sd);
        e2 = cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, su);
        e3 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(down_blocks, kd, kNT, sd);
        e4 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(up_blocks, ku, kNT, su);
    }
    if (e1 || e2 || e3 || e4) return BMG_ERR_DEVICE;
    return BMG_OK;
}

bmg_status fused_down(Ctx& c, int l) {
    const FusedLevel& F = c.fused[l];
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    if (!f32) return launch_down<double, double>(c, F, c.stream);
    if (l == 0) return launch_down<float, double>(c, F, c.stream);
    return launch_down<float, float>(c, F, c.stream);
}

bmg_status fused_up(Ctx& c, int l, void* out) {
    const FusedLevel& F = c.fused[l];
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    if (!f32) return launch_up<double, double, double>(c, F, c.stream, out);
    if (l == 0) return launch_up<float, double, double>(c, F, c.stream, out);
    return launch_up<float, float, float>(c, F, c.stream, out);
}

}  // namespace bmg
