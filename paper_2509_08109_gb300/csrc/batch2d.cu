// batch2d.cu -- many independent 2-D problems, several right-hand sides
// each, solved together on the device: the batched form of the mixed-
// precision solve (FP64 iterative refinement around an FP32 flexible CG
// preconditioned by the FP32 V-cycle of Sec. 2.2, "Solution phase" step 3),
// one V-cycle per right-hand side per inner iteration.
//
// Layout.  Every problem keeps the hierarchy its own context built
// (bmg_setup).  The batch copies the FP32 operators and interpolation
// weights of every streamed level (n >= 65) into class-contiguous storage:
// all (problem, level) members with the same n form a size class whose
// arrays carry one more dimension, the member, so one TMA tensor map covers
// the class.  Vectors are interleaved, kBatchR values per node (one per
// right-hand side), so each stencil and weight value a kernel stages serves
// every right-hand side.
//
// Work.  One inner iteration of the whole batch is: the down kernels of the
// size classes from the finest down (each a persistent grid walking the
// class's work-list of (member, tile) items), one tail launch (a CTA per
// problem for the levels n <= 33), the up kernels from the coarsest class
// up (the finest members also form each system's flexible-CG beta), the
// batched operator product p = z + beta p_old, q = A p with alpha, and the
// update x += alpha p, r -= alpha q.  That sequence is captured once as a
// CUDA graph (per parity of the alternating z buffers) and replayed.  All
// systems iterate in lockstep; between refinements the host reads every
// system's FP64 residual, retires the converged ones, and gives every
// active system its own number of inner iterations for the next run (the
// single-problem rule); the run lasts as long as the largest, and a system
// whose count is used up, or whose r.z has fallen by the run's goal, freezes
// (no further updates) until the next refinement.  A problem whose systems
// are all frozen is skipped by every batched kernel of the iteration.
//
// Reductions are deterministic: per-tile partial sums, summed in a fixed
// order by the last CTA of each problem (arrival counter per problem).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "common.cuh"

namespace bmg {
namespace {

constexpr int R = kBatchR;
constexpr int kBThreads = 256;                 // batched vector kernels: 64 columns x R
constexpr int kBCols = kBThreads / R;
constexpr int kRowBlocks = 32;                 // blocks per problem of the row-parallel kernels

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

bool dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Stencil planes of a class: (x = column, row, plane, member), box of
// box_x columns, 2 rows, all planes, one member.
bool map_planes(CUtensorMap* m, const float* base, int ld, int n, int planes, long long plane, int members,
                int box_x) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)ld, (cuuint64_t)n, (cuuint64_t)planes, (cuuint64_t)members};
    cuuint64_t strides[3] = {(cuuint64_t)ld * 4, (cuuint64_t)plane * 4, (cuuint64_t)plane * planes * 4};
    cuuint32_t box[4] = {(cuuint32_t)box_x, 2, (cuuint32_t)planes, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Interleaved vectors of a class, viewed as (g nodes x R values, column
// group, row, member) so that the innermost box extent is g * R floats
// (128 bytes for g = 8) rather than one node's R values; box of box_x
// columns (a multiple of g), box_y rows, one member.  The shared-memory
// image is the same as the rows' natural order.
bool map_vec(CUtensorMap* m, const float* base, int ld, int n, long long plane, int members, int box_x, int box_y,
             int g) {
    auto fn = encode_fn();
    if (!fn || box_x % g || ld % g) return false;
    cuuint64_t dims[4] = {(cuuint64_t)g * R, (cuuint64_t)(ld / g), (cuuint64_t)n, (cuuint64_t)members};
    cuuint64_t strides[3] = {(cuuint64_t)g * R * 4, (cuuint64_t)ld * R * 4, (cuuint64_t)plane * R * 4};
    cuuint32_t box[4] = {(cuuint32_t)(g * R), (cuuint32_t)(box_x / g), (cuuint32_t)box_y, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Per-problem view used by the batched vector kernels.
struct BProbDev {
    int n, ld;
    long long plane;
    const double* A64;     // FP64 operator (5 planes)
    const float* A32;      // FP32 finest operator (the class copy, 5 planes)
    const float* rs;       // FP32 row sums of the finest operator (the context's)
    double* x;             // FP64 iterate, R per node
    const double* b;       // FP64 right-hand side, R per node
    float* r;              // FP32 inner residual (the finest member's class right-hand side)
    float* z[2];           // FP32 preconditioned residuals (alternating)
    float* p[2];           // FP32 search directions (alternating)
    float* q;              // FP32 A p
    int sp_tiles_x, sp_tiles;   // tiles of the operator product
    long long sp_part;     // first partial of the operator product
};

// Item of the batched operator product: one tile of one problem.
struct SpItem {
    int prob, tile;
};

// Compensated FP32 accumulator (as in the single-problem kernels).
struct AccB {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Sums v over the threads of each right-hand side (thread t carries
// right-hand side t % R); valid in threads 0 .. R-1.  Fixed order.
__device__ __forceinline__ double block_sum_r(double v, double* red) {
    const int tid = threadIdx.x;
    __syncthreads();
    red[tid] = v;
    __syncthreads();
    double a = 0.0;
    if (tid < 32) {
        for (int k = tid; k < (int)blockDim.x; k += 32) a += red[k];
        for (int o = 16; o >= R; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    }
    return a;
}

// ---------------------------------------------------------------- layout
// dst (padded, R per node) <- the R caller vectors src[r] (n x n, i fastest);
// null sources give zero; boundary entries zero.  grid (blocks, 1).
__global__ void k_bpack(int n, int ld, const double* s0, const double* s1, const double* s2, const double* s3,
                        double* __restrict__ dst) {
    const double* src[4] = {s0, s1, s2, s3};
    const long long tot = (long long)n * ld * R;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        const int rh = (int)(k % R);
        const long long node = k / R;
        const int j = (int)(node / ld), i = (int)(node - (long long)j * ld);
        const bool in = i >= 1 && i <= n - 2 && j >= 1 && j <= n - 2;
        dst[k] = (in && src[rh]) ? src[rh][(long long)j * n + i] : 0.0;
    }
}

__global__ void k_bunpack(int n, int ld, const double* __restrict__ src, double* d0, double* d1, double* d2,
                          double* d3) {
    double* dst[4] = {d0, d1, d2, d3};
    const long long tot = (long long)n * n * R;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        const int rh = (int)(k % R);
        const long long node = k / R;
        const int j = (int)(node / n), i = (int)(node - (long long)j * n);
        if (dst[rh]) dst[rh][node] = src[((long long)j * ld + i) * R + rh];
    }
}

// x = 0 in the lanes of the systems with a zero right-hand side (their
// solution), problem blockIdx.y.
__global__ void __launch_bounds__(kBThreads) k_bclear(const BProbDev* __restrict__ probs,
                                                      const SysState* __restrict__ sys, int nrhs) {
    const int pi = blockIdx.y;
    const BProbDev P = probs[pi];
    const int rh = threadIdx.x % R;
    if (rh >= nrhs || sys[(long long)pi * R + rh].bb != 0.0) return;
    const long long tot = P.plane * R;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x)
        P.x[k] = 0.0;
}

// Table-driven forms for right-hand sides and solutions in device memory:
// one launch for every problem (blockIdx.y).
struct PackEnt {
    const double* src[4];
    double* dst[4];
};

__global__ void k_bpack_all(const BProbDev* __restrict__ probs, const PackEnt* __restrict__ tab, int which) {
    const int pi = blockIdx.y;
    const BProbDev P = probs[pi];
    const PackEnt e = tab[pi];
    double* dst = which == 0 ? (double*)P.b : P.x;
    const int n = P.n, ld = P.ld;
    const long long tot = P.plane * R;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        const int rh = (int)(k % R);
        const long long node = k / R;
        const int j = (int)(node / ld), i = (int)(node - (long long)j * ld);
        const bool in = i >= 1 && i <= n - 2 && j >= 1 && j <= n - 2;
        dst[k] = (in && e.src[rh]) ? e.src[rh][(long long)j * n + i] : 0.0;
    }
}

__global__ void k_bunpack_all(const BProbDev* __restrict__ probs, const PackEnt* __restrict__ tab) {
    const int pi = blockIdx.y;
    const BProbDev P = probs[pi];
    const PackEnt e = tab[pi];
    const int n = P.n, ld = P.ld;
    const long long tot = (long long)n * n * R;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot;
         k += (long long)gridDim.x * blockDim.x) {
        const int rh = (int)(k % R);
        const long long node = k / R;
        const int j = (int)(node / n), i = (int)(node - (long long)j * n);
        if (e.dst[rh]) e.dst[rh][node] = P.x[((long long)j * ld + i) * R + rh];
    }
}

// ---------------------------------------------------------------- FP64 residual
// r = (float)(b - A x) for every right-hand side of problem blockIdx.y,
// ||r||^2 (and, with bb, ||b||^2) per system; the last block of the problem
// stores them and restarts the inner CG of its active systems.  Rows whose x
// neighbourhood is zero take r = b without the FP64 products.
__global__ void __launch_bounds__(kBThreads) k_bresidual(const BProbDev* __restrict__ probs, SysState* sys,
                                                         double* partials, unsigned* counters, int bb) {
    __shared__ double red[kBThreads];
    __shared__ bool last;
    const int pi = blockIdx.y;
    const BProbDev P = probs[pi];
    const int rh = threadIdx.x % R, col = threadIdx.x / R;
    const int n = P.n, ld = P.ld;
    const long long pl = P.plane;
    double acc = 0.0, accb = 0.0;
    for (int j = 1 + blockIdx.x; j <= n - 2; j += gridDim.x) {
        for (int i = 1 + col; i <= n - 2; i += kBCols) {
            const long long o = (long long)j * ld + i;
            const double* A = P.A64;
            auto X = [&](long long q) { return P.x[q * R + rh]; };
            auto bits = [](double v) { return (unsigned long long)__double_as_longlong(v) << 1; };
            const unsigned long long zx = bits(X(o)) | bits(X(o - 1)) | bits(X(o + 1)) | bits(X(o - ld)) |
                                          bits(X(o + ld)) | bits(X(o - ld - 1)) | bits(X(o + ld + 1)) |
                                          bits(X(o + ld - 1)) | bits(X(o - ld + 1));
            const double bv = P.b[o * R + rh];
            double v = bv;
            if (zx != 0) {
                double s = A[C2 * pl + o] * X(o);
                s += A[W2 * pl + o] * X(o - 1);
                s += A[W2 * pl + o + 1] * X(o + 1);
                s += A[S2 * pl + o] * X(o - ld);
                s += A[S2 * pl + o + ld] * X(o + ld);
                s += A[SW2 * pl + o] * X(o - ld - 1);
                s += A[SW2 * pl + o + ld + 1] * X(o + ld + 1);
                s += A[NW2 * pl + o] * X(o + ld - 1);
                s += A[NW2 * pl + o - ld + 1] * X(o - ld + 1);
                v = bv - s;
            }
            P.r[o * R + rh] = (float)v;
            acc += v * v;
            accb += bv * bv;
        }
    }
    const double t1 = block_sum_r(acc, red);
    const double t2 = bb ? block_sum_r(accb, red) : 0.0;
    double* part = partials + ((long long)pi * gridDim.x + blockIdx.x) * 2 * R;
    if (threadIdx.x < R) {
        part[2 * threadIdx.x] = t1;
        part[2 * threadIdx.x + 1] = t2;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&counters[pi], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < R) {
        const double* base = partials + (long long)pi * gridDim.x * 2 * R;
        double s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < (int)gridDim.x; k++) {
            s1 += ((volatile const double*)base)[(long long)k * 2 * R + 2 * threadIdx.x];
            s2 += ((volatile const double*)base)[(long long)k * 2 * R + 2 * threadIdx.x + 1];
        }
        SysState& sy = sys[(long long)pi * R + threadIdx.x];
        sy.rr = s1;
        if (bb) sy.bb = s2;
        if (sy.active) sy.first = 1;
    }
    if (threadIdx.x == 0) counters[pi] = 0u;
}

// ---------------------------------------------------------------- operator product
__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 operator+(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 operator-(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 operator*(float a, float4 b) { return make_float4(a * b.x, a * b.y, a * b.z, a * b.w); }
__device__ __forceinline__ float4 operator*(float4 a, float4 b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

// p = z + beta p_old, then q = A p in difference form (FP64 row sums), p.q
// per system; the last tile of a problem forms alpha = r.z / p.q for each of
// its systems.  One CTA per item: kBThreads interior columns x H rows of
// one problem, a thread per column with the R right-hand sides of a node as
// one float4; a four-row ring of p (one halo column per side) and of the W,
// SW, NW planes (one halo column on the right), the loads of row j+2 in
// flight while row j is formed.  The arithmetic and its order are those of
// the single-problem kernel, per right-hand side.
static_assert(R == 4, "the batched vector kernels carry the right-hand sides of a node as a float4");
__global__ void __launch_bounds__(kBThreads, 3) k_bpspmv(const BProbDev* __restrict__ probs,
                                                      const SpItem* __restrict__ items, int H, int parity,
                                                      SysState* sys, double* partials, unsigned* counters,
                                                      KState* st) {
    constexpr int TW = kBThreads;
    __shared__ float4 sP[4][TW + 2];
    __shared__ float sW[4][TW + 1];
    __shared__ float sSW[4][TW + 1];
    __shared__ float sNW[4][TW + 1];
    __shared__ double red[kBThreads];
    __shared__ bool last;
    const SpItem it = items[blockIdx.x];
    const BProbDev P = probs[it.prob];
    const int t = threadIdx.x;
    const int n = P.n, ld = P.ld;
    const long long pl = P.plane;
    const float* A = P.A32;
    const float4* z = (const float4*)P.z[parity];
    const float4* pold = (const float4*)P.p[parity ^ 1];
    float4* pnew = (float4*)P.p[parity];
    float4* q = (float4*)P.q;
    const SysState* sy = sys + (long long)it.prob * R;
    const float4 beta = make_float4((float)sy[0].beta, (float)sy[1].beta, (float)sy[2].beta, (float)sy[3].beta);
    const int tx = it.tile % P.sp_tiles_x, ty = it.tile / P.sp_tiles_x;
    const int i0 = 1 + tx * TW;
    const int j0 = 1 + ty * H;
    const int j1 = min(j0 + H, n - 1);
    const int i = i0 + t;
    const bool act = i <= n - 2;
    const int il = i0 - 1, ir = i0 + TW;
    struct Row {
        float4 z, po, hz, hpo;
        float w, sw, nw, s, r, hw, hsw, hnw;
    };
    const float4 zero4 = f4(0.f);
    auto load = [&](int j, Row& v) {
        v.z = v.po = v.hz = v.hpo = zero4;
        v.w = v.sw = v.nw = v.s = v.r = v.hw = v.hsw = v.hnw = 0.f;
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
            v.r = P.rs[k];
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
    AccB acc[R];
    // a problem none of whose systems takes this iteration contributes zero
    // partials (its systems get alpha = 0 below)
    if (!batch_frozen(sys, it.prob)) {
    Row nx;
    load(j0 - 1, nx);
    put(j0 - 1, nx);
    load(j0, nx);
    put(j0, nx);
    float rs_j = nx.r, s_j = nx.s;
    load(j0 + 1, nx);
    for (int j = j0; j < j1; j++) {
        put(j + 1, nx);
        const float s_n = nx.s, rs_n = nx.r;
        load(j + 2, nx);
        __syncthreads();
        if (act) {
            const int sm = (j - 1) & 3, s0 = j & 3, sp = (j + 1) & 3;
            const float4 pv = sP[s0][t + 1];
            float4 v = rs_j * pv;
            v = v + sW[s0][t] * (sP[s0][t] - pv);
            v = v + sW[s0][t + 1] * (sP[s0][t + 2] - pv);
            v = v + s_j * (sP[sm][t + 1] - pv);
            v = v + s_n * (sP[sp][t + 1] - pv);
            v = v + sSW[s0][t] * (sP[sm][t] - pv);
            v = v + sSW[sp][t + 1] * (sP[sp][t + 2] - pv);
            v = v + sNW[s0][t] * (sP[sp][t] - pv);
            v = v + sNW[sm][t + 1] * (sP[sm][t + 2] - pv);
            const long long k = (long long)j * ld + i;
            pnew[k] = pv;
            q[k] = v;
            const float4 pq = pv * v;
            acc[0].add(pq.x);
            acc[1].add(pq.y);
            acc[2].add(pq.z);
            acc[3].add(pq.w);
        }
        rs_j = rs_n;
        s_j = s_n;
    }
    }
    // per right-hand side: warp shuffle trees, then the warps' sums in order
    // (a fixed order: deterministic), then the tile partial
    double v[R];
    for (int r = 0; r < R; r++) {
        v[r] = acc[r].value();
        for (int o = 16; o > 0; o >>= 1) v[r] += __shfl_down_sync(0xffffffffu, v[r], o);
    }
    const int warp = t >> 5, lane = t & 31;
    if (lane == 0)
        for (int r = 0; r < R; r++) red[warp * R + r] = v[r];
    __syncthreads();
    double* part = partials + P.sp_part * R;
    if (t < R) {
        double sum = 0.0;
        for (int w = 0; w < kBThreads / 32; w++) sum += red[w * R + t];
        part[(long long)it.tile * R + t] = sum;
    }
    __threadfence();
    __syncthreads();
    if (t == 0) last = atomicAdd(&counters[it.prob], 1u) == (unsigned)P.sp_tiles - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // fixed-order sum over the problem's tiles, per right-hand side
    const int rh = t % R;
    double s = 0.0;
    for (int k = t / R; k < P.sp_tiles; k += kBThreads / R)
        s += ((volatile const double*)part)[(long long)k * R + rh];
    s = block_sum_r(s, red);
    if (t < R) {
        SysState& sw = sys[(long long)it.prob * R + t];
        const bool live = sw.active && sw.left > 0;
        sw.pq = s;
        if (!live || sw.rz == 0.0) {
            sw.alpha = 0.0;
        } else if (!(s > 0.0)) {
            set_err(st, BMG_ERR_NOT_SPD);
            sw.alpha = 0.0;
        } else {
            sw.alpha = sw.rz / s;
        }
        if (live) {
            sw.left--;
            sw.taken++;
        }
    }
    if (t == 0) counters[it.prob] = 0u;
}

// x += alpha p straight into the FP64 iterate, r -= alpha q in FP32, for the
// systems of problem blockIdx.y that took this iteration (alpha != 0; a
// frozen system has alpha = 0 and keeps x and r).  A thread per node, the R
// right-hand sides as vectors.
__global__ void __launch_bounds__(kBThreads) k_bupdate(const BProbDev* __restrict__ probs, int parity,
                                                       const SysState* __restrict__ sys) {
    const int pi = blockIdx.y;
    const BProbDev P = probs[pi];
    const SysState* sy = sys + (long long)pi * R;
    double al[R];
    for (int r = 0; r < R; r++) al[r] = sy[r].active ? sy[r].alpha : 0.0;
    if (al[0] == 0.0 && al[1] == 0.0 && al[2] == 0.0 && al[3] == 0.0) return;
    const float4 a32 = make_float4((float)al[0], (float)al[1], (float)al[2], (float)al[3]);
    const float4* p = (const float4*)P.p[parity];
    const float4* q = (const float4*)P.q;
    float4* rr = (float4*)P.r;
    double2* x = (double2*)P.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < P.plane;
         k += (long long)gridDim.x * blockDim.x) {
        const float4 pv = p[k];
        const float4 qv = q[k];
        double2 x0 = x[2 * k], x1 = x[2 * k + 1];
        x0.x += al[0] * (double)pv.x;
        x0.y += al[1] * (double)pv.y;
        x1.x += al[2] * (double)pv.z;
        x1.y += al[3] * (double)pv.w;
        x[2 * k] = x0;
        x[2 * k + 1] = x1;
        rr[k] = rr[k] - a32 * qv;
    }
}

}  // namespace

// ---------------------------------------------------------------- batch object
struct BClass {
    int n = 0, ld = 0, nc = 0, ldc = 0;
    long long plane = 0, cplane = 0;
    bool tail = false;                  // the tails' first level (n <= 33): vectors only
    std::vector<int> prob, level;       // member -> (problem, level)
    float *A = nullptr, *P = nullptr, *b = nullptr, *xp = nullptr, *xf = nullptr;
    BatchMember *mdown = nullptr, *mup = nullptr;   // device member tables
    int coarse = -1;                    // index of the coarse level's class
    int wc = 32, hc = 0, tiles_x = 0, tiles_y = 0, grid_down = 0, grid_up = 0;
    CUtensorMap mA, mF, mXp, mXc;
    long long part0 = 0;                // first partial of its finest members (finest up kernel)
};

struct Batch {
    int count = 0;
    std::vector<Ctx*> ctx;
    int device = -1;
    cudaStream_t stream = nullptr;
    size_t ws_need = 0;
    char* ws = nullptr;
    bool attached = false;
    std::vector<BClass> cls;            // fused classes by decreasing n, then the tail class
    int tail_cls = -1;
    std::vector<int> cls_of;            // [problem * kMaxLevels + level] -> class (-1: below the tail)
    std::vector<int> mem_of;            // member index within that class
    std::vector<BProbDev> prob_h;
    BProbDev* prob_d = nullptr;
    std::vector<SpItem> sp_h;
    SpItem* sp_d = nullptr;
    int sp_h_rows = 0;
    TailArgs* targs = nullptr;
    size_t tail_smem = 0;
    SysState* sys = nullptr;            // device, count * R
    SysState* sys_h = nullptr;          // pinned mirror
    KState* st = nullptr;               // device error word
    KState* st_h = nullptr;
    unsigned* counters = nullptr;       // count (finest up) + count (product) + count (residual)
    double* part_up = nullptr;          // finest up kernel partials
    double* part_sp = nullptr;          // operator product partials
    double* part_res = nullptr;         // residual partials (count * kRowBlocks * 2R)
    double* stage = nullptr;            // host staging (largest n^2 * R doubles)
    PackEnt* ptab = nullptr;            // device: 3 * count pack/unpack entries
    PackEnt* ptab_h = nullptr;          // pinned mirror
    long long stage_elems = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    long long exec_kernels[2] = {0, 0};
    long long launches = 0;
    bool use_graphs = true;
    bool alias = false;                 // one problem: the classes view the context's own FP32 levels
};

namespace {

// Walks the workspace layout; with base == nullptr it only measures.
size_t carve_batch(Batch& B, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = a256(off);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    // finest-up partials: room for the most tiles any legal shape gives
    // (strip width 16, kBatchK rows per tile); offsets are set at configure
    long long parts_up = 0;
    for (const BClass& K : B.cls)
        if (!K.tail)
            for (size_t m = 0; m < K.prob.size(); m++)
                if (K.level[m] == 0) parts_up += (long long)cdiv(K.nc - 1, 16) * cdiv(K.nc - 1, kBatchK);
    for (BClass& K : B.cls) {
        const long long nm = (long long)K.prob.size();
        if (!K.tail) {
            if (!B.alias) {
                K.A = (float*)take(sizeof(float) * NS2 * K.plane * nm);
                K.P = (float*)take(sizeof(float) * NP2 * K.cplane * nm);
            }
            K.xp = (float*)take(sizeof(float) * R * K.plane * nm);
        }
        K.b = (float*)take(sizeof(float) * R * K.plane * nm);
        K.xf = (float*)take(sizeof(float) * R * K.plane * nm);
        K.mdown = (BatchMember*)take(sizeof(BatchMember) * nm);
        K.mup = (BatchMember*)take(sizeof(BatchMember) * nm);
    }
    long long parts_sp = 0;
    for (int p = 0; p < B.count; p++) {
        BProbDev& P = B.prob_h[p];
        const long long v = P.plane * R;
        P.x = (double*)take(sizeof(double) * v);
        P.b = (const double*)take(sizeof(double) * v);
        P.z[0] = (float*)take(sizeof(float) * v);
        P.z[1] = (float*)take(sizeof(float) * v);
        P.p[0] = (float*)take(sizeof(float) * v);
        P.p[1] = (float*)take(sizeof(float) * v);
        P.q = (float*)take(sizeof(float) * v);
        P.sp_part = parts_sp;
        parts_sp += P.sp_tiles;
    }
    B.prob_d = (BProbDev*)take(sizeof(BProbDev) * B.count);
    B.sp_d = (SpItem*)take(sizeof(SpItem) * B.sp_h.size());
    B.targs = (TailArgs*)take(sizeof(TailArgs) * B.count);
    B.sys = (SysState*)take(sizeof(SysState) * B.count * R);
    B.st = (KState*)take(sizeof(KState));
    B.counters = (unsigned*)take(sizeof(unsigned) * 3 * B.count);
    B.part_up = (double*)take(sizeof(double) * 2 * R * (parts_up > 0 ? parts_up : 1));
    B.part_sp = (double*)take(sizeof(double) * R * (parts_sp > 0 ? parts_sp : 1));
    B.part_res = (double*)take(sizeof(double) * 2 * R * kRowBlocks * B.count);
    B.stage = (double*)take(sizeof(double) * B.stage_elems);
    B.ptab = (PackEnt*)take(sizeof(PackEnt) * 3 * B.count);
    return a256(off);
}

// Rows per tile of a class: minimise waves x (2 hc + 3) over the class's
// items at the kernels' occupancy (a multiple of the rows per step).
void model_class_rows(BClass& K, int occ, int sms) {
    const int m = K.nc - 1;
    K.tiles_x = cdiv(m, K.wc);
    const long long slots = (long long)occ * sms;
    const long long nm = (long long)K.prob.size();
    long long best = -1;
    for (int ty = 1; ty <= m; ty++) {
        const int hc = cdiv(cdiv(m, ty), kBatchK) * kBatchK;
        const int tyr = cdiv(m, hc);
        const long long waves = cdiv(nm * K.tiles_x * tyr, slots);
        const long long cost = waves * (2LL * hc + 3);
        if (best < 0 || cost < best) {
            best = cost;
            K.hc = hc;
            K.tiles_y = tyr;
        }
    }
}

bmg_status make_maps(Batch& B, BClass& K) {
    if (K.tail) return BMG_OK;
    const int WW = 2 * K.wc + 16, WWc = K.wc + 8;
    const int nm = (int)K.prob.size();
    bool ok = map_planes(&K.mA, K.A, K.ld, K.n, NS2, K.plane, nm, WW);
    ok = ok && map_vec(&K.mF, K.b, K.ld, K.n, K.plane, nm, WW, 2, 8);
    ok = ok && map_vec(&K.mXp, K.xp, K.ld, K.n, K.plane, nm, WW, 2, 8);
    const BClass& C = B.cls[K.coarse];
    ok = ok && map_vec(&K.mXc, C.xf, C.ld, C.n, C.plane, (int)C.prob.size(), WWc, 1, 4);
    return ok ? BMG_OK : BMG_ERR_DEVICE;
}

FusedArgs class_args(Batch& B, const BClass& K, bool up, int parity) {
    FusedArgs a{};
    a.nf = K.n;
    a.nc = K.nc;
    a.ldf = K.ld;
    a.ldc = K.ldc;
    a.wc = K.wc;
    a.hc = K.hc;
    a.plc = K.cplane;
    a.st = B.st;
    a.partials = up ? B.part_up : nullptr;
    a.mem = up ? K.mup : K.mdown;
    a.nmem = (int)K.prob.size();
    a.tiles_x = K.tiles_x;
    a.tiles_y = K.tiles_y;
    a.parity = parity;
    a.sys = B.sys;
    a.counters = B.counters;
    return a;
}

// Member tables (device) of every class; host data from the layout.
bmg_status upload_tables(Batch& B) {
    for (size_t c = 0; c < B.cls.size(); c++) {
        BClass& K = B.cls[c];
        const int nm = (int)K.prob.size();
        if (K.tail) continue;
        std::vector<BatchMember> d(nm), u(nm);
        long long part = K.part0;
        for (int m = 0; m < nm; m++) {
            const int p = K.prob[m], l = K.level[m];
            const int cc = B.cls_of[p * kMaxLevels + l + 1], cm = B.mem_of[p * kMaxLevels + l + 1];
            const BClass& C = B.cls[cc];
            BatchMember& D = d[m];
            BatchMember& U = u[m];
            D = BatchMember{};
            U = BatchMember{};
            float* xp = K.xp + (long long)m * R * K.plane;
            float* xf = K.xf + (long long)m * R * K.plane;
            D.x[0] = D.x[1] = xp;
            D.bc = C.b + (long long)cm * R * C.plane;
            D.P = K.P + (long long)m * NP2 * K.cplane;
            D.cmem = cm;
            D.prob = p;
            D.finest = l == 0;
            U = D;
            U.bc = nullptr;
            if (l == 0) {
                U.x[0] = B.prob_h[p].z[0];
                U.x[1] = B.prob_h[p].z[1];
                U.zold[0] = B.prob_h[p].z[1];
                U.zold[1] = B.prob_h[p].z[0];
                U.part = part;
                part += (long long)K.tiles_x * K.tiles_y;
            } else {
                U.x[0] = U.x[1] = xf;
            }
        }
        BMG_CUDA(cudaMemcpyAsync(K.mdown, d.data(), sizeof(BatchMember) * nm, cudaMemcpyHostToDevice, B.stream));
        BMG_CUDA(cudaMemcpyAsync(K.mup, u.data(), sizeof(BatchMember) * nm, cudaMemcpyHostToDevice, B.stream));
    }
    BMG_CUDA(cudaStreamSynchronize(B.stream));
    return BMG_OK;
}

bmg_status configure_classes(Batch& B) {
    int sms = 0;
    BMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B.device));
    for (BClass& K : B.cls) {
        if (K.tail) continue;
        int od = 0, ou = 0;
        BMG_TRY(batch_occupancy(K.wc, &od, &ou));
        const int occ = std::max(1, std::min(od, ou));
        if (K.hc <= 0) model_class_rows(K, occ, sms);
        K.tiles_x = cdiv(K.nc - 1, K.wc);
        K.tiles_y = cdiv(K.nc - 1, K.hc);
        const long long items = (long long)K.prob.size() * K.tiles_x * K.tiles_y;
        K.grid_down = (int)std::min<long long>(items, (long long)std::max(1, od) * sms);
        K.grid_up = (int)std::min<long long>(items, (long long)std::max(1, ou) * sms);
        BMG_TRY(make_maps(B, K));
    }
    long long parts_up = 0;
    for (BClass& K : B.cls) {
        K.part0 = parts_up;
        if (!K.tail)
            for (size_t m = 0; m < K.prob.size(); m++)
                if (K.level[m] == 0) parts_up += (long long)K.tiles_x * K.tiles_y;
    }
    for (int p = 0; p < 2; p++)
        if (B.exec[p]) {
            cudaGraphExecDestroy(B.exec[p]);
            B.exec[p] = nullptr;
        }
    return BMG_OK;
}

// One inner iteration of every system (parity: z buffer written).
bmg_status enqueue_iteration(Batch& B, int parity) {
    const int nf = (int)B.cls.size();
    for (int c = 0; c < nf; c++) {
        const BClass& K = B.cls[c];
        if (K.tail) continue;
        BMG_TRY(batch_down(K.mA, K.mF, class_args(B, K, false, parity), K.grid_down, B.stream));
        B.launches++;
    }
    BMG_TRY(batch_tail(B.targs, B.count, B.tail_smem, B.stream));
    B.launches++;
    for (int c = nf - 1; c >= 0; c--) {
        const BClass& K = B.cls[c];
        if (K.tail) continue;
        BMG_TRY(batch_up(K.mA, K.mF, K.mXp, K.mXc, class_args(B, K, true, parity), K.grid_up, B.stream));
        B.launches++;
    }
    k_bpspmv<<<(int)B.sp_h.size(), kBThreads, 0, B.stream>>>(B.prob_d, B.sp_d, B.sp_h_rows, parity, B.sys,
                                                             B.part_sp, B.counters + B.count, B.st);
    int maxblk = 1;
    for (const BProbDev& P : B.prob_h) maxblk = std::max(maxblk, cdiv(P.plane, kBThreads * 4));
    k_bupdate<<<dim3(std::min(maxblk, 512), B.count), kBThreads, 0, B.stream>>>(B.prob_d, parity, B.sys);
    B.launches += 2;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status run_iteration(Batch& B, int parity) {
    if (!B.use_graphs) return enqueue_iteration(B, parity);
    if (!B.exec[parity]) {
        if (!B.cap) BMG_CUDA(cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking));
        cudaStream_t user = B.stream;
        B.stream = B.cap;
        cudaGraph_t g = nullptr;
        bmg_status st = BMG_OK;
        if (cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = BMG_ERR_DEVICE;
        const long long before = B.launches;
        if (st == BMG_OK) st = enqueue_iteration(B, parity);
        B.exec_kernels[parity] = B.launches - before;
        B.launches = before;
        const cudaError_t e = cudaStreamEndCapture(B.cap, &g);
        B.stream = user;
        if (st != BMG_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return BMG_ERR_DEVICE;
        cudaGraphExec_t ex = nullptr;
        const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) return BMG_ERR_DEVICE;
        B.exec[parity] = ex;
    }
    BMG_CUDA(cudaGraphLaunch(B.exec[parity], B.stream));
    B.launches += B.exec_kernels[parity];
    return BMG_OK;
}

bmg_status residual(Batch& B, bool bb) {
    k_bresidual<<<dim3(kRowBlocks, B.count), kBThreads, 0, B.stream>>>(B.prob_d, B.sys, B.part_res,
                                                                       B.counters + 2 * B.count, bb ? 1 : 0);
    B.launches++;
    BMG_CUDA(cudaGetLastError());
    return BMG_OK;
}

bmg_status read_sys(Batch& B) {
    BMG_CUDA(cudaMemcpyAsync(B.sys_h, B.sys, sizeof(SysState) * B.count * R, cudaMemcpyDeviceToHost, B.stream));
    BMG_CUDA(cudaMemcpyAsync(B.st_h, B.st, sizeof(KState), cudaMemcpyDeviceToHost, B.stream));
    BMG_CUDA(cudaStreamSynchronize(B.stream));
    return BMG_OK;
}

}  // namespace

// ---------------------------------------------------------------- entry points
// Eligibility of a context from its options and shape alone.
bool batch_eligible_shape(const Ctx& c) {
    return c.dim == 2 && c.opts.precision == BMG_PREC_FP32 && c.opts.outer == BMG_OUTER_REFINEMENT &&
           !(c.opts.flags & BMG_FLAG_UNFUSED) && c.nlev >= 2 && c.lev[0].n >= 65;
}

// sizing: lay out from the contexts' shapes only (no attach or setup needed).
bmg_status batch_build(int count, Ctx* const* ctxs, int flags, bool sizing, bool alias, Batch** out) {
    *out = nullptr;
    if (count < 1) return BMG_ERR_ARG;
    if (alias && count != 1) return BMG_ERR_ARG;
    Batch* B = new (std::nothrow) Batch();
    if (!B) return BMG_ERR_ARG;
    B->count = count;
    B->alias = alias;
    B->use_graphs = !(flags & BMG_FLAG_NO_GRAPHS);
    B->ctx.assign(ctxs, ctxs + count);
    B->cls_of.assign((size_t)count * kMaxLevels, -1);
    B->mem_of.assign((size_t)count * kMaxLevels, -1);
    B->prob_h.resize(count);
    auto fail = [&](bmg_status s) {
        delete B;
        return s;
    };
    // size classes: every streamed level (n > 33) by its n, and the tails' first level
    std::vector<int> sizes;
    for (int p = 0; p < count; p++) {
        const Ctx* c = ctxs[p];
        if (!c || !batch_eligible_shape(*c)) return fail(BMG_ERR_ARG);
        if (!sizing) {
            if (!c->attached || !c->use_fused || !c->tail_pack) return fail(BMG_ERR_ARG);
            if (!c->have_setup) return fail(BMG_ERR_STATE);
            if (p > 0 && c->device != ctxs[0]->device) return fail(BMG_ERR_ARG);
        }
        const int t = tail_first_level(*c);
        if (c->lev[t].n != kTailMaxN) return fail(BMG_ERR_SHAPE);
        for (int l = 0; l < t; l++)
            if (std::find(sizes.begin(), sizes.end(), c->lev[l].n) == sizes.end()) sizes.push_back(c->lev[l].n);
    }
    std::sort(sizes.begin(), sizes.end(), std::greater<int>());
    for (int n : sizes) {
        BClass K;
        K.n = n;
        K.ld = (n + 31) & ~31;
        K.nc = (n + 1) / 2;
        K.ldc = (K.nc + 31) & ~31;
        K.plane = (long long)K.ld * n;
        K.cplane = (long long)K.ldc * K.nc;
        K.wc = n >= 129 ? 32 : 16;
        B->cls.push_back(K);
    }
    {
        BClass K;
        K.tail = true;
        K.n = kTailMaxN;
        K.ld = (kTailMaxN + 31) & ~31;
        K.plane = (long long)K.ld * K.n;
        B->cls.push_back(K);
        B->tail_cls = (int)B->cls.size() - 1;
    }
    for (int p = 0; p < count; p++) {
        const Ctx* c = ctxs[p];
        const int t = tail_first_level(*c);
        for (int l = 0; l <= t; l++) {
            const int ci = l == t ? B->tail_cls
                                  : (int)(std::find(sizes.begin(), sizes.end(), c->lev[l].n) - sizes.begin());
            BClass& K = B->cls[ci];
            B->cls_of[p * kMaxLevels + l] = ci;
            B->mem_of[p * kMaxLevels + l] = (int)K.prob.size();
            K.prob.push_back(p);
            K.level.push_back(l);
        }
    }
    for (size_t ci = 0; ci < B->cls.size(); ci++) {
        BClass& K = B->cls[ci];
        if (K.tail) continue;
        const int ncn = K.nc;
        if (ncn == kTailMaxN) {
            K.coarse = B->tail_cls;
        } else {
            K.coarse = (int)(std::find(sizes.begin(), sizes.end(), ncn) - sizes.begin());
        }
        K.tiles_x = cdiv(K.nc - 1, K.wc);   // rows per tile are modelled at attach
    }
    // per problem: the operator-product tiles and the staging size
    int H = 32;
    B->sp_h_rows = H;
    for (int p = 0; p < count; p++) {
        const Ctx* c = ctxs[p];
        BProbDev& P = B->prob_h[p];
        P = BProbDev{};
        P.n = c->lev[0].n;
        P.ld = c->lev[0].ld;
        P.plane = c->lev[0].plane;
        const int m = P.n - 2;
        P.sp_tiles_x = cdiv(m, kBThreads);
        P.sp_tiles = P.sp_tiles_x * cdiv(m, H);
        for (int t = 0; t < P.sp_tiles; t++) B->sp_h.push_back(SpItem{p, t});
        B->stage_elems = std::max<long long>(B->stage_elems, (long long)P.n * P.n * R);
    }
    B->ws_need = carve_batch(*B, nullptr);
    *out = B;
    return BMG_OK;
}

bmg_status batch_create(int count, Ctx* const* ctxs, int flags, Batch** out) {
    return batch_build(count, ctxs, flags, false, false, out);
}

size_t batch_ws_bytes(const Batch& B) { return B.ws_need; }

// Workspace of the one-problem batch a context uses for several right-hand
// sides (0 if the context is not eligible); shapes only.
size_t batch_single_bytes(Ctx& c) {
    if (!batch_eligible_shape(c)) return 0;
    Ctx* cs[1] = {&c};
    Batch* B = nullptr;
    if (batch_build(1, cs, c.opts.flags, true, true, &B) != BMG_OK) return 0;
    const size_t n = B->ws_need;
    delete B;
    return n;
}

bmg_status batch_single_create(Ctx& c, Batch** out) {
    Ctx* cs[1] = {&c};
    return batch_build(1, cs, c.opts.flags, false, true, out);
}

bmg_status batch_attach(Batch& B, void* ws, size_t bytes, void* stream) {
    if (!ws || ((uintptr_t)ws & 255) != 0) return BMG_ERR_ARG;
    if (bytes < B.ws_need) return BMG_ERR_WORKSPACE;
    if (!dev_ptr(ws)) return BMG_ERR_ARG;
    int dev = -1;
    BMG_CUDA(cudaGetDevice(&dev));
    if (dev != B.ctx[0]->device) return BMG_ERR_ARG;
    B.device = dev;
    B.stream = (cudaStream_t)stream;
    B.ws = (char*)ws;
    carve_batch(B, B.ws);
    if (!B.sys_h) BMG_CUDA(cudaMallocHost((void**)&B.sys_h, sizeof(SysState) * B.count * R));
    if (!B.st_h) BMG_CUDA(cudaMallocHost((void**)&B.st_h, sizeof(KState)));
    if (!B.ptab_h) BMG_CUDA(cudaMallocHost((void**)&B.ptab_h, sizeof(PackEnt) * 3 * B.count));
    BMG_CUDA(cudaMemsetAsync(B.ws, 0, B.ws_need, B.stream));
    // class copies of the FP32 operators and weights, in member order (one
    // problem: the classes view the context's own levels)
    for (BClass& K : B.cls) {
        if (K.tail) continue;
        if (B.alias) {
            const Level& L = B.ctx[0]->lev[K.level[0]];
            K.A = L.A32;
            K.P = L.P32;
            continue;
        }
        for (size_t m = 0; m < K.prob.size(); m++) {
            const Ctx& c = *B.ctx[K.prob[m]];
            const Level& L = c.lev[K.level[m]];
            BMG_CUDA(cudaMemcpyAsync(K.A + (long long)m * NS2 * K.plane, L.A32, sizeof(float) * NS2 * K.plane,
                                     cudaMemcpyDeviceToDevice, B.stream));
            BMG_CUDA(cudaMemcpyAsync(K.P + (long long)m * NP2 * K.cplane, L.P32, sizeof(float) * NP2 * K.cplane,
                                     cudaMemcpyDeviceToDevice, B.stream));
        }
    }
    // per-problem views: the finest member's class right-hand side is the inner residual
    for (int p = 0; p < B.count; p++) {
        BProbDev& P = B.prob_h[p];
        const Ctx& c = *B.ctx[p];
        const BClass& K = B.cls[B.cls_of[p * kMaxLevels]];
        const int m = B.mem_of[p * kMaxLevels];
        P.A64 = c.lev[0].A64;
        P.A32 = K.A + (long long)m * NS2 * K.plane;
        P.rs = c.rs32;
        P.r = K.b + (long long)m * R * K.plane;
    }
    BMG_CUDA(cudaMemcpyAsync(B.prob_d, B.prob_h.data(), sizeof(BProbDev) * B.count, cudaMemcpyHostToDevice,
                             B.stream));
    BMG_CUDA(cudaMemcpyAsync(B.sp_d, B.sp_h.data(), sizeof(SpItem) * B.sp_h.size(), cudaMemcpyHostToDevice,
                             B.stream));
    // tails: each problem's tail reads the tail class's right-hand side and
    // writes its final iterate there (the up kernels of n = 65 read it)
    {
        std::vector<TailArgs> ta(B.count);
        const BClass& T = B.cls[B.tail_cls];
        for (int p = 0; p < B.count; p++) {
            const Ctx& c = *B.ctx[p];
            const int t = tail_first_level(c);
            const int m = B.mem_of[p * kMaxLevels + t];
            BMG_TRY(tail_args(c, T.b + (long long)m * R * T.plane, T.xf + (long long)m * R * T.plane, T.ld, B.st,
                              &ta[p]));
            ta[p].sys = B.sys + (long long)p * R;
            if (p == 0) B.tail_smem = batch_tail_smem(ta[0].ns, ta[0].nlev);
        }
        BMG_CUDA(cudaMemcpyAsync(B.targs, ta.data(), sizeof(TailArgs) * B.count, cudaMemcpyHostToDevice, B.stream));
        BMG_CUDA(cudaStreamSynchronize(B.stream));
    }
    for (BClass& K : B.cls) K.hc = 0;   // re-modelled at the device's occupancy
    BMG_TRY(configure_classes(B));
    BMG_TRY(upload_tables(B));
    B.attached = true;
    return BMG_OK;
}

// Tile shape of a size class: wc (16 or 32) coarse columns and hc coarse
// rows (a positive multiple of kBatchK) per item.
bmg_status batch_set_tiles(Batch& B, int cls, int wc, int hc) {
    if (!B.attached || cls < 0 || cls >= (int)B.cls.size() || B.cls[cls].tail) return BMG_ERR_ARG;
    if ((wc != 16 && wc != 32) || hc < kBatchK || hc % kBatchK) return BMG_ERR_ARG;
    B.cls[cls].wc = wc;
    B.cls[cls].hc = hc;
    BMG_TRY(configure_classes(B));
    return upload_tables(B);
}

bmg_status batch_get_tiles(const Batch& B, int cls, int* n, int* wc, int* hc, int* members) {
    if (cls < 0 || cls >= (int)B.cls.size()) return BMG_ERR_ARG;
    const BClass& K = B.cls[cls];
    if (n) *n = K.n;
    if (wc) *wc = K.tail ? 0 : K.wc;
    if (hc) *hc = K.tail ? 0 : K.hc;
    if (members) *members = (int)K.prob.size();
    return BMG_OK;
}

// Times every legal tile shape of each size class (its down and up kernels
// over all members, CUDA events, best of reps; the vectors the kernels use
// hold no state between V-cycles) and keeps the fastest.  Candidates: strip
// width 16 and 32, each with the modelled rows, half and twice that.
bmg_status batch_autotune(Batch& B, int reps, double* ms_total) {
    if (!B.attached) return BMG_ERR_STATE;
    if (reps < 1) reps = 1;
    cudaEvent_t e0, e1;
    BMG_CUDA(cudaEventCreate(&e0));
    BMG_CUDA(cudaEventCreate(&e1));
    int sms = 0;
    BMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B.device));
    // every system live, so that the kernels skip no problem while timed
    // (batch_solve sets the states afresh)
    const int S = B.count * R;
    for (int s = 0; s < S; s++) {
        B.sys_h[s] = SysState{};
        B.sys_h[s].active = 1;
        B.sys_h[s].left = 1 << 30;
    }
    BMG_CUDA(cudaMemcpyAsync(B.sys, B.sys_h, sizeof(SysState) * S, cudaMemcpyHostToDevice, B.stream));
    double total = 0.0;
    for (size_t ci = 0; ci < B.cls.size(); ci++) {
        BClass& K = B.cls[ci];
        if (K.tail) continue;
        int bw = K.wc, bh = K.hc;
        float best = -1.f;
        for (int wc = 16; wc <= 32; wc += 16) {
            int od = 0, ou = 0;
            BMG_TRY(batch_occupancy(wc, &od, &ou));
            BClass probe = K;
            probe.wc = wc;
            model_class_rows(probe, std::max(1, std::min(od, ou)), sms);
            const int cands[3] = {probe.hc, (probe.hc / 2 / kBatchK) * kBatchK, probe.hc * 2};
            for (int c = 0; c < 3; c++) {
                const int hc = cands[c];
                if (hc < kBatchK || (c > 0 && hc == probe.hc) || hc > cdiv(K.nc - 1, kBatchK) * kBatchK + kBatchK)
                    continue;
                K.wc = wc;
                K.hc = hc;
                BMG_TRY(configure_classes(B));
                BMG_TRY(upload_tables(B));
                float tb = -1.f;
                for (int r = 0; r <= reps; r++) {   // the first run is a warm-up
                    BMG_CUDA(cudaMemsetAsync(B.stage, 0, sizeof(double) * B.stage_elems, B.stream));
                    BMG_CUDA(cudaEventRecord(e0, B.stream));
                    BMG_TRY(batch_down(K.mA, K.mF, class_args(B, K, false, 0), K.grid_down, B.stream));
                    BMG_TRY(batch_up(K.mA, K.mF, K.mXp, K.mXc, class_args(B, K, true, 0), K.grid_up, B.stream));
                    BMG_CUDA(cudaEventRecord(e1, B.stream));
                    BMG_CUDA(cudaEventSynchronize(e1));
                    float t = 0.f;
                    BMG_CUDA(cudaEventElapsedTime(&t, e0, e1));
                    if (r > 0 && (tb < 0 || t < tb)) tb = t;
                }
                if (best < 0 || tb < best) {
                    best = tb;
                    bw = wc;
                    bh = hc;
                }
            }
        }
        K.wc = bw;
        K.hc = bh;
        total += best > 0 ? best : 0.0;
    }
    BMG_TRY(configure_classes(B));
    BMG_TRY(upload_tables(B));
    // the tuning launches left arrival counters and partials untouched only
    // if every finest class ran to the end; clear them before the next solve
    BMG_CUDA(cudaMemsetAsync(B.counters, 0, sizeof(unsigned) * 3 * B.count, B.stream));
    BMG_CUDA(cudaStreamSynchronize(B.stream));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_total) *ms_total = total;
    return BMG_OK;
}

bmg_status batch_solve(Batch& B, int nrhs, const double* const* b, double* const* x, double tol, int maxit,
                       bmg_info* infos) {
    if (!B.attached) return BMG_ERR_WORKSPACE;
    if (nrhs < 1 || nrhs > R || !b || !x || maxit < 0 || !(tol > 0)) return BMG_ERR_ARG;
    const int S = B.count * R;
    // right-hand sides and initial guesses into the interleaved FP64 vectors:
    // one table-driven launch when every array is in device memory, else
    // per problem through the staging buffer
    bool all_dev = true;
    for (long long k = 0; k < (long long)B.count * nrhs && all_dev; k++) {
        if (!b[k] || !x[k]) return BMG_ERR_ARG;
        all_dev = dev_ptr(b[k]) && dev_ptr(x[k]);
    }
    int maxpk = 1;
    for (const BProbDev& P : B.prob_h) maxpk = std::max(maxpk, cdiv(P.plane * R, kBThreads * 4));
    maxpk = std::min(maxpk, 256);
    if (all_dev) {
        for (int p = 0; p < B.count; p++)
            for (int r = 0; r < R; r++) {
                const bool have = r < nrhs;
                B.ptab_h[p].src[r] = have ? b[(long long)p * nrhs + r] : nullptr;
                B.ptab_h[B.count + p].src[r] = have ? x[(long long)p * nrhs + r] : nullptr;
                B.ptab_h[2 * B.count + p].dst[r] = have ? x[(long long)p * nrhs + r] : nullptr;
            }
        BMG_CUDA(cudaMemcpyAsync(B.ptab, B.ptab_h, sizeof(PackEnt) * 3 * B.count, cudaMemcpyHostToDevice, B.stream));
        k_bpack_all<<<dim3(maxpk, B.count), kBThreads, 0, B.stream>>>(B.prob_d, B.ptab, 0);
        k_bpack_all<<<dim3(maxpk, B.count), kBThreads, 0, B.stream>>>(B.prob_d, B.ptab + B.count, 1);
        B.launches += 2;
    }
    for (int p = 0; p < B.count && !all_dev; p++) {
        BProbDev& P = B.prob_h[p];
        const long long nn = (long long)P.n * P.n;
        const double* src[R] = {nullptr, nullptr, nullptr, nullptr};
        const double* xs[R] = {nullptr, nullptr, nullptr, nullptr};
        for (int r = 0; r < nrhs; r++) {
            const double* bb = b[(long long)p * nrhs + r];
            const double* xx = x[(long long)p * nrhs + r];
            if (!bb || !xx) return BMG_ERR_ARG;
            src[r] = bb;
            xs[r] = xx;
        }
        const int blocks = std::min(cdiv(P.plane * R, kBThreads), 1024);
        for (int pass = 0; pass < 2; pass++) {
            const double** s = pass == 0 ? src : xs;
            const double* d[R];
            for (int r = 0; r < R; r++) {
                d[r] = s[r];
                if (s[r] && !dev_ptr(s[r])) {
                    BMG_CUDA(cudaMemcpyAsync(B.stage + r * nn, s[r], sizeof(double) * nn, cudaMemcpyHostToDevice,
                                             B.stream));
                    d[r] = B.stage + r * nn;
                }
            }
            k_bpack<<<blocks, kBThreads, 0, B.stream>>>(P.n, P.ld, d[0], d[1], d[2], d[3],
                                                        pass == 0 ? (double*)P.b : P.x);
            B.launches++;
        }
    }
    BMG_CUDA(cudaGetLastError());
    // every system starts active; zero right-hand sides (and the padding
    // systems) are retired below with x = 0
    for (int s = 0; s < S; s++) {
        B.sys_h[s] = SysState{};
        B.sys_h[s].active = (s % R) < nrhs ? 1 : 0;
    }
    BMG_CUDA(cudaMemcpyAsync(B.sys, B.sys_h, sizeof(SysState) * S, cudaMemcpyHostToDevice, B.stream));
    BMG_CUDA(cudaMemsetAsync(B.st, 0, sizeof(KState), B.stream));
    BMG_TRY(residual(B, true));
    BMG_TRY(read_sys(B));
    std::vector<double> bb(S), rr(S), rr0(S), rho(S, 0.3);
    std::vector<int> it(S, 0), refs(S, 0), status(S, BMG_OK), lastm(S, 0);
    std::vector<char> act(S, 0);
    bool zero_x = false;
    for (int s = 0; s < S; s++) {
        bb[s] = B.sys_h[s].bb;
        rr[s] = rr0[s] = B.sys_h[s].rr;
        act[s] = (s % R) < nrhs && bb[s] > 0.0;
        if ((s % R) < nrhs && bb[s] == 0.0) zero_x = true;
    }
    if (zero_x) {
        // a zero right-hand side has the solution x = 0 (residual 0)
        int maxblk = 1;
        for (const BProbDev& P : B.prob_h) maxblk = std::max(maxblk, cdiv(P.plane * R, kBThreads * 8));
        k_bclear<<<dim3(std::min(maxblk, 512), B.count), kBThreads, 0, B.stream>>>(B.prob_d, B.sys, nrhs);
        B.launches++;
        BMG_CUDA(cudaGetLastError());
        for (int s = 0; s < S; s++)
            if ((s % R) < nrhs && bb[s] == 0.0) rr[s] = rr0[s] = 0.0;
    }
    bmg_status first_err = BMG_OK;
    int global_it = 0;
    std::vector<int> m_of(S, 0);
    std::vector<double> want_of(S, 1.0);
    while (true) {
        int m_need = 0;
        for (int s = 0; s < S; s++) {
            m_of[s] = 0;
            if (!act[s]) continue;
            const double lim = tol * tol * bb[s];
            if (rr[s] <= lim) {
                act[s] = 0;
                continue;
            }
            if (it[s] >= maxit) {
                act[s] = 0;
                status[s] = BMG_ERR_NOT_CONVERGED;
                continue;
            }
            double want = sqrt(lim / rr[s]);
            if (want < 1e-6) want = 1e-6;
            int m = (int)ceil(log(want) / log(rho[s])) + 1;
            if (m < 2) m = 2;
            if (m > kMaxInner) m = kMaxInner;
            if (m > maxit - it[s]) m = maxit - it[s];
            m_of[s] = m;
            want_of[s] = want;
            m_need = std::max(m_need, m);
        }
        if (m_need == 0) break;
        for (int s = 0; s < S; s++) {
            B.sys_h[s].active = act[s];
            B.sys_h[s].left = act[s] ? m_of[s] : 0;
            // the run also ends for a system once its r.z has fallen by the
            // square of the reduction it aims at (the recursive residual in
            // the preconditioner's norm): a fast system stops there instead
            // of iterating past what its FP32 inner solve can deliver
            // (not after a run in which it took no iteration: then it takes
            // its full count, which maxit bounds)
            B.sys_h[s].stop = act[s] && !(refs[s] > 0 && lastm[s] == 0) ? want_of[s] * want_of[s] : 0.0;
            B.sys_h[s].taken = 0;
        }
        BMG_CUDA(cudaMemcpyAsync(B.sys, B.sys_h, sizeof(SysState) * S, cudaMemcpyHostToDevice, B.stream));
        for (int k = 0; k < m_need; k++) BMG_TRY(run_iteration(B, (global_it + k) & 1));
        global_it += m_need;
        BMG_TRY(residual(B, false));
        BMG_TRY(read_sys(B));
        if (B.st_h->err) {
            first_err = (bmg_status)B.st_h->err;
            break;
        }
        for (int s = 0; s < S; s++) {
            if (!act[s]) continue;
            const int m = B.sys_h[s].taken;
            it[s] += m;
            refs[s]++;
            const double nr = B.sys_h[s].rr;
            const double red = sqrt(nr / rr[s]);
            if (m > 0 && red > 0 && red < 1) {
                const double r1 = pow(red, 1.0 / m);
                if (r1 > 0.02 && r1 < 0.999) rho[s] = r1;
            }
            rr[s] = nr;
            lastm[s] = m;
        }
    }
    // solutions back to the caller
    if (all_dev) {
        k_bunpack_all<<<dim3(maxpk, B.count), kBThreads, 0, B.stream>>>(B.prob_d, B.ptab + 2 * B.count);
        B.launches++;
    }
    for (int p = 0; p < B.count && !all_dev; p++) {
        BProbDev& P = B.prob_h[p];
        const long long nn = (long long)P.n * P.n;
        double* d[R] = {nullptr, nullptr, nullptr, nullptr};
        bool host = false;
        for (int r = 0; r < nrhs; r++) {
            double* xx = x[(long long)p * nrhs + r];
            if (dev_ptr(xx)) {
                d[r] = xx;
            } else {
                d[r] = B.stage + r * nn;
                host = true;
            }
        }
        const int blocks = std::min(cdiv(nn * R, kBThreads), 1024);
        k_bunpack<<<blocks, kBThreads, 0, B.stream>>>(P.n, P.ld, P.x, d[0], d[1], d[2], d[3]);
        B.launches++;
        if (host) {
            for (int r = 0; r < nrhs; r++) {
                double* xx = x[(long long)p * nrhs + r];
                if (!dev_ptr(xx))
                    BMG_CUDA(cudaMemcpyAsync(xx, B.stage + r * nn, sizeof(double) * nn, cudaMemcpyDeviceToHost,
                                             B.stream));
            }
        }
    }
    BMG_CUDA(cudaStreamSynchronize(B.stream));
    BMG_CUDA(cudaGetLastError());
    bmg_status ret = first_err;
    for (int p = 0; p < B.count; p++)
        for (int r = 0; r < nrhs; r++) {
            const int s = p * R + r;
            if (infos) {
                bmg_info& in = infos[(long long)p * nrhs + r];
                memset(&in, 0, sizeof(in));
                in.iterations = it[s];
                in.refinements = refs[s];
                in.relres = bb[s] > 0 ? sqrt(rr[s] / bb[s]) : 0.0;
                in.true_relres = in.relres;
                in.rho = (it[s] > 0 && rr0[s] > 0 && rr[s] > 0) ? pow(rr[s] / rr0[s], 0.5 / it[s]) : 0.0;
                const Ctx& c = *B.ctx[p];
                double n0 = (double)(c.lev[0].n - 2) * (c.lev[0].n - 2), g = 0.0;
                for (int l = 0; l < c.nlev; l++) g += (double)(c.lev[l].n - 2) * (c.lev[l].n - 2);
                in.levels = c.nlev;
                in.grid_complexity = in.operator_complexity = g / n0;
                in.status = first_err ? first_err : status[s];
            }
            if (ret == BMG_OK && status[s] != BMG_OK) ret = (bmg_status)status[s];
        }
    return ret;
}

void batch_destroy(Batch* B) {
    if (!B) return;
    for (int p = 0; p < 2; p++)
        if (B->exec[p]) cudaGraphExecDestroy(B->exec[p]);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->sys_h) cudaFreeHost(B->sys_h);
    if (B->st_h) cudaFreeHost(B->st_h);
    if (B->ptab_h) cudaFreeHost(B->ptab_h);
    delete B;
}

long long batch_launches(const Batch& B) { return B.launches; }
int batch_classes(const Batch& B) { return (int)B.cls.size(); }

}  // namespace bmg

// ---------------------------------------------------------------- C ABI
struct bmg_batch {
    bmg::Batch* b;
};

extern "C" {

bmg_status bmg_batch_create(int count, bmg_ctx* const* ctxs, int flags, bmg_batch** out) {
    if (!out) return BMG_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !ctxs) return BMG_ERR_ARG;
    std::vector<bmg::Ctx*> cs(count);
    for (int p = 0; p < count; p++) {
        if (!ctxs[p]) return BMG_ERR_ARG;
        cs[p] = &ctxs[p]->c;
    }
    bmg::Batch* B = nullptr;
    BMG_TRY(bmg::batch_create(count, cs.data(), flags, &B));
    bmg_batch* h = new (std::nothrow) bmg_batch{B};
    if (!h) {
        bmg::batch_destroy(B);
        return BMG_ERR_ARG;
    }
    *out = h;
    return BMG_OK;
}

bmg_status bmg_batch_workspace_bytes(const bmg_batch* b, size_t* bytes) {
    if (!b || !bytes) return BMG_ERR_ARG;
    *bytes = bmg::batch_ws_bytes(*b->b);
    return BMG_OK;
}

bmg_status bmg_batch_attach(bmg_batch* b, void* ws, size_t bytes, void* stream) {
    if (!b) return BMG_ERR_ARG;
    return bmg::batch_attach(*b->b, ws, bytes, stream);
}

bmg_status bmg_batch_solve(bmg_batch* b, int nrhs, const double* const* rhs, double* const* x, double tol, int maxit,
                           bmg_info* infos) {
    if (!b) return BMG_ERR_ARG;
    return bmg::batch_solve(*b->b, nrhs, rhs, x, tol, maxit, infos);
}

bmg_status bmg_batch_autotune(bmg_batch* b, int reps, double* ms) {
    if (!b) return BMG_ERR_ARG;
    return bmg::batch_autotune(*b->b, reps, ms);
}

int bmg_batch_classes(const bmg_batch* b) { return b ? bmg::batch_classes(*b->b) : 0; }

bmg_status bmg_batch_get_tiles(const bmg_batch* b, int cls, int* n, int* wc, int* hc, int* members) {
    if (!b) return BMG_ERR_ARG;
    return bmg::batch_get_tiles(*b->b, cls, n, wc, hc, members);
}

bmg_status bmg_batch_set_tiles(bmg_batch* b, int cls, int wc, int hc) {
    if (!b) return BMG_ERR_ARG;
    return bmg::batch_set_tiles(*b->b, cls, wc, hc);
}

long long bmg_batch_launch_count(const bmg_batch* b) { return b ? bmg::batch_launches(*b->b) : 0; }

void bmg_batch_destroy(bmg_batch* b) {
    if (!b) return;
    bmg::batch_destroy(b->b);
    delete b;
}

}  // extern "C"
