// common.cuh -- internal types and device helpers of libbmg.
//
// Internal layout.  Every level l of the hierarchy stores its grid
// (n_l nodes per side) with a padded row length ld_l (a multiple of 32
// elements, so every row starts on a 128-byte boundary in FP32 and a
// 256-byte boundary in FP64); one "plane" holds ld_l * n_l^(d-1) values,
// i fastest.  Padding and boundary entries are kept at zero in every array.
//
// Operators are stored as the symmetric half of the 9-point (2-D) or
// 27-point (3-D) stencil, one plane per stored offset (the symmetric
// storage of Sec. 4.1: five values per node in 2-D):
//   2-D: C (0,0), W (-1,0), S (0,-1), SW (-1,-1), NW (-1,+1);
//        a(+d) at node i is a(-d) stored at node i+d.
//   3-D: C and the 13 offsets that are lexicographically negative
//        (dz<0, or dz==0 and dy<0, or dz==dy==0 and dx<0).
// Interpolation P_l (level l+1 -> level l) is stored on the coarse grid,
// one plane per weight of the fine points owned by coarse node (I,J[,K])
// (the fine points 2I+{0,1}, 2J+{0,1}[, 2K+{0,1}] other than the C point):
//   2-D: PXL PXR  (2I+1,2J)   -> (I,J), (I+1,J)
//        PYS PYN  (2I,2J+1)   -> (I,J), (I,J+1)
//        PSW PSE PNW PNE (2I+1,2J+1) -> (I,J), (I+1,J), (I,J+1), (I+1,J+1)
//   3-D: 26 planes, see setup3d.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bmg.h"
#include "fused2d.cuh"

namespace bmg {

constexpr int kMaxLevels = 20;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;       // partials buffer size for reductions (two sums per block)
// refinement mode: most FP32 inner iterations between two FP64 residuals
// (slowly converging problems, e.g. the 3-D shell, need hundreds per solve)
constexpr int kMaxInner = 400;

enum Plane2 { C2 = 0, W2 = 1, S2 = 2, SW2 = 3, NW2 = 4, NS2 = 5 };
enum PPlane2 { PXL = 0, PXR = 1, PYS = 2, PYN = 3, PSW = 4, PSE = 5, PNW = 6, PNE = 7, NP2 = 8 };
constexpr int NS3 = 14;
constexpr int NP3 = 26;

// Device error word values mirror bmg_status.
struct KState {
    double bb;        // ||b||^2
    double rr;        // ||r||^2 (last reduction)
    double rz;        // r.z of the previous iteration
    double rzn;       // r.z of this iteration
    double rzo;       // r.z_old (flexible CG)
    double pq;        // p.Aq
    double alpha, beta;
    double dot;       // scratch result of a plain dot product
    int err;          // first device error (bmg_status), 0 = none
    int first;        // 1 on the first iteration (p = z, no beta)
    unsigned int counter[8];
};

// CG scalars of one system (one right-hand side of one problem) in a
// batched solve; mirrors the fields of KState that the batched kernels use.
struct SysState {
    double bb;        // ||b||^2
    double rr;        // ||r||^2 of the last FP64 residual
    double rz;        // r.z of the previous inner iteration
    double pq;        // p.Ap
    double alpha, beta;
    double rz0;       // r.z of the first inner iteration of the current run
    double stop;      // the run ends for this system once r.z <= stop * rz0 (0: it takes its full count)
    int first;        // 1: the next inner iteration takes p = z
    int active;       // 0: converged, zero right-hand side or out of iterations: no updates
    int left;         // inner iterations this system still takes in the current run (its own
                      // count, as the single-problem refinement sizes it); at 0 it freezes
    int taken;        // inner iterations it took in the current run
};

// Right-hand sides per problem and row pairs per step of the batched
// streaming kernels (FP32 V-cycle).
constexpr int kBatchR = 4;
constexpr int kBatchK = 2;

// True when no system of problem p takes the current inner iteration: the
// batched kernels then skip the problem's work (its results would not be
// used: every one of its systems has alpha = 0 for the iteration).
__device__ __forceinline__ bool batch_frozen(const SysState* sys, int p) {
    const SysState* s = sys + (long long)p * kBatchR;
    for (int r = 0; r < kBatchR; r++)
        if (s[r].active && s[r].left > 0) return false;
    return true;
}

struct Level {
    int n = 0;            // nodes per side
    int ld = 0;           // padded row length
    long long plane = 0;  // elements per plane
    double* A64 = nullptr;
    float* A32 = nullptr;
    double* P64 = nullptr;    // interpolation from level+1 (planes on level+1's grid)
    float* P32 = nullptr;
    void* b = nullptr;        // V-cycle right-hand side (V-cycle precision)
    void* x = nullptr;        // V-cycle iterate
    void* r = nullptr;        // residual scratch
    float* cb = nullptr;      // 3-D FP32: full 27-entry rows in colour blocks (smoother)
};

struct ProfSlot {
    std::vector<cudaEvent_t> ev;   // start/end pairs
    int used = 0;
    double bytes = 0.0;
};

struct Batch;

struct Ctx {
    bmg_opts opts{};
    int dim = 2;
    int nlev = 0;
    int ns = 5, np = 8;       // stored stencil / interpolation planes
    Level lev[kMaxLevels];
    size_t ws_need = 0;
    char* ws = nullptr;
    cudaStream_t stream = nullptr;
    int device = -1;
    bool attached = false, have_op = false, have_setup = false;
    bool op_tensor = false;       // operator assembled from a diffusion tensor (no dL/dkappa)
    // finest-level FP64 Krylov vectors (internal padded layout)
    double *bvec = nullptr, *x = nullptr, *r = nullptr, *z[2] = {nullptr, nullptr};
    double *p = nullptr, *q = nullptr;
    double *stage_in = nullptr, *stage_out = nullptr;   // n^d doubles each, host staging
    // iterative refinement: FP32 inner CG vectors
    float *r32 = nullptr, *z32[2] = {nullptr, nullptr}, *p32 = nullptr, *q32 = nullptr;
    float* p32s[2] = {nullptr, nullptr};   // search directions, alternating (p is formed while p_old is read)
    float* rs32 = nullptr;        // FP32 row sums of the finest operator (difference-form products)
    FusedLevel fused_ir0;         // level-0 streaming kernels reading r32 (FP32)
    double* partials = nullptr;
    KState* st = nullptr;         // device
    KState* st_host = nullptr;    // pinned mirror
    long long launches = 0;
    int red_blocks = 0;           // fixed grid of the reducing kernels (deterministic)
    int spmv_h = 0, spmv_tiles_x = 0, spmv_tiles = 0;   // tiles of the 2-D refinement-mode operator product
    bool prof_on = false;
    ProfSlot prof[BMG_PROF_KINDS];
    bool use_fused = false;       // streaming V-cycle kernels (2-D)
    bool use_hs3 = false;         // 3-D: half-sweep kernels (one launch per colour parity of k)
    void* tail_pack = nullptr;    // 2-D: operators and weights of the tail levels, packed (tail2d.cu)
    // CUDA graphs of one inner/outer iteration (two, for the alternating z buffers)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t it_exec[2] = {nullptr, nullptr};
    long long it_kernels[2] = {0, 0};
    bool use_graphs = true;
    // bumped whenever launch shapes change (tile choices): graphs that other
    // objects capture around this context's kernels compare it
    unsigned long long shape_epoch = 0;
    FusedLevel fused[kMaxLevels];
    // several right-hand sides (opts.max_rhs > 1 on an eligible context): a
    // one-problem batch in a reserved part of the workspace, built on first use
    Batch* mrhs = nullptr;
    char* mrhs_ws = nullptr;
    size_t mrhs_bytes = 0;
};

// Event brackets around profiled launches (finest level only).
inline void prof_begin(Ctx& c, int kind, int level) {
    if (!c.prof_on || level != 0) return;
    ProfSlot& s = c.prof[kind];
    if ((size_t)(2 * s.used + 2) > s.ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        s.ev.push_back(a);
        s.ev.push_back(b);
    }
    cudaEventRecord(s.ev[2 * s.used], c.stream);
}

inline void prof_end(Ctx& c, int kind, int level, double bytes) {
    if (!c.prof_on || level != 0) return;
    ProfSlot& s = c.prof[kind];
    cudaEventRecord(s.ev[2 * s.used + 1], c.stream);
    s.used++;
    s.bytes += bytes;
}

// ------------------------------------------------------------------ helpers
#define BMG_CUDA(call)                                                      \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return BMG_ERR_DEVICE;                       \
    } while (0)

#define BMG_TRY(call)                                                       \
    do {                                                                    \
        bmg_status s_ = (call);                                             \
        if (s_ != BMG_OK) return s_;                                        \
    } while (0)

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

__device__ __forceinline__ void set_err(KState* st, int code) {
    atomicCAS(&st->err, 0, code);
}

// Symmetric-half 2-D stencil view.  a(i,j; dx,dy) for |dx|,|dy| <= 1.
template <typename T>
struct Sten2 {
    const T* a;
    int ld;
    long long pl;
    __device__ __forceinline__ T at(int p, int i, int j) const {
        return a[(long long)p * pl + (long long)j * ld + i];
    }
    __device__ __forceinline__ T c(int i, int j) const { return at(C2, i, j); }
    __device__ __forceinline__ T full(int i, int j, int dx, int dy) const {
        if (dx == 0 && dy == 0) return at(C2, i, j);
        if (dy == 0) return dx < 0 ? at(W2, i, j) : at(W2, i + 1, j);
        if (dx == 0) return dy < 0 ? at(S2, i, j) : at(S2, i, j + 1);
        if (dx < 0 && dy < 0) return at(SW2, i, j);
        if (dx > 0 && dy > 0) return at(SW2, i + 1, j + 1);
        if (dx < 0 && dy > 0) return at(NW2, i, j);
        return at(NW2, i + 1, j - 1);   // dx > 0, dy < 0
    }
};

// Block-wide sum (blockDim.x == kThreads), result valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        s = l < kThreads / 32 ? sh[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// Two sums at once (same scheme as grid_sum; partials holds 2 per block).
__device__ __forceinline__ bool grid_sum2(double v1, double v2, double* partials, unsigned int* counter,
                                          double* t1, double* t2) {
    __shared__ bool last2;
    double b1 = block_sum(v1);
    double b2 = block_sum(v2);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = b1;
        partials[2 * blockIdx.x + 1] = b2;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        last2 = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last2) return false;
    __threadfence();
    double s1 = 0.0, s2 = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
        s1 += ((volatile double*)partials)[2 * k];
        s2 += ((volatile double*)partials)[2 * k + 1];
    }
    s1 = block_sum(s1);
    s2 = block_sum(s2);
    if (threadIdx.x == 0) {
        *counter = 0u;
        *t1 = s1;
        *t2 = s2;
        return true;
    }
    return false;
}

// Deterministic grid reduction: each block stores its partial; the last
// block to arrive sums the partials in a fixed order.  Returns true (in
// thread 0 of the last block only) with the total in *total.
__device__ __forceinline__ bool grid_sum(double v, double* partials, unsigned int* counter,
                                         double* total) {
    __shared__ bool last;
    double b = block_sum(v);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = b;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) s += ((volatile double*)partials)[k];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        *counter = 0u;
        *total = s;
        return true;
    }
    return false;
}

// ------------------------------------------------------------------ host launchers
// setup2d.cu
bmg_status assemble2d(Ctx& c, const double* coords, const double* kappa);
bmg_status assemble_tensor2d(Ctx& c, const double* coords, const double* D);
bmg_status boundary_rhs2d(Ctx& c, const double* coords, const double* kappa, const double* g, double* out);
bmg_status set_stencil2d(Ctx& c, const double* full);
bmg_status setup_level2d(Ctx& c, int l);
bmg_status export_stencil2d(Ctx& c, int l, double* out);
bmg_status export_interp2d(Ctx& c, int l, double* out);
bmg_status adjoint_cells2d(Ctx& c, const double* coords, const double* u, const double* lam, double* g);
// setup3d.cu
bmg_status assemble3d(Ctx& c, const double* coords, const double* kappa);
bmg_status assemble_tensor3d(Ctx& c, const double* coords, const double* D);
bmg_status boundary_rhs3d(Ctx& c, const double* coords, const double* kappa, const double* g, double* out);
bmg_status set_stencil3d(Ctx& c, const double* full);
bmg_status setup_level3d(Ctx& c, int l);
bmg_status export_stencil3d(Ctx& c, int l, double* out);
bmg_status export_interp3d(Ctx& c, int l, double* out);
bmg_status adjoint_cells3d(Ctx& c, const double* coords, const double* u, const double* lam, double* g);
// setup2d.cu / setup3d.cu, context-free: assembly into given half planes, then export
bmg_status assemble_export2d(int n, int ld, long long pl, const double* coords, const double* kappa, double* A,
                             KState* st, double* out, cudaStream_t s);
bmg_status assemble_export3d(int n, int ld, long long pl, const double* coords, const double* kappa, double* A,
                             KState* st, double* out, cudaStream_t s);
// batch2d.cu
bmg_status batch_attach(Batch& B, void* ws, size_t bytes, void* stream);
bmg_status batch_solve(Batch& B, int nrhs, const double* const* b, double* const* x, double tol, int maxit,
                       bmg_info* infos);
void batch_destroy(Batch* B);
size_t batch_single_bytes(Ctx& c);
bmg_status batch_single_create(Ctx& c, Batch** out);
// vcycle.cu: z = M r on the finest level (FP64 in/out, internal layout)
bmg_status vcycle(Ctx& c, const double* r, double* z);
// fused2d.cu / tmaps.cu
int fused_rows_per_step(bool f32);
int fused_down_smem(bool f32, bool f64in, int wc);
int fused_up_smem(bool f32, bool f64in, int wc);
bmg_status fused_occupancy(bool f32, bool f64in, int wc, int* down_blocks, int* up_blocks);
bmg_status fused_down(Ctx& c, int l, bool ir = false);
bmg_status fused_up(Ctx& c, int l, void* out, bool ir = false, const float* zold = nullptr);
bmg_status vcycle_f32(Ctx& c, float* z32, const float* zold = nullptr);
// batched streaming kernels (fused2d.cu): FP32, kBatchR right-hand sides, strip width 16 or 32
int batch_down_smem(int wc);
int batch_up_smem(int wc);
bmg_status batch_occupancy(int wc, int* down_blocks, int* up_blocks);
bmg_status batch_down(const CUtensorMap& mA, const CUtensorMap& mF, const FusedArgs& a, int grid, cudaStream_t s);
bmg_status batch_up(const CUtensorMap& mA, const CUtensorMap& mF, const CUtensorMap& mXp, const CUtensorMap& mXc,
                    const FusedArgs& a, int grid, cudaStream_t s);
// vcycle3d.cu: colour-blocked full rows of the FP32 levels (after demotion)
bmg_status colour_blocks3d(Ctx& c);
// interior nodes of colour col (parities col&1, col>>1&1, col>>2) on an n-grid,
// and the offset of that colour's block (27 entries per node) in Level::cb
__host__ __device__ inline int cb_side(int n, int parity) { return parity ? (n - 1) / 2 : (n - 2) / 2; }
__host__ __device__ inline long long cb_count(int n, int col) {
    return (long long)cb_side(n, col & 1) * cb_side(n, (col >> 1) & 1) * cb_side(n, col >> 2);
}
__host__ __device__ inline long long cb_offset(int n, int col) {
    long long o = 0;
    for (int q = 0; q < col; q++) o += 27 * cb_count(n, q);
    return o;
}
// tail2d.cu: the levels from the first one with n <= kTailMaxN (at least
// level 1) down to the coarsest, in one single-CTA launch
constexpr int kTailMaxN = 33;
struct TailArgs {
    int nlev;                     // levels in the tail (the last one has 3 nodes)
    int ns[kMaxLevels];           // nodes per side of each tail level
    const void* pack;             // packed operators and weights (shared-memory image)
    unsigned pack_bytes;          // its size, a multiple of 16
    const void* b0;               // right-hand side of the first tail level
    void* x0;                     // finished iterate of the first tail level
    int ld0;                      // row length of b0 and x0 (in nodes)
    const double* a64c;           // FP64 centre entry of the coarsest operator
    KState* st;
    const SysState* sys = nullptr;   // batched: the problem's systems (skips a frozen problem)
};
int tail_first_level(const Ctx& c);
bmg_status tail_args(const Ctx& c, const void* b0, void* x0, int ld0, KState* st, TailArgs* a);
size_t batch_tail_smem(const int* ns, int L);
bmg_status batch_tail(const TailArgs* args, int count, size_t smem, cudaStream_t s);
size_t tail_smem_bytes(const Ctx& c, int t);
size_t tail_pack_bytes(const Ctx& c);             // packed tail operators (0 outside 2-D)
bmg_status tail_pack(Ctx& c);                     // fills c.tail_pack (bmg_setup)
bmg_status tail_vcycle(Ctx& c, int t);
// z32 = M r32 (FP32 in and out); with zold and the streaming kernels the
// finest up kernel also forms r.z, r.z_old and the flexible-CG beta
bool vcycle_forms_beta(const Ctx& c);
template <typename T>
bmg_status vcycle3d_impl(Ctx& c, const T* b0, T* x0, T* xout);
bmg_status fused_prepare(Ctx& c);
bmg_status fused_configure(Ctx& c, int l, int wc, int hc, int hc_up);
bmg_status fused_autotune(Ctx& c, int reps, double* best_ms_total);
bmg_status demote_levels(Ctx& c);
// krylov.cu
bmg_status k_pack(Ctx& c, const double* src, double* dst);      // n^d -> padded, boundary zeroed
bmg_status k_unpack(Ctx& c, const double* src, double* dst);    // padded -> n^d
bmg_status k_residual(Ctx& c, const double* b, const double* x, double* r);  // r = b - A x; st.rr
bmg_status k_dot(Ctx& c, const double* a, const double* b, double* slot);    // *slot (device) = a.b
bmg_status k_spmv_pq(Ctx& c, const double* p, double* q);        // q = A p; alpha = rz / p.q
bmg_status k_update_xr(Ctx& c);                                   // x += alpha p; r -= alpha q; rr
bmg_status k_rz_beta(Ctx& c, const double* z, const double* zold, bool flexible);
bmg_status k_p_update(Ctx& c, const double* z);                   // p = z + beta p (or z)
// FP32 inner CG of the refinement mode
bmg_status k_row_sums32(Ctx& c);                // rs32 = row sums of A (computed in FP64)
bmg_status k_residual_to32(Ctx& c);             // r32 = (float)(b - A x); rr; resets the inner CG state
bmg_status k_rz_beta32(Ctx& c, const float* z, const float* zo);
bmg_status k_update_dr32(Ctx& c, int parity);    // x (FP64) += alpha p; r32 -= alpha q
bmg_status pspmv_prepare(Ctx& c);                // tile shape of the 2-D operator product
bmg_status k_pspmv32(Ctx& c, const float* z, int parity);   // p = z + beta p_old; q = A p; alpha

}  // namespace bmg

// The opaque context of the C ABI.
struct bmg_ctx {
    bmg::Ctx c;
};
