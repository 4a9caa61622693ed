// api.cu -- the C ABI (include/bmg.h): context, workspace carving, the
// setup/solve sequence of Sec. 2.2 ("Setup phase", "Solution phase") with a
// preconditioned-CG outer loop, host/device staging, diagnostics.
#include <algorithm>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"

using namespace bmg;

namespace {

long long ipow(long long b, int e) {
    long long r = 1;
    while (e-- > 0) r *= b;
    return r;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Walks the workspace layout; with base == nullptr it only measures.
size_t carve(Ctx& c, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = align256(off);
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    const size_t vt = f32 ? sizeof(float) : sizeof(double);
    for (int l = 0; l < c.nlev; l++) {
        Level& L = c.lev[l];
        L.A64 = (double*)take(sizeof(double) * c.ns * L.plane);
        L.A32 = f32 ? (float*)take(sizeof(float) * c.ns * L.plane) : nullptr;
        if (l < c.nlev - 1) {
            const Level& K = c.lev[l + 1];
            L.P64 = (double*)take(sizeof(double) * c.np * K.plane);
            L.P32 = f32 ? (float*)take(sizeof(float) * c.np * K.plane) : nullptr;
        } else {
            L.P64 = nullptr;
            L.P32 = nullptr;
        }
        // colour-blocked rows serve only the per-colour 3-D smoother
        L.cb = (f32 && c.dim == 3 && l < c.nlev - 1 && (c.opts.flags & BMG_FLAG_UNFUSED))
                   ? (float*)take(sizeof(float) * 27 * ipow(L.n - 2, 3))
                   : nullptr;
        L.b = (l > 0 || f32) ? take(vt * L.plane) : nullptr;
        L.x = take(vt * L.plane);
        L.r = take(vt * L.plane);
    }
    const long long pl0 = c.lev[0].plane;
    c.bvec = (double*)take(sizeof(double) * pl0);
    c.x = (double*)take(sizeof(double) * pl0);
    c.r = (double*)take(sizeof(double) * pl0);
    c.z[0] = (double*)take(sizeof(double) * pl0);
    c.z[1] = (double*)take(sizeof(double) * pl0);
    c.p = (double*)take(sizeof(double) * pl0);
    c.q = (double*)take(sizeof(double) * pl0);
    if (c.opts.outer == BMG_OUTER_REFINEMENT) {
        c.r32 = (float*)take(sizeof(float) * pl0);
        c.z32[0] = (float*)take(sizeof(float) * pl0);
        c.z32[1] = (float*)take(sizeof(float) * pl0);
        c.p32 = (float*)take(sizeof(float) * pl0);
        c.p32s[0] = c.p32;
        c.p32s[1] = (float*)take(sizeof(float) * pl0);
        c.q32 = (float*)take(sizeof(float) * pl0);
        c.rs32 = (float*)take(sizeof(float) * pl0);
    }
    const long long nn = ipow(c.lev[0].n, c.dim);
    c.stage_in = (double*)take(sizeof(double) * nn);
    c.stage_out = (double*)take(sizeof(double) * nn);
    c.partials = (double*)take(sizeof(double) * kMaxBlocks);
    c.st = (KState*)take(sizeof(KState));
    const size_t tp = tail_pack_bytes(c);
    c.tail_pack = tp ? take(tp) : nullptr;
    c.mrhs_ws = c.mrhs_bytes ? take(c.mrhs_bytes) : nullptr;
    return align256(off);
}

// Drops the one-problem batch of several right-hand sides (its class views
// and tile shapes follow the hierarchy, so it is rebuilt after a setup).
void drop_mrhs(Ctx& c) {
    if (c.mrhs) {
        batch_destroy(c.mrhs);
        c.mrhs = nullptr;
    }
}

bmg_status read_state(Ctx& c, KState& h) {
    BMG_CUDA(cudaMemcpyAsync(&h, c.st, sizeof(KState), cudaMemcpyDeviceToHost, c.stream));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return BMG_OK;
}

bmg_status reset_state(Ctx& c) {
    KState z;
    memset(&z, 0, sizeof(z));
    BMG_CUDA(cudaMemcpyAsync(c.st, &z, sizeof(KState), cudaMemcpyHostToDevice, c.stream));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return BMG_OK;
}

bmg_status check_ready(const bmg_ctx* ctx) {
    if (!ctx) return BMG_ERR_ARG;
    if (!ctx->c.attached) return BMG_ERR_WORKSPACE;
    return BMG_OK;
}

}  // namespace

namespace bmg {
// Copies an n^d array from the caller (host or device) into the padded dst.
bmg_status stage_in_async(Ctx& c, const double* src, double* dst) {
    const long long nn = ipow(c.lev[0].n, c.dim);
    const double* dsrc = src;
    if (!is_device_ptr(src)) {
        BMG_CUDA(cudaMemcpyAsync(c.stage_in, src, sizeof(double) * nn, cudaMemcpyHostToDevice, c.stream));
        dsrc = c.stage_in;
    }
    return k_pack(c, dsrc, dst);
}

bmg_status stage_out_async(Ctx& c, const double* src, double* dst) {
    const long long nn = ipow(c.lev[0].n, c.dim);
    if (is_device_ptr(dst)) return k_unpack(c, src, dst);
    BMG_TRY(k_unpack(c, src, c.stage_out));
    BMG_CUDA(cudaMemcpyAsync(dst, c.stage_out, sizeof(double) * nn, cudaMemcpyDeviceToHost, c.stream));
    return BMG_OK;
}

void fill_complexity_info(const Ctx& c, bmg_info* info) {
    double n0 = (double)ipow(c.lev[0].n - 2, c.dim), s = 0.0;
    for (int l = 0; l < c.nlev; l++) s += (double)ipow(c.lev[l].n - 2, c.dim);
    info->levels = c.nlev;
    info->grid_complexity = s / n0;
    info->operator_complexity = s / n0;   // same stored entries per node on every level
}
}  // namespace bmg

namespace {
bmg_status stage_in(Ctx& c, const double* src, double* dst) { return stage_in_async(c, src, dst); }
bmg_status stage_out(Ctx& c, const double* src, double* dst) { return stage_out_async(c, src, dst); }
void fill_complexity(const Ctx& c, bmg_info* info) { fill_complexity_info(c, info); }

}  // namespace

namespace bmg {

// One iteration's launches on c.stream: refinement mode (FP32 inner CG) or
// the FP64 outer CG.  parity selects the z buffer written this iteration.
bmg_status enqueue_iteration(Ctx& c, int parity) {
    if (c.opts.outer == BMG_OUTER_REFINEMENT) {
        float* zn = c.z32[parity];
        float* zo = c.z32[parity ^ 1];
        if (vcycle_forms_beta(c)) {
            BMG_TRY(vcycle_f32(c, zn, zo));     // the finest up kernel also forms beta
        } else {
            BMG_TRY(vcycle_f32(c, zn));
            BMG_TRY(k_rz_beta32(c, zn, zo));
        }
        BMG_TRY(k_pspmv32(c, zn, parity));
        BMG_TRY(k_update_dr32(c, parity));
    } else {
        double* zn = c.z[parity];
        double* zo = c.z[parity ^ 1];
        BMG_TRY(vcycle(c, c.r, zn));
        BMG_TRY(k_rz_beta(c, zn, zo, c.opts.outer == BMG_OUTER_FLEXIBLE_CG));
        BMG_TRY(k_p_update(c, zn));
        BMG_TRY(k_spmv_pq(c, c.p, c.q));
        BMG_TRY(k_update_xr(c));
    }
    return BMG_OK;
}

// Captures one iteration into a CUDA graph (one per parity) on the library's
// capture stream; a no-op when graphs are off or already captured.
bmg_status capture_iteration(Ctx& c, int parity) {
    if (!c.use_graphs || c.prof_on || c.it_exec[parity]) return BMG_OK;
    if (!c.cap_stream) BMG_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c.stream;
    c.stream = c.cap_stream;
    cudaGraph_t g = nullptr;
    bmg_status st = BMG_OK;
    if (cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) st = BMG_ERR_DEVICE;
    const long long before = c.launches;
    if (st == BMG_OK) st = enqueue_iteration(c, parity);
    c.it_kernels[parity] = c.launches - before;
    c.launches = before;
    cudaError_t e = cudaStreamEndCapture(c.cap_stream, &g);
    c.stream = user;
    if (st != BMG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return BMG_ERR_DEVICE;
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return BMG_ERR_DEVICE;
    c.it_exec[parity] = ex;
    return BMG_OK;
}

// Launches one iteration: a replay of its graph, or the kernels themselves
// while profiling (per-launch events) or with graphs disabled.
bmg_status run_iteration(Ctx& c, int parity) {
    if (!c.use_graphs || c.prof_on) return enqueue_iteration(c, parity);
    BMG_TRY(capture_iteration(c, parity));
    BMG_CUDA(cudaGraphLaunch(c.it_exec[parity], c.stream));
    c.launches += c.it_kernels[parity];   // kernels the graph replays
    return BMG_OK;
}

bmg_status stage_in_async(Ctx& c, const double* src, double* dst);
bmg_status stage_out_async(Ctx& c, const double* src, double* dst);
void fill_complexity_info(const Ctx& c, bmg_info* info);
bmg_status solve_many(Ctx** cs, int count, int nrhs, const double* const* b, double* const* x, double tol,
                      int maxit, bmg_info* infos);

}  // namespace bmg

namespace {

// Iterative refinement: FP64 residual, inner FP32 flexible CG (FP32 V-cycle)
// on A d = r for m iterations whose updates go straight into the FP64 iterate
// x; m is chosen from the contraction seen
// so far so that one inner solve aims at the remaining reduction (bounded
// below by what FP32 can deliver).  The first run, whose prediction has no
// contraction to go by, goes on in steps of max(8, m/4) instead of
// restarting while its r.z is still more than 100 times above its goal
// (want^2 times its first r.z): on the 257^3 shell the solve took 520 inner
// iterations instead of 604 (532 when every run could go on).  maxit caps
// the total inner iterations.
bmg_status pcg_ir(Ctx& c, double tol, int maxit, bmg_info* info) {
    KState h;
    BMG_TRY(reset_state(c));
    BMG_TRY(k_dot(c, c.bvec, c.bvec, &c.st->bb));
    BMG_TRY(k_residual_to32(c));
    BMG_TRY(read_state(c, h));
    const double bb = h.bb;
    double rr = h.rr;
    const double rr0 = rr;
    int it = 0, refinements = 0;
    bmg_status status = BMG_OK;
    double rho = 0.3;                 // contraction per inner iteration, updated as we go
    const double floor_red = 1e-6;    // reduction one FP32 inner solve can deliver
    if (bb == 0.0) {
        BMG_CUDA(cudaMemsetAsync(c.x, 0, sizeof(double) * c.lev[0].plane, c.stream));
        rr = 0.0;
    } else {
        const double lim = tol > 0 ? tol * tol * bb : -1.0;
        while (!(rr <= lim) && it < maxit) {
            double want = tol > 0 ? sqrt(lim / rr) : floor_red;
            if (want < floor_red) want = floor_red;
            int m = (int)ceil(log(want) / log(rho)) + 1;
            if (m < 2) m = 2;
            if (m > kMaxInner) m = kMaxInner;
            if (m > maxit - it) m = maxit - it;
            // the predicted run.  The first run has no contraction to go by:
            // while its r.z stays far above the run's goal (more than 100x
            // want^2 times its first value, kept on the device in rzn) it
            // goes on instead of restarting
            BMG_TRY(run_iteration(c, it & 1));
            it++;
            BMG_CUDA(cudaMemcpyAsync(&c.st->rzn, &c.st->rz, sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            int done = 1, mm = m - 1;
            for (;;) {
                for (int k = 0; k < mm; k++) BMG_TRY(run_iteration(c, (it + k) & 1));
                it += mm;
                done += mm;
                if (done >= kMaxInner || it >= maxit || refinements > 0) break;
                BMG_TRY(read_state(c, h));
                if (h.err || !(h.rz > 100.0 * want * want * h.rzn)) break;
                mm = std::min(std::max(8, m / 4), std::min(kMaxInner - done, maxit - it));
            }
            m = done;
            BMG_TRY(k_residual_to32(c));
            BMG_TRY(read_state(c, h));
            refinements++;
            if (h.err) {
                status = (bmg_status)h.err;
                break;
            }
            const double red = sqrt(h.rr / rr);
            if (red > 0 && red < 1) {
                const double r1 = pow(red, 1.0 / m);
                if (r1 > 0.02 && r1 < 0.999) rho = r1;
            }
            rr = h.rr;
        }
        if (status == BMG_OK && tol > 0 && !(rr <= lim)) status = BMG_ERR_NOT_CONVERGED;
    }
    if (info) {
        info->iterations = it;
        info->refinements = refinements;
        info->relres = bb > 0 ? sqrt(rr / bb) : 0.0;
        info->true_relres = info->relres;   // the FP64 residual of the final iterate
        info->rho = (it > 0 && rr0 > 0 && rr > 0) ? pow(rr / rr0, 0.5 / it) : 0.0;
        fill_complexity(c, info);
        info->status = status;
    }
    return status;
}

// PCG with M = one V-cycle.  x (padded, in c.x) holds the initial guess.
bmg_status pcg(Ctx& c, double tol, int maxit, bmg_info* info) {
    if (c.opts.outer == BMG_OUTER_REFINEMENT) return pcg_ir(c, tol, maxit, info);
    BMG_TRY(reset_state(c));
    KState h;
    BMG_TRY(k_dot(c, c.bvec, c.bvec, &c.st->bb));
    BMG_TRY(k_residual(c, c.bvec, c.x, c.r));
    {   // the first iteration takes p = z
        int first = 1;
        BMG_CUDA(cudaMemcpyAsync(&c.st->first, &first, sizeof(int), cudaMemcpyHostToDevice, c.stream));
    }
    BMG_TRY(read_state(c, h));
    const double bb = h.bb;
    double rr = h.rr;
    const double rr0 = rr;
    int it = 0;
    bmg_status status = BMG_OK;
    if (bb == 0.0) {
        BMG_CUDA(cudaMemsetAsync(c.x, 0, sizeof(double) * c.lev[0].plane, c.stream));
        rr = 0.0;
    } else {
        const double lim = tol > 0 ? tol * tol * bb : -1.0;
        bool done = rr <= lim;
        while (!done && it < maxit) {
            BMG_TRY(run_iteration(c, it & 1));
            it++;
            BMG_TRY(read_state(c, h));
            if (h.err) {
                status = (bmg_status)h.err;
                break;
            }
            rr = h.rr;
            if (rr <= lim) {
                BMG_TRY(k_residual(c, c.bvec, c.x, c.r));   // true residual replaces r
                BMG_TRY(read_state(c, h));
                rr = h.rr;
                done = rr <= lim;
            }
        }
        if (status == BMG_OK && tol > 0 && !done) status = BMG_ERR_NOT_CONVERGED;
    }
    if (info) {
        info->iterations = it;
        info->refinements = 0;
        info->relres = bb > 0 ? sqrt(rr / bb) : 0.0;
        info->rho = (it > 0 && rr0 > 0 && rr > 0) ? pow(rr / rr0, 0.5 / it) : 0.0;
        // true residual of the final iterate, into q (scratch)
        BMG_TRY(k_residual(c, c.bvec, c.x, c.q));
        BMG_TRY(read_state(c, h));
        info->true_relres = bb > 0 ? sqrt(h.rr / bb) : 0.0;
        fill_complexity(c, info);
        info->status = status;
    }
    return status;
}

}  // namespace

extern "C" {

void bmg_default_opts(bmg_opts* o) {
    if (!o) return;
    o->dim = 2;
    o->n = 65;
    o->precision = BMG_PREC_FP64;
    o->outer = BMG_OUTER_CG;
    o->flags = 0;
    o->max_rhs = 1;
}

bmg_status bmg_create(const bmg_opts* opts, bmg_ctx** out) {
    if (!out) return BMG_ERR_ARG;
    *out = nullptr;
    if (!opts) return BMG_ERR_ARG;
    if (opts->dim != 2 && opts->dim != 3) return BMG_ERR_SHAPE;
    const int n = opts->n;
    if (n < 3 || ((n - 1) & (n - 2)) != 0) return BMG_ERR_SHAPE;
    if (opts->precision != BMG_PREC_FP64 && opts->precision != BMG_PREC_FP32) return BMG_ERR_ARG;
    if (opts->outer != BMG_OUTER_CG && opts->outer != BMG_OUTER_FLEXIBLE_CG && opts->outer != BMG_OUTER_REFINEMENT)
        return BMG_ERR_ARG;
    if (opts->outer == BMG_OUTER_REFINEMENT && opts->precision != BMG_PREC_FP32) return BMG_ERR_ARG;
    if (opts->max_rhs < 0 || opts->max_rhs > kBatchR) return BMG_ERR_ARG;
    bmg_ctx* ctx = new (std::nothrow) bmg_ctx();
    if (!ctx) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    c.opts = *opts;
    c.dim = opts->dim;
    c.ns = c.dim == 2 ? NS2 : NS3;
    c.np = c.dim == 2 ? NP2 : NP3;
    int nl = n, l = 0;
    while (true) {
        if (l >= kMaxLevels) {
            delete ctx;
            return BMG_ERR_SHAPE;
        }
        Level& L = c.lev[l];
        L.n = nl;
        L.ld = (nl + 31) & ~31;
        L.plane = (long long)L.ld * ipow(nl, c.dim - 1);
        l++;
        if (nl == 3) break;
        nl = (nl + 1) / 2;
    }
    c.nlev = l;
    if (c.opts.max_rhs < 1) c.opts.max_rhs = 1;
    c.mrhs_bytes = c.opts.max_rhs > 1 ? batch_single_bytes(c) : 0;
    c.ws_need = carve(c, nullptr);
    const long long rows = ipow(c.lev[0].n, c.dim - 1);
    c.red_blocks = (int)(rows > 152 * 8 ? 152 * 8 : rows);
    *out = ctx;
    return BMG_OK;
}

bmg_status bmg_workspace_bytes(const bmg_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return BMG_ERR_ARG;
    *bytes = ctx->c.ws_need;
    return BMG_OK;
}

bmg_status bmg_attach(bmg_ctx* ctx, void* ws, size_t bytes, void* stream) {
    if (!ctx || !ws) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (((uintptr_t)ws & 255) != 0) return BMG_ERR_ARG;
    if (bytes < c.ws_need) return BMG_ERR_WORKSPACE;
    if (!is_device_ptr(ws)) return BMG_ERR_ARG;
    BMG_CUDA(cudaGetDevice(&c.device));
    drop_mrhs(c);
    c.stream = (cudaStream_t)stream;
    if (!c.st_host) BMG_CUDA(cudaMallocHost((void**)&c.st_host, sizeof(KState)));
    c.ws = (char*)ws;
    carve(c, c.ws);
    BMG_CUDA(cudaMemsetAsync(c.ws, 0, c.ws_need, c.stream));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    c.use_fused = c.dim == 2 && !(c.opts.flags & BMG_FLAG_UNFUSED) && c.nlev >= 2;
    // FP64 3-D V-cycles are bound by FP64 arithmetic: the half sweeps'
    // recomputed halo would cost more than their saved traffic
    c.use_hs3 = c.dim == 3 && c.opts.precision == BMG_PREC_FP32 && !(c.opts.flags & BMG_FLAG_UNFUSED);
    c.use_graphs = !(c.opts.flags & BMG_FLAG_NO_GRAPHS);
    if (c.use_fused) BMG_TRY(fused_prepare(c));
    c.attached = true;
    c.have_op = c.have_setup = false;
    return BMG_OK;
}

bmg_status bmg_assemble(bmg_ctx* ctx, const double* coords, const double* kappa) {
    BMG_TRY(check_ready(ctx));
    if (!coords || !kappa) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!is_device_ptr(coords) || !is_device_ptr(kappa)) return BMG_ERR_ARG;
    BMG_TRY(reset_state(c));
    BMG_TRY(c.dim == 2 ? assemble2d(c, coords, kappa) : assemble3d(c, coords, kappa));
    KState h;
    BMG_TRY(read_state(c, h));
    c.have_setup = false;
    c.op_tensor = false;
    if (h.err) {
        c.have_op = false;
        return (bmg_status)h.err;
    }
    c.have_op = true;
    return BMG_OK;
}

bmg_status bmg_assemble_tensor(bmg_ctx* ctx, const double* coords, const double* D) {
    BMG_TRY(check_ready(ctx));
    if (!coords || !D) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!is_device_ptr(coords) || !is_device_ptr(D)) return BMG_ERR_ARG;
    BMG_TRY(reset_state(c));
    BMG_TRY(c.dim == 2 ? assemble_tensor2d(c, coords, D) : assemble_tensor3d(c, coords, D));
    KState h;
    BMG_TRY(read_state(c, h));
    c.have_setup = false;
    c.op_tensor = true;
    if (h.err) {
        c.have_op = false;
        return (bmg_status)h.err;
    }
    c.have_op = true;
    return BMG_OK;
}

bmg_status bmg_boundary_rhs(bmg_ctx* ctx, const double* coords, const double* kappa, const double* g,
                            double* out) {
    BMG_TRY(check_ready(ctx));
    if (!coords || !kappa || !g || !out) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!is_device_ptr(coords) || !is_device_ptr(kappa) || !is_device_ptr(g) || !is_device_ptr(out))
        return BMG_ERR_ARG;
    BMG_TRY(reset_state(c));
    BMG_TRY(c.dim == 2 ? boundary_rhs2d(c, coords, kappa, g, out) : boundary_rhs3d(c, coords, kappa, g, out));
    KState h;
    BMG_TRY(read_state(c, h));
    return h.err ? (bmg_status)h.err : BMG_OK;
}

bmg_status bmg_set_stencil(bmg_ctx* ctx, const double* stencil) {
    BMG_TRY(check_ready(ctx));
    if (!stencil || !is_device_ptr(stencil)) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    BMG_TRY(c.dim == 2 ? set_stencil2d(c, stencil) : set_stencil3d(c, stencil));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    c.have_op = true;
    c.have_setup = false;
    return BMG_OK;
}

bmg_status bmg_setup(bmg_ctx* ctx) {
    BMG_TRY(check_ready(ctx));
    Ctx& c = ctx->c;
    if (!c.have_op) return BMG_ERR_STATE;
    drop_mrhs(c);
    BMG_TRY(reset_state(c));
    for (int l = 0; l < c.nlev - 1; l++) BMG_TRY(c.dim == 2 ? setup_level2d(c, l) : setup_level3d(c, l));
    BMG_TRY(demote_levels(c));
    if (c.use_fused) BMG_TRY(tail_pack(c));
    if (c.rs32) BMG_TRY(k_row_sums32(c));
    BMG_TRY(pspmv_prepare(c));
    KState h;
    BMG_TRY(read_state(c, h));
    if (h.err) {
        c.have_setup = false;
        return (bmg_status)h.err;
    }
    c.have_setup = true;
    return BMG_OK;
}

bmg_status bmg_vcycle(bmg_ctx* ctx, const double* r, double* z) {
    BMG_TRY(check_ready(ctx));
    if (!r || !z) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.have_setup) return BMG_ERR_STATE;
    BMG_TRY(stage_in(c, r, c.r));
    BMG_TRY(vcycle(c, c.r, c.z[0]));
    BMG_TRY(stage_out(c, c.z[0], z));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return BMG_OK;
}

}  // extern "C"

namespace {

// One right-hand side through the single-problem path.
bmg_status solve_one(Ctx& c, const double* b, double* x, double tol, int maxit, bmg_info* info) {
    BMG_TRY(stage_in(c, b, c.bvec));
    BMG_TRY(stage_in(c, x, c.x));
    bmg_status st = pcg(c, tol, maxit, info);
    if (st == BMG_ERR_DEVICE) return st;
    BMG_TRY(stage_out(c, c.x, x));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return st;
}

// nrhs right-hand sides b + r n^d: together (groups of max_rhs, the
// one-problem batch) where the context has room for it, else in turn.
bmg_status solve_rhs(Ctx& c, int nrhs, const double* b, double* x, double tol, int maxit, bmg_info* info) {
    const long long nn = ipow(c.lev[0].n, c.dim);
    bmg_status first = BMG_OK;
    if (nrhs > 1 && c.mrhs_bytes && c.opts.max_rhs > 1 && tol > 0) {
        if (!c.mrhs) {
            BMG_TRY(batch_single_create(c, &c.mrhs));
            const bmg_status a = batch_attach(*c.mrhs, c.mrhs_ws, c.mrhs_bytes, c.stream);
            if (a != BMG_OK) {
                drop_mrhs(c);
                return a;
            }
        }
        for (int r0 = 0; r0 < nrhs; r0 += c.opts.max_rhs) {
            const int g = nrhs - r0 < c.opts.max_rhs ? nrhs - r0 : c.opts.max_rhs;
            const double* bp[kBatchR];
            double* xp[kBatchR];
            for (int r = 0; r < g; r++) {
                bp[r] = b + (r0 + r) * nn;
                xp[r] = x + (r0 + r) * nn;
            }
            const bmg_status st = batch_solve(*c.mrhs, g, bp, xp, tol, maxit, info ? info + r0 : nullptr);
            if (st == BMG_ERR_DEVICE || st == BMG_ERR_ARG) return st;
            if (first == BMG_OK) first = st;
        }
        return first;
    }
    for (int r = 0; r < nrhs; r++) {
        const bmg_status st = solve_one(c, b + r * nn, x + r * nn, tol, maxit, info ? info + r : nullptr);
        if (st == BMG_ERR_DEVICE) return st;
        if (first == BMG_OK) first = st;
    }
    return first;
}

}  // namespace

extern "C" {

bmg_status bmg_solve(bmg_ctx* ctx, int nrhs, const double* b, double* x, double tol, int maxit, bmg_info* info) {
    BMG_TRY(check_ready(ctx));
    if (!b || !x || maxit < 0 || nrhs < 1) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.have_setup) return BMG_ERR_STATE;
    return solve_rhs(c, nrhs, b, x, tol, maxit, info);
}

bmg_status bmg_adjoint_grad(bmg_ctx* ctx, int nrhs, const double* coords, const double* u, const double* dLdu,
                            double* lambda, double* dLdkappa, double tol, int maxit, bmg_info* info) {
    BMG_TRY(check_ready(ctx));
    if (!coords || !u || !dLdu || !lambda || !dLdkappa || nrhs < 1) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.have_setup || c.op_tensor) return BMG_ERR_STATE;
    if (!is_device_ptr(coords) || !is_device_ptr(u) || !is_device_ptr(dLdu) || !is_device_ptr(lambda) ||
        !is_device_ptr(dLdkappa))
        return BMG_ERR_ARG;
    const long long nn = ipow(c.lev[0].n, c.dim);
    const long long ne = ipow(c.lev[0].n - 1, c.dim);
    // A lambda = dL/du from a zero guess, for every right-hand side
    BMG_CUDA(cudaMemsetAsync(lambda, 0, sizeof(double) * nn * nrhs, c.stream));
    bmg_status st = solve_rhs(c, nrhs, dLdu, lambda, tol, maxit, info);
    if (st == BMG_ERR_DEVICE || st == BMG_ERR_ARG) return st;
    BMG_CUDA(cudaMemsetAsync(&c.st->err, 0, sizeof(c.st->err), c.stream));
    for (int r = 0; r < nrhs; r++)
        BMG_TRY(c.dim == 2 ? adjoint_cells2d(c, coords, u + r * nn, lambda + r * nn, dLdkappa + r * ne)
                           : adjoint_cells3d(c, coords, u + r * nn, lambda + r * nn, dLdkappa + r * ne));
    KState h;
    BMG_TRY(read_state(c, h));
    if (h.err && st == BMG_OK) st = (bmg_status)h.err;
    return st;
}

bmg_status bmg_adjoint_cells(bmg_ctx* ctx, const double* coords, const double* u, const double* lambda,
                             double* dLdkappa) {
    BMG_TRY(check_ready(ctx));
    if (!coords || !u || !lambda || !dLdkappa) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.have_setup || c.op_tensor) return BMG_ERR_STATE;
    if (!is_device_ptr(coords) || !is_device_ptr(u) || !is_device_ptr(lambda) || !is_device_ptr(dLdkappa))
        return BMG_ERR_ARG;
    BMG_CUDA(cudaMemsetAsync(&c.st->err, 0, sizeof(c.st->err), c.stream));
    BMG_TRY(c.dim == 2 ? adjoint_cells2d(c, coords, u, lambda, dLdkappa)
                       : adjoint_cells3d(c, coords, u, lambda, dLdkappa));
    KState h;
    BMG_TRY(read_state(c, h));
    return h.err ? (bmg_status)h.err : BMG_OK;
}

bmg_status bmg_solve_many(bmg_ctx* const* ctxs, int count, int nrhs, const double* const* b, double* const* x,
                          double tol, int maxit, bmg_info* infos) {
    if (!ctxs || count < 0 || nrhs < 1 || !b || !x || maxit < 0 || !(tol > 0)) return BMG_ERR_ARG;
    std::vector<Ctx*> cs(count);
    for (int p = 0; p < count; p++) {
        BMG_TRY(check_ready(ctxs[p]));
        Ctx& c = ctxs[p]->c;
        if (!c.have_setup) return BMG_ERR_STATE;
        if (c.opts.outer != BMG_OUTER_REFINEMENT) return BMG_ERR_ARG;
        for (int r = 0; r < nrhs; r++)
            if (!b[(long long)p * nrhs + r] || !x[(long long)p * nrhs + r]) return BMG_ERR_ARG;
        cs[p] = &c;
    }
    return solve_many(cs.data(), count, nrhs, b, x, tol, maxit, infos);
}

int bmg_levels(const bmg_ctx* ctx) { return ctx ? ctx->c.nlev : 0; }

int bmg_level_n(const bmg_ctx* ctx, int level) {
    if (!ctx || level < 0 || level >= ctx->c.nlev) return 0;
    return ctx->c.lev[level].n;
}

bmg_status bmg_get_stencil(bmg_ctx* ctx, int level, double* out) {
    BMG_TRY(check_ready(ctx));
    Ctx& c = ctx->c;
    if (!out || level < 0 || level >= c.nlev || !is_device_ptr(out)) return BMG_ERR_ARG;
    if (level > 0 && !c.have_setup) return BMG_ERR_STATE;
    if (level == 0 && !c.have_op) return BMG_ERR_STATE;
    BMG_TRY(c.dim == 2 ? export_stencil2d(c, level, out) : export_stencil3d(c, level, out));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return BMG_OK;
}

bmg_status bmg_get_interp(bmg_ctx* ctx, int level, double* out) {
    BMG_TRY(check_ready(ctx));
    Ctx& c = ctx->c;
    if (!out || level < 0 || level >= c.nlev - 1 || !is_device_ptr(out)) return BMG_ERR_ARG;
    if (!c.have_setup) return BMG_ERR_STATE;
    BMG_TRY(c.dim == 2 ? export_interp2d(c, level, out) : export_interp3d(c, level, out));
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return BMG_OK;
}

bmg_status bmg_profile(bmg_ctx* ctx, int enable) {
    if (!ctx) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    if (enable) {
        if (c.attached) BMG_CUDA(cudaStreamSynchronize(c.stream));
        for (int k = 0; k < BMG_PROF_KINDS; k++) {
            c.prof[k].used = 0;
            c.prof[k].bytes = 0.0;
        }
    }
    c.prof_on = enable != 0;
    return BMG_OK;
}

bmg_status bmg_profile_read(bmg_ctx* ctx, int kind, double* ms, long long* launches, double* bytes) {
    if (!ctx || kind < 0 || kind >= BMG_PROF_KINDS) return BMG_ERR_ARG;
    Ctx& c = ctx->c;
    ProfSlot& s = c.prof[kind];
    double tot = 0.0;
    if (s.used > 0) {
        BMG_CUDA(cudaStreamSynchronize(c.stream));
        for (int i = 0; i < s.used; i++) {
            float t = 0.f;
            BMG_CUDA(cudaEventElapsedTime(&t, s.ev[2 * i], s.ev[2 * i + 1]));
            tot += t;
        }
    }
    if (ms) *ms = tot;
    if (launches) *launches = s.used;
    if (bytes) *bytes = s.bytes;
    return BMG_OK;
}

bmg_status bmg_get_tiles(const bmg_ctx* ctx, int level, int* wc, int* hc, int* hc_up) {
    if (!ctx || !wc || !hc || !hc_up) return BMG_ERR_ARG;
    const Ctx& c = ctx->c;
    if (!c.use_fused || level < 0 || level >= c.nlev - 1) return BMG_ERR_ARG;
    *wc = c.fused[level].wc;
    *hc = c.fused[level].hc;
    *hc_up = c.fused[level].hc_up;
    return BMG_OK;
}

bmg_status bmg_set_tiles(bmg_ctx* ctx, int level, int wc, int hc, int hc_up) {
    BMG_TRY(check_ready(ctx));
    Ctx& c = ctx->c;
    if (!c.use_fused || level < 0 || level >= c.nlev - 1) return BMG_ERR_ARG;
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    return fused_configure(c, level, wc, hc, hc_up);
}

bmg_status bmg_autotune(bmg_ctx* ctx, int reps, double* ms) {
    BMG_TRY(check_ready(ctx));
    Ctx& c = ctx->c;
    if (!c.have_setup) return BMG_ERR_STATE;
    if (reps < 1) return BMG_ERR_ARG;
    BMG_CUDA(cudaStreamSynchronize(c.stream));
    const bool prof = c.prof_on;
    c.prof_on = false;
    bmg_status st = fused_autotune(c, reps, ms);
    c.prof_on = prof;
    if (st != BMG_OK) return st;
    KState h;
    BMG_TRY(read_state(c, h));
    return h.err ? (bmg_status)h.err : BMG_OK;
}

long long bmg_launch_count(const bmg_ctx* ctx) { return ctx ? ctx->c.launches : 0; }

void bmg_destroy(bmg_ctx* ctx) {
    if (!ctx) return;
    drop_mrhs(ctx->c);
    for (int p = 0; p < 2; p++)
        if (ctx->c.it_exec[p]) cudaGraphExecDestroy(ctx->c.it_exec[p]);
    if (ctx->c.cap_stream) cudaStreamDestroy(ctx->c.cap_stream);
    if (ctx->c.st_host) cudaFreeHost(ctx->c.st_host);
    for (int k = 0; k < BMG_PROF_KINDS; k++)
        for (cudaEvent_t e : ctx->c.prof[k].ev) cudaEventDestroy(e);
    delete ctx;
}

const char* bmg_status_str(bmg_status s) {
    switch (s) {
        case BMG_OK: return "ok";
        case BMG_ERR_ARG: return "invalid argument";
        case BMG_ERR_SHAPE: return "unsupported shape (n must be 2^k+1, dim 2 or 3)";
        case BMG_ERR_DEVICE: return "CUDA runtime error";
        case BMG_ERR_WORKSPACE: return "workspace missing or too small";
        case BMG_ERR_MAP_FOLDED: return "map folded: det J <= 0 at a quadrature point";
        case BMG_ERR_SETUP_BREAKDOWN: return "setup breakdown: zero collapsed denominator or non-positive diagonal";
        case BMG_ERR_NOT_SPD: return "CG breakdown: p^T A p <= 0";
        case BMG_ERR_NOT_CONVERGED: return "not converged within maxit";
        case BMG_ERR_TIMEOUT: return "bounded device wait expired";
        case BMG_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

}  // extern "C"
