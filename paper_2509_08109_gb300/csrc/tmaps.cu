// tmaps.cu -- host side of the streaming 2-D V-cycle: tile shapes per level
// (sized to fill whole waves of resident CTAs on the device) and the TMA
// tensor maps of every array the kernels stream.
#include <cudaTypedefs.h>

#include "common.cuh"

namespace bmg {
namespace {

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

// rank-2 or rank-3 row-major map: x = i (fastest), y = row, z = plane
bool make_map(CUtensorMap* m, bool f64, const void* base, int ld, int rows, int planes, long long plane_elems,
              int box_x, int box_y) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t es = f64 ? 8 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)ld, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)ld * es, (cuuint64_t)plane_elems * es};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)planes};
    cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = planes > 1 ? 3 : 2;
    CUresult r = fn(m, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

// Resident CTAs per SM of the down and up kernels of level l at strip width wc.
static bmg_status level_occupancy(Ctx& c, int l, int wc, int* od, int* ou) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    BMG_TRY(fused_occupancy(f32, f32 && l == 0 && !c.r32, wc, od, ou));
    if (*od < 1 || *ou < 1) return BMG_ERR_DEVICE;
    return BMG_OK;
}

// Rows per CTA (a multiple of the rows per step) for a given column width
// and occ resident CTAs per SM: minimise waves x (rows + pre-roll).
int model_rows(Ctx& c, int l, int wc, int occ) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess || sms < 1) sms = 1;
    const int m = c.lev[l + 1].n - 1;
    const int tiles_x = cdiv(m, wc);
    const long long slots = (long long)(occ < 1 ? 1 : occ) * sms;
    const int K = fused_rows_per_step(f32);
    long long best = -1;
    int hc_best = K;
    for (int ty = 1; ty <= m; ty++) {
        const int hc = cdiv(cdiv(m, ty), K) * K;
        const int tyr = cdiv(m, hc);
        const long long waves = cdiv((long long)tiles_x * tyr, slots);
        const long long cost = waves * (2LL * hc + 3);
        if (best < 0 || cost < best) {
            best = cost;
            hc_best = hc;
        }
    }
    return hc_best;
}

// Tile shape (wc coarse columns, hc coarse rows per CTA) of level l: kernel
// arguments and the TMA maps, whose boxes depend on wc.
bmg_status fused_configure(Ctx& c, int l, int wc, int hc, int hc_up) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    const int K = fused_rows_per_step(f32);
    // wc a multiple of 8: the TMA x coordinates 2 I0 - 10 and I0 - 5 then
    // start on 16-byte boundaries in FP32 and FP64
    if (wc < 8 || wc > 64 || wc % 8) return BMG_ERR_ARG;
    if (hc < K || hc % K || hc_up < K || hc_up % K) return BMG_ERR_ARG;
    FusedLevel& F = c.fused[l];
    const Level& Lf = c.lev[l];
    const Level& Lc = c.lev[l + 1];
    // Tiles cover coarse indices 1 .. nc-1: coarse index J owns the fine rows
    // 2J-1 and 2J, so the boundary index nc-1 still owns fine row nf-2.
    const int m = Lc.n - 1;
    F.wc = wc;
    F.hc = hc;
    F.tiles_x = cdiv(m, wc);
    F.tiles_y = cdiv(m, hc);
    F.hc_up = hc_up;
    F.tiles_y_up = cdiv(m, hc_up);
    const int WW = 2 * F.wc + 16, WWc = F.wc + 8;
    const void* A = f32 ? (const void*)Lf.A32 : (const void*)Lf.A64;
    const void* P = f32 ? (const void*)Lf.P32 : (const void*)Lf.P64;
    const void* f = l == 0 ? (const void*)c.r : Lf.b;
    const bool f_is64 = l == 0 || !f32;
    bool ok = make_map(&F.mA, !f32, A, Lf.ld, Lf.n, c.ns, Lf.plane, WW, 2);
    ok = ok && make_map(&F.mF, f_is64, f, Lf.ld, Lf.n, 1, Lf.plane, WW, 2);
    ok = ok && make_map(&F.mXp, !f32, Lf.x, Lf.ld, Lf.n, 1, Lf.plane, WW, 2);
    ok = ok && make_map(&F.mXc, !f32, Lc.r, Lc.ld, Lc.n, 1, Lc.plane, WWc, 1);
    if (!ok) return BMG_ERR_DEVICE;
    F.down = FusedArgs{Lf.n, Lc.n, Lf.ld, Lc.ld, F.wc, F.hc, Lf.x, Lc.b, P, Lc.plane, c.st, nullptr, nullptr};
    F.up = FusedArgs{Lf.n, Lc.n, Lf.ld, Lc.ld, F.wc, F.hc_up, nullptr, nullptr, P, Lc.plane, c.st, nullptr, nullptr};
    F.ready = true;
    if (l == 0 && c.r32) {
        // refinement mode: the level-0 kernels read the FP32 inner residual
        FusedLevel& G = c.fused_ir0;
        G = F;
        int od2 = 0, ou2 = 0;
        BMG_TRY(fused_occupancy(true, false, F.wc, &od2, &ou2));
        if (!make_map(&G.mF, false, c.r32, Lf.ld, Lf.n, 1, Lf.plane, WW, 2)) return BMG_ERR_DEVICE;
    }
    // captured iteration graphs hold the old launch shapes
    c.shape_epoch++;
    for (int p = 0; p < 2; p++)
        if (c.it_exec[p]) {
            cudaGraphExecDestroy(c.it_exec[p]);
            c.it_exec[p] = nullptr;
        }
    return BMG_OK;
}

// Default strip width of level l: the widest multiple of 8 up to a size
// cap that maximises useful columns in flight per SM, occupancy x wc (the
// kernels are bound by the bytes their TMA rings keep in flight).
int default_wc(Ctx& c, int l) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    const int m = c.lev[l + 1].n - 1;
    const int cap = m >= 512 ? 64 : m >= 128 ? 32 : m >= 32 ? 16 : 8;
    int best = 8, best_score = -1;
    for (int wc = cap; wc >= 8; wc -= 8) {
        int od = 0, ou = 0;
        if (fused_occupancy(f32, f32 && l == 0 && !c.r32, wc, &od, &ou) != BMG_OK) continue;
        const int score = (od < ou ? od : ou) * wc;
        if (score > best_score) {
            best_score = score;
            best = wc;
        }
    }
    return best;
}

bmg_status fused_prepare(Ctx& c) {
    for (int l = 0; l + 1 < c.nlev; l++) {
        const int wc = default_wc(c, l);
        int od = 0, ou = 0;
        BMG_TRY(level_occupancy(c, l, wc, &od, &ou));
        BMG_TRY(fused_configure(c, l, wc, model_rows(c, l, wc, od), model_rows(c, l, wc, ou)));
    }
    return BMG_OK;
}

// Measures candidate tile shapes of every level and keeps the fastest: the
// strip width is common to the level's down and up kernels (the TMA boxes
// depend on it), the rows per CTA are chosen for each kernel.  Candidates:
// each legal width with the rows the wave model gives at the kernel's
// occupancy and at one CTA per SM less, half and twice the first; each
// candidate runs the down and the up kernel (CUDA events before, between
// and after; best of reps per kernel).  Runs the kernels on the context's
// scratch vectors (they hold no state between V-cycles).  Before every
// timed rep the host staging buffers (2 n^d doubles) are overwritten, which
// evicts the level's data from L2 when the problem is larger than L2:
// inside a V-cycle the finer levels have evicted it too, and a warm L2
// would hide the halo re-reads of narrow strips.
bmg_status fused_autotune(Ctx& c, int reps, double* best_ms_total) {
    if (!c.use_fused) return BMG_OK;
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    const int K = fused_rows_per_step(f32);
    cudaEvent_t ev[3];
    for (int i = 0; i < 3; i++) BMG_CUDA(cudaEventCreate(&ev[i]));
    double total = 0.0;
    const bool ir = c.opts.outer == BMG_OUTER_REFINEMENT;
    void* out0 = ir ? (void*)c.z32[0] : (void*)c.z[0];
    size_t stage_bytes = sizeof(double);
    for (int d = 0; d < c.dim; d++) stage_bytes *= (size_t)c.lev[0].n;
    bmg_status st = BMG_OK;
    for (int l = 0; st == BMG_OK && l + 1 < c.nlev; l++) {
        const int m = c.lev[l + 1].n - 1;
        int best_wc = c.fused[l].wc, best_hd = c.fused[l].hc, best_hu = c.fused[l].hc_up;
        float best = -1.f;
        for (int wc = 8; st == BMG_OK && wc <= 64; wc += 8) {
            if (cdiv(m, wc) < 1 || (wc > 8 && m < wc / 2)) continue;
            int od = 0, ou = 0;
            if ((st = level_occupancy(c, l, wc, &od, &ou)) != BMG_OK) break;
            const int occ = od > ou ? od : ou;
            int cands[8], nc = 0;
            auto add = [&](int hc) {
                hc = hc / K * K;
                if (hc < K || hc > cdiv(m, K) * K + K) return;
                for (int i = 0; i < nc; i++)
                    if (cands[i] == hc) return;
                cands[nc++] = hc;
            };
            const int h0 = model_rows(c, l, wc, occ);
            add(h0);
            if (occ > 1) add(model_rows(c, l, wc, occ - 1));
            if (od != ou) add(model_rows(c, l, wc, od < ou ? od : ou));
            add(h0 / 2);
            add(h0 * 2);
            float bd = -1.f, bu = -1.f;
            int hd = cands[0], hu = cands[0];
            for (int ci = 0; st == BMG_OK && ci < nc; ci++) {
                const int hc = cands[ci];
                if ((st = fused_configure(c, l, wc, hc, hc)) != BMG_OK) break;
                void* out = l == 0 ? out0 : c.lev[l].r;
                if ((st = fused_down(c, l, ir)) != BMG_OK || (st = fused_up(c, l, out, ir)) != BMG_OK) break;
                for (int r = 0; st == BMG_OK && r < reps; r++) {
                    if (cudaMemsetAsync(c.stage_in, 0, stage_bytes, c.stream) != cudaSuccess ||
                        cudaMemsetAsync(c.stage_out, 0, stage_bytes, c.stream) != cudaSuccess ||
                        cudaEventRecord(ev[0], c.stream) != cudaSuccess) {
                        st = BMG_ERR_DEVICE;
                        break;
                    }
                    if ((st = fused_down(c, l, ir)) != BMG_OK) break;
                    if (cudaEventRecord(ev[1], c.stream) != cudaSuccess) {
                        st = BMG_ERR_DEVICE;
                        break;
                    }
                    if ((st = fused_up(c, l, out, ir)) != BMG_OK) break;
                    float td = 0.f, tu = 0.f;
                    if (cudaEventRecord(ev[2], c.stream) != cudaSuccess || cudaEventSynchronize(ev[2]) != cudaSuccess ||
                        cudaEventElapsedTime(&td, ev[0], ev[1]) != cudaSuccess ||
                        cudaEventElapsedTime(&tu, ev[1], ev[2]) != cudaSuccess) {
                        st = BMG_ERR_DEVICE;
                        break;
                    }
                    if (bd < 0 || td < bd) {
                        bd = td;
                        hd = hc;
                    }
                    if (bu < 0 || tu < bu) {
                        bu = tu;
                        hu = hc;
                    }
                }
            }
            if (st == BMG_OK && bd >= 0 && (best < 0 || bd + bu < best)) {
                best = bd + bu;
                best_wc = wc;
                best_hd = hd;
                best_hu = hu;
            }
        }
        if (st == BMG_OK) st = fused_configure(c, l, best_wc, best_hd, best_hu);
        total += best;
    }
    for (int i = 0; i < 3; i++) cudaEventDestroy(ev[i]);
    if (best_ms_total) *best_ms_total = total;
    return st;
}

}  // namespace bmg
