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

bmg_status fused_prepare(Ctx& c) {
    const bool f32 = c.opts.precision == BMG_PREC_FP32;
    int sms = 0;
    BMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device));
    for (int l = 0; l + 1 < c.nlev; l++) {
        FusedLevel& F = c.fused[l];
        const Level& Lf = c.lev[l];
        const Level& Lc = c.lev[l + 1];
        // Tiles cover coarse indices 1 .. nc-1: coarse index J owns the fine rows
        // 2J-1 and 2J, so the boundary index nc-1 still owns fine row nf-2.
        const int m = Lc.n - 1;
        F.wc = m >= 512 ? 64 : m >= 128 ? 32 : m >= 32 ? 16 : 8;
        F.tiles_x = cdiv(m, F.wc);
        int od = 0, ou = 0;
        BMG_TRY(fused_occupancy(f32, f32 && l == 0, F.wc, &od, &ou));
        const int occ = od < ou ? od : ou;
        if (occ < 1) return BMG_ERR_DEVICE;
        const long long slots = (long long)occ * sms;
        // rows per CTA (a multiple of the rows per step): minimise waves x (rows + pre-roll)
        const int K = fused_rows_per_step(f32);
        long long best = -1;
        for (int ty = 1; ty <= m; ty++) {
            const int hc = cdiv(cdiv(m, ty), K) * K;
            const int tyr = cdiv(m, hc);
            const long long waves = cdiv((long long)F.tiles_x * tyr, slots);
            const long long cost = waves * (2LL * hc + 3);
            if (best < 0 || cost < best) {
                best = cost;
                F.hc = hc;
                F.tiles_y = tyr;
            }
        }
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
        F.down = FusedArgs{Lf.n, Lc.n, Lf.ld, Lc.ld, F.wc, F.hc, Lf.x, Lc.b, P, Lc.plane, c.st};
        F.up = FusedArgs{Lf.n, Lc.n, Lf.ld, Lc.ld, F.wc, F.hc, nullptr, nullptr, P, Lc.plane, c.st};
        F.ready = true;
        if (l == 0 && c.r32) {
            // refinement mode: the level-0 kernels read the FP32 inner residual
            FusedLevel& G = c.fused_ir0;
            G = F;
            int od2 = 0, ou2 = 0;
            BMG_TRY(fused_occupancy(true, false, F.wc, &od2, &ou2));
            if (!make_map(&G.mF, false, c.r32, Lf.ld, Lf.n, 1, Lf.plane, WW, 2)) return BMG_ERR_DEVICE;
        }
    }
    return BMG_OK;
}

}  // namespace bmg
