// noalloc.cu -- operator assembly that allocates nothing.
//
// bmg_assemble works in the caller's workspace, which the caller has to
// allocate and attach to a context first.  Some callers cannot do that: code
// that runs while another allocator owns the device memory (a framework's
// caching pool that must not be bypassed), code under a hard memory cap, or
// code on a path where an allocation would synchronise the device or is not
// permitted at all.  For them bmg_assemble_noalloc produces the same finest
// operator without a context, a workspace or any allocating call: its
// working storage (the device error word and the half-plane operator) is a
// fixed static device array of BMG_NOALLOC_SCRATCH_BYTES, and the result is
// written, as full 3^d-entry rows, into the caller's buffer.
#include <mutex>

#include "common.cuh"

namespace {

// Working storage: [0, 256) the error word (a KState), then the half planes.
constexpr size_t kStateBytes = 256;
static_assert(sizeof(bmg::KState) <= kStateBytes, "KState must fit its reserved slot");

__device__ __align__(256) unsigned char g_scratch[BMG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// True for device (or managed) memory of the calling thread's current
// device; a pointer into another GPU's memory is refused rather than
// dereferenced as a peer access.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == dev;
    return a.type == cudaMemoryTypeManaged;
}

// Whether the half-plane operator of an n-node grid (2-D: 5 planes of ld*n
// doubles; 3-D: 14 planes of ld*n*n) and the error word fit the static
// array.  n is bounded first, so none of the products can overflow.
bool fits_scratch(int dim, int n) {
    if (n < 3 || n > 4096) return false;
    const unsigned long long ld = ((unsigned long long)n + 31) & ~31ull;
    const unsigned long long pl = dim == 2 ? ld * n : ld * n * (unsigned long long)n;
    const unsigned long long planes = dim == 2 ? bmg::NS2 : bmg::NS3;
    return kStateBytes + planes * pl * sizeof(double) <= (unsigned long long)BMG_NOALLOC_SCRATCH_BYTES;
}

// Address of the static array on the current device, resolved once per device.
bmg_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BMG_ERR_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return BMG_ERR_DEVICE;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return BMG_OK;
}

}  // namespace

extern "C" bmg_status bmg_assemble_noalloc(int dim, int n, const double* coords, const double* kappa,
                                           double* stencil, void* stream) {
    if (dim != 2 && dim != 3) return BMG_ERR_SHAPE;
    if (!fits_scratch(dim, n)) return BMG_ERR_SHAPE;   // checked on n before any size arithmetic
    const long long ld = (n + 31) & ~31;
    const long long pl = dim == 2 ? ld * n : ld * n * (long long)n;
    if (!coords || !kappa || !stencil) return BMG_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BMG_ERR_DEVICE;
    if (!on_device(coords, dev) || !on_device(kappa, dev) || !on_device(stencil, dev)) return BMG_ERR_ARG;
    void* base = nullptr;
    BMG_TRY(scratch_address(&base));
    bmg::KState* st = (bmg::KState*)base;
    double* A = (double*)((unsigned char*)base + kStateBytes);
    cudaStream_t s = (cudaStream_t)stream;
    // the error word must start at zero; the half planes are written in full
    BMG_CUDA(cudaMemsetAsync(st, 0, sizeof(bmg::KState), s));
    BMG_TRY(dim == 2 ? bmg::assemble_export2d(n, (int)ld, pl, coords, kappa, A, st, stencil, s)
                     : bmg::assemble_export3d(n, (int)ld, pl, coords, kappa, A, st, stencil, s));
    // `err` is pageable stack memory: the asynchronous copy into it is only
    // complete, and `err` only safe to read or leave, after the stream
    // synchronisation that follows.  Keep the two together.
    int err = 0;
    BMG_CUDA(cudaMemcpyAsync(&err, &st->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BMG_CUDA(cudaStreamSynchronize(s));
    return err ? (bmg_status)err : BMG_OK;
}
