// fused2d.cuh -- launch descriptors of the streaming 2-D V-cycle kernels.
#pragma once

#include <cuda.h>

namespace bmg {

struct KState;
struct SysState;

// One (problem, level) of a batch size class: where the batched kernels
// write and read what is not streamed through the class's tensor maps.
// Vectors are interleaved, R values per node (one per right-hand side).
struct BatchMember {
    void* x[2];          // down: pre-smoothed iterate (x[0]); up: final iterate, per parity of the
                         // z buffers on a problem's finest level (x[0] == x[1] on the others)
    void* bc;            // down: coarse right-hand side
    const void* P;       // interpolation planes of the level (coarse grid), scalar
    const void* zold[2]; // up, finest level: z_old per parity (null on the other levels)
    int cmem;            // member index of the coarse level in its class (coarse iterate map)
    int prob;            // problem index; its systems are prob*R .. prob*R+R-1
    int finest;          // 1: the problem's finest level (its up kernel also forms the CG beta)
    long long part;      // first tile partial of this member (finest up kernel)
};

// Kernel arguments shared by the down and up kernels of one level pair.
struct FusedArgs {
    int nf, nc;      // nodes per side, fine and coarse
    int ldf, ldc;    // padded row lengths
    int wc, hc;      // coarse columns / rows owned by one CTA
    void* x;         // down: pre-smoothed fine iterate (out); up: final fine iterate (out)
    void* bc;        // down: coarse right-hand side (out)
    const void* P;   // interpolation planes (coarse grid)
    long long plc;   // plane stride of P
    KState* st;
    // up kernel, finest level of the refinement mode: r.z and r.z_old of the
    // owned nodes (r = this kernel's right-hand side, z = its output) reduced
    // into the CG coefficient; null when not wanted
    const void* zold;
    double* partials;
    // batched kernels: a persistent grid walks the work-list of (member,
    // tile) items of one size class; members describe each (problem, level)
    const BatchMember* mem = nullptr;
    int nmem = 0, tiles_x = 0, tiles_y = 0;
    int parity = 0;              // z buffer written by the finest up kernels
    SysState* sys = nullptr;     // per-system CG scalars
    unsigned int* counters = nullptr;   // per-problem arrival counters (finest up kernel)
};

// Per fine level: tile shape and TMA descriptors (built at attach time).
struct FusedLevel {
    bool ready = false;
    // one strip width for both kernels (the TMA boxes depend on it); rows per
    // CTA for each kernel (hc: down, hc_up: up)
    int wc = 0, hc = 0, tiles_x = 0, tiles_y = 0, hc_up = 0, tiles_y_up = 0;
    CUtensorMap mA;    // stencil planes, 3-D box (2*wc+16) x 2 rows x planes
    CUtensorMap mF;    // right-hand side rows
    CUtensorMap mXp;   // pre-smoothed iterate rows
    CUtensorMap mXc;   // coarse final iterate rows
    FusedArgs down, up;
};

}  // namespace bmg
