// fused2d.cuh -- launch descriptors of the streaming 2-D V-cycle kernels.
#pragma once

#include <cuda.h>

namespace bmg {

struct KState;

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
};

// Per fine level: tile shape and TMA descriptors (built at attach time).
struct FusedLevel {
    bool ready = false;
    int wc = 0, hc = 0, tiles_x = 0, tiles_y = 0;
    CUtensorMap mA;    // stencil planes, 3-D box (2*wc+16) x 2 rows x planes
    CUtensorMap mF;    // right-hand side rows
    CUtensorMap mXp;   // pre-smoothed iterate rows
    CUtensorMap mXc;   // coarse final iterate rows
    FusedArgs down, up;
};

}  // namespace bmg
