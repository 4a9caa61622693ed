// grid3.cuh -- 3-D stencil and interpolation accessors (device).
//
// Node (i,j,k) of a level lives at i + ld*(j + n*k).  Offsets d in
// {-1,0,1}^3 are numbered o = (dx+1) + 3(dy+1) + 9(dz+1); o = 13 is the centre
// and o < 13 are the lexicographically negative offsets.  The symmetric half
// is stored as planes 0..13 (plane o holds offset o at the node);
// a(+d) at node i is plane 26-o at node i+d.
//
// Interpolation: the 7 fine points owned by coarse node (I,J,K) are
// (2I,2J,2K) + b with b a non-zero parity mask m (bit 0: x, 1: y, 2: z).
// Point m has 2^popcount(m) weights, to the coarse nodes (I,J,K) + s with s a
// subset of m; they are stored in planes kPBase[m] + compress(s, m).
#pragma once

#include "common.cuh"

namespace bmg {

__host__ __device__ constexpr int kPBase(int m) {
    return m == 1 ? 0 : m == 2 ? 2 : m == 4 ? 4 : m == 3 ? 6 : m == 5 ? 10 : m == 6 ? 14 : 18;
}

__host__ __device__ __forceinline__ int off_x(int o) { return o % 3 - 1; }
__host__ __device__ __forceinline__ int off_y(int o) { return (o / 3) % 3 - 1; }
__host__ __device__ __forceinline__ int off_z(int o) { return o / 9 - 1; }

// index of the subset s of m in the compressed numbering (bits of s at m's set bits)
__host__ __device__ __forceinline__ int compress3(int s, int m) {
    int r = 0, b = 0;
    for (int a = 0; a < 3; a++)
        if ((m >> a) & 1) {
            r |= ((s >> a) & 1) << b;
            b++;
        }
    return r;
}

template <typename T>
struct Sten3 {
    const T* a;
    int n, ld;
    long long pl;
    __device__ __forceinline__ long long idx(int i, int j, int k) const {
        return (long long)i + (long long)ld * (j + (long long)n * k);
    }
    __device__ __forceinline__ T full(int i, int j, int k, int o) const {
        if (o <= 13) return a[(long long)o * pl + idx(i, j, k)];
        return a[(long long)(26 - o) * pl + idx(i + off_x(o), j + off_y(o), k + off_z(o))];
    }
};

// Weight of fine node (fi,fj,fk) of an nf-grid to coarse node (KI,KJ,KK);
// P planes live on the coarse grid (ldc, nc, plane stride plc).
template <typename T>
__device__ __forceinline__ T pweight3(const T* __restrict__ P, int ldc, int nc, long long plc, int nf, int fi, int fj,
                                      int fk, int KI, int KJ, int KK) {
    if (fi < 1 || fj < 1 || fk < 1 || fi > nf - 2 || fj > nf - 2 || fk > nf - 2) return (T)0;
    const int m = (fi & 1) | ((fj & 1) << 1) | ((fk & 1) << 2);
    const int I = fi >> 1, J = fj >> 1, K = fk >> 1;
    const int dI = KI - I, dJ = KJ - J, dK = KK - K;
    if (dI < 0 || dJ < 0 || dK < 0 || dI > (m & 1) || dJ > ((m >> 1) & 1) || dK > ((m >> 2) & 1)) return (T)0;
    if (m == 0) return (T)1;
    const int s = dI | (dJ << 1) | (dK << 2);
    const int plane = kPBase(m) + compress3(s, m);
    return P[(long long)plane * plc + (long long)I + (long long)ldc * (J + (long long)nc * K)];
}

}  // namespace bmg
