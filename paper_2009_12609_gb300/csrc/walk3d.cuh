// walk3d.cuh -- integer ray walk through a regular N^3 grid (Sect. 2.2).
//
// The ray lattice is defined in fixed point so that every implementation
// finds the same cells and lengths: one root cell is H = 2^F units, axes
// with a negative direction component are mirrored so the ray moves towards
// +main, +a, +b, and the root line (i, j) passes at main-axis coordinate z
// through A(z) = o + i H + floor(q_a z / 2^F) (mod N H), likewise B(z), with
// o = H / 2.  A segment is a maximal run of integer z inside one cell.
// Because q <= 2^F the transverse coordinate moves by at most one unit per
// unit of z, so boundaries are met one at a time and the next crossing of a
// boundary at offset `target` is z = ceil(target 2^F / q).
#pragma once

#include "loc_internal.cuh"

namespace loc {

__device__ __forceinline__ long long next_cross(long long q, long long target)
{
    if (q <= 0) return LLONG_MAX;
    const unsigned long long num = (unsigned long long)target << kFixedBits;
    return (long long)((num + (unsigned long long)q - 1ull) / (unsigned long long)q);
}

// Walks root line (i, j) of direction D on an N^3 grid and calls
// f(cell, dz) for every segment in order.  All lanes of a warp may run it
// redundantly (uniform control flow).
template <class F>
__device__ __forceinline__ void walk_grid3d(const Dir3D &D, int N, long long i, long long j, F &&f)
{
    const long long H = 1ll << kFixedBits;
    const long long E = (long long)N * H;
    const long long o = H >> 1;
    long long ta = H - o;           // next a-boundary, relative to A(0)
    long long tb = H - o;
    long long za = next_cross(D.qa, ta);
    long long zb = next_cross(D.qb, tb);
    int ia = (int)i, ib = (int)j, im = 0;   // (o + i H) / H = i
    long long z = 0;
    while (z < E) {
        const long long zm = (long long)(im + 1) * H;
        long long zn = zm;
        if (za < zn) zn = za;
        if (zb < zn) zn = zb;
        int idx[3];
        idx[D.m] = im;
        idx[D.a] = ia;
        idx[D.b] = ib;
        const int ix = D.flip[0] ? N - 1 - idx[0] : idx[0];
        const int iy = D.flip[1] ? N - 1 - idx[1] : idx[1];
        const int iz = D.flip[2] ? N - 1 - idx[2] : idx[2];
        const long long cell = ((long long)iz * N + iy) * N + ix;
        f(cell, zn - z);
        z = zn;
        if (z == zm) im++;
        if (z == za) { ia = (ia + 1 == N) ? 0 : ia + 1; ta += H; za = next_cross(D.qa, ta); }
        if (z == zb) { ib = (ib + 1 == N) ? 0 : ib + 1; tb += H; zb = next_cross(D.qb, tb); }
    }
}

}  // namespace loc
