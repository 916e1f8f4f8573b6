// walk3d.cuh -- integer ray walk through a regular N^3 grid (Sect. 2.2).
//
// The ray lattice is defined in fixed point so that every implementation
// finds the same cells and lengths: one root cell is H = 2^F units, axes
// with a negative direction component are mirrored so the ray moves towards
// +main, +a, +b, and the root line (i, j) passes at main-axis coordinate z
// through A(z) = o + i H + floor(q_a z / 2^F) (mod N H), likewise B(z), with
// o = H / 2.  A segment is a maximal run of integer z inside one cell.
// Because q <= 2^F the transverse coordinate moves by at most one unit per
// unit of z, so boundaries are met one at a time; the crossing of the
// boundary at offset `target` is z = ceil(target 2^F / q).  Successive
// targets differ by H, so the walk carries the quotient and remainder of
// target 2^F / q and advances them by the per-direction constants
// H 2^F = D q + r: no division inside the walk.
#pragma once

#include "loc_internal.cuh"

namespace loc {

// z, the crossings and the main-axis boundary fit in 32 bits for grids of up
// to 255 root cells per side (255 x 2^24 < 2^32); the quotient / remainder
// state stays 64-bit and is only touched when a crossing happens.
constexpr unsigned kNever = 0xffffffffu;

__device__ __forceinline__ unsigned sat32(long long v)
{
    return (v >= (long long)kNever) ? kNever : (unsigned)v;
}

struct GridWalk {
    unsigned z, za, zb;         // current z, next a / b crossing
    long long Qa, Ra, Qb, Rb;   // quotient / remainder of the current targets
    int ia, ib, im;             // (mirrored) cell indices along a, b, main

    __device__ __forceinline__ void init(const Dir3D &D, long long i, long long j)
    {
        z = 0;
        ia = (int)i;
        ib = (int)j;
        im = 0;
        Qa = D.Qa0; Ra = D.Ra0;
        Qb = D.Qb0; Rb = D.Rb0;
        za = (D.qa > 0) ? sat32(Qa + (Ra > 0)) : kNever;
        zb = (D.qb > 0) ? sat32(Qb + (Rb > 0)) : kNever;
    }

    __device__ __forceinline__ bool done(int N) const
    {
        return z >= ((unsigned)N << kFixedBits);
    }

    // Current segment's cell (x fastest) and length; advances the walk.
    __device__ __forceinline__ void step(const Dir3D &D, int N, long long &cell, long long &dz)
    {
        const unsigned zm = (unsigned)(im + 1) << kFixedBits;
        unsigned zn = zm;
        if (za < zn) zn = za;
        if (zb < zn) zn = zb;
        int idx[3];
        idx[D.m] = im;
        idx[D.a] = ia;
        idx[D.b] = ib;
        const int ix = D.flip[0] ? N - 1 - idx[0] : idx[0];
        const int iy = D.flip[1] ? N - 1 - idx[1] : idx[1];
        const int iz = D.flip[2] ? N - 1 - idx[2] : idx[2];
        cell = ((long long)iz * N + iy) * N + ix;
        dz = (long long)(zn - z);
        z = zn;
        if (z == zm) im++;
        if (z == za) {
            ia = (ia + 1 == N) ? 0 : ia + 1;
            Qa += D.Da; Ra += D.ra;
            if (Ra >= D.qa) { Ra -= D.qa; Qa++; }
            za = sat32(Qa + (Ra > 0));
        }
        if (z == zb) {
            ib = (ib + 1 == N) ? 0 : ib + 1;
            Qb += D.Db; Rb += D.rb;
            if (Rb >= D.qb) { Rb -= D.qb; Qb++; }
            zb = sat32(Qb + (Rb > 0));
        }
    }
};

// Walks root line (i, j) of direction D and calls f(cell, dz) per segment.
template <class F>
__device__ __forceinline__ void walk_grid3d(const Dir3D &D, int N, long long i, long long j, F &&f)
{
    GridWalk w;
    w.init(D, i, j);
    while (!w.done(N)) {
        long long c, dz;
        w.step(D, N, c, dz);
        f(c, dz);
    }
}

}  // namespace loc
