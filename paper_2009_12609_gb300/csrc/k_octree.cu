// k_octree.cu -- ray march over octree grids (Sect. 2.2).
//
// Ray lattice as for regular grids (walk3d.cuh), at every refinement level:
// line (lam, i, j) passes through A(z) = o + i (H0 >> lam) + floor(q_a z / 2^F)
// (likewise B) with the common offset o = (H0 >> Lmax) / 2, so coarser
// lattices are contained in finer ones.  A line's creation level lam is the
// coarsest level whose lattice holds it; it is active in a leaf iff the leaf's
// level >= lam.  This is the effect of the paper's rules -- rays split into
// four at the upstream border of a refined cell, side rays added where a
// neighbour is less refined, rays terminated on entering coarser cells,
// re-entry on the opposite side -- and gives every level-L leaf exactly the
// level-L lattice, i.e. a constant path length per cell and direction.
//
// Every refined cell C (level k) is entered through its upstream face by
// exactly one active line of level <= k.  When that line reaches the face it
// creates C's new rays: the level-(k+1) lines that become active inside C,
// through the face (split) or through a side face (side rays), each
// starting with the creating line's intensity at the face.  New rays are
// followed first (depth first, "higher levels first"), then the creating
// line resumes: one stack frame per refinement level, holding one intensity
// snapshot that both initialises the new rays and restores the parent.
//
// GB300 mapping: persistent warps take (direction, root line, line group)
// items from a counter; lanes over channels in the per-step update
// (march_step, shared with the other geometries); the 25 candidate lines of
// a refined cell are examined one per lane (entry point, and whether the line
// was inactive just before -- one octree descent each) and collected with a
// ballot; point location is an integer descent through the child array.
#include <algorithm>

#include "k_march.cuh"

namespace loc {

constexpr int kOctWarpsPerBlock = 4;
static_assert(kOctWarpsPerBlock <= kWarpsPerBlock, "march_step's per-warp tiles are sized for kWarpsPerBlock warps");
constexpr int kOctBlocksPerSM = 4;
constexpr int kOctMaxBlocksPerSM = 8;       // replay: up to 32 warps per SM
constexpr int kOctMaxDepth = 10;

// floor(n / q) with minv = floor((2^64 - 1) / q): one correction step
__device__ __forceinline__ unsigned long long udivq(unsigned long long n, unsigned long long q,
                                                    unsigned long long minv)
{
    unsigned long long t = __umul64hi(n, minv);
    if (n - t * q >= q) t++;
    return t;
}

// smallest z with floor(q z / 2^F) >= target (target >= 1, q > 0)
__device__ __forceinline__ long long cross_z(long long target, long long q, unsigned long long minv)
{
    const unsigned long long num = ((unsigned long long)target << kFixedBits) + (unsigned long long)q - 1ull;
    return (long long)udivq(num, (unsigned long long)q, minv);
}

__device__ __forceinline__ long long fq(long long q, long long z) { return (q * z) >> kFixedBits; }

// A lattice coordinate A = A0 + floor(q z / 2^F) reduced modulo the model
// width E: A0 < E (line offset) and floor(q z / 2^F) <= z < E (slope <= 1),
// so A < 2 E and one conditional subtraction replaces a 64-bit division.
__device__ __forceinline__ long long wrap_e(long long A, long long E) { return A >= E ? A - E : A; }

// v mod M in [0, M) for v within a few M of that range (no 64-bit division)
__device__ __forceinline__ long long mod_near(long long v, long long M)
{
    while (v < 0) v += M;
    while (v >= M) v -= M;
    return v;
}

struct OctGeo {
    Dir3D D;
    long long E, o;
    int N, Lmax;
};

__device__ __forceinline__ void oct_point(const OctGeo &g, long long Au, long long Bu, long long z, long long p[3])
{
    long long mm[3];
    mm[g.D.m] = z;
    mm[g.D.a] = wrap_e(Au, g.E);
    mm[g.D.b] = wrap_e(Bu, g.E);
#pragma unroll
    for (int ax = 0; ax < 3; ax++) p[ax] = g.D.flip[ax] ? g.E - 1 - mm[ax] : mm[ax];
}

// cell containing p, descending at most max_level levels; level receives it
__device__ __forceinline__ int oct_locate(const DevModel &m, const OctGeo &g, const long long p[3],
                                          int max_level, int &level)
{
    const int F = kFixedBits;
    int c = (int)(((p[2] >> F) * g.N + (p[1] >> F)) * g.N + (p[0] >> F));
    int L = 0;
    while (L < max_level) {
        const int ch = __ldg(m.child + c);
        if (ch < 0) break;
        L++;
        const int sh = F - L;
        c = ch + (int)(((p[0] >> sh) & 1) | (((p[1] >> sh) & 1) << 1) | (((p[2] >> sh) & 1) << 2));
    }
    level = L;
    return c;
}

// Ancestor cache of the last point located by a warp's march: the point and
// its leaf level (registers, the same in every lane) and the cells of its
// path from the root (shared memory, path[0..L]).  The next point shares
// every level whose box holds both points, so its descent restarts from the
// deepest such ancestor -- usually the parent -- instead of the root.
struct OctPathCache {
    long long p[3];
    int L;                  // -1: empty
};

__device__ __forceinline__ int oct_locate_cached(const DevModel &m, const OctGeo &g, const long long p[3],
                                                 int &level, OctPathCache &pc, int *path, int lane)
{
    const int F = kFixedBits;
    const unsigned long long x = (unsigned long long)((p[0] ^ pc.p[0]) | (p[1] ^ pc.p[1]) | (p[2] ^ pc.p[2]));
    int s;                  // deepest level whose cell holds both points
    if (pc.L < 0 || (x >> F) != 0) s = -1;
    else if (x == 0) s = pc.L;
    else s = min(F - 1 - (63 - __clzll((long long)x)), pc.L);
    int c, L;
    if (s < 0) {
        c = (int)(((p[2] >> F) * g.N + (p[1] >> F)) * g.N + (p[0] >> F));
        L = 0;
        if (lane == 0) path[0] = c;
    } else {
        c = path[s];
        L = s;
    }
    while (L < g.Lmax) {
        const int ch = __ldg(m.child + c);
        if (ch < 0) break;
        L++;
        const int sh = F - L;
        c = ch + (int)(((p[0] >> sh) & 1) | (((p[1] >> sh) & 1) << 1) | (((p[2] >> sh) & 1) << 2));
        if (lane == 0) path[L] = c;
    }
    __syncwarp();
    pc.p[0] = p[0];
    pc.p[1] = p[1];
    pc.p[2] = p[2];
    pc.L = L;
    level = L;
    return c;
}

// mirrored lower corner of the level-L box containing original coordinate v
__device__ __forceinline__ long long oct_mlo(const OctGeo &g, int ax, long long v, int L)
{
    const int sh = kFixedBits - L;
    const long long H = 1ll << sh;
    const long long lo = (v >> sh) << sh;
    return g.D.flip[ax] ? g.E - lo - H : lo;
}

struct OctLine {
    int lam, i, j;
    long long z;
};

// Per-warp frame of the depth-first traversal (shared memory).
struct OctFrame {
    int lam, i, j;          // paused creating line
    long long z;            // its position (the face where it created rays)
    int n_kids, next;       // new rays of this frame, next one to start
};

// Creates the rays of refined cell (level k) entered by line `cur` at its
// upstream face cur.z; appends them to kids[] from index *nk.  All lanes.
__device__ __forceinline__ void oct_spawn(const DevModel &m, const OctGeo &g, const OctLine &cur,
                                          const long long p[3], int k, int4 *kids, int &nk, int lane)
{
    const long long H0 = 1ll << kFixedBits;
    const long long H = H0 >> k, Hc = H >> 1;
    const long long zf = cur.z;
    const long long ma0 = oct_mlo(g, g.D.a, p[g.D.a], k);
    const long long mb0 = oct_mlo(g, g.D.b, p[g.D.b], k);
    const long long fa = fq(g.D.qa, zf), fb = fq(g.D.qb, zf);
    const long long da = fq(g.D.qa, zf + H - 1) - fa, db = fq(g.D.qb, zf + H - 1) - fb;
    const long long Mc = (long long)g.N << (k + 1);
    // first candidate index along each axis: lattice position >= box lower bound - drift
    // (ma0, fa < E; da <= H, o < H0 <= E: the argument lies in (-3E, E))
    const long long xa = mod_near(ma0 - da - g.o - fa, g.E);
    const long long xb = mod_near(mb0 - db - g.o - fb, g.E);
    const int shc = kFixedBits - k - 1;                 // Hc = 2^shc
    const long long ia0 = (xa + Hc - 1) >> shc, jb0 = (xb + Hc - 1) >> shc;
    bool is_new = false;
    int ci = 0, cj = 0;
    long long zin = 0;
    // at most 4 lattice lines per axis can meet the box; small lattices (fewer
    // than 5 lines) are enumerated once each instead of wrapping onto themselves
    const int nu = (int)min(5ll, Mc);
    const int cu = lane / 5, cv = lane % 5;
    if (lane < 25 && cu < nu && cv < nu) {
        ci = (int)mod_near(ia0 + cu, Mc);               // ia0 <= Mc: at most Mc + 4
        cj = (int)mod_near(jb0 + cv, Mc);
        if ((ci & 1) || (cj & 1)) {                      // creation level k + 1
            const long long A0 = g.o + (long long)ci * Hc, B0 = g.o + (long long)cj * Hc;
            // offset from the box's lower bound: [0, H) inside, otherwise taken
            // as before the box (the line may still drift into it)
            long long ar = mod_near(A0 + fa - ma0, g.E);     // argument in (-E, 2E)
            if (ar >= H) ar -= g.E;
            long long br = mod_near(B0 + fb - mb0, g.E);
            if (br >= H) br -= g.E;
            const long long NEVER = 1ll << 62;
            bool ok = (ar >= -da) && (ar < H) && (br >= -db) && (br < H);
            long long za_in = zf, zb_in = zf, za_out = NEVER, zb_out = NEVER;
            if (ok) {
                if (ar < 0) za_in = (g.D.qa > 0) ? cross_z(fa - ar, g.D.qa, g.D.ma) : NEVER;
                if (br < 0) zb_in = (g.D.qb > 0) ? cross_z(fb - br, g.D.qb, g.D.mb) : NEVER;
                if (g.D.qa > 0) za_out = cross_z(fa - ar + H, g.D.qa, g.D.ma);
                if (g.D.qb > 0) zb_out = cross_z(fb - br + H, g.D.qb, g.D.mb);
                zin = max(zf, max(za_in, zb_in));
                const long long zout = min(zf + H, min(za_out, zb_out));
                ok = zin < zout;
            }
            if (ok) {
                if (zin == 0) {
                    is_new = true;
                } else {                                  // inactive just before entering?
                    long long q[3];
                    oct_point(g, A0 + fq(g.D.qa, zin - 1), B0 + fq(g.D.qb, zin - 1), zin - 1, q);
                    int lev;
                    oct_locate(m, g, q, k + 1, lev);
                    is_new = lev < k + 1;
                }
            }
        }
    }
    const unsigned mask = __ballot_sync(kFull, is_new);
    if (is_new) {
        const int slot = nk + __popc(mask & ((1u << lane) - 1u));
        if (slot < kOctMaxKids) kids[slot] = make_int4(k + 1, ci, cj, (int)(unsigned)zin);
    }
    nk += __popc(mask);
}

// Path records of a root-ray family, in the order of the depth-first
// traversal: one 64-bit word per active step or intensity copy.
//   step:  leaf (bits 0-31), dz (bits 32-56, at most 2^24), leaf level
//          (bits 57-60), type 0 (bits 61-63)
//   save:  type 1, frame depth in bits 0-31 (snapshot I before new rays)
//   load:  type 2, frame depth in bits 0-31 (I from that snapshot: the start
//          of a new ray, or the creating line resuming)
constexpr unsigned kRecStep = 0, kRecSave = 1, kRecLoad = 2;

__device__ __forceinline__ unsigned long long rec_step(int leaf, long long dz, int level)
{
    return (unsigned long long)(unsigned)leaf | ((unsigned long long)dz << 32) |
           ((unsigned long long)level << 57);
}

__device__ __forceinline__ unsigned long long rec_ctrl(unsigned type, int depth)
{
    return (unsigned long long)(unsigned)depth | ((unsigned long long)type << 61);
}

// Weight of a step of main-axis length dz through a level-L leaf, dz / H_L
// / n_dir (H_L = 2^(24 - L) units): the division by a power of two is exact,
// so it is a multiplication by 2^(L - 24).
__device__ __forceinline__ float oct_weight(long long dz, int L, float wscale)
{
    return (float)(int)dz * __int_as_float((127 + L - kFixedBits) << 23) * wscale;
}

// Visitors of the traversal: the march applies each step to the warp's
// intensities (kNeedI); the others only see the geometry.
struct OctMarchVisitor {
    static constexpr bool kNeedI = true;
    __device__ void step(int, const OctLine &, long long, int, int) {}
    __device__ void save(int, int) {}
    __device__ void load(int, int) {}
};

struct OctTraceVisitor {
    static constexpr bool kNeedI = false;
    long long *out;            // records {level, i, j, z0, dz, leaf, leaf level}
    long long cap;
    unsigned long long *count;
    unsigned long long *sums;  // optional per-leaf sum of dz
    int dir;
    unsigned local;            // active steps of the current family (added to *count
                               // once per family when nothing is listed)
    unsigned ctrl;             // intensity copies (saves and loads) of the family
    __device__ void step(int lane, const OctLine &cur, long long dz, int leaf, int Lc)
    {
        local++;
        if (lane == 0) {
            if (sums) atomicAdd(sums + leaf, (unsigned long long)dz);
            if (count && out) {                  // listing: one slot per step
                const unsigned long long n = atomicAdd(count, 1ull);
                if ((long long)n < cap) {
                    long long *o = out + 7 * n;
                    o[0] = cur.lam; o[1] = cur.i; o[2] = cur.j; o[3] = cur.z; o[4] = dz;
                    o[5] = leaf; o[6] = Lc;
                }
            }
        }
    }
    __device__ void save(int, int) { ctrl++; }
    __device__ void load(int, int) { ctrl++; }
};

// Writes the path records of one family to rec[0 .. n).  Every lane calls
// put with the same record; lane k keeps record k of the current block of
// 32, and each full block is written by one coalesced store of the warp
// (flush once more at the end of the family for a partial block).
struct OctRecVisitor {
    static constexpr bool kNeedI = false;
    unsigned long long *rec;
    long long n, cap;
    unsigned long long buf;
    __device__ void flush(int lane)
    {
        const long long k = ((n - 1) & ~31ll) + lane;
        if (k < n && k < cap) rec[k] = buf;
    }
    __device__ void put(int lane, unsigned long long w)
    {
        if (lane == (int)(n & 31)) buf = w;
        n++;
        if ((n & 31) == 0) flush(lane);
    }
    __device__ void step(int lane, const OctLine &, long long dz, int leaf, int Lc)
    {
        put(lane, rec_step(leaf, dz, Lc));
    }
    __device__ void save(int lane, int depth) { put(lane, rec_ctrl(kRecSave, depth)); }
    __device__ void load(int lane, int depth) { put(lane, rec_ctrl(kRecLoad, depth)); }
};

// Depth-first traversal of the rays created from root line (i, j).
template <int G, int ACC, class V>
__device__ void oct_traverse(const DevModel &m, const MarchArgs &a, const OctGeo &g, int i, int j,
                             float *I, float *snap, int4 *kids_all, OctFrame *fr, int *path, int lane,
                             V &vis, long long &nw)
{
    const long long H0 = 1ll << kFixedBits;
    const int snap_n = a.per * m.n_ch;
    const float wscale = 1.0f / (float)m.n_dir;
    (void)wscale;
    OctLine cur = {0, i, j, 0};
    long long skip_z = -1;          // a resumed line does not create rays twice at one face
    int depth = 0;
    OctPathCache pc;
    pc.p[0] = pc.p[1] = pc.p[2] = 0;
    pc.L = -1;
    MarchState pend = march_state();
    if (V::kNeedI) init_ray<G>(m, a, I, lane);
    while (true) {
        bool done_line = cur.z >= g.E;
        long long p[3];
        int Lc = 0;
        int cell = 0;
        long long Au = 0, Bu = 0;
        if (!done_line) {
            Au = g.o + (long long)cur.i * (H0 >> cur.lam) + fq(g.D.qa, cur.z);
            Bu = g.o + (long long)cur.j * (H0 >> cur.lam) + fq(g.D.qb, cur.z);
            oct_point(g, Au, Bu, cur.z, p);
            cell = oct_locate_cached(m, g, p, Lc, pc, path, lane);
            done_line = Lc < cur.lam;                       // entered a coarser leaf: terminated
        }
        if (!done_line && cur.z != skip_z) {
            // new rays of the refined cells whose upstream face this line enters now
            // (a line at depth d has creation level >= d, so depth < Lmax here)
            int nk = 0;
            if (depth < kOctMaxDepth) {
                int4 *kids = kids_all + depth * kOctMaxKids;
                for (int k = cur.lam; k < Lc; k++)
                    if (oct_mlo(g, g.D.m, p[g.D.m], k) == cur.z) oct_spawn(m, g, cur, p, k, kids, nk, lane);
            } else {
                for (int k = cur.lam; k < Lc; k++)
                    if (oct_mlo(g, g.D.m, p[g.D.m], k) == cur.z && lane == 0) atomicExch(m.oct_err, 3);
            }
            if (nk > kOctMaxKids) {
                if (lane == 0) atomicExch(m.oct_err, 1);
                nk = kOctMaxKids;
            }
            if (nk > 0) {
                if (depth >= kOctMaxDepth) {
                    if (lane == 0) atomicExch(m.oct_err, 2);
                } else {
                    if (lane == 0) {
                        fr[depth].lam = cur.lam; fr[depth].i = cur.i; fr[depth].j = cur.j;
                        fr[depth].z = cur.z; fr[depth].n_kids = nk; fr[depth].next = 0;
                    }
                    if (V::kNeedI) {
                        float *sn = snap + (size_t)depth * snap_n;
                        for (int q = lane; q < snap_n; q += 32) sn[q] = I[q];
                    }
                    vis.save(lane, depth);
                    depth++;
                    __syncwarp();
                    done_line = true;                       // switch to the first new ray below
                    skip_z = -1;
                }
            }
        }
        if (!done_line) {
            // one step through leaf `cell`
            const long long HL = H0 >> Lc;
            long long zn = oct_mlo(g, g.D.m, p[g.D.m], Lc) + HL;
            if (g.D.qa > 0) {
                const long long T = Au - wrap_e(Au, g.E) + oct_mlo(g, g.D.a, p[g.D.a], Lc) + HL;
                zn = min(zn, cross_z(T - (Au - fq(g.D.qa, cur.z)), g.D.qa, g.D.ma));
            }
            if (g.D.qb > 0) {
                const long long T = Bu - wrap_e(Bu, g.E) + oct_mlo(g, g.D.b, p[g.D.b], Lc) + HL;
                zn = min(zn, cross_z(T - (Bu - fq(g.D.qb, cur.z)), g.D.qb, g.D.mb));
            }
            zn = min(zn, g.E);
            const long long dz = zn - cur.z;
            const int leaf = __ldg(m.leaf_of + cell);
            if constexpr (V::kNeedI) {
                Step<G> st;
                st.cell = leaf;
                const float4 cv = m.vel[leaf];
                st.vlos = cv.x * g.D.d[0] + cv.y * g.D.d[1] + cv.z * g.D.d[2];
                st.inv = cv.w;
                st.s = (float)(int)dz * g.D.unit;       // dz <= one leaf <= 2^24 units
                st.w = oct_weight(dz, Lc, wscale);
                load_lines<G>(m, a, st, lane);
                nw += (long long)march_step<G, ACC>(m, a, I, st, lane, pend) * a.n_lines;
                __syncwarp();
            } else {
                vis.step(lane, cur, dz, leaf, Lc);
            }
            cur.z = zn;
            skip_z = -1;
            continue;
        }
        // the current line is finished (or paused): start the next new ray of
        // the innermost frame, or resume the line that created them
        if (depth == 0) {
            if (V::kNeedI) march_state_end<ACC>(m, a, pend, lane);
            break;
        }
        const int fi = depth - 1;
        OctFrame &f = fr[fi];
        const int nxt = f.next;
        const int nkids = f.n_kids;
        __syncwarp();
        if (nxt < nkids) {
            const int4 kd = kids_all[fi * kOctMaxKids + nxt];
            if (lane == 0) f.next = nxt + 1;
            cur.lam = kd.x; cur.i = kd.y; cur.j = kd.z; cur.z = (long long)(unsigned)kd.w;
            skip_z = -1;
        } else {
            cur.lam = f.lam; cur.i = f.i; cur.j = f.j; cur.z = f.z;
            skip_z = cur.z;
            depth = fi;
        }
        // new rays and the resumed line both start from the frame's snapshot
        if (V::kNeedI) {
            const float *src = snap + (size_t)fi * snap_n;
            for (int q = lane; q < snap_n; q += 32) I[q] = src[q];
        }
        vis.load(lane, fi);
        __syncwarp();
    }
}

template <int G, int ACC>
__global__ void __launch_bounds__(kOctWarpsPerBlock * 32) march_octree_kernel(DevModel m, MarchArgs a0,
                                                                               unsigned *counter)
{
    extern __shared__ float smem[];
    __shared__ OctFrame frames[kOctWarpsPerBlock][kOctMaxDepth];
    __shared__ int paths[kOctWarpsPerBlock][kOctMaxDepth + 1];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kOctWarpsPerBlock + wid;
    float *I = smem + (size_t)wid * a0.per * m.n_ch;
    float *snap = m.oct_scratch + (size_t)gw * kOctMaxDepth * a0.per * m.n_ch;
    int4 *kids = m.oct_kids + (size_t)gw * kOctMaxDepth * kOctMaxKids;
    const long long per_dir = (long long)m.N * m.N;
    const long long total = per_dir * m.n_dir * a0.n_groups;
    OctMarchVisitor vis;
    long long nw = 0;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((long long)it >= total) break;
        const long long fam = (long long)it / a0.n_groups;     // most work first
        const long long item = m.oct_order ? (long long)m.oct_order[fam] : fam;
        const int dir = (int)(item / per_dir);
        if (dir < a0.dir0 || dir >= a0.dir1) continue;          // another rank's direction
        const MarchArgs a = warp_args(m, a0, (int)((long long)it - fam * a0.n_groups));
        const long long r = item - (long long)dir * per_dir;
        OctGeo g;
        g.D = m.dirs[dir];
        g.N = m.N;
        g.Lmax = m.Lmax;
        g.E = (long long)m.N << kFixedBits;
        g.o = ((1ll << kFixedBits) >> m.Lmax) / 2;
        oct_traverse<G, ACC>(m, a, g, (int)(r / m.N), (int)(r % m.N), I, snap, kids, frames[wid], paths[wid],
                             lane, vis, nw);
    }
    if (a0.count && lane == 0) atomicAdd(m.upd_count, (unsigned long long)nw);   // nw counts lines
}

// Geometry of a traversal without intensities (tracing and recording).
__device__ __forceinline__ OctGeo oct_geo(const DevModel &m)
{
    OctGeo g;
    g.N = m.N;
    g.Lmax = m.Lmax;
    g.E = (long long)m.N << kFixedBits;
    g.o = ((1ll << kFixedBits) >> m.Lmax) / 2;
    return g;
}

__device__ __forceinline__ MarchArgs oct_geo_args()
{
    MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.per = 1;
    a.n_groups = 1;
    a.n_lines = 1;
    return a;
}

// fam_work[f]: active steps of family f; fam_rec[f]: its path records
// (steps, saves and loads); either may be null.
__global__ void __launch_bounds__(kOctWarpsPerBlock * 32) trace_octree_kernel(DevModel m, int dir,
                                                                               OctTraceVisitor vis,
                                                                               unsigned *counter,
                                                                               unsigned *fam_work,
                                                                               unsigned *fam_rec)
{
    __shared__ OctFrame frames[kOctWarpsPerBlock][kOctMaxDepth];
    __shared__ int paths[kOctWarpsPerBlock][kOctMaxDepth + 1];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kOctWarpsPerBlock + wid;
    int4 *kids = m.oct_kids + (size_t)gw * kOctMaxDepth * kOctMaxKids;
    const long long per_dir = (long long)m.N * m.N;
    const MarchArgs a = oct_geo_args();
    long long nw = 0;
    OctGeo g = oct_geo(m);
    // dir >= 0: the root lines of that direction; dir < 0: of every direction
    const long long total = dir >= 0 ? per_dir : per_dir * m.n_dir;
    while (true) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((long long)it >= total) break;
        const int d = dir >= 0 ? dir : (int)((long long)it / per_dir);
        const long long r = dir >= 0 ? (long long)it : (long long)it - (long long)d * per_dir;
        g.D = m.dirs[d];
        vis.local = 0;
        vis.ctrl = 0;
        oct_traverse<1, kAccPlain>(m, a, g, (int)(r / m.N), (int)(r % m.N), nullptr, nullptr, kids, frames[wid],
                        paths[wid], lane, vis, nw);
        if (vis.count && !vis.out && lane == 0 && vis.local) atomicAdd(vis.count, (unsigned long long)vis.local);
        if (fam_work && lane == 0) fam_work[(long long)d * per_dir + r] = vis.local;
        if (fam_rec && lane == 0) fam_rec[(long long)d * per_dir + r] = vis.local + vis.ctrl;
    }
}

// Path records of every family f (direction f / N^2, root line f % N^2) at
// m.oct_rec + m.oct_rec_off[f], by the traversal the march uses; families
// taken in decreasing order of work (m.oct_order) when it is known.  A
// family whose record count differs from its slot raises error flag 4.
__global__ void __launch_bounds__(kOctWarpsPerBlock * 32) record_octree_kernel(DevModel m, unsigned *counter)
{
    __shared__ OctFrame frames[kOctWarpsPerBlock][kOctMaxDepth];
    __shared__ int paths[kOctWarpsPerBlock][kOctMaxDepth + 1];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kOctWarpsPerBlock + wid;
    int4 *kids = m.oct_kids + (size_t)gw * kOctMaxDepth * kOctMaxKids;
    const long long per_dir = (long long)m.N * m.N;
    const MarchArgs a = oct_geo_args();
    long long nw = 0;
    OctGeo g = oct_geo(m);
    const long long total = per_dir * m.n_dir;
    while (true) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((long long)it >= total) break;
        const long long f = m.oct_order ? (long long)m.oct_order[it] : (long long)it;
        const int d = (int)(f / per_dir);
        const long long r = f - (long long)d * per_dir;
        g.D = m.dirs[d];
        OctRecVisitor vis;
        const long long r0 = m.oct_rec_off[f];
        vis.rec = m.oct_rec + r0;
        vis.cap = m.oct_rec_off[f + 1] - r0;
        vis.n = 0;
        vis.buf = 0ull;
        oct_traverse<1, kAccPlain>(m, a, g, (int)(r / m.N), (int)(r % m.N), nullptr, nullptr, kids, frames[wid],
                        paths[wid], lane, vis, nw);
        if (vis.n & 31) vis.flush(lane);
        if (vis.n != vis.cap && lane == 0) atomicExch(m.oct_err, 4);
    }
}

// ----------------------------------------------------------------------------
// Recording in one traversal.  The families' record counts are not known
// before the walk, so each warp appends its family's records to chunks of
// kPoolChunk records taken from a pool (one atomic per chunk, next[c] links
// a family's chunks); the walk also yields the families' work and record
// counts.  The host then lays the records out contiguously
// (compact_octree_kernel).  A pool too small for the model raises flag 5
// (the counts stay exact; the caller records again with the two-pass
// scheme).
// ----------------------------------------------------------------------------
constexpr int kPoolChunk = (int)kOctPoolChunk;   // a multiple of 32

struct OctPoolVisitor {
    static constexpr bool kNeedI = false;
    unsigned long long *pool;
    int *next;
    unsigned *chunks;           // chunks handed out so far
    long long cap;              // chunks in the pool
    int *err;
    long long n;                // records of the family so far
    unsigned steps;             // active steps of the family
    long long chunk;            // current chunk (-1: none, the pool ran out)
    long long head;             // first chunk of the family
    unsigned long long buf;     // lane k: record k of the current block of 32
    __device__ void flush(int lane)
    {
        const long long b = (n - 1) & ~31ll;            // first record of the block
        if (chunk >= 0 && b + lane < n)
            pool[(size_t)chunk * kPoolChunk + (size_t)(b & (kPoolChunk - 1)) + lane] = buf;
    }
    __device__ void put(int lane, unsigned long long w)
    {
        if ((n & (kPoolChunk - 1)) == 0) {
            unsigned c = 0;
            if (lane == 0) c = atomicAdd(chunks, 1u);
            c = __shfl_sync(kFull, c, 0);
            long long nc = (long long)c < cap ? (long long)c : -1;
            if (nc < 0 && lane == 0) atomicExch(err, 5);
            if (n == 0) head = nc;
            else if (chunk >= 0 && lane == 0) next[chunk] = (int)nc;
            if (chunk < 0 && n > 0) nc = -1;            // a broken chain stays broken
            chunk = nc;
        }
        if (lane == (int)(n & 31)) buf = w;
        n++;
        if ((n & 31) == 0) flush(lane);
    }
    __device__ void step(int lane, const OctLine &, long long dz, int leaf, int Lc)
    {
        steps++;
        put(lane, rec_step(leaf, dz, Lc));
    }
    __device__ void save(int lane, int depth) { put(lane, rec_ctrl(kRecSave, depth)); }
    __device__ void load(int lane, int depth) { put(lane, rec_ctrl(kRecLoad, depth)); }
};

// walk_order (or null): the families in the order to walk them (the
// host's estimate of decreasing work, so that the longest walks start first)
__global__ void __launch_bounds__(kOctWarpsPerBlock * 32) pool_octree_kernel(DevModel m, unsigned *counter,
                                                                              OctPoolVisitor v0,
                                                                              unsigned *fam_work,
                                                                              unsigned *fam_rec, int *fam_head,
                                                                              const int *walk_order)
{
    __shared__ OctFrame frames[kOctWarpsPerBlock][kOctMaxDepth];
    __shared__ int paths[kOctWarpsPerBlock][kOctMaxDepth + 1];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kOctWarpsPerBlock + wid;
    int4 *kids = m.oct_kids + (size_t)gw * kOctMaxDepth * kOctMaxKids;
    const long long per_dir = (long long)m.N * m.N;
    const MarchArgs a = oct_geo_args();
    long long nw = 0;
    OctGeo g = oct_geo(m);
    const long long total = per_dir * m.n_dir;
    while (true) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((long long)it >= total) break;
        const long long f = walk_order ? (long long)walk_order[it] : (long long)it;
        const int d = (int)(f / per_dir);
        const long long r = f - (long long)d * per_dir;
        g.D = m.dirs[d];
        OctPoolVisitor vis = v0;
        vis.n = 0;
        vis.steps = 0;
        vis.chunk = -1;
        vis.head = -1;
        vis.buf = 0ull;
        oct_traverse<1, kAccPlain>(m, a, g, (int)(r / m.N), (int)(r % m.N), nullptr, nullptr, kids, frames[wid],
                        paths[wid], lane, vis, nw);
        if (vis.n & 31) vis.flush(lane);
        if (lane == 0) {
            fam_work[f] = vis.steps;
            fam_rec[f] = (unsigned)vis.n;
            fam_head[f] = (int)vis.head;
        }
    }
}

// Copies family f's records from its pool chunks to m.oct_rec +
// m.oct_rec_off[f] (one warp per family, coalesced loads and stores).
__global__ void compact_octree_kernel(DevModel m, const unsigned long long *pool, const int *next,
                                      const int *fam_head, long long fams)
{
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long f = w0; f < fams; f += nwarps) {
        const long long r0 = m.oct_rec_off[f], n = m.oct_rec_off[f + 1] - r0;
        int c = fam_head[f];
        for (long long k = 0; k < n && c >= 0; k += kPoolChunk) {
            const unsigned long long *src = pool + (size_t)c * kPoolChunk;
            const long long len = min((long long)kPoolChunk, n - k);
            for (long long q = lane; q < len; q += 32) m.oct_rec[r0 + k + q] = src[q];
            if (k + kPoolChunk < n) c = next[c];
        }
    }
}

// ----------------------------------------------------------------------------
// Replay of the recorded paths: the march without the traversal.  A warp
// takes (family, line group) items in decreasing order of work, streams the
// family's records (32 per coalesced load, broadcast by shuffle) and applies
// each step with march_step; save / load records copy the intensities to or
// from the warp's snapshot frames exactly where the traversal does, so every
// step sees the intensities the walking march gives it.  The next step's
// cell data is loaded while the current step computes.
// ----------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ void replay_load(const DevModel &m, const MarchArgs &a, const Dir3D &D,
                                            float wscale, unsigned long long x, Step<G> &st, int lane)
{
    const int leaf = (int)(unsigned)(x & 0xffffffffull);
    const long long dz = (long long)((x >> 32) & 0x1ffffffull);
    const int Lc = (int)((x >> 57) & 0xfull);
    st.cell = leaf;
    const float4 cv = m.vel[leaf];
    st.vlos = cv.x * D.d[0] + cv.y * D.d[1] + cv.z * D.d[2];
    st.inv = cv.w;
    st.s = (float)(int)dz * D.unit;
    st.w = oct_weight(dz, Lc, wscale);
    load_lines<G>(m, a, st, lane);
}

template <int G, int ACC>
__device__ long long replay_family(const DevModel &m, const MarchArgs &a, const Dir3D &D, long long r0,
                                   long long r1, float *I, float *snap, int lane)
{
    const unsigned long long *rec = m.oct_rec;
    const int snap_n = a.per * m.n_ch;
    const float wscale = 1.0f / (float)m.n_dir;
    long long nw = 0;
    long long b0 = r0;                                   // first record of the current block
    unsigned long long rb = (b0 + lane < r1) ? rec[b0 + lane] : 0ull;
    unsigned long long rn = (b0 + 32 + lane < r1) ? rec[b0 + 32 + lane] : 0ull;
    Step<G> cur, nxt;
    MarchState pend = march_state();
    bool pre = false;                                    // cur holds the data of record q
    for (long long q = r0; q < r1; q++) {
        if (q - b0 == 32) {
            b0 += 32;
            rb = rn;
            rn = (b0 + 32 + lane < r1) ? rec[b0 + 32 + lane] : 0ull;
        }
        const int r = (int)(q - b0);
        const unsigned long long x = __shfl_sync(kFull, rb, r);
        const unsigned long long y1 = __shfl_sync(kFull, rb, (r + 1) & 31);
        const unsigned long long y2 = __shfl_sync(kFull, rn, 0);
        const unsigned long long y = (r < 31) ? y1 : y2;
        const unsigned type = (unsigned)(x >> 61);
        if (type == kRecStep) {
            if (!pre) replay_load<G>(m, a, D, wscale, x, cur, lane);
            const bool nstep = (q + 1 < r1) && ((unsigned)(y >> 61) == kRecStep);
            if (nstep) replay_load<G>(m, a, D, wscale, y, nxt, lane);
            nw += (long long)march_step<G, ACC>(m, a, I, cur, lane, pend) * a.n_lines;
            __syncwarp();
            if (nstep) cur = nxt;
            pre = nstep;
        } else {
            const int depth = (int)(unsigned)(x & 0xffffffffull);
            float *sn = snap + (size_t)depth * snap_n;
            if (type == kRecSave) {
                for (int k = lane; k < snap_n; k += 32) sn[k] = I[k];
            } else {
                for (int k = lane; k < snap_n; k += 32) I[k] = sn[k];
            }
            __syncwarp();
            pre = false;
        }
    }
    march_state_end<ACC>(m, a, pend, lane);
    return nw;
}

// registers capped so that 5 blocks (20 warps) fit per SM, 4 for the
// largest line groups
template <int G, int ACC>
__global__ void __launch_bounds__(kOctWarpsPerBlock * 32, G <= 11 ? 5 : 4) replay_octree_kernel(DevModel m, MarchArgs a0,
                                                                                unsigned *counter)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * kOctWarpsPerBlock + wid;
    float *I = smem + (size_t)wid * a0.per * m.n_ch;
    float *snap = m.oct_scratch + (size_t)gw * kOctMaxDepth * a0.per * m.n_ch;
    const long long per_dir = (long long)m.N * m.N;
    const long long total = per_dir * m.n_dir * a0.n_groups;
    long long nw = 0;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((long long)it >= total) break;
        const long long fam = (long long)it / a0.n_groups;     // most work first
        const long long item = m.oct_order ? (long long)m.oct_order[fam] : fam;
        const int dir = (int)(item / per_dir);
        if (dir < a0.dir0 || dir >= a0.dir1) continue;          // another rank's direction
        const MarchArgs a = warp_args(m, a0, (int)((long long)it - fam * a0.n_groups));
        const Dir3D D = m.dirs[dir];
        init_ray<G>(m, a, I, lane);
        nw += replay_family<G, ACC>(m, a, D, m.oct_rec_off[item], m.oct_rec_off[item + 1], I, snap, lane);
    }
    if (a0.count && lane == 0) atomicAdd(m.upd_count, (unsigned long long)nw);   // nw counts lines
}

// ----------------------------------------------------------------------------
// 3D map of an octree: one warp per pixel = lattice line (lam, i, j) of
// direction dir, walked once through the periodic model across every leaf it
// meets (a line of sight: the activation rules of the ray simulation do not
// apply), with the step boundaries of the march and the cached descent; all
// channels in registers, no accumulation.
// ----------------------------------------------------------------------------
template <int CMAX>
__global__ void __launch_bounds__(kOctWarpsPerBlock * 32) map_octree_kernel(DevModel m, int t, int dir, int lam,
                                                                             float *Tout)
{
    __shared__ int paths[kOctWarpsPerBlock][kOctMaxDepth + 1];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long Mp = (long long)m.N << lam;
    const long long pix = (long long)blockIdx.x * kOctWarpsPerBlock + wid;
    if (pix >= Mp * Mp) return;
    const long long H0 = 1ll << kFixedBits;
    OctGeo g;
    g.D = m.dirs[dir];
    g.N = m.N;
    g.Lmax = m.Lmax;
    g.E = (long long)m.N << kFixedBits;
    g.o = (H0 >> m.Lmax) / 2;
    const long long A0 = g.o + (pix / Mp) * (H0 >> lam), B0 = g.o + (pix % Mp) * (H0 >> lam);
    OctPathCache pc;
    pc.p[0] = pc.p[1] = pc.p[2] = 0;
    pc.L = -1;
    const int nchunk = (m.n_ch + 30) / 31;
    const float nb = m.nbg[t];
    const float inv_dv = (float)(1.0 / m.dv), dv = (float)m.dv, vmin = (float)m.v_min;
    float dI[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; c++) dI[c] = 0.f;
    long long z = 0;
    while (z < g.E) {
        const long long Au = A0 + fq(g.D.qa, z), Bu = B0 + fq(g.D.qb, z);
        long long p[3];
        oct_point(g, Au, Bu, z, p);
        int Lc;
        const int cell = oct_locate_cached(m, g, p, Lc, pc, paths[wid], lane);
        const long long HL = H0 >> Lc;
        long long zn = oct_mlo(g, g.D.m, p[g.D.m], Lc) + HL;
        if (g.D.qa > 0) {
            const long long T = Au - wrap_e(Au, g.E) + oct_mlo(g, g.D.a, p[g.D.a], Lc) + HL;
            zn = min(zn, cross_z(T - A0, g.D.qa, g.D.ma));
        }
        if (g.D.qb > 0) {
            const long long T = Bu - wrap_e(Bu, g.E) + oct_mlo(g, g.D.b, p[g.D.b], Lc) + HL;
            zn = min(zn, cross_z(T - B0, g.D.qb, g.D.mb));
        }
        zn = min(zn, g.E);
        const int leaf = __ldg(m.leaf_of + cell);
        const float4 cv = m.vel[leaf];
        const float vlos = cv.x * g.D.d[0] + cv.y * g.D.d[1] + cv.z * g.D.d[2];
        const float2 ks = m.ks[(long long)leaf * m.T + t];
        los_step<CMAX>(dI, nchunk, lane, ks.x * ((float)(int)(zn - z) * g.D.unit), ks.y - nb,
                       (vmin + vlos) * inv_dv, dv * cv.w);
        z = zn;
    }
    los_store<CMAX>(dI, nchunk, m.n_ch, lane, (float)(kH * m.line_nu[t] / kKB), pix, Tout);
}

template <int CMAX>
static loc_status launch_map_oct_c(const DevModel &m, int t, int dir, int lam, float *T_dev, cudaStream_t st)
{
    const long long Mp = (long long)m.N << lam;
    const long long nb = (Mp * Mp + kOctWarpsPerBlock - 1) / kOctWarpsPerBlock;
    map_octree_kernel<CMAX><<<(unsigned)nb, kOctWarpsPerBlock * 32, 0, st>>>(m, t, dir, lam, T_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_map_octree(const DevModel &m, int t, int dir, int lam, float *T_dev, cudaStream_t st)
{
    const int nchunk = (m.n_ch + 30) / 31;
    if (nchunk <= 2) return launch_map_oct_c<2>(m, t, dir, lam, T_dev, st);
    if (nchunk <= 5) return launch_map_oct_c<5>(m, t, dir, lam, T_dev, st);
    if (nchunk <= 9) return launch_map_oct_c<9>(m, t, dir, lam, T_dev, st);
    if (nchunk <= 17) return launch_map_oct_c<17>(m, t, dir, lam, T_dev, st);
    return launch_map_oct_c<34>(m, t, dir, lam, T_dev, st);
}

static int octree_sms()
{
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        nsm = 152;
    }
    return nsm;
}

// warps of the walking kernels, and the most warps any octree march launches
// (the per-warp snapshot scratch is sized for it)
int octree_persistent_warps(const DevModel &m)
{
    (void)m;
    return octree_sms() * kOctBlocksPerSM * kOctWarpsPerBlock;
}

int octree_max_warps(const DevModel &m)
{
    (void)m;
    return octree_sms() * kOctMaxBlocksPerSM * kOctWarpsPerBlock;
}

// persistent blocks per SM of a march kernel: what the occupancy calculator
// allows (registers, shared memory), at least kOctBlocksPerSM
template <class K>
static int oct_blocks_per_sm(K kernel, size_t smem)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kOctWarpsPerBlock * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        nb = 0;
    }
    return std::max(kOctBlocksPerSM, std::min(nb, kOctMaxBlocksPerSM));
}

struct LaunchOctree {
    const DevModel &m;
    const MarchArgs &a;
    unsigned *counter;
    cudaStream_t st;
    template <int G, int ACC>
    loc_status go() const
    {
        const size_t smem = (size_t)kOctWarpsPerBlock * a.per * m.n_ch * sizeof(float);
        if (m.oct_rec) {
            auto k = replay_octree_kernel<G, ACC>;
            LOC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int blocks = octree_sms() * oct_blocks_per_sm(k, smem);
            k<<<blocks, kOctWarpsPerBlock * 32, smem, st>>>(m, a, counter);
        } else {
            auto k = march_octree_kernel<G, ACC>;
            LOC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            const int blocks = octree_persistent_warps(m) / kOctWarpsPerBlock;
            k<<<blocks, kOctWarpsPerBlock * 32, smem, st>>>(m, a, counter);
        }
        LOC_CUDA_TRY(cudaGetLastError());
        return LOC_OK;
    }
};

// counter: one unsigned of device scratch right after the error flag
loc_status launch_march_octree(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    unsigned *counter = (unsigned *)(m.oct_err + 1);
    LOC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    return march_dispatch(a, LaunchOctree{m, a, counter, st});
}

loc_status launch_trace_octree(const DevModel &m, int dir, long long *out, long long cap,
                               unsigned long long *count, cudaStream_t st, unsigned long long *sums,
                               unsigned *fam_work, unsigned *fam_rec)
{
    unsigned *counter = (unsigned *)(m.oct_err + 1);
    LOC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    if (count) LOC_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), st));
    OctTraceVisitor vis;
    vis.out = out;
    vis.cap = cap;
    vis.count = count;
    vis.sums = sums;
    vis.dir = dir;
    vis.local = 0;
    vis.ctrl = 0;
    const int blocks = octree_persistent_warps(m) / kOctWarpsPerBlock;
    trace_octree_kernel<<<blocks, kOctWarpsPerBlock * 32, 0, st>>>(m, dir, vis, counter, fam_work, fam_rec);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_pool_octree(const DevModel &m, unsigned long long *pool, int *next, long long cap_chunks,
                              unsigned *chunk_ctr, unsigned *fam_work, unsigned *fam_rec, int *fam_head,
                              const int *walk_order, cudaStream_t st)
{
    unsigned *counter = (unsigned *)(m.oct_err + 1);
    LOC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    LOC_CUDA_TRY(cudaMemsetAsync(chunk_ctr, 0, sizeof(unsigned), st));
    OctPoolVisitor v;
    memset(&v, 0, sizeof(v));
    v.pool = pool;
    v.next = next;
    v.chunks = chunk_ctr;
    v.cap = cap_chunks;
    v.err = m.oct_err;
    const int blocks = octree_persistent_warps(m) / kOctWarpsPerBlock;
    pool_octree_kernel<<<blocks, kOctWarpsPerBlock * 32, 0, st>>>(m, counter, v, fam_work, fam_rec, fam_head,
                                                                   walk_order);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_compact_octree(const DevModel &m, const unsigned long long *pool, const int *next,
                                 const int *fam_head, long long fams, cudaStream_t st)
{
    const long long blocks = std::min<long long>((fams + 7) / 8, (long long)octree_sms() * 16);
    compact_octree_kernel<<<(unsigned)std::max(1ll, blocks), 256, 0, st>>>(m, pool, next, fam_head, fams);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_record_octree(const DevModel &m, cudaStream_t st)
{
    unsigned *counter = (unsigned *)(m.oct_err + 1);
    LOC_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
    const int blocks = octree_persistent_warps(m) / kOctWarpsPerBlock;
    record_octree_kernel<<<blocks, kOctWarpsPerBlock * 32, 0, st>>>(m, counter);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

}  // namespace loc
