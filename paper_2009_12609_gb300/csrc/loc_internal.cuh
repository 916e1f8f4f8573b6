// loc_internal.cuh -- device-side data layout and shared helpers of the
// GB300 LOC library.  Everything here is internal to the shared library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/loc.h"

namespace loc {

// CGS constants (CODATA 2018 exact SI values).
constexpr double kH = 6.62607015e-27;
constexpr double kKB = 1.380649e-16;
constexpr double kC = 2.99792458e10;
constexpr double kAMU = 1.66053906660e-24;
constexpr double kPI = 3.14159265358979323846;

// One root cell is 2^kFixedBits integer units in the 3D ray geometry.
constexpr int kFixedBits = 24;
constexpr int kMaxLevels = 32;      // molecule levels supported by the SE
constexpr int kMaxLines = 64;       // radiative lines
constexpr int kMaxChannels = 1024;
constexpr int kMaxLinesPerWarp = 15;

// One step of a 1D ray through one shell, precomputed at model creation:
// cell index, path length s (cm), line-of-sight velocity at the step's
// start (cm/s) and the step's weight w = A_j s / W_c.
struct Seg1D {
    int cell;
    float s;
    float vlos;
    float w;
};

// Per-direction integer description of the 3D ray lattice.
struct Dir3D {
    int m, a, b;            // main / transverse axes
    int flip[3];            // mirrored axes
    long long qa, qb;       // slopes in units of 2^-F
    long long Da, ra, Db, rb;       // H 2^F = D q + r (crossing increments)
    long long Qa0, Ra0, Qb0, Rb0;   // first target (H/2) 2^F = Q q + R
    unsigned long long ma, mb;      // floor((2^64 - 1) / q): division by q
    float d[3];             // true unit direction (for v . d)
    float unit;             // cm per fixed-point unit along the ray
};

// Device view of one model.  All pointers are device memory.
struct DevModel {
    int geometry;
    long long n_cells;
    int n_ch;
    double v_min, dv;
    float vmin_f, dv_f;                 // the channel grid in FP32 (the march uses no FP64)
    double t_bg;

    // static per-cell data
    double *n_h2, *t_kin, *abundance;   // FP64: line parameters and SE
    float *inv_s2sig;                   // 1 / (sqrt(2) sigma) per cell
    float4 *vel;                        // 3D: {vx, vy, vz, inv_s2sig}

    // 1D geometry
    int K, n_rays;
    double ray_power;                   // impact parameters R ((j + 1/2) / n_rays)^ray_power (<= 0: 1)
    int trunc;                          // per-cell line truncation on (lines marked off by line_params)
    long long n_segs;
    double *radius;                     // [K]
    float *v1d;                         // [K] radial velocity
    int *ray_off;                       // [n_rays + 1]
    Seg1D *segs;                        // [n_segs]

    // 3D geometry
    int N, n_dir;
    double h0;
    Dir3D *dirs;                        // [n_dir]

    // octree (cells level ordered; data arrays above are per leaf)
    int Lmax;                           // refinement levels below the root
    long long n_tree;                   // cells of all levels
    int *child;                         // [n_tree] first child or -1
    int *leaf_of;                       // [n_tree] leaf index or -1
    float *oct_scratch;                 // per persistent warp: frame snapshots
    int4 *oct_kids;                     // per persistent warp: child lines
    int *oct_err;                       // device flag: frame capacity exceeded
    int *oct_order;                     // root-ray families, most work first (or null)
    int *leaf_perm;                     // octree: [n_cells] level-ordered index of each leaf (the
                                        // leaves are stored depth first; null for other geometries)
    unsigned long long *oct_rec;        // recorded paths of all families (or null: walk)
    long long *oct_rec_off;             // [families + 1] first record of each family

    // molecule
    int L, T, P;
    double mass_amu;
    double *energy_K, *g;               // [L]
    int *line_u, *line_l;               // [T]
    double *line_A, *line_nu;           // [T]
    int *coll_u, *coll_l;               // [P]
    double *coll_k;                     // [P]
    double2 *coll_rates;                // [n_cells][P] {C_ul, C_lu}, or null: computed in the solve
    int *hf_off;                        // [T + 1] hyperfine components of each line (or null: none)
    float *hf_o, *hf_w;                 // component offsets (channels, v / dv) and strengths
    float hf_olo, hf_ohi;               // smallest (<= 0) and largest (>= 0) offset, channels
    float *nbg;                         // [T] background occupation
    double *nbg64;                      // [T]

    // iteration state
    double *x;                          // [n_cells][L] populations
    double *x_new;                      // [n_cells][L]
    float2 *ks;                         // [n_cells][T] {K (per unit phi and length), S}
    float2 *acc;                        // [n_cells][T] {SIJ, ESC}
    float *norm;                        // [n_cells]
    float2 *acc_c;                      // [n_cells][T] rounding errors of acc's additions (or null)
    float *norm_c;                      // [n_cells] rounding errors of norm's additions (or null)
    double *acc64;                      // [n_cells][T][2] (FP64 accumulation)
    double *norm64;                     // [n_cells]
    unsigned int *dtex_bits;            // device scalar: max rel dTex (float bits)
    unsigned long long *maser_count;    // device scalar
    unsigned long long *upd_count;      // device scalar: computed updates (profiling)
    unsigned long long *nom_count;      // device scalar: nominal updates (profiling)
};

// Parameters of one march launch.
struct MarchArgs {
    int per;            // lines per warp (line group size)
    int n_groups;       // line groups: a work item is (ray, group)
    int line0;          // first line of the warp's group (set per warp)
    int n_lines;        // lines in the warp's group (set per warp)
    float window;       // window half-width in sigma (0 = all channels)
    float inv_dv;       // 1 / channel width (s/cm)
    int fp64_acc;       // accumulate in FP64
    int comp;           // FP32 accumulation compensated (acc_c, norm_c collect the rounding errors)
    int do_norm;        // the warp also accumulates NORM (group 0)
    int count;          // count computed channel updates into upd_count
    // 1D rays cut into runs of `chunk` consecutive steps (0: whole rays);
    // see march1d_affine_kernel
    int chunk;
    long long n_chunks;     // runs over all rays
    const int *chunk_off;   // [n_rays + 1] first run of each ray
    const int *chunk_ray;   // [n_chunks] ray of each run
    float2 *ab;             // [n_chunks][T][n_ch] run maps {alpha, beta}, then {I_in, -}
    int2 *run_rng;          // [n_chunks] channels [lo, hi) the run's step windows touch
    int tile;               // channels per shared-memory tile of the run maps (>= every run's union)
    int dir0, dir1;         // 3D: the march covers directions [dir0, dir1) of the model's table
    // 1D sub-iterations of the sub_k innermost shells: the rays j < n_rays
    // reach them, and the intensity a ray carries into them (at step
    // K - sub_k of its list) is kept in sub_I[j][line][channel]
    int sub_k;              // 0: none
    int sub_mode;           // 0: full march, storing sub_I; 1: march the region's steps from sub_I
    float *sub_I;
};

// ----------------------------------------------------------------------------
// Per-cell accumulators as the solve reads them: the FP32 sums plus the
// rounding errors of their additions (compensated accumulation), or the FP64
// sums of the FP64-accumulation mode.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double2 acc_value(const DevModel &m, long long o, int fp64_acc)
{
    if (fp64_acc) return make_double2(m.acc64[2 * o], m.acc64[2 * o + 1]);
    const float2 a = m.acc[o];
    if (!m.acc_c) return make_double2(a.x, a.y);
    const float2 e = m.acc_c[o];
    return make_double2((double)a.x + (double)e.x, (double)a.y + (double)e.y);
}

__device__ __forceinline__ double norm_value(const DevModel &m, long long c, int fp64_acc)
{
    if (fp64_acc) return m.norm64[c];
    const double n = m.norm[c];
    return m.norm_c ? n + (double)m.norm_c[c] : n;
}

// clears the accumulators of entry o = c T + t (and NORM of cell c if first)
__device__ __forceinline__ void acc_zero(const DevModel &m, long long o, long long c, int fp64_acc, bool first)
{
    if (fp64_acc) {
        m.acc64[2 * o] = 0.0;
        m.acc64[2 * o + 1] = 0.0;
        if (first) m.norm64[c] = 0.0;
    } else {
        m.acc[o] = make_float2(0.f, 0.f);
        if (m.acc_c) m.acc_c[o] = make_float2(0.f, 0.f);
        if (first) {
            m.norm[c] = 0.f;
            if (m.norm_c) m.norm_c[c] = 0.f;
        }
    }
}

// ----------------------------------------------------------------------------
// host-side helpers (implemented in loc_api.cu)
// ----------------------------------------------------------------------------
void set_error(const char *fmt, ...);
#define LOC_CUDA_TRY(call)                                                        \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            ::loc::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), \
                             __FILE__, __LINE__);                                 \
            return LOC_ECUDA;                                                     \
        }                                                                         \
    } while (0)

// true when no two of the n level pairs (u[i], l[i]) join the same two
// levels (in either order); levels in [0, L), L <= kMaxLevels
inline bool distinct_level_pairs(const int32_t *u, const int32_t *l, int n, int L)
{
    bool seen[kMaxLevels * kMaxLevels] = {};
    for (int i = 0; i < n; i++) {
        const int a = u[i] < l[i] ? u[i] : l[i], b = u[i] < l[i] ? l[i] : u[i];
        if (a < 0 || b >= L) return false;
        if (seen[a * kMaxLevels + b]) return false;
        seen[a * kMaxLevels + b] = true;
    }
    return true;
}

// kernel launchers (one per translation unit)
loc_status launch_geom1d(const DevModel &m, cudaStream_t st);
loc_status launch_geom1d_scratch(const DevModel &m, cudaStream_t st, int *tan, double *W);
loc_status launch_line_params(const DevModel &m, cudaStream_t st, int zero_acc = 0, double cutoff = 0.0);
loc_status launch_march(const DevModel &m, const MarchArgs &a, cudaStream_t st);
loc_status launch_march1d(const DevModel &m, const MarchArgs &a, cudaStream_t st);
loc_status launch_march1d_chunked(const DevModel &m, const MarchArgs &a, cudaStream_t st);
loc_status launch_march1d_ranges(const DevModel &m, const MarchArgs &a, int *max_w_dev, cudaStream_t st);
loc_status launch_march3d(const DevModel &m, const MarchArgs &a, cudaStream_t st);
// want_dtex = 0: skip the convergence metric (nothing reads it this iteration)
// next = 1: the solve also computes the next iteration's line parameters
// from the new populations (with cutoff) and clears its accumulators
loc_status launch_se(const DevModel &m, int ali, int fp64_acc, cudaStream_t st, int want_dtex = 1,
                     int next = 0, double cutoff = 0.0);
loc_status launch_lte(const DevModel &m, cudaStream_t st);
loc_status launch_coll_rates(const DevModel &m, double2 *out, cudaStream_t st);
loc_status launch_bg(const DevModel &m, cudaStream_t st);
loc_status launch_tex(const DevModel &m, int t, double *out_dev, cudaStream_t st);
loc_status launch_dtex(const DevModel &m, const double *x0, cudaStream_t st);
// rows of w doubles between the internal leaf order and the level order:
// to_api = 1: dst[perm[i]] = src[i]; 0: dst[i] = src[perm[i]]
loc_status launch_permute_rows(const int *perm, long long n, int w, const double *src, double *dst,
                               int to_api, cudaStream_t st);
loc_status launch_spectra1d(const DevModel &m, int t, const double *p_dev, int n_p, float4 *rec,
                            int *nsteps, float *T_dev, cudaStream_t st);
loc_status launch_trace3d(const DevModel &m, int dir, long long i, long long j,
                          long long *cells, long long *dz, long long cap,
                          long long *n_out, cudaStream_t st);
loc_status launch_count3d(const DevModel &m, unsigned long long *total_dev, cudaStream_t st);
loc_status launch_dir_setup(const double *dirs_dev, int n_dir, double h0, Dir3D *out,
                            cudaStream_t st);
loc_status launch_cell_setup(const DevModel &m, const double *sigma_turb, const double *vx,
                             const double *vy, const double *vz, cudaStream_t st);
loc_status launch_march_octree(const DevModel &m, const MarchArgs &a, cudaStream_t st);
loc_status launch_trace_octree(const DevModel &m, int dir, long long *out, long long cap,
                               unsigned long long *count, cudaStream_t st,
                               unsigned long long *sums = nullptr, unsigned *fam_work = nullptr,
                               unsigned *fam_rec = nullptr);
loc_status launch_record_octree(const DevModel &m, cudaStream_t st);
// one traversal into a chunk pool (records, work and record counts per
// family; flag 5 when the pool ran out), then the contiguous layout
constexpr long long kOctPoolChunk = 256;
loc_status launch_pool_octree(const DevModel &m, unsigned long long *pool, int *next, long long cap_chunks,
                              unsigned *chunk_ctr, unsigned *fam_work, unsigned *fam_rec, int *fam_head,
                              const int *walk_order, cudaStream_t st);
loc_status launch_compact_octree(const DevModel &m, const unsigned long long *pool, const int *next,
                                 const int *fam_head, long long fams, cudaStream_t st);
int octree_persistent_warps(const DevModel &m);
int octree_max_warps(const DevModel &m);
loc_status launch_map_grid3d(const DevModel &m, int t, int dir, float *T_dev, cudaStream_t st);
loc_status launch_map_octree(const DevModel &m, int t, int dir, int lam, float *T_dev, cudaStream_t st);
constexpr int kOctMaxKids = 96;         // child lines one frame can hold
loc_status launch_acc_to_f64(const DevModel &m, int fp64_acc, double *sij, double *esc,
                             double *norm, cudaStream_t st);

}  // namespace loc
