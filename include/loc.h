/*
 * loc.h -- C ABI of the GB300 LOC line radiative-transfer library.
 *
 * The library runs the hot path of the accelerated lambda iteration (ALI)
 * of Juvela's LOC (arXiv:2009.12609): for every ray and velocity channel a
 * ray march across 1D shells or 3D cells evaluates the Doppler-shifted
 * Gaussian profile, applies the formal solution I <- I e^-tau + S (1 - e^-tau)
 * and accumulates each cell's absorbed-photon sum (SIJ) and escape term
 * (ESC, the diagonal lambda operator), followed by a per-cell statistical-
 * equilibrium solve (Sect. 2 of the paper, Eq. 1-3).  All steps run as
 * CUDA kernels on one GPU (sm_103a); there is no CPU fallback.
 *
 * Conventions
 *  - Every function returns a loc_status; LOC_OK is 0, errors are negative.
 *    loc_last_error() returns a thread-local message describing the last
 *    error (valid until the next call on the same thread).
 *  - All array arguments are HOST pointers unless stated otherwise.  The
 *    library copies what it needs; the caller keeps ownership.  Outputs are
 *    caller-allocated host buffers whose capacity n_out is checked first:
 *    too small -> LOC_EINVAL and nothing is written.
 *  - Units are CGS: cm, cm/s, cm^-3, K, Hz, s^-1, cm^3 s^-1.
 *  - Handles are not thread-safe; use one handle per thread.
 *  - Device memory comes from the allocator in loc_model_desc (or
 *    cudaMalloc when it is NULL); work is queued on the given stream.
 *  - No C++ exception crosses this interface.
 */
#ifndef LOC_H
#define LOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int loc_status;
#define LOC_OK        0
#define LOC_EINVAL   -1   /* bad argument (size, range, NULL, layout)      */
#define LOC_ENOMEM   -2   /* device or host allocation failed              */
#define LOC_ECUDA    -3   /* a CUDA call failed (message has the details)  */
#define LOC_ETIMEOUT -4   /* a bounded wait gave up                        */
#define LOC_ENOTCONV -5   /* tolerance not reached within max_iter         */
#define LOC_ESTATE   -6   /* call out of order (e.g. no molecule yet)      */
#define LOC_EBUSY    -7   /* server has no free slot / memory              */

/* Geometry kinds (Sect. 2.1 and 2.2). */
#define LOC_SHELLS_1D 1
#define LOC_GRID_3D   2
#define LOC_OCTREE_3D 3

/* Accumulation precision of the ray march (Eq. 2: the per-cell sums of
 * absorbed photons and escape terms over all ray steps). */
#define LOC_FP32_MARCH 0  /* FP32 march; FP32 per-cell accumulators whose
                             additions are compensated: the exact rounding
                             error of every atomic addition (TwoSum on the
                             value it found) goes to a second FP32 word, and
                             the solve reads the sum of both (the default) */
#define LOC_FP64_ACC   1  /* FP32 march, FP64 per-cell accumulators         */
#define LOC_FP32_PLAIN 2  /* FP32 march, plain FP32 accumulators (no
                             compensation; for error comparisons)           */

/* Optional device allocator; alloc returns NULL on failure. */
typedef struct loc_allocator {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} loc_allocator;

/*
 * Model description (Sect. 2.1 for shells, Sect. 2.2 for 3D grids).
 *  geometry     LOC_SHELLS_1D, LOC_GRID_3D or LOC_OCTREE_3D (see octree_*);
 *               for octrees the model's cells (populations, radiation,
 *               T_ex) are the leaves, in level-ordered cell order.
 *  n_shells     1D: number of concentric shells K >= 1.
 *  radius       1D: [K] outer radii, strictly increasing, > 0.
 *  n_rays       1D: number of impact parameters (0 -> n_shells); ray j
 *               passes at p_j = R ((j + 1/2) / n_rays)^ray_power and stands
 *               for the annulus between R (j / n_rays)^ray_power and
 *               R ((j + 1) / n_rays)^ray_power (Sect. 2.1).
 *  n_root, h0   3D: N^3 root cells of size h0 (cm), 1 <= N <= 255; cells
 *               are indexed x fastest: idx = (iz N + iy) N + ix.
 *  n_dir, dirs  3D: [n_dir][3] unit ray directions (e.g. HEALPix centres).
 *  octree_levels, octree_refine, octree_n_cells
 *               octree (1 <= n_root <= 255, levels <= 10): number of
 *               levels below the root, and per cell a
 *               refine flag (0 = leaf, 1 = split into 8 children) in level
 *               order: level-0 cells in raster order, then the children of
 *               every refined level-L cell, in the order of their parents,
 *               each as the 8 octants (cx + 2 cy + 4 cz).  Per-cell field
 *               arrays then follow this same order (values of refined
 *               cells are ignored).
 *  n_h2, t_kin, sigma_turb, abundance
 *               per cell: H2 density, kinetic temperature, micro-turbulent
 *               1D dispersion (cm/s), fractional abundance.
 *  v            1D: [K] radial velocity (cm/s, > 0 outwards).
 *  vx, vy, vz   3D: per-cell velocity (cm/s).
 *  n_ch, v_min, dv  velocity channels: channel k covers
 *               [v_min + k dv, v_min + (k+1) dv]; 1 <= n_ch <= 1024.
 *  t_bg         background (CMB) temperature of the entering rays.
 *  stream       cudaStream_t to queue all work on (NULL: legacy default).
 *  allocator    optional device allocator (NULL: cudaMalloc / cudaFree).
 *  ray_power    1D: exponent of the impact-parameter power law; 0 or 1 give
 *               equidistant rays (the default), > 1 concentrates rays towards
 *               the centre (small inner shells), (0, 1) towards the edge;
 *               at most 10.
 *  octree_paths octree: 0 (default) records the paths of all rays once,
 *               at creation (8 bytes per active ray step or intensity copy
 *               of the split / side-ray rules of Sect. 2.2), when they fit
 *               in device memory, and every ray simulation replays them;
 *               1 walks the tree in every ray simulation (no records).  The
 *               results are the same either way: the replay applies the
 *               same steps, in the same order, as the walk.  Recording
 *               takes one traversal into a temporary pool of at most 40 %
 *               of the free device memory, or, when the pool does not fit,
 *               one traversal that counts and one that records; 2 asks for
 *               the latter outright (same records).
 */
typedef struct loc_model_desc {
    int geometry;
    int n_shells;
    const double *radius;
    int n_rays;
    int n_root;
    double h0;
    int n_dir;
    const double *dirs;
    int octree_levels;
    const int32_t *octree_refine;
    int64_t octree_n_cells;
    const double *n_h2, *t_kin, *sigma_turb, *abundance;
    const double *v;
    const double *vx, *vy, *vz;
    int n_ch;
    double v_min, dv;
    double t_bg;
    void *stream;
    const loc_allocator *allocator;
    double ray_power;
    int octree_paths;
} loc_model_desc;

/*
 * Molecule description.  Levels 0..n_levels-1 with energies E/k (K) and
 * statistical weights; radiative lines u -> l with Einstein A and rest
 * frequency; collisional pairs u > l with a constant downward rate
 * coefficient k_ul (partner H2; upward rates follow from detailed balance).
 * 2 <= n_levels <= 32.
 * Hyperfine structure (1D models, Sect. 2.1; NULL hf_n: none): hf_n[t]
 * components of line t (0: the plain profile, at most 16), with velocity
 * offsets hf_v (cm/s) and relative strengths hf_w (>= 0, summing to 1 per
 * line within 1e-6), concatenated in line order.  The components are in
 * LTE with each other: the line is one transition whose channel profile is
 * the strength-weighted sum of the components' profiles, each shifted by
 * its offset.  The channel band should hold every component.
 */
typedef struct loc_molecule_desc {
    int n_levels;
    const double *energy_K;
    const double *g;
    double mass_amu;
    int n_lines;
    const int32_t *line_u, *line_l;
    const double *line_A, *line_nu;
    int n_coll;
    const int32_t *coll_u, *coll_l;
    const double *coll_k;
    const int32_t *hf_n;
    const double *hf_v, *hf_w;
} loc_molecule_desc;

/*
 * Iteration options.
 *  max_iter       number of ALI iterations to run (>= 1).
 *  tol_tex        stop early once max |dT_ex|/|T_ex| < tol_tex (0: run
 *                 exactly max_iter iterations).  The metric covers lines
 *                 whose upper level holds >= 1e-6 of the molecules.
 *  ali            1: accelerated lambda iteration with the diagonal
 *                 operator (Sect. 2); 0: plain lambda iteration.
 *  precision      LOC_FP32_MARCH (default), LOC_FP64_ACC or LOC_FP32_PLAIN.
 *  lines_per_pass 0: automatic (the value chosen by loc_autotune, else all
 *                 lines per warp, or fewer when the launch would leave
 *                 SMs idle); k > 0: each warp carries k lines through the
 *                 rays (the paper's one-line-at-a-time mode is k = 1,
 *                 Sect. 2).  Results do not depend on it beyond rounding.
 *  window_sigmas  0: update every channel; w > 0: skip channels farther
 *                 than w sigma from the local line centre (Sect. A.2).
 *  profile        1: time every kernel with CUDA events on the model's
 *                 stream and count the channel updates actually computed
 *                 (fills the *_ms and computed_updates report fields).
 *  steps_per_chunk  1D models only.  0: automatic (the value chosen by
 *                 loc_autotune, else whole rays when the rays fill the GPU
 *                 and runs of steps otherwise); c > 0: every ray is cut
 *                 into runs of c consecutive steps marched by separate
 *                 warps (each run's intensity map composed first, then the
 *                 runs' entering intensities by a scan along the ray);
 *                 c < 0: whole rays, one warp each.  Results equal the
 *                 whole-ray march up to rounding.  Ignored for 3D models.
 *  level_cutoff   per-cell line truncation in the ALI loop (the paper's
 *                 suggestion to skip, cell by cell, transitions between
 *                 levels that are not populated, Sect. 4): 0 = off; c > 0:
 *                 in a cell where both levels of a line hold less than c of
 *                 the molecules, the line is left out of that iteration's
 *                 ray simulation there (its opacity is taken as zero) and
 *                 the equilibrium solve uses the background intensity with
 *                 beta = 1 for it.  A ray step whose lines of one pass
 *                 (lines_per_pass) are all left out is skipped, so the
 *                 saving grows as lines_per_pass shrinks.  At most 1e-6
 *                 (below the convergence metric's 1e-6 population floor).
 *                 Emergent spectra and maps never truncate.
 *  dir_begin, dir_end  3D models: the ray simulation covers directions
 *                 [dir_begin, dir_end) of the model's table only (both 0:
 *                 all).  The directions of one simulation are independent
 *                 (Sect. 2.2), so N devices can each march a share and sum
 *                 their accumulators (loc_radiation_buffers) before
 *                 loc_solve; loc_iterate with a range solves from that
 *                 share alone.  Ignored for 1D models.
 *  sub_iters, sub_shells  1D models, loc_iterate: after every full ALI
 *                 iteration, sub_iters sub-iterations of the region of the
 *                 sub_shells innermost shells (Sect. 4 suggests updating
 *                 optically thick regions more often): line parameters of
 *                 the region, a ray simulation of the rays that reach it --
 *                 only their steps inside it, from the intensity each ray
 *                 carried into the region in the full iteration -- and the
 *                 equilibrium of the region's cells; the populations outside
 *                 the region are held.  max_iter and tol_tex count full
 *                 iterations; the metric compares the populations before
 *                 and after the whole iteration.  Whole rays are marched
 *                 (steps_per_chunk is ignored); level_cutoff must be 0.
 *                 Afterwards the accumulators hold the last sub-iteration's
 *                 sums of the region.  0: none.
 */
typedef struct loc_iter_opts {
    int max_iter;
    double tol_tex;
    int ali;
    int precision;
    int lines_per_pass;
    double window_sigmas;
    int profile;
    int steps_per_chunk;
    double level_cutoff;
    int dir_begin, dir_end;
    int sub_iters, sub_shells;
} loc_iter_opts;

/* Iteration report. */
typedef struct loc_iter_report {
    int iterations;            /* iterations performed                      */
    double max_rel_dtex;       /* metric of the last iteration              */
    int64_t segments;          /* ray-cell steps per ray simulation         */
    double updates;            /* (step, channel, line) updates, all iters  */
    double kernel_ms;          /* device time of the iterations (events)    */
    int64_t n_maser_cells;     /* (line, cell) pairs with negative opacity  */
    /* filled when opts.profile = 1 (0 otherwise) */
    double march_ms;           /* summed duration of the march launches     */
    double se_ms;              /* summed duration of the equilibrium solves */
    double params_ms;          /* summed duration of the line-parameter step*/
    int64_t march_launches;    /* number of march launches                  */
    double computed_updates;   /* updates inside the channel windows        */
    double nominal_updates;    /* updates of every channel of every line not
                                  left out by level_cutoff in the step's cell */
    /* how the work was done (always filled) */
    int64_t path_records;      /* octree: recorded path records the march
                                  replays (0: it walks the tree)             */
    int coll_table;            /* 1: collision rates read from the model's
                                  table; 0: recomputed in every solve       */
} loc_iter_report;

typedef struct loc_model loc_model;

/* Message of the last failed call on this thread ("" if none). */
const char *loc_last_error(void);

/* Library version string. */
const char *loc_version(void);

/* Build a model on the device (Sect. 2.1 / 2.2): validates and copies the
 * description, precomputes the ray geometry.  *out receives the handle. */
loc_status loc_create_model(loc_model **out, const loc_model_desc *d);

/* Attach the molecule and reset the populations to LTE at T_kin (the
 * iteration's starting point, Sect. 3.3.2).  May be called again. */
loc_status loc_set_molecule(loc_model *m, const loc_molecule_desc *mol);

/* Run ALI iterations (Sect. 2): per iteration, line parameters from the
 * populations, one ray simulation accumulating SIJ / ESC / NORM, and the
 * statistical-equilibrium solve.  r may be NULL.  Returns LOC_ENOTCONV
 * (with the work done) if tol_tex > 0 was not reached in max_iter. */
loc_status loc_iterate(loc_model *m, const loc_iter_opts *o, loc_iter_report *r);

/* Reset the populations to LTE at T_kin (the starting point of the
 * iteration, Sect. 3.3.2) without re-uploading the molecule. */
loc_status loc_reset_populations(loc_model *m);

/* One ray simulation (Sect. 2) with the current populations, without the
 * equilibrium solve: clears and fills the per-cell accumulators read by
 * loc_get_radiation and loc_radiation_buffers.  For 3D models
 * o->dir_begin / dir_end restrict it to that range of the direction table
 * (one device's share; loc_solve then takes the summed accumulators).
 * LOC_ESTATE before loc_set_molecule, LOC_EINVAL for invalid options, the
 * octree flags' LOC_ECUDA if a traversal limit was hit. */
loc_status loc_march(loc_model *m, const loc_iter_opts *o);

/* Choose the launch shape of the march: the number of lines each warp
 * carries (more lines per warp share the profile and the walk, fewer give
 * more warps and fewer registers per thread) and, for 1D models, the run
 * length steps_per_chunk (whole rays or runs of 128 / 64 / 32 / 16 / 8 steps),
 * by timing one ray simulation per candidate with CUDA events on the
 * model's stream; the fastest is used by later calls whose lines_per_pass
 * (steps_per_chunk) is 0.  Runs ray simulations with the current
 * populations and o->level_cutoff (overwrites the accumulators and the line
 * parameters).  best_per, best_chunk (-1:
 * whole rays) and best_ms (each may be NULL) receive the choice and its
 * time. */
loc_status loc_autotune(loc_model *m, const loc_iter_opts *o, int *best_per, int *best_chunk,
                        double *best_ms);

/* Per-cell accumulators of the last ray simulation, as FP64:
 * sij, esc [n_lines][n_cells] and norm [n_cells] (any may be NULL).
 * J_ext = SIJ / NORM and beta = ESC / NORM enter the rate equations. */
loc_status loc_get_radiation(const loc_model *m, double *sij, double *esc,
                             double *norm, size_t n_out_lines_cells,
                             size_t n_out_cells);

/* Device addresses of a model's per-cell accumulators (the sums SIJ, ESC
 * and NORM of Sect. 2 over all ray steps; Sect. 2.2 makes the directions of
 * one simulation independent), valid until the model is destroyed
 * (loc_set_molecule reallocates them).  LOC_EINVAL for NULL arguments,
 * LOC_ESTATE before loc_set_molecule (*out is cleared on success first).
 * All are DEVICE pointers owned by the library, every one allocated by
 * loc_set_molecule whatever the precision:
 *  acc, acc_c     [n_cells][n_lines][2] FP32 {SIJ, ESC} and the
 *                 compensation words of their additions (zero unless the
 *                 precision is LOC_FP32_MARCH);
 *  norm, norm_c   [n_cells] FP32 NORM and its compensation word;
 *  acc64, norm64  the FP64 accumulators of LOC_FP64_ACC, same layout.
 * Every array is a plain sum over ray steps, so the accumulators of several
 * devices that marched disjoint direction ranges of the same model combine
 * by element-wise addition of each array (an all-reduce with sum), after
 * which loc_solve gives every device the populations of the whole ray
 * simulation.  Octree leaves are in the library's storage order (depth
 * first), the same on every device that holds the same model; the other
 * calls of this interface use the level order.  Reading or writing them
 * while the model's stream has work queued races with that work. */
typedef struct loc_radiation_buffers_t {
    int64_t n_cells;
    int n_lines;
    float *acc, *acc_c, *norm, *norm_c;
    double *acc64, *norm64;
} loc_radiation_buffers_t;

loc_status loc_radiation_buffers(loc_model *m, loc_radiation_buffers_t *out);

/* The statistical-equilibrium half of one ALI iteration (Sect. 2): every
 * cell's rate equations from the accumulators as they are now (after
 * loc_march, and after any summation of several devices' accumulators),
 * the new populations in place of the old, and the convergence metric
 * between them in r->max_rel_dtex (r may be NULL).  o->ali, o->precision
 * (which must be the last march's) and o->level_cutoff apply.  LOC_ESTATE
 * if no ray simulation has run. */
loc_status loc_solve(loc_model *m, const loc_iter_opts *o, loc_iter_report *r);

/* Level populations x[cell][level] (fractions summing to 1 per cell). */
loc_status loc_get_populations(const loc_model *m, double *out, size_t n_out);

/* Replace the populations (e.g. resume from a checkpoint); layout as above. */
loc_status loc_set_populations(loc_model *m, const double *in, size_t n);

/* Excitation temperatures of line t for all cells:
 * T_ex = (h nu / k) / ln(g_u x_l / (g_l x_u)); 0 where a population is 0. */
loc_status loc_get_tex(const loc_model *m, int t, double *out, size_t n_out);

/* Emergent spectra of a 1D model (the final line-of-sight integration of
 * Sect. 2): for each impact parameter p_cm[i] the ray is followed through
 * the shells with the current populations; T_out[i][k] is the Rayleigh-
 * Jeans brightness (h nu / k)(n_k - n_bg) of line t in channel k. */
loc_status loc_spectra(const loc_model *m, int t, const double *p_cm, int n_p,
                       double *T_out, size_t n_out);

/* Emergent map of a 3D model (the final line-of-sight integration of
 * Sect. 2, for grids and octrees) seen along direction `dir` of the model's
 * direction table, with the current populations.  One pixel per lattice
 * line (i, j) of level `level` of that direction (0 for grids, 0 ..
 * octree_levels for octrees): M = n_root << level pixels per side, i along
 * the direction's first transverse axis a, j along the second b (the two
 * axes other than the main axis m = argmax |d|, a < b), both counted in the
 * direction of travel (mirrored where the direction component is negative).
 * Each pixel's ray starts with the background at the upstream face, crosses
 * the periodic model once along the main axis through every cell it meets
 * (every octree leaf, whatever its level) and is updated with Eq. 3, no
 * accumulation.  T_out[(i M + j) n_ch + k] is the Rayleigh-Jeans
 * brightness (h nu / k)(n_k - n_bg) of line t in channel k.  At most 2^26
 * pixels per call; n_out >= M^2 n_ch, else LOC_EINVAL. */
loc_status loc_map3d(const loc_model *m, int t, int dir, int level, double *T_out, size_t n_out);

/* Number of cells (shells, grid cells or octree leaves+parents as given). */
loc_status loc_model_info(const loc_model *m, int64_t *n_cells, int *n_levels,
                          int *n_lines, int64_t *segments_per_sim);

/* Segment list of one ray of a 3D model, traced on the device by the same
 * walk the march uses: direction index dir, root line (i, j).  cells[k] is
 * the cell index (x fastest for grids), dz[k] the main-axis length in
 * fixed-point units (one root cell = 2^24).  *n_seg receives the count;
 * LOC_EINVAL if it exceeds cap (nothing written). */
loc_status loc_trace_ray(const loc_model *m, int dir, int64_t i, int64_t j,
                         int64_t *cells, int64_t *dz, int64_t cap,
                         int64_t *n_seg);

/*
 * Radiation field of a 1D model for given line parameters, allocating no
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- a host application whose device
 * memory belongs to another allocator, or a latency-critical loop in which
 * cudaMalloc / cudaFree would synchronise the device.
 *
 * All pointers are DEVICE pointers owned by the caller:
 *  radius     [n_shells] FP64 outer radii (cm), strictly increasing
 *  v_rad      [n_shells] radial velocity (cm/s)
 *  inv_s2sig  [n_shells] 1 / (sqrt(2) sigma) of the line profile (s/cm)
 *  ks         [n_shells][n_lines][2] FP32 {K, S}: opacity per unit profile
 *             fraction and path length, and source function (occupation)
 *  nbg        [n_lines] background occupation number of each line
 *  j_ext, beta  outputs [n_shells][n_lines]: J_ext = SIJ / NORM and
 *             beta = ESC / NORM (background and 1 for a shell no ray crossed)
 * n_rays = 0 means one ray per shell; the channel grid and window are those
 * of loc_iter_opts / loc_model_desc.  Limits: n_shells <= 256, n_rays <= 256,
 * n_lines <= 64, n_ch <= 1024; larger sizes return LOC_EINVAL.
 * Intermediates live in one fixed 2.5 MiB device array that every GPU which
 * loads the library keeps until the process exits.  The first call on a
 * device looks up that array's address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and corrupt each other; serialise them.  The work is
 * queued on `stream` (cudaStream_t, NULL: legacy default) and the function
 * returns without waiting for it.
 */
loc_status loc_radiation1d_noalloc(int n_shells, int n_rays, const double *radius,
                                   const float *v_rad, const float *inv_s2sig, int n_ch,
                                   double v_min, double dv, int n_lines, const float *ks,
                                   const float *nbg, double window_sigmas, float *j_ext,
                                   float *beta, void *stream);

/* ------------------------------------------------------------------------
 * Continuous-batching server for 1D models.
 *
 * Many independent spherical models (the inverse-problem workload of the
 * paper's introduction) are solved to convergence together: a host thread
 * admits submitted models into free slots while the device-memory budget
 * allows, keeps their populations on the device, and runs their ALI
 * iterations (Sect. 2) as one batch -- one persistent launch per step kind,
 * work items ordered longest ray first, iters_per_launch iterations per
 * captured CUDA graph.  Models that arrive while others run join at the
 * next graph boundary; converged models leave and free their slot.
 * Thread-safe: submit and poll may be called from any thread.
 * ------------------------------------------------------------------------ */
typedef struct loc_server loc_server;

typedef struct loc_server_opts {
    int max_slots;             /* models resident at once (1..65536)          */
    size_t mem_budget_bytes;   /* device memory admitted models may use       */
    int iters_per_launch;      /* ALI iterations per graph launch (1..64)     */
    double window_sigmas;      /* channel window of the march (0 = all)       */
    int device;                /* CUDA device index                           */
    int max_queue;             /* pending requests before LOC_EBUSY (0: no cap) */
} loc_server_opts;

typedef struct loc_result {
    uint64_t ticket;
    loc_status status;         /* LOC_OK, or LOC_ENOTCONV if tol not reached  */
    int iterations;
    double max_rel_dtex;       /* convergence metric of the last iteration    */
    double latency_ms;         /* submit -> result available                  */
    int64_t n_cells;
    int n_levels;
    double updates;            /* (step, channel, line) updates performed     */
} loc_result;

typedef struct loc_server_counters {
    int64_t submitted, completed, active, queued;
    int64_t device_bytes_in_use;
    double p50_ms, p99_ms, mean_ms;   /* latency of completed requests        */
    double models_per_s;              /* completed / (last completion - first submit) */
} loc_server_counters;

/* Start a server (allocates its tables, stream and host thread). */
loc_status loc_server_create(loc_server **out, const loc_server_opts *o);

/* Queue one 1D model (geometry LOC_SHELLS_1D; allocator and stream fields
 * ignored) with its molecule and iteration options (max_iter, tol_tex, ali;
 * FP32 march).  The arrays are copied before return.  *ticket identifies
 * the result.  LOC_EBUSY if max_queue requests are already waiting. */
loc_status loc_server_submit(loc_server *s, const loc_model_desc *d, const loc_molecule_desc *mol,
                             const loc_iter_opts *o, uint64_t *ticket);

/* Wait up to timeout_ms (0: do not wait) for a result.  On success fills
 * *out, copies the populations [n_cells][n_levels] into `populations` (may be
 * NULL; n_out checked) and releases the result.  LOC_ETIMEOUT if not done in
 * time (the request keeps running). */
loc_status loc_server_poll(loc_server *s, uint64_t ticket, int timeout_ms, loc_result *out,
                           double *populations, size_t n_out);

/* Counters and latency percentiles; returns the server's fatal status. */
loc_status loc_server_stats(loc_server *s, loc_server_counters *st);

/* Stop the server: running and queued requests are abandoned. */
void loc_server_destroy(loc_server *s);

/* Active segments of one direction of an octree model (Sect. 2.2), traced
 * on the device by the same traversal the march uses (root rays, rays
 * created at refined cells, terminations).  Record k of out7 is
 * {creation level, i, j, z0, dz, leaf, leaf level}: the lattice line
 * (level, i, j), its segment start z0 and length dz in fixed-point units
 * (one root cell = 2^24), and the leaf index (leaves numbered in the
 * level-ordered cell order).  *n_seg receives the total count; at most cap
 * records are written (beyond cap an unspecified subset is kept, which
 * serves for sampling). */
loc_status loc_trace_octree(const loc_model *m, int dir, int64_t *out7, int64_t cap, int64_t *n_seg);

/* Per-leaf total main-axis length (fixed-point units) of the active
 * segments of one direction of an octree model: the constant-path-length
 * property (Sect. 2.2) makes it exactly 2^24 >> level for every leaf. */
loc_status loc_octree_path_sums(const loc_model *m, int dir, int64_t *out, size_t n_out);

/* Numerical self-check, not a step of the method: r[i] = the reciprocal
 * that the equilibrium solve and the line parameters use in place of an FP64
 * division (an FP32 seed refined by two Newton-Raphson steps, within about
 * one FP64 ulp of 1 / d[i]; zero, subnormal, huge, infinite and NaN inputs
 * give 1.0 / d[i]), evaluated on the current device.  d and r are host
 * arrays of n doubles owned by the caller.  LOC_EINVAL for a NULL buffer
 * with n > 0, LOC_ENOMEM / LOC_ECUDA on device failures. */
loc_status loc_check_recip(const double *d, double *r, size_t n);

/* Wait for all queued work of the model. */
loc_status loc_sync(loc_model *m);

/* Free the model and its device memory. */
void loc_destroy(loc_model *m);

#ifdef __cplusplus
}
#endif
#endif /* LOC_H */
