// loc_api.cu -- the C ABI (include/loc.h): model and molecule set-up, the
// ALI iteration loop, result getters.  Argument marshalling, validation and
// launch sequencing only; every step of the method runs in the kernels of
// k_geom.cu, k_march.cu and k_se.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "loc_internal.cuh"

namespace loc {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

}  // namespace loc

using namespace loc;

struct loc_model {
    DevModel d;
    cudaStream_t st = nullptr;
    loc_allocator alloc{};
    bool custom_alloc = false;
    std::vector<void *> geo_mem;     // lives as long as the model
    std::vector<void *> mol_mem;     // replaced by loc_set_molecule
    std::vector<int> oct_child, oct_leaf;       // octree index arrays (host copies)
    std::vector<int> leaf_api;                  // octree: level-ordered index of each stored leaf
    std::vector<double> leaf_f[7];              // octree per-leaf fields (host staging)
    double *sigma_turb = nullptr;    // device copies kept for set_molecule
    double *vx = nullptr, *vy = nullptr, *vz = nullptr;
    bool has_mol = false;
    bool has_rad = false;
    int last_fp64 = 0;
    long long segs_per_sim = 0;
    int n_sm = 152;
    int tuned_per = 0;               // lines per warp chosen by loc_autotune (0: heuristic)
    int tuned_chunk = 0;             // 1D run length chosen by loc_autotune (0: heuristic, -1: whole rays)
    std::vector<int> ray_off_h;      // 1D: first step of each ray (host copy, n_rays + 1)
    int run_len = 0;                 // 1D: run length of the current run tables (0: none)
    long long run_n = 0;             // runs in the current tables
    int *run_off = nullptr, *run_ray = nullptr;
    int2 *run_rng = nullptr;         // channel range each run's windows touch
    int *run_maxw = nullptr;         // device scalar: widest range
    int rng_len = 0;                 // run length and window of the current ranges
    double rng_window = -1.0;
    int run_tile = 0;                // widest range, rounded up to 32 channels
    float2 *run_ab = nullptr;        // run maps / entering intensities
    size_t run_ab_bytes = 0;
    std::vector<void *> run_mem, run_ab_mem;
    size_t oct_scratch_floats = 0;   // octree traversal scratch currently allocated
    std::vector<void *> oct_mem;
    long long path_records = 0;      // octree: recorded path records (0: the march walks the tree)
    std::vector<void *> path_mem;
    std::vector<void *> tmp_mem;     // buffers of one call (the octree record pool)
    // 1D sub-iterations (set for the duration of a loc_iterate call)
    int sub_k = 0;                   // region: the sub_k innermost shells (0: none)
    int sub_mode = 0;                // 0: full march storing sub_I, 1: region march
    int sub_rays = 0;                // rays that reach the region
    float *sub_I = nullptr;          // [sub_rays][T][n_ch] intensities at the region's boundary
    double *sub_x0 = nullptr;        // populations at the start of the iteration
    size_t sub_bytes = 0;
    std::vector<void *> sub_mem;
};

static void *dev_alloc(loc_model *m, size_t bytes, std::vector<void *> &owner)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (m->custom_alloc) {
        p = m->alloc.alloc(bytes, m->alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) owner.push_back(p);
    return p;
}

static void dev_free_all(loc_model *m, std::vector<void *> &owner)
{
    for (void *p : owner) {
        if (m->custom_alloc) m->alloc.free(p, m->alloc.ctx);
        else cudaFree(p);
    }
    owner.clear();
}

template <class T>
static loc_status upload(loc_model *m, T **dst, const T *src, size_t n, std::vector<void *> &owner,
                         const char *what)
{
    *dst = (T *)dev_alloc(m, sizeof(T) * n, owner);
    if (!*dst) {
        set_error("device allocation of %s (%zu bytes) failed", what, sizeof(T) * n);
        return LOC_ENOMEM;
    }
    if (src) LOC_CUDA_TRY(cudaMemcpyAsync(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, m->st));
    return LOC_OK;
}

#define TRY(x)                          \
    do {                                \
        loc_status _s = (x);            \
        if (_s != LOC_OK) return _s;    \
    } while (0)

#define CHECK(cond, ...)                \
    do {                                \
        if (!(cond)) {                  \
            set_error(__VA_ARGS__);     \
            return LOC_EINVAL;          \
        }                               \
    } while (0)

static bool finite_pos(const double *a, long long n, bool allow_zero)
{
    for (long long i = 0; i < n; i++) {
        if (!std::isfinite(a[i])) return false;
        if (allow_zero ? a[i] < 0.0 : a[i] <= 0.0) return false;
    }
    return true;
}

static bool finite_all(const double *a, long long n)
{
    for (long long i = 0; i < n; i++)
        if (!std::isfinite(a[i])) return false;
    return true;
}

extern "C" {

const char *loc_last_error(void) { return g_err; }

const char *loc_version(void) { return "loc-gb300 0.1 (sm_103a)"; }

// Records of the path walk into a chunk pool (launch_pool_octree), kept
// until they are laid out contiguously; the buffers are the model's tmp_mem.
struct OctPool {
    unsigned long long *pool = nullptr;
    int *next = nullptr;
    int *head = nullptr;
};

// One traversal of every family into a pool sized for about four records
// per leaf and direction (measured clouds need 2.2) plus a partial chunk per
// family, at most 40 % of the free device memory.  Fills fam_work and
// fam_rec and sets ok when every record fit; ok == false (pool not
// allocated, or too small) leaves the two-pass scheme to the caller.
static loc_status pool_octree_paths(loc_model *m, long long fams, unsigned *work, unsigned *nrec, OctPool &P,
                                    bool &ok)
{
    DevModel &D = m->d;
    ok = false;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return LOC_OK;
    }
    const long long chunk_b = kOctPoolChunk * (long long)sizeof(unsigned long long) + (long long)sizeof(int);
    long long cap = (4ll * D.n_cells * D.n_dir + kOctPoolChunk - 1) / kOctPoolChunk + fams;
    cap = std::min(cap, (long long)(0.4 * (double)free_b) / chunk_b);
    cap = std::min(cap, (long long)INT32_MAX);
    if (cap < fams) return LOC_OK;
    P.pool = (unsigned long long *)dev_alloc(m, (size_t)cap * kOctPoolChunk * sizeof(unsigned long long), m->tmp_mem);
    P.next = (int *)dev_alloc(m, (size_t)cap * sizeof(int), m->tmp_mem);
    P.head = (int *)dev_alloc(m, (size_t)fams * sizeof(int), m->tmp_mem);
    unsigned *ctr = (unsigned *)dev_alloc(m, sizeof(unsigned), m->tmp_mem);
    if (!P.pool || !P.next || !P.head || !ctr) {
        dev_free_all(m, m->tmp_mem);
        return LOC_OK;
    }
    // walk order: families by decreasing estimated work, the leaves of the
    // root cells their root line crosses (lateral drift at each root layer's
    // centre, mirrored axes as the march mirrors them), so that the longest
    // walks start first.  The estimate reads N^3 root cells per direction
    // (70 ms of host time for a 64^3 root and 48 directions, but 1.3 s for
    // 128^3 and 10 s for 255^3, strided); beyond 2^25 reads the families
    // are walked in index order.
    int *order_d = nullptr;
    if ((long long)D.N * D.N * D.N * D.n_dir <= (1ll << 25)) {
        const int N = D.N;
        const long long per_dir = (long long)N * N;
        std::vector<Dir3D> dirs(D.n_dir);
        LOC_CUDA_TRY(cudaMemcpyAsync(dirs.data(), D.dirs, sizeof(Dir3D) * D.n_dir, cudaMemcpyDeviceToHost, m->st));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        std::vector<long long> leaves(m->oct_child.size(), 1);
        for (long long c = (long long)leaves.size() - 1; c >= 0; c--) {
            const int ch = m->oct_child[c];
            if (ch >= 0) {
                long long n = 0;
                for (int o = 0; o < 8; o++) n += leaves[ch + o];
                leaves[c] = n;
            }
        }
        std::vector<long long> est(fams, 0);
        const double inv_one = 1.0 / (double)(1ll << kFixedBits);
        const long long stride[3] = {1, N, (long long)N * N};
        std::vector<int> sh_a(N), sh_b(N);
        std::vector<long long> base(N);
        for (int d = 0; d < D.n_dir; d++) {
            const Dir3D &q = dirs[d];
            const double sa = (double)q.qa * inv_one, sb = (double)q.qb * inv_one;   // slopes <= 1
            for (int k = 0; k < N; k++) {
                sh_a[k] = (int)std::floor(sa * (k + 0.5)) % N;
                sh_b[k] = (int)std::floor(sb * (k + 0.5)) % N;
                base[k] = (long long)(q.flip[q.m] ? N - 1 - k : k) * stride[q.m];
            }
            const long long step_a = q.flip[q.a] ? -stride[q.a] : stride[q.a];
            const long long step_b = q.flip[q.b] ? -stride[q.b] : stride[q.b];
            const long long org = (q.flip[q.a] ? (long long)(N - 1) * stride[q.a] : 0) +
                                  (q.flip[q.b] ? (long long)(N - 1) * stride[q.b] : 0);
            for (int i = 0; i < N; i++) {
                for (int j = 0; j < N; j++) {
                    long long w = 0;
                    for (int k = 0; k < N; k++) {
                        int xa = i + sh_a[k], xb = j + sh_b[k];
                        if (xa >= N) xa -= N;
                        if (xb >= N) xb -= N;
                        w += leaves[base[k] + org + xa * step_a + xb * step_b];
                    }
                    est[d * per_dir + (long long)i * N + j] = w;
                }
            }
        }
        std::vector<int> order(fams);
        for (long long f = 0; f < fams; f++) order[f] = (int)f;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return est[x] > est[y]; });
        order_d = (int *)dev_alloc(m, sizeof(int) * (size_t)fams, m->tmp_mem);
        if (order_d)
            LOC_CUDA_TRY(cudaMemcpyAsync(order_d, order.data(), sizeof(int) * (size_t)fams, cudaMemcpyHostToDevice,
                                         m->st));
    }
    TRY(launch_pool_octree(D, P.pool, P.next, cap, ctr, work, nrec, P.head, order_d, m->st));
    int flag = 0;
    LOC_CUDA_TRY(cudaMemcpyAsync(&flag, D.oct_err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    if (flag == 5) {                                  // pool too small: counts exact, records not
        LOC_CUDA_TRY(cudaMemsetAsync(D.oct_err, 0, sizeof(int), m->st));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        dev_free_all(m, m->tmp_mem);
        return LOC_OK;
    }
    if (flag) {
        set_error("tracing the octree paths failed (code %d)", flag);
        return LOC_ECUDA;
    }
    ok = true;
    return LOC_OK;
}

// Records of the octree paths (see record_octree_kernel): offsets from the
// per-family record counts, one device buffer for all records, filled by one
// more traversal, or copied from the pool of pool_octree_paths when given.
// A failed allocation leaves the model walking the tree.
static loc_status record_octree_paths(loc_model *m, const std::vector<unsigned> &nrec, const OctPool *P = nullptr)
{
    DevModel &D = m->d;
    const size_t fams = nrec.size();
    std::vector<long long> off(fams + 1, 0);
    for (size_t f = 0; f < fams; f++) off[f + 1] = off[f] + nrec[f];
    const long long total = off[fams];
    unsigned long long *rec = (unsigned long long *)dev_alloc(m, sizeof(unsigned long long) * (size_t)std::max(total, 1ll), m->path_mem);
    if (!rec) {
        m->path_records = 0;
        return LOC_OK;
    }
    long long *offd = (long long *)dev_alloc(m, sizeof(long long) * (fams + 1), m->path_mem);
    if (!offd) {
        dev_free_all(m, m->path_mem);
        m->path_records = 0;
        return LOC_OK;
    }
    LOC_CUDA_TRY(cudaMemcpyAsync(offd, off.data(), sizeof(long long) * (fams + 1), cudaMemcpyHostToDevice, m->st));
    D.oct_rec = rec;
    D.oct_rec_off = offd;
    if (P) TRY(launch_compact_octree(D, P->pool, P->next, P->head, (long long)fams, m->st));
    else TRY(launch_record_octree(D, m->st));
    int flag = 0;
    LOC_CUDA_TRY(cudaMemcpyAsync(&flag, D.oct_err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    if (flag) {
        set_error("recording the octree paths failed (code %d)", flag);
        return LOC_ECUDA;
    }
    m->path_records = total;
    return LOC_OK;
}

static loc_status create_impl(loc_model *m, const loc_model_desc *d)
{
    DevModel &D = m->d;
    memset(&D, 0, sizeof(D));
    D.geometry = d->geometry;
    D.n_ch = d->n_ch;
    D.v_min = d->v_min;
    D.dv = d->dv;
    D.vmin_f = (float)d->v_min;
    D.dv_f = (float)d->dv;
    D.t_bg = d->t_bg;
    CHECK(d->n_ch >= 1 && d->n_ch <= kMaxChannels, "n_ch must be in [1, %d], got %d", kMaxChannels, d->n_ch);
    CHECK(std::isfinite(d->v_min) && d->dv > 0.0 && std::isfinite(d->dv), "channel grid: need finite v_min and dv > 0");
    CHECK(std::isfinite(d->t_bg) && d->t_bg >= 0.0, "t_bg must be >= 0");
    long long nc = 0;
    if (d->geometry == LOC_SHELLS_1D) {
        CHECK(d->n_shells >= 1 && d->n_shells <= (1 << 16), "n_shells must be in [1, 65536]");
        CHECK(d->radius && d->v, "1D model needs radius and v");
        const int K = d->n_shells;
        CHECK(finite_pos(d->radius, K, false), "radius must be finite and > 0");
        for (int k = 1; k < K; k++) CHECK(d->radius[k] > d->radius[k - 1], "radius must increase strictly");
        CHECK(finite_all(d->v, K), "v must be finite");
        nc = K;
        D.K = K;
        D.n_rays = d->n_rays > 0 ? d->n_rays : K;
        CHECK(D.n_rays <= (1 << 16), "n_rays must be <= 65536");
        CHECK(d->ray_power == 0.0 || (d->ray_power > 0.0 && d->ray_power <= 10.0),
              "ray_power must be 0 (equidistant) or in (0, 10]");
        D.ray_power = d->ray_power > 0.0 ? d->ray_power : 1.0;
    } else if (d->geometry == LOC_GRID_3D) {
        CHECK(d->n_root >= 1 && d->n_root <= 255, "n_root must be in [1, 255]");
        CHECK(d->h0 > 0.0 && std::isfinite(d->h0), "h0 must be > 0");
        CHECK(d->n_dir >= 1 && d->dirs, "3D model needs directions");
        for (int i = 0; i < d->n_dir; i++) {
            const double *v = d->dirs + 3 * i;
            const double n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            CHECK(std::isfinite(n2) && fabs(n2 - 1.0) < 1e-6, "direction %d is not a unit vector", i);
        }
        CHECK(d->vx && d->vy && d->vz, "3D model needs vx, vy, vz");
        nc = (long long)d->n_root * d->n_root * d->n_root;
        D.N = d->n_root;
        D.n_dir = d->n_dir;
        D.h0 = d->h0;
    } else if (d->geometry == LOC_OCTREE_3D) {
        CHECK(d->n_root >= 1 && d->n_root <= 255, "n_root must be in [1, 255]");
        CHECK(d->h0 > 0.0 && std::isfinite(d->h0), "h0 must be > 0");
        CHECK(d->n_dir >= 1 && d->dirs, "3D model needs directions");
        for (int i = 0; i < d->n_dir; i++) {
            const double *v = d->dirs + 3 * i;
            const double n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            CHECK(std::isfinite(n2) && fabs(n2 - 1.0) < 1e-6, "direction %d is not a unit vector", i);
        }
        CHECK(d->octree_levels >= 0 && d->octree_levels <= 10, "octree_levels must be in [0, 10]");
        CHECK(d->octree_paths >= 0 && d->octree_paths <= 2, "octree_paths must be 0, 1 or 2");
        CHECK(d->octree_refine && d->vx && d->vy && d->vz, "octree model needs refine flags and velocities");
        const long long N3 = (long long)d->n_root * d->n_root * d->n_root;
        CHECK(d->octree_n_cells >= N3 && d->octree_n_cells < (1ll << 31), "octree_n_cells out of range");
        D.N = d->n_root;
        D.n_dir = d->n_dir;
        D.h0 = d->h0;
        D.Lmax = d->octree_levels;
        D.n_tree = d->octree_n_cells;
        m->oct_child.assign(D.n_tree, -1);
        m->oct_leaf.assign(D.n_tree, -1);
        std::vector<signed char> lev(D.n_tree, 0);
        long long nxt = N3, nleaf = 0;
        for (long long c = 0; c < D.n_tree; c++) {
            const int r = d->octree_refine[c];
            CHECK(r == 0 || r == 1, "refine flag of cell %lld must be 0 or 1", c);
            CHECK(c < nxt, "refine flags inconsistent: cell %lld has no parent", c);
            if (r) {
                CHECK(lev[c] < D.Lmax, "cell %lld refined below the deepest level", c);
                CHECK(nxt + 8 <= D.n_tree, "refine flags need more than octree_n_cells cells");
                m->oct_child[c] = (int)nxt;
                for (int o = 0; o < 8; o++) lev[nxt + o] = (signed char)(lev[c] + 1);
                nxt += 8;
            } else {
                m->oct_leaf[c] = (int)nleaf++;
            }
        }
        CHECK(nxt == D.n_tree, "refine flags describe %lld cells, octree_n_cells is %lld", nxt, (long long)D.n_tree);
        nc = nleaf;
        // the leaves are stored depth first (root cells in raster order, the
        // children of a refined cell in octant order): a ray's consecutive
        // leaves, and the rays of neighbouring lattice lines, then touch
        // nearby memory.  The interface keeps the level order: leaf_api maps
        // a stored leaf to its level-ordered index.
        m->leaf_api.assign(nleaf, 0);
        {
            std::vector<int> dfs(D.n_tree, -1);
            long long next_id = 0;
            std::vector<long long> stack;
            for (long long r = N3 - 1; r >= 0; r--) stack.push_back(r);
            while (!stack.empty()) {
                const long long c = stack.back();
                stack.pop_back();
                if (m->oct_child[c] >= 0) {
                    for (int o = 7; o >= 0; o--) stack.push_back(m->oct_child[c] + o);
                } else {
                    dfs[c] = (int)next_id++;
                }
            }
            for (long long c = 0; c < D.n_tree; c++)
                if (m->oct_leaf[c] >= 0) {
                    m->leaf_api[dfs[c]] = m->oct_leaf[c];
                    m->oct_leaf[c] = dfs[c];
                }
        }
        // per-leaf copies of the per-cell fields (values of refined cells are ignored)
        auto gather = [&](const double *src, std::vector<double> &dst) {
            dst.resize(nleaf);
            for (long long c = 0; c < D.n_tree; c++)
                if (m->oct_leaf[c] >= 0) dst[m->oct_leaf[c]] = src[c];
        };
        CHECK(d->n_h2 && d->t_kin && d->sigma_turb && d->abundance, "per-cell arrays missing");
        gather(d->n_h2, m->leaf_f[0]);
        gather(d->t_kin, m->leaf_f[1]);
        gather(d->sigma_turb, m->leaf_f[2]);
        gather(d->abundance, m->leaf_f[3]);
        gather(d->vx, m->leaf_f[4]);
        gather(d->vy, m->leaf_f[5]);
        gather(d->vz, m->leaf_f[6]);
    } else {
        CHECK(false, "unknown geometry %d", d->geometry);
    }
    D.n_cells = nc;
    const bool oct = d->geometry == LOC_OCTREE_3D;
    const double *f_n = oct ? m->leaf_f[0].data() : d->n_h2;
    const double *f_t = oct ? m->leaf_f[1].data() : d->t_kin;
    const double *f_s = oct ? m->leaf_f[2].data() : d->sigma_turb;
    const double *f_a = oct ? m->leaf_f[3].data() : d->abundance;
    CHECK(f_n && f_t && f_s && f_a, "per-cell arrays missing");
    CHECK(finite_pos(f_n, nc, true), "n_h2 must be finite and >= 0");
    CHECK(finite_pos(f_t, nc, false), "t_kin must be finite and > 0");
    CHECK(finite_pos(f_s, nc, true), "sigma_turb must be finite and >= 0");
    CHECK(finite_pos(f_a, nc, true), "abundance must be finite and >= 0");

    TRY(upload(m, &D.n_h2, f_n, nc, m->geo_mem, "n_h2"));
    TRY(upload(m, &D.t_kin, f_t, nc, m->geo_mem, "t_kin"));
    TRY(upload(m, &D.abundance, f_a, nc, m->geo_mem, "abundance"));
    TRY(upload(m, &m->sigma_turb, f_s, nc, m->geo_mem, "sigma_turb"));
    TRY(upload<float>(m, &D.inv_s2sig, nullptr, nc, m->geo_mem, "inv_s2sig"));

    if (d->geometry == LOC_SHELLS_1D) {
        const int K = D.K;
        TRY(upload(m, &D.radius, d->radius, K, m->geo_mem, "radius"));
        std::vector<float> v1(K);
        for (int k = 0; k < K; k++) v1[k] = (float)d->v[k];
        TRY(upload(m, &D.v1d, v1.data(), K, m->geo_mem, "v"));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));     // v1 leaves scope
        TRY(upload<int>(m, &D.ray_off, nullptr, D.n_rays + 1, m->geo_mem, "ray offsets"));
        const long long cap = 2ll * D.n_rays * (K + 1);
        TRY(upload<Seg1D>(m, &D.segs, nullptr, cap, m->geo_mem, "ray steps"));
        TRY(launch_geom1d(D, m->st));
        int total = 0;
        LOC_CUDA_TRY(cudaMemcpyAsync(&total, D.ray_off + D.n_rays, sizeof(int), cudaMemcpyDeviceToHost, m->st));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        D.n_segs = total;
        m->segs_per_sim = total;
        m->ray_off_h.resize(D.n_rays + 1);
        LOC_CUDA_TRY(cudaMemcpy(m->ray_off_h.data(), D.ray_off, sizeof(int) * (D.n_rays + 1),
                                cudaMemcpyDeviceToHost));
    } else {
        const double *vx = oct ? m->leaf_f[4].data() : d->vx;
        const double *vy = oct ? m->leaf_f[5].data() : d->vy;
        const double *vz = oct ? m->leaf_f[6].data() : d->vz;
        CHECK(finite_all(vx, nc) && finite_all(vy, nc) && finite_all(vz, nc), "velocities must be finite");
        TRY(upload(m, &m->vx, vx, nc, m->geo_mem, "vx"));
        TRY(upload(m, &m->vy, vy, nc, m->geo_mem, "vy"));
        TRY(upload(m, &m->vz, vz, nc, m->geo_mem, "vz"));
        if (oct) {
            TRY(upload(m, &D.child, m->oct_child.data(), D.n_tree, m->geo_mem, "octree children"));
            TRY(upload(m, &D.leaf_of, m->oct_leaf.data(), D.n_tree, m->geo_mem, "octree leaves"));
            TRY(upload(m, &D.leaf_perm, m->leaf_api.data(), nc, m->geo_mem, "leaf order"));
            TRY(upload<int>(m, &D.oct_err, nullptr, 4, m->geo_mem, "octree flags"));
            LOC_CUDA_TRY(cudaMemsetAsync(D.oct_err, 0, 4 * sizeof(int), m->st));
            const size_t kid_n = (size_t)octree_persistent_warps(D) * 10 * kOctMaxKids;
            TRY(upload<int4>(m, &D.oct_kids, nullptr, kid_n, m->geo_mem, "octree frames"));
        }
        TRY(upload<float4>(m, &D.vel, nullptr, nc, m->geo_mem, "velocity records"));
        double *dirs = nullptr;
        TRY(upload(m, &dirs, d->dirs, 3 * (size_t)d->n_dir, m->geo_mem, "dirs"));
        TRY(upload<Dir3D>(m, &D.dirs, nullptr, d->n_dir, m->geo_mem, "direction records"));
        TRY(launch_dir_setup(dirs, d->n_dir, d->h0, D.dirs, m->st));
        unsigned long long *cnt = nullptr, total = 0;
        TRY(upload<unsigned long long>(m, &cnt, nullptr, 1, m->geo_mem, "segment count"));
        if (oct) {
            // count the active steps of every root-ray family; the march takes
            // the families in order of decreasing work (fewer idle warps at
            // the end of a persistent launch)
            const long long fams = (long long)D.N * D.N * D.n_dir;
            unsigned *work = nullptr, *nrec = nullptr;
            TRY(upload<unsigned>(m, &work, nullptr, fams, m->geo_mem, "family work"));
            TRY(upload<unsigned>(m, &nrec, nullptr, fams, m->geo_mem, "family records"));
            // recording: one walk into a pool when it fits, else a counting
            // walk here and a recording walk below
            OctPool pool;
            bool pooled = false;
            const bool record = d->octree_paths != 1;
            if (d->octree_paths == 0) {
                TRY(pool_octree_paths(m, fams, work, nrec, pool, pooled));
            }
            if (!pooled) {
                TRY(launch_trace_octree(D, -1, nullptr, 0, cnt, m->st, nullptr, work, nrec));
                LOC_CUDA_TRY(cudaMemcpyAsync(&total, cnt, sizeof(total), cudaMemcpyDeviceToHost, m->st));
                LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
            }
            std::vector<unsigned> wh(fams), rh(fams);
            LOC_CUDA_TRY(cudaMemcpy(wh.data(), work, sizeof(unsigned) * fams, cudaMemcpyDeviceToHost));
            LOC_CUDA_TRY(cudaMemcpy(rh.data(), nrec, sizeof(unsigned) * fams, cudaMemcpyDeviceToHost));
            if (pooled) {
                total = 0;
                for (long long f = 0; f < fams; f++) total += wh[f];
            }
            std::vector<int> order(fams);
            for (long long f = 0; f < fams; f++) order[f] = (int)f;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return wh[x] > wh[y]; });
            TRY(upload(m, &D.oct_order, order.data(), fams, m->geo_mem, "family order"));
            LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
            // the paths never change: record them once (8 bytes per step or
            // intensity copy) and let every ray simulation replay them,
            // unless the caller asked to walk the tree or the records do not
            // fit in device memory
            if (record) {
                const loc_status rs = record_octree_paths(m, rh, pooled ? &pool : nullptr);
                if (!m->tmp_mem.empty()) {
                    cudaStreamSynchronize(m->st);
                    dev_free_all(m, m->tmp_mem);
                }
                if (rs != LOC_OK) return rs;
            }
        } else {
            TRY(launch_count3d(D, cnt, m->st));
            LOC_CUDA_TRY(cudaMemcpyAsync(&total, cnt, sizeof(total), cudaMemcpyDeviceToHost, m->st));
            LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        }
        m->segs_per_sim = (long long)total;
    }
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    return LOC_OK;
}

loc_status loc_create_model(loc_model **out, const loc_model_desc *d)
{
    if (!out || !d) { set_error("NULL argument"); return LOC_EINVAL; }
    *out = nullptr;
    loc_model *m = new (std::nothrow) loc_model();
    if (!m) { set_error("host allocation failed"); return LOC_ENOMEM; }
    m->st = (cudaStream_t)d->stream;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            m->n_sm = nsm;
        cudaGetLastError();
    }
    if (d->allocator) {
        if (!d->allocator->alloc || !d->allocator->free) {
            delete m;
            set_error("allocator needs alloc and free");
            return LOC_EINVAL;
        }
        m->alloc = *d->allocator;
        m->custom_alloc = true;
    }
    loc_status s = create_impl(m, d);
    if (s != LOC_OK) {
        loc_destroy(m);               // every buffer list, not only the geometry
        return s;
    }
    *out = m;
    return LOC_OK;
}

static loc_status set_molecule_impl(loc_model *m, const loc_molecule_desc *mol)
{
    DevModel &D = m->d;
    CHECK(mol->n_levels >= 2 && mol->n_levels <= kMaxLevels, "n_levels must be in [2, %d]", kMaxLevels);
    CHECK(mol->n_lines >= 1 && mol->n_lines <= kMaxLines, "n_lines must be in [1, %d]", kMaxLines);
    CHECK(mol->n_coll >= 0, "n_coll must be >= 0");
    CHECK(mol->energy_K && mol->g && mol->line_u && mol->line_l && mol->line_A && mol->line_nu,
          "molecule arrays missing");
    CHECK(mol->n_coll == 0 || (mol->coll_u && mol->coll_l && mol->coll_k), "collision arrays missing");
    CHECK(mol->mass_amu > 0.0 && std::isfinite(mol->mass_amu), "mass_amu must be > 0");
    const int L = mol->n_levels;
    CHECK(finite_pos(mol->g, L, false), "g must be > 0");
    CHECK(finite_all(mol->energy_K, L), "energies must be finite");
    for (int t = 0; t < mol->n_lines; t++) {
        const int u = mol->line_u[t], l = mol->line_l[t];
        CHECK(u >= 0 && u < L && l >= 0 && l < L && u != l, "line %d: bad levels", t);
        CHECK(mol->line_A[t] >= 0.0 && mol->line_nu[t] > 0.0, "line %d: bad A or nu", t);
    }
    for (int p = 0; p < mol->n_coll; p++) {
        const int u = mol->coll_u[p], l = mol->coll_l[p];
        CHECK(u >= 0 && u < L && l >= 0 && l < L && u != l, "collision %d: bad levels", p);
        CHECK(mol->coll_k[p] >= 0.0 && std::isfinite(mol->coll_k[p]), "collision %d: bad rate", p);
    }
    CHECK(distinct_level_pairs(mol->line_u, mol->line_l, mol->n_lines, L),
          "two lines join the same pair of levels");
    CHECK(distinct_level_pairs(mol->coll_u, mol->coll_l, mol->n_coll, L),
          "two collision entries join the same pair of levels");
    // hyperfine components: offsets in channel units, per-line ranges
    std::vector<int> hf_off;
    std::vector<float> hf_o, hf_w;
    float olo = 0.f, ohi = 0.f;
    if (mol->hf_n) {
        CHECK(D.geometry == LOC_SHELLS_1D, "hyperfine lines are supported for 1D models");
        hf_off.assign(mol->n_lines + 1, 0);
        int total = 0;
        for (int t = 0; t < mol->n_lines; t++) {
            CHECK(mol->hf_n[t] >= 0 && mol->hf_n[t] <= 16, "line %d: hyperfine components must be 0..16", t);
            total += mol->hf_n[t];
            hf_off[t + 1] = total;
        }
        CHECK(total == 0 || (mol->hf_v && mol->hf_w), "hyperfine offsets and strengths missing");
        for (int t = 0; t < mol->n_lines; t++) {
            double wsum = 0.0;
            for (int c = hf_off[t]; c < hf_off[t + 1]; c++) {
                CHECK(std::isfinite(mol->hf_v[c]) && std::isfinite(mol->hf_w[c]) && mol->hf_w[c] >= 0.0,
                      "line %d: bad hyperfine component %d", t, c - hf_off[t]);
                wsum += mol->hf_w[c];
                const float o = (float)(mol->hf_v[c] / D.dv);
                hf_o.push_back(o);
                hf_w.push_back((float)mol->hf_w[c]);
                olo = std::min(olo, o);
                ohi = std::max(ohi, o);
            }
            CHECK(hf_off[t + 1] == hf_off[t] || fabs(wsum - 1.0) <= 1e-6,
                  "line %d: hyperfine strengths sum to %g, not 1", t, wsum);
        }
        if (total == 0) hf_off.clear();
    }
    D.L = L;
    D.T = mol->n_lines;
    D.P = mol->n_coll;
    D.mass_amu = mol->mass_amu;
    std::vector<int> lu(mol->line_u, mol->line_u + D.T), ll(mol->line_l, mol->line_l + D.T);
    std::vector<int> cu(mol->coll_u, mol->coll_u + D.P), cl(mol->coll_l, mol->coll_l + D.P);
    TRY(upload(m, &D.energy_K, mol->energy_K, L, m->mol_mem, "energies"));
    TRY(upload(m, &D.g, mol->g, L, m->mol_mem, "weights"));
    TRY(upload(m, &D.line_u, lu.data(), D.T, m->mol_mem, "line_u"));
    TRY(upload(m, &D.line_l, ll.data(), D.T, m->mol_mem, "line_l"));
    TRY(upload(m, &D.line_A, mol->line_A, D.T, m->mol_mem, "line_A"));
    TRY(upload(m, &D.line_nu, mol->line_nu, D.T, m->mol_mem, "line_nu"));
    TRY(upload(m, &D.coll_u, cu.data(), D.P, m->mol_mem, "coll_u"));
    TRY(upload(m, &D.coll_l, cl.data(), D.P, m->mol_mem, "coll_l"));
    TRY(upload(m, &D.coll_k, mol->coll_k, D.P, m->mol_mem, "coll_k"));
    D.hf_off = nullptr;
    D.hf_o = D.hf_w = nullptr;
    D.hf_olo = olo;
    D.hf_ohi = ohi;
    if (!hf_off.empty()) {
        TRY(upload(m, &D.hf_off, hf_off.data(), hf_off.size(), m->mol_mem, "hyperfine ranges"));
        TRY(upload(m, &D.hf_o, hf_o.data(), hf_o.size(), m->mol_mem, "hyperfine offsets"));
        TRY(upload(m, &D.hf_w, hf_w.data(), hf_w.size(), m->mol_mem, "hyperfine strengths"));
    }
    const long long nc = D.n_cells;
    TRY(upload<float>(m, &D.nbg, nullptr, D.T, m->mol_mem, "nbg"));
    TRY(upload<double>(m, &D.nbg64, nullptr, D.T, m->mol_mem, "nbg64"));
    TRY(upload<double>(m, &D.x, nullptr, nc * L, m->mol_mem, "populations"));
    TRY(upload<double>(m, &D.x_new, nullptr, nc * L, m->mol_mem, "populations"));
    TRY(upload<float2>(m, &D.ks, nullptr, nc * D.T, m->mol_mem, "line parameters"));
    TRY(upload<float2>(m, &D.acc, nullptr, nc * D.T, m->mol_mem, "accumulators"));
    TRY(upload<float>(m, &D.norm, nullptr, nc, m->mol_mem, "norm"));
    TRY(upload<float2>(m, &D.acc_c, nullptr, nc * D.T, m->mol_mem, "accumulator compensation"));
    TRY(upload<float>(m, &D.norm_c, nullptr, nc, m->mol_mem, "norm compensation"));
    LOC_CUDA_TRY(cudaMemsetAsync(D.acc_c, 0, sizeof(float2) * nc * D.T, m->st));
    LOC_CUDA_TRY(cudaMemsetAsync(D.norm_c, 0, sizeof(float) * nc, m->st));
    TRY(upload<double>(m, &D.acc64, nullptr, 2 * nc * D.T, m->mol_mem, "accumulators64"));
    TRY(upload<double>(m, &D.norm64, nullptr, nc, m->mol_mem, "norm64"));
    TRY(upload<unsigned int>(m, &D.dtex_bits, nullptr, 1, m->mol_mem, "dtex"));
    TRY(upload<unsigned long long>(m, &D.maser_count, nullptr, 1, m->mol_mem, "maser count"));
    TRY(upload<unsigned long long>(m, &D.upd_count, nullptr, 1, m->mol_mem, "update count"));
    TRY(upload<unsigned long long>(m, &D.nom_count, nullptr, 1, m->mol_mem, "nominal update count"));
    // collision rates depend only on n_H2 and T_kin: tabulated once when the
    // table (16 B per cell and pair) takes at most a quarter of the free
    // device memory and 16 GiB, else computed inside every solve (an FP64
    // exponential per pair and cell, the costliest part of a large solve)
    D.coll_rates = nullptr;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
    const double table_b = 16.0 * (double)nc * (double)D.P;
    if (D.P > 0 && table_b <= std::min(0.25 * (double)free_b, 16.0 * (1ull << 30))) {
        TRY(upload<double2>(m, &D.coll_rates, nullptr, nc * D.P, m->mol_mem, "collision rates"));
        TRY(launch_coll_rates(D, D.coll_rates, m->st));
    }
    TRY(launch_cell_setup(D, m->sigma_turb, m->vx, m->vy, m->vz, m->st));
    TRY(launch_bg(D, m->st));
    TRY(launch_lte(D, m->st));
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));    // host vectors leave scope
    return LOC_OK;
}

loc_status loc_set_molecule(loc_model *m, const loc_molecule_desc *mol)
{
    if (!m || !mol) { set_error("NULL argument"); return LOC_EINVAL; }
    cudaStreamSynchronize(m->st);
    dev_free_all(m, m->mol_mem);
    m->has_mol = false;
    m->has_rad = false;
    m->rng_len = 0;                  // line widths change with the molecule
    loc_status s = set_molecule_impl(m, mol);
    if (s != LOC_OK) {
        cudaStreamSynchronize(m->st);
        dev_free_all(m, m->mol_mem);
        return s;
    }
    m->has_mol = true;
    return LOC_OK;
}

loc_status loc_reset_populations(loc_model *m)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("no molecule"); return LOC_ESTATE; }
    TRY(launch_lte(m->d, m->st));
    m->has_rad = false;
    return LOC_OK;
}

// octree traversal status flag (set by the kernel when a frame overflows)
static loc_status octree_status(loc_model *m)
{
    if (m->d.geometry != LOC_OCTREE_3D) return LOC_OK;
    int flag = 0;
    LOC_CUDA_TRY(cudaMemcpyAsync(&flag, m->d.oct_err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    if (flag) {
        set_error("octree traversal capacity exceeded (code %d): too many new rays in one cell face", flag);
        return LOC_ECUDA;
    }
    return LOC_OK;
}

static loc_status check_opts(const loc_iter_opts *o)
{
    CHECK(o, "NULL options");
    CHECK(o->max_iter >= 1, "max_iter must be >= 1");
    CHECK(o->tol_tex >= 0.0 && std::isfinite(o->tol_tex), "tol_tex must be >= 0");
    CHECK(o->precision == LOC_FP32_MARCH || o->precision == LOC_FP64_ACC || o->precision == LOC_FP32_PLAIN,
          "unknown precision");
    CHECK(o->lines_per_pass >= 0, "lines_per_pass must be >= 0");
    CHECK(o->window_sigmas >= 0.0 && std::isfinite(o->window_sigmas), "window_sigmas must be >= 0");
    CHECK(o->profile == 0 || o->profile == 1, "profile must be 0 or 1");
    CHECK(o->level_cutoff >= 0.0 && o->level_cutoff <= 1e-6, "level_cutoff must be in [0, 1e-6]");
    CHECK(o->dir_begin >= 0 && o->dir_end >= 0, "direction range must be >= 0");
    CHECK(o->sub_iters >= 0 && o->sub_iters <= 1000, "sub_iters must be in [0, 1000]");
    CHECK(o->sub_iters == 0 || o->level_cutoff == 0.0, "sub-iterations and level_cutoff do not combine");
    return LOC_OK;
}

// lines per warp: the requested group size, or (0) all lines when the
// launch has enough rays to fill the GPU, otherwise smaller groups so that
// more warps share each ray's lines
static int lines_per_warp(const loc_model *m, const loc_iter_opts *o)
{
    const DevModel &D = m->d;
    if (o->lines_per_pass == 0 && m->tuned_per > 0 && m->tuned_per <= D.T) return m->tuned_per;
    int per = o->lines_per_pass > 0 ? o->lines_per_pass : D.T;
    if (per > kMaxLinesPerWarp) per = kMaxLinesPerWarp;
    if (per > D.T) per = D.T;
    if (o->lines_per_pass == 0) {
        const long long items = (D.geometry == LOC_SHELLS_1D) ? (long long)D.n_rays
                                                              : (long long)D.N * D.N * D.n_dir;
        // octree walked in every march: at most 6 lines share one traversal
        // (measured best on the 32^3- and 64^3-root clouds; more lines per
        // warp cost occupancy); replayed paths carry every line per warp
        if (D.geometry == LOC_OCTREE_3D && !D.oct_rec && per > 6) per = (D.T + (D.T + 5) / 6 - 1) / ((D.T + 5) / 6);
        const long long target = 32ll * m->n_sm;
        while (per > 1 && items * ((D.T + per - 1) / per) < target) per = (per + 1) / 2;
    }
    // shared memory: 4 warps x per x n_ch floats per block
    while (per > 1 && 4ll * per * D.n_ch * 4 > 200 * 1024) per--;
    return per;
}

// 1D run length (steps per run; 0: whole rays): the requested one, the
// tuned one, or automatically whole rays when the (ray, line group) items
// fill the GPU, else the longest power-of-two run (>= 16 steps) that gives
// at least 64 warps per SM
static int steps_per_run(const loc_model *m, const loc_iter_opts *o, int per)
{
    const DevModel &D = m->d;
    if (D.geometry != LOC_SHELLS_1D) return 0;
    if (m->sub_k > 0) return 0;                  // sub-iterations march whole rays
    if (D.hf_off) return 0;                      // so do hyperfine lines
    int c = o->steps_per_chunk != 0 ? o->steps_per_chunk : m->tuned_chunk;
    if (c < 0) return 0;
    if (c > 0) return c;
    const long long groups = (D.T + per - 1) / per;
    const long long target = 64ll * m->n_sm;
    if ((long long)D.n_rays * groups >= target) return 0;
    int longest = 0;
    for (int j = 0; j < D.n_rays; j++) longest = std::max(longest, m->ray_off_h[j + 1] - m->ray_off_h[j]);
    int len = 16;
    for (int cand = 4096; cand >= 16; cand >>= 1) {
        long long runs = 0;
        for (int j = 0; j < D.n_rays; j++) runs += (m->ray_off_h[j + 1] - m->ray_off_h[j] + cand - 1) / cand;
        len = cand;
        if (runs * groups >= target) break;
    }
    return len >= longest ? 0 : len;
}

// run tables of length len ([n_rays + 1] first run of each ray, [runs] ray
// of each run) and the run-map buffer [runs][T][n_ch]
static loc_status ensure_runs(loc_model *m, int len)
{
    DevModel &D = m->d;
    if (m->run_len != len) {
        std::vector<int> off(D.n_rays + 1, 0), ray;
        for (int j = 0; j < D.n_rays; j++) {
            const int nr = (m->ray_off_h[j + 1] - m->ray_off_h[j] + len - 1) / len;
            for (int c = 0; c < nr; c++) ray.push_back(j);
            off[j + 1] = off[j] + nr;
        }
        if (ray.empty()) ray.push_back(0);
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));   // the old tables may be in use
        dev_free_all(m, m->run_mem);
        m->run_len = 0;
        TRY(upload(m, &m->run_off, off.data(), off.size(), m->run_mem, "run offsets"));
        TRY(upload(m, &m->run_ray, ray.data(), ray.size(), m->run_mem, "run rays"));
        TRY(upload<int2>(m, &m->run_rng, nullptr, ray.size(), m->run_mem, "run ranges"));
        TRY(upload<int>(m, &m->run_maxw, nullptr, 1, m->run_mem, "run range width"));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));   // host tables leave scope
        m->run_len = len;
        m->run_n = off[D.n_rays];
        m->rng_len = 0;
    }
    const size_t need = sizeof(float2) * (size_t)std::max(m->run_n, 1ll) * D.T * D.n_ch;
    if (need > m->run_ab_bytes) {
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        dev_free_all(m, m->run_ab_mem);
        m->run_ab_bytes = 0;
        m->run_ab = (float2 *)dev_alloc(m, need, m->run_ab_mem);
        if (!m->run_ab) { set_error("device allocation of the run maps (%zu bytes) failed", need); return LOC_ENOMEM; }
        m->run_ab_bytes = need;
    }
    return LOC_OK;
}

// one ray simulation: zero the accumulators, then the march over all
// (ray, line group) work items -- one launch, or for 1D rays cut into runs
// the affine / scan / run launches
static loc_status march_impl(loc_model *m, const loc_iter_opts *o, bool zeroed = false)
{
    DevModel &D = m->d;
    const int fp64 = o->precision == LOC_FP64_ACC;
    if (zeroed) {
        // the line-parameter launch of this iteration cleared the accumulators
    } else if (fp64) {
        LOC_CUDA_TRY(cudaMemsetAsync(D.acc64, 0, sizeof(double) * 2 * D.T * D.n_cells, m->st));
        LOC_CUDA_TRY(cudaMemsetAsync(D.norm64, 0, sizeof(double) * D.n_cells, m->st));
    } else {
        LOC_CUDA_TRY(cudaMemsetAsync(D.acc, 0, sizeof(float2) * D.T * D.n_cells, m->st));
        LOC_CUDA_TRY(cudaMemsetAsync(D.norm, 0, sizeof(float) * D.n_cells, m->st));
        LOC_CUDA_TRY(cudaMemsetAsync(D.acc_c, 0, sizeof(float2) * D.T * D.n_cells, m->st));
        LOC_CUDA_TRY(cudaMemsetAsync(D.norm_c, 0, sizeof(float) * D.n_cells, m->st));
    }
    MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.per = lines_per_warp(m, o);
    const int run = steps_per_run(m, o, a.per);
    a.window = (float)o->window_sigmas;
    a.inv_dv = (float)(1.0 / D.dv);
    a.dir0 = 0;
    a.dir1 = D.n_dir;
    if (D.geometry != LOC_SHELLS_1D && (o->dir_begin != 0 || o->dir_end != 0)) {
        CHECK(o->dir_begin >= 0 && o->dir_begin < o->dir_end && o->dir_end <= D.n_dir,
              "direction range [%d, %d) outside [0, %d) or empty", o->dir_begin, o->dir_end, D.n_dir);
        a.dir0 = o->dir_begin;
        a.dir1 = o->dir_end;
    }
    if (run > 0) {
        TRY(ensure_runs(m, run));
        a.chunk = run;
        a.n_chunks = m->run_n;
        a.chunk_off = m->run_off;
        a.chunk_ray = m->run_ray;
        a.ab = m->run_ab;
        a.run_rng = m->run_rng;
        // each run's window union depends only on the model, the run length
        // and the window: found once, it sizes the affine launch's tiles
        if (m->rng_len != run || m->rng_window != o->window_sigmas) {
            int w = 0;
            if (a.n_chunks > 0) {
                LOC_CUDA_TRY(cudaMemsetAsync(m->run_maxw, 0, sizeof(int), m->st));
                TRY(launch_march1d_ranges(D, a, m->run_maxw, m->st));
                LOC_CUDA_TRY(cudaMemcpyAsync(&w, m->run_maxw, sizeof(int), cudaMemcpyDeviceToHost, m->st));
                LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
            }
            m->run_tile = std::min(D.n_ch, std::max(32, (w + 31) / 32 * 32));
            m->rng_len = run;
            m->rng_window = o->window_sigmas;
        }
        a.tile = m->run_tile;
        // the affine launch keeps two [per][tile] arrays per warp in shared memory
        while (a.per > 1 && 32ll * a.per * a.tile > 200 * 1024) a.per--;
    }
    if (D.geometry == LOC_OCTREE_3D) {
        const size_t need = (size_t)octree_max_warps(D) * 10 * a.per * D.n_ch;
        if (need > m->oct_scratch_floats) {
            LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
            dev_free_all(m, m->oct_mem);
            D.oct_scratch = (float *)dev_alloc(m, sizeof(float) * need, m->oct_mem);
            if (!D.oct_scratch) { set_error("device allocation of octree scratch failed"); return LOC_ENOMEM; }
            m->oct_scratch_floats = need;
        }
    }
    a.n_groups = (D.T + a.per - 1) / a.per;
    a.fp64_acc = fp64;
    a.comp = o->precision == LOC_FP32_MARCH;
    a.count = o->profile;
    a.sub_k = m->sub_k;
    a.sub_mode = m->sub_mode;
    a.sub_I = m->sub_I;
    if (run > 0) {
        if (a.n_chunks > 0) TRY(launch_march1d_chunked(D, a, m->st));
    } else if (m->sub_k > 0 && m->sub_mode == 1) {
        DevModel R = D;                          // the rays that reach the region
        R.n_rays = m->sub_rays;
        if (R.n_rays > 0) TRY(launch_march(R, a, m->st));
    } else {
        TRY(launch_march(D, a, m->st));
    }
    m->has_rad = true;
    m->last_fp64 = fp64;
    return LOC_OK;
}

loc_status loc_autotune(loc_model *m, const loc_iter_opts *o, int *best_per, int *best_chunk,
                        double *best_ms)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    TRY(check_opts(o));
    if (!m->has_mol) { set_error("loc_set_molecule has not been called"); return LOC_ESTATE; }
    const DevModel &D = m->d;
    m->tuned_per = 0;
    m->tuned_chunk = 0;
    std::vector<int> cand;
    for (int parts = 1; parts <= D.T; parts++) {
        int per = (D.T + parts - 1) / parts;
        if (per > kMaxLinesPerWarp) continue;
        if (4ll * per * D.n_ch * 4 > 200 * 1024) continue;
        bool seen = false;
        for (int c : cand) seen |= (c == per);
        if (!seen) cand.push_back(per);
        if (cand.size() >= 6) break;
    }
    if (cand.empty()) cand.push_back(1);
    // 1D: whole rays (-1) and runs shorter than the longest ray
    std::vector<int> runs = {-1};
    if (D.geometry == LOC_SHELLS_1D) {
        int longest = 0;
        for (int j = 0; j < D.n_rays; j++) longest = std::max(longest, m->ray_off_h[j + 1] - m->ray_off_h[j]);
        for (int len : {128, 64, 32, 16, 8})
            if (len < longest) runs.push_back(len);
    }
    // timed with the per-cell line truncation the iterations will use
    TRY(launch_line_params(m->d, m->st, 0, o->level_cutoff));
    cudaEvent_t e0, e1;
    LOC_CUDA_TRY(cudaEventCreate(&e0));
    LOC_CUDA_TRY(cudaEventCreate(&e1));
    m->d.trunc = o->level_cutoff > 0.0 ? 1 : 0;        // reset below on every path
    int best = cand[0], best_run = -1;
    float best_t = 1e30f;
    loc_iter_opts oo = *o;
    loc_status st = LOC_OK;
    for (int run : runs) {
        for (int per : cand) {
            // run mode keeps twice the shared memory per warp
            if (run > 0 && 32ll * per * D.n_ch > 200 * 1024) continue;
            oo.lines_per_pass = per;
            oo.steps_per_chunk = run;
            float t_min = 1e30f;
            for (int rep = 0; rep < 2 && st == LOC_OK; rep++) {
                cudaEventRecord(e0, m->st);
                st = march_impl(m, &oo);
                cudaEventRecord(e1, m->st);
                if (cudaEventSynchronize(e1) != cudaSuccess) { set_error("autotune march failed"); st = LOC_ECUDA; }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < t_min) t_min = ms;
            }
            if (st != LOC_OK) break;
            if (t_min < best_t) { best_t = t_min; best = per; best_run = run; }
        }
        if (st != LOC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->d.trunc = 0;
    if (st != LOC_OK) return st;
    m->tuned_per = best;
    m->tuned_chunk = best_run;
    if (best_per) *best_per = best;
    if (best_chunk) *best_chunk = best_run;
    if (best_ms) *best_ms = best_t;
    return LOC_OK;
}

loc_status loc_march(loc_model *m, const loc_iter_opts *o)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    TRY(check_opts(o));
    if (!m->has_mol) { set_error("loc_set_molecule has not been called"); return LOC_ESTATE; }
    TRY(launch_line_params(m->d, m->st));
    TRY(march_impl(m, o));
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    return octree_status(m);
}

// Sub-iterations (1D): the region is the sub_shells innermost shells; the
// rays that reach it are those whose step list is longer than the 2 (K -
// sub_shells) steps outside it (impact parameters grow with the ray index,
// so they are the first sub_rays rays).  Buffers for the intensities at the
// region's boundary and for the populations at the start of an iteration.
static loc_status sub_setup(loc_model *m, const loc_iter_opts *o)
{
    DevModel &D = m->d;
    CHECK(D.geometry == LOC_SHELLS_1D, "sub-iterations need a 1D model");
    CHECK(o->sub_shells >= 1 && o->sub_shells <= D.K, "sub_shells must be in [1, %d]", D.K);
    const int outer = D.K - o->sub_shells;
    int rays = 0;
    for (int j = 0; j < D.n_rays; j++)
        if (m->ray_off_h[j + 1] - m->ray_off_h[j] > 2 * outer) rays = j + 1;
    const size_t bI = sizeof(float) * (size_t)std::max(rays, 1) * D.T * D.n_ch;
    const size_t bx = sizeof(double) * (size_t)D.n_cells * D.L;
    if (bI + bx > m->sub_bytes) {
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        dev_free_all(m, m->sub_mem);
        m->sub_bytes = 0;
        m->sub_I = (float *)dev_alloc(m, bI, m->sub_mem);
        m->sub_x0 = (double *)dev_alloc(m, bx, m->sub_mem);
        if (!m->sub_I || !m->sub_x0) { set_error("device allocation for sub-iterations failed"); return LOC_ENOMEM; }
        m->sub_bytes = bI + bx;
    }
    m->sub_k = o->sub_shells;
    m->sub_rays = rays;
    m->sub_mode = 0;
    return LOC_OK;
}

// n_sub sub-iterations of the region after a full iteration: line
// parameters of the region's cells (accumulators cleared), the region's
// steps of the rays that reach it from the intensities stored at its
// boundary, the equilibrium of the region's cells, whose new populations
// replace the old ones (the cells outside keep theirs).
static loc_status sub_iterations(loc_model *m, const loc_iter_opts *o)
{
    DevModel &D = m->d;
    DevModel R = D;
    R.n_cells = m->sub_k;
    const int fp64 = o->precision == LOC_FP64_ACC;
    for (int q = 0; q < o->sub_iters; q++) {
        TRY(launch_line_params(R, m->st, fp64 ? 2 : 1, 0.0));
        m->sub_mode = 1;
        const loc_status st = march_impl(m, o, true);
        m->sub_mode = 0;
        TRY(st);
        R.x = D.x;
        R.x_new = D.x_new;
        TRY(launch_se(R, o->ali, fp64, m->st, 0, 0, 0.0));
        LOC_CUDA_TRY(cudaMemcpyAsync(D.x, D.x_new, sizeof(double) * (size_t)m->sub_k * D.L,
                                     cudaMemcpyDeviceToDevice, m->st));
    }
    return LOC_OK;
}

loc_status loc_iterate(loc_model *m, const loc_iter_opts *o, loc_iter_report *r)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    TRY(check_opts(o));
    if (!m->has_mol) { set_error("loc_set_molecule has not been called"); return LOC_ESTATE; }
    DevModel &D = m->d;
    const bool prof = o->profile == 1;
    std::vector<cudaEvent_t> ev;              // 4 per iteration when profiling
    auto mark = [&](size_t idx) -> cudaError_t {
        if (!prof) return cudaSuccess;
        while (ev.size() <= idx) {
            cudaEvent_t e;
            cudaError_t ce = cudaEventCreate(&e);
            if (ce != cudaSuccess) return ce;
            ev.push_back(e);
        }
        return cudaEventRecord(ev[idx], m->st);
    };
    cudaEvent_t e0, e1;
    LOC_CUDA_TRY(cudaEventCreate(&e0));
    LOC_CUDA_TRY(cudaEventCreate(&e1));
    LOC_CUDA_TRY(cudaMemsetAsync(D.maser_count, 0, sizeof(unsigned long long), m->st));
    LOC_CUDA_TRY(cudaMemsetAsync(D.upd_count, 0, sizeof(unsigned long long), m->st));
    LOC_CUDA_TRY(cudaMemsetAsync(D.nom_count, 0, sizeof(unsigned long long), m->st));
    LOC_CUDA_TRY(cudaEventRecord(e0, m->st));
    int it = 0;
    float dtex = 0.f;
    bool converged = false;
    const bool sub = o->sub_iters > 0;
    if (sub) TRY(sub_setup(m, o));
    const bool fuse = !(o->tol_tex > 0.0) && !sub;
    D.trunc = o->level_cutoff > 0.0 ? 1 : 0;           // reset after the loop on every path
    loc_status st = LOC_OK;
    // NVTX ranges mark the host-side phases of every iteration for timeline
    // tools (no cost without an attached tool)
    nvtxRangePushA("loc_iterate");
    for (it = 0; it < o->max_iter; it++) {
        const size_t b = 5 * (size_t)it;
        if (mark(b) != cudaSuccess) { st = LOC_ECUDA; break; }
        if (sub && cudaMemcpyAsync(m->sub_x0, D.x, sizeof(double) * D.n_cells * D.L, cudaMemcpyDeviceToDevice,
                                   m->st) != cudaSuccess) { st = LOC_ECUDA; break; }
        // with a fixed iteration count (no tolerance) the first iteration's
        // line parameters (and cleared accumulators) come from their own
        // launch and every later iteration's from the previous iteration's
        // solve; with a tolerance, a converged call must leave the last ray
        // simulation's accumulators readable, so every iteration launches them
        if (it == 0 || !fuse) {
            nvtxRangePushA("line parameters");
            st = launch_line_params(D, m->st, o->precision == LOC_FP64_ACC ? 2 : 1, o->level_cutoff);
            nvtxRangePop();
            if (st != LOC_OK) break;
        }
        if (mark(b + 1) != cudaSuccess) { st = LOC_ECUDA; break; }
        nvtxRangePushA("ray march");
        st = march_impl(m, o, true);
        nvtxRangePop();
        if (st != LOC_OK) break;
        if (mark(b + 2) != cudaSuccess) { st = LOC_ECUDA; break; }
        // the metric is read when a tolerance is set, and after the last iteration
        const int want = (o->tol_tex > 0.0 || it == o->max_iter - 1) ? 1 : 0;
        if (want && it > 0 && fuse) {
            if (cudaMemsetAsync(D.dtex_bits, 0, sizeof(unsigned), m->st) != cudaSuccess) { st = LOC_ECUDA; break; }
        }
        const int next = (fuse && it < o->max_iter - 1) ? 1 : 0;
        nvtxRangePushA("statistical equilibrium");
        st = launch_se(D, o->ali, o->precision == LOC_FP64_ACC, m->st, sub ? 0 : want, next, o->level_cutoff);
        nvtxRangePop();
        if (st != LOC_OK) break;
        if (mark(b + 3) != cudaSuccess) { st = LOC_ECUDA; break; }
        std::swap(D.x, D.x_new);
        if (sub) {
            nvtxRangePushA("sub-iterations");
            st = sub_iterations(m, o);
            if (st == LOC_OK && want) {
                // the metric of the whole iteration: populations before and after
                if (cudaMemsetAsync(D.dtex_bits, 0, sizeof(unsigned), m->st) != cudaSuccess) st = LOC_ECUDA;
                else st = launch_dtex(D, m->sub_x0, m->st);
            }
            nvtxRangePop();
            if (st != LOC_OK) break;
        }
        if (mark(b + 4) != cudaSuccess) { st = LOC_ECUDA; break; }
        if (o->tol_tex > 0.0 || it == o->max_iter - 1) {
            unsigned bits = 0;
            if (cudaMemcpyAsync(&bits, D.dtex_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
                cudaStreamSynchronize(m->st) != cudaSuccess) {
                set_error("reading the convergence metric failed: %s", cudaGetErrorString(cudaGetLastError()));
                st = LOC_ECUDA;
                break;
            }
            memcpy(&dtex, &bits, sizeof(float));
            if (o->tol_tex > 0.0 && dtex < o->tol_tex) { converged = true; it++; break; }
        }
    }
    nvtxRangePop();
    D.trunc = 0;
    m->sub_k = 0;
    m->sub_mode = 0;
    if (st == LOC_ECUDA && g_err[0] == 0) set_error("CUDA error in the iteration: %s", cudaGetErrorString(cudaGetLastError()));
    cudaEventRecord(e1, m->st);
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    double t_par = 0.0, t_mar = 0.0, t_se = 0.0;
    if (prof && st == LOC_OK && ce == cudaSuccess) {
        // sub-iterations (line parameters, march and solve of the region)
        // count as march time
        for (size_t b = 0; b + 4 < ev.size() && b / 5 < (size_t)it; b += 5) {
            float a = 0.f, c = 0.f, d = 0.f, e = 0.f;
            cudaEventElapsedTime(&a, ev[b], ev[b + 1]);
            cudaEventElapsedTime(&c, ev[b + 1], ev[b + 2]);
            cudaEventElapsedTime(&d, ev[b + 2], ev[b + 3]);
            cudaEventElapsedTime(&e, ev[b + 3], ev[b + 4]);
            t_par += a; t_mar += c + e; t_se += d;
        }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LOC_OK) return st;
    if (ce != cudaSuccess) { set_error("iteration failed: %s", cudaGetErrorString(ce)); return LOC_ECUDA; }
    TRY(octree_status(m));
    if (r) {
        memset(r, 0, sizeof(*r));
        r->iterations = it;
        r->max_rel_dtex = dtex;
        r->segments = m->segs_per_sim;
        r->updates = (double)m->segs_per_sim * D.n_ch * D.T * it;
        r->kernel_ms = ms;
        unsigned long long mc = 0, uc = 0, nc = 0;
        cudaMemcpy(&mc, D.maser_count, sizeof(mc), cudaMemcpyDeviceToHost);
        cudaMemcpy(&uc, D.upd_count, sizeof(uc), cudaMemcpyDeviceToHost);
        cudaMemcpy(&nc, D.nom_count, sizeof(nc), cudaMemcpyDeviceToHost);
        r->n_maser_cells = (int64_t)mc;
        r->path_records = m->path_records;
        r->coll_table = D.coll_rates ? 1 : 0;
        if (prof) {
            r->march_ms = t_mar;
            r->se_ms = t_se;
            r->params_ms = t_par;
            r->march_launches = (int64_t)it;
            r->computed_updates = (double)uc;
            r->nominal_updates = (double)nc;
        }
    }
    if (o->tol_tex > 0.0 && !converged) {
        set_error("not converged: max |dTex/Tex| = %g after %d iterations", dtex, it);
        return LOC_ENOTCONV;
    }
    return LOC_OK;
}

loc_status loc_get_radiation(const loc_model *m, double *sij, double *esc, double *norm,
                             size_t n_lc, size_t n_c)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    if (!m->has_rad) { set_error("no ray simulation has run"); return LOC_ESTATE; }
    const DevModel &D = m->d;
    const size_t nlc = (size_t)D.T * D.n_cells;
    if ((sij || esc) && n_lc < nlc) { set_error("sij/esc buffers need %zu elements", nlc); return LOC_EINVAL; }
    if (norm && n_c < (size_t)D.n_cells) { set_error("norm buffer needs %lld elements", D.n_cells); return LOC_EINVAL; }
    double *buf = nullptr;
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(double) * (2 * nlc + D.n_cells)));
    loc_status s = launch_acc_to_f64(D, m->last_fp64, buf, buf + nlc, buf + 2 * nlc, m->st);
    if (s == LOC_OK) {
        cudaError_t e = cudaSuccess;
        if (sij) e = cudaMemcpyAsync(sij, buf, sizeof(double) * nlc, cudaMemcpyDeviceToHost, m->st);
        if (esc && e == cudaSuccess) e = cudaMemcpyAsync(esc, buf + nlc, sizeof(double) * nlc, cudaMemcpyDeviceToHost, m->st);
        if (norm && e == cudaSuccess) e = cudaMemcpyAsync(norm, buf + 2 * nlc, sizeof(double) * D.n_cells, cudaMemcpyDeviceToHost, m->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
        if (e != cudaSuccess) { set_error("copy failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    }
    cudaFree(buf);
    return s;
}

loc_status loc_radiation_buffers(loc_model *m, loc_radiation_buffers_t *out)
{
    if (!m || !out) { set_error("NULL argument"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("loc_set_molecule has not been called"); return LOC_ESTATE; }
    const DevModel &D = m->d;
    memset(out, 0, sizeof(*out));
    out->n_cells = D.n_cells;
    out->n_lines = D.T;
    out->acc = (float *)D.acc;
    out->acc_c = (float *)D.acc_c;
    out->norm = D.norm;
    out->norm_c = D.norm_c;
    out->acc64 = D.acc64;
    out->norm64 = D.norm64;
    return LOC_OK;
}

// The statistical-equilibrium half of an ALI iteration: the solve of every
// cell from the accumulators as they are now (after loc_march, and after
// the caller summed the accumulators of several devices' marches), the
// convergence metric against the populations before, and the new
// populations in place.
loc_status loc_solve(loc_model *m, const loc_iter_opts *o, loc_iter_report *r)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    TRY(check_opts(o));
    if (!m->has_mol) { set_error("loc_set_molecule has not been called"); return LOC_ESTATE; }
    if (!m->has_rad) { set_error("no ray simulation has run"); return LOC_ESTATE; }
    DevModel &D = m->d;
    if ((o->precision == LOC_FP64_ACC) != (m->last_fp64 != 0)) {
        set_error("precision differs from the last ray simulation's");
        return LOC_EINVAL;
    }
    D.trunc = o->level_cutoff > 0.0 ? 1 : 0;
    LOC_CUDA_TRY(cudaMemsetAsync(D.dtex_bits, 0, sizeof(unsigned), m->st));
    loc_status st = launch_se(D, o->ali, o->precision == LOC_FP64_ACC, m->st, 1, 0, o->level_cutoff);
    D.trunc = 0;
    TRY(st);
    std::swap(D.x, D.x_new);
    unsigned bits = 0;
    LOC_CUDA_TRY(cudaMemcpyAsync(&bits, D.dtex_bits, sizeof(unsigned), cudaMemcpyDeviceToHost, m->st));
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    float dtex = 0.f;
    memcpy(&dtex, &bits, sizeof(float));
    if (r) {
        memset(r, 0, sizeof(*r));
        r->iterations = 1;
        r->max_rel_dtex = dtex;
        r->segments = m->segs_per_sim;
        r->path_records = m->path_records;
        r->coll_table = D.coll_rates ? 1 : 0;
    }
    return LOC_OK;
}

loc_status loc_get_populations(const loc_model *m, double *out, size_t n_out)
{
    if (!m || !out) { set_error("NULL argument"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("no molecule"); return LOC_ESTATE; }
    const size_t n = (size_t)m->d.n_cells * m->d.L;
    if (n_out < n) { set_error("output needs %zu elements", n); return LOC_EINVAL; }
    if (!m->d.leaf_perm) {
        LOC_CUDA_TRY(cudaMemcpyAsync(out, m->d.x, sizeof(double) * n, cudaMemcpyDeviceToHost, m->st));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        return LOC_OK;
    }
    double *buf = nullptr;                      // octree: stored order -> level order
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(double) * n));
    loc_status s = launch_permute_rows(m->d.leaf_perm, m->d.n_cells, m->d.L, m->d.x, buf, 1, m->st);
    cudaError_t e = cudaSuccess;
    if (s == LOC_OK) e = cudaMemcpyAsync(out, buf, sizeof(double) * n, cudaMemcpyDeviceToHost, m->st);
    if (s == LOC_OK && e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) { set_error("copy failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    cudaFree(buf);
    return s;
}

loc_status loc_set_populations(loc_model *m, const double *in, size_t n_in)
{
    if (!m || !in) { set_error("NULL argument"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("no molecule"); return LOC_ESTATE; }
    const size_t n = (size_t)m->d.n_cells * m->d.L;
    if (n_in != n) { set_error("populations need exactly %zu elements", n); return LOC_EINVAL; }
    if (!finite_pos(in, (long long)n, true)) { set_error("populations must be finite and >= 0"); return LOC_EINVAL; }
    if (!m->d.leaf_perm) {
        LOC_CUDA_TRY(cudaMemcpyAsync(m->d.x, in, sizeof(double) * n, cudaMemcpyHostToDevice, m->st));
        LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
        m->has_rad = false;
        return LOC_OK;
    }
    double *buf = nullptr;                      // octree: level order -> stored order
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(double) * n));
    loc_status s = LOC_OK;
    cudaError_t e = cudaMemcpyAsync(buf, in, sizeof(double) * n, cudaMemcpyHostToDevice, m->st);
    if (e == cudaSuccess) s = launch_permute_rows(m->d.leaf_perm, m->d.n_cells, m->d.L, buf, m->d.x, 0, m->st);
    if (e == cudaSuccess && s == LOC_OK) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) { set_error("copy failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    cudaFree(buf);
    m->has_rad = false;
    return s;
}

loc_status loc_get_tex(const loc_model *m, int t, double *out, size_t n_out)
{
    if (!m || !out) { set_error("NULL argument"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("no molecule"); return LOC_ESTATE; }
    if (t < 0 || t >= m->d.T) { set_error("line index %d out of range", t); return LOC_EINVAL; }
    if (n_out < (size_t)m->d.n_cells) { set_error("output needs %lld elements", m->d.n_cells); return LOC_EINVAL; }
    double *buf = nullptr;
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(double) * m->d.n_cells));
    loc_status s = launch_tex(m->d, t, buf, m->st);
    if (s == LOC_OK) {
        cudaError_t e = cudaMemcpyAsync(out, buf, sizeof(double) * m->d.n_cells, cudaMemcpyDeviceToHost, m->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
        if (e != cudaSuccess) { set_error("copy failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    }
    cudaFree(buf);
    return s;
}

loc_status loc_spectra(const loc_model *m, int t, const double *p_cm, int n_p, double *T_out,
                       size_t n_out)
{
    if (!m || (!p_cm && n_p > 0) || (!T_out && n_p > 0)) { set_error("NULL argument"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("no molecule"); return LOC_ESTATE; }
    if (m->d.geometry != LOC_SHELLS_1D) { set_error("loc_spectra supports 1D models"); return LOC_EINVAL; }
    if (t < 0 || t >= m->d.T) { set_error("line index %d out of range", t); return LOC_EINVAL; }
    if (n_p < 0) { set_error("n_p must be >= 0"); return LOC_EINVAL; }
    if (n_p == 0) return LOC_OK;
    const size_t n = (size_t)n_p * m->d.n_ch;
    if (n_out < n) { set_error("output needs %zu elements", n); return LOC_EINVAL; }
    for (int i = 0; i < n_p; i++)
        if (!(p_cm[i] >= 0.0) || !std::isfinite(p_cm[i])) { set_error("impact parameter %d invalid", i); return LOC_EINVAL; }
    // temporaries from the model's allocator: impact parameters, per-step
    // records [n_p][2 K], step counts, brightness
    loc_model *mm = const_cast<loc_model *>(m);
    std::vector<void *> tmp_mem;
    double *pd = (double *)dev_alloc(mm, sizeof(double) * n_p, tmp_mem);
    float4 *rec = (float4 *)dev_alloc(mm, sizeof(float4) * (size_t)n_p * 2 * m->d.K, tmp_mem);
    int *nst = (int *)dev_alloc(mm, sizeof(int) * n_p, tmp_mem);
    float *Td = (float *)dev_alloc(mm, sizeof(float) * n, tmp_mem);
    if (!pd || !rec || !nst || !Td) {
        dev_free_all(mm, tmp_mem);
        set_error("allocation of the spectra buffers failed");
        return LOC_ENOMEM;
    }
    std::vector<float> tmp(n);
    loc_status s = LOC_OK;
    cudaError_t e = cudaMemcpyAsync(pd, p_cm, sizeof(double) * n_p, cudaMemcpyHostToDevice, m->st);
    if (e == cudaSuccess) {
        s = launch_line_params(m->d, m->st);
        if (s == LOC_OK) s = launch_spectra1d(m->d, t, pd, n_p, rec, nst, Td, m->st);
        if (s == LOC_OK) {
            e = cudaMemcpyAsync(tmp.data(), Td, sizeof(float) * n, cudaMemcpyDeviceToHost, m->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
        }
    }
    if (e != cudaSuccess) { set_error("spectra failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    if (s == LOC_OK) for (size_t i = 0; i < n; i++) T_out[i] = tmp[i];
    cudaStreamSynchronize(m->st);
    dev_free_all(mm, tmp_mem);
    return s;
}

loc_status loc_map3d(const loc_model *m, int t, int dir, int level, double *T_out, size_t n_out)
{
    if (!m || !T_out) { set_error("NULL argument"); return LOC_EINVAL; }
    if (!m->has_mol) { set_error("no molecule"); return LOC_ESTATE; }
    const DevModel &D = m->d;
    if (D.geometry != LOC_GRID_3D && D.geometry != LOC_OCTREE_3D) { set_error("loc_map3d needs a 3D model"); return LOC_EINVAL; }
    if (t < 0 || t >= D.T) { set_error("line index %d out of range", t); return LOC_EINVAL; }
    if (dir < 0 || dir >= D.n_dir) { set_error("direction index %d out of range [0, %d)", dir, D.n_dir); return LOC_EINVAL; }
    const int lmax = (D.geometry == LOC_OCTREE_3D) ? D.Lmax : 0;
    if (level < 0 || level > lmax) { set_error("map level must be in [0, %d]", lmax); return LOC_EINVAL; }
    const long long Mp = (long long)D.N << level;
    if (Mp * Mp > (1ll << 26)) { set_error("map of %lld^2 pixels exceeds 2^26 pixels", Mp); return LOC_EINVAL; }
    const size_t n = (size_t)(Mp * Mp) * D.n_ch;
    if (n_out < n) { set_error("output needs %zu elements", n); return LOC_EINVAL; }
    loc_model *mm = const_cast<loc_model *>(m);
    std::vector<void *> tmp_mem;
    float *Td = (float *)dev_alloc(mm, sizeof(float) * n, tmp_mem);
    if (!Td) { set_error("allocation of the map buffer failed"); return LOC_ENOMEM; }
    std::vector<float> tmp;
    try { tmp.resize(n); } catch (...) { dev_free_all(mm, tmp_mem); set_error("host allocation failed"); return LOC_ENOMEM; }
    loc_status s = launch_line_params(D, m->st);
    if (s == LOC_OK) s = (D.geometry == LOC_GRID_3D) ? launch_map_grid3d(D, t, dir, Td, m->st)
                                                     : launch_map_octree(D, t, dir, level, Td, m->st);
    cudaError_t e = cudaSuccess;
    if (s == LOC_OK) {
        e = cudaMemcpyAsync(tmp.data(), Td, sizeof(float) * n, cudaMemcpyDeviceToHost, m->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
        if (e != cudaSuccess) { set_error("map failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    }
    if (s == LOC_OK) for (size_t i = 0; i < n; i++) T_out[i] = tmp[i];
    cudaStreamSynchronize(m->st);
    dev_free_all(mm, tmp_mem);
    return s;
}

loc_status loc_model_info(const loc_model *m, int64_t *n_cells, int *n_levels, int *n_lines,
                          int64_t *segments_per_sim)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    if (n_cells) *n_cells = m->d.n_cells;
    if (n_levels) *n_levels = m->has_mol ? m->d.L : 0;
    if (n_lines) *n_lines = m->has_mol ? m->d.T : 0;
    if (segments_per_sim) *segments_per_sim = m->segs_per_sim;
    return LOC_OK;
}

loc_status loc_trace_ray(const loc_model *m, int dir, int64_t i, int64_t j, int64_t *cells,
                         int64_t *dz, int64_t cap, int64_t *n_seg)
{
    if (!m || !n_seg) { set_error("NULL argument"); return LOC_EINVAL; }
    if (m->d.geometry != LOC_GRID_3D) { set_error("loc_trace_ray needs a 3D grid model"); return LOC_EINVAL; }
    if (dir < 0 || dir >= m->d.n_dir) { set_error("direction %d out of range", dir); return LOC_EINVAL; }
    if (i < 0 || j < 0 || i >= m->d.N || j >= m->d.N) { set_error("root line out of range"); return LOC_EINVAL; }
    if (cap < 0 || (cap > 0 && (!cells || !dz))) { set_error("bad output buffers"); return LOC_EINVAL; }
    long long *buf = nullptr;
    const long long dcap = cap > 0 ? cap : 1;
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(long long) * (2 * dcap + 1)));
    loc_status s = launch_trace3d(m->d, dir, i, j, buf, buf + dcap, dcap, buf + 2 * dcap, m->st);
    long long n = 0;
    if (s == LOC_OK) {
        cudaError_t e = cudaMemcpyAsync(&n, buf + 2 * dcap, sizeof(long long), cudaMemcpyDeviceToHost, m->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
        if (e != cudaSuccess) { set_error("trace failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    }
    if (s == LOC_OK) {
        *n_seg = n;
        if (n > cap) {
            set_error("ray has %lld segments, capacity %lld", n, (long long)cap);
            s = LOC_EINVAL;
        } else if (n > 0) {
            cudaError_t e = cudaMemcpy(cells, buf, sizeof(long long) * n, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(dz, buf + dcap, sizeof(long long) * n, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { set_error("copy failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
        }
    }
    cudaFree(buf);
    return s;
}

loc_status loc_trace_octree(const loc_model *mc, int dir, int64_t *out7, int64_t cap, int64_t *n_seg)
{
    loc_model *m = (loc_model *)mc;
    if (!m || !n_seg) { set_error("NULL argument"); return LOC_EINVAL; }
    if (m->d.geometry != LOC_OCTREE_3D) { set_error("loc_trace_octree needs an octree model"); return LOC_EINVAL; }
    if (dir < 0 || dir >= m->d.n_dir) { set_error("direction %d out of range", dir); return LOC_EINVAL; }
    if (cap < 0 || (cap > 0 && !out7)) { set_error("bad output buffer"); return LOC_EINVAL; }
    long long *buf = nullptr;
    unsigned long long *cnt = nullptr;
    const long long dcap = cap > 0 ? cap : 1;
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(long long) * 7 * dcap));
    if (cudaMalloc(&cnt, sizeof(unsigned long long)) != cudaSuccess) { cudaFree(buf); set_error("allocation failed"); return LOC_ENOMEM; }
    loc_status s = launch_trace_octree(m->d, dir, buf, cap, cnt, m->st);
    unsigned long long n = 0;
    if (s == LOC_OK) {
        cudaError_t e = cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, m->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
        if (e != cudaSuccess) { set_error("trace failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    }
    if (s == LOC_OK) s = octree_status(m);
    if (s == LOC_OK) {
        *n_seg = (int64_t)n;
        const long long w = ((long long)n < cap) ? (long long)n : cap;
        if (w > 0) {
            const cudaError_t e = cudaMemcpy(out7, buf, sizeof(long long) * 7 * w, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { set_error("copy failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
            else for (long long k = 0; k < w; k++) out7[7 * k + 5] = m->leaf_api[out7[7 * k + 5]];
        }
    }
    cudaFree(buf);
    cudaFree(cnt);
    return s;
}

loc_status loc_octree_path_sums(const loc_model *mc, int dir, int64_t *out, size_t n_out)
{
    loc_model *m = (loc_model *)mc;
    if (!m || !out) { set_error("NULL argument"); return LOC_EINVAL; }
    if (m->d.geometry != LOC_OCTREE_3D) { set_error("loc_octree_path_sums needs an octree model"); return LOC_EINVAL; }
    if (dir < 0 || dir >= m->d.n_dir) { set_error("direction %d out of range", dir); return LOC_EINVAL; }
    if (n_out < (size_t)m->d.n_cells) { set_error("output needs %lld elements", m->d.n_cells); return LOC_EINVAL; }
    unsigned long long *buf = nullptr;
    LOC_CUDA_TRY(cudaMalloc(&buf, sizeof(unsigned long long) * (m->d.n_cells + 1)));
    loc_status s = LOC_OK;
    cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(unsigned long long) * (m->d.n_cells + 1), m->st);
    if (e == cudaSuccess) s = launch_trace_octree(m->d, dir, nullptr, 0, buf + m->d.n_cells, m->st, buf);
    if (e == cudaSuccess && s == LOC_OK) e = cudaMemcpyAsync(out, buf, sizeof(int64_t) * m->d.n_cells, cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess && s == LOC_OK) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) { set_error("path sums failed: %s", cudaGetErrorString(e)); s = LOC_ECUDA; }
    cudaFree(buf);
    if (s == LOC_OK) s = octree_status(m);
    if (s == LOC_OK) {                          // stored order -> level order
        std::vector<int64_t> tmp(out, out + m->d.n_cells);
        for (long long i = 0; i < m->d.n_cells; i++) out[m->leaf_api[i]] = tmp[i];
    }
    return s;
}

loc_status loc_sync(loc_model *m)
{
    if (!m) { set_error("NULL model"); return LOC_EINVAL; }
    LOC_CUDA_TRY(cudaStreamSynchronize(m->st));
    return LOC_OK;
}

void loc_destroy(loc_model *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->st);
    dev_free_all(m, m->oct_mem);
    dev_free_all(m, m->path_mem);
    dev_free_all(m, m->tmp_mem);
    dev_free_all(m, m->sub_mem);
    dev_free_all(m, m->run_mem);
    dev_free_all(m, m->run_ab_mem);
    dev_free_all(m, m->mol_mem);
    dev_free_all(m, m->geo_mem);
    delete m;
}

}  // extern "C"
