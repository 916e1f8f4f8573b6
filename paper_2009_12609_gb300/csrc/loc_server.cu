// loc_server.cu -- continuous-batching server for 1D models (the inverse-
// problem use of the method: many small spherical models solved to
// convergence, Sect. 1 and 2.1).
//
// A host thread owns one CUDA stream and a table of slots.  Each round it
//   1. admits queued requests while a slot is free and the device-memory
//      budget allows (per request: one arena allocation holding the model,
//      molecule, ray steps, populations and accumulators; set-up kernels
//      build the ray geometry and LTE populations on the device);
//   2. rebuilds the work tables when the composition changed ((slot, ray,
//      line group) items ordered longest ray first, (slot, cell) items);
//   3. launches one CUDA graph holding k ALI iterations of every active slot
//      (k_batch.cu); slots that converge stop inside the graph;
//   4. reads the per-slot done flags, copies finished populations to host
//      result buffers, frees their arenas and wakes the pollers.
// Populations stay on the device for the whole solve; requests that arrive
// while others run join at the next round boundary.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <new>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "k_batch.cuh"

using Clock = std::chrono::steady_clock;

namespace loc {

static size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

// Arena layout of one admitted model; offsets in bytes.
struct ArenaLayout {
    size_t n_h2, t_kin, abundance, sigma, radius, v1d, energy, g, line_u, line_l, line_A, line_nu,
        coll_u, coll_l, coll_k;       // uploaded inputs (contiguous prefix)
    size_t inputs_end;
    size_t inv, ray_off, segs, tan, W, nbg, nbg64, x, x_new, ks, acc, norm, acc_c, norm_c, dtex, maser, upd, coll;
    size_t total;
};

struct Request {
    uint64_t ticket = 0;
    int K = 0, n_rays = 0, n_ch = 0;
    double ray_power = 1.0;
    double v_min = 0, dv = 0, t_bg = 0;
    int L = 0, T = 0, P = 0;
    double mass = 0;
    int max_iter = 1, ali = 1;
    double cutoff = 0.0;
    float tol = 0.f;
    ArenaLayout lay{};
    std::vector<unsigned char> staged;   // inputs in arena order
    long long steps_per_sim = 0;
    Clock::time_point t_submit;
};

struct Finished {
    loc_result r{};
    std::vector<double> pops;
};

struct SlotHost {
    bool used = false;
    Request *req = nullptr;
    void *arena = nullptr;
    int cls = 0;
    int per = 1, n_groups = 1;
    std::vector<int> ray_steps;
};

static ArenaLayout layout_for(const Request &q)
{
    ArenaLayout a{};
    size_t o = 0;
    auto put = [&](size_t bytes) { const size_t r = o; o += al256(bytes); return r; };
    const size_t K = q.K, L = q.L, T = q.T, P = q.P, R = q.n_rays;
    a.n_h2 = put(8 * K); a.t_kin = put(8 * K); a.abundance = put(8 * K); a.sigma = put(8 * K);
    a.radius = put(8 * K); a.v1d = put(4 * K);
    a.energy = put(8 * L); a.g = put(8 * L);
    a.line_u = put(4 * T); a.line_l = put(4 * T); a.line_A = put(8 * T); a.line_nu = put(8 * T);
    a.coll_u = put(4 * (P ? P : 1)); a.coll_l = put(4 * (P ? P : 1)); a.coll_k = put(8 * (P ? P : 1));
    a.inputs_end = o;
    a.inv = put(4 * K); a.ray_off = put(4 * (R + 1)); a.segs = put(sizeof(Seg1D) * 2 * R * (K + 1));
    a.tan = put(4 * R); a.W = put(8 * K); a.nbg = put(4 * T); a.nbg64 = put(8 * T);
    a.x = put(8 * K * L); a.x_new = put(8 * K * L); a.ks = put(8 * K * T); a.acc = put(8 * K * T);
    a.norm = put(4 * K); a.acc_c = put(8 * K * T); a.norm_c = put(4 * K);
    a.dtex = put(4); a.maser = put(8); a.upd = put(8);
    a.coll = put(16 * K * (P ? P : 1));   // collision rates per cell and pair, tabulated once
    a.total = o;
    return a;
}

}  // namespace loc

using namespace loc;

struct loc_server {
    loc_server_opts opt{};
    int device = 0;
    cudaStream_t st = nullptr;
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Finished> done;
    std::atomic<uint64_t> next_ticket{1};
    bool stop = false;
    loc_status fatal = LOC_OK;
    char fatal_msg[512] = "";

    // device state
    std::vector<SlotHost> slots;
    BatchSlot *slots_d = nullptr;
    int *done_d = nullptr, *done_h = nullptr;
    int4 *items_d[kBatchClasses] = {};
    size_t items_cap[kBatchClasses] = {};
    int2 *cells_d = nullptr;
    size_t cells_cap = 0;
    int *counts_d = nullptr;       // [kBatchClasses + 1]
    unsigned *counters_d = nullptr;
    int *counts_h = nullptr;       // pinned staging of the counts
    cudaGraphExec_t graph = nullptr;
    bool need_capture = true;
    cudaStream_t side[kBatchClasses] = {};
    cudaEvent_t fork = nullptr, join[kBatchClasses] = {};
    int n_sm = 152;
    size_t mem_used = 0;

    // stats
    int64_t submitted = 0, completed = 0;
    std::vector<double> latencies_ms;
    Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;
};

static void server_fail(loc_server *s, loc_status st, const char *msg)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal == LOC_OK) {
        s->fatal = st;
        snprintf(s->fatal_msg, sizeof(s->fatal_msg), "%s", msg);
    }
    s->stop = true;
    s->cv_done.notify_all();
}

// device memory for the work tables; growth forces a new graph capture
static bool ensure_tables(loc_server *s, const size_t need_items[kBatchClasses], size_t need_cells)
{
    for (int c = 0; c < kBatchClasses; c++) {
        if (need_items[c] <= s->items_cap[c] && s->items_d[c]) continue;
        size_t cap = std::max<size_t>(1024, s->items_cap[c]);
        while (cap < need_items[c]) cap *= 2;
        if (s->items_d[c]) cudaFreeAsync(s->items_d[c], s->st);
        if (cudaMallocAsync(&s->items_d[c], sizeof(int4) * cap, s->st) != cudaSuccess) return false;
        s->items_cap[c] = cap;
        s->need_capture = true;
    }
    if (!(need_cells <= s->cells_cap && s->cells_d)) {
        size_t cap = std::max<size_t>(4096, s->cells_cap);
        while (cap < need_cells) cap *= 2;
        if (s->cells_d) cudaFreeAsync(s->cells_d, s->st);
        if (cudaMallocAsync(&s->cells_d, sizeof(int2) * cap, s->st) != cudaSuccess) return false;
        s->cells_cap = cap;
        s->need_capture = true;
    }
    return true;
}

static bool rebuild_tables(loc_server *s)
{
    std::vector<int4> items[kBatchClasses];
    std::vector<int2> cells;
    for (int si = 0; si < (int)s->slots.size(); si++) {
        const SlotHost &h = s->slots[si];
        if (!h.used) continue;
        for (int j = 0; j < h.req->n_rays; j++)
            for (int g = 0; g < h.n_groups; g++)
                items[h.cls].push_back(make_int4(si, j, g, h.ray_steps[j]));
        for (int c = 0; c < h.req->K; c++) cells.push_back(make_int2(si, c));
    }
    size_t need[kBatchClasses];
    for (int c = 0; c < kBatchClasses; c++) {
        // longest rays first (counting sort on the step count, descending)
        std::stable_sort(items[c].begin(), items[c].end(),
                         [](const int4 &a, const int4 &b) { return a.w > b.w; });
        need[c] = items[c].size();
    }
    if (!ensure_tables(s, need, cells.size())) return false;
    for (int c = 0; c < kBatchClasses; c++) {
        s->counts_h[c] = (int)items[c].size();
        if (!items[c].empty() &&
            cudaMemcpyAsync(s->items_d[c], items[c].data(), sizeof(int4) * items[c].size(),
                            cudaMemcpyHostToDevice, s->st) != cudaSuccess)
            return false;
    }
    s->counts_h[kBatchClasses] = (int)cells.size();
    if (!cells.empty() &&
        cudaMemcpyAsync(s->cells_d, cells.data(), sizeof(int2) * cells.size(), cudaMemcpyHostToDevice,
                        s->st) != cudaSuccess)
        return false;
    if (cudaMemcpyAsync(s->counts_d, s->counts_h, sizeof(int) * (kBatchClasses + 1),
                        cudaMemcpyHostToDevice, s->st) != cudaSuccess)
        return false;
    // pageable sources: wait before the vectors go out of scope
    return cudaStreamSynchronize(s->st) == cudaSuccess;
}

static bool capture_graph(loc_server *s)
{
    if (s->graph) { cudaGraphExecDestroy(s->graph); s->graph = nullptr; }
    BatchLaunch b{};
    b.slots = s->slots_d;
    b.n_slots = (int)s->slots.size();
    for (int c = 0; c < kBatchClasses; c++) b.items[c] = s->items_d[c];
    b.n_items = s->counts_d;
    b.cells = s->cells_d;
    b.n_cells = s->counts_d + kBatchClasses;
    b.counters = s->counters_d;
    b.done_out = s->done_d;
    b.window = (float)s->opt.window_sigmas;
    b.n_sm = s->n_sm;
    b.blocks_per_sm = 4;
    for (int c = 0; c < kBatchClasses; c++) { b.side[c] = s->side[c]; b.join[c] = s->join[c]; }
    b.fork = s->fork;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    bool ok = true;
    for (int k = 0; k < s->opt.iters_per_launch && ok; k++) ok = batch_launch_iteration(b, s->st) == LOC_OK;
    const cudaError_t e = cudaStreamEndCapture(s->st, &g);
    if (!ok || e != cudaSuccess) { if (g) cudaGraphDestroy(g); return false; }
    const cudaError_t ei = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return false;
    s->need_capture = false;
    return true;
}

// upload a request into a free slot; returns false on a CUDA error
static bool admit(loc_server *s, int si, Request *q)
{
    SlotHost &h = s->slots[si];
    void *arena = nullptr;
    if (cudaMallocAsync(&arena, q->lay.total, s->st) != cudaSuccess) return false;
    unsigned char *b = (unsigned char *)arena;
    if (cudaMemcpyAsync(b, q->staged.data(), q->lay.inputs_end, cudaMemcpyHostToDevice, s->st) != cudaSuccess)
        return false;
    const ArenaLayout &a = q->lay;
    BatchSlot bs;
    memset(&bs, 0, sizeof(bs));
    DevModel &m = bs.m;
    m.geometry = LOC_SHELLS_1D;
    m.n_cells = q->K;
    m.n_ch = q->n_ch;
    m.v_min = q->v_min;
    m.dv = q->dv;
    m.vmin_f = (float)q->v_min;
    m.dv_f = (float)q->dv;
    m.t_bg = q->t_bg;
    m.n_h2 = (double *)(b + a.n_h2);
    m.t_kin = (double *)(b + a.t_kin);
    m.abundance = (double *)(b + a.abundance);
    m.inv_s2sig = (float *)(b + a.inv);
    m.K = q->K;
    m.n_rays = q->n_rays;
    m.ray_power = q->ray_power;
    m.trunc = q->cutoff > 0.0 ? 1 : 0;
    m.radius = (double *)(b + a.radius);
    m.v1d = (float *)(b + a.v1d);
    m.ray_off = (int *)(b + a.ray_off);
    m.segs = (Seg1D *)(b + a.segs);
    m.L = q->L;
    m.T = q->T;
    m.P = q->P;
    m.mass_amu = q->mass;
    m.energy_K = (double *)(b + a.energy);
    m.g = (double *)(b + a.g);
    m.line_u = (int *)(b + a.line_u);
    m.line_l = (int *)(b + a.line_l);
    m.line_A = (double *)(b + a.line_A);
    m.line_nu = (double *)(b + a.line_nu);
    m.coll_u = (int *)(b + a.coll_u);
    m.coll_l = (int *)(b + a.coll_l);
    m.coll_k = (double *)(b + a.coll_k);
    m.nbg = (float *)(b + a.nbg);
    m.nbg64 = (double *)(b + a.nbg64);
    m.x = (double *)(b + a.x);
    m.x_new = (double *)(b + a.x_new);
    m.ks = (float2 *)(b + a.ks);
    m.acc = (float2 *)(b + a.acc);
    m.norm = (float *)(b + a.norm);
    m.acc_c = (float2 *)(b + a.acc_c);
    m.norm_c = (float *)(b + a.norm_c);
    m.dtex_bits = (unsigned *)(b + a.dtex);
    m.maser_count = (unsigned long long *)(b + a.maser);
    m.upd_count = (unsigned long long *)(b + a.upd);
    m.coll_rates = q->P > 0 ? (double2 *)(b + a.coll) : nullptr;
    if (cudaMemsetAsync(m.dtex_bits, 0, 4, s->st) != cudaSuccess) return false;
    if (launch_geom1d_scratch(m, s->st, (int *)(b + a.tan), (double *)(b + a.W)) != LOC_OK) return false;
    if (launch_cell_setup(m, (const double *)(b + a.sigma), nullptr, nullptr, nullptr, s->st) != LOC_OK) return false;
    if (m.coll_rates && launch_coll_rates(m, m.coll_rates, s->st) != LOC_OK) return false;
    if (launch_bg(m, s->st) != LOC_OK) return false;
    if (launch_lte(m, s->st) != LOC_OK) return false;
    // lines per warp: per x n_ch <= 2048 floats of shared memory, rounded
    // down to a compiled group size
    int per_max = std::min(q->T, std::min(15, std::max(1, kBatchLineFloats / q->n_ch)));
    int cls = 0;
    while (cls + 1 < kBatchClasses && kBatchClassG[cls + 1] <= per_max) cls++;
    const int per = kBatchClassG[cls];
    bs.active = 1;
    bs.done = 0;
    bs.iter = 0;
    bs.max_iter = q->max_iter;
    bs.tol = q->tol;
    bs.ali = q->ali;
    bs.per = per;
    bs.n_groups = (q->T + per - 1) / per;
    bs.inv_dv = (float)(1.0 / q->dv);
    bs.cutoff = q->cutoff;
    if (cudaMemcpyAsync(s->slots_d + si, &bs, sizeof(bs), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
        return false;
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return false;    // bs leaves scope
    h.used = true;
    h.req = q;
    h.arena = arena;
    h.cls = cls;
    h.per = per;
    h.n_groups = bs.n_groups;
    // step counts of the equidistant rays (ordering of the work items)
    h.ray_steps.assign(q->n_rays, 0);
    const double *R = (const double *)(q->staged.data() + a.radius);
    const double Rout = R[q->K - 1];
    long long tot = 0;
    for (int j = 0; j < q->n_rays; j++) {
        const double p = (q->ray_power == 1.0) ? (j + 0.5) * Rout / q->n_rays
                                               : Rout * std::pow((j + 0.5) / q->n_rays, q->ray_power);
        const int t = (int)(std::upper_bound(R, R + q->K, p) - R);
        h.ray_steps[j] = (t < q->K) ? 2 * (q->K - t) : 0;
        tot += h.ray_steps[j];
    }
    q->steps_per_sim = tot;
    return true;
}

static bool retire(loc_server *s, int si)
{
    SlotHost &h = s->slots[si];
    BatchSlot bs;
    if (cudaMemcpyAsync(&bs, s->slots_d + si, sizeof(bs), cudaMemcpyDeviceToHost, s->st) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return false;
    Finished f;
    const Request *q = h.req;
    f.pops.resize((size_t)q->K * q->L);
    if (cudaMemcpyAsync(f.pops.data(), bs.m.x, sizeof(double) * f.pops.size(), cudaMemcpyDeviceToHost, s->st) != cudaSuccess)
        return false;
    BatchSlot zero;
    memset(&zero, 0, sizeof(zero));
    if (cudaMemcpyAsync(s->slots_d + si, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->st) != cudaSuccess) return false;
    if (cudaFreeAsync(h.arena, s->st) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return false;
    const auto now = Clock::now();
    f.r.ticket = q->ticket;
    f.r.status = (q->tol > 0.f && !(bs.last_dtex < q->tol)) ? LOC_ENOTCONV : LOC_OK;
    f.r.iterations = bs.iter;
    f.r.max_rel_dtex = bs.last_dtex;
    f.r.latency_ms = std::chrono::duration<double, std::milli>(now - q->t_submit).count();
    f.r.n_cells = q->K;
    f.r.n_levels = q->L;
    f.r.updates = (double)q->steps_per_sim * q->n_ch * q->T * bs.iter;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->mem_used -= q->lay.total;
        s->completed++;
        s->latencies_ms.push_back(f.r.latency_ms);
        s->t_last_done = now;
        s->done[q->ticket] = std::move(f);
    }
    delete h.req;
    h = SlotHost();
    s->cv_done.notify_all();
    return true;
}

static void server_loop(loc_server *s)
{
    if (cudaSetDevice(s->device) != cudaSuccess) { server_fail(s, LOC_ECUDA, "cudaSetDevice failed"); return; }
    bool changed = false;
    while (true) {
        // 1. admission
        std::vector<std::pair<int, Request *>> admits;
        int active = 0;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) break;
            for (auto &h : s->slots) active += h.used;
            if (active == 0 && s->pending.empty()) {
                s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            int free_slot = 0;
            while (!s->pending.empty()) {
                while (free_slot < (int)s->slots.size() &&
                       (s->slots[free_slot].used ||
                        std::any_of(admits.begin(), admits.end(), [&](auto &p) { return p.first == free_slot; })))
                    free_slot++;
                if (free_slot >= (int)s->slots.size()) break;
                Request *q = s->pending.front();
                if (s->mem_used + q->lay.total > s->opt.mem_budget_bytes && (active + (int)admits.size()) > 0) break;
                s->pending.pop_front();
                s->mem_used += q->lay.total;
                admits.emplace_back(free_slot, q);
            }
        }
        for (auto &p : admits) {
            if (!admit(s, p.first, p.second)) {
                server_fail(s, LOC_ECUDA, "admission failed (device allocation or set-up kernel)");
                return;
            }
            changed = true;
        }
        active = 0;
        for (auto &h : s->slots) active += h.used;
        if (active == 0) continue;
        // 2. tables and graph
        if (changed) {
            if (!rebuild_tables(s)) { server_fail(s, LOC_ECUDA, "work-table upload failed"); return; }
            changed = false;
        }
        if (s->need_capture && !capture_graph(s)) { server_fail(s, LOC_ECUDA, "graph capture failed"); return; }
        // 3. k iterations of every active slot
        nvtxRangePushA("server round");
        const bool round_ok = cudaGraphLaunch(s->graph, s->st) == cudaSuccess;
        nvtxRangePop();
        if (!round_ok ||
            cudaMemcpyAsync(s->done_h, s->done_d, sizeof(int) * s->slots.size(), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
            cudaStreamSynchronize(s->st) != cudaSuccess) {
            char msg[256];
            snprintf(msg, sizeof(msg), "batched iteration failed: %s", cudaGetErrorString(cudaGetLastError()));
            server_fail(s, LOC_ECUDA, msg);
            return;
        }
        // 4. retirement
        for (int si = 0; si < (int)s->slots.size(); si++) {
            if (!s->slots[si].used || !s->done_h[si]) continue;
            if (!retire(s, si)) { server_fail(s, LOC_ECUDA, "retirement copy failed"); return; }
            changed = true;
        }
    }
}

extern "C" {

loc_status loc_server_create(loc_server **out, const loc_server_opts *o)
{
    if (!out || !o) { set_error("NULL argument"); return LOC_EINVAL; }
    *out = nullptr;
    if (o->max_slots < 1 || o->max_slots > 65536) { set_error("max_slots must be in [1, 65536]"); return LOC_EINVAL; }
    if (o->iters_per_launch < 1 || o->iters_per_launch > 64) { set_error("iters_per_launch must be in [1, 64]"); return LOC_EINVAL; }
    if (!(o->window_sigmas >= 0.0)) { set_error("window_sigmas must be >= 0"); return LOC_EINVAL; }
    if (o->mem_budget_bytes == 0) { set_error("mem_budget_bytes must be > 0"); return LOC_EINVAL; }
    loc_server *s = new (std::nothrow) loc_server();
    if (!s) { set_error("host allocation failed"); return LOC_ENOMEM; }
    s->opt = *o;
    s->device = o->device;
    s->slots.resize(o->max_slots);
    auto fail = [&](const char *what) {
        set_error("loc_server_create: %s: %s", what, cudaGetErrorString(cudaGetLastError()));
        if (s->st) cudaStreamDestroy(s->st);
        delete s;
        return LOC_ECUDA;
    };
    if (cudaSetDevice(s->device) != cudaSuccess) return fail("cudaSetDevice");
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess && nsm > 0) s->n_sm = nsm;
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) return fail("stream");
    if (batch_prepare() != LOC_OK) return fail("kernel attributes");
    for (int c = 0; c < kBatchClasses; c++) {
        if (cudaStreamCreateWithFlags(&s->side[c], cudaStreamNonBlocking) != cudaSuccess) return fail("stream");
        if (cudaEventCreateWithFlags(&s->join[c], cudaEventDisableTiming) != cudaSuccess) return fail("event");
    }
    if (cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess) return fail("event");
    if (cudaMalloc(&s->slots_d, sizeof(BatchSlot) * o->max_slots) != cudaSuccess) return fail("slot table");
    if (cudaMemset(s->slots_d, 0, sizeof(BatchSlot) * o->max_slots) != cudaSuccess) return fail("slot table");
    if (cudaMalloc(&s->done_d, sizeof(int) * o->max_slots) != cudaSuccess) return fail("flags");
    if (cudaMemset(s->done_d, 0, sizeof(int) * o->max_slots) != cudaSuccess) return fail("flags");
    if (cudaMallocHost(&s->done_h, sizeof(int) * o->max_slots) != cudaSuccess) return fail("flags");
    if (cudaMalloc(&s->counts_d, sizeof(int) * (kBatchClasses + 1)) != cudaSuccess) return fail("counts");
    if (cudaMemset(s->counts_d, 0, sizeof(int) * (kBatchClasses + 1)) != cudaSuccess) return fail("counts");
    if (cudaMallocHost(&s->counts_h, sizeof(int) * (kBatchClasses + 1)) != cudaSuccess) return fail("counts");
    if (cudaMalloc(&s->counters_d, sizeof(unsigned) * kBatchCounters) != cudaSuccess) return fail("counters");
    s->thr = std::thread(server_loop, s);
    *out = s;
    return LOC_OK;
}

loc_status loc_server_submit(loc_server *s, const loc_model_desc *d, const loc_molecule_desc *mol,
                             const loc_iter_opts *o, uint64_t *ticket)
{
    if (!s || !d || !mol || !o || !ticket) { set_error("NULL argument"); return LOC_EINVAL; }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != LOC_OK) { set_error("server stopped: %s", s->fatal_msg); return s->fatal; }
        if (s->stop) { set_error("server is shutting down"); return LOC_ESTATE; }
        if (s->opt.max_queue > 0 && (int)s->pending.size() >= s->opt.max_queue) {
            set_error("queue full (%d requests)", s->opt.max_queue);
            return LOC_EBUSY;
        }
    }
    if (d->geometry != LOC_SHELLS_1D) { set_error("the server takes 1D models"); return LOC_EINVAL; }
    if (mol->hf_n) {
        for (int t = 0; t < mol->n_lines; t++)
            if (mol->hf_n[t] != 0) { set_error("the server takes lines without hyperfine structure"); return LOC_EINVAL; }
    }
    const int K = d->n_shells;
    if (K < 1 || K > 4096 || !d->radius || !d->v || !d->n_h2 || !d->t_kin || !d->sigma_turb || !d->abundance) {
        set_error("1D model: need 1 <= n_shells <= 4096 and all per-shell arrays");
        return LOC_EINVAL;
    }
    for (int k = 0; k < K; k++) {
        if (!(d->radius[k] > 0.0) || (k && !(d->radius[k] > d->radius[k - 1])) || !(d->t_kin[k] > 0.0) ||
            !(d->n_h2[k] >= 0.0) || !(d->abundance[k] >= 0.0) || !(d->sigma_turb[k] >= 0.0) ||
            !std::isfinite(d->v[k]) || !std::isfinite(d->n_h2[k])) {
            set_error("1D model: invalid values at shell %d", k);
            return LOC_EINVAL;
        }
    }
    const int n_rays = d->n_rays > 0 ? d->n_rays : K;
    if (n_rays > 4096 || d->n_ch < 1 || d->n_ch > kMaxChannels || !(d->dv > 0.0) ||
        !(d->ray_power == 0.0 || (d->ray_power > 0.0 && d->ray_power <= 10.0))) {
        set_error("1D model: bad ray count or channel grid");
        return LOC_EINVAL;
    }
    const int L = mol->n_levels, T = mol->n_lines, P = mol->n_coll;
    if (L < 2 || L > 32 || T < 1 || T > 31 || P < 0 || P > 496 || T + P > kBatchMaxRates || !mol->energy_K ||
        !mol->g || !mol->line_u || !mol->line_l || !mol->line_A || !mol->line_nu ||
        (P && (!mol->coll_u || !mol->coll_l || !mol->coll_k)) || !(mol->mass_amu > 0.0)) {
        set_error("molecule: need 2 <= levels <= 32, 1 <= lines <= 31, pairs <= 496 and all arrays");
        return LOC_EINVAL;
    }
    for (int t = 0; t < T; t++)
        if (mol->line_u[t] < 0 || mol->line_u[t] >= L || mol->line_l[t] < 0 || mol->line_l[t] >= L ||
            mol->line_u[t] == mol->line_l[t] || !(mol->line_nu[t] > 0.0) || !(mol->line_A[t] >= 0.0)) {
            set_error("molecule: bad line %d", t);
            return LOC_EINVAL;
        }
    for (int p = 0; p < P; p++)
        if (mol->coll_u[p] < 0 || mol->coll_u[p] >= L || mol->coll_l[p] < 0 || mol->coll_l[p] >= L ||
            mol->coll_u[p] == mol->coll_l[p] || !(mol->coll_k[p] >= 0.0)) {
            set_error("molecule: bad collision pair %d", p);
            return LOC_EINVAL;
        }
    if (!distinct_level_pairs(mol->line_u, mol->line_l, T, L) ||
        !distinct_level_pairs(mol->coll_u, mol->coll_l, P, L)) {
        set_error("molecule: two lines or two collision entries join the same pair of levels");
        return LOC_EINVAL;
    }
    if (o->max_iter < 1 || !(o->tol_tex >= 0.0) || !(o->level_cutoff >= 0.0 && o->level_cutoff <= 1e-6)) {
        set_error("options: max_iter >= 1, tol_tex >= 0, level_cutoff in [0, 1e-6]");
        return LOC_EINVAL;
    }
    Request *q = new (std::nothrow) Request();
    if (!q) { set_error("host allocation failed"); return LOC_ENOMEM; }
    q->K = K;
    q->n_rays = n_rays;
    q->ray_power = d->ray_power > 0.0 ? d->ray_power : 1.0;
    q->n_ch = d->n_ch;
    q->v_min = d->v_min;
    q->dv = d->dv;
    q->t_bg = d->t_bg;
    q->L = L;
    q->T = T;
    q->P = P;
    q->mass = mol->mass_amu;
    q->max_iter = o->max_iter;
    q->cutoff = o->level_cutoff;
    q->tol = (float)o->tol_tex;
    q->ali = o->ali;
    q->lay = layout_for(*q);
    q->staged.assign(q->lay.inputs_end, 0);
    unsigned char *b = q->staged.data();
    const ArenaLayout &a = q->lay;
    memcpy(b + a.n_h2, d->n_h2, 8 * K);
    memcpy(b + a.t_kin, d->t_kin, 8 * K);
    memcpy(b + a.abundance, d->abundance, 8 * K);
    memcpy(b + a.sigma, d->sigma_turb, 8 * K);
    memcpy(b + a.radius, d->radius, 8 * K);
    float *v1 = (float *)(b + a.v1d);
    for (int k = 0; k < K; k++) v1[k] = (float)d->v[k];
    memcpy(b + a.energy, mol->energy_K, 8 * L);
    memcpy(b + a.g, mol->g, 8 * L);
    memcpy(b + a.line_u, mol->line_u, 4 * T);
    memcpy(b + a.line_l, mol->line_l, 4 * T);
    memcpy(b + a.line_A, mol->line_A, 8 * T);
    memcpy(b + a.line_nu, mol->line_nu, 8 * T);
    if (P) {
        memcpy(b + a.coll_u, mol->coll_u, 4 * P);
        memcpy(b + a.coll_l, mol->coll_l, 4 * P);
        memcpy(b + a.coll_k, mol->coll_k, 8 * P);
    }
    q->ticket = s->next_ticket.fetch_add(1);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->any_submit) { s->any_submit = true; s->t_first_submit = q->t_submit; }
        s->submitted++;
        s->pending.push_back(q);
    }
    s->cv_work.notify_one();
    *ticket = q->ticket;
    return LOC_OK;
}

loc_status loc_server_poll(loc_server *s, uint64_t ticket, int timeout_ms, loc_result *out,
                           double *populations, size_t n_out)
{
    if (!s || !out) { set_error("NULL argument"); return LOC_EINVAL; }
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (true) {
        auto it = s->done.find(ticket);
        if (it != s->done.end()) {
            Finished &f = it->second;
            const size_t n = f.pops.size();
            if (populations) {
                if (n_out < n) { set_error("populations buffer needs %zu elements", n); return LOC_EINVAL; }
                memcpy(populations, f.pops.data(), sizeof(double) * n);
            }
            *out = f.r;
            s->done.erase(it);
            return LOC_OK;
        }
        if (s->fatal != LOC_OK) { set_error("server stopped: %s", s->fatal_msg); return s->fatal; }
        if (ticket == 0 || ticket >= s->next_ticket.load()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return LOC_EINVAL; }
        if (timeout_ms <= 0 || s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            if (s->done.count(ticket)) continue;
            set_error("ticket %llu not finished within %d ms", (unsigned long long)ticket, timeout_ms);
            return LOC_ETIMEOUT;
        }
    }
}

loc_status loc_server_stats(loc_server *s, loc_server_counters *st)
{
    if (!s || !st) { set_error("NULL argument"); return LOC_EINVAL; }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->queued = (int64_t)s->pending.size();
    int64_t act = 0;
    for (auto &h : s->slots) act += h.used;
    st->active = act;
    st->device_bytes_in_use = (int64_t)s->mem_used;
    if (!s->latencies_ms.empty()) {
        std::vector<double> v = s->latencies_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, std::ceil(p * v.size()) - 1));
            return v[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / v.size();
        const double span = std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count();
        st->models_per_s = span > 0 ? s->completed / span : 0.0;
    }
    return s->fatal;
}

void loc_server_destroy(loc_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->st);
    for (auto &h : s->slots) {
        if (h.arena) cudaFree(h.arena);
        delete h.req;
    }
    for (Request *q : s->pending) delete q;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (int c = 0; c < kBatchClasses; c++) if (s->items_d[c]) cudaFree(s->items_d[c]);
    if (s->cells_d) cudaFree(s->cells_d);
    cudaFree(s->slots_d);
    cudaFree(s->done_d);
    cudaFreeHost(s->done_h);
    cudaFree(s->counts_d);
    cudaFreeHost(s->counts_h);
    cudaFree(s->counters_d);
    for (int c = 0; c < kBatchClasses; c++) {
        if (s->side[c]) cudaStreamDestroy(s->side[c]);
        if (s->join[c]) cudaEventDestroy(s->join[c]);
    }
    if (s->fork) cudaEventDestroy(s->fork);
    cudaStreamDestroy(s->st);
    delete s;
}

}  // extern "C"
