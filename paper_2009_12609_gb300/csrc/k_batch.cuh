// k_batch.cuh -- device layout of the batched 1D engine (k_batch.cu) and the
// server that feeds it (loc_server.cu).
#pragma once

#include "loc_internal.cuh"

namespace loc {

// One model of the batch.
struct BatchSlot {
    DevModel m;          // the model's device buffers
    int active;          // 1 while it iterates
    int done;            // 1 once converged or out of iterations
    int iter, max_iter;
    float tol, last_dtex;
    int ali;
    int per, n_groups;   // lines per warp, line groups
    float inv_dv;        // 1 / channel width in FP32
    double cutoff;       // per-cell line truncation (loc_iter_opts.level_cutoff)
};

// Line-group classes of the batched march (compile-time group sizes) and
// the intensity floats each warp of a class keeps in shared memory: a slot
// with per lines per warp joins the smallest class G >= per, and per is
// capped so that per x n_ch <= 2048.
constexpr int kBatchClasses = 5;
constexpr int kBatchClassG[kBatchClasses] = {1, 2, 4, 8, 15};
constexpr int kBatchClassFloats[kBatchClasses] = {1024, 2048, 4 * 682, 8 * 409, 15 * 227};
constexpr int kBatchLineFloats = 2048;
constexpr int kBatchCounters = kBatchClasses + 1;
constexpr int kBatchMaxRates = 31 + 496;   // lines + collision pairs of a 32-level molecule

struct BatchLaunch {
    BatchSlot *slots;            // [n_slots]
    int n_slots;
    int4 *items[kBatchClasses];  // (slot, ray, group, steps), longest first
    int *n_items;                // [kBatchClasses] device counts
    int2 *cells;                 // (slot, cell)
    int *n_cells;                // device count
    unsigned *counters;          // [kBatchCounters]
    int *done_out;               // [n_slots] copy of BatchSlot::done
    float window;
    int n_sm, blocks_per_sm;
    cudaStream_t side[kBatchClasses];        // one branch per line-group class
    cudaEvent_t fork, join[kBatchClasses];   // fork / join of the branches
};

loc_status batch_prepare();
loc_status batch_launch_iteration(const BatchLaunch &b, cudaStream_t st);

}  // namespace loc
