// k_batch.cu -- batched ALI iterations over many 1D models at once.
//
// Every model of the batch keeps its own device buffers (a DevModel in the
// slot table); the kernels here run one ALI iteration (Sect. 2: line
// parameters -> ray simulation -> statistical equilibrium) for all active
// slots together:
//   batch_clear / batch_params   one block per slot
//   batch_march<G>               persistent warps that take (slot, ray, line
//                                group) work items from a device counter;
//                                items are ordered longest ray first
//   batch_se                     persistent warps over (slot, cell) items
//   batch_flags                  per slot: iteration count, convergence
//                                test against the slot's tolerance, swap of
//                                the population buffers, retirement
// The per-step update, the ray loop and the equilibrium solve are the same
// device routines as the single-model kernels (k_march.cuh, k_se.cuh).  The
// item counts are read from device memory, so one captured CUDA graph serves
// any batch composition.
#include "k_batch.cuh"
#include "k_march.cuh"
#include "k_se.cuh"

namespace loc {

constexpr int kBatchSeLmax = 32;

__global__ void batch_clear_kernel(BatchSlot *slots, int n_slots)
{
    const int s = blockIdx.x;
    if (s >= n_slots || !slots[s].active) return;
    const DevModel &m = slots[s].m;
    const long long n = (long long)m.n_cells * m.T;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) acc_zero(m, i, i / m.T, 0, (i % m.T) == 0);
}

__global__ void batch_params_kernel(BatchSlot *slots, int n_slots)
{
    const int s = blockIdx.x;
    if (s >= n_slots || !slots[s].active) return;
    const DevModel m = slots[s].m;
    const long long n = (long long)m.n_cells * m.T;
    const double cutoff = slots[s].cutoff;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) line_params_one(m, i, cutoff);
}

template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
batch_march_kernel(BatchSlot *slots, const int4 *items, const int *n_items, unsigned *counter,
                   float window, int warp_floats)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    float *I = smem + (size_t)wid * warp_floats;
    const int total = *n_items;
    while (true) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((int)it >= total) break;
        const int4 w = items[it];
        const BatchSlot *S = slots + w.x;
        if (!S->active) continue;
        const DevModel m = S->m;
        MarchArgs a0;
        memset(&a0, 0, sizeof(a0));
        a0.per = S->per;
        a0.n_groups = S->n_groups;
        a0.window = window;
        a0.inv_dv = S->inv_dv;
        a0.fp64_acc = 0;
        a0.comp = m.acc_c != nullptr;
        a0.count = 0;
        const MarchArgs a = warp_args(m, a0, w.z);
        march_ray1d<G, kAccComp>(m, a, I, w.y, lane);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kSeWarps * 32)
batch_se_kernel(BatchSlot *slots, const int2 *cells, const int *n_cells, unsigned *counter)
{
    constexpr int W = kBatchSeLmax + 2;
    extern __shared__ double se_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double *M = se_smem + (size_t)wid * (kBatchSeLmax * W + kBatchSeLmax);
    const int total = *n_cells;
    while (true) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if ((int)it >= total) break;
        const int2 w = cells[it];
        const BatchSlot *S = slots + w.x;
        if (!S->active) continue;
        const DevModel m = S->m;
        float d = se_seg_cell<kBatchSeLmax, 32>(m, w.y, true, S->ali, 0, lane, M, M + kBatchSeLmax * W);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d = fmaxf(d, __shfl_xor_sync(kFull, d, off));
        if (lane == 0 && d > 0.f) atomicMax(m.dtex_bits, __float_as_uint(d));
        __syncwarp();
    }
}

__global__ void batch_flags_kernel(BatchSlot *slots, int n_slots, int *done_out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    BatchSlot &S = slots[s];
    if (!S.active) { done_out[s] = S.done; return; }
    const float d = __uint_as_float(*S.m.dtex_bits);
    *S.m.dtex_bits = 0u;
    double *tmp = S.m.x;                 // the solve wrote x_new
    S.m.x = S.m.x_new;
    S.m.x_new = tmp;
    S.iter += 1;
    S.last_dtex = d;
    if ((S.tol > 0.f && d < S.tol) || S.iter >= S.max_iter) {
        S.active = 0;
        S.done = 1;
    }
    done_out[s] = S.done;
}

static size_t se_smem_bytes()
{
    return sizeof(double) * kSeWarps * (kBatchSeLmax * (kBatchSeLmax + 2) + kBatchSeLmax);
}

// kernel attributes, set once outside any stream capture
loc_status batch_prepare()
{
#define LOC_BATCH_ATTR(CI)                                                                        \
    LOC_CUDA_TRY(cudaFuncSetAttribute(batch_march_kernel<kBatchClassG[CI]>,                        \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                                      (int)(sizeof(float) * kWarpsPerBlock * kBatchClassFloats[CI])));
    LOC_BATCH_ATTR(0)
    LOC_BATCH_ATTR(1)
    LOC_BATCH_ATTR(2)
    LOC_BATCH_ATTR(3)
    LOC_BATCH_ATTR(4)
#undef LOC_BATCH_ATTR
    LOC_CUDA_TRY(cudaFuncSetAttribute(batch_se_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)se_smem_bytes()));
    return LOC_OK;
}

loc_status batch_launch_iteration(const BatchLaunch &b, cudaStream_t st)
{
    LOC_CUDA_TRY(cudaMemsetAsync(b.counters, 0, sizeof(unsigned) * kBatchCounters, st));
    batch_clear_kernel<<<b.n_slots, 256, 0, st>>>(b.slots, b.n_slots);
    batch_params_kernel<<<b.n_slots, 256, 0, st>>>(b.slots, b.n_slots);
    const unsigned grid = (unsigned)(b.n_sm * b.blocks_per_sm);
    // the classes run as parallel branches (fork / join through events), so
    // one class's tail overlaps the others' work
    LOC_CUDA_TRY(cudaEventRecord(b.fork, st));
#define LOC_BATCH_LAUNCH(CI)                                                                      \
    LOC_CUDA_TRY(cudaStreamWaitEvent(b.side[CI], b.fork, 0));                                      \
    batch_march_kernel<kBatchClassG[CI]><<<grid, kWarpsPerBlock * 32,                              \
                                           sizeof(float) * kWarpsPerBlock * kBatchClassFloats[CI], \
                                           b.side[CI]>>>(                                          \
        b.slots, b.items[CI], b.n_items + CI, b.counters + CI, b.window, kBatchClassFloats[CI]);  \
    LOC_CUDA_TRY(cudaEventRecord(b.join[CI], b.side[CI]));                                         \
    LOC_CUDA_TRY(cudaStreamWaitEvent(st, b.join[CI], 0));
    LOC_BATCH_LAUNCH(0)
    LOC_BATCH_LAUNCH(1)
    LOC_BATCH_LAUNCH(2)
    LOC_BATCH_LAUNCH(3)
    LOC_BATCH_LAUNCH(4)
#undef LOC_BATCH_LAUNCH
    batch_se_kernel<<<(unsigned)(b.n_sm * 4), kSeWarps * 32, se_smem_bytes(), st>>>(
        b.slots, b.cells, b.n_cells, b.counters + kBatchClasses);
    batch_flags_kernel<<<(b.n_slots + 127) / 128, 128, 0, st>>>(b.slots, b.n_slots, b.done_out);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

}  // namespace loc
