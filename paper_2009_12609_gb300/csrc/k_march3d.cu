// k_march3d.cu -- ray march over a regular 3D grid (Sect. 2.2); the walk is
// GridWalk in walk3d.cuh, the per-step update march_step in k_march.cuh.
#include "k_march.cuh"

namespace loc {

// 3D regular grid: one warp per (direction, root line, line group).
// registers capped for 4 blocks per SM up to 8 lines per warp, 3 above
template <int G, int ACC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, G <= 8 ? 4 : 3) march3d_kernel(DevModel m, MarchArgs a0)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item0 = (long long)blockIdx.x * kWarpsPerBlock + wid;
    const long long per_dir = (long long)m.N * m.N;
    if (item0 >= per_dir * (a0.dir1 - a0.dir0) * a0.n_groups) return;
    const long long item = item0 / a0.n_groups;
    const MarchArgs a = warp_args(m, a0, (int)(item0 - item * a0.n_groups));
    const int dir = a0.dir0 + (int)(item / per_dir);
    const long long r = item - (long long)(dir - a0.dir0) * per_dir;
    const long long i = r / m.N, j = r - (r / m.N) * m.N;
    float *I = smem + (size_t)wid * a.per * m.n_ch;
    init_ray<G>(m, a, I, lane);
    const Dir3D D = m.dirs[dir];
    const float wscale = 1.0f / ((float)(1ll << kFixedBits) * (float)m.n_dir);
    GridWalk wk;
    wk.init(D, i, j);
    auto fetch = [&](Step<G> &st) {
        long long dz;
        wk.step(D, m.N, st.cell, dz);
        const float4 cv = m.vel[st.cell];
        st.vlos = cv.x * D.d[0] + cv.y * D.d[1] + cv.z * D.d[2];
        st.inv = cv.w;
        st.s = (float)(int)dz * D.unit;             // dz <= one cell = 2^24 units
        st.w = (float)(int)dz * wscale;
        load_lines<G>(m, a, st, lane);
    };
    long long nw = 0;
    Step<G> cur, nxt;
    MarchState pend = march_state();
    fetch(cur);
    while (true) {
        const bool more = !wk.done(m.N);
        if (more) fetch(nxt);
        nw += march_step<G, ACC>(m, a, I, cur, lane, pend);
        __syncwarp();
        if (!more) break;
        cur = nxt;
    }
    march_state_end<ACC>(m, a, pend, lane);
    flush_count(m, a, nw, lane);
}


struct Launch3D {
    const DevModel &m;
    const MarchArgs &a;
    cudaStream_t st;
    template <int G, int ACC>
    loc_status go() const
    {
        const size_t smem = (size_t)kWarpsPerBlock * a.per * m.n_ch * sizeof(float);
        const long long items = (long long)m.N * m.N * (a.dir1 - a.dir0) * a.n_groups;
        const long long nb = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
        LOC_CUDA_TRY(cudaFuncSetAttribute(march3d_kernel<G, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        march3d_kernel<G, ACC><<<(unsigned)nb, kWarpsPerBlock * 32, smem, st>>>(m, a);
        LOC_CUDA_TRY(cudaGetLastError());
        return LOC_OK;
    }
};

loc_status launch_march3d(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    return march_dispatch(a, Launch3D{m, a, st});
}

loc_status launch_march(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    const size_t smem = (size_t)kWarpsPerBlock * a.per * m.n_ch * sizeof(float);
    if (smem > 227 * 1024 || a.per > kMaxLinesPerWarp || a.per < 1 ||
        a.n_groups != (m.T + a.per - 1) / a.per) {
        set_error("march: %d lines per warp x %d channels need %zu B of shared memory per block",
                  a.per, m.n_ch, smem);
        return LOC_EINVAL;
    }
    if (m.geometry == LOC_SHELLS_1D) return launch_march1d(m, a, st);
    if (m.geometry == LOC_OCTREE_3D) return launch_march_octree(m, a, st);
    return launch_march3d(m, a, st);
}

// ----------------------------------------------------------------------------
// 3D map of a regular grid (Sect. 2: final line-of-sight integration): one
// warp per pixel = root line (i, j) of direction dir, walked by the march's
// integer DDA once through the periodic model, all channels (CMAX chunks of
// 31 in registers), no accumulation.
// ----------------------------------------------------------------------------
template <int CMAX>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) map_grid3d_kernel(DevModel m, int t, int dir, float *Tout)
{
    const int lane = threadIdx.x & 31;
    const long long pix = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (pix >= (long long)m.N * m.N) return;
    const Dir3D D = m.dirs[dir];
    GridWalk wk;
    wk.init(D, pix / m.N, pix % m.N);
    const int nchunk = (m.n_ch + 30) / 31;
    const float nb = m.nbg[t];
    const float inv_dv = (float)(1.0 / m.dv), dv = (float)m.dv, vmin = (float)m.v_min;
    float dI[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; c++) dI[c] = 0.f;
    while (true) {
        long long cell, dz;
        wk.step(D, m.N, cell, dz);
        const float4 cv = m.vel[cell];
        const float vlos = cv.x * D.d[0] + cv.y * D.d[1] + cv.z * D.d[2];
        const float2 ks = m.ks[cell * m.T + t];
        los_step<CMAX>(dI, nchunk, lane, ks.x * ((float)(int)dz * D.unit), ks.y - nb, (vmin + vlos) * inv_dv,
                       dv * cv.w);
        if (wk.done(m.N)) break;
    }
    los_store<CMAX>(dI, nchunk, m.n_ch, lane, (float)(kH * m.line_nu[t] / kKB), pix, Tout);
}

template <int CMAX>
static loc_status launch_map_grid_c(const DevModel &m, int t, int dir, float *T_dev, cudaStream_t st)
{
    const long long np = (long long)m.N * m.N;
    map_grid3d_kernel<CMAX><<<(unsigned)((np + kWarpsPerBlock - 1) / kWarpsPerBlock), kWarpsPerBlock * 32, 0, st>>>(
        m, t, dir, T_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_map_grid3d(const DevModel &m, int t, int dir, float *T_dev, cudaStream_t st)
{
    const int nchunk = (m.n_ch + 30) / 31;
    if (nchunk <= 2) return launch_map_grid_c<2>(m, t, dir, T_dev, st);
    if (nchunk <= 5) return launch_map_grid_c<5>(m, t, dir, T_dev, st);
    if (nchunk <= 9) return launch_map_grid_c<9>(m, t, dir, T_dev, st);
    if (nchunk <= 17) return launch_map_grid_c<17>(m, t, dir, T_dev, st);
    return launch_map_grid_c<34>(m, t, dir, T_dev, st);
}

}  // namespace loc
