// k_march1d.cu -- ray march over 1D shells (Sect. 2.1) and the 1D emergent
// spectra; the per-step update is march_step in k_march.cuh.
#include "k_march.cuh"

namespace loc {

template <int G, int ACC, bool HF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, G <= 11 ? 5 : 3) march1d_kernel(DevModel m, MarchArgs a0)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * kWarpsPerBlock + wid;
    if (item >= (long long)m.n_rays * a0.n_groups) return;
    const int j = (int)(item / a0.n_groups);
    const MarchArgs a = warp_args(m, a0, (int)(item - (long long)j * a0.n_groups));
    float *I = smem + (size_t)wid * a.per * m.n_ch;
    const long long nw = march_ray1d<G, ACC, HF>(m, a, I, j, lane);
    flush_count(m, a, nw, lane);
}

struct Launch1D {
    const DevModel &m;
    const MarchArgs &a;
    cudaStream_t st;
    template <int G, int ACC>
    loc_status go() const
    {
        const size_t smem = (size_t)kWarpsPerBlock * a.per * m.n_ch * sizeof(float);
        const long long items = (long long)m.n_rays * a.n_groups;
        const long long nb = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
        // models with hyperfine lines take the kernel that evaluates them
        auto k = m.hf_off ? march1d_kernel<G, ACC, true> : march1d_kernel<G, ACC, false>;
        LOC_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k<<<(unsigned)nb, kWarpsPerBlock * 32, smem, st>>>(m, a);
        LOC_CUDA_TRY(cudaGetLastError());
        return LOC_OK;
    }
};

loc_status launch_march1d(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    return march_dispatch(a, Launch1D{m, a, st});
}

// ----------------------------------------------------------------------------
// Rays cut into runs.  A ray's steps are sequential only through the
// intensity, and one step (Eq. 3) maps every channel's intensity affinely,
// I <- I e^-tau + S (1 - e^-tau); so a run of consecutive steps maps the
// intensity entering it to A I_in + B.  Three launches replace the one
// warp-per-ray march, so that a long ray is worked on by many warps at once:
//   affine:  per (run, line group) the run's {A, B} per line and channel
//            (every run except the last of its ray),
//   scan:    per (ray, line, channel) I_in of each run, from the background
//            through the runs' maps in ray order (written over A),
//   march:   per (run, line group) march_step over the run from its I_in,
//            accumulating SIJ / ESC / NORM exactly as the whole-ray march.
// ----------------------------------------------------------------------------
// Channels [lo, hi) touched by the windows of steps s0 .. s0 + n - 1 (the
// union of step_window over the run; lo = hi = 0 if none): all lanes.
template <int G>
__device__ __forceinline__ int2 run_window_union(const DevModel &m, const MarchArgs &a, int s0, int n, int lane)
{
    int lo = m.n_ch, hi = 0;
    for (int q = lane; q < n; q += 32) {
        const Seg1D rec = m.segs[s0 + q];
        Step<G> st;
        st.vlos = rec.vlos;
        st.inv = m.inv_s2sig[rec.cell];
        float u0, db;
        int klo, khi;
        step_window(m, a, st, u0, db, klo, khi);
        if (khi > klo) {
            lo = min(lo, klo);
            hi = max(hi, khi);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = min(lo, __shfl_xor_sync(kFull, lo, off));
        hi = max(hi, __shfl_xor_sync(kFull, hi, off));
    }
    return (lo < hi) ? make_int2(lo, hi) : make_int2(0, 0);
}

// warp per run: the run's window union, and the widest union of all runs
// (sizes the affine launch's shared-memory tiles)
__global__ void __launch_bounds__(kWarpsPerBlock * 32) march1d_ranges_kernel(DevModel m, MarchArgs a, int *max_w)
{
    const int lane = threadIdx.x & 31;
    const long long gc = (long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (gc >= a.n_chunks) return;
    const int j = a.chunk_ray[gc];
    const int c = (int)(gc - a.chunk_off[j]);
    const int n = m.ray_off[j + 1] - m.ray_off[j];
    const int q0 = c * a.chunk;
    const int2 rng = run_window_union<1>(m, a, m.ray_off[j] + q0, min(a.chunk, n - q0), lane);
    if (lane == 0) {
        a.run_rng[gc] = rng;
        atomicMax(max_w, rng.y - rng.x);
    }
}

loc_status launch_march1d_ranges(const DevModel &m, const MarchArgs &a, int *max_w_dev, cudaStream_t st)
{
    const long long nb = (a.n_chunks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    march1d_ranges_kernel<<<(unsigned)nb, kWarpsPerBlock * 32, 0, st>>>(m, a, max_w_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) march1d_affine_kernel(DevModel m, MarchArgs a0)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * kWarpsPerBlock + wid;
    if (item >= a0.n_chunks * a0.n_groups) return;
    const long long gc = item / a0.n_groups;
    const MarchArgs a = warp_args(m, a0, (int)(item - gc * a0.n_groups));
    const int j = a.chunk_ray[gc];
    const int c = (int)(gc - a.chunk_off[j]);
    const int n = m.ray_off[j + 1] - m.ray_off[j];
    const int q0 = c * a.chunk;
    const int s0 = m.ray_off[j] + q0;
    if (q0 + a.chunk >= n) return;                 // last run of the ray: map not needed
    const int2 rng = a.run_rng[gc];                // the channels this run touches
    const int nch = m.n_ch, tile = a.tile;
    float *A = smem + (size_t)wid * 2 * a.per * tile;
    float *B = A + a.per * tile;
    // channel tiles of the union: each tile composes its own channels' maps
    for (int tlo = rng.x; tlo < rng.y; tlo += tile) {
        const int thi = min(rng.y, tlo + tile), w = thi - tlo;
        for (int i = lane; i < a.per * w; i += 32) {       // the tiles hold a.per <= G lines
            const int t = i / w;
            A[t * tile + i - t * w] = 1.f;
            B[t * tile + i - t * w] = 0.f;
        }
        __syncwarp();
        walk_steps1d<G>(m, a, s0, a.chunk, lane, [&](const Step<G> &st) {
            affine_step<G>(m, a, A, B, st, lane, tlo, thi);
            return 0ll;
        });
        float2 *out = a.ab + ((size_t)gc * m.T + a.line0) * nch + tlo;
        for (int i = lane; i < a.n_lines * w; i += 32) {
            const int t = i / w, k = i - t * w;
            out[(size_t)t * nch + k] = make_float2(A[t * tile + k], B[t * tile + k]);
        }
        __syncwarp();
    }
}

// thread per (ray, line, channel): the entering intensity of every run of
// the ray, from the background through the runs' maps in ray order; a run
// whose windows miss the channel leaves it unchanged and needs no value.
// Maps are loaded eight runs at a time ahead of the dependent updates.
__global__ void march1d_scan_kernel(DevModel m, MarchArgs a)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nch = m.n_ch, T = m.T;
    if (idx >= (long long)m.n_rays * T * nch) return;
    const int j = (int)(idx / ((long long)T * nch));
    const int rem = (int)(idx - (long long)j * T * nch);      // t * nch + k
    const int t = rem / nch, k = rem - t * nch;
    float I = m.nbg[t];
    const int c0 = a.chunk_off[j], c1 = a.chunk_off[j + 1];
    constexpr int kB = 8;
    for (int cb = c0; cb < c1; cb += kB) {
        float2 v[kB];
        bool in[kB];
#pragma unroll
        for (int q = 0; q < kB; q++) {
            const int c = cb + q;
            in[q] = false;
            if (c < c1) {
                const int2 r = a.run_rng[c];
                in[q] = (k >= r.x && k < r.y);
                if (in[q] && c + 1 < c1) v[q] = a.ab[(size_t)c * T * nch + rem];
            }
        }
#pragma unroll
        for (int q = 0; q < kB; q++) {
            const int c = cb + q;
            if (c < c1 && in[q]) {
                a.ab[(size_t)c * T * nch + rem].x = I;
                if (c + 1 < c1) I = fmaf(v[q].x, I, v[q].y);
            }
        }
    }
}

// registers capped for 5 blocks per SM up to 11 lines per warp
template <int G, int ACC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, G <= 11 ? 5 : 3) march1d_run_kernel(DevModel m, MarchArgs a0)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * kWarpsPerBlock + wid;
    if (item >= a0.n_chunks * a0.n_groups) return;
    const long long gc = item / a0.n_groups;
    const MarchArgs a = warp_args(m, a0, (int)(item - gc * a0.n_groups));
    const int j = a.chunk_ray[gc];
    const int c = (int)(gc - a.chunk_off[j]);
    const int n = m.ray_off[j + 1] - m.ray_off[j];
    const int q0 = c * a.chunk;
    const int len = min(a.chunk, n - q0);
    const int nch = m.n_ch;
    float *I = smem + (size_t)wid * a.per * nch;
    // entering intensities of the channels the run's windows touch (the
    // march reads no other channel)
    const int2 rng = a.run_rng[gc];
    const int w = rng.y - rng.x;
    const float2 *in = a.ab + ((size_t)gc * m.T + a.line0) * nch + rng.x;
    for (int i = lane; i < a.n_lines * w; i += 32) {
        const int t = i / w, k = i - t * w;
        I[t * nch + rng.x + k] = in[(size_t)t * nch + k].x;
    }
    __syncwarp();
    MarchState pend = march_state();
    const long long nw = walk_steps1d<G>(m, a, m.ray_off[j] + q0, len, lane, [&](const Step<G> &st) {
        return (long long)march_step<G, ACC>(m, a, I, st, lane, pend);
    });
    march_state_end<ACC>(m, a, pend, lane);
    flush_count(m, a, nw, lane);
}

struct Launch1DRuns {
    const DevModel &m;
    const MarchArgs &a;
    cudaStream_t st;
    template <int G, int ACC>
    loc_status go() const
    {
        const long long items = a.n_chunks * a.n_groups;
        const long long nb = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
        const size_t smem_a = (size_t)kWarpsPerBlock * 2 * a.per * a.tile * sizeof(float);
        const size_t smem_r = (size_t)kWarpsPerBlock * a.per * m.n_ch * sizeof(float);
        LOC_CUDA_TRY(cudaFuncSetAttribute(march1d_affine_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a));
        LOC_CUDA_TRY(cudaFuncSetAttribute(march1d_run_kernel<G, ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r));
        march1d_affine_kernel<G><<<(unsigned)nb, kWarpsPerBlock * 32, smem_a, st>>>(m, a);
        LOC_CUDA_TRY(cudaGetLastError());
        const long long ns = (long long)m.n_rays * m.T * m.n_ch;
        march1d_scan_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(m, a);
        LOC_CUDA_TRY(cudaGetLastError());
        march1d_run_kernel<G, ACC><<<(unsigned)nb, kWarpsPerBlock * 32, smem_r, st>>>(m, a);
        LOC_CUDA_TRY(cudaGetLastError());
        return LOC_OK;
    }
};

loc_status launch_march1d_chunked(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    return march_dispatch(a, Launch1DRuns{m, a, st});
}

// ----------------------------------------------------------------------------
// 1D emergent spectra (the final line-of-sight integration, Sect. 2).  Two
// launches:
//   spectra1d_geom:  one thread per (impact parameter, step): the step's
//                    shell, FP64 chord length and entry cosine as in the
//                    march, reduced to an FP32 record {K s, S - n_bg, u0, db}
//                    of line t (FP64 work once per step, not per channel);
//   spectra1d:       one warp per (impact parameter, 31-channel chunk), all
//                    channels, tracking dI = I - n_bg so that the brightness
//                    T = (h nu / k) dI keeps relative accuracy in the wings.
// ----------------------------------------------------------------------------
__global__ void spectra1d_geom_kernel(DevModel m, int t, const double *pv, int n_p, float4 *rec,
                                      int *nsteps)
{
    const int K = m.K, S2 = 2 * K;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_p * S2) return;
    const int ip = (int)(idx / S2), st = (int)(idx - (long long)ip * S2);
    const double p = pv[ip];
    // tangent shell: the first shell whose outer radius exceeds p (radii
    // strictly increasing)
    int lo = 0, hi = K;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (m.radius[mid] > p) hi = mid;
        else lo = mid + 1;
    }
    const int tsh = lo;
    const int n = 2 * (K - tsh);
    if (st == 0) nsteps[ip] = n;
    if (st >= n) return;
    int k;
    double s, cosv;
    if (st < K - tsh) {                      // inbound: K-1 .. tsh
        k = K - 1 - st;
        const double zo = sqrt(m.radius[k] * m.radius[k] - p * p);
        if (k > tsh) {
            const double zi = sqrt(m.radius[k - 1] * m.radius[k - 1] - p * p);
            s = zo - zi;
        } else {
            s = zo;
        }
        cosv = -zo / m.radius[k];
    } else {                                 // outbound: tsh .. K-1
        k = tsh + (st - (K - tsh));
        const double zo = sqrt(m.radius[k] * m.radius[k] - p * p);
        if (k > tsh) {
            const double zi = sqrt(m.radius[k - 1] * m.radius[k - 1] - p * p);
            s = zo - zi;
            cosv = zi / m.radius[k - 1];
        } else {
            s = zo;
            cosv = 0.0;
        }
    }
    const float vlos = (float)((double)m.v1d[k] * cosv);
    const float dv = (float)m.dv;
    const float2 ks = m.ks[(long long)k * m.T + t];
    rec[idx] = make_float4(ks.x * (float)s, ks.y - m.nbg[t], ((float)m.v_min + vlos) / dv,
                           dv * m.inv_s2sig[k]);
}

__global__ void spectra1d_kernel(DevModel m, int t, int n_p, const float4 *rec, const int *nsteps,
                                 float *Tout)
{
    const int lane = threadIdx.x & 31;
    const int nch = m.n_ch;
    const int nchunk = (nch + 30) / 31;
    const long long item = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= (long long)n_p * nchunk) return;
    const int ip = (int)(item / nchunk);
    const int ch = (int)(item - (long long)ip * nchunk) * 31 + lane;
    const int n = nsteps[ip];
    const float4 *r = rec + (size_t)ip * 2 * m.K;
    const int hc0 = m.hf_off ? m.hf_off[t] : 0, hc1 = m.hf_off ? m.hf_off[t + 1] : 0;
    float dI = 0.f;
    for (int b = 0; b < n; b += 32) {
        const float4 my = (b + lane < n) ? r[b + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int nb = min(32, n - b);
        for (int q = 0; q < nb; q++) {
            const float Ksv = __shfl_sync(kFull, my.x, q);
            const float src = __shfl_sync(kFull, my.y, q);
            const float u0 = __shfl_sync(kFull, my.z, q);
            const float db = __shfl_sync(kFull, my.w, q);
            // lane l: Gaussian tail at the lower edge of channel ch, the upper
            // edge from lane l + 1
            const float b0 = ((float)ch + u0) * db;
            const float e0 = 0.5f * erfcf(fabsf(b0));
            const float b1 = __shfl_down_sync(kFull, b0, 1);
            const float e1 = __shfl_down_sync(kFull, e0, 1);
            float phi = (b0 >= 0.f) ? (e0 - e1) : ((b1 <= 0.f) ? (e1 - e0) : (1.f - e0 - e1));
            if (hc1 > hc0) {                 // hyperfine components of line t
                phi = 0.f;
                for (int c = hc0; c < hc1; c++) {
                    const float bc = ((float)ch + u0 - m.hf_o[c]) * db;
                    const float ec = 0.5f * erfcf(fabsf(bc));
                    const float bc1 = __shfl_down_sync(kFull, bc, 1);
                    const float ec1 = __shfl_down_sync(kFull, ec, 1);
                    phi += m.hf_w[c] * ((bc >= 0.f) ? (ec - ec1) : ((bc1 <= 0.f) ? (ec1 - ec) : (1.f - ec - ec1)));
                }
            }
            const float tm = one_minus_exp(Ksv * phi);
            dI = fmaf(src - dI, tm, dI);
        }
    }
    if (lane < 31 && ch < nch) Tout[(long long)ip * nch + ch] = (float)(kH * m.line_nu[t] / kKB) * dI;
}

loc_status launch_spectra1d(const DevModel &m, int t, const double *p_dev, int n_p, float4 *rec,
                            int *nsteps, float *T_dev, cudaStream_t st)
{
    const long long ng = (long long)n_p * 2 * m.K;
    spectra1d_geom_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(m, t, p_dev, n_p, rec, nsteps);
    LOC_CUDA_TRY(cudaGetLastError());
    const long long items = (long long)n_p * ((m.n_ch + 30) / 31);
    const int wpb = 4;
    spectra1d_kernel<<<(unsigned)((items + wpb - 1) / wpb), wpb * 32, 0, st>>>(m, t, n_p, rec, nsteps, T_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

}  // namespace loc
