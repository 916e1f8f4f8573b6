// k_march.cu -- the ray march: one radiation-field simulation (Sect. 2).
//
// For every ray and velocity channel the march crosses the cells in order
// and, per step of length s through cell c, evaluates the channel-integrated
// Gaussian profile phi_k Doppler-shifted by the line-of-sight velocity at the
// step's start, the optical depth tau_k = K phi_k s, and
//   SIJ_c += w sum_k phi_k I_k f_k,   ESC_c += w sum_k phi_k f_k,
//   NORM_c += w sum_k phi_k,          I_k <- I_k e^-tau_k + S (1 - e^-tau_k),
// with f = (1 - e^-tau) / tau (the external term of Eq. 2 and, through ESC,
// the local term that ALI removes; Eq. 3 for the update).  Since
// phi_k f_k = (1 - e^-tau_k) / (K s), the per-channel sums only need
// t_k = 1 - e^-tau_k and one division per (step, line).
//
// GB300 mapping: one warp per ray (and group of at most 15 lines), lanes
// over channels, the ray's intensities I[line][channel] in shared memory,
// the profile computed once per step and channel and reused by every line
// of the group, channels optionally restricted to a window around the local
// line centre (Sect. A.2).  The per-step sums {SIJ_t, ESC_t, NORM} of all
// lanes are combined by a transpose-reduction that leaves line t's totals
// in lane t, so each step ends with one coalesced vector atomic {SIJ, ESC}
// per line into the cell's contiguous [cell][line] record.  The next step's
// cell data is loaded while the current step computes.
#include "loc_internal.cuh"
#include "walk3d.cuh"

namespace loc {

constexpr int kWarpsPerBlock = 4;
constexpr unsigned kFull = 0xffffffffu;

// Channel fraction of a Gaussian between b0 and b0 + db (arguments in units
// of sqrt(2) sigma), written with upper tails so both wings keep relative
// accuracy.
__device__ __forceinline__ float chan_phi(float b0, float db)
{
    const float b1 = b0 + db;
    const float e0 = 0.5f * erfcf(fabsf(b0));
    const float e1 = 0.5f * erfcf(fabsf(b1));
    return (b0 >= 0.f) ? (e0 - e1) : ((b1 <= 0.f) ? (e1 - e0) : (1.f - e0 - e1));
}

// 1 - e^-tau: series for |tau| < 1/8 (truncation < 1e-9 relative), the
// exponential otherwise; both evaluated, no divergence.
__device__ __forceinline__ float one_minus_exp(float tau)
{
    float p = 1.f - tau * (1.f / 6.f);
    p = 1.f - tau * (1.f / 5.f) * p;
    p = 1.f - tau * (1.f / 4.f) * p;
    p = 1.f - tau * (1.f / 3.f) * p;
    p = 1.f - tau * 0.5f * p;
    const float e = __expf(-tau);
    return (fabsf(tau) < 0.125f) ? tau * p : 1.f - e;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

// Sum of v[i] over the 32 lanes for all i at once; lane l receives the
// total of index l (recursive halving: 31 shuffles for 32 values).
__device__ __forceinline__ float transpose_reduce32(float (&v)[32], int lane)
{
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < m; i++) {
            const float send = up ? v[i] : v[i + m];
            const float keep = up ? v[i + m] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, m);
        }
    }
    return v[0];
}

// Data of one ray step.
template <int G>
struct Step {
    long long cell;
    float s, w;          // path length (cm), weight of the step
    float vlos, inv;     // line-of-sight velocity, 1/(sqrt(2) sigma)
    float2 ks[G];        // {K, S} of the lines of this pass
};

template <int G>
__device__ __forceinline__ void load_lines(const DevModel &m, const MarchArgs &a, Step<G> &st)
{
    const float2 *p = m.ks + st.cell * m.T + a.line0;
#pragma unroll
    for (int t = 0; t < G; t++) st.ks[t] = (t < a.n_lines) ? p[t] : make_float2(0.f, 0.f);
}

// Process one step.  All lanes call it with identical arguments.  Returns
// the number of channels computed.
template <int G>
__device__ __forceinline__ int march_step(const DevModel &m, const MarchArgs &a, float *I,
                                          const Step<G> &st, int lane)
{
    const int nch = m.n_ch;
    const float dv = (float)m.dv;
    const float u0 = ((float)m.v_min + st.vlos) / dv;   // channel coordinate offset
    const float db = dv * st.inv;                        // channel width in b units
    int klo = 0, khi = nch;
    if (a.window > 0.f) {
        const float hw = a.window / (1.41421356f * db);  // window half-width, channels
        const float cen = -u0;
        klo = (int)fminf(fmaxf(floorf(cen - hw), 0.f), (float)nch);
        khi = (int)fminf(fmaxf(ceilf(cen + hw), 0.f), (float)nch);
    }
    float Ks[G], sij[G], esc[G];
#pragma unroll
    for (int t = 0; t < G; t++) {
        float k = st.ks[t].x * st.s;
        // keep |K s| >= 1e-20 so that (1 - e^-tau) / (K s) stays phi
        if (fabsf(k) < 1e-20f) k = (k < 0.f) ? -1e-20f : 1e-20f;
        Ks[t] = k;
        sij[t] = 0.f;
        esc[t] = 0.f;
    }
    float nrm = 0.f;
    for (int base = klo; base < khi; base += 32) {
        const int k = base + lane;
        if (k < khi) {
            const float phi = chan_phi(((float)k + u0) * db, db);
            nrm += phi;
#pragma unroll
            for (int t = 0; t < G; t++) {
                if (t < a.n_lines) {
                    const float tm = one_minus_exp(Ks[t] * phi);
                    float *ip = I + t * nch + k;
                    const float iv = *ip;
                    sij[t] = fmaf(iv, tm, sij[t]);
                    esc[t] += tm;
                    *ip = fmaf(st.ks[t].y - iv, tm, iv);
                }
            }
        }
    }
    // lane t < n_lines ends with line t's {SIJ, ESC}; lane 15 with NORM
    float my_sij, my_esc, my_nrm;
    if (G <= 2) {
        my_sij = 0.f;
        my_esc = 0.f;
#pragma unroll
        for (int t = 0; t < G; t++) {
            const float a1 = warp_sum(sij[t]), a2 = warp_sum(esc[t]);
            if (lane == t) { my_sij = a1; my_esc = a2; }
        }
        my_nrm = a.do_norm ? warp_sum(nrm) : 0.f;
    } else {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
#pragma unroll
        for (int t = 0; t < G; t++) { v[t] = sij[t]; v[16 + t] = esc[t]; }
        v[15] = nrm;
        const float r = transpose_reduce32(v, lane);
        my_sij = r;
        my_esc = __shfl_down_sync(kFull, r, 16);
        my_nrm = r;   // meaningful in lane 15
    }
    if (a.do_norm && lane == 15) {
        if (a.fp64_acc) atomicAdd(m.norm64 + st.cell, (double)st.w * (double)my_nrm);
        else atomicAdd(m.norm + st.cell, st.w * my_nrm);
    }
    if (lane < a.n_lines) {
        float my_ks = 1.f;
#pragma unroll
        for (int t = 0; t < G; t++) if (lane == t) my_ks = Ks[t];
        const long long o = st.cell * m.T + a.line0 + lane;
        if (a.fp64_acc) {
            const double f = (double)st.w / (double)my_ks;
            atomicAdd(m.acc64 + 2 * o, f * (double)my_sij);
            atomicAdd(m.acc64 + 2 * o + 1, f * (double)my_esc);
        } else {
            const float f = st.w / my_ks;
            atomicAdd(m.acc + o, make_float2(my_sij * f, my_esc * f));
        }
    }
    return khi - klo;
}

template <int G>
__device__ __forceinline__ void init_ray(const DevModel &m, const MarchArgs &a, float *I, int lane)
{
    for (int t = 0; t < a.n_lines; t++) {
        const float nb = m.nbg[a.line0 + t];
        for (int k = lane; k < m.n_ch; k += 32) I[t * m.n_ch + k] = nb;
    }
    __syncwarp();
}

// add this warp's computed-update count (profiling)
__device__ __forceinline__ void flush_count(const DevModel &m, const MarchArgs &a, long long nw,
                                            int lane)
{
    if (a.count && lane == 0) atomicAdd(m.upd_count, (unsigned long long)(nw * a.n_lines));
}

// 1D shells: one warp per (equidistant ray j, line group).  Step records
// are fetched 32 at a time (one coalesced load) and broadcast by shuffle.
// The work item of a warp is (ray, line group); the group fixes line0 and
// n_lines, and group 0 also accumulates NORM.
__device__ __forceinline__ MarchArgs warp_args(const DevModel &m, MarchArgs a, int g)
{
    a.line0 = g * a.per;
    a.n_lines = min(a.per, m.T - a.line0);
    a.do_norm = (g == 0);
    return a;
}

template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) march1d_kernel(DevModel m, MarchArgs a0)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * kWarpsPerBlock + wid;
    if (item >= (long long)m.n_rays * a0.n_groups) return;
    const int j = (int)(item / a0.n_groups);
    const MarchArgs a = warp_args(m, a0, (int)(item - (long long)j * a0.n_groups));
    float *I = smem + (size_t)wid * a.per * m.n_ch;
    init_ray<G>(m, a, I, lane);
    const int s0 = m.ray_off[j], n = m.ray_off[j + 1] - s0;
    if (n <= 0) return;
    Seg1D rec = {0, 0.f, 0.f, 0.f};
    // step q of the ray (0 <= q < n); a new block of 32 records every 32 steps
    auto fetch = [&](int q, Step<G> &st) {
        const int r = q & 31;
        if (r == 0 && q + lane < n) rec = m.segs[s0 + q + lane];
        st.cell = __shfl_sync(kFull, rec.cell, r);
        st.s = __shfl_sync(kFull, rec.s, r);
        st.vlos = __shfl_sync(kFull, rec.vlos, r);
        st.w = __shfl_sync(kFull, rec.w, r);
        st.inv = m.inv_s2sig[st.cell];
        load_lines<G>(m, a, st);
    };
    long long nw = 0;
    Step<G> cur, nxt;
    fetch(0, cur);
    for (int q = 0; q < n; q++) {
        const bool more = q + 1 < n;
        if (more) fetch(q + 1, nxt);
        nw += march_step<G>(m, a, I, cur, lane);
        __syncwarp();
        if (more) cur = nxt;
    }
    flush_count(m, a, nw, lane);
}

// 3D regular grid: one warp per (direction, root line, line group).
template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) march3d_kernel(DevModel m, MarchArgs a0)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item0 = (long long)blockIdx.x * kWarpsPerBlock + wid;
    const long long per_dir = (long long)m.N * m.N;
    if (item0 >= per_dir * m.n_dir * a0.n_groups) return;
    const long long item = item0 / a0.n_groups;
    const MarchArgs a = warp_args(m, a0, (int)(item0 - item * a0.n_groups));
    const int dir = (int)(item / per_dir);
    const long long r = item - (long long)dir * per_dir;
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
        st.s = (float)dz * D.unit;
        st.w = (float)dz * wscale;
        load_lines<G>(m, a, st);
    };
    long long nw = 0;
    Step<G> cur, nxt;
    fetch(cur);
    while (true) {
        const bool more = !wk.done(m.N);
        if (more) fetch(nxt);
        nw += march_step<G>(m, a, I, cur, lane);
        __syncwarp();
        if (!more) break;
        cur = nxt;
    }
    flush_count(m, a, nw, lane);
}

template <int G>
static loc_status launch_march_g(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    const size_t smem = (size_t)kWarpsPerBlock * a.per * m.n_ch * sizeof(float);
    long long items;
    if (m.geometry == LOC_SHELLS_1D) items = (long long)m.n_rays * a.n_groups;
    else items = (long long)m.N * m.N * m.n_dir * a.n_groups;
    const long long nb = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (m.geometry == LOC_SHELLS_1D) {
        LOC_CUDA_TRY(cudaFuncSetAttribute(march1d_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        march1d_kernel<G><<<(unsigned)nb, kWarpsPerBlock * 32, smem, st>>>(m, a);
    } else {
        LOC_CUDA_TRY(cudaFuncSetAttribute(march3d_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        march3d_kernel<G><<<(unsigned)nb, kWarpsPerBlock * 32, smem, st>>>(m, a);
    }
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
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
    if (a.per <= 1) return launch_march_g<1>(m, a, st);
    if (a.per <= 2) return launch_march_g<2>(m, a, st);
    if (a.per <= 4) return launch_march_g<4>(m, a, st);
    if (a.per <= 8) return launch_march_g<8>(m, a, st);
    if (a.per <= 12) return launch_march_g<12>(m, a, st);
    return launch_march_g<15>(m, a, st);
}

// ----------------------------------------------------------------------------
// 1D emergent spectra: one warp per impact parameter, all channels, FP64 path
// geometry as in the march; tracks dI = I - n_bg so that the brightness
// T = (h nu / k) dI keeps relative accuracy in the line wings.
// ----------------------------------------------------------------------------
__global__ void spectra1d_kernel(DevModel m, int t, const double *pv, int n_p, float *Tout)
{
    const int lane = threadIdx.x & 31;
    const int ip = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (ip >= n_p) return;
    const double p = pv[ip];
    const int nch = m.n_ch;
    const int K = m.K;
    constexpr int CMAX = kMaxChannels / 32;
    float dI[CMAX];
#pragma unroll
    for (int i = 0; i < CMAX; i++) dI[i] = 0.f;
    const float nb = m.nbg[t];
    const float dv = (float)m.dv;
    int tsh = 0;
    while (tsh < K && !(m.radius[tsh] > p)) tsh++;
    const int nsteps = (tsh < K) ? 2 * (K - tsh) : 0;
    for (int st = 0; st < nsteps; st++) {
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
        const float inv = m.inv_s2sig[k];
        const float u0 = ((float)m.v_min + vlos) / dv;
        const float db = dv * inv;
        const float2 ks = m.ks[(long long)k * m.T + t];
        const float Ksv = ks.x * (float)s;
        const float src = ks.y - nb;
#pragma unroll
        for (int i = 0; i < CMAX; i++) {
            const int ch = i * 32 + lane;
            if (ch < nch) {
                const float phi = chan_phi(((float)ch + u0) * db, db);
                const float tm = one_minus_exp(Ksv * phi);
                dI[i] = fmaf(src - dI[i], tm, dI[i]);
            }
        }
    }
    const float T0 = (float)(kH * m.line_nu[t] / kKB);
#pragma unroll
    for (int i = 0; i < CMAX; i++) {
        const int ch = i * 32 + lane;
        if (ch < nch) Tout[(long long)ip * nch + ch] = T0 * dI[i];
    }
}

loc_status launch_spectra1d(const DevModel &m, int t, const double *p_dev, int n_p,
                            float *T_dev, cudaStream_t st)
{
    const int wpb = 4;
    spectra1d_kernel<<<(n_p + wpb - 1) / wpb, wpb * 32, 0, st>>>(m, t, p_dev, n_p, T_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

}  // namespace loc
