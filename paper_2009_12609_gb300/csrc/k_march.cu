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
// GB300 mapping: one warp per ray (and group of lines), lanes over channels,
// the ray's intensities I[line][channel] in shared memory, profile computed
// once per step and channel and reused by every line of the group, channels
// optionally restricted to a window around the local line centre (Sect.
// A.2), per-step sums reduced across the warp and added to the cell with one
// vector atomic {SIJ, ESC} per line (FP32) or FP64 atomics.
#include "loc_internal.cuh"
#include "walk3d.cuh"

namespace loc {

constexpr int kWarpsPerBlock = 4;

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

// 1 - e^-tau: series for |tau| < 1/8 (truncation < 1e-9 relative), MUFU
// exponential otherwise.
__device__ __forceinline__ float one_minus_exp(float tau)
{
    if (fabsf(tau) < 0.125f) {
        float p = 1.f - tau * (1.f / 6.f);
        p = 1.f - tau * (1.f / 5.f) * p;
        p = 1.f - tau * (1.f / 4.f) * p;
        p = 1.f - tau * (1.f / 3.f) * p;
        p = 1.f - tau * 0.5f * p;
        return tau * p;
    }
    return 1.f - __expf(-tau);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Process one step through `cell`.  All lanes call it with identical
// arguments.  vlos: line-of-sight velocity; inv: 1/(sqrt(2) sigma).
template <int G>
__device__ __forceinline__ int march_step(const DevModel &m, const MarchArgs &a, float *I,
                                           long long cell, float s, float vlos, float inv,
                                           float w, int lane)
{
    const int nch = m.n_ch;
    const float dv = (float)m.dv;
    const float u0 = ((float)m.v_min + vlos) / dv;   // channel coordinate offset
    const float db = dv * inv;                        // channel width in b units
    int klo = 0, khi = nch;
    if (a.window > 0.f) {
        const float hw = a.window / (1.41421356f * db);   // window half-width, channels
        const float cen = -u0;
        klo = (int)fminf(fmaxf(floorf(cen - hw), 0.f), (float)nch);
        khi = (int)fminf(fmaxf(ceilf(cen + hw), 0.f), (float)nch);
    }
    float Ks[G], Sv[G], sij[G], esc[G];
#pragma unroll
    for (int t = 0; t < G; t++) {
        sij[t] = 0.f;
        esc[t] = 0.f;
        if (t < a.n_lines) {
            const float2 ks = m.ks[(long long)(a.line0 + t) * m.n_cells + cell];
            float k = ks.x * s;
            // keep |K s| >= 1e-20 so that (1 - e^-tau) / (K s) stays phi
            if (fabsf(k) < 1e-20f) k = (k < 0.f) ? -1e-20f : 1e-20f;
            Ks[t] = k;
            Sv[t] = ks.y;
        } else {
            Ks[t] = 1e-20f;
            Sv[t] = 0.f;
        }
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
                    *ip = fmaf(Sv[t] - iv, tm, iv);
                }
            }
        }
    }
    // reduce across lanes; lane t adds line t
    if (a.do_norm) {
        nrm = warp_sum(nrm);
        if (lane == 31) {
            if (a.fp64_acc) atomicAdd(m.norm64 + cell, (double)w * (double)nrm);
            else atomicAdd(m.norm + cell, w * nrm);
        }
    }
#pragma unroll
    for (int t = 0; t < G; t++) {
        if (t < a.n_lines) {
            const float ss = warp_sum(sij[t]);
            const float se = warp_sum(esc[t]);
            if (lane == t) {
                const float f = w / Ks[t];
                const long long o = (long long)(a.line0 + t) * m.n_cells + cell;
                if (a.fp64_acc) {
                    const double fd = (double)w / (double)Ks[t];
                    atomicAdd(m.acc64 + 2 * o, fd * (double)ss);
                    atomicAdd(m.acc64 + 2 * o + 1, fd * (double)se);
                } else {
                    atomicAdd(m.acc + o, make_float2(ss * f, se * f));
                }
            }
        }
    }
    return khi - klo;
}

// add this warp's computed-update count (profiling)
__device__ __forceinline__ void flush_count(const DevModel &m, const MarchArgs &a, long long nw,
                                            int lane)
{
    if (a.count && lane == 0) atomicAdd(m.upd_count, (unsigned long long)(nw * a.n_lines));
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

// 1D shells: one warp per equidistant ray j.
template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) march1d_kernel(DevModel m, MarchArgs a)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int j = blockIdx.x * kWarpsPerBlock + wid;
    if (j >= m.n_rays) return;
    float *I = smem + (size_t)wid * a.n_lines * m.n_ch;
    init_ray<G>(m, a, I, lane);
    const int s0 = m.ray_off[j], s1 = m.ray_off[j + 1];
    long long nw = 0;
    for (int si = s0; si < s1; si++) {
        const Seg1D sg = m.segs[si];
        nw += march_step<G>(m, a, I, sg.cell, sg.s, sg.vlos, m.inv_s2sig[sg.cell], sg.w, lane);
        __syncwarp();
    }
    flush_count(m, a, nw, lane);
}

// 3D regular grid: one warp per (direction, root line).
template <int G>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) march3d_kernel(DevModel m, MarchArgs a)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const long long item = (long long)blockIdx.x * kWarpsPerBlock + wid;
    const long long per_dir = (long long)m.N * m.N;
    if (item >= per_dir * m.n_dir) return;
    const int dir = (int)(item / per_dir);
    const long long r = item - (long long)dir * per_dir;
    const long long i = r / m.N, j = r - (r / m.N) * m.N;
    float *I = smem + (size_t)wid * a.n_lines * m.n_ch;
    init_ray<G>(m, a, I, lane);
    const Dir3D D = m.dirs[dir];
    const float wscale = 1.0f / ((float)(1ll << kFixedBits) * (float)m.n_dir);
    long long nw = 0;
    walk_grid3d(D, m.N, i, j, [&](long long cell, long long dz) {
        const float4 cv = m.vel[cell];
        const float vlos = cv.x * D.d[0] + cv.y * D.d[1] + cv.z * D.d[2];
        const float s = (float)dz * D.unit;
        const float w = (float)dz * wscale;
        nw += march_step<G>(m, a, I, cell, s, vlos, cv.w, w, lane);
        __syncwarp();
    });
    flush_count(m, a, nw, lane);
}

template <int G>
static loc_status launch_march_g(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    const size_t smem = (size_t)kWarpsPerBlock * a.n_lines * m.n_ch * sizeof(float);
    long long items;
    if (m.geometry == LOC_SHELLS_1D) items = m.n_rays;
    else items = (long long)m.N * m.N * m.n_dir;
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
    const size_t smem = (size_t)kWarpsPerBlock * a.n_lines * m.n_ch * sizeof(float);
    if (smem > 227 * 1024) {
        set_error("march: %d lines x %d channels need %zu B of shared memory per block",
                  a.n_lines, m.n_ch, smem);
        return LOC_EINVAL;
    }
    if (a.n_lines <= 1) return launch_march_g<1>(m, a, st);
    if (a.n_lines <= 2) return launch_march_g<2>(m, a, st);
    if (a.n_lines <= 4) return launch_march_g<4>(m, a, st);
    if (a.n_lines <= 8) return launch_march_g<8>(m, a, st);
    if (a.n_lines <= 12) return launch_march_g<12>(m, a, st);
    return launch_march_g<16>(m, a, st);
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
        const float2 ks = m.ks[(long long)t * m.n_cells + k];
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
