// k_march1d.cu -- ray march over 1D shells (Sect. 2.1) and the 1D emergent
// spectra; the per-step update is march_step in k_march.cuh.
#include "k_march.cuh"

namespace loc {

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
    const long long nw = march_ray1d<G>(m, a, I, j, lane);
    flush_count(m, a, nw, lane);
}

// instantiate every group size 1..15 so no predicated-off line is issued
template <int G>
static loc_status launch_g(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    const size_t smem = (size_t)kWarpsPerBlock * a.per * m.n_ch * sizeof(float);
    const long long items = (long long)m.n_rays * a.n_groups;
    const long long nb = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
    LOC_CUDA_TRY(cudaFuncSetAttribute(march1d_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    march1d_kernel<G><<<(unsigned)nb, kWarpsPerBlock * 32, smem, st>>>(m, a);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_march1d(const DevModel &m, const MarchArgs &a, cudaStream_t st)
{
    switch (a.per) {
    case 1: return launch_g<1>(m, a, st);
    case 2: return launch_g<2>(m, a, st);
    case 3: return launch_g<3>(m, a, st);
    case 4: return launch_g<4>(m, a, st);
    case 5: return launch_g<5>(m, a, st);
    case 6: return launch_g<6>(m, a, st);
    case 7: return launch_g<7>(m, a, st);
    case 8: return launch_g<8>(m, a, st);
    case 9: return launch_g<9>(m, a, st);
    case 10: return launch_g<10>(m, a, st);
    case 11: return launch_g<11>(m, a, st);
    case 12: return launch_g<12>(m, a, st);
    case 13: return launch_g<13>(m, a, st);
    case 14: return launch_g<14>(m, a, st);
    default: return launch_g<15>(m, a, st);
    }
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
