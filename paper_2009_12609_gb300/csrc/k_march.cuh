// k_march.cuh -- the ray march: one radiation-field simulation (Sect. 2).
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
// in lane t, so each step ends with one
// coalesced vector atomic {SIJ, ESC} per line into the cell's contiguous
// [cell][line] record.  The FP32 atomics are compensated: each lane keeps
// the value its last atomic found and, one step later (when it has long
// arrived), adds the exact rounding error of that addition (TwoSum) to a
// compensation word of the same element.  The next step's cell data is
// loaded while the current step computes.
#pragma once

#include "loc_internal.cuh"
#include "walk3d.cuh"

namespace loc {

constexpr int kWarpsPerBlock = 4;
constexpr unsigned kFull = 0xffffffffu;

// Accumulation of the per-cell sums, fixed when a march kernel is compiled:
// plain FP32 atomics, compensated FP32 atomics, or FP64 atomics.
constexpr int kAccPlain = 0, kAccComp = 1, kAccF64 = 2;

inline int acc_mode(const MarchArgs &a) { return a.fp64_acc ? kAccF64 : (a.comp ? kAccComp : kAccPlain); }

// Register-array sizes (lines per warp) the march kernels are compiled for:
// a group of `per` lines runs in the smallest of them >= per.
__host__ __device__ constexpr int march_g(int per)
{
    return per <= 4 ? per : per <= 6 ? 6 : per <= 8 ? 8 : per <= 11 ? 11 : 15;
}

// f.template go<G, ACC>() for the compiled G of a.per and a's accumulation
template <int G, class F>
loc_status march_dispatch_acc(int mode, const F &f)
{
    switch (mode) {
    case kAccComp: return f.template go<G, kAccComp>();
    case kAccF64: return f.template go<G, kAccF64>();
    default: return f.template go<G, kAccPlain>();
    }
}

template <class F>
loc_status march_dispatch(const MarchArgs &a, const F &f)
{
    const int mode = acc_mode(a);
    switch (march_g(a.per)) {
    case 1: return march_dispatch_acc<1>(mode, f);
    case 2: return march_dispatch_acc<2>(mode, f);
    case 3: return march_dispatch_acc<3>(mode, f);
    case 4: return march_dispatch_acc<4>(mode, f);
    case 6: return march_dispatch_acc<6>(mode, f);
    case 8: return march_dispatch_acc<8>(mode, f);
    case 11: return march_dispatch_acc<11>(mode, f);
    default: return march_dispatch_acc<15>(mode, f);
    }
}

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

// e^-tau as 2^(-tau log2 e) on the SFU, results below the smallest normal
// float flushed to zero (they only ever enter as 1 - e^-tau)
__device__ __forceinline__ float exp_neg(float tau)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(tau * -1.44269504088896341f));
    return y;
}

// 1 - e^-tau: for |tau| < 1/16 the Taylor series tau (1 - tau/2 + tau^2/6 -
// tau^3/24) in Horner form (truncation tau^4/120 < 1.3e-7 relative), the
// exponential otherwise (at tau = 1/16 the SFU's absolute error becomes
// < 3e-6 relative to 1 - e^-tau); both evaluated, no divergence.
__device__ __forceinline__ float one_minus_exp(float tau)
{
    float p = fmaf(tau, -1.f / 24.f, 1.f / 6.f);
    p = fmaf(p, tau, -0.5f);
    p = fmaf(p, tau, 1.f);
    const float e = exp_neg(tau);
    return (fabsf(tau) < 0.0625f) ? tau * p : 1.f - e;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

// Exact rounding error of the FP32 sum a + b (Knuth's TwoSum): with s the
// rounded sum, a + b = s + err exactly.  Explicit round-to-nearest
// operations keep the compiler from contracting or reordering them.
__device__ __forceinline__ float two_sum_err(float a, float b)
{
    const float sum = __fadd_rn(a, b);
    const float bb = __fsub_rn(sum, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(b, bb));
}

// State a lane carries from step to step of one ray: its last compensated
// atomic -- the element, the value added and the value the atomic found
// there (the atomic rounds old + v to nearest, so two_sum_err(old, v) is
// exactly what the stored sum lacks) -- and, when counting, the (step, line)
// pairs of the steps so far whose line is not truncated in the step's cell
// (each stands for n_ch nominal channel updates).
struct MarchState {
    float2 old, v;
    long long o;
    int kind;               // 0 none, 1 {SIJ, ESC} of element o, 2 NORM of cell o
    long long nom;
};

__device__ __forceinline__ void acc_flush(const DevModel &m, MarchState &p)
{
    if (p.kind == 1)
        atomicAdd(m.acc_c + p.o, make_float2(two_sum_err(p.old.x, p.v.x), two_sum_err(p.old.y, p.v.y)));
    else if (p.kind == 2)
        atomicAdd(m.norm_c + p.o, two_sum_err(p.old.x, p.v.x));
    p.kind = 0;
}

__device__ __forceinline__ MarchState march_state()
{
    MarchState p;
    p.old = make_float2(0.f, 0.f);
    p.v = make_float2(0.f, 0.f);
    p.o = 0;
    p.kind = 0;
    p.nom = 0;
    return p;
}

// end of a ray: the pending compensation, and the nominal count (profiling;
// p.nom counts (step, line) pairs, each worth n_ch channel updates)
template <int ACC>
__device__ __forceinline__ void march_state_end(const DevModel &m, const MarchArgs &a, MarchState &p, int lane)
{
    if constexpr (ACC == kAccComp) acc_flush(m, p);
    if (a.count && lane == 0 && p.nom) atomicAdd(m.nom_count, (unsigned long long)p.nom * (unsigned long long)m.n_ch);
    p.nom = 0;
}

// Sum of v[i] over the 32 lanes for all i at once; lane l receives the
// total of index l (recursive halving: 31 shuffles for 32 values).  LIVE
// marks the indices that may be non-zero (the others are 0 in every lane):
// a pair of indices that are both 0 everywhere stays 0 without a shuffle, so
// a step with 2 G + 1 sums of a G-line group issues fewer shuffles; the sums
// that are formed, and their order, do not change.
template <unsigned LIVE = 0xffffffffu>
__device__ __forceinline__ float transpose_reduce32(float (&v)[32], int lane)
{
    unsigned live = LIVE;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < m; i++) {
            if (((live >> i) | (live >> (i + m))) & 1u) {
                const float send = up ? v[i] : v[i + m];
                const float keep = up ? v[i + m] : v[i];
                v[i] = keep + __shfl_xor_sync(kFull, send, m);
            }
        }
        live = (live | (live >> m)) & ((1u << m) - 1u);
    }
    return v[0];
}

// Data of one ray step.  The lines' parameters are spread over the lanes:
// lane t < n_lines holds {K, S} of line t of the pass (one coalesced load
// per step), the others {0, 0}; march_step broadcasts them by shuffle.
template <int G>
struct Step {
    long long cell;
    float s, w;          // path length (cm), weight of the step
    float vlos, inv;     // line-of-sight velocity, 1/(sqrt(2) sigma)
    float2 kl;           // {K, S} of this lane's line
};

template <int G>
__device__ __forceinline__ void load_lines(const DevModel &m, const MarchArgs &a, Step<G> &st, int lane)
{
    st.kl = (lane < a.n_lines) ? m.ks[st.cell * m.T + a.line0 + lane] : make_float2(0.f, 0.f);
}

// Channel coordinate offset u0 (the local line centre sits at channel -u0),
// channel width db in units of sqrt(2) sigma, and the channel range [klo, khi)
// of the step's window (all channels when the window is 0).
template <int G>
__device__ __forceinline__ void step_window(const DevModel &m, const MarchArgs &a, const Step<G> &st,
                                            float &u0, float &db, int &klo, int &khi)
{
    const int nch = m.n_ch;
    u0 = (m.vmin_f + st.vlos) * a.inv_dv;
    db = m.dv_f * st.inv;
    klo = 0;
    khi = nch;
    if (a.window > 0.f) {
        const float hw = __fdividef(a.window, 1.41421356f * db);  // window half-width, channels
        const float cen = -u0;
        klo = (int)fminf(fmaxf(floorf(cen - hw), 0.f), (float)nch);
        khi = (int)fminf(fmaxf(ceilf(cen + hw), 0.f), (float)nch);
    }
}

// K s of a line on a step, kept at |K s| >= 1e-20 so that (1 - e^-tau) / (K s)
// stays phi
__device__ __forceinline__ float step_ks(float K, float s)
{
    float k = K * s;
    if (fabsf(k) < 1e-20f) k = (k < 0.f) ? -1e-20f : 1e-20f;
    return k;
}

// Per-cell line truncation marks a line off in a cell with {K, S} = {-0, 0}:
// K s is then clamped to 1e-20 (step_ks), so the line leaves I unchanged to
// within 1e-20 relative and its SIJ / ESC are not used by the solve.  A step
// whose lines are all off in its cell is skipped outright by the warps that
// do not sum NORM.
template <int G>
__device__ __forceinline__ bool lines_off(const DevModel &m, const MarchArgs &a, const Step<G> &st, int lane)
{
    if (!m.trunc || a.do_norm) return false;
    return __ballot_sync(kFull, lane < a.n_lines && __float_as_uint(st.kl.x) != 0x80000000u) == 0u;
}

// Lane of a warp that adds the step's NORM (lanes t < n_lines <= G add the
// lines' {SIJ, ESC}); the transpose reduction leaves NORM in lane 15.
template <int G>
__device__ __forceinline__ constexpr int norm_lane() { return G <= 2 ? 2 * G : 15; }

// Adds one step's totals to the cell: lane t < n_lines holds line t's
// channel sums {sum I t_k, sum t_k} (t_k = 1 - e^-tau_k), which become
// {SIJ, ESC} with the factor w / ks (ks = line t's K s, step_ks); lane
// norm_lane<G>() holds sum phi_k.
// Compensated FP32: the previous atomic of the lane gets its rounding error
// added first (its result has arrived by now), then the new one is issued
// and remembered.
template <int G, int ACC>
__device__ __forceinline__ void step_commit(const DevModel &m, const MarchArgs &a, long long cell, float ks,
                                            float w, int lane, float my_sij, float my_esc, float my_nrm,
                                            MarchState &pend)
{
    if (lane < a.n_lines) {
        const long long o = cell * m.T + a.line0 + lane;
        if constexpr (ACC == kAccF64) {
            const double f = (double)w / (double)ks;
            atomicAdd(m.acc64 + 2 * o, f * (double)my_sij);
            atomicAdd(m.acc64 + 2 * o + 1, f * (double)my_esc);
        } else {
            const float f = __fdividef(w, ks);
            const float2 v = make_float2(my_sij * f, my_esc * f);
            if constexpr (ACC == kAccPlain) {
                atomicAdd(m.acc + o, v);
            } else {
                acc_flush(m, pend);
                pend.old = atomicAdd(m.acc + o, v);
                pend.v = v;
                pend.o = o;
                pend.kind = 1;
            }
        }
    } else if (a.do_norm && lane == norm_lane<G>()) {
        if constexpr (ACC == kAccF64) {
            atomicAdd(m.norm64 + cell, (double)w * (double)my_nrm);
        } else {
            const float v = w * my_nrm;
            if constexpr (ACC == kAccPlain) {
                atomicAdd(m.norm + cell, v);
            } else {
                acc_flush(m, pend);
                pend.old = make_float2(atomicAdd(m.norm + cell, v), 0.f);
                pend.v = make_float2(v, 0.f);
                pend.o = cell;
                pend.kind = 2;
            }
        }
    }
}

// Narrow windows (at most 16 channels): the lanes take (line, channel) pairs,
// 32 / Wp lines per chunk with Wp the window rounded up to a power of two.
// The profile is evaluated once per step (lane c holds channel klo + c), the
// line parameters come from the lane that holds them, and a segmented
// reduction over each Wp-lane segment gives every lane of the segment line
// t's sums; lane t collects them for step_commit.
template <int G, int ACC>
__device__ __forceinline__ int march_step_packed(const DevModel &m, const MarchArgs &a, float *I,
                                                 const Step<G> &st, int lane, int klo, int khi,
                                                 float u0, float db, MarchState &pend)
{
    const int W = khi - klo;
    if (W <= 0) return 0;
    int Wp = 1;
    while (Wp < W) Wp <<= 1;
    const int P = 32 / Wp;                         // lines per chunk
    const int nch = m.n_ch;
    // profile of the window: lane c (c <= W) evaluates the lower edge of
    // channel klo + c and takes the upper edge from lane c + 1
    const float b0 = ((float)(klo + lane) + u0) * db;
    const float e0 = 0.5f * erfcf(fabsf(b0));
    const float b1 = __shfl_down_sync(kFull, b0, 1);
    const float e1 = __shfl_down_sync(kFull, e0, 1);
    const float phi_c = (lane < W) ? ((b0 >= 0.f) ? (e0 - e1) : ((b1 <= 0.f) ? (e1 - e0) : (1.f - e0 - e1)))
                                   : 0.f;
    // line parameters: lane t holds line t's K s and S
    const float my_k = (lane < G) ? step_ks(st.kl.x, st.s) : 1e-20f;
    const float my_s = (lane < G) ? st.kl.y : 0.f;
    const int tl = lane / Wp, kk = lane - tl * Wp;
    float g_sij = 0.f, g_esc = 0.f;
    for (int base = 0; base < a.n_lines; base += P) {
        const int t = base + tl;
        const bool act = (kk < W) && (t < a.n_lines);
        const float phi = __shfl_sync(kFull, phi_c, kk);
        const float Kt = __shfl_sync(kFull, my_k, t < 32 ? t : 0);
        const float St = __shfl_sync(kFull, my_s, t < 32 ? t : 0);
        float ps = 0.f, pe = 0.f;
        if (act) {
            const float tm = one_minus_exp(Kt * phi);
            float *ip = I + t * nch + klo + kk;
            const float iv = *ip;
            ps = iv * tm;
            pe = tm;
            *ip = fmaf(St - iv, tm, iv);
        }
        for (int off = Wp >> 1; off > 0; off >>= 1) {
            ps += __shfl_xor_sync(kFull, ps, off);
            pe += __shfl_xor_sync(kFull, pe, off);
        }
        // line base + j's sums sit in segment j: lane base + j takes them
        const int j = lane - base;
        const int src = (j >= 0 && j < P) ? j * Wp : 0;
        const float vs = __shfl_sync(kFull, ps, src), ve = __shfl_sync(kFull, pe, src);
        if (j >= 0 && j < P) {
            g_sij = vs;
            g_esc = ve;
        }
    }
    const float nrm = a.do_norm ? warp_sum(phi_c) : 0.f;
    step_commit<G, ACC>(m, a, st.cell, my_k, st.w, lane, g_sij, g_esc, nrm, pend);
    return W;
}

// Process one step.  All lanes call it with identical arguments.  Returns
// the number of channels computed (0 for a skipped step).  pend carries the
// lane's last compensated atomic from step to step (acc_flush after the
// last step).
// HF: the model's lines may have hyperfine components (1D): line t's
// profile is the strength-weighted sum of its components' channel
// fractions, each shifted by its offset, and the window widens to hold every
// component; NORM keeps the unshifted profile.
template <int G, int ACC, bool HF = false>
__device__ __forceinline__ int march_step(const DevModel &m, const MarchArgs &a, float *I,
                                          const Step<G> &st, int lane, MarchState &pend)
{
    if (lines_off<G>(m, a, st, lane)) return 0;
    const int nch = m.n_ch;
    if (a.count) {
        int on = a.n_lines;
        if (m.trunc)
            on = __popc(__ballot_sync(kFull, lane < a.n_lines && __float_as_uint(st.kl.x) != 0x80000000u));
        pend.nom += on;
    }
    float u0, db;
    int klo, khi;
    step_window(m, a, st, u0, db, klo, khi);
    int hc0[HF ? G : 1], hc1[HF ? G : 1];
    if constexpr (HF) {
        if (a.window > 0.f) {
            klo = max(0, klo + (int)floorf(m.hf_olo));
            khi = min(nch, khi + (int)ceilf(m.hf_ohi));
        }
#pragma unroll
        for (int t = 0; t < G; t++) {
            hc0[t] = (t < a.n_lines) ? m.hf_off[a.line0 + t] : 0;
            hc1[t] = (t < a.n_lines) ? m.hf_off[a.line0 + t + 1] : 0;
        }
        if (khi <= klo) return 0;
    } else {
        if (khi - klo <= 16) return march_step_packed<G, ACC>(m, a, I, st, lane, klo, khi, u0, db, pend);
    }
    // lane t < n_lines: K s of its line, then broadcast to every lane
    const float my_ks = step_ks(st.kl.x, st.s);
    float Ks[G], Sv[G], sij[G], esc[G];
#pragma unroll
    for (int t = 0; t < G; t++) {
        Ks[t] = __shfl_sync(kFull, my_ks, t);
        Sv[t] = __shfl_sync(kFull, st.kl.y, t);
        sij[t] = 0.f;
        esc[t] = 0.f;
    }
    // channels in chunks of 31: lane l evaluates the Gaussian tail at the
    // lower edge of channel base + l and takes the upper edge from lane l + 1;
    // a full group (n_lines == G) runs without per-line predicates
    const bool full = (a.n_lines == G);
    float nrm = 0.f;
    auto chunk = [&](int base) {
        const int k = base + lane;
        const float b0 = ((float)k + u0) * db;
        const float e0 = 0.5f * erfcf(fabsf(b0));
        const float b1 = __shfl_down_sync(kFull, b0, 1);
        const float e1 = __shfl_down_sync(kFull, e0, 1);
        float ph[HF ? G : 1];
        if constexpr (HF) {
            // every lane takes part in the components' shuffles
#pragma unroll
            for (int t = 0; t < G; t++) {
                ph[t] = 0.f;
                if (hc1[t] > hc0[t]) {
                    float sum = 0.f;
                    for (int c = hc0[t]; c < hc1[t]; c++) {
                        const float bc = ((float)k + u0 - m.hf_o[c]) * db;
                        const float ec = 0.5f * erfcf(fabsf(bc));
                        const float bc1 = __shfl_down_sync(kFull, bc, 1);
                        const float ec1 = __shfl_down_sync(kFull, ec, 1);
                        sum += m.hf_w[c] * ((bc >= 0.f) ? (ec - ec1) : ((bc1 <= 0.f) ? (ec1 - ec) : (1.f - ec - ec1)));
                    }
                    ph[t] = sum;
                }
            }
        }
        if (lane < 31 && k < khi) {
            const float phi = (b0 >= 0.f) ? (e0 - e1) : ((b1 <= 0.f) ? (e1 - e0) : (1.f - e0 - e1));
            nrm += phi;
            float *ip = I + k;
            if (full) {
#pragma unroll
                for (int t = 0; t < G; t++) {
                    const float tm = one_minus_exp(Ks[t] * ((HF && hc1[HF ? t : 0] > hc0[HF ? t : 0]) ? ph[HF ? t : 0] : phi));
                    const float iv = ip[t * nch];
                    sij[t] = fmaf(iv, tm, sij[t]);
                    esc[t] += tm;
                    ip[t * nch] = fmaf(Sv[t] - iv, tm, iv);
                }
            } else {
#pragma unroll
                for (int t = 0; t < G; t++) {
                    if (t < a.n_lines) {
                        const float tm = one_minus_exp(Ks[t] * ((HF && hc1[HF ? t : 0] > hc0[HF ? t : 0]) ? ph[HF ? t : 0] : phi));
                        const float iv = ip[t * nch];
                        sij[t] = fmaf(iv, tm, sij[t]);
                        esc[t] += tm;
                        ip[t * nch] = fmaf(Sv[t] - iv, tm, iv);
                    }
                }
            }
        }
    };
    if constexpr (G <= 2) {
        // few lines per warp: two independent chunks per pass (more ILP on
        // the latency-bound path of a single long ray)
        int base = klo;
        for (; base + 31 < khi; base += 62) {
            chunk(base);
            chunk(base + 31);
        }
        if (base < khi) chunk(base);
    } else {
        for (int base = klo; base < khi; base += 31) chunk(base);
    }
    // lane t < n_lines ends with line t's {SIJ, ESC}; norm_lane<G>() with NORM
    float my_sij = 0.f, my_esc = 0.f, my_nrm = 0.f;
    if constexpr (G <= 2) {
#pragma unroll
        for (int t = 0; t < G; t++) {
            const float a1 = warp_sum(sij[t]), a2 = warp_sum(esc[t]);
            if (lane == t) { my_sij = a1; my_esc = a2; }
        }
        my_nrm = a.do_norm ? warp_sum(nrm) : 0.f;
    } else {
        // SIJ of line t in value t, ESC in 16 + t, NORM in 15 (= norm_lane)
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; i++) v[i] = 0.f;
#pragma unroll
        for (int t = 0; t < G; t++) { v[t] = sij[t]; v[16 + t] = esc[t]; }
        v[15] = nrm;
        constexpr unsigned kLines = (G >= 15) ? 0x7fffu : ((1u << G) - 1u);
        const float r = transpose_reduce32<kLines | (1u << 15) | (kLines << 16)>(v, lane);
        my_sij = r;
        my_esc = __shfl_down_sync(kFull, r, 16);
        my_nrm = r;
    }
    step_commit<G, ACC>(m, a, st.cell, my_ks, st.w, lane, my_sij, my_esc, my_nrm, pend);
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

// The work item of a warp is (ray, line group); the group fixes line0 and
// n_lines, and group 0 also accumulates NORM.
__device__ __forceinline__ MarchArgs warp_args(const DevModel &m, MarchArgs a, int g)
{
    a.line0 = g * a.per;
    a.n_lines = min(a.per, m.T - a.line0);
    a.do_norm = (g == 0);
    return a;
}


// The 1D step records s0 .. s0 + n - 1 in order, each handed to fn (all
// lanes, identical arguments); records are fetched 32 at a time (one
// coalesced load) and broadcast by shuffle, the next step's line data is
// prefetched.  Returns the sum of fn's results.
template <int G, class F>
__device__ __forceinline__ long long walk_steps1d(const DevModel &m, const MarchArgs &a, int s0, int n,
                                                  int lane, F &&fn)
{
    if (n <= 0) return 0;
    Seg1D rec = {0, 0.f, 0.f, 0.f};
    // step q of the run (0 <= q < n); a new block of 32 records every 32 steps
    auto fetch = [&](int q, Step<G> &st) {
        const int r = q & 31;
        if (r == 0 && q + lane < n) rec = m.segs[s0 + q + lane];
        st.cell = __shfl_sync(kFull, rec.cell, r);
        st.s = __shfl_sync(kFull, rec.s, r);
        st.vlos = __shfl_sync(kFull, rec.vlos, r);
        st.w = __shfl_sync(kFull, rec.w, r);
        st.inv = m.inv_s2sig[st.cell];
        load_lines<G>(m, a, st, lane);
    };
    long long nw = 0;
    Step<G> cur, nxt;
    fetch(0, cur);
    for (int q = 0; q < n; q++) {
        const bool more = q + 1 < n;
        if (more) fetch(q + 1, nxt);
        nw += fn(cur);
        __syncwarp();
        if (more) cur = nxt;
    }
    return nw;
}

// One 1D ray (equidistant ray j) through all its steps for the warp's line
// group.  Returns the number of channels computed.
// Copies the warp's intensities of its line group to (to_store) or from the
// region-boundary buffer of ray j.
__device__ __forceinline__ void sub_boundary(const DevModel &m, const MarchArgs &a, float *I, int j, int lane,
                                             bool to_store)
{
    float *b = a.sub_I + ((size_t)j * m.T + a.line0) * m.n_ch;
    for (int i = lane; i < a.n_lines * m.n_ch; i += 32) {
        if (to_store) b[i] = I[i];
        else I[i] = b[i];
    }
    __syncwarp();
}

template <int G, int ACC, bool HF = false>
__device__ __forceinline__ long long march_ray1d(const DevModel &m, const MarchArgs &a, float *I,
                                                 int j, int lane)
{
    const int s0 = m.ray_off[j], n = m.ray_off[j + 1] - s0;
    MarchState pend = march_state();
    auto fn = [&](const Step<G> &st) { return (long long)march_step<G, ACC, HF>(m, a, I, st, lane, pend); };
    long long nw = 0;
    const int outer = m.K - a.sub_k;                  // steps before the region (sub_k > 0)
    if (a.sub_k > 0 && a.sub_mode == 1) {
        // a sub-iteration: the region's steps of the ray, from the intensity
        // the full march left at the region's boundary
        sub_boundary(m, a, I, j, lane, false);
        nw = walk_steps1d<G>(m, a, s0 + outer, n - 2 * outer, lane, fn);
    } else if (a.sub_k > 0 && a.sub_I && n > 2 * outer) {
        // full march of a ray that reaches the region: keep its intensity there
        init_ray<G>(m, a, I, lane);
        nw = walk_steps1d<G>(m, a, s0, outer, lane, fn);
        sub_boundary(m, a, I, j, lane, true);
        nw += walk_steps1d<G>(m, a, s0 + outer, n - outer, lane, fn);
    } else {
        init_ray<G>(m, a, I, lane);
        nw = walk_steps1d<G>(m, a, s0, n, lane, fn);
    }
    march_state_end<ACC>(m, a, pend, lane);
    return nw;
}

// Eq. 3 on a step without accumulation, applied to the affine map of a run
// of steps: with I_out = A I_in + B for the steps so far, the step's
// I <- I + (S - I)(1 - e^-tau) gives A <- A - A t, B <- B + (S - B) t,
// t = 1 - e^-tau.  The channel window, profile and t are evaluated exactly
// as in march_step, so the run's map reproduces the sequential march up to
// rounding.  Only channels [tlo, thi) are updated; A and B hold them at
// A[t * tile + k - tlo].
template <int G>
__device__ __forceinline__ void affine_step(const DevModel &m, const MarchArgs &a, float *A, float *B,
                                            const Step<G> &st, int lane, int tlo, int thi)
{
    if (lines_off<G>(m, a, st, lane)) return;             // identity map
    float u0, db;
    int klo, khi;
    step_window(m, a, st, u0, db, klo, khi);
    klo = max(klo, tlo);
    khi = min(khi, thi);
    const float my_ks = step_ks(st.kl.x, st.s);
    float Ks[G], Sv[G];
#pragma unroll
    for (int t = 0; t < G; t++) {
        Ks[t] = __shfl_sync(kFull, my_ks, t);
        Sv[t] = __shfl_sync(kFull, st.kl.y, t);
    }
    const bool full = (a.n_lines == G);
    const int tile = a.tile;
    for (int base = klo; base < khi; base += 31) {
        const int k = base + lane;
        const float b0 = ((float)k + u0) * db;
        const float e0 = 0.5f * erfcf(fabsf(b0));
        const float b1 = __shfl_down_sync(kFull, b0, 1);
        const float e1 = __shfl_down_sync(kFull, e0, 1);
        if (lane < 31 && k < khi) {
            const float phi = (b0 >= 0.f) ? (e0 - e1) : ((b1 <= 0.f) ? (e1 - e0) : (1.f - e0 - e1));
#pragma unroll
            for (int t = 0; t < G; t++) {
                if (full || t < a.n_lines) {
                    const float tm = one_minus_exp(Ks[t] * phi);
                    const int o = t * tile + k - tlo;
                    const float av = A[o], bv = B[o];
                    A[o] = fmaf(-av, tm, av);
                    B[o] = fmaf(Sv[t] - bv, tm, bv);
                }
            }
        }
    }
}

// Line-of-sight integration without accumulation (3D maps): lane l keeps
// dI = I - n_bg of channel 31 c + l in dI[c] (c < nchunk, all channels of the
// band) and applies Eq. 3 for one step with K s = Ksv and S - n_bg = src;
// lane 31 only supplies the upper profile edge of lane 30.
template <int CMAX>
__device__ __forceinline__ void los_step(float (&dI)[CMAX], int nchunk, int lane, float Ksv, float src,
                                         float u0, float db)
{
#pragma unroll
    for (int c = 0; c < CMAX; c++) {
        if (c < nchunk) {
            const float b0 = ((float)(31 * c + lane) + u0) * db;
            const float e0 = 0.5f * erfcf(fabsf(b0));
            const float b1 = __shfl_down_sync(kFull, b0, 1);
            const float e1 = __shfl_down_sync(kFull, e0, 1);
            const float phi = (b0 >= 0.f) ? (e0 - e1) : ((b1 <= 0.f) ? (e1 - e0) : (1.f - e0 - e1));
            const float tm = one_minus_exp(Ksv * phi);
            dI[c] = fmaf(src - dI[c], tm, dI[c]);
        }
    }
}

// Writes the brightness T0 dI of the warp's channels for pixel `pix`.
template <int CMAX>
__device__ __forceinline__ void los_store(const float (&dI)[CMAX], int nchunk, int n_ch, int lane, float T0,
                                          long long pix, float *Tout)
{
#pragma unroll
    for (int c = 0; c < CMAX; c++) {
        const int ch = 31 * c + lane;
        if (c < nchunk && lane < 31 && ch < n_ch) Tout[pix * n_ch + ch] = T0 * dI[c];
    }
}

}  // namespace loc
