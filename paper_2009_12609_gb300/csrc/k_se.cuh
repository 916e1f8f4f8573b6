// k_se.cuh -- per-cell device routines of the level-population step
// (line parameters, statistical equilibrium, excitation temperature), shared
// by the single-model kernels (k_se.cu) and the batched ones (k_batch.cu).
// The equations are those listed at the top of k_se.cu.
#pragma once

#include "loc_internal.cuh"

namespace loc {

constexpr int kSeWarps = 4;   // warps per block of the segment-per-cell solve

// 1/d in FP64 without a division (the solve is bound by FP64 instruction
// throughput on GB300, and a division costs several FP64 instructions): the
// exponent of d is handled as an integer, the leading 23 fraction bits get an
// FP32 reciprocal from the SFU (rcp.approx, relative error about 2^-23), and
// two Newton-Raphson steps r <- r + r (1 - d r) square the relative error
// each time (2^-23 -> 2^-46 -> below the rounding of the last step), so the
// result is within about one FP64 ulp of 1/d.  Zero, subnormal, huge,
// infinite and NaN inputs (biased exponent outside [2, 2044]) take 1.0 / d.
__device__ __forceinline__ double recip(double d)
{
    const long long b = __double_as_longlong(d);
    const int be = (int)((b >> 52) & 0x7ff);
    if (be < 2 || be > 2044) return 1.0 / d;
    const float mf = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));   // mantissa in [1, 2)
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));                      // in (0.5, 1]
    const int rb = __float_as_int(rf);
    const long long e = (long long)(((rb >> 23) & 0xff) - 127 + 2046 - be);        // in [1, 2046]
    double r = __longlong_as_double((b & (long long)0x8000000000000000ull) | (e << 52) |
                                    ((long long)(rb & 0x7fffff) << 29));
    double t = fma(-d, r, 1.0);
    r = fma(r, t, r);
    t = fma(-d, r, 1.0);
    return fma(r, t, r);
}

// {K, S} of a line switched off in this cell by the truncation below
__device__ __forceinline__ bool line_off(float2 ks)
{
    return __float_as_uint(ks.x) == 0x80000000u;
}

// cutoff > 0: a line whose two levels both hold less than cutoff of the
// molecules in this cell is marked off there: {K, S} = {-0, 0} (an ordinary
// line never has K = -0)
__device__ __forceinline__ void line_params_at(const DevModel &m, long long c, int t, double xl, double xu,
                                               double cutoff)
{
    const long long idx = c * m.T + t;             // layout [cell][line]
    const int u = m.line_u[t], l = m.line_l[t];
    const double nu = m.line_nu[t];
    const double gu = m.g[u], gl = m.g[l];
    const double diff = gu * xl - gl * xu;
    float2 ks;
    if (cutoff > 0.0 && xl < cutoff && xu < cutoff) {
        ks = make_float2(-0.f, 0.f);                            // line off in this cell
    } else if (fabs(diff) <= 1e-30 * gu * xl || (xl == 0.0 && xu == 0.0)) {
        ks = make_float2(0.f, 0.f);
    } else {
        const double pre = kC * kC * kC * m.line_A[t] * recip(8.0 * kPI * nu * nu * nu * m.dv * gl);
        const double K = pre * m.n_h2[c] * m.abundance[c] * diff;
        float kf = (float)K;
        if (kf == 0.f) kf = 0.f;                    // an underflow to -0 is not the mark
        ks = make_float2(kf, (float)(gl * xu * recip(diff)));
        if (K < 0.0) atomicAdd(m.maser_count, 1ull);
    }
    m.ks[idx] = ks;
}

// entry idx = c T + t from the current populations m.x
__device__ __forceinline__ void line_params_one(const DevModel &m, long long idx, double cutoff = 0.0)
{
    const long long c = idx / m.T;
    const int t = (int)(idx - c * m.T);
    line_params_at(m, c, t, m.x[c * m.L + m.line_l[t]], m.x[c * m.L + m.line_u[t]], cutoff);
}

// The solve of one ALI iteration prepares the next one in the same pass:
// line t's {K, S} from the cell's new populations xn, and its accumulators
// cleared (lane `first` also clears NORM) -- what line_params_kernel does at
// the start of an iteration, without the launch.
__device__ __forceinline__ void next_line_params(const DevModel &m, long long c, int t, const double *xn,
                                                 int fp64_acc, double cutoff, bool first)
{
    line_params_at(m, c, t, xn[m.line_l[t]], xn[m.line_u[t]], cutoff);
    acc_zero(m, c * m.T + t, c, fp64_acc, first);
}

__device__ __forceinline__ double tex_of(const DevModel &m, int t, const double *x)
{
    const int u = m.line_u[t], l = m.line_l[t];
    const double xu = x[u], xl = x[l];
    if (!(xu > 0.0) || !(xl > 0.0)) return 0.0;
    return (kH * m.line_nu[t] / kKB) / log(m.g[u] * xl / (m.g[l] * xu));
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Collision rates of pair p in cell c: {C_ul, C_lu} with C_ul = n_H2 k_ul and
// C_lu = C_ul (g_u / g_l) exp(-(E_u - E_l) / T_kin) (detailed balance); from
// the per-model table when the model has one (T_kin and n_H2 are fixed).
__device__ __forceinline__ double2 coll_rate(const DevModel &m, long long c, int p)
{
    if (m.coll_rates) return m.coll_rates[c * m.P + p];
    const int u = m.coll_u[p], l = m.coll_l[p];
    const double cul = m.n_h2[c] * m.coll_k[p];
    return make_double2(cul, cul * (m.g[u] / m.g[l]) * exp(-(m.energy_K[u] - m.energy_K[l]) / m.t_kin[c]));
}

// Statistical equilibrium of cell c by a segment of LW lanes (LW a power of
// two <= 32, L <= LMAX <= LW; sl = lane within the segment; every segment of
// the warp runs the same control flow).  M: L x W matrix (W = LMAX + 2; L
// columns and the right-hand side), F: LMAX scratch, both in shared memory
// and owned by the segment.  With valid == false the segment repeats the work
// of a real cell but stores nothing.  Returns this lane's part of the
// convergence metric (0 when want_dtex is false).
//
// Balance of level i: sum_j x_j R(j -> i) - x_i sum_j R(i -> j) = 0, i.e.
// M[i][j] = R(j -> i) off the diagonal and M[i][i] = -sum_j M[j][i].  Each
// level pair carries at most one line and one collision pair (checked when
// the molecule is set), so the lanes of one pass write distinct entries: lines
// first, then collisions, then the diagonal as column sums -- a fixed order.
// Elimination with partial pivoting runs with lanes over columns; back
// substitution with lanes over rows, one broadcast per unknown.
// next: also prepare the next iteration (next_line_params) with `cutoff`.
template <int LMAX, int LW>
__device__ __forceinline__ float se_seg_cell(const DevModel &m, long long c, bool valid, int ali,
                                             int fp64_acc, int sl, double *M, double *F,
                                             bool want_dtex = true, bool next = false,
                                             double cutoff = 0.0)
{
    constexpr int W = LMAX + 2;
    const int L = m.L;
    for (int i = sl; i < L * W; i += LW) M[i] = 0.0;
    __syncwarp();
    const double nrm = norm_value(m, c, fp64_acc);
    const double inv_nrm = (nrm > 0.0) ? recip(nrm) : 0.0;
    for (int b = 0; b < m.T; b += LW) {
        const int t = b + sl;
        if (t < m.T) {
            const int u = m.line_u[t], l = m.line_l[t];
            const double A = m.line_A[t];
            const long long o = c * m.T + t;
            double J, beta;
            if (m.trunc && line_off(m.ks[o])) {              // line off in this cell
                J = m.nbg64[t];
                beta = 1.0;
            } else if (nrm > 0.0) {
                double sj, ej;
                const double2 a = acc_value(m, o, fp64_acc);
                sj = a.x;
                ej = a.y;
                J = sj * inv_nrm;
                beta = ej * inv_nrm;
                if (!ali) { J = J + (double)m.ks[o].y * (1.0 - beta); beta = 1.0; }
            } else {
                J = m.nbg64[t];
                beta = 1.0;
            }
            M[l * W + u] += A * (beta + J);                     // u -> l
            M[u * W + l] += m.g[u] * recip(m.g[l]) * A * J;     // l -> u
        }
    }
    __syncwarp();
    // collision rates: the pairs of four rounds are fetched before any is
    // added (independent loads in flight instead of one load per round trip)
    for (int b = 0; b < m.P; b += 4 * LW) {
        double2 cr[4];
        int pu[4], pl[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int p = b + q * LW + sl;
            pu[q] = -1;
            if (p < m.P) {
                pu[q] = m.coll_u[p];
                pl[q] = m.coll_l[p];
                cr[q] = coll_rate(m, c, p);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (pu[q] >= 0) {
                M[pl[q] * W + pu[q]] += cr[q].x;
                M[pu[q] * W + pl[q]] += cr[q].y;
            }
        }
    }
    __syncwarp();
    for (int j = sl; j < L; j += LW) {
        double out = 0.0;
        for (int i = 0; i < L; i++)
            if (i != j) out += M[i * W + j];
        M[j * W + j] = -out;
    }
    __syncwarp();
    for (int j = sl; j <= L; j += LW) M[j] = 1.0;               // row 0: sum(x) = 1
    __syncwarp();
    double my_inv = 0.0;                                         // lane p: 1 / U[p][p]
    for (int p = 0; p < L; p++) {
        // pivot: the first row i >= p with the largest |M[i][p]|.  The
        // magnitudes are compared as the bit patterns of non-negative doubles,
        // which order like their values, so the search issues integer
        // compares instead of FP64 ones; -1 marks rows outside [p, L)
        long long v = (sl >= p && sl < L) ? __double_as_longlong(fabs(M[sl * W + p])) : -1ll;
        int idx = sl;
#pragma unroll
        for (int off = LW / 2; off > 0; off >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, v, off);
            const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        if (idx != p) {
            for (int j = p + sl; j <= L; j += LW) {
                const double tmp = M[p * W + j];
                M[p * W + j] = M[idx * W + j];
                M[idx * W + j] = tmp;
            }
        }
        __syncwarp();
        const double inv = recip(M[p * W + p]);
        if (sl == p) my_inv = inv;
        if (sl > p && sl < L) F[sl] = M[sl * W + p] * inv;
        __syncwarp();
        for (int j = p + sl; j <= L; j += LW) {
            const double pj = M[p * W + j];
            for (int i = p + 1; i < L; i++) M[i * W + j] -= F[i] * pj;
        }
        __syncwarp();
    }
    // back substitution: lane r keeps the reduced right-hand side of row r
    double rhs = (sl < L) ? M[sl * W + L] : 0.0;
    double xi = 0.0;
    for (int i = L - 1; i >= 0; i--) {
        const double x = __shfl_sync(0xffffffffu, rhs * my_inv, i, LW);
        if (sl == i) xi = x;
        if (sl < i) rhs = fma(-M[sl * W + i], x, rhs);
    }
    __syncwarp();
    if (sl < L) {
        if (valid) m.x_new[c * L + sl] = xi;
        F[sl] = xi;
    }
    __syncwarp();
    float my_d = 0.f;
    if (valid && want_dtex) {
        const double *xo = m.x + c * L;
        for (int t = sl; t < m.T; t += LW) {
            if (F[m.line_u[t]] < 1e-6) continue;
            const double a = tex_of(m, t, xo);
            if (a == 0.0) continue;
            const double b = tex_of(m, t, F);
            my_d = fmaxf(my_d, (float)(fabs(b - a) / fabs(a)));
        }
    }
    if (valid && next)
        for (int t = sl; t < m.T; t += LW) next_line_params(m, c, t, F, fp64_acc, cutoff, t == 0);
    __syncwarp();
    return my_d;
}

}  // namespace loc
