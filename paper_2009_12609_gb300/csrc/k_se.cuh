// k_se.cuh -- per-cell device routines of the level-population step
// (line parameters, statistical equilibrium, excitation temperature), shared
// by the single-model kernels (k_se.cu) and the batched ones (k_batch.cu).
// The equations are those listed at the top of k_se.cu.
#pragma once

#include "loc_internal.cuh"

namespace loc {

constexpr int kSeWarps = 4;   // warps per block of the warp-per-cell solve

__device__ __forceinline__ void line_params_one(const DevModel &m, long long idx)
{
    const long long c = idx / m.T;                 // layout [cell][line]
    const int t = (int)(idx - c * m.T);
    const int u = m.line_u[t], l = m.line_l[t];
    const double nu = m.line_nu[t];
    const double gu = m.g[u], gl = m.g[l];
    const double xl = m.x[c * m.L + l], xu = m.x[c * m.L + u];
    const double diff = gu * xl - gl * xu;
    float2 ks;
    if (fabs(diff) <= 1e-30 * gu * xl || (xl == 0.0 && xu == 0.0)) {
        ks = make_float2(0.f, 0.f);
    } else {
        const double pre = kC * kC * kC * m.line_A[t] / (8.0 * kPI * nu * nu * nu * m.dv);
        const double K = pre * m.n_h2[c] * m.abundance[c] * diff / gl;
        ks = make_float2((float)K, (float)(gl * xu / diff));
        if (K < 0.0) atomicAdd(m.maser_count, 1ull);
    }
    m.ks[idx] = ks;
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

// Statistical equilibrium of cell c by one warp; M: LMAX x (LMAX+2) matrix,
// F: LMAX scratch, R: 2 (T + P) rates, all in shared memory.  Returns this
// lane's part of the convergence metric (reduce over the warp).
template <int LMAX>
__device__ __forceinline__ float se_warp_cell(const DevModel &m, long long c, int ali, int fp64_acc,
                                              int lane, double *M, double *F, double *R)
{
    constexpr int W = LMAX + 2;
    const int nrate = m.T + m.P;
    float my_d = 0.f;
    {
        const int L = m.L;
        const double nrm = fp64_acc ? m.norm64[c] : (double)m.norm[c];
        for (int t = lane; t < m.T; t += 32) {
            const int u = m.line_u[t], l = m.line_l[t];
            const double A = m.line_A[t];
            const long long o = c * m.T + t;
            double J, beta;
            if (nrm > 0.0) {
                double sj, ej;
                if (fp64_acc) { sj = m.acc64[2 * o]; ej = m.acc64[2 * o + 1]; }
                else { const float2 a = m.acc[o]; sj = a.x; ej = a.y; }
                J = sj / nrm;
                beta = ej / nrm;
            } else {
                J = m.nbg64[t];
                beta = 1.0;
            }
            if (!ali) { J = J + (double)m.ks[o].y * (1.0 - beta); beta = 1.0; }
            R[2 * t] = A * (beta + J);                          // u -> l
            R[2 * t + 1] = (m.g[u] / m.g[l]) * A * J;           // l -> u
        }
        const double Tk = m.t_kin[c], nh = m.n_h2[c];
        for (int p = lane; p < m.P; p += 32) {
            const int u = m.coll_u[p], l = m.coll_l[p];
            const double cul = nh * m.coll_k[p];
            R[2 * (m.T + p)] = cul;
            R[2 * (m.T + p) + 1] = cul * (m.g[u] / m.g[l]) * exp(-(m.energy_K[u] - m.energy_K[l]) / Tk);
        }
        for (int i = lane; i < L * W; i += 32) M[i] = 0.0;
        __syncwarp();
        // balance of level i: sum_j x_j R(j -> i) - x_i sum_j R(i -> j) = 0
        if (lane < L) {
            double *row = M + lane * W;
            for (int q = 0; q < nrate; q++) {
                int u, l;
                if (q < m.T) { u = m.line_u[q]; l = m.line_l[q]; }
                else { u = m.coll_u[q - m.T]; l = m.coll_l[q - m.T]; }
                const double rd = R[2 * q], ru = R[2 * q + 1];
                if (lane == l) { row[u] += rd; row[l] -= ru; }
                if (lane == u) { row[u] -= rd; row[l] += ru; }
            }
        }
        __syncwarp();
        for (int j = lane; j <= L; j += 32) M[j] = 1.0;         // row 0: sum(x) = 1
        __syncwarp();
        for (int p = 0; p < L; p++) {
            // pivot: the first row i >= p with the largest |M[i][p]|
            double v = (lane >= p && lane < L) ? fabs(M[lane * W + p]) : -1.0;
            int idx = lane;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, v, off);
                const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
                if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
            }
            if (idx != p) {
                for (int j = lane; j <= L; j += 32) {
                    const double tmp = M[p * W + j];
                    M[p * W + j] = M[idx * W + j];
                    M[idx * W + j] = tmp;
                }
            }
            __syncwarp();
            const double inv = 1.0 / M[p * W + p];
            if (lane > p && lane < L) F[lane] = M[lane * W + p] * inv;
            __syncwarp();
            for (int j = p + lane; j <= L; j += 32) {
                const double pj = M[p * W + j];
                for (int i = p + 1; i < L; i++) M[i * W + j] -= F[i] * pj;
            }
            __syncwarp();
        }
        double xi = 0.0;
        for (int i = L - 1; i >= 0; i--) {
            const double part = warp_sum_d((lane > i && lane < L) ? M[i * W + lane] * xi : 0.0);
            const double xv = (M[i * W + L] - part) / M[i * W + i];
            if (lane == i) xi = xv;
        }
        __syncwarp();
        if (lane < L) {
            m.x_new[c * L + lane] = xi;
            F[lane] = xi;
        }
        __syncwarp();
        const double *xo = m.x + c * L;
        for (int t = lane; t < m.T; t += 32) {
            if (F[m.line_u[t]] < 1e-6) continue;
            const double a = tex_of(m, t, xo);
            if (a == 0.0) continue;
            const double b = tex_of(m, t, F);
            my_d = fmaxf(my_d, (float)(fabs(b - a) / fabs(a)));
        }
    }
    return my_d;
}

}  // namespace loc
