// k_se.cu -- level populations: LTE start, background, line parameters,
// statistical-equilibrium solve and excitation temperatures.
//
// Line parameters (Eq. 2, Eq. 3): the optical depth of a step of length s in
// channel k is tau = K phi_k s with
//   K = c^3 A / (8 pi nu^3 dv) n_mol (x_l g_u / g_l - x_u)
// and the source function in occupation units is
//   S = g_l x_u / (g_u x_l - g_l x_u).
// A vanishing population difference (|g_u x_l - g_l x_u| <= 1e-30 g_u x_l)
// gives K = 0, S = 0; inverted populations (K < 0) are kept and counted.
//
// Statistical equilibrium (Sect. 2, ALI paragraph): the radiative rates use
// the cell averages J_ext = SIJ / NORM and beta = ESC / NORM in place of
// B_lu I_nu; with ALI the locally absorbed photons are removed from J and
// A_ul is scaled by beta:
//   R_lu = (g_u / g_l) A J_ext,   R_ul = A (beta + J_ext);
// without ALI J = J_ext + S (1 - beta) and beta = 1.  Collisions with H2:
// C_ul = n_H2 k_ul, C_lu = C_ul (g_u / g_l) exp(-(E_u - E_l) / T_kin).  The
// first balance equation is replaced by sum(x) = 1 and the system is solved
// in FP64 by Gaussian elimination with partial pivoting, one cell per
// warp.  The same kernel reports max |dT_ex| / |T_ex| over cells and lines
// whose upper level holds at least 1e-6 of the molecules.
#include "k_se.cuh"

namespace loc {

__global__ void lte_kernel(DevModel m)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.n_cells) return;
    double z = 0.0;
    double *x = m.x + c * m.L;
    for (int i = 0; i < m.L; i++) {
        x[i] = m.g[i] * exp(-m.energy_K[i] / m.t_kin[c]);
        z += x[i];
    }
    for (int i = 0; i < m.L; i++) x[i] /= z;
}

// FP64 elementwise kernels of small models run in 32-thread blocks so that
// their warps spread over the SMs' FP64 pipes
static int fp64_block(long long n) { return n <= 152ll * 256 ? 32 : 256; }

loc_status launch_lte(const DevModel &m, cudaStream_t st)
{
    const int bs = fp64_block(m.n_cells);
    lte_kernel<<<(unsigned)((m.n_cells + bs - 1) / bs), bs, 0, st>>>(m);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// background occupation n_bg = 1 / (exp(h nu / k T_bg) - 1) per line (Eq. 1:
// rays enter carrying the background field)
__global__ void bg_kernel(DevModel m)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m.T) return;
    const double n = (m.t_bg > 0.0) ? 1.0 / expm1(kH * m.line_nu[t] / (kKB * m.t_bg)) : 0.0;
    m.nbg64[t] = n;
    m.nbg[t] = (float)n;
}

loc_status launch_bg(const DevModel &m, cudaStream_t st)
{
    bg_kernel<<<(m.T + 63) / 64, 64, 0, st>>>(m);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// zero_acc: 0 keep the accumulators; 1 (2) also clear the FP32 (FP64)
// accumulators of entry idx, NORM of its cell and the convergence metric,
// the start of a ray simulation in the ALI loop
__global__ void line_params_kernel(DevModel m, int zero_acc, double cutoff)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m.T * m.n_cells) return;
    line_params_one(m, idx, cutoff);
    if (zero_acc) {
        acc_zero(m, idx, idx / m.T, zero_acc == 2, (idx % m.T) == 0);
        if (idx == 0) *m.dtex_bits = 0u;
    }
}

loc_status launch_line_params(const DevModel &m, cudaStream_t st, int zero_acc, double cutoff)
{
    const long long n = (long long)m.T * m.n_cells;
    const int bs = fp64_block(n);
    line_params_kernel<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(m, zero_acc, cutoff);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// One thread per cell (large models: enough cells to fill the GPU, FP64
// throughput is the limit).  Same rate assembly order as the warp version.
template <int LMAX>
__global__ void __launch_bounds__(128) se_thread_kernel(DevModel m, int ali, int fp64_acc, int want_dtex,
                                                        int next, double cutoff)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float my_d = 0.f;
    if (c < m.n_cells) {
        const int L = m.L;
        double M[LMAX][LMAX + 1];
        for (int i = 0; i < L; i++)
            for (int j = 0; j <= L; j++) M[i][j] = 0.0;
        const double nrm = norm_value(m, c, fp64_acc);
        for (int t = 0; t < m.T; t++) {
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
                const double inv_nrm = recip(nrm);
                J = sj * inv_nrm;
                beta = ej * inv_nrm;
                if (!ali) { J = J + (double)m.ks[o].y * (1.0 - beta); beta = 1.0; }
            } else {
                J = m.nbg64[t];
                beta = 1.0;
            }
            const double rd = A * (beta + J);
            const double ru = m.g[u] * recip(m.g[l]) * A * J;
            M[l][u] += rd; M[l][l] -= ru;
            M[u][u] -= rd; M[u][l] += ru;
        }
        for (int p = 0; p < m.P; p++) {
            const int u = m.coll_u[p], l = m.coll_l[p];
            const double2 cr = coll_rate(m, c, p);
            M[l][u] += cr.x; M[l][l] -= cr.y;
            M[u][u] -= cr.x; M[u][l] += cr.y;
        }
        for (int j = 0; j < L; j++) M[0][j] = 1.0;
        M[0][L] = 1.0;
        for (int p = 0; p < L; p++) {
            // magnitudes compared as the bit patterns of non-negative
            // doubles (ordered like the values; integer compares)
            int piv = p;
            long long best = __double_as_longlong(fabs(M[p][p]));
            for (int i = p + 1; i < L; i++) {
                const long long a = __double_as_longlong(fabs(M[i][p]));
                if (a > best) { best = a; piv = i; }
            }
            if (piv != p)
                for (int j = p; j <= L; j++) { const double tmp = M[p][j]; M[p][j] = M[piv][j]; M[piv][j] = tmp; }
            const double inv = recip(M[p][p]);
            for (int i = p + 1; i < L; i++) {
                const double f = M[i][p] * inv;
                if ((__double_as_longlong(f) << 1) == 0) continue;     // f == +-0, integer test
                for (int j = p; j <= L; j++) M[i][j] -= f * M[p][j];
            }
        }
        double xs[LMAX];
        for (int i = L - 1; i >= 0; i--) {
            double a = M[i][L];
            for (int j = i + 1; j < L; j++) a -= M[i][j] * xs[j];
            xs[i] = a * recip(M[i][i]);
        }
        const double *xo = m.x + c * L;
        double *xn = m.x_new + c * L;
        for (int i = 0; i < L; i++) xn[i] = xs[i];
        for (int t = 0; want_dtex && t < m.T; t++) {
            if (xs[m.line_u[t]] < 1e-6) continue;
            const double a = tex_of(m, t, xo);
            if (a == 0.0) continue;
            const double b = tex_of(m, t, xs);
            my_d = fmaxf(my_d, (float)(fabs(b - a) / fabs(a)));
        }
        for (int t = 0; next && t < m.T; t++) next_line_params(m, c, t, xs, fp64_acc, cutoff, t == 0);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) my_d = fmaxf(my_d, __shfl_xor_sync(0xffffffffu, my_d, off));
    if ((threadIdx.x & 31) == 0 && my_d > 0.f) atomicMax(m.dtex_bits, __float_as_uint(my_d));
}

// Small models: one segment of LMAX lanes per cell, 32 / LMAX cells per warp
// (se_seg_cell in k_se.cuh).  On GB300 an FP64 warp instruction occupies the
// FP64 pipe for many cycles whatever the number of active lanes, so packing
// cells into one warp divides the FP64 instructions per cell.
// at or above this many cells one thread per cell already fills the GPU
constexpr long long kSeThreadCells = 1ll << 16;

template <int LMAX>
__global__ void __launch_bounds__(kSeWarps * 32) se_kernel(DevModel m, int ali, int fp64_acc, int want_dtex,
                                                            int next, double cutoff)
{
    constexpr int LW = LMAX;                        // lanes per cell
    constexpr int CPW = 32 / LW;                    // cells per warp
    constexpr int W = LMAX + 2;                     // row stride: L columns + rhs + pad
    constexpr int SEG = LMAX * W + LMAX;            // doubles per segment
    extern __shared__ double se_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int seg = lane / LW, sl = lane - seg * LW;
    double *M = se_smem + (size_t)(wid * CPW + seg) * SEG;
    const long long c0 = ((long long)blockIdx.x * (blockDim.x >> 5) + wid) * CPW;
    if (c0 >= m.n_cells) return;                    // whole warp
    long long c = c0 + seg;
    const bool valid = c < m.n_cells;
    if (!valid) c = m.n_cells - 1;                  // repeat a real cell, store nothing
    float my_d = se_seg_cell<LMAX, LW>(m, c, valid, ali, fp64_acc, sl, M, M + LMAX * W, want_dtex != 0,
                                       next != 0, cutoff);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) my_d = fmaxf(my_d, __shfl_xor_sync(0xffffffffu, my_d, off));
    if (lane == 0 && my_d > 0.f) atomicMax(m.dtex_bits, __float_as_uint(my_d));
}

template <int LMAX>
static loc_status launch_se_l(const DevModel &m, int ali, int fp64_acc, int want_dtex, int next,
                              double cutoff, cudaStream_t st)
{
    if (m.n_cells >= kSeThreadCells) {
        const unsigned nbt = (unsigned)((m.n_cells + 127) / 128);
        se_thread_kernel<LMAX><<<nbt, 128, 0, st>>>(m, ali, fp64_acc, want_dtex, next, cutoff);
        LOC_CUDA_TRY(cudaGetLastError());
        return LOC_OK;
    }
    constexpr int CPW = 32 / LMAX;
    // the FP64 pipes are per SM: a small model spreads its warps one per
    // block (one per SM) instead of packing kSeWarps warps on fewer SMs
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 152;
    }
    const long long warps = (m.n_cells + CPW - 1) / CPW;
    const int wpb = (warps <= 2ll * nsm) ? 1 : kSeWarps;
    const size_t smem = sizeof(double) * wpb * CPW * (LMAX * (LMAX + 2) + LMAX);
    LOC_CUDA_TRY(cudaFuncSetAttribute(se_kernel<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const long long cells_per_block = (long long)wpb * CPW;
    const unsigned nb = (unsigned)((m.n_cells + cells_per_block - 1) / cells_per_block);
    se_kernel<LMAX><<<nb, wpb * 32, smem, st>>>(m, ali, fp64_acc, want_dtex, next, cutoff);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_se(const DevModel &m, int ali, int fp64_acc, cudaStream_t st, int want_dtex, int next,
                     double cutoff)
{
    if (m.L <= 4) return launch_se_l<4>(m, ali, fp64_acc, want_dtex, next, cutoff, st);
    if (m.L <= 8) return launch_se_l<8>(m, ali, fp64_acc, want_dtex, next, cutoff, st);
    if (m.L <= 16) return launch_se_l<16>(m, ali, fp64_acc, want_dtex, next, cutoff, st);
    return launch_se_l<32>(m, ali, fp64_acc, want_dtex, next, cutoff, st);
}

// Collision rate table of the model (n_H2 and T_kin are fixed): one thread
// per (cell, pair).
__global__ void coll_rates_kernel(DevModel m, double2 *out)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m.n_cells * m.P) return;
    const long long c = idx / m.P;
    const int p = (int)(idx - c * m.P);
    const int u = m.coll_u[p], l = m.coll_l[p];
    const double cul = m.n_h2[c] * m.coll_k[p];
    out[idx] = make_double2(cul, cul * (m.g[u] / m.g[l]) * exp(-(m.energy_K[u] - m.energy_K[l]) / m.t_kin[c]));
}

loc_status launch_coll_rates(const DevModel &m, double2 *out, cudaStream_t st)
{
    const long long n = m.n_cells * m.P;
    if (n == 0) return LOC_OK;
    coll_rates_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, out);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

__global__ void tex_kernel(DevModel m, int t, double *out)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.n_cells) return;
    out[m.leaf_perm ? m.leaf_perm[c] : c] = tex_of(m, t, m.x + c * m.L);
}

__global__ void permute_rows_kernel(const int *perm, long long n, int w, const double *src, double *dst,
                                    int to_api)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * w) return;
    const long long i = idx / w, l = idx - i * w;
    if (to_api) dst[(long long)perm[i] * w + l] = src[idx];
    else dst[idx] = src[(long long)perm[i] * w + l];
}

loc_status launch_permute_rows(const int *perm, long long n, int w, const double *src, double *dst,
                               int to_api, cudaStream_t st)
{
    const long long tot = n * w;
    if (tot == 0) return LOC_OK;
    permute_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(perm, n, w, src, dst, to_api);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_tex(const DevModel &m, int t, double *out_dev, cudaStream_t st)
{
    tex_kernel<<<(unsigned)((m.n_cells + 255) / 256), 256, 0, st>>>(m, t, out_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// Convergence metric between the populations x0 and m.x: max over cells
// and over lines whose upper level now holds >= 1e-6 of |dT_ex| / |T_ex|,
// as the solve computes it (one thread per (cell, line)).
__global__ void dtex_kernel(DevModel m, const double *x0)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (idx < (long long)m.T * m.n_cells) {
        const long long c = idx / m.T;
        const int t = (int)(idx - c * m.T);
        const double *xn = m.x + c * m.L;
        if (!(xn[m.line_u[t]] < 1e-6)) {
            const double a = tex_of(m, t, x0 + c * m.L);
            if (a != 0.0) d = (float)(fabs(tex_of(m, t, xn) - a) / fabs(a));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, off));
    if ((threadIdx.x & 31) == 0 && d > 0.f) atomicMax(m.dtex_bits, __float_as_uint(d));
}

loc_status launch_dtex(const DevModel &m, const double *x0, cudaStream_t st)
{
    const long long n = (long long)m.T * m.n_cells;
    dtex_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, x0);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// accumulators -> FP64 arrays (diagnostics)
__global__ void acc_to_f64_kernel(DevModel m, int fp64_acc, double *sij, double *esc, double *norm)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)m.T * m.n_cells;
    if (idx < n) {                               // idx = c * T + t -> out[t][c] (level order)
        const long long c = idx / m.T;
        const long long t = idx - c * m.T;
        const long long o = t * m.n_cells + (m.leaf_perm ? m.leaf_perm[c] : c);
        const double2 a = acc_value(m, idx, fp64_acc);
        if (sij) sij[o] = a.x;
        if (esc) esc[o] = a.y;
    }
    if (idx < m.n_cells && norm) norm[m.leaf_perm ? m.leaf_perm[idx] : idx] = norm_value(m, idx, fp64_acc);
}

loc_status launch_acc_to_f64(const DevModel &m, int fp64_acc, double *sij, double *esc,
                             double *norm, cudaStream_t st)
{
    const long long n = (long long)m.T * m.n_cells;
    acc_to_f64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m, fp64_acc, sij, esc, norm);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

}  // namespace loc

namespace {
__global__ void recip_check_kernel(const double *in, double *out, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = loc::recip(in[i]);
}
}  // namespace

// Numerical self-check of the solve's reciprocal (see recip in k_se.cuh).
extern "C" loc_status loc_check_recip(const double *d, double *r, size_t n)
{
    if (n == 0) return LOC_OK;
    if (!d || !r) { loc::set_error("loc_check_recip: NULL buffer"); return LOC_EINVAL; }
    double *buf = nullptr;
    if (cudaMalloc(&buf, 2 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        loc::set_error("loc_check_recip: device allocation failed");
        return LOC_ENOMEM;
    }
    loc_status st = LOC_OK;
    if (cudaMemcpy(buf, d, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) st = LOC_ECUDA;
    if (st == LOC_OK) {
        recip_check_kernel<<<(unsigned)((n + 255) / 256), 256>>>(buf, buf + n, (long long)n);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(r, buf + n, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = LOC_ECUDA;
    }
    if (st != LOC_OK) loc::set_error("loc_check_recip: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(buf);
    return st;
}
