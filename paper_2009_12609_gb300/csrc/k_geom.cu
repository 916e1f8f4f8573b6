// k_geom.cu -- ray geometry set-up kernels.
//
// 1D (Sect. 2.1): concentric shells with outer radii R_k, parallel rays with
// impact parameters p_j = R ((j + 1/2) / n_rays)^a, each standing for the
// annulus between R (j / n_rays)^a and R ((j + 1) / n_rays)^a (a = 1, the
// default, gives equidistant rays and A_j = pi R^2 ((j+1)^2 - j^2) / n_rays^2).  A ray visits
// shells K-1 .. t+1, its tangent shell t (smallest k with R_k > p) in two
// halves, then t+1 .. K-1; step lengths are differences of
// sqrt(R_k^2 - p^2).  The path lengths are precomputed once (the paper does
// the same to speed up its kernel), in FP64, together with the line-of-sight
// velocity at each step's start (Sect. 3.1: Doppler shift at the beginning of
// the step; the outbound half of the tangent shell starts at cos = 0) and the
// step's share of the cell's emission, w = A_j s / W_c with
// W_c = sum over steps in c of A_j s (Sect. 2: with deterministic rays the
// total path length through each cell is available).
//
// 3D (Sect. 2.2): per direction the main axis, the mirrored axes and the
// fixed-point slopes of the ray lattice (see walk3d.cuh).
#include "loc_internal.cuh"
#include "walk3d.cuh"

namespace loc {

// ray j passes at p_j = R ((j + 1/2) / n)^a and stands for the annulus
// between R (j / n)^a and R ((j + 1) / n)^a (a = 1: equidistant rays)
__device__ __forceinline__ double ray_p(const DevModel &m, int j)
{
    const double R = m.radius[m.K - 1];
    if (!(m.ray_power > 0.0) || m.ray_power == 1.0) return (j + 0.5) * R / m.n_rays;
    return R * pow((j + 0.5) / m.n_rays, m.ray_power);
}

__device__ __forceinline__ double ray_area(const DevModel &m, int j)
{
    const double R = m.radius[m.K - 1];
    if (!(m.ray_power > 0.0) || m.ray_power == 1.0)
        return kPI * R * R * ((j + 1.0) * (j + 1.0) - (double)j * j) / ((double)m.n_rays * m.n_rays);
    const double b0 = R * pow((double)j / m.n_rays, m.ray_power);
    const double b1 = R * pow((j + 1.0) / m.n_rays, m.ray_power);
    return kPI * (b1 * b1 - b0 * b0);
}

__device__ __forceinline__ int tangent_shell(const DevModel &m, double p)
{
    int lo = 0, hi = m.K;            // first k with R_k > p (binary search)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (m.radius[mid] > p) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// segment lengths of ray p through shell k (k > t): both crossings equal
__device__ __forceinline__ double shell_chord(const DevModel &m, int k, double p)
{
    const double zo = sqrt(m.radius[k] * m.radius[k] - p * p);
    const double zi = sqrt(m.radius[k - 1] * m.radius[k - 1] - p * p);
    return zo - zi;
}

// one block of kOffThreads threads: tangent shells and per-ray step counts,
// then offsets by an exclusive prefix sum.  Thread i takes a contiguous range
// of rays, so the scan is a per-thread sum, a block scan of those sums and a
// second pass over each range.
constexpr int kOffThreads = 1024;

__global__ void __launch_bounds__(kOffThreads) geom1d_offsets(DevModel m, int *tan)
{
    __shared__ int part[kOffThreads];
    const int tid = threadIdx.x;
    const int per = (m.n_rays + kOffThreads - 1) / kOffThreads;
    const int j0 = min(m.n_rays, tid * per), j1 = min(m.n_rays, j0 + per);
    int sum = 0;
    for (int j = j0; j < j1; j++) {
        const int t = tangent_shell(m, ray_p(m, j));
        tan[j] = t;
        sum += (t < m.K) ? 2 * (m.K - t) : 0;
    }
    part[tid] = sum;
    __syncthreads();
    for (int w = 1; w < kOffThreads; w <<= 1) {          // inclusive scan (Hillis-Steele)
        const int v = (tid >= w) ? part[tid - w] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int off = part[tid] - sum;
    for (int j = j0; j < j1; j++) {
        m.ray_off[j] = off;
        const int t = tan[j];
        off += (t < m.K) ? 2 * (m.K - t) : 0;
    }
    if (tid == kOffThreads - 1) m.ray_off[m.n_rays] = part[tid];
}

// block per shell: W_k = sum_j A_j (length of ray j inside shell k), the
// rays split over the block's threads and summed by a fixed-order reduction
__global__ void geom1d_weights(DevModel m, const int *tan, double *W)
{
    const int k = blockIdx.x;
    if (k >= m.K) return;
    double acc = 0.0;
    for (int j = threadIdx.x; j < m.n_rays; j += blockDim.x) {
        const int t = tan[j];
        if (t > k) continue;
        const double p = ray_p(m, j);
        const double s = (t == k) ? sqrt(m.radius[k] * m.radius[k] - p * p) : shell_chord(m, k, p);
        acc += ray_area(m, j) * 2.0 * s;     // two steps per shell
    }
    __shared__ double red[128];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) W[k] = red[0];
}

// block per ray: step q of ray j (0 <= q < 2 (K - t)), all steps in parallel
__global__ void geom1d_fill(DevModel m, const int *tan, const double *W)
{
    const int j = blockIdx.x;
    if (j >= m.n_rays) return;
    const int t = tan[j];
    if (t >= m.K) return;
    const double p = ray_p(m, j);
    const double A = ray_area(m, j);
    Seg1D *out = m.segs + m.ray_off[j];
    const int nin = m.K - t;                       // inbound steps K-1 .. t
    for (int q = threadIdx.x; q < 2 * nin; q += blockDim.x) {
        int k;
        double s, cosv;
        if (q < nin) {                             // inbound: shell K-1-q
            k = m.K - 1 - q;
            const double zo = sqrt(m.radius[k] * m.radius[k] - p * p);
            s = (k > t) ? zo - sqrt(m.radius[k - 1] * m.radius[k - 1] - p * p) : zo;
            cosv = -zo / m.radius[k];
        } else {                                   // outbound: shell t + (q - nin)
            k = t + (q - nin);
            const double zo = sqrt(m.radius[k] * m.radius[k] - p * p);
            if (k > t) {
                const double zi = sqrt(m.radius[k - 1] * m.radius[k - 1] - p * p);
                s = zo - zi;
                cosv = zi / m.radius[k - 1];
            } else {
                s = zo;
                cosv = 0.0;
            }
        }
        Seg1D sg;
        sg.cell = k;
        sg.s = (float)s;
        sg.vlos = (float)((double)m.v1d[k] * cosv);
        sg.w = (float)((W[k] > 0.0) ? A * s / W[k] : 0.0);
        out[q] = sg;
    }
}

loc_status launch_geom1d(const DevModel &m, cudaStream_t st)
{
    int *tan = nullptr;
    double *W = nullptr;
    LOC_CUDA_TRY(cudaMallocAsync(&tan, sizeof(int) * m.n_rays, st));
    LOC_CUDA_TRY(cudaMallocAsync(&W, sizeof(double) * m.K, st));
    geom1d_offsets<<<1, kOffThreads, 0, st>>>(m, tan);
    geom1d_weights<<<m.K, 128, 0, st>>>(m, tan, W);
    geom1d_fill<<<m.n_rays, 128, 0, st>>>(m, tan, W);
    LOC_CUDA_TRY(cudaGetLastError());
    LOC_CUDA_TRY(cudaFreeAsync(tan, st));
    LOC_CUDA_TRY(cudaFreeAsync(W, st));
    return LOC_OK;
}

// Same set-up with caller-provided temporaries (tan: n_rays ints, W: K
// doubles) instead of stream-ordered allocations.
loc_status launch_geom1d_scratch(const DevModel &m, cudaStream_t st, int *tan, double *W)
{
    geom1d_offsets<<<1, kOffThreads, 0, st>>>(m, tan);
    geom1d_weights<<<m.K, 128, 0, st>>>(m, tan, W);
    geom1d_fill<<<m.n_rays, 128, 0, st>>>(m, tan, W);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// ----------------------------------------------------------------------------
// 3D: trace one root line and record its segments (tests / diagnostics)
// ----------------------------------------------------------------------------
__global__ void trace3d_kernel(DevModel m, int dir, long long i, long long j,
                               long long *cells, long long *dz, long long cap,
                               long long *n_out)
{
    if (threadIdx.x != 0) return;
    const Dir3D D = m.dirs[dir];
    long long n = 0;
    walk_grid3d(D, m.N, i, j, [&](long long c, long long d) {
        if (n < cap) { cells[n] = c; dz[n] = d; }
        n++;
    });
    *n_out = n;
}

// thread per root line: number of segments of one ray simulation
__global__ void count3d_kernel(DevModel m, unsigned long long *total)
{
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per_dir = (long long)m.N * m.N;
    if (item >= per_dir * m.n_dir) return;
    const int dir = (int)(item / per_dir);
    const long long r = item - (long long)dir * per_dir;
    const Dir3D D = m.dirs[dir];
    unsigned long long n = 0;
    walk_grid3d(D, m.N, r / m.N, r % m.N, [&](long long, long long) { n++; });
    atomicAdd(total, n);
}

loc_status launch_count3d(const DevModel &m, unsigned long long *total_dev, cudaStream_t st)
{
    const long long items = (long long)m.N * m.N * m.n_dir;
    LOC_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(unsigned long long), st));
    count3d_kernel<<<(unsigned)((items + 127) / 128), 128, 0, st>>>(m, total_dev);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

loc_status launch_trace3d(const DevModel &m, int dir, long long i, long long j,
                          long long *cells, long long *dz, long long cap,
                          long long *n_out, cudaStream_t st)
{
    trace3d_kernel<<<1, 32, 0, st>>>(m, dir, i, j, cells, dz, cap, n_out);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}


// ----------------------------------------------------------------------------
// 3D direction decomposition (FP64, same arithmetic as the lattice definition)
// ----------------------------------------------------------------------------
__global__ void dir_setup_kernel(const double *dirs, int n_dir, double h0, Dir3D *out)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_dir) return;
    const double d[3] = {dirs[3 * id], dirs[3 * id + 1], dirs[3 * id + 2]};
    int mm = 0;
    if (fabs(d[1]) > fabs(d[mm])) mm = 1;
    if (fabs(d[2]) > fabs(d[mm])) mm = 2;
    Dir3D D;
    D.m = mm;
    D.a = (mm == 0) ? 1 : 0;
    D.b = (mm == 2) ? 1 : 2;
    const double scale = ldexp(1.0, kFixedBits);
    for (int k = 0; k < 3; k++) { D.flip[k] = d[k] < 0.0; D.d[k] = (float)d[k]; }
    D.qa = (long long)floor(scale * fabs(d[D.a]) / fabs(d[mm]) + 0.5);
    D.qb = (long long)floor(scale * fabs(d[D.b]) / fabs(d[mm]) + 0.5);
    const unsigned long long H = 1ull << kFixedBits;
    const unsigned long long step = H << kFixedBits;            // H 2^F
    const unsigned long long first = (H - H / 2) << kFixedBits; // (H - o) 2^F
    const unsigned long long qa = D.qa > 0 ? (unsigned long long)D.qa : 1ull;
    const unsigned long long qb = D.qb > 0 ? (unsigned long long)D.qb : 1ull;
    D.Da = (long long)(step / qa); D.ra = (long long)(step % qa);
    D.Db = (long long)(step / qb); D.rb = (long long)(step % qb);
    D.Qa0 = (long long)(first / qa); D.Ra0 = (long long)(first % qa);
    D.Qb0 = (long long)(first / qb); D.Rb0 = (long long)(first % qb);
    D.ma = ~0ull / qa;
    D.mb = ~0ull / qb;
    D.unit = (float)(h0 / scale / fabs(d[mm]));
    out[id] = D;
}

loc_status launch_dir_setup(const double *dirs_dev, int n_dir, double h0, Dir3D *out,
                            cudaStream_t st)
{
    dir_setup_kernel<<<(n_dir + 63) / 64, 64, 0, st>>>(dirs_dev, n_dir, h0, out);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

// per cell: 1 / (sqrt(2) sigma) with sigma^2 = sigma_turb^2 + k T / m, and the
// packed 3D record {vx, vy, vz, 1/(sqrt(2) sigma)}
__global__ void cell_setup_kernel(DevModel m, const double *sigma_turb, const double *vx,
                                  const double *vy, const double *vz)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m.n_cells) return;
    const double sig = sqrt(sigma_turb[c] * sigma_turb[c] + kKB * m.t_kin[c] / (m.mass_amu * kAMU));
    const float inv = (float)(1.0 / (sqrt(2.0) * sig));
    m.inv_s2sig[c] = inv;
    if (m.vel) m.vel[c] = make_float4((float)vx[c], (float)vy[c], (float)vz[c], inv);
}

loc_status launch_cell_setup(const DevModel &m, const double *sigma_turb, const double *vx,
                             const double *vy, const double *vz, cudaStream_t st)
{
    const long long nb = (m.n_cells + 255) / 256;
    cell_setup_kernel<<<(unsigned)nb, 256, 0, st>>>(m, sigma_turb, vx, vy, vz);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}

}  // namespace loc
