// k_noalloc.cu -- radiation field of a 1D model without any device allocation.
//
// Some callers of this library cannot call cudaMalloc: code that runs inside
// a host application whose device memory is owned by another allocator (a
// framework pool that must see every byte), or a latency-critical loop where
// cudaMalloc / cudaFree would synchronise the device and stall other work.
// loc_radiation1d_noalloc serves them: the caller passes its own device
// buffers for the inputs and outputs, and every intermediate (ray steps,
// per-shell weights, the SIJ / ESC / NORM accumulators) lives in one
// file-scope device array of fixed size, kNoAllocScratchBytes (2.5 MiB),
// that every GPU which loads the library holds until the process exits.
//
// Host code may not use the array's name as a device address: on the host it
// is only a stand-in symbol.  Its device address is looked up once per device
// with cudaGetSymbolAddress (on the first call made with that device
// current) and reused afterwards.
#include <mutex>

#include "loc_internal.cuh"

namespace loc {

constexpr int kNoAllocMaxShells = 256;
constexpr int kNoAllocMaxRays = 256;
constexpr int kNoAllocMaxLines = 64;
constexpr size_t kNoAllocScratchBytes = 2621440;   // 2.5 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// device address of the scratch array on the current device
static loc_status noalloc_scratch(void **out)
{
    int dev = -1;
    LOC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("loc_radiation1d_noalloc: device index %d not supported", dev);
        return LOC_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("loc_radiation1d_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return LOC_ECUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LOC_OK;
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

// J_ext = SIJ / NORM and beta = ESC / NORM per (shell, line); a shell that
// no ray crossed (NORM = 0) gets the background and beta = 1, as in the
// equilibrium solve.
__global__ void noalloc_finalize(const float2 *acc, const float *norm, const float *nbg,
                                 int K, int T, float *j_ext, float *beta)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * T) return;
    const int c = idx / T, t = idx - (idx / T) * T;
    const float n = norm[c];
    if (n > 0.f) {
        const float2 a = acc[idx];
        j_ext[idx] = a.x / n;
        beta[idx] = a.y / n;
    } else {
        j_ext[idx] = nbg[t];
        beta[idx] = 1.f;
    }
}

}  // namespace loc

using namespace loc;

extern "C" loc_status loc_radiation1d_noalloc(int n_shells, int n_rays, const double *radius,
                                              const float *v_rad, const float *inv_s2sig, int n_ch,
                                              double v_min, double dv, int n_lines, const float *ks,
                                              const float *nbg, double window_sigmas, float *j_ext,
                                              float *beta, void *stream)
{
    if (n_rays == 0) n_rays = n_shells;
    if (n_shells < 1 || n_shells > kNoAllocMaxShells) {
        set_error("loc_radiation1d_noalloc: n_shells = %d, must be in [1, %d]", n_shells, kNoAllocMaxShells);
        return LOC_EINVAL;
    }
    if (n_rays < 1 || n_rays > kNoAllocMaxRays) {
        set_error("loc_radiation1d_noalloc: n_rays = %d, must be in [1, %d]", n_rays, kNoAllocMaxRays);
        return LOC_EINVAL;
    }
    if (n_lines < 1 || n_lines > kNoAllocMaxLines) {
        set_error("loc_radiation1d_noalloc: n_lines = %d, must be in [1, %d]", n_lines, kNoAllocMaxLines);
        return LOC_EINVAL;
    }
    if (n_ch < 1 || n_ch > kMaxChannels || !(dv > 0.0) || !(window_sigmas >= 0.0)) {
        set_error("loc_radiation1d_noalloc: bad channel grid or window");
        return LOC_EINVAL;
    }
    if (!radius || !v_rad || !inv_s2sig || !ks || !nbg || !j_ext || !beta) {
        set_error("loc_radiation1d_noalloc: NULL pointer argument");
        return LOC_EINVAL;
    }
    const int K = n_shells, T = n_lines;
    const long long max_steps = 2ll * n_rays * (K + 1);
    const size_t o_off = 0;
    const size_t o_tan = o_off + align256(sizeof(int) * (n_rays + 1));
    const size_t o_W = o_tan + align256(sizeof(int) * n_rays);
    const size_t o_seg = o_W + align256(sizeof(double) * K);
    const size_t o_acc = o_seg + align256(sizeof(Seg1D) * max_steps);
    const size_t o_norm = o_acc + align256(sizeof(float2) * (size_t)K * T);
    const size_t total = o_norm + align256(sizeof(float) * K);
    if (total > kNoAllocScratchBytes) {
        set_error("loc_radiation1d_noalloc: needs %zu bytes of scratch, maximum %zu", total,
                  kNoAllocScratchBytes);
        return LOC_EINVAL;
    }
    void *base = nullptr;
    loc_status s = noalloc_scratch(&base);
    if (s != LOC_OK) return s;
    unsigned char *b = (unsigned char *)base;
    const cudaStream_t st = (cudaStream_t)stream;

    DevModel m;
    memset(&m, 0, sizeof(m));
    m.geometry = LOC_SHELLS_1D;
    m.n_cells = K;
    m.n_ch = n_ch;
    m.v_min = v_min;
    m.vmin_f = (float)v_min;
    m.dv = dv;
    m.dv_f = (float)dv;
    m.K = K;
    m.n_rays = n_rays;
    m.radius = (double *)radius;
    m.v1d = (float *)v_rad;
    m.inv_s2sig = (float *)inv_s2sig;
    m.ray_off = (int *)(b + o_off);
    m.segs = (Seg1D *)(b + o_seg);
    m.T = T;
    m.ks = (float2 *)ks;
    m.nbg = (float *)nbg;
    m.acc = (float2 *)(b + o_acc);
    m.norm = (float *)(b + o_norm);

    // the array keeps the previous call's contents: clear the accumulators
    LOC_CUDA_TRY(cudaMemsetAsync(m.acc, 0, sizeof(float2) * (size_t)K * T, st));
    LOC_CUDA_TRY(cudaMemsetAsync(m.norm, 0, sizeof(float) * K, st));
    s = launch_geom1d_scratch(m, st, (int *)(b + o_tan), (double *)(b + o_W));
    if (s != LOC_OK) return s;

    // lines per warp as in loc_march: enough warps to cover the GPU
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
        cudaGetLastError();
        nsm = 152;
    }
    int per = T < kMaxLinesPerWarp ? T : kMaxLinesPerWarp;
    while (per > 1 && (long long)n_rays * ((T + per - 1) / per) < 32ll * nsm) per = (per + 1) / 2;
    while (per > 1 && 4ll * per * n_ch * 4 > 200 * 1024) per--;
    MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.per = per;
    a.n_groups = (T + per - 1) / per;
    a.window = (float)window_sigmas;
    a.inv_dv = (float)(1.0 / dv);
    s = launch_march(m, a, st);
    if (s != LOC_OK) return s;
    noalloc_finalize<<<(K * T + 255) / 256, 256, 0, st>>>(m.acc, m.norm, nbg, K, T, j_ext, beta);
    LOC_CUDA_TRY(cudaGetLastError());
    return LOC_OK;
}
