// noalloc.cu -- allocation-free entry point of libafns (declared in include/afns.h).
//
// af_dt_max_noalloc computes the CFL time step of Eq. (13) for a 2D FP64 state
// that the caller already holds on the device, without allocating anything. Its
// only scratch is a file-scope device array: one (inviscid, viscous) pair of
// maxima per chunk of AF_NOALLOC_CHUNK cells, for at most AF_NOALLOC_MAX_CHUNKS
// chunks. Every GPU that loads the library keeps that array until the process
// exits. The paper has no counterpart of this call.
#include <cuda.h>   // CUcontext (the driver calls go through the runtime's entry-point query)
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "afns.h"

namespace {

constexpr int kChunk = AF_NOALLOC_CHUNK;          // cells per block
constexpr int kMaxChunks = AF_NOALLOC_MAX_CHUNKS;  // blocks per call
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

// Partial maxima of one call; every call overwrites the slots it uses. A chunk
// holding an inadmissible or non-finite cell average stores NaN as its
// inviscid maximum.
static __device__ __align__(256) double g_dt_scratch[2 * kMaxChunks];

// Device address of g_dt_scratch per device, with the id of the CUDA context it
// was taken in (host code may not use the symbol itself: on the host it names a
// stand-in, not device memory). A new context on the device (after a device
// reset) gets the address looked up again.
struct ScratchAddr {
    unsigned long long ctx_id;
    double *addr;
};
ScratchAddr g_scratch[kMaxDevices] = {};
std::mutex g_setup_lock;

__global__ void __launch_bounds__(kThreads) k_noalloc_partial(const double *avg, long long cells, double dx, double dy,
                                                              double gamma, double mu, double Pr, double cfl_c,
                                                              double cfl_v, double *scratch)
{
    const long long begin = (long long)blockIdx.x * kChunk;
    const long long end = begin + kChunk < cells ? begin + kChunk : cells;
    double m1 = 0.0, m2 = 0.0;
    int bad = 0;
    const double g1 = gamma - 1.0;
    for (long long t = begin + threadIdx.x; t < end; t += blockDim.x) {
        const double rho = avg[t], mx = avg[cells + t], my = avg[2 * cells + t], E = avg[3 * cells + t];
        const double p = g1 * (E - (mx * mx + my * my) / (2.0 * rho));
        // the bound of Eq. (13) is defined on admissible states only
        if (!(rho > 0.0) || !(p > 0.0) || !isfinite(rho) || !isfinite(mx) || !isfinite(my) || !isfinite(E)) {
            bad = 1;
            continue;
        }
        const double c = sqrt(gamma * p / rho);
        const double rv = fmax(4.0 * mu / (3.0 * rho), gamma * mu / (Pr * rho));
        m1 = fmax(m1, fmax((fabs(mx / rho) + c) / (cfl_c * dx), (fabs(my / rho) + c) / (cfl_c * dy)));
        m2 = fmax(m2, fmax(rv / (cfl_v * dx * dx), rv / (cfl_v * dy * dy)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __shared__ double s1[kThreads / 32], s2[kThreads / 32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s1[wid] = m1, s2[wid] = m2;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) m1 = fmax(m1, s1[k]), m2 = fmax(m2, s2[k]);
        scratch[2 * blockIdx.x] = bad ? (double)NAN : m1;
        scratch[2 * blockIdx.x + 1] = m2;
    }
}

__global__ void __launch_bounds__(kThreads) k_noalloc_final(const double *scratch, int nchunks, double *dt_out)
{
    double m1 = 0.0, m2 = 0.0;
    int bad = 0;
    for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
        const double a = scratch[2 * k];
        if (isnan(a)) bad = 1;
        else m1 = fmax(m1, a);
        m2 = fmax(m2, scratch[2 * k + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __shared__ double s1[kThreads / 32], s2[kThreads / 32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s1[wid] = m1, s2[wid] = m2;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) m1 = fmax(m1, s1[k]), m2 = fmax(m2, s2[k]);
        *dt_out = bad ? (double)NAN : 1.0 / (m1 + m2);
    }
}

typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

// Id of the calling thread's current CUDA context (0 if there is none yet).
static cudaError_t current_context_id(unsigned long long *id)
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f)
            return cudaErrorNotSupported;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess || !g)
            return cudaErrorNotSupported;
        get_current = (PfnCtxGetCurrent)f;
        get_id = (PfnCtxGetId)g;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

// Device address of the scratch array on the current device: looked up with
// cudaGetSymbolAddress once per device and CUDA context (the lookup also makes
// the runtime's primary context current), then reused.
static cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_setup_lock);
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    if (id == 0 || g_scratch[dev].addr == nullptr || g_scratch[dev].ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dt_scratch);
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        g_scratch[dev].addr = (double *)p;
        g_scratch[dev].ctx_id = id;
    }
    *out = g_scratch[dev].addr;
    return cudaSuccess;
}

}  // namespace

extern "C" af_status af_dt_max_noalloc(const af_grid *grid, double gamma, double mu, double Pr, const af_opts *opts,
                                       const double *avg_dev, double *dt_dev, void *cuda_stream)
{
    if (!grid || !avg_dev || !dt_dev || grid->dim != 2) return AF_EINVAL;
    if (grid->n[0] < 1 || grid->n[1] < 1 || !(grid->hi[0] > grid->lo[0]) || !(grid->hi[1] > grid->lo[1]))
        return AF_EINVAL;
    if (!(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0)) return AF_EINVAL;
    const long long cells = (long long)grid->n[0] * grid->n[1];
    const long long nchunks = (cells + kChunk - 1) / kChunk;
    if (nchunks > kMaxChunks) return AF_EINVAL;   // larger than the static scratch: nothing launched
    af_opts d;
    if (!opts) {
        af_opts_default(2, &d);
        opts = &d;
    }
    if (!(opts->cfl_c > 0.0) || !(opts->cfl_v > 0.0)) return AF_EINVAL;
    if (opts->kappa_off != 0 && opts->kappa_off != 1) return AF_EINVAL;
    // without heat conduction the bound has no conduction term (as in af_create)
    const double pr_cfl = opts->kappa_off ? INFINITY : Pr;
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return AF_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const double dx = (grid->hi[0] - grid->lo[0]) / grid->n[0], dy = (grid->hi[1] - grid->lo[1]) / grid->n[1];
    double cfl_c = opts->cfl_c, cfl_v = opts->cfl_v;
    int nch = (int)nchunks;
    // launched through cudaLaunchKernel so that each launch's own status is read
    // (an error left over from unrelated earlier work is not reported as ours)
    void *a1[] = {(void *)&avg_dev, (void *)&cells, (void *)&dx, (void *)&dy, (void *)&gamma, (void *)&mu,
                  (void *)&pr_cfl, (void *)&cfl_c, (void *)&cfl_v, (void *)&scratch};
    if (cudaLaunchKernel((const void *)k_noalloc_partial, dim3((unsigned)nchunks), dim3(kThreads), a1, 0, st) !=
        cudaSuccess)
        return AF_ECUDA;
    void *a2[] = {(void *)&scratch, (void *)&nch, (void *)&dt_dev};
    if (cudaLaunchKernel((const void *)k_noalloc_final, dim3(1), dim3(kThreads), a2, 0, st) != cudaSuccess)
        return AF_ECUDA;
    return AF_OK;
}
