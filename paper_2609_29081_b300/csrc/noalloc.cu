// noalloc.cu -- allocation-free entry point of libafns (declared in include/afns.h).
//
// af_dt_max_noalloc computes the CFL time step of Eq. (13) for a 2D FP64 state
// that the caller already holds on the device, without allocating anything. Its
// only scratch is a file-scope device array: one (inviscid, viscous) pair of
// maxima per chunk of AF_NOALLOC_CHUNK cells, for at most AF_NOALLOC_MAX_CHUNKS
// chunks. Every GPU that loads the library keeps that array until the process
// exits. The paper has no counterpart of this call.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "afns.h"

namespace {

constexpr int kChunk = AF_NOALLOC_CHUNK;          // cells per block
constexpr int kMaxChunks = AF_NOALLOC_MAX_CHUNKS;  // blocks per call
constexpr int kMaxDevices = 64;

// Partial maxima of one call; every call overwrites the slots it uses.
static __device__ __align__(256) double g_dt_scratch[2 * kMaxChunks];

// Device address of g_dt_scratch per device (host code may not use the symbol
// itself: on the host it names a stand-in, not device memory).
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_lock;

__global__ void k_noalloc_partial(const double *avg, long long cells, double dx, double dy, double gamma, double mu,
                                  double Pr, double cfl_c, double cfl_v, double *scratch)
{
    const long long begin = (long long)blockIdx.x * kChunk;
    const long long end = begin + kChunk < cells ? begin + kChunk : cells;
    double m1 = 0.0, m2 = 0.0;
    const double g1 = gamma - 1.0;
    for (long long t = begin + threadIdx.x; t < end; t += blockDim.x) {
        double rho = avg[t], mx = avg[cells + t], my = avg[2 * cells + t], E = avg[3 * cells + t];
        double p = g1 * (E - (mx * mx + my * my) / (2.0 * rho));
        double c = sqrt(gamma * p / rho);
        double rv = fmax(4.0 * mu / (3.0 * rho), gamma * mu / (Pr * rho));
        m1 = fmax(m1, fmax((fabs(mx / rho) + c) / (cfl_c * dx), (fabs(my / rho) + c) / (cfl_c * dy)));
        m2 = fmax(m2, fmax(rv / (cfl_v * dx * dx), rv / (cfl_v * dy * dy)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __shared__ double s1[32], s2[32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s1[wid] = m1, s2[wid] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m1 = fmax(m1, s1[k]), m2 = fmax(m2, s2[k]);
        scratch[2 * blockIdx.x] = m1;
        scratch[2 * blockIdx.x + 1] = m2;
    }
}

__global__ void k_noalloc_final(const double *scratch, int nchunks, double *dt_out)
{
    double m1 = 0.0, m2 = 0.0;
    for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
        m1 = fmax(m1, scratch[2 * k]);
        m2 = fmax(m2, scratch[2 * k + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    __shared__ double s1[32], s2[32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s1[wid] = m1, s2[wid] = m2;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m1 = fmax(m1, s1[k]), m2 = fmax(m2, s2[k]);
        *dt_out = 1.0 / (m1 + m2);
    }
}

// Device address of the scratch array on the current device (looked up once per device).
static cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dt_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (double *)p;
    }
    *out = g_scratch_addr[dev];
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
    if (nchunks > kMaxChunks) {   // larger than the static scratch
        std::fprintf(stderr, "af_dt_max_noalloc: %lld cells exceed the fixed scratch limit of %lld cells\n", cells,
                     (long long)kChunk * kMaxChunks);
        return AF_EINVAL;
    }
    af_opts d;
    if (!opts) {
        af_opts_default(2, &d);
        opts = &d;
    }
    if (!(opts->cfl_c > 0.0) || !(opts->cfl_v > 0.0)) return AF_EINVAL;
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return AF_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const double dx = (grid->hi[0] - grid->lo[0]) / grid->n[0], dy = (grid->hi[1] - grid->lo[1]) / grid->n[1];
    k_noalloc_partial<<<(unsigned)nchunks, 256, 0, st>>>(avg_dev, cells, dx, dy, gamma, mu, Pr, opts->cfl_c,
                                                         opts->cfl_v, scratch);
    k_noalloc_final<<<1, 256, 0, st>>>(scratch, (int)nchunks, dt_dev);
    return cudaGetLastError() == cudaSuccess ? AF_OK : AF_ECUDA;
}
