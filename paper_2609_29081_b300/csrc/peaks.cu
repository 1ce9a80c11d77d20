// peaks.cu -- measured FP32 / FP64 FMA throughput of the device (the ALU
// roofline denominators of the stage kernels; the paper has no counterpart).
//
// Every thread runs eight independent FMA chains (enough independent work to
// cover the FMA pipe latency at full occupancy) for a fixed number of
// iterations; the grid is 8 CTAs of 256 threads per SM. Rate = 2 flops per FMA
// x FMAs issued / CUDA-event time of the launch (after one warm-up launch).
#include <cuda_runtime.h>

#include "afns.h"

namespace {

template <class R>
__global__ void __launch_bounds__(256) k_fma_chains(R *out, R m, R c, int iters)
{
    R a0 = (R)threadIdx.x, a1 = a0 + (R)1, a2 = a0 + (R)2, a3 = a0 + (R)3;
    R a4 = a0 + (R)4, a5 = a0 + (R)5, a6 = a0 + (R)6, a7 = a0 + (R)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            a0 = a0 * m + c;
            a1 = a1 * m + c;
            a2 = a2 * m + c;
            a3 = a3 * m + c;
            a4 = a4 * m + c;
            a5 = a5 * m + c;
            a6 = a6 * m + c;
            a7 = a7 * m + c;
        }
    }
    out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

template <class R>
cudaError_t run_probe(int iters, double *tflops)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int threads = 256, blocks = nsm * 8;
    R *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&out, sizeof(R) * (size_t)blocks * threads);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms = 0.f;
    if (e == cudaSuccess) {
        // m slightly below 1 keeps every chain bounded (a -> c / (1 - m)).
        const R m = (R)0.999999, c = (R)1e-3;
        k_fma_chains<R><<<blocks, threads, 0, st>>>(out, m, c, iters);
        cudaEventRecord(a, st);
        k_fma_chains<R><<<blocks, threads, 0, st>>>(out, m, c, iters);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    if (e == cudaSuccess) {
        double fma = (double)blocks * threads * iters * 16.0 * 8.0;
        *tflops = 2.0 * fma / (ms * 1e-3) / 1e12;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return e;
}

}  // namespace

extern "C" af_status af_alu_peak(int precision, double *tflops)
{
    if (!tflops || (precision != AF_FP64 && precision != AF_MIXED)) return AF_EINVAL;
    *tflops = 0.0;
    cudaGetLastError();
    // FP32: 16384 x 128 FMA per thread (~1 ms at full rate); FP64 1/32 of that.
    cudaError_t e = precision == AF_MIXED ? run_probe<float>(16384, tflops) : run_probe<double>(512, tflops);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return AF_ECUDA;
    }
    return AF_OK;
}
