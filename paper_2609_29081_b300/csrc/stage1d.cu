// stage1d.cu -- host-side launchers of the 1D kernels (stage1d_kernels.cuh).
#include <algorithm>

#include "stage1d_kernels.cuh"

namespace afns {

cudaError_t launch_dt_final(const double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st);

cudaError_t launch_ghost1d_fp64(const Layout &L, double *buf, cudaStream_t st)
{
    k_ghost1d<double><<<1, 32, 0, st>>>(L, buf);
    return cudaGetLastError();
}

cudaError_t launch_ghost1d_f32(const Layout &L, float *buf, cudaStream_t st)
{
    k_ghost1d<float><<<1, 32, 0, st>>>(L, buf);
    return cudaGetLastError();
}

cudaError_t launch_exact_ghost1d_fp64(const Layout &L, double *buf, const Ctl *ctl, double ct, ExactParams ep,
                                      cudaStream_t st)
{
    k_exact_ghost1d<double><<<1, 32, 0, st>>>(L, buf, ctl, ct, ep);
    return cudaGetLastError();
}

cudaError_t launch_exact_ghost1d_f32(const Layout &L, float *buf, const Ctl *ctl, double ct, ExactParams ep,
                                     cudaStream_t st)
{
    k_exact_ghost1d<float><<<1, 32, 0, st>>>(L, buf, ctl, ct, ep);
    return cudaGetLastError();
}

template <class R>
static cudaError_t launch_stage1d_t(const StageArgs &A, cudaStream_t st)
{
    constexpr int TX = 64;
    using T = Tile1<TX>;
    size_t smem = sizeof(R) * (size_t)T::total;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_stage1d<R, R, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_stage1d<R, R, TX><<<(A.L.n1 + TX - 1) / TX, 128, smem, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_stage1d_fp64(const StageArgs &A, cudaStream_t st) { return launch_stage1d_t<double>(A, st); }

// Mixed precision: FP32 storage and stencils, FP64 limiters and cell update.
cudaError_t launch_stage1d_mixed(const StageArgs &A, cudaStream_t st) { return launch_stage1d_t<float>(A, st); }

cudaError_t launch_dt1d_fp64(const Layout &L, const double *buf, double gamma, double mu, double Pr, double cfl_c,
                             double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st)
{
    k_dt_partial1d<double><<<nparts, 256, 0, st>>>(L, buf, gamma, mu, Pr, cfl_c, cfl_v, partial);
    return launch_dt_final(partial, nparts, ctl, clip, st);
}

cudaError_t launch_dt1d_f32(const Layout &L, const float *buf, double gamma, double mu, double Pr, double cfl_c,
                            double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st)
{
    k_dt_partial1d<float><<<nparts, 256, 0, st>>>(L, buf, gamma, mu, Pr, cfl_c, cfl_v, partial);
    return launch_dt_final(partial, nparts, ctl, clip, st);
}

cudaError_t launch_validate1d_fp64(const Layout &L, const double *buf, double gamma, int *flag, cudaStream_t st)
{
    int blocks = std::min((2 * L.n1 + 1 + 255) / 256, 148 * 8);
    k_validate1d<double><<<blocks, 256, 0, st>>>(L, buf, gamma, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate1d_f32(const Layout &L, const float *buf, double gamma, int *flag, cudaStream_t st)
{
    int blocks = std::min((2 * L.n1 + 1 + 255) / 256, 148 * 8);
    k_validate1d<float><<<blocks, 256, 0, st>>>(L, buf, gamma, flag);
    return cudaGetLastError();
}

}  // namespace afns
