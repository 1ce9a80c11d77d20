// stage2d.cu -- host-side launchers of the 2D kernels (stage2d_kernels.cuh).
#include <algorithm>

#include "stage2d_kernels.cuh"

namespace afns {

// ---------------------------------------------------------------------------
// Host-side launchers (called from the C-ABI driver)
// ---------------------------------------------------------------------------
template <class S>
cudaError_t launch_ghost2d(const Layout &L, S *buf, cudaStream_t st)
{
    const int total = 4 * 5 * ((L.n2 + 1) + (L.n1 + 5));
    k_ghost2d_once<S><<<(total + 255) / 256, 256, 0, st>>>(L, buf);
    return cudaGetLastError();
}

template <class R, class S, int TX, int TY, int NTH>
cudaError_t launch_stage2d_n(const StageArgs &A, const CUtensorMap *const *maps, cudaStream_t st)
{
    using T = Tile2<TX, TY>;
    size_t smem = T::template bytes<R>();
    static int resident = 0;   // CTAs of this configuration that fit on the GPU at once
    if (!resident) {
        cudaError_t e = cudaFuncSetAttribute(k_stage2d<R, S, TX, TY, NTH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        // the whole unified L1 as shared memory: without a preference the driver
        // may pick a smaller carveout and fit fewer tiles per SM
        e = cudaFuncSetAttribute(k_stage2d<R, S, TX, TY, NTH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage2d<R, S, TX, TY, NTH>, NTH, smem);
        if (e != cudaSuccess) return e;
        resident = std::max(1, nsm * per_sm);
    }
    const long long ntiles = (long long)((A.L.n1 + TX - 1) / TX) * ((A.L.n2 + TY - 1) / TY);
    const int grid = (int)std::min<long long>(ntiles, resident);
    k_stage2d<R, S, TX, TY, NTH><<<grid, NTH, smem, st>>>(A, *maps[0], *maps[1], *maps[2], *maps[3]);
    return cudaGetLastError();
}

// threads: 128 or 256 per CTA (a compile-time constant of the kernel)
template <class R, class S, int TX, int TY>
cudaError_t launch_stage2d_t(const StageArgs &A, const CUtensorMap *const *maps, cudaStream_t st, int threads = 256)
{
    if (threads == 128) return launch_stage2d_n<R, S, TX, TY, 128>(A, maps, st);
    return launch_stage2d_n<R, S, TX, TY, 256>(A, maps, st);
}

// Tile shapes: FP64 16x8 or 16x16 (the 32x8 FP64 tile exceeds shared memory);
// FP32 16x8, 32x8, 16x16 or 32x16. threads: 256 or 128 per CTA (every phase
// loops over its items); the 32x16 FP32 tile (185 KB, one CTA per SM) runs 512.
cudaError_t launch_stage2d_fp64(const StageArgs &A, int tx, int ty, int threads, const CUtensorMap *const *maps,
                                cudaStream_t st)
{
    (void)tx;
    if (ty == 16) return launch_stage2d_t<double, double, 16, 16>(A, maps, st, threads > 0 ? threads : 256);
    return launch_stage2d_t<double, double, 16, 8>(A, maps, st, threads > 0 ? threads : 256);
}

cudaError_t launch_dt2d_fp64(const Layout &L, const double *buf, double gamma, double mu, double Pr, double cfl_c,
                             double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st)
{
    k_dt_partial2d<double><<<nparts, 256, 0, st>>>(L, buf, cfl_const(gamma, mu, Pr, cfl_c, cfl_v, L.dx, L.dy),
                                                   partial);
    k_dt_final<<<1, 256, 0, st>>>(partial, nparts, ctl, clip);
    return cudaGetLastError();
}

cudaError_t launch_tile_consts5(const StageArgs &A, const StageCoef *ks, void *out, int stride_bytes, int fp32,
                                cudaStream_t st)
{
    StageCoef5 k5;
    for (int s = 0; s < 5; ++s) k5.k[s] = ks[s];
    if (fp32) k_tile_consts5<float><<<1, 32, 0, st>>>(A, k5, (char *)out, stride_bytes);
    else k_tile_consts5<double><<<1, 32, 0, st>>>(A, k5, (char *)out, stride_bytes);
    return cudaGetLastError();
}

cudaError_t launch_tile_consts(const StageArgs &A, void *out, int fp32, cudaStream_t st)
{
    if (fp32) k_tile_consts<float><<<1, 32, 0, st>>>(A, (TileConst<float> *)out);
    else k_tile_consts<double><<<1, 32, 0, st>>>(A, (TileConst<double> *)out);
    return cudaGetLastError();
}

cudaError_t launch_dt_final(const double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st)
{
    k_dt_final<<<1, 256, 0, st>>>(partial, nparts, ctl, clip);
    return cudaGetLastError();
}

cudaError_t launch_ghost2d_fp64(const Layout &L, double *buf, cudaStream_t st) { return launch_ghost2d<double>(L, buf, st); }

template <class S>
static cudaError_t launch_validate2d(const Layout &L, const S *buf, double gamma, int *flag, cudaStream_t st)
{
    long long total = (long long)(L.n1 + 1) * (L.n2 + 1) * 4;
    int blocks = (int)std::min<long long>((total + 255) / 256, 148 * 16);
    k_validate2d<S><<<blocks, 256, 0, st>>>(L, buf, gamma, flag);
    return cudaGetLastError();
}

cudaError_t launch_validate2d_fp64(const Layout &L, const double *buf, double gamma, int *flag, cudaStream_t st)
{
    return launch_validate2d<double>(L, buf, gamma, flag, st);
}


}  // namespace afns

// ---------------------------------------------------------------------------
// Mixed precision: FP32 stencils and storage, FP64 islands, float-float averages
// ---------------------------------------------------------------------------
namespace afns {

cudaError_t launch_stage2d_mixed(const StageArgs &A, int tx, int ty, int threads, const CUtensorMap *const *maps,
                                 cudaStream_t st)
{
    if (tx == 32 && ty == 16) return launch_stage2d_n<float, float, 32, 16, 512>(A, maps, st);
    if (tx == 32) return launch_stage2d_t<float, float, 32, 8>(A, maps, st, threads > 0 ? threads : 256);
    if (ty == 16) return launch_stage2d_t<float, float, 16, 16>(A, maps, st, threads > 0 ? threads : 256);
    return launch_stage2d_t<float, float, 16, 8>(A, maps, st, threads > 0 ? threads : 256);
}

cudaError_t launch_ghost2d_f32(const Layout &L, float *buf, cudaStream_t st) { return launch_ghost2d<float>(L, buf, st); }

cudaError_t launch_dt2d_f32(const Layout &L, const float *buf, double gamma, double mu, double Pr, double cfl_c,
                            double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st)
{
    k_dt_partial2d<float><<<nparts, 256, 0, st>>>(L, buf, cfl_const(gamma, mu, Pr, cfl_c, cfl_v, L.dx, L.dy),
                                                  partial);
    return launch_dt_final(partial, nparts, ctl, clip, st);
}

// FP64 state planes -> FP32 planes; the cell-average planes (the first nc) also
// get their rounding residue in the compensation planes that follow the nplanes.
__global__ void k_to_f32(const double *src, float *dst, long long plane, int nplanes, int nc)
{
    long long total = plane * nplanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        double x = src[e];
        float h = __double2float_rn(x);
        dst[e] = h;
        long long p = e / plane;
        if (p < nc) dst[(long long)nplanes * plane + e] = __double2float_rn(x - (double)h);
    }
}

__global__ void k_to_f64(const float *src, double *dst, long long plane, int nplanes, int nc, int use_lo)
{
    long long total = plane * nplanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        double x = (double)src[e];
        long long p = e / plane;
        if (use_lo && p < nc) x += (double)src[(long long)nplanes * plane + e];
        dst[e] = x;
    }
}

// One DoF site's packed array (components in turn, x fastest, no ghosts) into the
// pitched planes of a state buffer: one coalesced pass, so that a host upload is
// one contiguous copy per site instead of one strided copy per component. In 2D
// the same pass checks the uploaded values (bit 1 of *flag: a DoF that is not
// finite, has rho <= 0 or p <= 0; bit 2: a periodic duplicate point that differs
// from its partner), so no separate validation pass reads the state again.
template <class T>
__global__ void k_unpack_site(Layout L, const T *src, T *buf, int site, int w, int h, int *flag)
{
    const int wh = w * h, nc = L.nc;
    const bool ptx = site == 1 || site == 3, pty = site == 2 || site == 3;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < wh; e += gridDim.x * blockDim.x) {
        const int j = e / w, i = e - j * w;
        const long long off = L.dim == 2 ? cell_off(L, i, j) : 2 + i;
        T U[4] = {T(0), T(0), T(0), T(0)};
        for (int c = 0; c < nc; ++c) {
            const T v = src[(long long)c * wh + e];
            buf[plane_of(L, site, c) + off] = v;
            U[c] = v;
        }
        if (L.dim != 2 || !flag) continue;
        if (!admissible_input2(U)) atomicOr(flag, 1);
        const int si = (ptx && i == L.n1 && L.bc[0] == BC_PERIODIC) ? 0 : i;
        const int sj = (pty && j == L.n2 && L.bc[2] == BC_PERIODIC) ? 0 : j;
        if (si != i || sj != j) {
            const int e2 = sj * w + si;
            for (int c = 0; c < nc; ++c)
                if (src[(long long)c * wh + e2] != src[(long long)c * wh + e]) atomicOr(flag, 2);
        }
    }
}

// The inverse of k_unpack_site for a download: one DoF site's pitched planes
// into a packed array (components in turn, x fastest, no ghosts), so that the
// host copy is one contiguous transfer instead of one strided copy per component.
template <class T>
__global__ void k_pack_site(Layout L, const T *buf, T *dst, int site, int w, int h)
{
    const int wh = w * h, nc = L.nc;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < wh; e += gridDim.x * blockDim.x) {
        const int j = e / w, i = e - j * w;
        const long long off = L.dim == 2 ? cell_off(L, i, j) : 2 + i;
        for (int c = 0; c < nc; ++c) dst[(long long)c * wh + e] = buf[plane_of(L, site, c) + off];
    }
}

cudaError_t launch_pack_site_f32(const Layout &L, const float *buf, float *dst, int site, int w, int h, cudaStream_t st)
{
    const long long n = (long long)w * h;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148 * 16);
    k_pack_site<float><<<blocks, 256, 0, st>>>(L, buf, dst, site, w, h);
    return cudaGetLastError();
}

cudaError_t launch_unpack_site_f32(const Layout &L, const float *src, float *buf, int site, int w, int h, int *flag,
                                   cudaStream_t st)
{
    const long long n = (long long)w * h;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 148 * 16);
    k_unpack_site<float><<<blocks, 256, 0, st>>>(L, src, buf, site, w, h, flag);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const Layout &L, const double *src, float *dst, cudaStream_t st)
{
    int np = L.nsite * L.nc;
    k_to_f32<<<148 * 8, 256, 0, st>>>(src, dst, L.plane, np, L.nc);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(const Layout &L, const float *src, double *dst, int use_lo, cudaStream_t st)
{
    int np = L.nsite * L.nc;
    k_to_f64<<<148 * 8, 256, 0, st>>>(src, dst, L.plane, np, L.nc, use_lo);
    return cudaGetLastError();
}

}  // namespace afns
