// afns_dev.cuh -- device-side layout, physics and stencil helpers of libafns.
//
// State layout in HBM (one "state buffer"): structure of arrays, one plane per
// (DoF site, conservative component). 2D sites: 0 = cell average, 1 = x-edge
// point, 2 = y-edge point, 3 = vertex point; 1D sites: 0 = cell average,
// 1 = interface point. Every plane covers indices i in [-2, n1+2],
// j in [-2, n2+2] (two ghost layers), element (i, j) at (j+2)*pitch + (i+2).
// The mixed-precision form adds one FP32 compensation plane per cell-average
// component (the average is hi + lo).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace afns {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_SYMMETRY = 2, BC_TRANSMISSIVE = 3, BC_EXACT = 4, BC_MOVING = 5 };
enum { LIM_NONE = 0, LIM_PP = 1, LIM_S_PP = 2 };

struct Layout {
    int dim;        // 1 or 2
    int nc;         // components: dim + 2
    int n1, n2;     // cells (n2 = 1 in 1D)
    int pitch;      // elements per row
    int rows;       // rows per plane
    long long plane;  // elements per plane (multiple of 64)
    int nsite;      // 4 in 2D, 2 in 1D
    int comp;       // compensation planes present (mixed precision)
    int bc[4];
    double wall_speed[4];  // tangential velocity of BC_MOVING sides
    double lo[2];   // domain origin (x, y)
    double dx, dy;
    // reciprocal stencil factors per direction, set on the host by layout_finish
    // (so no kernel divides by the grid spacing): 1/dx_l, 1/(6 dx_l),
    // 1/(3 dx_l^2), 4/dx_l^2, 1/(2 dx_l)
    double idx[2], i6[2], i3h2[2], f4h2[2], i2[2];
};

inline void layout_finish(Layout *L)
{
    const double h[2] = {L->dx, L->dy};
    for (int l = 0; l < 2; ++l) {
        L->idx[l] = 1.0 / h[l];
        L->i6[l] = 1.0 / (6.0 * h[l]);
        L->i3h2[l] = 1.0 / (3.0 * h[l] * h[l]);
        L->f4h2[l] = 4.0 / (h[l] * h[l]);
        L->i2[l] = 1.0 / (2.0 * h[l]);
    }
}

// Plane index of (site, component); compensation plane of cell-average comp c.
__host__ __device__ __forceinline__ long long plane_of(const Layout &L, int site, int c)
{
    return (long long)(site * L.nc + c) * L.plane;
}
__host__ __device__ __forceinline__ long long comp_plane(const Layout &L, int c)
{
    return (long long)(L.nsite * L.nc + c) * L.plane;
}
__host__ __device__ __forceinline__ long long cell_off(const Layout &L, int i, int j)
{
    return (long long)(j + 2) * L.pitch + (i + 2);
}

// Gas constants in the compute precision.
template <class R>
struct Gas {
    R gamma, gm1, mu, kappa, eps;
};

// Control block in device memory shared by the kernels of one step.
struct Ctl {
    double dt;        // step size used by the stage kernels
    double t;         // current time
    double t_end;     // clip target of the CFL step (<= t: no clip)
    double dt_cfl;    // last CFL bound
    int notpp;        // a low-order state the limiters evaluate left G
    int err;          // a tile load of a stage kernel timed out (result invalid)
    // the two maxima of Eq. (13) over the cell averages a step's last stage wrote
    // (bit patterns of non-negative doubles, merged by atomic max): the next
    // step's CFL bound without another pass over the state
    unsigned long long cfl_mx[2];
};

// Parameters of the exact moving viscous shock used as 1D boundary data.
struct ExactParams {
    double gamma, mu, Pr, M0, uinf;
};

// SSP-RK54 stage combination: out = a0 u0 + a1 uin + a2 aux + cl dt L(uin);
// with acc: aux <- b2 aux + b1 uin + bl dt L(uin). Residual mode writes L itself.
struct StageCoef {
    double a0, a1, a2, cl;
    double b1, b2, bl;
    double ct;        // time of the stage input: t + ct dt (manufactured sources)
    int acc;
    int residual;
    int wall_fix;
    int cfl_out;      // 2D: merge the CFL maxima of the output cell averages into Ctl.cfl_mx
};

// --- ghost index images (two ghost layers; walls mirror about the boundary node,
// periodic wraps). "pt" = point-like along the direction (index i <-> lattice 2i),
// otherwise cell-like (index i <-> lattice 2i+1).
__host__ __device__ __forceinline__ int ghost_image(int i, int n, bool pt, int kind_lo, int kind_hi, int *side)
{
    // returns the interior index; *side = 0 (lo), 1 (hi), or -1 (not a ghost)
    if (pt) {
        if (i < 0) {
            *side = 0;
            return kind_lo == BC_PERIODIC ? i + n : -i;
        }
        if (i > n || (i == n && kind_hi == BC_PERIODIC)) {
            *side = 1;
            return kind_hi == BC_PERIODIC ? i - n : 2 * n - i;
        }
    } else {
        if (i < 0) {
            *side = 0;
            return kind_lo == BC_PERIODIC ? i + n : -i - 1;
        }
        if (i >= n) {
            *side = 1;
            return kind_hi == BC_PERIODIC ? i - n : 2 * n - 1 - i;
        }
    }
    *side = -1;
    return i;
}

// Momentum sign of component c (1..dim) under the mirror of a side of kind `kind`
// normal to direction l.
__host__ __device__ __forceinline__ double mirror_sign(int kind, int l, int c, int dim)
{
    if (c < 1 || c > dim) return 1.0;
    if (kind == BC_WALL || kind == BC_MOVING) return -1.0;
    if (kind == BC_SYMMETRY && c - 1 == l) return -1.0;
    return 1.0;
}

// Ghost value across a moving no-slip wall: the mirrored state v (both momenta
// already negated) gets its tangential velocity shifted by 2 U_w, i.e. the ghost
// velocity is 2 U_w - u_image, with the internal energy of the image kept.
template <class S>
__device__ __forceinline__ void moving_wall_ghost(const Layout &L, int side, S v[4])
{
    if (L.bc[side] != BC_MOVING) return;
    const int t = 1 + (1 - (side >> 1));
    const double r = v[0], m1 = v[1], m2 = v[2];
    double w[3] = {0.0, m1, m2};
    w[t] += 2.0 * r * L.wall_speed[side];
    const double m2_old = m1 * m1 + m2 * m2, m2_new = w[1] * w[1] + w[2] * w[2];
    v[t] = (S)w[t];
    v[3] = (S)((double)v[3] + (m2_new - m2_old) / (2.0 * r));
}

// Theta of Sec. 3.3 (limiter blending toward the low-order value).
template <class R>
__device__ __forceinline__ R theta_fn(R zL, R zH, R eps)
{
    return zH < eps ? (zL - eps) / (zL - zH) : R(1);
}

template <class R>
__device__ __forceinline__ R dmax(R a, R b)
{
    return b > a ? b : a;   // a NaN in b is ignored
}
template <class R>
__device__ __forceinline__ R dmin(R a, R b)
{
    return a < b ? a : b;
}

// --- float-float ("double-single") arithmetic for the compensated cell-average
// accumulation of the mixed-precision path: a value is hi + lo with |lo| <= ulp(hi)/2.
struct ff {
    float h, l;
};
__device__ __forceinline__ ff ff_quick(float a, float b)
{
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.h, b.h);
    return ff_quick(s.h, s.l + a.l + b.l);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return ff_quick(p, e);
}
__device__ __forceinline__ ff ff_from(double x)
{
    float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

// --- asynchronous global -> shared copies of single 4- or 8-byte elements
// (cp.async), used for the per-tile constants: the words are issued while the
// tile's TMA copies are in flight, then one wait and a barrier publish them. The
// host-compiler pass of this header (never executed on the GPU) copies
// synchronously.
template <class T>
__device__ __forceinline__ void cp_async_elem(T *dst_shared, const T *src_global)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
#ifdef __CUDA_ARCH__
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src_global) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src_global) : "memory");
#else
    *dst_shared = *src_global;
#endif
}

// Wait until every cp.async this thread issued has landed in shared memory
// (other threads see them after the next barrier).
__device__ __forceinline__ void cp_async_wait_all()
{
#ifdef __CUDA_ARCH__
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
#endif
}

// --- TMA tile loads: one mbarrier per CTA; thread 0 arms it with the byte count
// and issues 3D tensor copies (x = element in row, y = row, z = plane) into
// shared memory; every thread then waits on the barrier's phase with a bounded
// number of polls. The host-compiler pass of this header is never executed on
// the GPU and compiles to nothing.
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
#ifdef __CUDA_ARCH__
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(b), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
#endif
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
#ifdef __CUDA_ARCH__
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
#endif
}

// Bring one box of a 3D tensor map into L2 without a shared-memory destination
// (no barrier; the data is then read by ordinary loads at L2 latency).
__device__ __forceinline__ void tma_prefetch_l2_3d(const void *tmap, int x, int y, int z)
{
#ifdef __CUDA_ARCH__
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(tmap), "r"(x), "r"(y),
                 "r"(z)
                 : "memory");
#endif
}

__device__ __forceinline__ void tma_load_3d(void *dst_shared, const void *tmap, int x, int y, int z, uint64_t *bar)
{
#ifdef __CUDA_ARCH__
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_shared);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(d),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(b)
        : "memory");
#endif
}

// Poll the barrier's phase `parity` until it completes (true) or max_ns of the
// global timer have passed (false): a wait that can end, whatever happens to the
// copies it waits for.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long max_ns)
{
#ifdef __CUDA_ARCH__
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t0));
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
        if (t - t0 > max_ns) return false;
    }
#else
    return true;
#endif
}

}  // namespace afns
