// afns.cu -- host driver and C-ABI of libafns (declared in include/afns.h).
//
// Owns the device workspace (or borrows the caller's), lays the state out as
// padded structure-of-arrays planes with two ghost layers, and sequences the
// kernels of one SSP-RK54 step: CFL reduction, then per stage a ghost fill and
// one fused stage kernel, then a 4-byte read of the restart flag (Remark 3.2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <cuda.h>

#include "afns.h"
#include "stage2d.cuh"

namespace {
// bytes between the tile-constant records of the five stages of a step
constexpr int kTconstStride = (int)((sizeof(afns::TileConst<double>) + 255) / 256 * 256);
}

namespace afns {
cudaError_t launch_stage2d_fp64(const StageArgs &A, int tx, int ty, int threads, const CUtensorMap *const *maps,
                                cudaStream_t st);
cudaError_t launch_dt2d_fp64(const Layout &L, const double *buf, double gamma, double mu, double Pr, double cfl_c,
                             double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st);
cudaError_t launch_ghost2d_fp64(const Layout &L, double *buf, cudaStream_t st);
cudaError_t launch_validate2d_fp64(const Layout &L, const double *buf, double gamma, int *flag, cudaStream_t st);
cudaError_t launch_ghost1d_fp64(const Layout &L, double *buf, cudaStream_t st);
cudaError_t launch_stage1d_fp64(const StageArgs &A, cudaStream_t st);
cudaError_t launch_dt1d_fp64(const Layout &L, const double *buf, double gamma, double mu, double Pr, double cfl_c,
                             double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st);
cudaError_t launch_validate1d_fp64(const Layout &L, const double *buf, double gamma, int *flag, cudaStream_t st);
cudaError_t launch_ghost1d_f32(const Layout &L, float *buf, cudaStream_t st);
cudaError_t launch_exact_ghost1d_fp64(const Layout &L, double *buf, const Ctl *ctl, double ct, ExactParams ep,
                                      cudaStream_t st);
cudaError_t launch_exact_ghost1d_f32(const Layout &L, float *buf, const Ctl *ctl, double ct, ExactParams ep,
                                     cudaStream_t st);
cudaError_t launch_validate1d_f32(const Layout &L, const float *buf, double gamma, int *flag, cudaStream_t st);
cudaError_t launch_stage1d_mixed(const StageArgs &A, cudaStream_t st);
cudaError_t launch_dt1d_f32(const Layout &L, const float *buf, double gamma, double mu, double Pr, double cfl_c,
                            double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st);
cudaError_t launch_stage2d_mixed(const StageArgs &A, int tx, int ty, int threads, const CUtensorMap *const *maps,
                                 cudaStream_t st);
cudaError_t launch_ghost2d_f32(const Layout &L, float *buf, cudaStream_t st);
cudaError_t launch_tile_consts5(const StageArgs &A, const StageCoef *ks, void *out, int stride_bytes, int fp32,
                                cudaStream_t st);
cudaError_t launch_dt2d_f32(const Layout &L, const float *buf, double gamma, double mu, double Pr, double cfl_c,
                            double cfl_v, double *partial, int nparts, Ctl *ctl, int clip, cudaStream_t st);
cudaError_t launch_to_f32(const Layout &L, const double *src, float *dst, cudaStream_t st);
cudaError_t launch_pack_site_f32(const Layout &L, const float *buf, float *dst, int site, int w, int h, cudaStream_t st);
cudaError_t launch_unpack_site_f32(const Layout &L, const float *src, float *buf, int site, int w, int h, int *flag,
                                   cudaStream_t st);
cudaError_t launch_tile_consts(const StageArgs &A, void *out, int fp32, cudaStream_t st);
cudaError_t launch_to_f64(const Layout &L, const float *src, double *dst, int use_lo, cudaStream_t st);

__global__ void k_set_ctl(Ctl *ctl, double dt, double t, double t_end)
{
    ctl->dt = dt;
    ctl->t = t;
    ctl->t_end = t_end;
    ctl->notpp = 0;
    ctl->err = 0;
}
// The CFL step of Eq. (13) from the maxima the previous step's last stage
// merged into the control block (same formula as k_dt_final), clipped to t_end
// when asked; the rest as k_set_ctl.
__global__ void k_set_ctl_cfl(Ctl *ctl, double t, double t_end, int clip)
{
    const double m1 = __longlong_as_double((long long)ctl->cfl_mx[0]);
    const double m2 = __longlong_as_double((long long)ctl->cfl_mx[1]);
    double dt = 1.0 / (m1 + m2);
    ctl->dt_cfl = dt;
    if (clip && t_end > t && t + dt > t_end) dt = t_end - t;
    ctl->dt = dt;
    ctl->t = t;
    ctl->t_end = t_end;
    ctl->notpp = 0;
    ctl->err = 0;
}
__global__ void k_halve_ctl(Ctl *ctl)
{
    ctl->dt *= 0.5;
    ctl->notpp = 0;
}
}  // namespace afns

using namespace afns;

// SSP-RK54, Spiteri-Ruuth SSPRK(5,4), Shu-Osher form (Sec. 2.3; the paper names
// the method but does not print its coefficients).
static const double kRK_a[5][5] = {
    {1.0, 0, 0, 0, 0},
    {0.444370493651235, 0.555629506348765, 0, 0, 0},
    {0.620101851488403, 0, 0.379898148511597, 0, 0},
    {0.178079954393132, 0, 0, 0.821920045606868, 0},
    {0, 0, 0.517231671970585, 0.096059710526147, 0.386708617503269},
};
static const double kRK_b[5] = {0.391752226571890, 0.368410593050371, 0.251891774271694, 0.544974750228521,
                                0.226007483236906};
static const double kRK_b43 = 0.063692468666290;

struct afns_ctx {
    int dim = 2;
    int n1 = 0, n2 = 1;
    double lo[2] = {0, 0}, hi[2] = {1, 1};
    double gamma = 1.4, mu = 0, Pr = 1, kappa = 0;
    double Pr_cfl = 1;           // Pr in the CFL bound (infinite without heat conduction)
    int bc[4] = {0, 0, 0, 0};
    af_opts opts{};
    cudaStream_t st = nullptr;
    Layout L{};
    size_t state_bytes = 0;
    char *ws = nullptr;
    bool own_ws = false;
    void *U[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // u^n, u1/u3/u5, u2/acc, u4, residual
    double *stage64 = nullptr;   // FP64 staging state of the mixed path
    bool mixed = false;
    int tile_x = 16, tile_y = 8; // 2D tile: 16x8, 16x16, or 32x8 (mixed path)
    int threads = 128;           // threads per CTA of the stage kernel
    // TMA tensor maps of the five state buffers for the 2D stage kernel, per tile
    // shape (16x8, 32x8, 16x16): 3D (element of a row, row, plane), box (TX+4, TY+4, 4)
    CUtensorMap maps[4][5];      // per tile shape (16x8, 32x8, 16x16, 32x16) and buffer
    CUtensorMap rmaps[4][5];     // the same, with the row box of the cell-update inputs
    void *map_buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // buffer of maps[.][k] (U[] rotates)
    void *tconst = nullptr;      // per-stage tile constants (2D stage kernel)
    int debug_extra_tx = 0;      // test hook of af_debug_tile_wait
    Ctl *ctl = nullptr;
    Ctl *h_ctl = nullptr;   // pinned mirror
    double *partial = nullptr;
    int nparts = 0;
    double *theta = nullptr;
    int *flag = nullptr;
    int *h_flag = nullptr;
    size_t nfaces = 0;
    // profiling: CUDA events around every stage-kernel launch, launch counters
    int profiling = 0;
    cudaEvent_t ev[5][2] = {};
    int ev_used = 0;
    double stage_ms = 0;
    long long stage_launches = 0;
    long long launches = 0;
    double t = 0;
    bool has_state = false;
    CflConst cflk{};             // constants of Eq. (13)
    bool cfl_ready = false;      // Ctl.cfl_mx holds the maxima of the current state (2D, after a step)
    std::string err;
};

static af_status fail(afns_ctx *c, af_status s, const std::string &m)
{
    if (c) c->err = m;
    return s;
}

static af_status cuda_check(afns_ctx *c, cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return AF_OK;
    cudaGetLastError();   // clear the runtime's record of the error so it is not reported again later
    return fail(c, AF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void make_layout(const af_grid *g, const int *bc, Layout *L, const double *wall_speed = nullptr)
{
    std::memset(L, 0, sizeof(*L));
    L->dim = g->dim;
    L->nc = g->dim + 2;
    L->n1 = g->n[0];
    L->n2 = g->dim == 2 ? g->n[1] : 1;
    L->nsite = g->dim == 2 ? 4 : 2;
    L->pitch = ((L->n1 + 5) + 31) / 32 * 32;
    L->rows = g->dim == 2 ? L->n2 + 5 : 1;
    long long pl = (long long)L->pitch * L->rows;
    L->plane = (pl + 63) / 64 * 64;
    for (int k = 0; k < 4; ++k) L->bc[k] = bc[k];
    for (int k = 0; k < 4; ++k) L->wall_speed[k] = wall_speed && bc[k] == AF_BC_MOVING_WALL ? wall_speed[k] : 0.0;
    L->dx = (g->hi[0] - g->lo[0]) / g->n[0];
    L->dy = g->dim == 2 ? (g->hi[1] - g->lo[1]) / g->n[1] : 1.0;
    L->lo[0] = g->lo[0];
    L->lo[1] = g->dim == 2 ? g->lo[1] : 0.0;
    layout_finish(L);
}

struct WsPlan {
    size_t state, stage64, ctl, partial, theta, flag, tconst, total;
    int nparts;
    size_t nfaces;
};

static WsPlan plan_ws(const Layout &L, const af_opts *o)
{
    WsPlan p{};
    size_t esz = o->precision == AF_MIXED ? sizeof(float) : sizeof(double);
    size_t planes = (size_t)L.nsite * L.nc + (o->precision == AF_MIXED ? L.nc : 0);
    p.state = align256(planes * (size_t)L.plane * esz);
    p.ctl = align256(sizeof(Ctl));
    p.nparts = 148 * 4;
    p.partial = align256(sizeof(double) * 2 * p.nparts);
    p.nfaces = L.dim == 2 ? (size_t)(L.n1 + 1) * L.n2 + (size_t)L.n1 * (L.n2 + 1) : (size_t)L.n1 + 1;
    p.theta = align256(sizeof(double) * 2 * p.nfaces);
    p.flag = align256(sizeof(int) * 4);
    // the mixed path converts to / from the FP64 public layout through a staging state
    p.stage64 = o->precision == AF_MIXED ? align256((size_t)L.nsite * L.nc * (size_t)L.plane * sizeof(double)) : 0;
    p.tconst = align256(5 * kTconstStride);
    p.total = 5 * p.state + p.stage64 + p.ctl + p.partial + p.theta + p.flag + p.tconst;
    return p;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        cudaGetLastError();
    }
    return fn;
}

// Tensor map of one 2D state buffer for tiles of TX x TY cells: the box covers
// the tile's cells with two of halo in each direction (TX+4 elements from the
// 16-byte aligned row start i0, TY+4 rows) and the 4 component planes of a site.
// With `rows` (cell-update inputs) the box is TX+4 elements by the tile's TY
// rows, and the planes reach the compensation planes of a mixed buffer.
// (Also used by the batched path for its per-problem maps.)
bool make_stage_map(CUtensorMap *m, void *buf, const Layout &L, size_t esz, int tx, int ty, bool rows)
{
    EncodeTiledFn f = encode_tiled();
    if (!f) return false;
    const cuuint64_t planes = (cuuint64_t)L.nsite * L.nc + (rows && esz == 4 ? (cuuint64_t)L.nc : 0);
    const cuuint64_t gdim[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, planes};
    const cuuint64_t gstride[2] = {(cuuint64_t)L.pitch * esz, (cuuint64_t)L.plane * esz};
    const cuuint32_t box[3] = {(cuuint32_t)(tx + 4), (cuuint32_t)(rows ? ty : ty + 4), 4};
    const cuuint32_t estride[3] = {1, 1, 1};
    return f(m, esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, buf, gdim, gstride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Why the calling thread's last af_create was refused (there is no context to
// hold the message).
static thread_local std::string g_create_error;

static af_status check_args(const af_grid *g, double gamma, double mu, double Pr, const af_bc *bc, const af_opts *o,
                            std::string *why)
{
    if (!g || !bc) return *why = "grid and bc are required", AF_EINVAL;
    if (g->dim != 1 && g->dim != 2) return *why = "dim must be 1 or 2", AF_EINVAL;
    for (int l = 0; l < g->dim; ++l) {
        if (g->n[l] < 4) return *why = "need at least 4 cells per direction", AF_EINVAL;
        if (!(g->hi[l] > g->lo[l])) return *why = "need hi > lo", AF_EINVAL;
    }
    // the per-site kernels index one site's elements (ghosts included) with
    // 32-bit integers; such grids would not fit in device memory anyway
    if (g->dim == 2 && (long long)(g->n[0] + 5) * (g->n[1] + 5) >= (1ll << 31))
        return *why = "grid too large: (n1+5)(n2+5) must stay below 2^31", AF_EINVAL;
    if (g->dim == 1 && g->n[0] >= (1 << 30)) return *why = "grid too large: n1 must stay below 2^30", AF_EINVAL;
    if (!(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0)) return *why = "need gamma > 1, mu >= 0, Pr > 0", AF_EINVAL;
    for (int l = 0; l < g->dim; ++l) {
        int a = bc->side[2 * l], b = bc->side[2 * l + 1];
        if (a < 0 || a > 5 || b < 0 || b > 5) return *why = "unknown boundary kind", AF_EINVAL;
        if ((a == AF_BC_EXACT || b == AF_BC_EXACT) && g->dim != 1)
            return *why = "exact boundary data are one-dimensional", AF_EINVAL;
        if ((a == AF_BC_MOVING_WALL || b == AF_BC_MOVING_WALL) && g->dim != 2)
            return *why = "moving walls are two-dimensional", AF_EINVAL;
        for (int s = 2 * l; s < 2 * l + 2; ++s)
            if (bc->side[s] == AF_BC_MOVING_WALL && !std::isfinite(bc->wall_speed[s]))
                return *why = "wall speed must be finite", AF_EINVAL;
        if ((a == AF_BC_PERIODIC) != (b == AF_BC_PERIODIC)) return *why = "periodic sides come in pairs", AF_EINVAL;
    }
    if (o->precision != AF_FP64 && o->precision != AF_MIXED) return *why = "unknown precision", AF_EINVAL;
    if (o->limiter < 0 || o->limiter > 2) return *why = "unknown limiter", AF_EINVAL;
    if (o->source != AF_SRC_NONE && o->source != AF_SRC_TAYLOR_GREEN) return *why = "unknown source", AF_EINVAL;
    if (o->source == AF_SRC_TAYLOR_GREEN && g->dim != 2)
        return *why = "the Taylor-Green source is two-dimensional", AF_EINVAL;
    if (o->kappa_off != 0 && o->kappa_off != 1) return *why = "kappa_off must be 0 or 1", AF_EINVAL;
    if (o->threads != 0 && o->threads != 128 && o->threads != 256)
        return *why = "threads per CTA must be 128 or 256", AF_EINVAL;
    if (!(o->cfl_c > 0) || !(o->cfl_v > 0) || !(o->eps > 0) || o->max_halvings < 0)
        return *why = "bad CFL numbers, eps or max_halvings", AF_EINVAL;
    return AF_OK;
}

extern "C" {

af_status af_opts_default(int dim, af_opts *o)
{
    if (!o || (dim != 1 && dim != 2)) return AF_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->precision = AF_FP64;
    o->limiter = AF_LIM_S_PP;
    o->c_s = 1.0;
    o->cfl_c = 1.04 / dim;
    // C^v of Eq. (13): 0.33 in 1D as printed; in 2D 0.13, just below the von
    // Neumann limit 0.1307 of the 2D viscous operator of Eq. (12) under SSP-RK54
    // where heat conduction dominates the bound (the Simpson centres and edge
    // averages couple the directions, so the printed 0.33/2 lets a high-frequency
    // mode grow)
    o->cfl_v = dim == 1 ? 0.33 : 0.13;
    o->eps = 1e-13;
    o->max_halvings = 30;
    o->source = AF_SRC_NONE;
    o->src_p0 = 100.0;
    o->ex_M0 = 3.0;
    o->ex_uinf = 0.2;
    o->threads = 128;
    o->kappa_off = 0;
    return AF_OK;
}

af_status af_workspace_bytes(const af_grid *grid, const af_opts *opts, size_t *bytes)
{
    if (!grid || !bytes) return AF_EINVAL;
    af_opts d;
    if (!opts) {
        if (af_opts_default(grid->dim, &d) != AF_OK) return AF_EINVAL;
        opts = &d;
    }
    int bc[4] = {0, 0, 0, 0};
    Layout L;
    make_layout(grid, bc, &L);
    *bytes = plan_ws(L, opts).total;
    return AF_OK;
}

af_status af_create(const af_grid *grid, double gamma, double mu, double Pr, const af_bc *bc, const af_opts *opts,
                    void *cuda_stream, void *workspace, size_t workspace_bytes, afns_ctx **out)
{
    if (!out) return AF_EINVAL;
    *out = nullptr;
    af_opts d;
    if (!opts) {
        if (!grid || af_opts_default(grid->dim, &d) != AF_OK) return AF_EINVAL;
        opts = &d;
    }
    std::string why;
    af_status s = check_args(grid, gamma, mu, Pr, bc, opts, &why);
    if (s != AF_OK) {
        g_create_error = why;   // af_last_error(NULL) returns it
        return s;
    }
    afns_ctx *c = new (std::nothrow) afns_ctx();
    if (!c) return AF_ENOMEM;
    c->dim = grid->dim;
    c->n1 = grid->n[0];
    c->n2 = grid->dim == 2 ? grid->n[1] : 1;
    for (int l = 0; l < 2; ++l) c->lo[l] = grid->lo[l], c->hi[l] = grid->hi[l];
    c->gamma = gamma;
    c->mu = mu;
    c->Pr = Pr;
    c->kappa = opts->kappa_off ? 0.0 : gamma * mu / ((gamma - 1.0) * Pr);
    c->Pr_cfl = opts->kappa_off ? INFINITY : Pr;
    for (int k = 0; k < 4; ++k) c->bc[k] = grid->dim == 2 || k < 2 ? bc->side[k] : AF_BC_PERIODIC;
    c->opts = *opts;
    c->st = (cudaStream_t)cuda_stream;
    make_layout(grid, c->bc, &c->L, bc->wall_speed);
    c->cflk = cfl_const(gamma, mu, c->Pr_cfl, opts->cfl_c, opts->cfl_v, c->L.dx, c->L.dy);
    WsPlan p = plan_ws(c->L, opts);
    if (workspace) {
        if (workspace_bytes < p.total || ((uintptr_t)workspace & 255)) {
            delete c;
            return AF_ENOMEM;
        }
        c->ws = (char *)workspace;
    } else {
        if (cudaMalloc((void **)&c->ws, p.total) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return AF_ENOMEM;
        }
        c->own_ws = true;
    }
    char *q = c->ws;
    c->state_bytes = p.state;
    for (int k = 0; k < 5; ++k) c->U[k] = q, q += p.state;
    c->mixed = opts->precision == AF_MIXED;
    c->L.comp = c->mixed ? 1 : 0;
    c->stage64 = c->mixed ? (double *)q : nullptr;
    c->tile_x = (c->mixed && opts->tile_x == 32) ? 32 : 16;
    c->tile_y = opts->tile_y == 16 ? 16 : 8;
    c->threads = opts->threads == 256 ? 256 : 128;
    q += p.stage64;
    c->ctl = (Ctl *)q;
    q += p.ctl;
    c->partial = (double *)q;
    q += p.partial;
    c->nparts = p.nparts;
    c->theta = (double *)q;
    q += p.theta;
    c->flag = (int *)q;
    q += p.flag;
    c->tconst = q;
    c->nfaces = p.nfaces;
    if (cudaMallocHost((void **)&c->h_ctl, sizeof(Ctl) + 16) != cudaSuccess) {
        cudaGetLastError();
        if (c->own_ws) cudaFree(c->ws);
        delete c;
        return AF_ENOMEM;
    }
    c->h_flag = (int *)(c->h_ctl + 1);
    // NaN-free workspace: ghost rows of unused padding are never read, but zero it once
    cudaError_t e = cudaMemsetAsync(c->ws, 0, p.total, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        af_destroy(c);
        return AF_ECUDA;
    }
    if (c->dim == 2) {
        const size_t esz = c->mixed ? sizeof(float) : sizeof(double);
        for (int k = 0; k < 5; ++k) c->map_buf[k] = c->U[k];
        static const int shape[4][2] = {{16, 8}, {32, 8}, {16, 16}, {32, 16}};
        for (int w = 0; w < 4; ++w)
            for (int k = 0; k < 5; ++k)
                if (!make_stage_map(&c->maps[w][k], c->map_buf[k], c->L, esz, shape[w][0], shape[w][1], false) ||
                    !make_stage_map(&c->rmaps[w][k], c->map_buf[k], c->L, esz, shape[w][0], shape[w][1], true)) {
                    af_destroy(c);
                    return AF_ECUDA;   // tensor map encoding failed
                }
    }
    *out = c;
    return AF_OK;
}

af_status af_destroy(afns_ctx *c)
{
    if (!c) return AF_EINVAL;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    for (int k = 0; k < 5; ++k)
        for (int q = 0; q < 2; ++q)
            if (c->ev[k][q]) cudaEventDestroy(c->ev[k][q]);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    delete c;
    return AF_OK;
}

const char *af_last_error(const afns_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

af_status af_sizes(const afns_ctx *c, size_t *cells, size_t *faces, size_t *site_elems4)
{
    if (!c) return AF_EINVAL;
    if (cells) *cells = (size_t)c->n1 * c->n2;
    if (faces) *faces = c->nfaces;
    if (site_elems4) {
        if (c->dim == 2) {
            site_elems4[0] = (size_t)4 * c->n1 * c->n2;
            site_elems4[1] = (size_t)4 * (c->n1 + 1) * c->n2;
            site_elems4[2] = (size_t)4 * c->n1 * (c->n2 + 1);
            site_elems4[3] = (size_t)4 * (c->n1 + 1) * (c->n2 + 1);
        } else {
            site_elems4[0] = (size_t)3 * c->n1;
            site_elems4[1] = (size_t)3 * (c->n1 + 1);
            site_elems4[2] = site_elems4[3] = 0;
        }
    }
    return AF_OK;
}

}  // extern "C"

// Width/height of site s.
static void site_dims(const afns_ctx *c, int s, int *w, int *h)
{
    if (c->dim == 1) {
        *w = s == 1 ? c->n1 + 1 : c->n1;
        *h = 1;
        return;
    }
    *w = (s == 1 || s == 3) ? c->n1 + 1 : c->n1;
    *h = (s == 2 || s == 3) ? c->n2 + 1 : c->n2;
}

// Kernel dispatch by dimension.
static cudaError_t do_ghost(afns_ctx *c, void *buf, double ct = 0.0)
{
    if (c->dim == 1) {
        c->launches += 1;
        cudaError_t e = c->mixed ? launch_ghost1d_f32(c->L, (float *)buf, c->st)
                                 : launch_ghost1d_fp64(c->L, (double *)buf, c->st);
        if (e == cudaSuccess && (c->bc[0] == AF_BC_EXACT || c->bc[1] == AF_BC_EXACT)) {
            c->launches += 1;
            ExactParams ep{c->gamma, c->mu, c->Pr, c->opts.ex_M0, c->opts.ex_uinf};
            e = c->mixed ? launch_exact_ghost1d_f32(c->L, (float *)buf, c->ctl, ct, ep, c->st)
                         : launch_exact_ghost1d_fp64(c->L, (double *)buf, c->ctl, ct, ep, c->st);
        }
        return e;
    }
    c->launches += 1;
    if (c->mixed) return launch_ghost2d_f32(c->L, (float *)buf, c->st);
    return launch_ghost2d_fp64(c->L, (double *)buf, c->st);
}

static cudaError_t do_stage(afns_ctx *c, const StageArgs &A)
{
    c->launches += 1;
    if (c->dim == 1) return c->mixed ? launch_stage1d_mixed(A, c->st) : launch_stage1d_fp64(A, c->st);
    auto slot = [&](const void *b) {
        int k = 0;
        while (k < 5 && c->map_buf[k] != b) ++k;
        return k;
    };
    const int k = slot(A.uin), k0 = slot(A.u0), k2 = slot(A.aux);
    if (k == 5 || k0 == 5 || k2 == 5) return cudaErrorInvalidValue;
    const int w = c->tile_x == 32 ? (c->tile_y == 16 ? 3 : 1) : (c->tile_y == 16 ? 2 : 0);
    // the tile map of the stage input, the row maps of u^n, of the auxiliary
    // state and of the stage input
    const CUtensorMap *maps[4] = {&c->maps[w][k], &c->rmaps[w][k0], &c->rmaps[w][k2], &c->rmaps[w][k]};
    if (c->mixed) return launch_stage2d_mixed(A, c->tile_x, c->tile_y, c->threads, maps, c->st);
    return launch_stage2d_fp64(A, c->tile_x, c->tile_y, c->threads, maps, c->st);
}

// Public FP64 site arrays <-> state buffer. The FP64 path copies directly; the
// mixed path goes through the FP64 staging state and a conversion kernel.
static af_status sites_in(afns_ctx *c, void *buf, double *const site[4], int on_device);
static af_status sites_out(afns_ctx *c, void *buf, double *const site[4], int on_device, int use_lo);

static cudaError_t do_validate(afns_ctx *c, const void *buf)
{
    if (c->dim == 1) return launch_validate1d_fp64(c->L, (const double *)buf, c->gamma, c->flag, c->st);
    return launch_validate2d_fp64(c->L, (const double *)buf, c->gamma, c->flag, c->st);
}

// Copy between the public site arrays and a padded state buffer (dir 0: in, 1: out).
template <class T>
static af_status copy_sites_t(afns_ctx *c, void *buf, T *const site[4], int on_device, int dir)
{
    for (int s = 0; s < c->L.nsite; ++s) {
        if (!site[s]) return fail(c, AF_EINVAL, "null site pointer");
        int w, h;
        site_dims(c, s, &w, &h);
        for (int comp = 0; comp < c->L.nc; ++comp) {
            T *dev = (T *)buf + plane_of(c->L, s, comp) + (c->dim == 2 ? cell_off(c->L, 0, 0) : 2);
            T *host = site[s] + (size_t)comp * w * h;
            cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : (dir == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
            cudaError_t e = dir == 0 ? cudaMemcpy2DAsync(dev, c->L.pitch * sizeof(T), host, w * sizeof(T),
                                                        w * sizeof(T), h, k, c->st)
                                     : cudaMemcpy2DAsync(host, w * sizeof(T), dev, c->L.pitch * sizeof(T),
                                                         w * sizeof(T), h, k, c->st);
            if (e != cudaSuccess) return cuda_check(c, e, "state copy");
        }
    }
    return AF_OK;
}

static af_status copy_sites(afns_ctx *c, void *buf, double *const site[4], int on_device, int dir)
{
    return copy_sites_t<double>(c, buf, site, on_device, dir);
}

static af_status sites_in(afns_ctx *c, void *buf, double *const site[4], int on_device)
{
    void *dst = c->mixed ? (void *)c->stage64 : buf;
    af_status s = copy_sites(c, dst, site, on_device, 0);
    if (s != AF_OK) return s;
    cudaError_t e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->st);
    if (e == cudaSuccess) e = do_validate(c, dst);
    if (e == cudaSuccess && c->mixed) e = launch_to_f32(c->L, c->stage64, (float *)buf, c->st);
    return cuda_check(c, e, "state upload");
}

static af_status sites_out(afns_ctx *c, void *buf, double *const site[4], int on_device, int use_lo)
{
    if (!c->mixed) return copy_sites(c, buf, site, on_device, 1);
    cudaError_t e = launch_to_f64(c->L, (const float *)buf, c->stage64, use_lo, c->st);
    if (e != cudaSuccess) return cuda_check(c, e, "state conversion");
    return copy_sites(c, c->stage64, site, on_device, 1);
}

extern "C" af_status af_set_state(afns_ctx *c, const double *const site[4], int on_device, double t)
{
    if (!c || !site) return fail(c, AF_EINVAL, "null argument");
    af_status s = sites_in(c, c->U[0], const_cast<double *const *>(site), on_device);
    if (s != AF_OK) return s;
    cudaError_t e = cudaMemcpyAsync(c->h_flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_check(c, e, "af_set_state");
    if (*c->h_flag & 1) return fail(c, AF_EINVAL, "state has a DoF outside G (rho <= 0, p <= 0 or not finite)");
    if (*c->h_flag & 2) return fail(c, AF_EINVAL, "periodic duplicate point values differ from their partners");
    c->t = t;
    c->has_state = true;
    c->cfl_ready = false;
    return AF_OK;
}

extern "C" af_status af_get_state(afns_ctx *c, double *const site[4], int on_device, double *t)
{
    if (!c || !site) return fail(c, AF_EINVAL, "null argument");
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    cudaError_t e = do_ghost(c, c->U[0]);
    if (e != cudaSuccess) return cuda_check(c, e, "ghost fill");
    af_status s = sites_out(c, c->U[0], site, on_device, 1);
    if (s != AF_OK) return s;
    e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_check(c, e, "af_get_state");
    if (t) *t = c->t;
    return AF_OK;
}

// FP32 site arrays of a mixed-precision context: straight into / out of the
// FP32 state (the compensation words of the averages start at zero; on the way
// out the averages are their FP32 roundings hi = fl(hi + lo)).
extern "C" af_status af_set_state_f32(afns_ctx *c, const float *const site[4], int on_device, double t)
{
    if (!c || !site) return fail(c, AF_EINVAL, "null argument");
    if (!c->mixed) return fail(c, AF_EINVAL, "FP32 state arrays need an AF_MIXED context");
    // host arrays: one contiguous copy per site into the staging area, then a
    // kernel spreads them over the pitched planes (device arrays: the kernel
    // reads them in place)
    cudaError_t e = cudaMemsetAsync(c->flag, 0, sizeof(int), c->st);
    size_t off = 0;
    for (int s = 0; s < c->L.nsite && e == cudaSuccess; ++s) {
        if (!site[s]) return fail(c, AF_EINVAL, "null site pointer");
        int w, h;
        site_dims(c, s, &w, &h);
        const size_t bytes = sizeof(float) * (size_t)c->L.nc * w * h;
        const float *src = site[s];
        if (!on_device) {
            float *stg = (float *)((char *)c->stage64 + off);
            e = cudaMemcpyAsync(stg, site[s], bytes, cudaMemcpyHostToDevice, c->st);
            src = stg;
            off += align256(bytes);
        }
        if (e == cudaSuccess) e = launch_unpack_site_f32(c->L, src, (float *)c->U[0], s, w, h, c->flag, c->st);
    }
    if (e != cudaSuccess) return cuda_check(c, e, "state upload");
    float *lo = (float *)c->U[0] + comp_plane(c->L, 0);
    e = cudaMemsetAsync(lo, 0, sizeof(float) * (size_t)c->L.nc * c->L.plane, c->st);
    // 2D: the unpack pass has checked the values; 1D: one validation pass
    if (e == cudaSuccess && c->dim == 1)
        e = launch_validate1d_f32(c->L, (const float *)c->U[0], c->gamma, c->flag, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_check(c, e, "af_set_state_f32");
    if (*c->h_flag & 1) return fail(c, AF_EINVAL, "state has a DoF outside G (rho <= 0, p <= 0 or not finite)");
    if (*c->h_flag & 2) return fail(c, AF_EINVAL, "periodic duplicate point values differ from their partners");
    c->t = t;
    c->has_state = true;
    c->cfl_ready = false;
    return AF_OK;
}

extern "C" af_status af_get_state_f32(afns_ctx *c, float *const site[4], int on_device, double *t)
{
    if (!c || !site) return fail(c, AF_EINVAL, "null argument");
    if (!c->mixed) return fail(c, AF_EINVAL, "FP32 state arrays need an AF_MIXED context");
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    cudaError_t e = do_ghost(c, c->U[0]);
    if (e != cudaSuccess) return cuda_check(c, e, "ghost fill");
    // one pass packs each site (device arrays: straight into them; host arrays:
    // into the staging area, then one contiguous copy per site)
    size_t off = 0;
    for (int s = 0; s < c->L.nsite && e == cudaSuccess; ++s) {
        if (!site[s]) return fail(c, AF_EINVAL, "null site pointer");
        int w, h;
        site_dims(c, s, &w, &h);
        const size_t bytes = sizeof(float) * (size_t)c->L.nc * w * h;
        float *dst = on_device ? site[s] : (float *)((char *)c->stage64 + off);
        e = launch_pack_site_f32(c->L, (const float *)c->U[0], dst, s, w, h, c->st);
        if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(site[s], dst, bytes, cudaMemcpyDeviceToHost, c->st);
        off += align256(bytes);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_check(c, e, "af_get_state_f32");
    if (t) *t = c->t;
    return AF_OK;
}

static StageArgs base_args(afns_ctx *c)
{
    StageArgs A{};
    A.L = c->L;
    A.ctl = c->ctl;
    A.gamma = c->gamma;
    A.mu = c->mu;
    A.kappa = c->kappa;
    A.eps = c->opts.eps;
    A.c_s = c->opts.c_s;
    A.limiter = c->opts.limiter;
    A.source = c->opts.source;
    A.src_p0 = c->opts.src_p0;
    A.cfl = c->cflk;
    return A;
}

// One fused stage: ghost fill of the input, then the stage kernel.
// slot >= 0: the stage's tile constants were formed for the whole step (slot =
// stage index); slot < 0: form them for this stage alone.
static cudaError_t run_stage(afns_ctx *c, void *in, void *out, const StageCoef &k, double *theta, int slot = -1)
{
    cudaError_t e = do_ghost(c, in, k.ct);
    if (e != cudaSuccess) return e;
    StageArgs A = base_args(c);
    A.uin = in;
    A.u0 = c->U[0];
    A.aux = c->U[2];
    A.out = out;
    A.theta = theta;
    A.k = k;
    A.extra_tx = c->debug_extra_tx;
    if (c->dim == 2) {
        if (slot >= 0) {
            A.tconst = (char *)c->tconst + (size_t)slot * kTconstStride;
        } else {
            A.tconst = c->tconst;
            if ((e = launch_tile_consts(A, c->tconst, c->mixed ? 1 : 0, c->st)) != cudaSuccess) return e;
            c->launches += 1;
        }
    }
    bool prof = c->profiling && c->ev_used < 5;
    if (prof) cudaEventRecord(c->ev[c->ev_used][0], c->st);
    e = do_stage(c, A);
    if (prof) cudaEventRecord(c->ev[c->ev_used++][1], c->st);
    c->stage_launches += 1;
    return e;
}

// Accumulate the stage-kernel event times of the work issued so far (the stream
// has been synchronised by the caller).
static void harvest_events(afns_ctx *c)
{
    for (int k = 0; k < c->ev_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[k][0], c->ev[k][1]) == cudaSuccess) c->stage_ms += ms;
    }
    c->ev_used = 0;
}

// The five SSP-RK54 stages from U[0]; the result lands in U[1].
static cudaError_t run_rk(afns_ctx *c)
{
    bool walls = false;
    for (int k = 0; k < 4; ++k)
        walls |= c->bc[k] == AF_BC_WALL || c->bc[k] == AF_BC_SYMMETRY || c->bc[k] == AF_BC_MOVING_WALL;
    StageCoef k{};
    k.wall_fix = walls;
    // time of each stage input as a fraction of dt: c(u(s+1)) = a_ss c(u(s)) + b_s
    // (u(0) = u^n enters every combination at time 0)
    double ct[5] = {0.0};
    for (int s = 1; s < 5; ++s) ct[s] = kRK_a[s - 1][s - 1] * ct[s - 1] + kRK_b[s - 1];
    StageCoef ks[5];
    // u1 = u0 + b0 dt L(u0)
    k.a0 = 0; k.a1 = 1; k.a2 = 0; k.cl = kRK_b[0]; k.ct = ct[0];
    ks[0] = k;
    // u2 = a10 u0 + a11 u1 + b1 dt L(u1)
    k.a0 = kRK_a[1][0]; k.a1 = kRK_a[1][1]; k.cl = kRK_b[1]; k.ct = ct[1];
    ks[1] = k;
    // u3 = a20 u0 + a22 u2 + b2 dt L(u2)
    k.a0 = kRK_a[2][0]; k.a1 = kRK_a[2][2]; k.cl = kRK_b[2]; k.ct = ct[2];
    ks[2] = k;
    // u4 = a30 u0 + a33 u3 + b3 dt L(u3); acc = a42 u2 + a43 u3 + b43 dt L(u3)
    k.a0 = kRK_a[3][0]; k.a1 = kRK_a[3][3]; k.cl = kRK_b[3]; k.ct = ct[3];
    k.acc = 1; k.b2 = kRK_a[4][2]; k.b1 = kRK_a[4][3]; k.bl = kRK_b43;
    ks[3] = k;
    // u5 = acc + a44 u4 + b4 dt L(u4)
    k.acc = 0; k.a0 = 0; k.a2 = 1; k.a1 = kRK_a[4][4]; k.cl = kRK_b[4]; k.ct = ct[4];
    k.cfl_out = c->dim == 2;   // u5 = u^{n+1}: its CFL maxima give the next step
    ks[4] = k;
    cudaError_t e;
    int slot0 = -1;
    if (c->dim == 2) {   // the tile constants of all five stages in one launch
        if ((e = launch_tile_consts5(base_args(c), ks, c->tconst, kTconstStride, c->mixed ? 1 : 0, c->st)) != cudaSuccess)
            return e;
        c->launches += 1;
        slot0 = 0;
    }
    void *const in[5] = {c->U[0], c->U[1], c->U[2], c->U[1], c->U[3]};
    void *const out[5] = {c->U[1], c->U[2], c->U[1], c->U[3], c->U[1]};
    for (int st = 0; st < 5; ++st)
        if ((e = run_stage(c, in[st], out[st], ks[st], nullptr, slot0 < 0 ? -1 : st)) != cudaSuccess) return e;
    return cudaSuccess;
}

static af_status read_ctl(afns_ctx *c)
{
    cudaError_t e = cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e == cudaSuccess && c->profiling) harvest_events(c);
    if (e == cudaSuccess && c->h_ctl->err) return fail(c, AF_ECUDA, "a stage kernel's tile load timed out");
    return cuda_check(c, e, "control read");
}

// Step with the dt already in ctl; restarts with dt/2 on a non-PP low-order state.
static af_status step_from_ctl(afns_ctx *c, double *dt_taken, int *halvings)
{
    int h = 0;
    c->cfl_ready = false;
    for (;;) {
        cudaError_t e = run_rk(c);
        if (e != cudaSuccess) return cuda_check(c, e, "stage");
        af_status s = read_ctl(c);
        if (s != AF_OK) return s;
        if (!c->h_ctl->notpp) break;
        if (h >= c->opts.max_halvings) {
            if (halvings) *halvings = h;
            return fail(c, AF_ENOTPP, "low-order states not admissible after max_halvings restarts");
        }
        ++h;
        k_halve_ctl<<<1, 1, 0, c->st>>>(c->ctl);
        c->launches += 1;
    }
    std::swap(c->U[0], c->U[1]);
    c->t += c->h_ctl->dt;
    c->cfl_ready = c->dim == 2;   // the accepted attempt's last stage merged the maxima of U[0]
    if (dt_taken) *dt_taken = c->h_ctl->dt;
    if (halvings) *halvings = h;
    return AF_OK;
}

static cudaError_t launch_dt(afns_ctx *c, int clip)
{
    c->launches += 2;
    if (c->dim == 1 && c->mixed)
        return launch_dt1d_f32(c->L, (const float *)c->U[0], c->gamma, c->mu, c->Pr_cfl, c->opts.cfl_c, c->opts.cfl_v,
                               c->partial, c->nparts, c->ctl, clip, c->st);
    if (c->dim == 1)
        return launch_dt1d_fp64(c->L, (const double *)c->U[0], c->gamma, c->mu, c->Pr_cfl, c->opts.cfl_c, c->opts.cfl_v,
                                c->partial, c->nparts, c->ctl, clip, c->st);
    if (c->mixed)
        return launch_dt2d_f32(c->L, (const float *)c->U[0], c->gamma, c->mu, c->Pr_cfl, c->opts.cfl_c, c->opts.cfl_v,
                               c->partial, c->nparts, c->ctl, clip, c->st);
    return launch_dt2d_fp64(c->L, (const double *)c->U[0], c->gamma, c->mu, c->Pr_cfl, c->opts.cfl_c, c->opts.cfl_v,
                            c->partial, c->nparts, c->ctl, clip, c->st);
}

extern "C" af_status af_dt_max(afns_ctx *c, double *dt)
{
    if (!c || !dt) return fail(c, AF_EINVAL, "null argument");
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    k_set_ctl<<<1, 1, 0, c->st>>>(c->ctl, 0.0, c->t, c->t);
    cudaError_t e = launch_dt(c, 0);
    if (e != cudaSuccess) return cuda_check(c, e, "dt");
    af_status s = read_ctl(c);
    if (s != AF_OK) return s;
    *dt = c->h_ctl->dt_cfl;
    return AF_OK;
}

extern "C" af_status af_step(afns_ctx *c, double dt, double *dt_taken, int *halvings)
{
    if (!c) return AF_EINVAL;
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    c->launches += 1;
    if (dt > 0) {
        k_set_ctl<<<1, 1, 0, c->st>>>(c->ctl, dt, c->t, c->t);
    } else if (c->cfl_ready) {
        k_set_ctl_cfl<<<1, 1, 0, c->st>>>(c->ctl, c->t, c->t, 0);
    } else {
        k_set_ctl<<<1, 1, 0, c->st>>>(c->ctl, 0.0, c->t, c->t);
        cudaError_t e = launch_dt(c, 0);
        if (e != cudaSuccess) return cuda_check(c, e, "dt");
    }
    return step_from_ctl(c, dt_taken, halvings);
}

extern "C" af_status af_advance(afns_ctx *c, double t_end, int *steps, int *restarts)
{
    if (!c) return AF_EINVAL;
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    int ns = 0, nr = 0;
    af_status s = AF_OK;
    while (c->t < t_end) {
        c->launches += 1;
        if (c->cfl_ready) {
            k_set_ctl_cfl<<<1, 1, 0, c->st>>>(c->ctl, c->t, t_end, 1);
        } else {
            k_set_ctl<<<1, 1, 0, c->st>>>(c->ctl, 0.0, c->t, t_end);
            cudaError_t e = launch_dt(c, 1);
            if (e != cudaSuccess) {
                s = cuda_check(c, e, "dt");
                break;
            }
        }
        int h = 0;
        s = step_from_ctl(c, nullptr, &h);
        nr += h;
        if (s != AF_OK) break;
        ++ns;
    }
    if (steps) *steps = ns;
    if (restarts) *restarts = nr;
    return s;
}

extern "C" af_status af_residual(afns_ctx *c, double dt, double *const Lout[4], int on_device, int *notpp)
{
    if (!c || !Lout) return fail(c, AF_EINVAL, "null argument");
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    k_set_ctl<<<1, 1, 0, c->st>>>(c->ctl, dt, c->t, c->t);
    StageCoef k{};
    k.residual = 1;
    cudaError_t e = run_stage(c, c->U[0], c->U[4], k, c->theta);
    if (e == cudaSuccess) e = do_ghost(c, c->U[4]);   // periodic duplicates
    if (e != cudaSuccess) return cuda_check(c, e, "residual");
    af_status s = sites_out(c, c->U[4], Lout, on_device, 0);
    if (s != AF_OK) return s;
    s = read_ctl(c);
    if (s != AF_OK) return s;
    if (notpp) *notpp = c->h_ctl->notpp;
    return AF_OK;
}

extern "C" af_status af_debug_tile_wait(afns_ctx *c, int extra_bytes)
{
    if (!c || extra_bytes < 0 || extra_bytes % 16) return fail(c, AF_EINVAL, "extra_bytes: a multiple of 16, >= 0");
    c->debug_extra_tx = extra_bytes;
    return AF_OK;
}

extern "C" af_status af_get_limiter(afns_ctx *c, double *theta_s, double *theta_pp)
{
    if (!c) return AF_EINVAL;
    cudaError_t e = cudaSuccess;
    if (theta_s) e = cudaMemcpyAsync(theta_s, c->theta, c->nfaces * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && theta_pp)
        e = cudaMemcpyAsync(theta_pp, c->theta + c->nfaces, c->nfaces * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return cuda_check(c, e, "af_get_limiter");
}

extern "C" af_status af_set_profiling(afns_ctx *c, int on)
{
    if (!c) return AF_EINVAL;
    if (on && !c->ev[0][0]) {
        for (int k = 0; k < 5; ++k)
            for (int q = 0; q < 2; ++q)
                if (cudaEventCreate(&c->ev[k][q]) != cudaSuccess) return cuda_check(c, cudaGetLastError(), "event");
    }
    c->profiling = on ? 1 : 0;
    c->ev_used = 0;
    c->stage_ms = 0;
    c->stage_launches = 0;
    c->launches = 0;
    return AF_OK;
}

extern "C" af_status af_get_profile(afns_ctx *c, double *stage_ms, long long *stage_launches, long long *launches)
{
    if (!c) return AF_EINVAL;
    if (stage_ms) *stage_ms = c->stage_ms;
    if (stage_launches) *stage_launches = c->stage_launches;
    if (launches) *launches = c->launches;
    return AF_OK;
}

// Autotuner of the 2D stage kernel: times each candidate launch configuration
// (tile width, threads per CTA) on residual evaluations of the current state,
// which leave the state untouched, and keeps the fastest. Results do not depend
// on the configuration (every face and node is computed by the same arithmetic).
extern "C" af_status af_tune(afns_ctx *c, int *tile_x, int *tile_y, int *threads)
{
    if (!c) return AF_EINVAL;
    if (!c->has_state) return fail(c, AF_ESTATE, "no state set");
    if (c->dim == 2) {
        struct Cand {
            int tx, ty, th;
        };
        // 32-wide tiles in AF_MIXED only; the 32x16 tile always runs 512 threads
        const Cand cands[] = {{16, 8, 256}, {16, 8, 128}, {32, 8, 256}, {32, 8, 128},
                              {16, 16, 256}, {16, 16, 128}, {32, 16, 512}};
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
            return cuda_check(c, cudaGetLastError(), "tune events");
        float best = 1e30f;
        Cand pick{c->tile_x, c->tile_y, c->threads};
        int prof = c->profiling;
        c->profiling = 0;
        cudaError_t e = cudaSuccess;
        k_set_ctl<<<1, 1, 0, c->st>>>(c->ctl, 0.0, c->t, c->t);
        e = launch_dt(c, 0);
        StageCoef k{};
        k.residual = 1;
        for (const Cand &cd : cands) {
            if (e != cudaSuccess) break;
            if (cd.tx == 32 && !c->mixed) continue;
            c->tile_x = cd.tx;
            c->tile_y = cd.ty;
            c->threads = cd.th;
            e = run_stage(c, c->U[0], c->U[4], k, nullptr);   // warm-up (sets the shared-memory limit)
            if (e == cudaSuccess) e = cudaEventRecord(a, c->st);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = run_stage(c, c->U[0], c->U[4], k, nullptr);
            if (e == cudaSuccess) e = cudaEventRecord(b, c->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && ms < best) best = ms, pick = cd;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        c->profiling = prof;
        c->tile_x = pick.tx;
        c->tile_y = pick.ty;
        c->threads = pick.th;
        if (e != cudaSuccess) return cuda_check(c, e, "tune");
    }
    if (tile_x) *tile_x = c->tile_x;
    if (tile_y) *tile_y = c->tile_y;
    if (threads) *threads = c->threads;
    return AF_OK;
}
