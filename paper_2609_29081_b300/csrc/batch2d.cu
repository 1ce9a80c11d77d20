// batch2d.cu -- many independent 2D AF-NS problems advanced together.
//
// Every problem has its own grid, gas parameters, state buffers and control block
// (dt, restart flag). One batch step runs, for all problems at once:
//   CFL reduction  -- per-chunk maxima merged with 64-bit atomic max (positive
//                     doubles order like their bit patterns), then per problem dt;
//   5 RK stages    -- a ghost-fill pass pair and ONE persistent stage kernel over
//                     the (problem, tile) work list, each tile running the same
//                     fused stage code as the single-problem kernel;
//   commit         -- per problem: accept (swap u^n and u^{n+1}, t += dt) or
//                     reject (restart of Remark 3.2: keep u^n, halve dt; the next
//                     batch step recomputes this problem's step).
// Nothing in a batch step needs the host, so a whole step is captured once in a
// CUDA graph and replayed. The tile shape, CTA size and the order of the work
// list are chosen by a small autotuner that times candidate configurations on the
// actual batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "afns.h"
#include "stage2d_kernels.cuh"

namespace afns {

struct BatchProb {
    Layout L;
    void *U[5];                 // u^n, u1/u3/u5, u2/acc, u4, spare
    Ctl *ctl;
    unsigned long long *mx;     // 2 atomic-max slots (inviscid, viscous CFL terms)
    double gamma, mu, kappa, Pr;
    int tiles_x, tiles_y;
    int rejected;               // last step rejected: redo with the halved dt
    int halvings;               // consecutive halvings of the pending step
    int accepted;               // accepted steps
    int restarts;               // total rejected steps
    int failed;                 // max_halvings exceeded
    int buf_of[4];              // which of the problem's four buffers U[k] is (they rotate):
                                // selects its tensor map
};

struct BatchArgs {
    BatchProb *probs;
    const int *item_p;          // work list: problem of item
    const int *item_t;          // work list: tile of item within its problem
    int nitems;
    StageCoef k;
    int in_idx, out_idx;
    double eps, c_s;
    int limiter;
    void *tconst;               // per-problem tile constants of the stage (TileConst<R>[nprob])
    const CUtensorMap *maps;    // per problem, per buffer: tensor maps of this tile shape
    const CUtensorMap *rmaps;   // the same with the row box of the cell-update inputs
};

// The tensor maps of the batch (device memory, filled on the host at creation):
// problem p, tile shape s (0: 16x8, 1: 32x8), buffer b at [(p * kShapes + s) * 4 + b].
constexpr int kShapes = 2;

// --- CFL: chunks of 4096 cells
constexpr int kDtChunk = 4096;

template <class S>
__global__ void k_batch_dt_partial(BatchProb *probs, const int *chunk_p, const int *chunk_c, double cfl_c,
                                   double cfl_v)
{
    const int p = chunk_p[blockIdx.x];
    BatchProb &P = probs[p];
    if (P.rejected || P.failed) return;
    const Layout &L = P.L;
    const long long nc = (long long)L.n1 * L.n2;
    const long long b0 = (long long)chunk_c[blockIdx.x] * kDtChunk;
    const long long b1 = min(nc, b0 + kDtChunk);
    const S *buf = (const S *)P.U[0];
    // the per-cell terms of the single-problem kernel (same constants, same order)
    const CflConst k = cfl_const(P.gamma, P.mu, P.Pr, cfl_c, cfl_v, L.dx, L.dy);
    S f1 = 0, f2 = 0;
    for (long long t = b0 + threadIdx.x; t < b1; t += blockDim.x) {
        int i = (int)(t % L.n1), j = (int)(t / L.n1);
        long long off = cell_off(L, i, j);
        cfl_terms(k, buf[plane_of(L, 0, 0) + off], buf[plane_of(L, 0, 1) + off], buf[plane_of(L, 0, 2) + off],
                  buf[plane_of(L, 0, 3) + off], f1, f2);
    }
    double m1 = f1, m2 = f2;
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
    }
    if ((threadIdx.x & 31) == 0) {
        // positive doubles compare like their bit patterns
        atomicMax(&P.mx[0], (unsigned long long)__double_as_longlong(m1));
        atomicMax(&P.mx[1], (unsigned long long)__double_as_longlong(m2));
    }
}

__global__ void k_batch_dt_final(BatchProb *probs, int nprob)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    BatchProb &P = probs[p];
    if (!P.rejected && !P.failed) {
        double m1 = __longlong_as_double((long long)P.mx[0]), m2 = __longlong_as_double((long long)P.mx[1]);
        double dt = 1.0 / (m1 + m2);
        P.ctl->dt_cfl = dt;
        P.ctl->dt = dt;
    }
    P.mx[0] = 0ull;
    P.mx[1] = 0ull;
    P.ctl->notpp = 0;
}

// --- ghost fill of the stage input of every problem; blockIdx.y = problem
template <class S>
__global__ void k_batch_ghost(BatchProb *probs, int in_idx, int pass)
{
    BatchProb &P = probs[blockIdx.y];
    if (P.failed) return;
    const Layout &L = P.L;
    S *buf = (S *)P.U[in_idx];
    int span = pass == 0 ? (L.n2 + 1) : (L.n1 + 5);
    int total = 4 * span * 5;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int g = t % 5, r = (t / 5) % span, site = t / (5 * span);
        bool ptx = site == 1 || site == 3, pty = site == 2 || site == 3;
        int side, i, j, si, sj, l;
        if (pass == 0) {
            j = r;
            if (j > L.n2 - 1 + (pty ? 1 : 0)) continue;
            i = g < 2 ? g - 2 : L.n1 + (g - 2);
            si = ghost_image(i, L.n1, ptx, L.bc[0], L.bc[1], &side);
            sj = j;
            l = 0;
        } else {
            i = r - 2;
            j = g < 2 ? g - 2 : L.n2 + (g - 2);
            sj = ghost_image(j, L.n2, pty, L.bc[2], L.bc[3], &side);
            si = i;
            l = 1;
        }
        if (side < 0) continue;
        int kind = L.bc[2 * l + side];
        S v[4];
        for (int c = 0; c < 4; ++c) {
            v[c] = buf[plane_of(L, site, c) + cell_off(L, si, sj)];
            if (mirror_sign(kind, l, c, 2) < 0) v[c] = -v[c];
        }
        moving_wall_ghost(L, 2 * l + side, v);
        for (int c = 0; c < 4; ++c) buf[plane_of(L, site, c) + cell_off(L, i, j)] = v[c];
    }
}

// Stage arguments of problem p.
template <class R>
__device__ __forceinline__ StageArgs batch_stage_args(const BatchArgs &B, int p)
{
    const BatchProb &P = B.probs[p];
    StageArgs A{};   // every field not set below is zero (no test hook, no CFL output)
    A.L = P.L;
    A.uin = P.U[B.in_idx];
    A.u0 = P.U[0];
    A.aux = P.U[2];
    A.out = P.U[B.out_idx];
    A.ctl = P.ctl;
    A.theta = nullptr;
    A.k = B.k;
    A.gamma = P.gamma;
    A.mu = P.mu;
    A.kappa = P.kappa;
    A.eps = B.eps;
    A.c_s = B.c_s;
    A.limiter = B.limiter;
    A.source = 0;
    A.src_p0 = 0.0;
    A.tconst = reinterpret_cast<const TileConst<R> *>(B.tconst) + p;
    return A;
}

// The tile constants of every problem for one stage (its own step size), one
// thread per problem, before the stage kernel.
template <class R>
__global__ void k_batch_tile_consts(BatchArgs B, int nprob)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob || B.probs[p].failed) return;
    const StageArgs A = batch_stage_args<R>(B, p);
    tile_const_init<R>(reinterpret_cast<TileConst<R> *>(B.tconst)[p], A, A.ctl->dt);
}

// --- the persistent stage kernel over the work list
// Work item `item` at or after `from` (stride gridDim.x) whose problem has not
// failed, or nitems (uniform per block: every thread computes the same).
__device__ __forceinline__ int next_live_item(const BatchArgs &B, int from)
{
    int item = from;
    while (item < B.nitems && B.probs[B.item_p[item]].failed) item += gridDim.x;
    return item;
}

// Each CTA walks its items as the single-problem kernel walks its tiles: the
// tile is loaded by TMA through its problem's tensor map (buffer U[in_idx]), and
// the next item's copies are issued as soon as the current tile's point phase is
// done, through the next item's map, so they land while the face and cell
// phases run. Every item loads its problem's tile constants and keeps its own
// restart flag.
template <class R, class S, int TX, int TY, int NTH>
__global__ void __launch_bounds__(NTH, stage_min_ctas<R, TX, TY, NTH>()) k_batch_stage(BatchArgs B)
{
    extern __shared__ __align__(128) unsigned char smem_batch[];
    V4<R> *sm = reinterpret_cast<V4<R> *>(smem_batch);
    constexpr int shape = TX == 32 ? 1 : 0;
    int item = next_live_item(B, blockIdx.x);
    for (int it = 0; item < B.nitems; ++it) {
        const int p = B.item_p[item];
        const BatchProb &P = B.probs[p];
        const int tile = B.item_t[item];
        const StageArgs A = batch_stage_args<R>(B, p);
        const size_t mb = ((size_t)p * kShapes + shape) * 4;
        const CUtensorMap *map = B.maps + mb + P.buf_of[B.in_idx];
        const int next = next_live_item(B, item + gridDim.x);
        int nbx = -1, nby = -1;
        const CUtensorMap *nmap = nullptr;
        if (next < B.nitems) {
            const int np = B.item_p[next], nt = B.item_t[next];
            const BatchProb &Q = B.probs[np];
            nbx = nt % Q.tiles_x;
            nby = nt / Q.tiles_x;
            nmap = B.maps + ((size_t)np * kShapes + shape) * 4 + Q.buf_of[B.in_idx];
        }
        if (!stage_tile<R, S, TX, TY, NTH>(A, tile % P.tiles_x, tile / P.tiles_x, sm, map, it, nbx, nby, nmap, true,
                                           B.rmaps + mb + P.buf_of[0], B.rmaps + mb + P.buf_of[2],
                                           B.rmaps + mb + P.buf_of[B.in_idx]))
            break;
        // the next item's records overwrite this item's
        __syncthreads();
        item = next;
    }
}

__global__ void k_batch_commit(BatchProb *probs, int nprob, int max_halvings)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    BatchProb &P = probs[p];
    if (P.failed) return;
    if (P.ctl->notpp) {
        P.rejected = 1;
        P.restarts += 1;
        P.halvings += 1;
        P.ctl->dt *= 0.5;
        if (P.halvings > max_halvings) P.failed = 1;
    } else {
        void *t = P.U[0];
        P.U[0] = P.U[1];
        P.U[1] = t;
        const int b = P.buf_of[0];
        P.buf_of[0] = P.buf_of[1];
        P.buf_of[1] = b;
        P.ctl->t += P.ctl->dt;
        P.accepted += 1;
        P.rejected = 0;
        P.halvings = 0;
    }
    P.ctl->notpp = 0;
}

// --- FP64 <-> FP32 (+ compensation) conversion of one problem's state
__global__ void k_batch_to_f32(const double *src, float *dst, long long plane, int nplanes, int nc);
__global__ void k_batch_to_f64(const float *src, double *dst, long long plane, int nplanes, int nc);

__global__ void k_batch_to_f32(const double *src, float *dst, long long plane, int nplanes, int nc)
{
    long long total = plane * nplanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        double x = src[e];
        float h = __double2float_rn(x);
        dst[e] = h;
        if (e / plane < nc) dst[(long long)nplanes * plane + e] = __double2float_rn(x - (double)h);
    }
}

__global__ void k_batch_to_f64(const float *src, double *dst, long long plane, int nplanes, int nc)
{
    long long total = plane * nplanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        double x = (double)src[e];
        if (e / plane < nc) x += (double)src[(long long)nplanes * plane + e];
        dst[e] = x;
    }
}

template <class S>
__global__ void k_batch_validate(const S *buf, Layout L, double gamma, int *flag)
{
    const int n1 = L.n1, n2 = L.n2;
    const long long per_site[4] = {(long long)n1 * n2, (long long)(n1 + 1) * n2, (long long)n1 * (n2 + 1),
                                   (long long)(n1 + 1) * (n2 + 1)};
    const long long total = per_site[0] + per_site[1] + per_site[2] + per_site[3];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        long long r = t;
        int site = 0;
        while (r >= per_site[site]) r -= per_site[site++];
        int w = (site == 1 || site == 3) ? n1 + 1 : n1;
        long long off = cell_off(L, (int)(r % w), (int)(r / w));
        S U[4];
        for (int c = 0; c < 4; ++c) U[c] = buf[plane_of(L, site, c) + off];
        if (!admissible_input2(U)) atomicOr(flag, 1);
    }
}

}  // namespace afns

using namespace afns;

// Tensor map of one state buffer for TX x TY tiles (afns.cu).
bool make_stage_map(CUtensorMap *m, void *buf, const Layout &L, size_t esz, int tx, int ty, bool rows);

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct TileCfg {
    int tx, ty, threads, schedule;   // schedule 0: problem-major, 1: largest problems first, interleaved
};

struct afb_ctx {
    int nprob = 0;
    bool mixed = true;
    af_opts opts{};
    cudaStream_t st = nullptr;
    char *ws = nullptr;
    bool own_ws = false;
    std::vector<BatchProb> h_probs;     // host copies (pointers into ws)
    BatchProb *d_probs = nullptr;
    Ctl *d_ctl = nullptr;
    unsigned long long *d_mx = nullptr;
    int *d_chunk_p = nullptr, *d_chunk_c = nullptr;
    void *d_tconst = nullptr;           // per-problem tile constants of the current stage
    int nchunks = 0;
    int *d_items[3][2] = {};            // per tile config: item_p, item_t (configs share the schedule arrays)
    CUtensorMap *d_maps = nullptr;      // tensor maps of every problem, buffer and tile shape
    CUtensorMap *d_rmaps = nullptr;     // the same with the row box of the cell-update inputs
    int nitems[3] = {0, 0, 0};
    double *stage64 = nullptr;          // FP64 staging of the largest problem
    int *d_flag = nullptr;
    int *h_flag = nullptr;
    TileCfg cfg{16, 8, 256, 0};
    int stage_grid = 0;                 // persistent grid of the current configuration
    bool tuned = false;
    cudaGraphExec_t graph = nullptr;
    long long launches_per_step = 0;
    std::string err;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

static const TileCfg kCandidates[] = {
    {16, 8, 256, 0}, {16, 8, 128, 0}, {16, 8, 256, 1}, {16, 8, 128, 1}, {32, 8, 256, 0}, {32, 8, 256, 1},
};

static int tile_index(int tx) { return tx == 32 ? 1 : 0; }

// Persistent grid of the stage kernel for a configuration: one wave of resident
// CTAs (SM count x CTAs per SM). Sets the dynamic shared-memory limit; called
// outside any stream capture.
template <class R, class S, int TX, int TY, int NTH>
static cudaError_t batch_stage_grid_n(int nitems, int *grid)
{
    size_t smem = Tile2<TX, TY>::template bytes<R>();
    cudaError_t e = cudaFuncSetAttribute(k_batch_stage<R, S, TX, TY, NTH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // the whole unified L1 as shared memory, so that the occupancy computed
    // below is the one the launches get
    e = cudaFuncSetAttribute(k_batch_stage<R, S, TX, TY, NTH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 148, per_sm = 1;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_stage<R, S, TX, TY, NTH>, NTH, smem);
    if (e != cudaSuccess) return e;
    *grid = std::max(1, std::min(nitems, nsm * std::max(per_sm, 1)));
    return cudaSuccess;
}

// Persistent grid of the stage kernel for a configuration: one wave of resident
// CTAs (SM count x CTAs per SM). Sets the dynamic shared-memory limit; called
// outside any stream capture.
template <class R, class S, int TX, int TY>
static cudaError_t batch_stage_grid(int threads, int nitems, int *grid)
{
    if (threads == 128) return batch_stage_grid_n<R, S, TX, TY, 128>(nitems, grid);
    return batch_stage_grid_n<R, S, TX, TY, 256>(nitems, grid);
}

template <class R, class S, int TX, int TY>
static cudaError_t launch_batch_stage_t(const BatchArgs &B, int threads, int grid, cudaStream_t st)
{
    size_t smem = Tile2<TX, TY>::template bytes<R>();
    if (threads == 128) k_batch_stage<R, S, TX, TY, 128><<<grid, 128, smem, st>>>(B);
    else k_batch_stage<R, S, TX, TY, 256><<<grid, 256, smem, st>>>(B);
    return cudaGetLastError();
}

static cudaError_t prepare_config(afb_ctx *c)
{
    const TileCfg &t = c->cfg;
    int n = c->nitems[tile_index(t.tx)];
    if (c->mixed) {
        if (t.tx == 32) return batch_stage_grid<float, float, 32, 8>(t.threads, n, &c->stage_grid);
        return batch_stage_grid<float, float, 16, 8>(t.threads, n, &c->stage_grid);
    }
    return batch_stage_grid<double, double, 16, 8>(t.threads, n, &c->stage_grid);
}

static cudaError_t launch_batch_stage(afb_ctx *c, const BatchArgs &B)
{
    const TileCfg &t = c->cfg;
    if (c->mixed) {
        if (t.tx == 32) return launch_batch_stage_t<float, float, 32, 8>(B, t.threads, c->stage_grid, c->st);
        return launch_batch_stage_t<float, float, 16, 8>(B, t.threads, c->stage_grid, c->st);
    }
    return launch_batch_stage_t<double, double, 16, 8>(B, t.threads, c->stage_grid, c->st);
}

// SSP-RK54 coefficients (Spiteri-Ruuth SSPRK(5,4), Shu-Osher form; Sec. 2.3)
static const double kA[5][2] = {{0.0, 1.0},
                                {0.444370493651235, 0.555629506348765},
                                {0.620101851488403, 0.379898148511597},
                                {0.178079954393132, 0.821920045606868},
                                {0.0, 0.386708617503269}};
static const double kBw[5] = {0.391752226571890, 0.368410593050371, 0.251891774271694, 0.544974750228521,
                              0.226007483236906};

// Issue one batch step (no host synchronisation).
static cudaError_t issue_step(afb_ctx *c)
{
    const int tb = tile_index(c->cfg.tx);
    cudaError_t e;
    if (c->mixed)
        k_batch_dt_partial<float><<<c->nchunks, 256, 0, c->st>>>(c->d_probs, c->d_chunk_p, c->d_chunk_c,
                                                                 c->opts.cfl_c, c->opts.cfl_v);
    else
        k_batch_dt_partial<double><<<c->nchunks, 256, 0, c->st>>>(c->d_probs, c->d_chunk_p, c->d_chunk_c,
                                                                  c->opts.cfl_c, c->opts.cfl_v);
    k_batch_dt_final<<<(c->nprob + 127) / 128, 128, 0, c->st>>>(c->d_probs, c->nprob);
    int maxspan = 0;
    for (auto &P : c->h_probs) maxspan = std::max(maxspan, 4 * (std::max(P.L.n1, P.L.n2) + 5) * 5);
    dim3 gg((maxspan + 255) / 256, c->nprob);
    static const int in_idx[5] = {0, 1, 2, 1, 3}, out_idx[5] = {1, 2, 1, 3, 1};
    for (int s = 0; s < 5; ++s) {
        for (int pass = 0; pass < 2; ++pass) {
            if (c->mixed) k_batch_ghost<float><<<gg, 256, 0, c->st>>>(c->d_probs, in_idx[s], pass);
            else k_batch_ghost<double><<<gg, 256, 0, c->st>>>(c->d_probs, in_idx[s], pass);
        }
        BatchArgs B{};
        B.probs = c->d_probs;
        B.item_p = c->d_items[tb][0] + (c->cfg.schedule ? c->nitems[tb] : 0);
        B.item_t = c->d_items[tb][1] + (c->cfg.schedule ? c->nitems[tb] : 0);
        B.nitems = c->nitems[tb];
        B.in_idx = in_idx[s];
        B.out_idx = out_idx[s];
        B.eps = c->opts.eps;
        B.c_s = c->opts.c_s;
        B.limiter = c->opts.limiter;
        StageCoef &k = B.k;
        k.wall_fix = 1;
        k.a0 = kA[s][0];
        k.a1 = kA[s][1];
        k.cl = kBw[s];
        if (s == 4) {
            k.a0 = 0.0;
            k.a2 = 1.0;
        }
        if (s == 3) {
            k.acc = 1;
            k.b2 = 0.517231671970585;
            k.b1 = 0.096059710526147;
            k.bl = 0.063692468666290;
        }
        B.tconst = c->d_tconst;
        B.maps = c->d_maps;
        B.rmaps = c->d_rmaps;
        if (c->mixed) k_batch_tile_consts<float><<<(c->nprob + 127) / 128, 128, 0, c->st>>>(B, c->nprob);
        else k_batch_tile_consts<double><<<(c->nprob + 127) / 128, 128, 0, c->st>>>(B, c->nprob);
        if ((e = launch_batch_stage(c, B)) != cudaSuccess) return e;
    }
    k_batch_commit<<<(c->nprob + 127) / 128, 128, 0, c->st>>>(c->d_probs, c->nprob, c->opts.max_halvings);
    c->launches_per_step = 2 + 5 * 4 + 1;
    return cudaGetLastError();
}

static af_status bfail(afb_ctx *c, af_status s, const char *m)
{
    if (s == AF_ECUDA) cudaGetLastError();   // clear the runtime's record of the error
    if (c) c->err = m;
    return s;
}

extern "C" {

af_status afb_workspace_bytes(int nprob, const af_grid *grids, const af_opts *opts, size_t *bytes)
{
    if (nprob <= 0 || !grids || !bytes) return AF_EINVAL;
    af_opts d;
    if (!opts) af_opts_default(2, &d), d.precision = AF_MIXED, opts = &d;
    const bool mixed = opts->precision == AF_MIXED;
    size_t tot = 0, big = 0;
    for (int p = 0; p < nprob; ++p) {
        const af_grid &g = grids[p];
        if (g.dim != 2 || g.n[0] < 4 || g.n[1] < 4) return AF_EINVAL;
        long long pitch = ((g.n[0] + 5) + 31) / 32 * 32, rows = g.n[1] + 5;
        long long plane = (pitch * rows + 63) / 64 * 64;
        size_t st = al256((size_t)plane * (16 + (mixed ? 4 : 0)) * (mixed ? 4 : 8));
        tot += 4 * st + al256(sizeof(Ctl)) + al256(16);
        big = std::max(big, (size_t)plane * 16 * 8);
    }
    *bytes = tot + al256(big) + al256(sizeof(int) * 4);
    return AF_OK;
}

af_status afb_create(int nprob, const af_grid *grids, const double *gamma, const double *mu, const double *Pr,
                     const af_bc *bcs, const af_opts *opts, void *cuda_stream, void *workspace,
                     size_t workspace_bytes, afb_ctx **out)
{
    if (!out || nprob <= 0 || !grids || !gamma || !mu || !Pr || !bcs) return AF_EINVAL;
    *out = nullptr;
    af_opts d;
    if (!opts) af_opts_default(2, &d), d.precision = AF_MIXED, opts = &d;
    if (opts->source != AF_SRC_NONE) return AF_EINVAL;   // manufactured sources: single-problem contexts only
    size_t need = 0;
    if (afb_workspace_bytes(nprob, grids, opts, &need) != AF_OK) return AF_EINVAL;
    for (int p = 0; p < nprob; ++p) {
        if (!(gamma[p] > 1.0) || !(mu[p] >= 0.0) || !(Pr[p] > 0.0)) return AF_EINVAL;
        for (int l = 0; l < 2; ++l)
            if ((bcs[p].side[2 * l] == AF_BC_PERIODIC) != (bcs[p].side[2 * l + 1] == AF_BC_PERIODIC)) return AF_EINVAL;
        for (int k = 0; k < 4; ++k) {
            const int kind = bcs[p].side[k];
            if (kind < 0 || kind > AF_BC_MOVING_WALL || kind == AF_BC_EXACT) return AF_EINVAL;
            if (kind == AF_BC_MOVING_WALL && !std::isfinite(bcs[p].wall_speed[k])) return AF_EINVAL;
        }
    }
    afb_ctx *c = new (std::nothrow) afb_ctx();
    if (!c) return AF_ENOMEM;
    c->nprob = nprob;
    c->opts = *opts;
    c->mixed = opts->precision == AF_MIXED;
    c->st = (cudaStream_t)cuda_stream;
    if (workspace) {
        if (workspace_bytes < need || ((uintptr_t)workspace & 255)) {
            delete c;
            return AF_ENOMEM;
        }
        c->ws = (char *)workspace;
    } else {
        if (cudaMalloc((void **)&c->ws, need) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return AF_ENOMEM;
        }
        c->own_ws = true;
    }
    char *q = c->ws;
    c->h_probs.resize(nprob);
    size_t big = 0;
    std::vector<int> chunk_p, chunk_c;
    for (int p = 0; p < nprob; ++p) {
        BatchProb &P = c->h_probs[p];
        std::memset(&P, 0, sizeof(P));
        const af_grid &g = grids[p];
        Layout &L = P.L;
        L.dim = 2;
        L.nc = 4;
        L.n1 = g.n[0];
        L.n2 = g.n[1];
        L.nsite = 4;
        L.pitch = ((L.n1 + 5) + 31) / 32 * 32;
        L.rows = L.n2 + 5;
        L.plane = ((long long)L.pitch * L.rows + 63) / 64 * 64;
        L.comp = c->mixed ? 1 : 0;
        for (int k = 0; k < 4; ++k) L.bc[k] = bcs[p].side[k];
        for (int k = 0; k < 4; ++k) L.wall_speed[k] = bcs[p].side[k] == AF_BC_MOVING_WALL ? bcs[p].wall_speed[k] : 0.0;
        L.dx = (g.hi[0] - g.lo[0]) / g.n[0];
        L.dy = (g.hi[1] - g.lo[1]) / g.n[1];
        L.lo[0] = g.lo[0];
        L.lo[1] = g.lo[1];
        layout_finish(&L);
        size_t st = al256((size_t)L.plane * (16 + (c->mixed ? 4 : 0)) * (c->mixed ? 4 : 8));
        for (int k = 0; k < 4; ++k) P.U[k] = q, P.buf_of[k] = k, q += st;
        P.U[4] = nullptr;
        P.ctl = (Ctl *)q;
        q += al256(sizeof(Ctl));
        P.mx = (unsigned long long *)q;
        q += al256(16);
        P.gamma = gamma[p];
        P.mu = mu[p];
        P.Pr = Pr[p];
        P.kappa = gamma[p] * mu[p] / ((gamma[p] - 1.0) * Pr[p]);
        P.tiles_x = (L.n1 + 15) / 16;
        P.tiles_y = (L.n2 + 7) / 8;
        big = std::max(big, (size_t)L.plane * 16 * 8);
        long long nc = (long long)L.n1 * L.n2;
        for (long long k = 0; k * kDtChunk < nc; ++k) chunk_p.push_back(p), chunk_c.push_back((int)k);
    }
    c->stage64 = (double *)q;
    q += al256(big);
    c->d_flag = (int *)q;
    cudaError_t e = cudaMemsetAsync(c->ws, 0, need, c->st);
    // descriptors and work lists in their own small allocations
    c->nchunks = (int)chunk_p.size();
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_probs, sizeof(BatchProb) * nprob);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_chunk_p, sizeof(int) * c->nchunks * 2);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tconst, sizeof(TileConst<double>) * nprob);
    if (e == cudaSuccess) {
        c->d_chunk_c = c->d_chunk_p + c->nchunks;
        e = cudaMemcpy(c->d_chunk_p, chunk_p.data(), sizeof(int) * c->nchunks, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemcpy(c->d_chunk_c, chunk_c.data(), sizeof(int) * c->nchunks, cudaMemcpyHostToDevice);
    // work lists per tile width (16, 32); schedule 0 then schedule 1 stored back to back
    for (int tb = 0; tb < 2 && e == cudaSuccess; ++tb) {
        int tw = tb ? 32 : 16;
        std::vector<int> ip, it;
        std::vector<std::vector<std::pair<int, int>>> per(nprob);
        for (int p = 0; p < nprob; ++p) {
            int txn = (c->h_probs[p].L.n1 + tw - 1) / tw, tyn = c->h_probs[p].tiles_y;
            for (int t = 0; t < txn * tyn; ++t) per[p].push_back({p, t}), ip.push_back(p), it.push_back(t);
        }
        // schedule 1: problems by decreasing size, tiles of different problems interleaved
        std::vector<int> order(nprob);
        for (int p = 0; p < nprob; ++p) order[p] = p;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return per[a].size() > per[b].size(); });
        std::vector<int> ip2, it2;
        size_t maxn = 0;
        for (int p : order) maxn = std::max(maxn, per[p].size());
        for (size_t r = 0; r < maxn; ++r)
            for (int p : order)
                if (r < per[p].size()) ip2.push_back(per[p][r].first), it2.push_back(per[p][r].second);
        int n = (int)ip.size();
        c->nitems[tb] = n;
        int *dp = nullptr, *dt_ = nullptr;
        e = cudaMalloc((void **)&dp, sizeof(int) * 2 * n);
        if (e == cudaSuccess) e = cudaMalloc((void **)&dt_, sizeof(int) * 2 * n);
        if (e == cudaSuccess) e = cudaMemcpy(dp, ip.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dp + n, ip2.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dt_, it.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dt_ + n, it2.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
        c->d_items[tb][0] = dp;
        c->d_items[tb][1] = dt_;
    }
    // tensor maps of the four buffers of every problem for both tile shapes
    if (e == cudaSuccess) {
        std::vector<CUtensorMap> maps((size_t)nprob * kShapes * 4), rmaps(maps.size());
        const size_t esz = c->mixed ? sizeof(float) : sizeof(double);
        static const int shape_tile[kShapes][2] = {{16, 8}, {32, 8}};
        for (int p = 0; p < nprob && e == cudaSuccess; ++p)
            for (int sh = 0; sh < kShapes && e == cudaSuccess; ++sh)
                for (int b = 0; b < 4; ++b) {
                    const size_t m = ((size_t)p * kShapes + sh) * 4 + b;
                    if (!make_stage_map(&maps[m], c->h_probs[p].U[b], c->h_probs[p].L, esz, shape_tile[sh][0],
                                        shape_tile[sh][1], false) ||
                        !make_stage_map(&rmaps[m], c->h_probs[p].U[b], c->h_probs[p].L, esz, shape_tile[sh][0],
                                        shape_tile[sh][1], true)) {
                        e = cudaErrorInvalidValue;   // tensor map encoding failed
                        break;
                    }
                }
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_maps, sizeof(CUtensorMap) * maps.size());
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_rmaps, sizeof(CUtensorMap) * rmaps.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_rmaps, rmaps.data(), sizeof(CUtensorMap) * rmaps.size(), cudaMemcpyHostToDevice);
    }
    // tile counts of the 32-wide configuration live in the descriptors at launch time
    if (e == cudaSuccess) e = cudaMemcpy(c->d_probs, c->h_probs.data(), sizeof(BatchProb) * nprob, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_flag, 64);
    if (e == cudaSuccess) e = prepare_config(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        afb_destroy(c);
        return AF_ECUDA;
    }
    *out = c;
    return AF_OK;
}

af_status afb_destroy(afb_ctx *c)
{
    if (!c) return AF_EINVAL;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (int tb = 0; tb < 3; ++tb)
        for (int k = 0; k < 2; ++k)
            if (c->d_items[tb][k]) cudaFree(c->d_items[tb][k]);
    if (c->d_probs) cudaFree(c->d_probs);
    if (c->d_maps) cudaFree(c->d_maps);
    if (c->d_rmaps) cudaFree(c->d_rmaps);
    if (c->d_chunk_p) cudaFree(c->d_chunk_p);
    if (c->d_tconst) cudaFree(c->d_tconst);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->own_ws && c->ws) cudaFree(c->ws);
    delete c;
    return AF_OK;
}

const char *afb_last_error(const afb_ctx *c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"

// Pull the device descriptors back (counters, swapped buffer pointers).
static cudaError_t pull_probs(afb_ctx *c)
{
    cudaError_t e = cudaMemcpyAsync(c->h_probs.data(), c->d_probs, sizeof(BatchProb) * c->nprob,
                                    cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return e;
}

static cudaError_t push_probs(afb_ctx *c)
{
    return cudaMemcpyAsync(c->d_probs, c->h_probs.data(), sizeof(BatchProb) * c->nprob, cudaMemcpyHostToDevice,
                           c->st);
}

static void site_dims2(const Layout &L, int s, int *w, int *h)
{
    *w = (s == 1 || s == 3) ? L.n1 + 1 : L.n1;
    *h = (s == 2 || s == 3) ? L.n2 + 1 : L.n2;
}

extern "C" af_status afb_set_state(afb_ctx *c, int i, const double *const site[4], int on_device, double t)
{
    if (!c || i < 0 || i >= c->nprob || !site) return AF_EINVAL;
    cudaError_t e = pull_probs(c);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    BatchProb &P = c->h_probs[i];
    const Layout &L = P.L;
    double *dst = c->mixed ? c->stage64 : (double *)P.U[0];
    for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
        int w, h;
        site_dims2(L, s, &w, &h);
        for (int comp = 0; comp < 4 && e == cudaSuccess; ++comp)
            e = cudaMemcpy2DAsync(dst + plane_of(L, s, comp) + cell_off(L, 0, 0), L.pitch * sizeof(double),
                                  site[s] + (size_t)comp * w * h, w * sizeof(double), w * sizeof(double), h,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st);
    if (e == cudaSuccess) k_batch_validate<double><<<148 * 4, 256, 0, c->st>>>(dst, L, P.gamma, c->d_flag);
    if (e == cudaSuccess && c->mixed)
        k_batch_to_f32<<<148 * 8, 256, 0, c->st>>>(c->stage64, (float *)P.U[0], L.plane, 16, 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    if (*c->h_flag) return bfail(c, AF_EINVAL, "state has a DoF outside G");
    P.accepted = P.restarts = P.rejected = P.halvings = P.failed = 0;
    Ctl h{};
    h.t = t;
    e = cudaMemcpyAsync(P.ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = push_probs(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    return e == cudaSuccess ? AF_OK : bfail(c, AF_ECUDA, cudaGetErrorString(e));
}

extern "C" af_status afb_get_state(afb_ctx *c, int i, double *const site[4], int on_device, double *t)
{
    if (!c || i < 0 || i >= c->nprob || !site) return AF_EINVAL;
    cudaError_t e = pull_probs(c);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    const BatchProb &P = c->h_probs[i];
    const Layout &L = P.L;
    // ghost fill of u^n of this problem (periodic duplicates)
    dim3 gg((4 * (std::max(L.n1, L.n2) + 5) * 5 + 255) / 256, 1);
    for (int pass = 0; pass < 2; ++pass) {
        if (c->mixed) k_batch_ghost<float><<<gg, 256, 0, c->st>>>(c->d_probs + i, 0, pass);
        else k_batch_ghost<double><<<gg, 256, 0, c->st>>>(c->d_probs + i, 0, pass);
    }
    const double *src = (const double *)P.U[0];
    if (c->mixed) {
        k_batch_to_f64<<<148 * 8, 256, 0, c->st>>>((const float *)P.U[0], c->stage64, L.plane, 16, 4);
        src = c->stage64;
    }
    for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
        int w, h;
        site_dims2(L, s, &w, &h);
        for (int comp = 0; comp < 4 && e == cudaSuccess; ++comp)
            e = cudaMemcpy2DAsync(site[s] + (size_t)comp * w * h, w * sizeof(double),
                                  src + plane_of(L, s, comp) + cell_off(L, 0, 0), L.pitch * sizeof(double),
                                  w * sizeof(double), h, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->st);
    }
    Ctl h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    if (t) *t = h.t;
    return AF_OK;
}

// Autotuner: time every candidate configuration on the batch (from a saved copy
// of the states, restored afterwards) and keep the fastest.
static af_status tune(afb_ctx *c)
{
    // save all states u^n
    std::vector<void *> save(c->nprob, nullptr);
    cudaError_t e = pull_probs(c);
    size_t esz = c->mixed ? 4 : 8;
    for (int p = 0; p < c->nprob && e == cudaSuccess; ++p) {
        const Layout &L = c->h_probs[p].L;
        size_t bytes = (size_t)L.plane * (16 + (c->mixed ? 4 : 0)) * esz;
        e = cudaMalloc(&save[p], bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(save[p], c->h_probs[p].U[0], bytes, cudaMemcpyDeviceToDevice, c->st);
    }
    std::vector<BatchProb> saved_desc = c->h_probs;
    float best = 1e30f;
    TileCfg best_cfg = c->cfg;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (const TileCfg &cand : kCandidates) {
        if (e != cudaSuccess) break;
        if (!c->mixed && cand.tx == 32) continue;   // the FP64 32x8 tile exceeds shared memory
        c->cfg = cand;
        for (int p = 0; p < c->nprob; ++p) c->h_probs[p].tiles_x = (c->h_probs[p].L.n1 + cand.tx - 1) / cand.tx;
        e = prepare_config(c);
        if (e == cudaSuccess) e = push_probs(c);
        if (e == cudaSuccess) e = issue_step(c);   // warm-up
        cudaEventRecord(a, c->st);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = issue_step(c);
        cudaEventRecord(b, c->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms < best) best = ms, best_cfg = cand;
        // restore states and descriptors
        c->h_probs = saved_desc;
        for (int p = 0; p < c->nprob && e == cudaSuccess; ++p) {
            const Layout &L = c->h_probs[p].L;
            size_t bytes = (size_t)L.plane * (16 + (c->mixed ? 4 : 0)) * esz;
            e = cudaMemcpyAsync(c->h_probs[p].U[0], save[p], bytes, cudaMemcpyDeviceToDevice, c->st);
        }
        if (e == cudaSuccess) e = push_probs(c);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    for (void *s : save)
        if (s) cudaFree(s);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    c->cfg = best_cfg;
    for (int p = 0; p < c->nprob; ++p) c->h_probs[p].tiles_x = (c->h_probs[p].L.n1 + best_cfg.tx - 1) / best_cfg.tx;
    e = prepare_config(c);
    if (e == cudaSuccess) e = push_probs(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    c->tuned = true;
    return e == cudaSuccess ? AF_OK : bfail(c, AF_ECUDA, cudaGetErrorString(e));
}

extern "C" af_status afb_tune(afb_ctx *c, int *tile_x, int *tile_y, int *threads, int *schedule)
{
    if (!c) return AF_EINVAL;
    af_status s = tune(c);
    if (s != AF_OK) return s;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (tile_x) *tile_x = c->cfg.tx;
    if (tile_y) *tile_y = c->cfg.ty;
    if (threads) *threads = c->cfg.threads;
    if (schedule) *schedule = c->cfg.schedule;
    return AF_OK;
}

extern "C" af_status afb_step_all(afb_ctx *c, int nsteps, int use_graph)
{
    if (!c || nsteps < 0) return AF_EINVAL;
    cudaError_t e = cudaSuccess;
    if (use_graph && !c->graph) {
        if (!c->st) return bfail(c, AF_EINVAL, "graph replay needs a non-default CUDA stream");
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
        cudaError_t e2 = issue_step(c);
        e = cudaStreamEndCapture(c->st, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    }
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = use_graph ? cudaGraphLaunch(c->graph, c->st) : issue_step(c);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    return AF_OK;
}

extern "C" af_status afb_stats(afb_ctx *c, int i, int *accepted, int *restarts, int *failed, double *t)
{
    if (!c || i < 0 || i >= c->nprob) return AF_EINVAL;
    cudaError_t e = pull_probs(c);
    if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
    const BatchProb &P = c->h_probs[i];
    if (accepted) *accepted = P.accepted;
    if (restarts) *restarts = P.restarts;
    if (failed) *failed = P.failed;
    if (t) {
        Ctl h{};
        e = cudaMemcpy(&h, P.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bfail(c, AF_ECUDA, cudaGetErrorString(e));
        *t = h.t;
    }
    return AF_OK;
}

extern "C" af_status afb_sync(afb_ctx *c, long long *launches_per_step)
{
    if (!c) return AF_EINVAL;
    if (launches_per_step) *launches_per_step = c->launches_per_step;
    cudaError_t e = cudaStreamSynchronize(c->st);
    return e == cudaSuccess ? AF_OK : bfail(c, AF_ECUDA, cudaGetErrorString(e));
}
